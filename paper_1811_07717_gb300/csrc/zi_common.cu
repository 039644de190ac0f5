// Error state, status strings, the private device-memory pool and the
// device-wide exclusive scan used by the mesh and assembly stages.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "zi_internal.cuh"

namespace zi {

namespace {
thread_local int g_status = ZI_OK;
thread_local char g_msg[1024] = "no error";
}  // namespace

thread_local bool g_capturing = false;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t k) {
  if (!g_capturing) g_launches.fetch_add(k, std::memory_order_relaxed);
}

int64_t launches_total() { return g_launches.load(); }

int set_error(int status, const char* fmt, ...) {
  g_status = status;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  const char* base = strrchr(file, '/');
  base = base ? base + 1 : file;
  int st = (e == cudaErrorMemoryAllocation) ? ZI_ERR_NOMEM : ZI_ERR_CUDA;
  return set_error(st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base, line);
}

int device_error_to_status(int d) {
  if (d == 0) return ZI_OK;
  if (d & DEV_ERR_NONFINITE) return set_error(ZI_ERR_NONFINITE, "non-finite input value");
  if (d & DEV_ERR_BAD_VOLUME) return set_error(ZI_ERR_BAD_MESH, "element with non-positive volume");
  if (d & DEV_ERR_OVERLAP) return set_error(ZI_ERR_BAD_MESH, "electrode patches overlap");
  if (d & DEV_ERR_NO_PATCH) return set_error(ZI_ERR_BAD_MESH, "an electrode covers no boundary triangle");
  if (d & DEV_ERR_DUP_ELECTRODE) return set_error(ZI_ERR_BAD_MESH, "two point electrodes on the same node");
  if (d & DEV_ERR_OUTSIDE) return set_error(ZI_ERR_BAD_MESH, "point outside the mesh");
  if (d & DEV_ERR_VALENCE) return set_error(ZI_ERR_BAD_MESH, "node valence above the supported bound");
  if (d & DEV_ERR_NO_GROUND) return set_error(ZI_ERR_BAD_MESH, "no boundary node outside the electrodes");
  if (d & DEV_ERR_NOT_SPD) return set_error(ZI_ERR_BAD_MESH, "electrode Schur matrix is not positive definite");
  if (d & DEV_ERR_NONMANIFOLD) return set_error(ZI_ERR_BAD_MESH, "a face is shared by more than two elements");
  if (d & DEV_ERR_STENCIL)
    return set_error(ZI_ERR_BAD_MESH, "a source stencil cannot represent all three orientations");
  if (d & DEV_ERR_BAD_INDEX)
    return set_error(ZI_ERR_ARG, "node index outside the mesh (a source-matrix entry or an element vertex) or a "
                     "non-finite source weight");
  if (d & DEV_ERR_TIMEOUT) return set_error(ZI_ERR_TIMEOUT, "device-side wait exceeded its bound");
  return set_error(ZI_ERR_CUDA, "device error word 0x%x", d);
}

// ---------------------------------------------------------------------------
// memory pool
// ---------------------------------------------------------------------------

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64];
bool g_pool_init[64];
}  // namespace

int get_pool(cudaMemPool_t* out) {
  int dev = 0;
  ZI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(ZI_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_init[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    ZI_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
    uint64_t thr = UINT64_MAX;
    ZI_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool_init[dev] = true;
  }
  *out = g_pools[dev];
  return ZI_OK;
}

int dalloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = nullptr;
  ZI_CHECK(get_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    (void)cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? ZI_ERR_NOMEM : ZI_ERR_CUDA,
                     "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  return ZI_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 152;
  }
  return cached[dev];
}

// ---------------------------------------------------------------------------
// exclusive scan (three passes: block totals, scan of totals, block scans)
// ---------------------------------------------------------------------------

namespace {
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one int64 per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* excl) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  int64_t warp_off = wid ? warp_tot[wid - 1] : 0;
  *excl = warp_off + x - v;
  int64_t total = warp_tot[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return total;
}

__global__ void k_tile_totals(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ tot) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) s += in[base + k];
  int64_t ex;
  int64_t t = block_exclusive_scan(s, &ex);
  if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

// Single block: in-place exclusive scan of the tile totals.
__global__ void k_scan_totals(int64_t* __restrict__ tot, int64_t nt, int64_t* __restrict__ grand) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nt; base += SCAN_TILE) {
    int64_t b = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t loc[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      loc[k] = (b + k < nt) ? tot[b + k] : 0;
      s += loc[k];
    }
    int64_t ex;
    int64_t t = block_exclusive_scan(s, &ex);
    int64_t run = carry + ex;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      if (b + k < nt) tot[b + k] = run;
      run += loc[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += t;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_tile_scan(const int32_t* __restrict__ in, int64_t n, const int64_t* __restrict__ tot,
                            int32_t* __restrict__ out, const int64_t* __restrict__ grand) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t loc[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    loc[k] = (base + k < n) ? in[base + k] : 0;
    s += loc[k];
  }
  int64_t ex;
  block_exclusive_scan(s, &ex);
  int64_t run = tot[blockIdx.x] + ex;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = (int32_t)run;
    run += loc[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (int32_t)(*grand);
}
}  // namespace

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total, cudaStream_t s) {
  if (n < 0) return set_error(ZI_ERR_ARG, "scan of negative length");
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt == 0) nt = 1;
  DevTmp<int64_t> tot;
  ZI_CHECK(tot.alloc(nt + 1, s));
  k_tile_totals<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tot.p);
  ZI_LAUNCH_CHECK();
  k_scan_totals<<<1, SCAN_THREADS, 0, s>>>(tot.p, nt, tot.p + nt);
  ZI_LAUNCH_CHECK();
  k_tile_scan<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tot.p, out, tot.p + nt);
  ZI_LAUNCH_CHECK();
  if (total) {
    int64_t g = 0;
    ZI_CUDA(cudaMemcpyAsync(&g, tot.p + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ZI_CUDA(cudaStreamSynchronize(s));
    if (g > INT32_MAX) return set_error(ZI_ERR_ARG, "scan total %lld exceeds int32 range", (long long)g);
    *total = g;
  }
  return ZI_OK;
}

}  // namespace zi

extern "C" {

int zi_version(void) { return 10000; }

int64_t zi_kernel_launches(void) { return zi::launches_total(); }

int zi_memory_stats(int64_t* used_now, int64_t* used_high, int reset_high) {
  cudaMemPool_t pool = nullptr;
  ZI_CHECK(zi::get_pool(&pool));
  uint64_t cur = 0, high = 0;
  ZI_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur));
  ZI_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
  if (used_now) *used_now = (int64_t)cur;
  if (used_high) *used_high = (int64_t)high;
  if (reset_high) {
    uint64_t zero = 0;
    ZI_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  }
  return ZI_OK;
}

int zi_last_error(char* buf, size_t len) {
  if (buf && len) {
    strncpy(buf, zi::g_msg, len - 1);
    buf[len - 1] = '\0';
  }
  return zi::g_status;
}

const char* zi_status_string(int st) {
  switch (st) {
    case ZI_OK: return "ZI_OK";
    case ZI_ERR_ARG: return "ZI_ERR_ARG";
    case ZI_ERR_BAD_MESH: return "ZI_ERR_BAD_MESH";
    case ZI_ERR_NONFINITE: return "ZI_ERR_NONFINITE";
    case ZI_ERR_NOT_CONVERGED: return "ZI_ERR_NOT_CONVERGED";
    case ZI_ERR_TIMEOUT: return "ZI_ERR_TIMEOUT";
    case ZI_ERR_CUDA: return "ZI_ERR_CUDA";
    case ZI_ERR_NOMEM: return "ZI_ERR_NOMEM";
    default: return "ZI_ERR_UNKNOWN";
  }
}

}  // extern "C"
