// Internal declarations shared by the libzi translation units: error state,
// stream-ordered device memory, the system handle, and small device helpers
// (warp reductions, a device-wide exclusive scan).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "zi.h"

namespace zi {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

int set_error(int status, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define ZI_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t _e = (call);                                            \
    if (_e != cudaSuccess) return zi::cuda_error(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define ZI_CHECK(call)            \
  do {                            \
    int _s = (call);              \
    if (_s != ZI_OK) return _s;   \
  } while (0)

// Every kernel launch site is followed by ZI_LAUNCH_CHECK(), which also
// counts the launch (except while a CUDA graph is being captured: graph
// replays are counted by the code that replays them).
void count_launches(int64_t k);
#define ZI_LAUNCH_CHECK()        \
  do {                           \
    zi::count_launches(1);       \
    ZI_CUDA(cudaGetLastError()); \
  } while (0)

// Set while a graph is captured on the calling thread.
extern thread_local bool g_capturing;

// Device-side error word bits (written by kernels, read back by the host).
enum : int {
  DEV_ERR_BAD_VOLUME = 1,
  DEV_ERR_NONFINITE = 2,
  DEV_ERR_OVERLAP = 4,
  DEV_ERR_VALENCE = 8,
  DEV_ERR_OUTSIDE = 16,
  DEV_ERR_DUP_ELECTRODE = 32,
  DEV_ERR_TIMEOUT = 64,
  DEV_ERR_NO_PATCH = 128,
  DEV_ERR_NO_GROUND = 256,
  DEV_ERR_NOT_SPD = 512,
  DEV_ERR_NONMANIFOLD = 1024,
  DEV_ERR_STENCIL = 2048,
  DEV_ERR_BAD_INDEX = 4096,
};

int device_error_to_status(int dev_err);

// ---------------------------------------------------------------------------
// device memory: a private stream-ordered pool per device that keeps freed
// blocks cached, so repeated builds do not pay for cudaMalloc.
// ---------------------------------------------------------------------------

int dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
int get_pool(cudaMemPool_t* out);  // the library's pool of the current device

template <typename T>
int dalloc_n(T** p, size_t n, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0), s);
}

// RAII holder of a temporary device buffer, released stream-ordered.
template <typename T>
struct DevTmp {
  T* p = nullptr;
  cudaStream_t s = 0;
  DevTmp() = default;
  DevTmp(const DevTmp&) = delete;
  DevTmp& operator=(const DevTmp&) = delete;
  ~DevTmp() { if (p) dfree(p, s); }
  int alloc(size_t n, cudaStream_t st) {
    s = st;
    return dalloc_n(&p, n, st);
  }
};

// CUDA events that are destroyed on every exit path (timing helpers).
struct EventSet {
  std::vector<cudaEvent_t> ev;
  EventSet() = default;
  EventSet(const EventSet&) = delete;
  EventSet& operator=(const EventSet&) = delete;
  ~EventSet() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  // Creates k events; `flags` as for cudaEventCreateWithFlags.
  cudaError_t create(size_t k, unsigned flags = cudaEventDefault) {
    ev.assign(k, nullptr);
    for (auto& e : ev) {
      cudaError_t r = cudaEventCreateWithFlags(&e, flags);
      if (r != cudaSuccess) {
        e = nullptr;
        return r;
      }
    }
    return cudaSuccess;
  }
  cudaEvent_t operator[](size_t i) const { return ev[i]; }
};

// ---------------------------------------------------------------------------
// the system handle
// ---------------------------------------------------------------------------

struct SolverScratch;  // defined in zi_pcg.cu

}  // namespace zi

struct zi_system {
  int device = 0;
  int64_t n = 0, m = 0, nb = 0, nnz = 0, n_entries = 0;
  int32_t n_el = 0, n_rhs = 0, model = 0;
  int64_t ground = -1;
  int64_t n_patch_faces = 0;
  int64_t n_patch_nodes = 0;
  double el_radius = 0.0;

  // mesh (own copies)
  double* nodes = nullptr;      // n x 3
  int32_t* tets = nullptr;      // m x 4
  int32_t* bfaces = nullptr;    // nb x 3

  // element stiffness, 10 unique entries per tet: (00,01,02,03,11,12,13,22,23,33)
  double* Ke = nullptr;         // m x 10

  // CSR pattern of A (mesh graph) and the sorted element-entry -> nnz map
  int32_t* rowptr = nullptr;    // n + 1
  int32_t* colind = nullptr;    // nnz
  int32_t* diagpos = nullptr;   // n: position of (i,i) in the CSR
  int32_t* seg = nullptr;       // nnz + 1: entries of nnz k are perm[seg[k] .. seg[k+1])
  int32_t* perm = nullptr;      // n_entries: entry ids sorted by (row, col, id)
  double* vals = nullptr;       // nnz: grounded A

  // electrodes
  int32_t* face_el = nullptr;   // nb: electrode of each boundary face or -1
  double* face_w = nullptr;     // nb: area / z_l of patch faces (0 elsewhere)
  double* zinv = nullptr;       // L: 1 / z_l
  double* B = nullptr;          // n x n_rhs right-hand sides (dense, node-major)
  double* C = nullptr;          // L
  int32_t* el_nodes = nullptr;  // L (point model)
  int32_t* patch_nodes = nullptr;  // nodes with a nonzero B row (CEM), ascending

  // transfer matrix
  double* T = nullptr;          // n x n_rhs
  int has_T = 0;

  zi::SolverScratch* solver = nullptr;
};

namespace zi {

// Frees every buffer of a system (used by zi_system_destroy and error paths).
void system_free(zi_system* s);

// Helpers implemented in zi_pcg.cu / zi_leadfield.cu used across units.
int schur_matrix(zi_system* sys, double* S, cudaStream_t s);  // S = C - B^T T (L x L)
// L = R S^-1 H (CEM) or H (point electrodes) from Ht = (T^T F)^T, N x n_rhs;
// synchronises the stream.
int leadfield_finish(zi_system* sys, const double* Ht, int64_t N, double* Lout, cudaStream_t s);
// Ht[c][l] = sum_j Fw[c*K + j] * T[Fn[c*K + j]][l] for ncols columns (T: n x ncol); bad
// indices or weights set DEV_ERR_BAD_INDEX in *err (device) and zero that column.
int source_apply_ell(int64_t ncols, int K, const int32_t* Fn, const double* Fw, int64_t n, const double* T, int ncol,
                     double* Ht, int* err, cudaStream_t s);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive prefix sum of n int32 counts into out (n+1 entries, out[n] =
// total).  Returns the total through *total (host) when non-null (this
// synchronises the stream).  Totals above INT32_MAX are reported as an error.
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total, cudaStream_t s);

inline unsigned grid_for(int64_t n, int block, unsigned cap = 152u * 32u) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

int sm_count();

}  // namespace zi
