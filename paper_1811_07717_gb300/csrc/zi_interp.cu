// Source interpolation (Sec. 2.5 keeps an index array that links mesh nodes
// to DOFs; Sec. 3.2 groups DOFs around random centres by distance): for
// every point, the nearest DOF position, ties to the lowest index.  Squared distances are formed as
// (dx*dx + dy*dy) + dz*dz with every operation rounded once (no contraction),
// so the comparison, and the index it picks, is exact and reproducible.
//
// One thread per point; the DOF positions stream through shared memory in
// tiles of NN_TILE, so each block reads them once per tile.
#include <math.h>

#include "zi_internal.cuh"

namespace zi {
namespace {

constexpr int NN_TILE = 256;

__global__ void __launch_bounds__(NN_TILE) k_nearest(int64_t n, const double* __restrict__ X, int64_t P,
                                                     const double* __restrict__ S, int32_t* __restrict__ out,
                                                     int* __restrict__ err) {
  __shared__ double sx[NN_TILE], sy[NN_TILE], sz[NN_TILE];
  for (int64_t base = (int64_t)blockIdx.x * NN_TILE; base < n; base += (int64_t)gridDim.x * NN_TILE) {
    const int64_t i = base + threadIdx.x;
    const bool act = i < n;
    double x = 0.0, y = 0.0, z = 0.0;
    if (act) {
      x = X[3 * i];
      y = X[3 * i + 1];
      z = X[3 * i + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(err, DEV_ERR_NONFINITE);
    }
    double best = INFINITY;
    int32_t bi = -1;
    for (int64_t p0 = 0; p0 < P; p0 += NN_TILE) {
      __syncthreads();
      const int64_t p = p0 + threadIdx.x;
      if (p < P) {
        sx[threadIdx.x] = S[3 * p];
        sy[threadIdx.x] = S[3 * p + 1];
        sz[threadIdx.x] = S[3 * p + 2];
        if (!isfinite(sx[threadIdx.x]) || !isfinite(sy[threadIdx.x]) || !isfinite(sz[threadIdx.x]))
          atomicOr(err, DEV_ERR_NONFINITE);
      }
      __syncthreads();
      const int cnt = (P - p0 < NN_TILE) ? (int)(P - p0) : NN_TILE;
      if (act) {
        for (int j = 0; j < cnt; ++j) {
          const double dx = __dsub_rn(x, sx[j]), dy = __dsub_rn(y, sy[j]), dz = __dsub_rn(z, sz[j]);
          const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          if (d2 < best) {
            best = d2;
            bi = (int32_t)(p0 + j);
          }
        }
      }
    }
    if (act) out[i] = bi;
  }
}

}  // namespace
}  // namespace zi

using namespace zi;

extern "C" int zi_nearest_source(const double* points, int64_t n, const double* sources, int64_t P, int32_t* out,
                                 cudaStream_t s) {
  if (n < 0 || P < 1 || P > INT32_MAX) return set_error(ZI_ERR_ARG, "need n >= 0 points and 1..2^31-1 sources");
  if (n == 0) return ZI_OK;
  if (!points || !sources || !out) return set_error(ZI_ERR_ARG, "null input or output array");
  DevTmp<int> err;
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_nearest<<<grid_for(n, NN_TILE, 152u * 16u), NN_TILE, 0, s>>>(n, points, P, sources, out, err.p);
  ZI_LAUNCH_CHECK();
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}
