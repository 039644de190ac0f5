// IAS MAP inversion (App. B): for every data column y_t, `iters` rounds of
//   x-step      x = D L^T (L D L^T + nu^2 I)^-1 y,      D = diag(theta)
//   theta-step  gamma (G):          theta_i = theta0/2 (eta + sqrt(eta^2 + 2 x_i^2/theta0)), eta = beta - 3/2
//               inverse gamma (IG): theta_i = (theta0 + x_i^2/2) / kappa,                     kappa = beta + 3/2
// from theta = theta0.  The Le x Le matrix L D L^T of each column is a
// split-K FP64 product over the sources (the step the paper moves to the GPU,
// Sec. 2.3.2), factored by Cholesky on one block per column; x and the new
// theta come out of one pass over L.
#include <algorithm>
#include <cmath>

#include "zi_internal.cuh"

namespace zi {
namespace {

constexpr int GT = 32;        // output tile of the Gram product
constexpr int GRAM_KC = 32;   // sources per shared-memory stage

// part[s][t][a][b] = sum over the sources j of slice s of L[a][j] theta_t[j] L[b][j],
// for the tiles (ti, tj) with ti >= tj (the lower triangle).  Thread (ty, tx)
// of the 16 x 16 block owns rows ty, ty + 16 and columns tx, tx + 16 of the tile.
__global__ void __launch_bounds__(256) k_ias_gram(int Le, int64_t n, int64_t chunk, const double* __restrict__ L,
                                                  const double* __restrict__ theta, double* __restrict__ part) {
  __shared__ double As[GT][GRAM_KC + 1], Bs[GT][GRAM_KC + 1];
  // lower-triangle tile index -> (ti, tj)
  int ti = 0, rem = blockIdx.x;
  while (rem > ti) {
    rem -= ti + 1;
    ++ti;
  }
  const int tj = rem;
  const int s = blockIdx.y, t = blockIdx.z, T = gridDim.z;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t j0 = (int64_t)s * chunk, j1 = min(n, j0 + chunk);
  const double* th = theta + (int64_t)t * n;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t jb = j0; jb < j1; jb += GRAM_KC) {
    for (int e = threadIdx.x; e < GT * GRAM_KC; e += blockDim.x) {
      const int r = e / GRAM_KC, k = e % GRAM_KC;
      const int64_t j = jb + k;
      const int ra = ti * GT + r, rb = tj * GT + r;
      const bool in = j < j1;
      As[r][k] = (in && ra < Le) ? L[(int64_t)ra * n + j] * th[j] : 0.0;
      Bs[r][k] = (in && rb < Le) ? L[(int64_t)rb * n + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GRAM_KC; ++k) {
      const double a0 = As[ty][k], a1 = As[ty + 16][k];
      const double b0 = Bs[tx][k], b1 = Bs[tx + 16][k];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  double* P = part + ((int64_t)s * T + t) * Le * Le;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int a = ti * GT + ty + 16 * u, b = tj * GT + tx + 16 * v;
      if (a < Le && b < Le) P[(int64_t)a * Le + b] = acc[u][v];
    }
}

// M_t[a][b] = sum_s part[s][t][a][b] (slice order) + nu^2 delta_ab, a >= b.
__global__ void k_ias_reduce(int Le, int S, int T, const double* __restrict__ part, double nu2,
                             double* __restrict__ M) {
  const int64_t tot = (int64_t)T * Le * Le;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)((e / Le) % Le), b = (int)(e % Le);
    if (b > a) continue;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += part[(int64_t)s * tot + e];
    M[e] = v + (a == b ? nu2 : 0.0);
  }
}

// Cholesky M_t = G G^T of each column's matrix (one block per column): G in
// the lower triangle, G^T mirrored into the upper one.
__global__ void __launch_bounds__(1024) k_ias_chol(int Le, double* __restrict__ Mall, int* __restrict__ err) {
  double* A = Mall + (int64_t)blockIdx.x * Le * Le;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < Le; ++j) {
    const double d = A[(int64_t)j * Le + j];
    if (threadIdx.x == 0 && !(d > 0.0)) bad = 1;
    __syncthreads();
    if (bad) break;
    const double sd = sqrt(d);
    for (int i = j + 1 + threadIdx.x; i < Le; i += blockDim.x) {
      const double g = A[(int64_t)i * Le + j] / sd;
      A[(int64_t)i * Le + j] = g;
      A[(int64_t)j * Le + i] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)j * Le + j] = sd;
    // trailing update of the lower triangle, one row i per thread group
    for (int i = j + 1 + threadIdx.x / 32; i < Le; i += blockDim.x / 32) {
      const double gi = A[(int64_t)i * Le + j];
      for (int k = j + 1 + (threadIdx.x & 31); k <= i; k += 32) A[(int64_t)i * Le + k] -= gi * A[(int64_t)k * Le + j];
    }
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(err, DEV_ERR_NOT_SPD);
}

// z_t = M_t^-1 y_t (forward with G, backward with G^T), one warp per column.
__global__ void __launch_bounds__(32) k_ias_solve(int Le, const double* __restrict__ Mall,
                                                  const double* __restrict__ Y, double* __restrict__ Z,
                                                  const int* __restrict__ err) {
  if (*(volatile const int*)err) return;
  __shared__ double z[256];
  const int t = blockIdx.x, lane = threadIdx.x;
  const double* A = Mall + (int64_t)t * Le * Le;
  const double* y = Y + (int64_t)t * Le;
  for (int i = 0; i < Le; ++i) {
    double s = 0.0;
    for (int k = lane; k < i; k += 32) s += A[(int64_t)i * Le + k] * z[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[i] = (y[i] - s) / A[(int64_t)i * Le + i];
    __syncwarp();
  }
  for (int i = Le - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k < Le; k += 32) s += A[(int64_t)i * Le + k] * z[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[i] = (z[i] - s) / A[(int64_t)i * Le + i];
    __syncwarp();
  }
  for (int i = lane; i < Le; i += 32) Z[(int64_t)t * Le + i] = z[i];
}

// x_t[j] = theta_t[j] (L^T z_t)[j], then the theta-step from that x.
__global__ void k_ias_x_theta(int Le, int64_t n, const double* __restrict__ L, const double* __restrict__ Z,
                              double* __restrict__ theta, double* __restrict__ X, double theta0, double beta,
                              int hyper) {
  __shared__ double z[256];
  const int t = blockIdx.y;
  for (int a = threadIdx.x; a < Le; a += blockDim.x) z[a] = Z[(int64_t)t * Le + a];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int a = 0; a < Le; ++a) s += L[(int64_t)a * n + j] * z[a];
    const int64_t e = (int64_t)t * n + j;
    const double x = theta[e] * s;
    X[e] = x;
    if (hyper == ZI_HYPER_G) {
      const double eta = beta - 1.5;
      theta[e] = 0.5 * theta0 * (eta + sqrt(eta * eta + 2.0 * x * x / theta0));
    } else {
      theta[e] = (theta0 + 0.5 * x * x) / (beta + 1.5);
    }
  }
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

}  // namespace

int ias_map_impl(const double* L, int Le, int64_t n, const double* Y, int T, double nu, double theta0, double beta,
                 int hyper, int iters, double* X, double* Theta, cudaStream_t s) {
  // split-K: enough slices for a few waves of blocks, each slice a multiple of the stage width
  const int ntile = (Le + GT - 1) / GT;
  const int pairs = ntile * (ntile + 1) / 2;
  int S = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)4 * sm_count() / std::max(1, pairs * T),
                                                     (n + GRAM_KC - 1) / GRAM_KC));
  const int64_t chunk = ((n + S - 1) / S + GRAM_KC - 1) / GRAM_KC * GRAM_KC;
  S = (int)((n + chunk - 1) / chunk);
  DevTmp<double> part, M, Z;
  DevTmp<int> err;
  ZI_CHECK(part.alloc((size_t)S * T * Le * Le, s));
  ZI_CHECK(M.alloc((size_t)T * Le * Le, s));
  ZI_CHECK(Z.alloc((size_t)T * Le, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  // every part entry of a lower tile is written; the upper parts of off-diagonal tiles are never read
  k_fill<<<grid_for((int64_t)T * n, 256), 256, 0, s>>>((int64_t)T * n, theta0, Theta);
  ZI_LAUNCH_CHECK();
  k_fill<<<grid_for((int64_t)T * n, 256), 256, 0, s>>>((int64_t)T * n, 0.0, X);  // iters = 0: x = 0
  ZI_LAUNCH_CHECK();
  for (int k = 0; k < iters; ++k) {
    k_ias_gram<<<dim3(pairs, S, T), 256, 0, s>>>(Le, n, chunk, L, Theta, part.p);
    ZI_LAUNCH_CHECK();
    k_ias_reduce<<<grid_for((int64_t)T * Le * Le, 256), 256, 0, s>>>(Le, S, T, part.p, nu * nu, M.p);
    ZI_LAUNCH_CHECK();
    k_ias_chol<<<T, 1024, 0, s>>>(Le, M.p, err.p);
    ZI_LAUNCH_CHECK();
    k_ias_solve<<<T, 32, 0, s>>>(Le, M.p, Y, Z.p, err.p);
    ZI_LAUNCH_CHECK();
    k_ias_x_theta<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 4 * sm_count()), T), 256, 0, s>>>(
        Le, n, L, Z.p, Theta, X, theta0, beta, hyper);
    ZI_LAUNCH_CHECK();
  }
  int h = 0;
  ZI_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(h);
}

}  // namespace zi

extern "C" int zi_ias_map(const double* L, int32_t Le, int64_t n, const double* Y, int32_t T, double nu,
                          double theta0, double beta, int32_t hypermodel, int32_t iters, double* X, double* Theta,
                          cudaStream_t stream) {
  using namespace zi;
  if (!L || !Y || !X || !Theta) return set_error(ZI_ERR_ARG, "null pointer");
  if (Le < 1 || Le > 256) return set_error(ZI_ERR_ARG, "Le must be in [1, 256] (got %d)", Le);
  if (n < 1 || T < 1 || iters < 0) return set_error(ZI_ERR_ARG, "bad sizes (n=%lld, T=%d, iters=%d)", (long long)n, T, iters);
  if (!(nu > 0.0) || !(theta0 > 0.0) || !std::isfinite(nu) || !std::isfinite(theta0) || !std::isfinite(beta))
    return set_error(ZI_ERR_ARG, "nu and theta0 must be positive and finite");
  if (hypermodel != ZI_HYPER_G && hypermodel != ZI_HYPER_IG) return set_error(ZI_ERR_ARG, "unknown hypermodel");
  if (hypermodel == ZI_HYPER_IG && !(beta + 1.5 > 0.0)) return set_error(ZI_ERR_ARG, "IG needs beta > -3/2");
  return ias_map_impl(L, Le, n, Y, T, nu, theta0, beta, hypermodel, iters, X, Theta, stream);
}
