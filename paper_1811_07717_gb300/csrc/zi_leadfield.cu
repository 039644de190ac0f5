// EEG lead field (App. A.2, Eq. aku):
//   L = R (C - B^T T)^-1 T^T F            (complete electrode model)
//   L = T^T F                             (point electrodes, electrode 0 as reference)
// with F the partial-integration source matrix, F[i, 3p+d] = d psi_i / d x_d on
// the tet holding dipole p (the paper's G is -F).
//
// Kernels: the sparse source application H^T = F^T T (one warp per dipole,
// four gathered rows of T), the electrode Schur matrix S = C - B^T T over the
// patch nodes, a single-block Cholesky inverse of S, and a tiled FP64 product
// L = (R S^-1) H.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "zi_internal.cuh"
#include "zi_pcg.cuh"

namespace zi {
namespace {

// Ht[3p+d][l] = sum_a T[v_a][l] * d lambda_a / d x_d  on tet dip_tet[p].
__global__ void k_source_apply(int64_t P, const int32_t* __restrict__ dip_tet, int64_t m,
                               const int32_t* __restrict__ tets, const double* __restrict__ X,
                               const double* __restrict__ T, int ncol, double* __restrict__ Ht,
                               int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
    int32_t t = dip_tet[p];
    if (t < 0 || t >= m) {
      if (lane == 0) atomicOr(err, DEV_ERR_OUTSIDE);
      continue;
    }
    int4 v = reinterpret_cast<const int4*>(tets)[t];
    int32_t vv[4] = {v.x, v.y, v.z, v.w};
    double x0[3], e[3][3];
    for (int d = 0; d < 3; ++d) x0[d] = X[3 * (int64_t)v.x + d];
    for (int d = 0; d < 3; ++d) {
      e[0][d] = X[3 * (int64_t)v.y + d] - x0[d];
      e[1][d] = X[3 * (int64_t)v.z + d] - x0[d];
      e[2][d] = X[3 * (int64_t)v.w + d] - x0[d];
    }
    double g[4][3];
    g[1][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
    g[1][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
    g[1][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
    g[2][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
    g[2][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
    g[2][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
    g[3][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    g[3][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    g[3][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    double det = e[0][0] * g[1][0] + e[0][1] * g[1][1] + e[0][2] * g[1][2];
    double inv = 1.0 / det;
    for (int a = 1; a < 4; ++a)
      for (int d = 0; d < 3; ++d) g[a][d] *= inv;
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    for (int l = lane; l < ncol; l += 32) {
      double tv[4];
      for (int a = 0; a < 4; ++a) tv[a] = T[(int64_t)vv[a] * ncol + l];
      for (int d = 0; d < 3; ++d) {
        double h = 0.0;
        for (int a = 0; a < 4; ++a) h += tv[a] * g[a][d];
        Ht[(3 * p + d) * (int64_t)ncol + l] = h;
      }
    }
  }
}

// Ht[c][l] = sum_j Fw[c][j] * T[Fn[c][j]][l]: a source matrix F given column
// by column with K stored entries each (the H(div) stencils of
// zi_source_stencil, or any caller's F).  One warp per column; lane j < K
// holds entry j and broadcasts it, lanes then run over the columns of T.
__global__ void k_source_apply_ell(int64_t ncols, int K, const int32_t* __restrict__ Fn,
                                   const double* __restrict__ Fw, int64_t n, const double* __restrict__ T,
                                   int ncol, double* __restrict__ Ht, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncols; c += warps) {
    int32_t node = 0;
    double w = 0.0;
    if (lane < K) {
      node = Fn[c * K + lane];
      w = Fw[c * K + lane];
    }
    const bool bad = lane < K && (node < 0 || node >= n || !isfinite(w));
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) atomicOr(err, DEV_ERR_BAD_INDEX);
      for (int l = lane; l < ncol; l += 32) Ht[c * ncol + l] = 0.0;
      continue;
    }
    for (int l = lane; l < ncol; l += 32) {
      double h = 0.0;
      for (int j = 0; j < K; ++j) {
        const int32_t nj = __shfl_sync(0xffffffffu, node, j);
        const double wj = __shfl_sync(0xffffffffu, w, j);
        h = fma(wj, T[(int64_t)nj * ncol + l], h);
      }
      Ht[c * ncol + l] = h;
    }
  }
}

// S[k][l] = C_k delta_kl - sum over patch nodes i (ascending) of B[i][k] T[i][l].
// S = C - B^T T over the patch nodes (App. A.2).  Column k of B is nonzero
// only on electrode k's patch nodes, so block k first compacts, in node
// order, the patch nodes with b_ik != 0 (a ballot per warp, warp offsets in
// shared memory) and then sums over that short list; the FMA chain is the
// one over all patch nodes minus its zero terms.  Thread l owns column l
// (L <= blockDim.x).
__global__ void __launch_bounds__(256) k_schur(int L, int64_t np_, const int32_t* __restrict__ pn,
                                               const double* __restrict__ B, const double* __restrict__ T,
                                               const double* __restrict__ C, double* __restrict__ S) {
  const int k = blockIdx.x;
  __shared__ int32_t nodes[256];
  __shared__ double bval[256];
  __shared__ int wcnt[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t base = 0; base < np_; base += blockDim.x) {
    const int64_t q = base + threadIdx.x;
    int32_t i = -1;
    double b = 0.0;
    if (q < np_) {
      i = pn[q];
      b = B[(int64_t)i * L + k];
    }
    const unsigned m = __ballot_sync(0xffffffffu, b != 0.0);
    if (lane == 0) wcnt[w] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
      if (ww < w) off += wcnt[ww];
      tot += wcnt[ww];
    }
    if (b != 0.0) {
      const int pos = off + __popc(m & ((1u << lane) - 1u));
      nodes[pos] = i;
      bval[pos] = b;
    }
    __syncthreads();
    if (threadIdx.x < L)
      for (int t = 0; t < tot; ++t) s += bval[t] * T[(int64_t)nodes[t] * L + threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x < L) S[(int64_t)k * L + threadIdx.x] = (k == (int)threadIdx.x ? C[k] : 0.0) - s;
}

// Single block: Cholesky factor A = G G^T of the SPD L x L matrix, in place
// (G in the lower triangle, G^T mirrored into the upper one); a non-positive
// pivot sets DEV_ERR_NOT_SPD.  k_chol_solve then forms (R) A^-1.
__global__ void __launch_bounds__(1024) k_chol(int L, double* __restrict__ A, int* __restrict__ err) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < L; ++j) {
    // A[j][j] holds the updated pivot
    double d = A[(int64_t)j * L + j];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) bad = 1;
    }
    __syncthreads();
    if (bad) break;
    double sd = sqrt(d);
    for (int i = j + 1 + threadIdx.x; i < L; i += blockDim.x) {
      const double g = A[(int64_t)i * L + j] / sd;
      A[(int64_t)i * L + j] = g;
      A[(int64_t)j * L + i] = g;  // G^T in the upper triangle, for row-wise back substitution
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)j * L + j] = sd;
    // trailing update of the lower triangle: A[i][k] -= A[i][j] A[k][j], j < k <= i
    int64_t rem = L - j - 1;
    int64_t tot = rem * (rem + 1) / 2;
    for (int64_t q = threadIdx.x; q < tot; q += blockDim.x) {
      // map q -> (i, k) with k <= i inside the trailing block
      int64_t ii = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
      while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
      while (ii * (ii + 1) / 2 > q) --ii;
      int64_t kk = q - ii * (ii + 1) / 2;
      int64_t i = j + 1 + ii, k = j + 1 + kk;
      A[i * L + k] -= A[i * L + j] * A[k * L + j];
    }
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(err, DEV_ERR_NOT_SPD);
}

// Column c of Xout = A^-1 (A = G G^T from k_chol), one warp per column:
// forward G y = e_c and backward G^T x = y, each step a warp-wide dot (lane l
// takes k = l mod 32) over y / x held in shared memory.  avg_ref: then
// x -= mean(x) (the average-reference rows of R S^-1).
__global__ void __launch_bounds__(32) k_chol_solve(int L, const double* __restrict__ A, double* __restrict__ Xout,
                                                   int avg_ref, const int* __restrict__ err) {
  if (*(volatile const int*)err) return;
  __shared__ double y[256];
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int i = 0; i < L; ++i) {
    double s = 0.0;
    for (int k = lane; k < i; k += 32) s += A[(int64_t)i * L + k] * y[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = ((i == c ? 1.0 : 0.0) - s) / A[(int64_t)i * L + i];
    __syncwarp();
  }
  for (int i = L - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + lane; k < L; k += 32) s += A[(int64_t)i * L + k] * y[k];  // upper triangle = G^T
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = (y[i] - s) / A[(int64_t)i * L + i];
    __syncwarp();
  }
  double mean = 0.0;
  if (avg_ref) {
    for (int i = lane; i < L; i += 32) mean += y[i];
    for (int o = 16; o > 0; o >>= 1) mean += __shfl_xor_sync(0xffffffffu, mean, o);
    mean /= L;
  }
  for (int i = lane; i < L; i += 32) Xout[(int64_t)i * L + c] = y[i] - mean;
}

// Out[r][j] = sum_k A[r][k] * Ht[j][k]   (Out: Lr x N, A: Lr x K, Ht: N x K),
// 64 x 64 output tiles, 4 x 4 per thread, K in steps of 16 through shared memory.
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) k_gemm_abt(int Lr, int K, int64_t N, const double* __restrict__ A,
                                                  const double* __restrict__ Ht, double* __restrict__ Out) {
  __shared__ double sa[GK][GT + 1];
  __shared__ double sb[GK][GT + 1];
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  const int r0 = blockIdx.y * GT;
  const int64_t j0 = (int64_t)blockIdx.x * GT;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int q = threadIdx.x; q < GT * GK; q += blockDim.x) {
      int rr = q / GK, kk = q % GK;
      int r = r0 + rr, k = k0 + kk;
      sa[kk][rr] = (r < Lr && k < K) ? A[(int64_t)r * K + k] : 0.0;
      int64_t j = j0 + rr;
      sb[kk][rr] = (j < N && k < K) ? Ht[j * K + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = sa[kk][tr + 16 * u];
        b[u] = sb[kk][tc + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int r = r0 + tr + 16 * u;
    if (r >= Lr) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int64_t j = j0 + tc + 16 * v;
      if (j < N) Out[(int64_t)r * N + j] = acc[u][v];
    }
  }
}

// Out[r][j] = Ht[j][r]
__global__ void k_transpose(int R_, int64_t N, const double* __restrict__ Ht, double* __restrict__ Out) {
  __shared__ double tile[32][33];
  int64_t j0 = (int64_t)blockIdx.x * 32;
  int r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int64_t j = j0 + y;
    int r = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (j < N && r < R_) ? Ht[j * R_ + r] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int r = r0 + y;
    int64_t j = j0 + threadIdx.x;
    if (r < R_ && j < N) Out[(int64_t)r * N + j] = tile[threadIdx.x][y];
  }
}

}  // namespace

int read_dev_err(int* derr, cudaStream_t s) {
  int h = 0;
  ZI_CUDA(cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(h);
}

int schur_matrix(zi_system* S, double* Sm, cudaStream_t s) {
  const int L = S->n_el;
  if (L > 256) return set_error(ZI_ERR_ARG, "more than 256 electrodes");
  k_schur<<<L, 256, 0, s>>>(L, S->n_patch_nodes, S->patch_nodes, S->B, S->T, S->C, Sm);
  ZI_LAUNCH_CHECK();
  return ZI_OK;
}

// Xout = (R) S^-1 for the CEM Schur matrix; S is overwritten.
int schur_inverse(zi_system* S, double* Sm, double* Xout, int avg_ref, cudaStream_t s) {
  DevTmp<int> err;
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  if (S->n_el > 256) return set_error(ZI_ERR_ARG, "more than 256 electrodes");
  k_chol<<<1, 1024, 0, s>>>(S->n_el, Sm, err.p);
  ZI_LAUNCH_CHECK();
  k_chol_solve<<<S->n_el, 32, 0, s>>>(S->n_el, Sm, Xout, avg_ref, err.p);
  ZI_LAUNCH_CHECK();
  return read_dev_err(err.p, s);
}

int leadfield_impl(zi_system* S, const int32_t* dip_tet, int64_t P, double* Lout, cudaStream_t s) {
  const int ncol = S->n_rhs;
  DevTmp<double> Ht;
  DevTmp<int> err;
  ZI_CHECK(Ht.alloc((size_t)3 * P * ncol, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_source_apply<<<grid_for(P * 32, 256, 152u * 64u), 256, 0, s>>>(P, dip_tet, S->m, S->tets, S->nodes, S->T, ncol,
                                                                  Ht.p, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(read_dev_err(err.p, s));
  return leadfield_finish(S, Ht.p, 3 * P, Lout, s);
}

int source_apply_ell(int64_t ncols, int K, const int32_t* Fn, const double* Fw, int64_t n, const double* T, int ncol,
                     double* Ht, int* err, cudaStream_t s) {
  k_source_apply_ell<<<grid_for(ncols * 32, 256, 152u * 64u), 256, 0, s>>>(ncols, K, Fn, Fw, n, T, ncol, Ht, err);
  ZI_LAUNCH_CHECK();
  return ZI_OK;
}

int leadfield_sparse_impl(zi_system* S, const int32_t* Fn, const double* Fw, int64_t ncols, int K, double* Lout,
                          cudaStream_t s) {
  const int ncol = S->n_rhs;
  DevTmp<double> Ht;
  DevTmp<int> err;
  ZI_CHECK(Ht.alloc((size_t)ncols * ncol, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  ZI_CHECK(source_apply_ell(ncols, K, Fn, Fw, S->n, S->T, ncol, Ht.p, err.p, s));
  ZI_CHECK(read_dev_err(err.p, s));
  return leadfield_finish(S, Ht.p, ncols, Lout, s);
}

// L from Ht = (T^T F)^T (N x n_rhs): L = R S^-1 H (CEM) or H (point electrodes).
int leadfield_finish(zi_system* S, const double* Ht, int64_t N, double* Lout, cudaStream_t s) {
  const int ncol = S->n_rhs;
  if (S->model == ZI_ELECTRODE_CEM) {
    const int L = S->n_el;
    DevTmp<double> Sm, Wm;
    ZI_CHECK(Sm.alloc((size_t)L * L, s));
    ZI_CHECK(Wm.alloc((size_t)L * L, s));
    ZI_CHECK(schur_matrix(S, Sm.p, s));
    ZI_CHECK(schur_inverse(S, Sm.p, Wm.p, 1, s));
    dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((L + GT - 1) / GT));
    k_gemm_abt<<<grid, 256, 0, s>>>(L, L, N, Wm.p, Ht, Lout);
    ZI_LAUNCH_CHECK();
  } else {
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((ncol + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(ncol, N, Ht, Lout);
    ZI_LAUNCH_CHECK();
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}

}  // namespace zi

using namespace zi;

extern "C" int zi_leadfield(zi_system* S, const int32_t* dip_tet, int64_t P, const zi_solver_opts* o, double* L,
                            cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative dipole count");
  if (P > 0 && (!dip_tet || !L)) return set_error(ZI_ERR_ARG, "null dipole or output array");
  if (!S->has_T) {
    ZI_CHECK(check_opts(o));
    int st = transfer_impl(S, o, nullptr, nullptr, nullptr, s);
    if (st != ZI_OK && st != ZI_ERR_NOT_CONVERGED) return st;
    if (st == ZI_ERR_NOT_CONVERGED) {
      if (P > 0) ZI_CHECK(leadfield_impl(S, dip_tet, P, L, s));
      return set_error(ZI_ERR_NOT_CONVERGED, "transfer solve did not reach tol; L written from the last iterate");
    }
  }
  if (P == 0) return ZI_OK;
  return leadfield_impl(S, dip_tet, P, L, s);
}

extern "C" int zi_leadfield_sparse(zi_system* S, const int32_t* F_nodes, const double* F_w, int64_t ncols, int K,
                                   const zi_solver_opts* o, double* L, cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (ncols < 0) return set_error(ZI_ERR_ARG, "negative column count");
  if (K < 1 || K > 32) return set_error(ZI_ERR_ARG, "entries per column must be in 1..32 (got %d)", K);
  if (ncols > 0 && (!F_nodes || !F_w || !L)) return set_error(ZI_ERR_ARG, "null source or output array");
  if (!S->has_T) {
    ZI_CHECK(check_opts(o));
    int st = transfer_impl(S, o, nullptr, nullptr, nullptr, s);
    if (st != ZI_OK && st != ZI_ERR_NOT_CONVERGED) return st;
    if (st == ZI_ERR_NOT_CONVERGED) {
      if (ncols > 0) ZI_CHECK(leadfield_sparse_impl(S, F_nodes, F_w, ncols, K, L, s));
      return set_error(ZI_ERR_NOT_CONVERGED, "transfer solve did not reach tol; L written from the last iterate");
    }
  }
  if (ncols == 0) return ZI_OK;
  return leadfield_sparse_impl(S, F_nodes, F_w, ncols, K, L, s);
}

namespace zi {
namespace {
__global__ void k_flush_l2(int64_t n, float* __restrict__ buf, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = v;
}
}  // namespace
}  // namespace zi

extern "C" int zi_time_source_apply(zi_system* S, const int32_t* F_nodes, const double* F_w, int64_t ncols, int K,
                                    int reps, double* ms_per_launch, double* bytes_per_launch, cudaStream_t s) {
  if (!S || !S->has_T) return set_error(ZI_ERR_ARG, "need a system that holds T (run zi_transfer first)");
  if (ncols < 1 || K < 1 || K > 32 || reps < 1 || !F_nodes || !F_w || !ms_per_launch)
    return set_error(ZI_ERR_ARG, "bad arguments");
  const int ncol = S->n_rhs;
  DevTmp<double> Ht;
  DevTmp<int> err;
  DevTmp<float> flush;
  const int64_t nflush = 64ll << 20;  // 64 Mi floats = 256 MB, twice the L2
  ZI_CHECK(Ht.alloc((size_t)ncols * ncol, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CHECK(flush.alloc(nflush, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  EventSet ev;
  ZI_CUDA(ev.create(2 * (size_t)reps));
  for (int r = 0; r < reps; ++r) {
    k_flush_l2<<<sm_count() * 8, 256, 0, s>>>(nflush, flush.p, (float)r);
    ZI_LAUNCH_CHECK();
    ZI_CUDA(cudaEventRecord(ev[2 * r], s));
    ZI_CHECK(source_apply_ell(ncols, K, F_nodes, F_w, S->n, S->T, ncol, Ht.p, err.p, s));
    ZI_CUDA(cudaEventRecord(ev[2 * r + 1], s));
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  double tot = 0.0;
  for (int r = 0; r < reps; ++r) {
    float ms = 0.f;
    ZI_CUDA(cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]));
    tot += ms;
  }
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  *ms_per_launch = tot / reps;
  if (bytes_per_launch) {
    // distinct T rows per group of columns (a Cartesian source's three columns share their nodes)
    std::vector<int32_t> fn((size_t)ncols * K);
    ZI_CUDA(cudaMemcpy(fn.data(), F_nodes, sizeof(int32_t) * fn.size(), cudaMemcpyDeviceToHost));
    const int64_t grp = (ncols % 3 == 0) ? 3 : 1;
    double rows = 0.0;
    std::vector<int32_t> ids;
    for (int64_t c0 = 0; c0 < ncols; c0 += grp) {
      ids.assign(fn.begin() + c0 * K, fn.begin() + (c0 + grp) * K);
      std::sort(ids.begin(), ids.end());
      rows += (double)(std::unique(ids.begin(), ids.end()) - ids.begin());
    }
    *bytes_per_launch = (double)ncols * K * 12.0 + rows * ncol * 8.0 + (double)ncols * ncol * 8.0;
  }
  return ZI_OK;
}

// ---------------------------------------------------------------------------
// Lead field without device allocation: the same kernels as zi_leadfield, with
// their scratch (error word, H^T, S, (R) S^-1) in one fixed device array.
// ---------------------------------------------------------------------------

namespace zi {
namespace {

constexpr size_t NOALLOC_WORDS = ZI_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr size_t NOALLOC_HEAD = 256 / sizeof(double);  // error word lives here

// In host code this name is only a stand-in for the device array; kernels get
// the device address looked up below.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_WORDS];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64];

// Device address of the scratch on the current device, looked up once per
// device with that device current and kept for the life of the process: the
// cache assumes one primary context per device for the whole process (a
// cudaDeviceReset or a re-created context would leave a stale address).
int noalloc_scratch(void** out) {
  int dev = 0;
  ZI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(ZI_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return ZI_OK;
}

int noalloc_read_err(int* derr, cudaStream_t s) {
  int h = 0;
  ZI_CUDA(cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(h);
}

}  // namespace
}  // namespace zi

extern "C" int zi_leadfield_noalloc(zi_system* S, const int32_t* dip_tet, int64_t P, double* Lout, cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative dipole count");
  if (P > 0 && (!dip_tet || !Lout)) return set_error(ZI_ERR_ARG, "null dipole or output array");
  if (!S->has_T) return set_error(ZI_ERR_ARG, "the system holds no transfer matrix: run zi_transfer first");
  if (P == 0) return ZI_OK;
  const int ncol = S->n_rhs;
  const bool cem = S->model == ZI_ELECTRODE_CEM;
  const int L = S->n_el;
  const size_t avail = NOALLOC_WORDS - NOALLOC_HEAD;
  const double need = 3.0 * (double)P * ncol + (cem ? 2.0 * (double)L * L : 0.0);
  if (need > (double)avail)
    return set_error(ZI_ERR_ARG,
                     "zi_leadfield_noalloc needs %.0f doubles of scratch for P=%lld and %d rows; the fixed scratch "
                     "holds %zu (ZI_NOALLOC_SCRATCH_BYTES = %u)",
                     need, (long long)P, ncol, avail, (unsigned)ZI_NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  ZI_CHECK(noalloc_scratch(&base));
  int* err = static_cast<int*>(base);
  double* Ht = static_cast<double*>(base) + NOALLOC_HEAD;
  double* Sm = Ht + (size_t)3 * P * ncol;
  double* Wm = Sm + (size_t)L * L;
  // the error word keeps the previous call's value: clear it
  ZI_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_source_apply<<<grid_for(P * 32, 256, 152u * 64u), 256, 0, s>>>(P, dip_tet, S->m, S->tets, S->nodes, S->T, ncol,
                                                                  Ht, err);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(noalloc_read_err(err, s));
  const int64_t N = 3 * P;
  if (cem) {
    ZI_CHECK(schur_matrix(S, Sm, s));
    k_chol<<<1, 1024, 0, s>>>(L, Sm, err);
    ZI_LAUNCH_CHECK();
    k_chol_solve<<<L, 32, 0, s>>>(L, Sm, Wm, 1, err);
    ZI_LAUNCH_CHECK();
    ZI_CHECK(noalloc_read_err(err, s));
    dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((L + GT - 1) / GT));
    k_gemm_abt<<<grid, 256, 0, s>>>(L, L, N, Wm, Ht, Lout);
    ZI_LAUNCH_CHECK();
  } else {
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((ncol + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(ncol, N, Ht, Lout);
    ZI_LAUNCH_CHECK();
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}
