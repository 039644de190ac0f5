// Linearised EIT (App. A.3).  With M = C - B^T A^-1 B = C - B^T T,
//   y_p = R M^-1 I_p,
//   dy_{p,k} / d log s_m = -u_p^T K_m w_k,   u_p = T M^-1 I_p,  w_k = T M^-1 R e_k,
// where K_m is element m's stiffness at the current conductivity (the
// conductivity of element m is s_m times its tensor, so dA/d log s_m = K_m;
// the electrode terms do not depend on s).  The full Jacobian is contracted
// per tet from the four gathered rows of U and W; the vector-Jacobian product
// contracts U with V = W G^T instead, so it never forms the Jacobian.
#include <math.h>

#include <vector>

#include "zi_internal.cuh"
#include "zi_pcg.cuh"

namespace zi {

int read_dev_err(int* derr, cudaStream_t s);
int schur_inverse(zi_system* S, double* Sm, double* Xout, int avg_ref, cudaStream_t s);

namespace {

__constant__ int e_sym[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};

// Out (n x q) = T (n x L) * Cm (L x q), Cm staged in shared memory; one warp
// per row, lanes over q.
__global__ void k_right_mult(int64_t n, int L, int q, const double* __restrict__ T, const double* __restrict__ Cm,
                             double* __restrict__ Out) {
  extern __shared__ double sc[];
  for (int e = threadIdx.x; e < L * q; e += blockDim.x) sc[e] = Cm[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    for (int c0 = 0; c0 < q; c0 += 32) {
      int c = c0 + lane;
      double s = 0.0;
      for (int l = 0; l < L; ++l) {
        double t = T[i * L + l];
        if (c < q) s += t * sc[l * q + c];
      }
      if (c < q) Out[i * q + c] = s;
    }
  }
}

// Small dense products on one block: D (r x c) = A (r x k) * B (k x c), with
// optional transposes expressed through strides.
__global__ void k_small_gemm(int r, int c, int k, const double* __restrict__ A, int sar, int sak,
                             const double* __restrict__ Bm, int sbk, int sbc, double* __restrict__ D) {
  for (int e = threadIdx.x; e < r * c; e += blockDim.x) {
    int i = e / c, j = e % c;
    double s = 0.0;
    for (int q = 0; q < k; ++q) s += A[i * sar + q * sak] * Bm[q * sbk + j * sbc];
    D[e] = s;
  }
}

// D (c x r) = A^T for A (r x c).
__global__ void k_small_transpose(int r, int c, const double* __restrict__ A, double* __restrict__ D) {
  for (int e = threadIdx.x; e < r * c; e += blockDim.x) {
    int i = e / c, j = e % c;
    D[(int64_t)j * r + i] = A[e];
  }
}

// Full Jacobian: out[m][p][k] = -sum_{a,b} U[v_a][p] K_m[a][b] W[v_b][k].
// One warp per tet; lanes over k.
__global__ void k_eit_full(int64_t m, const int32_t* __restrict__ tets, const double* __restrict__ Ke, int np_,
                           int L, const double* __restrict__ U, const double* __restrict__ W,
                           double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < m; t += warps) {
    int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    int64_t v[4] = {v4.x, v4.y, v4.z, v4.w};
    double K[10];
    for (int e = 0; e < 10; ++e) K[e] = Ke[10 * t + e];
    double* o = out + t * (int64_t)np_ * L;
    for (int k0 = 0; k0 < L; k0 += 32) {
      int k = k0 + lane;
      double kw[4] = {0, 0, 0, 0};
      if (k < L) {
        double w[4];
        for (int b = 0; b < 4; ++b) w[b] = W[v[b] * L + k];
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) kw[a] += K[e_sym[a][b]] * w[b];
      }
      for (int p = 0; p < np_; ++p) {
        double u[4];
        for (int a = 0; a < 4; ++a) u[a] = U[v[a] * np_ + p];
        double s = -(u[0] * kw[0] + u[1] * kw[1] + u[2] * kw[2] + u[3] * kw[3]);
        if (k < L) o[(int64_t)p * L + k] = s;
      }
    }
  }
}

// VJP: g_m = -sum_{a,b} K_m[a][b] sum_p U[v_a][p] V[v_b][p].  One warp per
// tet, lanes over p, fixed-order warp reduction.
__global__ void k_eit_vjp(int64_t m, const int32_t* __restrict__ tets, const double* __restrict__ Ke, int np_,
                          const double* __restrict__ U, const double* __restrict__ V, double* __restrict__ g) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < m; t += warps) {
    int4 v4 = reinterpret_cast<const int4*>(tets)[t];
    int64_t v[4] = {v4.x, v4.y, v4.z, v4.w};
    double K[10];
    for (int e = 0; e < 10; ++e) K[e] = Ke[10 * t + e];
    double s = 0.0;
    for (int p = lane; p < np_; p += 32) {
      double u[4], w[4];
      for (int a = 0; a < 4; ++a) {
        u[a] = U[v[a] * np_ + p];
        w[a] = V[v[a] * np_ + p];
      }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) s += u[a] * K[e_sym[a][b]] * w[b];
    }
    s = warp_sum(s);
    if (lane == 0) g[t] = -s;
  }
}

}  // namespace

int eit_impl(zi_system* S, const double* I, int np_, int mode, const double* grad_y, double* out, double* y,
             cudaStream_t s) {
  const int L = S->n_el;
  const int64_t n = S->n;
  DevTmp<double> Sm, X, RX, Cu, Cw, Cv, U, W;
  ZI_CHECK(Sm.alloc((size_t)L * L, s));
  ZI_CHECK(X.alloc((size_t)L * L, s));
  ZI_CHECK(RX.alloc((size_t)L * L, s));
  ZI_CHECK(schur_matrix(S, Sm.p, s));
  ZI_CHECK(schur_inverse(S, Sm.p, X.p, 0, s));  // X = M^-1
  ZI_CHECK(schur_matrix(S, Sm.p, s));
  ZI_CHECK(schur_inverse(S, Sm.p, RX.p, 1, s));  // RX = R M^-1
  // y[p][k] = sum_m (R M^-1)[k][m] I[p][m]  ->  y = I (R M^-1)^T
  if (y) {
    k_small_gemm<<<1, 256, 0, s>>>(np_, L, L, I, L, 1, RX.p, 1, L, y);
    ZI_LAUNCH_CHECK();
  }
  if (!out) {
    ZI_CUDA(cudaStreamSynchronize(s));
    return ZI_OK;
  }
  // Cu = M^-1 I^T (L x np), Cw = M^-1 R (L x L) = (R M^-1)^T
  ZI_CHECK(Cu.alloc((size_t)L * np_, s));
  ZI_CHECK(Cw.alloc((size_t)L * L, s));
  k_small_gemm<<<1, 256, 0, s>>>(L, np_, L, X.p, L, 1, I, 1, L, Cu.p);
  ZI_LAUNCH_CHECK();
  k_small_transpose<<<1, 256, 0, s>>>(L, L, RX.p, Cw.p);  // Cw = M^-1 R = (R M^-1)^T
  ZI_LAUNCH_CHECK();
  size_t smem_u = sizeof(double) * (size_t)L * np_;
  if (smem_u > 200 * 1024) return set_error(ZI_ERR_ARG, "EIT pattern block too large for shared memory");
  ZI_CHECK(U.alloc((size_t)n * np_, s));
  ZI_CUDA(cudaFuncSetAttribute(k_right_mult, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  k_right_mult<<<grid_for(n * 32, 256, 152u * 16u), 256, smem_u, s>>>(n, L, np_, S->T, Cu.p, U.p);
  ZI_LAUNCH_CHECK();
  if (mode == ZI_EIT_FULL) {
    size_t smem_w = sizeof(double) * (size_t)L * L;
    if (smem_w > 200 * 1024) return set_error(ZI_ERR_ARG, "too many electrodes for the EIT kernels");
    ZI_CHECK(W.alloc((size_t)n * L, s));
    k_right_mult<<<grid_for(n * 32, 256, 152u * 16u), 256, smem_w, s>>>(n, L, L, S->T, Cw.p, W.p);
    ZI_LAUNCH_CHECK();
    k_eit_full<<<grid_for(S->m * 32, 256, 152u * 64u), 256, 0, s>>>(S->m, S->tets, S->Ke, np_, L, U.p, W.p, out);
    ZI_LAUNCH_CHECK();
  } else {
    // Cv = Cw G^T (L x np): Cv[l][p] = sum_k Cw[l][k] grad_y[p][k]
    ZI_CHECK(Cv.alloc((size_t)L * np_, s));
    k_small_gemm<<<1, 256, 0, s>>>(L, np_, L, Cw.p, L, 1, grad_y, 1, L, Cv.p);
    ZI_LAUNCH_CHECK();
    ZI_CHECK(W.alloc((size_t)n * np_, s));
    k_right_mult<<<grid_for(n * 32, 256, 152u * 16u), 256, smem_u, s>>>(n, L, np_, S->T, Cv.p, W.p);
    ZI_LAUNCH_CHECK();
    k_eit_vjp<<<grid_for(S->m * 32, 256, 152u * 64u), 256, 0, s>>>(S->m, S->tets, S->Ke, np_, U.p, W.p, out);
    ZI_LAUNCH_CHECK();
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}

}  // namespace zi

using namespace zi;

extern "C" int zi_eit_jacobian(zi_system* S, const double* I, int np_, int mode, const double* grad_y, double* out,
                               double* y, const zi_solver_opts* o, cudaStream_t s) {
  if (!S || !I) return set_error(ZI_ERR_ARG, "null system or current patterns");
  if (S->model != ZI_ELECTRODE_CEM) return set_error(ZI_ERR_ARG, "EIT needs complete-electrode-model systems");
  if (np_ < 1 || np_ > 4096) return set_error(ZI_ERR_ARG, "pattern count must be in 1..4096");
  if (mode != ZI_EIT_FULL && mode != ZI_EIT_VJP) return set_error(ZI_ERR_ARG, "unknown EIT mode %d", mode);
  if (mode == ZI_EIT_VJP && out && !grad_y) return set_error(ZI_ERR_ARG, "VJP mode needs grad_y");
  if (!S->has_T) {
    ZI_CHECK(check_opts(o));
    ZI_CHECK(transfer_impl(S, o, nullptr, nullptr, nullptr, s));
  }
  return eit_impl(S, I, np_, mode, grad_y, out, y, s);
}
