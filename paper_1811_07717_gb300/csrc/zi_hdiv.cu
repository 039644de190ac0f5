// H(div) source stencils (Sec. 2.1, primary current model).
//
// A Cartesian source (three orientations at a position x0) is a combination
// of the divergence-conforming basis functions of the tet T that holds it:
//   face source k (k = 0..3): lowest-order Raviart-Thomas function of the face
//     opposite vertex v_k, unit flux from T into the neighbour N_k.  Load
//     f = (e_{o_k} - e_{v_k}) / 4 (o_k: N_k's vertex off the face), moment
//     (x_{o_k} - x_{v_k}) / 4, position the face centroid; absent on the mesh
//     boundary.
//   edge source (a, b) (10-source stencil only): opposite unit monopoles at
//     the edge's end nodes, load e_{v_b} - e_{v_a}, moment x_{v_b} - x_{v_a},
//     position the edge midpoint.
// Position-based optimisation picks the coefficients w of orientation e_j:
// minimise  sum_{k,l} w_k w_l (d_k . d_l)(r_k . r_l) + lam sum_k (1 + |r_k|^2)|d_k|^2 w_k^2
// (r_k = (c_k - x0) / s, s the mean edge length of T: the first moment of the
// combined source about x0 plus a distance-weighted Tikhonov term) subject to
// sum_k w_k d_k = e_j.  With H that quadratic form, w = H^-1 D^T (D H^-1 D^T)^-1 e_j.
//
// The neighbour across each face comes from a node -> tet incidence list
// built here (counting sort of the 4m corners); the search result is unique,
// so the output does not depend on the incidence order.
#include <math.h>

#include "zi_internal.cuh"

namespace zi {
namespace {

constexpr int KMAX = 10;  // sources per stencil
constexpr int NW = 8;     // nodes per Cartesian source column (T's four + four across its faces)

__global__ void k_inc_count(int64_t m, const int32_t* __restrict__ tets, int64_t n, int32_t* __restrict__ cnt,
                            int* __restrict__ err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 4 * m; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = tets[q];
    if (v < 0 || v >= n) {
      atomicOr(err, DEV_ERR_BAD_INDEX);
      continue;
    }
    atomicAdd(&cnt[v], 1);
  }
}

__global__ void k_inc_fill(int64_t m, const int32_t* __restrict__ tets, int64_t n, const int32_t* __restrict__ start,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ inc) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 4 * m; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = tets[q];
    if (v < 0 || v >= n) continue;
    inc[start[v] + atomicAdd(&cursor[v], 1)] = (int32_t)(q >> 2);
  }
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One thread per source position p: neighbours, stencil, PBO coefficients,
// and the three columns 3p + j of F (NW entries each).
__global__ void __launch_bounds__(128) k_stencil(int64_t P, const double* __restrict__ pos,
                                                 const int32_t* __restrict__ dip_tet, int64_t m,
                                                 const int32_t* __restrict__ tets, int64_t n,
                                                 const double* __restrict__ X,
                                                 const int32_t* __restrict__ inc_start,
                                                 const int32_t* __restrict__ inc, int model, double lam,
                                                 int32_t* __restrict__ Fn, double* __restrict__ Fw,
                                                 int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t node[NW];
    double wn[NW][3];
    for (int i = 0; i < NW; ++i) {
      node[i] = 0;
      wn[i][0] = wn[i][1] = wn[i][2] = 0.0;
    }
    int bad = 0;
    const int32_t t = dip_tet[p];
    double x0[3];
    for (int d = 0; d < 3; ++d) {
      x0[d] = pos[3 * p + d];
      if (!isfinite(x0[d])) bad |= DEV_ERR_NONFINITE;
    }
    if (t < 0 || t >= m) bad |= DEV_ERR_OUTSIDE;
    int32_t v[4] = {0, 0, 0, 0};
    if (!bad) {
      const int4 tv = reinterpret_cast<const int4*>(tets)[t];
      v[0] = tv.x;
      v[1] = tv.y;
      v[2] = tv.z;
      v[3] = tv.w;
      for (int a = 0; a < 4; ++a)
        if (v[a] < 0 || v[a] >= n) bad |= DEV_ERR_BAD_INDEX;
    }
    if (!bad) {
      double xv[4][3];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) xv[a][d] = X[3 * (int64_t)v[a] + d];
      // the vertex across each face
      int32_t o[4];
      for (int k = 0; k < 4; ++k) {
        int32_t f[3];
        for (int j = 0, q = 0; j < 4; ++j)
          if (j != k) f[q++] = v[j];
        o[k] = -1;
        int found = 0;
        for (int32_t q = inc_start[f[0]]; q < inc_start[f[0] + 1]; ++q) {
          const int32_t u = inc[q];
          if (u == t) continue;
          const int4 uv4 = reinterpret_cast<const int4*>(tets)[u];
          const int32_t uv[4] = {uv4.x, uv4.y, uv4.z, uv4.w};
          int has1 = 0, has2 = 0, other = -1, nother = 0;
          for (int j = 0; j < 4; ++j) {
            if (uv[j] == f[1]) has1 = 1;
            else if (uv[j] == f[2]) has2 = 1;
            else if (uv[j] != f[0]) { other = uv[j]; ++nother; }
          }
          if (has1 && has2 && nother == 1) {
            ++found;
            o[k] = other;
          }
        }
        if (o[k] >= n) {  // o[k] < 0 only when nothing was found
          bad |= DEV_ERR_BAD_INDEX;
          o[k] = -1;
        }
        if (found > 1) {
          bad |= DEV_ERR_NONMANIFOLD;
          o[k] = -1;
        }
      }
      // stencil sources: moment d, position c, and where the load goes
      double dk[KMAX][3], rk[KMAX][3];
      int src_a[KMAX], src_b[KMAX];  // load: +s at slot src_b, -s at slot src_a (s = 1/4 faces, 1 edges)
      double src_s[KMAX];
      int K = 0;
      double s = 0.0;
      const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
      for (int e = 0; e < 6; ++e) {
        double u[3] = {xv[eb[e]][0] - xv[ea[e]][0], xv[eb[e]][1] - xv[ea[e]][1], xv[eb[e]][2] - xv[ea[e]][2]};
        s += sqrt(dot3(u, u));
      }
      s /= 6.0;
      for (int k = 0; k < 4; ++k) {
        if (o[k] < 0) continue;
        double c[3];
        for (int d = 0; d < 3; ++d) {
          const double xo = X[3 * (int64_t)o[k] + d];
          dk[K][d] = (xo - xv[k][d]) / 4.0;
          c[d] = 0.0;
          for (int j = 0; j < 4; ++j)
            if (j != k) c[d] += xv[j][d];
          c[d] /= 3.0;
          rk[K][d] = (c[d] - x0[d]) / s;
        }
        node[4 + k] = o[k];
        src_a[K] = k;
        src_b[K] = 4 + k;
        src_s[K] = 0.25;
        ++K;
      }
      if (model == ZI_SOURCE_PBO10) {
        for (int e = 0; e < 6; ++e) {
          for (int d = 0; d < 3; ++d) {
            dk[K][d] = xv[eb[e]][d] - xv[ea[e]][d];
            rk[K][d] = (0.5 * (xv[ea[e]][d] + xv[eb[e]][d]) - x0[d]) / s;
          }
          src_a[K] = ea[e];
          src_b[K] = eb[e];
          src_s[K] = 1.0;
          ++K;
        }
      }
      for (int a = 0; a < 4; ++a) node[a] = v[a];
      for (int k = 0; k < 4; ++k)
        if (o[k] < 0) node[4 + k] = v[k];  // weight stays 0
      // H (lower triangle, row-major packed) and its Cholesky factor in place
      double Hm[KMAX * (KMAX + 1) / 2];
      for (int k = 0; k < K; ++k)
        for (int l = 0; l <= k; ++l) {
          double h = dot3(dk[k], dk[l]) * dot3(rk[k], rk[l]);
          if (k == l) h += lam * (1.0 + dot3(rk[k], rk[k])) * dot3(dk[k], dk[k]);
          Hm[k * (k + 1) / 2 + l] = h;
        }
      for (int k = 0; k < K && !bad; ++k) {
        for (int l = 0; l <= k; ++l) {
          double a = Hm[k * (k + 1) / 2 + l];
          for (int q = 0; q < l; ++q) a -= Hm[k * (k + 1) / 2 + q] * Hm[l * (l + 1) / 2 + q];
          if (l == k) {
            if (!(a > 0.0)) {
              bad |= DEV_ERR_STENCIL;
              break;
            }
            Hm[k * (k + 1) / 2 + k] = sqrt(a);
          } else {
            Hm[k * (k + 1) / 2 + l] = a / Hm[l * (l + 1) / 2 + l];
          }
        }
      }
      if (!bad && K >= 3) {
        // Y = H^-1 D^T (K x 3): forward then backward substitution per column
        double Y[KMAX][3];
        for (int j = 0; j < 3; ++j) {
          for (int k = 0; k < K; ++k) {
            double a = dk[k][j];
            for (int q = 0; q < k; ++q) a -= Hm[k * (k + 1) / 2 + q] * Y[q][j];
            Y[k][j] = a / Hm[k * (k + 1) / 2 + k];
          }
          for (int k = K - 1; k >= 0; --k) {
            double a = Y[k][j];
            for (int q = k + 1; q < K; ++q) a -= Hm[q * (q + 1) / 2 + k] * Y[q][j];
            Y[k][j] = a / Hm[k * (k + 1) / 2 + k];
          }
        }
        // S = D Y (3 x 3, symmetric positive definite when the moments span R^3)
        double Sm[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += dk[k][a] * Y[k][b];
            Sm[a][b] = acc;
          }
        // S^-1 by cofactors; reject a near-singular S (moments not spanning R^3)
        const double c00 = Sm[1][1] * Sm[2][2] - Sm[1][2] * Sm[2][1];
        const double c01 = Sm[1][2] * Sm[2][0] - Sm[1][0] * Sm[2][2];
        const double c02 = Sm[1][0] * Sm[2][1] - Sm[1][1] * Sm[2][0];
        const double det = Sm[0][0] * c00 + Sm[0][1] * c01 + Sm[0][2] * c02;
        const double tr = Sm[0][0] + Sm[1][1] + Sm[2][2];
        if (!(det > 1e-12 * tr * tr * tr)) {
          bad |= DEV_ERR_STENCIL;
        } else {
          double Si[3][3];
          Si[0][0] = c00 / det;
          Si[1][0] = c01 / det;
          Si[2][0] = c02 / det;
          Si[0][1] = (Sm[0][2] * Sm[2][1] - Sm[0][1] * Sm[2][2]) / det;
          Si[1][1] = (Sm[0][0] * Sm[2][2] - Sm[0][2] * Sm[2][0]) / det;
          Si[2][1] = (Sm[0][1] * Sm[2][0] - Sm[0][0] * Sm[2][1]) / det;
          Si[0][2] = (Sm[0][1] * Sm[1][2] - Sm[0][2] * Sm[1][1]) / det;
          Si[1][2] = (Sm[0][2] * Sm[1][0] - Sm[0][0] * Sm[1][2]) / det;
          Si[2][2] = (Sm[0][0] * Sm[1][1] - Sm[0][1] * Sm[1][0]) / det;
          // w = Y S^-1; scatter each source's load into the node slots
          for (int k = 0; k < K; ++k)
            for (int j = 0; j < 3; ++j) {
              const double w = Y[k][0] * Si[0][j] + Y[k][1] * Si[1][j] + Y[k][2] * Si[2][j];
              wn[src_b[k]][j] += src_s[k] * w;
              wn[src_a[k]][j] -= src_s[k] * w;
            }
        }
      } else if (!bad) {
        bad |= DEV_ERR_STENCIL;
      }
      if (bad)
        for (int i = 0; i < NW; ++i) wn[i][0] = wn[i][1] = wn[i][2] = 0.0;
    }
    if (bad) atomicOr(err, bad);
    for (int j = 0; j < 3; ++j) {
      const int64_t col = 3 * p + j;
      for (int i = 0; i < NW; ++i) {
        Fn[col * NW + i] = node[i];
        Fw[col * NW + i] = wn[i][j];
      }
    }
  }
}

}  // namespace
}  // namespace zi

using namespace zi;

extern "C" int zi_source_stencil(zi_system* S, const double* pos, const int32_t* dip_tet, int64_t P, int model,
                                 double lambda, int32_t* F_nodes, double* F_w, cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative source count");
  if (model != ZI_SOURCE_WHITNEY4 && model != ZI_SOURCE_PBO10)
    return set_error(ZI_ERR_ARG, "unknown source model %d", model);
  if (lambda == 0.0) lambda = ZI_PBO_LAMBDA_DEFAULT;
  if (!(lambda > 0.0) || !isfinite(lambda)) return set_error(ZI_ERR_ARG, "lambda must be positive and finite");
  if (P > 0 && (!pos || !dip_tet || !F_nodes || !F_w)) return set_error(ZI_ERR_ARG, "null input or output array");
  if (P == 0) return ZI_OK;
  const int64_t n = S->n, m = S->m;
  DevTmp<int32_t> cnt, start, inc;
  DevTmp<int> err;
  ZI_CHECK(cnt.alloc(n, s));
  ZI_CHECK(start.alloc(n + 1, s));
  ZI_CHECK(inc.alloc(4 * m, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_inc_count<<<grid_for(4 * m, 256), 256, 0, s>>>(m, S->tets, n, cnt.p, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(exclusive_scan_i32(cnt.p, start.p, n, nullptr, s));
  ZI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n, s));
  k_inc_fill<<<grid_for(4 * m, 256), 256, 0, s>>>(m, S->tets, n, start.p, cnt.p, inc.p);
  ZI_LAUNCH_CHECK();
  k_stencil<<<grid_for(P, 128), 128, 0, s>>>(P, pos, dip_tet, m, S->tets, n, S->nodes, start.p, inc.p, model,
                                             lambda, F_nodes, F_w, err.p);
  ZI_LAUNCH_CHECK();
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}
