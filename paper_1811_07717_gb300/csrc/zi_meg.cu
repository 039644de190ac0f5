// MEG lead field by the Biot-Savart formula (App. A.2, by analogy with the
// EEG lead field).
//
// The field of the total current J^p - sigma grad u at sensor s (position
// r_s, unit orientation n_s) is the primary dipole's field plus the volume
// current's, Bm^T u with
//   Bm[i][s] = -mu0/(4 pi) sum_{e containing i} grad psi_i|_e . sigma_e (G_e(r_s) x n_s),
//   G_e(r)   = int_e (r - r') / |r - r'|^3 dV'   (4-point degree-2 rule),
// so the volume part of the lead field is (A^-1 Bm)^T F: one PCG solve per
// sensor (the EEG transfer solver on a view of the system with Bm as its
// right-hand sides), then the sparse source application.
//
// Bm is built in sensor chunks: k_meg_tet evaluates, per (tet, sensor),
// c_a = grad psi_a . sigma_e (G_e x n_s) for the tet's four vertices into a
// scratch array; k_meg_gather sums, per node, over the tets that contain it in
// ascending tet order (the diagonal entries of the assembly's sorted entry
// map), so Bm is bitwise reproducible.
#include <math.h>
#include <stdlib.h>

#include "zi_internal.cuh"
#include "zi_pcg.cuh"

namespace zi {
namespace {

constexpr double MU0_4PI = 1e-7;  // mu0 / (4 pi), T m / A
// the rule's barycentric weights: (5 + 3 sqrt 5) / 20 on one vertex, (5 - sqrt 5) / 20 on the others
constexpr double QUAD_A = 0.58541019662496845446;
constexpr double QUAD_B = 0.13819660112501051518;

// Gradients of the barycentric coordinates (g[a] = grad psi_a) and |det| of tet X.
__device__ __forceinline__ double tet_grads(const double x[4][3], double g[4][3]) {
  double e[3][3];
  for (int d = 0; d < 3; ++d) {
    e[0][d] = x[1][d] - x[0][d];
    e[1][d] = x[2][d] - x[0][d];
    e[2][d] = x[3][d] - x[0][d];
  }
  g[1][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
  g[1][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
  g[1][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
  g[2][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
  g[2][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
  g[2][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
  g[3][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
  g[3][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
  g[3][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  const double det = e[0][0] * g[1][0] + e[0][1] * g[1][1] + e[0][2] * g[1][2];
  const double inv = 1.0 / det;
  for (int a = 1; a < 4; ++a)
    for (int d = 0; d < 3; ++d) g[a][d] *= inv;
  for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  return fabs(det);
}

// W[(t*4 + a)*Sc + j] = grad psi_a|_t . sigma_t (G_t(r_s) x n_s) for sensor s = s0 + j.
__global__ void __launch_bounds__(256) k_meg_tet(int64_t m, const int32_t* __restrict__ tets,
                                                 const double* __restrict__ X, const double* __restrict__ sigma6,
                                                 int s0, int Sc, const double* __restrict__ spos,
                                                 const double* __restrict__ sdir, double* __restrict__ W,
                                                 int* __restrict__ err) {
  const int64_t total = m * (int64_t)Sc;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = q / Sc;
    const int j = (int)(q - t * Sc);
    const int s = s0 + j;
    const int4 v = reinterpret_cast<const int4*>(tets)[t];
    const int32_t vv[4] = {v.x, v.y, v.z, v.w};
    double x[4][3], g[4][3];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) x[a][d] = X[3 * (int64_t)vv[a] + d];
    const double vol = tet_grads(x, g) / 6.0;
    double xs[3], r[3], ns[3];
    for (int d = 0; d < 3; ++d) {
      xs[d] = x[0][d] + x[1][d] + x[2][d] + x[3][d];
      r[d] = spos[3 * s + d];
      ns[d] = sdir[3 * s + d];
    }
    double G[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
      double dv[3];
      for (int d = 0; d < 3; ++d) dv[d] = r[d] - (QUAD_B * xs[d] + (QUAD_A - QUAD_B) * x[k][d]);
      const double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
      const double w = 1.0 / (d2 * sqrt(d2));
      for (int d = 0; d < 3; ++d) G[d] += dv[d] * w;
    }
    for (int d = 0; d < 3; ++d) G[d] *= 0.25 * vol;
    const double c[3] = {G[1] * ns[2] - G[2] * ns[1], G[2] * ns[0] - G[0] * ns[2], G[0] * ns[1] - G[1] * ns[0]};
    const double* sg = sigma6 + 6 * t;  // (s11, s22, s33, s12, s13, s23)
    const double V[3] = {sg[0] * c[0] + sg[3] * c[1] + sg[4] * c[2], sg[3] * c[0] + sg[1] * c[1] + sg[5] * c[2],
                         sg[4] * c[0] + sg[5] * c[1] + sg[2] * c[2]};
    bool bad = false;
    for (int a = 0; a < 4; ++a) {
      const double ca = g[a][0] * V[0] + g[a][1] * V[1] + g[a][2] * V[2];
      bad |= !isfinite(ca);
      W[(t * 4 + a) * Sc + j] = ca;
    }
    if (bad) atomicOr(err, DEV_ERR_NONFINITE);
  }
}

// Bm[i][s0 + j] = -mu0/(4 pi) * sum over the tets holding i (ascending) of W[(t*4 + a)*Sc + j].
__global__ void k_meg_gather(int64_t n, int64_t m, const int32_t* __restrict__ diagpos,
                             const int32_t* __restrict__ seg, const int32_t* __restrict__ perm, int s0, int Sc,
                             const double* __restrict__ W, int Ns, int64_t ground, double* __restrict__ Bm) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t vol_ids = 16 * m;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const int k = diagpos[i];
    const int q0 = seg[k], q1 = seg[k + 1];
    for (int j = lane; j < Sc; j += 32) {
      double acc = 0.0;
      for (int q = q0; q < q1; ++q) {
        const int64_t id = (uint32_t)perm[q];
        if (id >= vol_ids) continue;  // electrode surface terms
        const int64_t t = id >> 4;
        const int a = (int)((id >> 2) & 3);
        acc += W[(t * 4 + a) * Sc + j];
      }
      Bm[i * Ns + s0 + j] = (i == ground) ? 0.0 : -MU0_4PI * acc;
    }
  }
}

// L[s][c] = primary field of unit dipole e_d at pos[p] (c = 3p + d) + Ht[c][s].
__global__ void k_meg_out(int Ns, int64_t ncols, const double* __restrict__ spos, const double* __restrict__ sdir,
                          const double* __restrict__ pos, const double* __restrict__ Ht, double* __restrict__ L) {
  __shared__ double tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int s0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y;
    const int s = s0 + threadIdx.x;
    tile[y][threadIdx.x] = (c < ncols && s < Ns) ? Ht[c * Ns + s] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int s = s0 + y;
    const int64_t c = c0 + threadIdx.x;
    if (s >= Ns || c >= ncols) continue;
    const int64_t p = c / 3;
    const int d = (int)(c - 3 * p);
    double a[3], n3[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = spos[3 * s + k] - pos[3 * p + k];
      n3[k] = sdir[3 * s + k];
    }
    // e_d . (a x n)
    const double cr = (d == 0) ? a[1] * n3[2] - a[2] * n3[1] : (d == 1) ? a[2] * n3[0] - a[0] * n3[2]
                                                                        : a[0] * n3[1] - a[1] * n3[0];
    const double r2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    L[(int64_t)s * ncols + c] = MU0_4PI * cr / (r2 * sqrt(r2)) + tile[threadIdx.x][y];
  }
}

// Partial-integration columns: F[v_a][3p + d] = d psi_a / d x_d on tet dip_tet[p].
__global__ void k_source_pi(int64_t P, const int32_t* __restrict__ dip_tet, int64_t m,
                            const int32_t* __restrict__ tets, const double* __restrict__ X,
                            int32_t* __restrict__ Fn, double* __restrict__ Fw, int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = dip_tet[p];
    int32_t vv[4] = {0, 0, 0, 0};
    double g[4][3] = {};
    if (t < 0 || t >= m) {
      atomicOr(err, DEV_ERR_OUTSIDE);
    } else {
      const int4 v = reinterpret_cast<const int4*>(tets)[t];
      vv[0] = v.x;
      vv[1] = v.y;
      vv[2] = v.z;
      vv[3] = v.w;
      double x[4][3];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) x[a][d] = X[3 * (int64_t)vv[a] + d];
      tet_grads(x, g);
    }
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 4; ++a) {
        Fn[(3 * p + d) * 4 + a] = vv[a];
        Fw[(3 * p + d) * 4 + a] = g[a][d];
      }
  }
}

int meg_rhs_impl(zi_system* S, const double* sigma6, const double* spos, const double* sdir, int Ns, double* Bm,
                 cudaStream_t s) {
  const int64_t m = S->m, n = S->n;
  // sensors per chunk: the per-(tet, vertex, sensor) scratch stays within 2 GiB
  int64_t sc = ((int64_t)1 << 31) / (32 * m);
  // ZI_MEG_SENSORS_PER_CHUNK lowers the chunk (tests use it to run the chunk
  // loop on small meshes; the result does not depend on the chunk size)
  if (const char* env = getenv("ZI_MEG_SENSORS_PER_CHUNK")) {
    const long v = strtol(env, nullptr, 10);
    if (v > 0 && v < sc) sc = v;
  }
  if (sc < 1) sc = 1;
  if (sc > Ns) sc = Ns;
  const int Sc = (int)sc;
  DevTmp<double> W;
  DevTmp<int> err;
  ZI_CHECK(W.alloc((size_t)m * 4 * Sc, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  for (int s0 = 0; s0 < Ns; s0 += Sc) {
    const int len = (Ns - s0 < Sc) ? Ns - s0 : Sc;
    k_meg_tet<<<grid_for(m * len, 256, 152u * 64u), 256, 0, s>>>(m, S->tets, S->nodes, sigma6, s0, len, spos, sdir,
                                                                  W.p, err.p);
    ZI_LAUNCH_CHECK();
    k_meg_gather<<<grid_for(n * 32, 256, 152u * 64u), 256, 0, s>>>(n, m, S->diagpos, S->seg, S->perm, s0, len, W.p,
                                                                    Ns, S->ground, Bm);
    ZI_LAUNCH_CHECK();
  }
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}

int check_sensors(zi_system* S, const double* sigma6, const double* spos, const double* sdir, int Ns) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (Ns < 1) return set_error(ZI_ERR_ARG, "sensor count must be positive");
  if (!sigma6 || !spos || !sdir) return set_error(ZI_ERR_ARG, "null conductivity or sensor array");
  if (16 * S->m > (int64_t)UINT32_MAX) return set_error(ZI_ERR_ARG, "too many elements for the entry map");
  return ZI_OK;
}

}  // namespace
}  // namespace zi

using namespace zi;

extern "C" int zi_meg_rhs(zi_system* S, const double* sigma6, const double* sens_pos, const double* sens_dir, int Ns,
                          double* Bm, cudaStream_t s) {
  ZI_CHECK(check_sensors(S, sigma6, sens_pos, sens_dir, Ns));
  if (!Bm) return set_error(ZI_ERR_ARG, "null output array");
  return meg_rhs_impl(S, sigma6, sens_pos, sens_dir, Ns, Bm, s);
}

extern "C" int zi_meg_transfer(zi_system* S, const double* sigma6, const double* sens_pos, const double* sens_dir,
                               int Ns, const zi_solver_opts* o, double* T_meg, int32_t* iters, double* relres,
                               cudaStream_t s) {
  ZI_CHECK(check_sensors(S, sigma6, sens_pos, sens_dir, Ns));
  if (!T_meg) return set_error(ZI_ERR_ARG, "null output array");
  ZI_CHECK(check_opts(o));
  DevTmp<double> Bm;
  ZI_CHECK(Bm.alloc((size_t)S->n * Ns, s));
  ZI_CHECK(meg_rhs_impl(S, sigma6, sens_pos, sens_dir, Ns, Bm.p, s));
  // a view of the system with the sensors' right-hand sides; the matrix and
  // pattern are shared, the solver scratch and solution are the view's own
  zi_system view = *S;
  view.B = Bm.p;
  view.n_rhs = Ns;
  view.T = nullptr;
  view.has_T = 0;
  view.solver = nullptr;
  int st = transfer_impl(&view, o, T_meg, iters, relres, s);
  // the view's internal stream may still run after an early error return
  cudaDeviceSynchronize();
  solver_scratch_free(&view);
  if (view.T) dfree(view.T, s);
  return st;
}

extern "C" int zi_meg_leadfield(zi_system* S, const double* T_meg, const double* sens_pos, const double* sens_dir,
                                int Ns, const double* pos, int64_t P, const int32_t* F_nodes, const double* F_w, int K,
                                double* L, cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (Ns < 1 || P < 0) return set_error(ZI_ERR_ARG, "bad sensor or source count");
  if (K < 1 || K > 32) return set_error(ZI_ERR_ARG, "entries per column must be in 1..32 (got %d)", K);
  if (P == 0) return ZI_OK;
  if (!T_meg || !sens_pos || !sens_dir || !pos || !F_nodes || !F_w || !L)
    return set_error(ZI_ERR_ARG, "null input or output array");
  const int64_t ncols = 3 * P;
  DevTmp<double> Ht;
  DevTmp<int> err;
  ZI_CHECK(Ht.alloc((size_t)ncols * Ns, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  ZI_CHECK(source_apply_ell(ncols, K, F_nodes, F_w, S->n, T_meg, Ns, Ht.p, err.p, s));
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  dim3 grid((unsigned)((ncols + 31) / 32), (unsigned)((Ns + 31) / 32));
  k_meg_out<<<grid, dim3(32, 8), 0, s>>>(Ns, ncols, sens_pos, sens_dir, pos, Ht.p, L);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}

extern "C" int zi_source_pi(zi_system* S, const int32_t* dip_tet, int64_t P, int32_t* F_nodes, double* F_w,
                            cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative source count");
  if (P == 0) return ZI_OK;
  if (!dip_tet || !F_nodes || !F_w) return set_error(ZI_ERR_ARG, "null input or output array");
  DevTmp<int> err;
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_source_pi<<<grid_for(P, 128), 128, 0, s>>>(P, dip_tet, S->m, S->tets, S->nodes, F_nodes, F_w, err.p);
  ZI_LAUNCH_CHECK();
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}
