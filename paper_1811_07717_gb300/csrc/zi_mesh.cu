// Regular-grid Kuhn mesher (stand-in for the paper's uniform tetrahedral mesh
// tool, Sec. 2.5) and grid point location of dipoles.
//
// Every integer output is decided by integer arithmetic or by FP64 comparisons
// formed in a fixed order (2R/h squared against an exact integer), so the
// outputs are reproducible bit for bit.
#include <math.h>

#include <vector>

#include "zi_internal.cuh"

namespace zi {
namespace {

// Axis permutations in lexicographic order; odd ones get their last two path
// vertices swapped to keep every tet positively oriented.
__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int c_odd[6] = {0, 1, 1, 0, 0, 1};
// Outward faces of a positively oriented tet, face f opposite vertex f.
__constant__ int c_face[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

constexpr int MAX_SHELLS = 8;
struct Shells {
  double thr[MAX_SHELLS];  // (2 R_s / h)^2
  int n;
};

struct Grid {
  int N;       // indices in [-N, N]
  int G;       // nodes per axis 2N+1
  int Gc;      // cubes per axis 2N
};

__global__ void k_cube_flags(Grid g, Shells sh, int32_t* __restrict__ keep, int8_t* __restrict__ label) {
  int64_t total = (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    int I = (int)(c / ((int64_t)g.Gc * g.Gc));
    int J = (int)((c / g.Gc) % g.Gc);
    int K = (int)(c % g.Gc);
    int64_t oi = 2 * (I - g.N) + 1, oj = 2 * (J - g.N) + 1, ok = 2 * (K - g.N) + 1;
    double sq = (double)(oi * oi + oj * oj + ok * ok);
    int kept = sq < sh.thr[sh.n - 1];
    int lab = 0;
    for (int s = 0; s < sh.n - 1; ++s) lab += (sq >= sh.thr[s]) ? 1 : 0;
    keep[c] = kept;
    if (label) label[c] = (int8_t)lab;
  }
}

__device__ __forceinline__ int cube_kept(const int32_t* keep, const Grid& g, int I, int J, int K) {
  if (I < 0 || J < 0 || K < 0 || I >= g.Gc || J >= g.Gc || K >= g.Gc) return 0;
  return keep[((int64_t)I * g.Gc + J) * g.Gc + K];
}

__global__ void k_node_flags(Grid g, const int32_t* __restrict__ keep, int32_t* __restrict__ nflag) {
  int64_t total = (int64_t)g.G * g.G * g.G;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total;
       v += (int64_t)gridDim.x * blockDim.x) {
    int I = (int)(v / ((int64_t)g.G * g.G));
    int J = (int)((v / g.G) % g.G);
    int K = (int)(v % g.G);
    int f = 0;
    for (int d = 0; d < 8 && !f; ++d)
      f = cube_kept(keep, g, I - (d >> 2 & 1), J - (d >> 1 & 1), K - (d & 1));
    nflag[v] = f;
  }
}

__global__ void k_nodes_out(Grid g, double h, const int32_t* __restrict__ nflag,
                            const int32_t* __restrict__ nid, double* __restrict__ nodes) {
  int64_t total = (int64_t)g.G * g.G * g.G;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!nflag[v]) continue;
    int I = (int)(v / ((int64_t)g.G * g.G));
    int J = (int)((v / g.G) % g.G);
    int K = (int)(v % g.G);
    int64_t id = nid[v];
    nodes[3 * id + 0] = __dmul_rn((double)(I - g.N), h);
    nodes[3 * id + 1] = __dmul_rn((double)(J - g.N), h);
    nodes[3 * id + 2] = __dmul_rn((double)(K - g.N), h);
  }
}

// Tet vertices (local order) of Kuhn tet k of cube (I,J,K) as node ids.
__device__ __forceinline__ void kuhn_tet(const Grid& g, const int32_t* nid, int I, int J, int K, int k,
                                         int32_t v[4]) {
  int p[3] = {I, J, K};
  int a = c_perm[k][0], b = c_perm[k][1];
  int path[4][3];
  path[0][0] = p[0]; path[0][1] = p[1]; path[0][2] = p[2];
  p[a] += 1;
  path[1][0] = p[0]; path[1][1] = p[1]; path[1][2] = p[2];
  p[b] += 1;
  path[2][0] = p[0]; path[2][1] = p[1]; path[2][2] = p[2];
  path[3][0] = I + 1; path[3][1] = J + 1; path[3][2] = K + 1;
  for (int s = 0; s < 4; ++s)
    v[s] = nid[((int64_t)path[s][0] * g.G + path[s][1]) * g.G + path[s][2]];
  if (c_odd[k]) {
    int32_t t = v[2]; v[2] = v[3]; v[3] = t;
  }
}

// Boundary faces of tet k of a kept cube: local face 0 lies on the cube's +a
// face, and the face opposite the far corner v0+(1,1,1) (local 3, or 2 after
// the swap) on its -c face; either is a boundary face iff the neighbouring
// cube across it is not kept.  The other two faces are inside the cube.
__device__ __forceinline__ int bface_mask(const Grid& g, const int32_t* keep, int I, int J, int K, int k) {
  int a = c_perm[k][0], c = c_perm[k][2];
  int q[3] = {I, J, K};
  q[a] += 1;
  int m = 0;
  if (!cube_kept(keep, g, q[0], q[1], q[2])) m |= 1;  // local face 0
  int r[3] = {I, J, K};
  r[c] -= 1;
  if (!cube_kept(keep, g, r[0], r[1], r[2])) m |= c_odd[k] ? 4 : 8;  // local face 2 or 3
  return m;
}

__global__ void k_tets_out(Grid g, const int32_t* __restrict__ keep, const int32_t* __restrict__ crank,
                           const int8_t* __restrict__ clabel, const int32_t* __restrict__ nid,
                           int32_t* __restrict__ tets, int32_t* __restrict__ labels,
                           int32_t* __restrict__ bcount) {
  int64_t total = (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[c]) continue;
    int I = (int)(c / ((int64_t)g.Gc * g.Gc));
    int J = (int)((c / g.Gc) % g.Gc);
    int K = (int)(c % g.Gc);
    int64_t r = crank[c];
    for (int k = 0; k < 6; ++k) {
      int64_t t = 6 * r + k;
      if (tets) {
        int32_t v[4];
        kuhn_tet(g, nid, I, J, K, k, v);
        tets[4 * t + 0] = v[0]; tets[4 * t + 1] = v[1];
        tets[4 * t + 2] = v[2]; tets[4 * t + 3] = v[3];
      }
      if (labels) labels[t] = clabel[c];
      if (bcount) bcount[t] = __popc(bface_mask(g, keep, I, J, K, k));
    }
  }
}

__global__ void k_bfaces_out(Grid g, const int32_t* __restrict__ keep, const int32_t* __restrict__ crank,
                             const int32_t* __restrict__ nid, const int32_t* __restrict__ boff,
                             int32_t* __restrict__ bfaces) {
  int64_t total = (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[c]) continue;
    int I = (int)(c / ((int64_t)g.Gc * g.Gc));
    int J = (int)((c / g.Gc) % g.Gc);
    int K = (int)(c % g.Gc);
    int64_t r = crank[c];
    for (int k = 0; k < 6; ++k) {
      int msk = bface_mask(g, keep, I, J, K, k);
      if (!msk) continue;
      int64_t t = 6 * r + k;
      int32_t v[4];
      kuhn_tet(g, nid, I, J, K, k, v);
      int64_t o = boff[t];
      for (int f = 0; f < 4; ++f) {
        if (!(msk >> f & 1)) continue;
        bfaces[3 * o + 0] = v[c_face[f][0]];
        bfaces[3 * o + 1] = v[c_face[f][1]];
        bfaces[3 * o + 2] = v[c_face[f][2]];
        ++o;
      }
    }
  }
}

int make_grid(double h, int n_shells, const double* radii, Grid* g, Shells* sh) {
  if (!(h > 0) || !isfinite(h)) return set_error(ZI_ERR_ARG, "grid step h must be positive and finite");
  if (n_shells < 1 || n_shells > MAX_SHELLS || !radii)
    return set_error(ZI_ERR_ARG, "need 1..%d shell radii", MAX_SHELLS);
  for (int s = 0; s < n_shells; ++s) {
    if (!(radii[s] > 0) || !isfinite(radii[s])) return set_error(ZI_ERR_ARG, "radii must be positive");
    if (s && !(radii[s] > radii[s - 1])) return set_error(ZI_ERR_ARG, "radii must ascend");
    volatile double t = 2.0 * radii[s] / h;  // formed in this order, then squared
    double tt = t;
    sh->thr[s] = tt * tt;
  }
  sh->n = n_shells;
  double q = ceil(radii[n_shells - 1] / h);
  if (q > 1200) return set_error(ZI_ERR_ARG, "grid too large (R/h = %g)", q);
  g->N = (int)q + 1;
  g->G = 2 * g->N + 1;
  g->Gc = 2 * g->N;
  return ZI_OK;
}

}  // namespace

int grid_cube_ranks(double h, int n_shells, const double* radii, int32_t** keep_out, int32_t** rank_out,
                    int* N_out, int64_t* n_kept, cudaStream_t s) {
  Grid g;
  Shells sh;
  ZI_CHECK(make_grid(h, n_shells, radii, &g, &sh));
  int64_t nc = (int64_t)g.Gc * g.Gc * g.Gc;
  int32_t *keep = nullptr, *rank = nullptr;
  ZI_CHECK(dalloc_n(&keep, nc, s));
  int st = dalloc_n(&rank, nc + 1, s);
  if (st) { dfree(keep, s); return st; }
  k_cube_flags<<<grid_for(nc, 256), 256, 0, s>>>(g, sh, keep, nullptr);
  st = exclusive_scan_i32(keep, rank, nc, n_kept, s);
  if (st) { dfree(keep, s); dfree(rank, s); return st; }
  *keep_out = keep;
  *rank_out = rank;
  *N_out = g.N;
  return ZI_OK;
}

}  // namespace zi

using namespace zi;

extern "C" int zi_mesh_from_grid(double h, int n_shells, const double* radii, int64_t* n_nodes,
                                 int64_t* n_tets, int64_t* n_bfaces, double* nodes, int32_t* tets,
                                 int32_t* labels, int32_t* bfaces, cudaStream_t s) {
  if (!n_nodes || !n_tets || !n_bfaces) return set_error(ZI_ERR_ARG, "size outputs must be non-null");
  int outs = (nodes != nullptr) + (tets != nullptr) + (labels != nullptr) + (bfaces != nullptr);
  if (outs != 0 && outs != 4) return set_error(ZI_ERR_ARG, "pass all four mesh outputs or none");
  Grid g;
  Shells sh;
  ZI_CHECK(make_grid(h, n_shells, radii, &g, &sh));
  int64_t nc = (int64_t)g.Gc * g.Gc * g.Gc;
  int64_t nv = (int64_t)g.G * g.G * g.G;
  DevTmp<int32_t> keep, crank, nflag, nid, bcnt, boff;
  DevTmp<int8_t> clabel;
  ZI_CHECK(keep.alloc(nc, s));
  ZI_CHECK(crank.alloc(nc + 1, s));
  ZI_CHECK(clabel.alloc(nc, s));
  ZI_CHECK(nflag.alloc(nv, s));
  ZI_CHECK(nid.alloc(nv + 1, s));
  k_cube_flags<<<grid_for(nc, 256), 256, 0, s>>>(g, sh, keep.p, clabel.p);
  ZI_LAUNCH_CHECK();
  int64_t n_cubes = 0, n = 0;
  ZI_CHECK(exclusive_scan_i32(keep.p, crank.p, nc, &n_cubes, s));
  k_node_flags<<<grid_for(nv, 256), 256, 0, s>>>(g, keep.p, nflag.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(exclusive_scan_i32(nflag.p, nid.p, nv, &n, s));
  int64_t m = 6 * n_cubes;
  if (m > INT32_MAX / 4) return set_error(ZI_ERR_ARG, "mesh too large for int32 indices");
  ZI_CHECK(bcnt.alloc(m, s));
  ZI_CHECK(boff.alloc(m + 1, s));
  k_tets_out<<<grid_for(nc, 256), 256, 0, s>>>(g, keep.p, crank.p, clabel.p, nid.p, tets, labels, bcnt.p);
  ZI_LAUNCH_CHECK();
  int64_t nb = 0;
  ZI_CHECK(exclusive_scan_i32(bcnt.p, boff.p, m, &nb, s));
  if (outs) {
    k_nodes_out<<<grid_for(nv, 256), 256, 0, s>>>(g, h, nflag.p, nid.p, nodes);
    ZI_LAUNCH_CHECK();
    k_bfaces_out<<<grid_for(nc, 256), 256, 0, s>>>(g, keep.p, crank.p, nid.p, boff.p, bfaces);
    ZI_LAUNCH_CHECK();
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  *n_nodes = n;
  *n_tets = m;
  *n_bfaces = nb;
  return ZI_OK;
}

namespace zi {
namespace {
__global__ void k_locate(int64_t P, const double* __restrict__ pos, double h, Grid g,
                         const int32_t* __restrict__ keep, const int32_t* __restrict__ crank,
                         int32_t* __restrict__ out, int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    double f[3];
    int ci[3];
    bool bad = false;
    for (int d = 0; d < 3; ++d) {
      double x = pos[3 * p + d];
      if (!isfinite(x)) { bad = true; break; }
      double sd = __ddiv_rn(x, h);
      double cell = floor(sd);
      f[d] = __dsub_rn(sd, cell);
      double c = cell + (double)g.N;
      if (c < 0 || c >= (double)g.Gc) { bad = true; break; }
      ci[d] = (int)c;
    }
    int64_t lin = bad ? 0 : ((int64_t)ci[0] * g.Gc + ci[1]) * g.Gc + ci[2];
    if (bad || !keep[lin]) {
      atomicOr(err, DEV_ERR_OUTSIDE);
      out[p] = -1;
      continue;
    }
    int kk = 5;
    for (int k = 0; k < 6; ++k) {
      int a = c_perm[k][0], b = c_perm[k][1], c = c_perm[k][2];
      if (f[a] >= f[b] && f[b] >= f[c]) { kk = k; break; }
    }
    out[p] = (int32_t)(6 * (int64_t)crank[lin] + kk);
  }
}
}  // namespace
}  // namespace zi

extern "C" int zi_locate_dipoles_grid(double h, int n_shells, const double* radii, const double* pos,
                                      int64_t P, int32_t* dip_tet, cudaStream_t s) {
  if (P < 0) return set_error(ZI_ERR_ARG, "negative point count");
  if (P > 0 && (!pos || !dip_tet)) return set_error(ZI_ERR_ARG, "null point or output array");
  Grid g;
  Shells sh;
  ZI_CHECK(make_grid(h, n_shells, radii, &g, &sh));
  if (P == 0) return ZI_OK;
  int64_t nc = (int64_t)g.Gc * g.Gc * g.Gc;
  DevTmp<int32_t> keep, crank;
  DevTmp<int> err;
  ZI_CHECK(keep.alloc(nc, s));
  ZI_CHECK(crank.alloc(nc + 1, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_cube_flags<<<grid_for(nc, 256), 256, 0, s>>>(g, sh, keep.p, nullptr);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(exclusive_scan_i32(keep.p, crank.p, nc, nullptr, s));
  k_locate<<<grid_for(P, 256), 256, 0, s>>>(P, pos, h, g, keep.p, crank.p, dip_tet, err.p);
  ZI_LAUNCH_CHECK();
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}
