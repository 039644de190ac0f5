// Regular-grid Kuhn mesher (stand-in for the paper's uniform tetrahedral mesh
// tool, Sec. 2.5) and grid point location of dipoles.
//
// Every integer output is decided by integer arithmetic or by FP64 comparisons
// formed in a fixed order (2R/h squared against an exact integer), so the
// outputs are reproducible bit for bit.
#include <math.h>
#include <string.h>

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
  // the output call writes into arrays sized by the counting call's counts
  if (outs && (*n_nodes != n || *n_tets != m))
    return set_error(ZI_ERR_ARG, "pass the counts of the counting call in n_nodes and n_tets");
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

// ---------------------------------------------------------------------------
// Mesher from a surface segmentation (Sec. 2.5, mesh tool): the same Kuhn
// grid, labelled from closed compartment surfaces.
//   node label: the first surface (innermost first) whose winding number at
//     the node is >= 1/2 (solid angles by Van Oosterom-Strackee), else outside;
//   tet label: the best-ranked label among its four nodes (rank = order by
//     (priority, index); outside ranks last); a tet with no inside node is
//     dropped;
//   kept nodes in grid order, kept tets in (cube, permutation) order,
//   boundary faces in (tet, local face) order, found by the Kuhn neighbour
//   across each face: across the face opposite path vertex 0 the tet
//   (b, c, a) of cube +e_a, opposite path vertex 3 the tet (c, a, b) of cube
//   -e_c, opposite path vertices 1 and 2 the tets (b, a, c) and (a, c, b) of
//   the same cube.
// ---------------------------------------------------------------------------

namespace zi {
namespace {

constexpr int SEG_MAX_SURF = 64;
struct SegParams {
  int C;                              // compartments
  int rank[SEG_MAX_SURF];             // rank of compartment c
  int order[SEG_MAX_SURF];            // compartment of rank r
  int64_t toff[SEG_MAX_SURF + 1];     // triangle range of surface c
};

__global__ void k_seg_maxabs(int64_t nv, const double* __restrict__ verts, unsigned long long* __restrict__ out,
                             int* __restrict__ err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * nv; q += (int64_t)gridDim.x * blockDim.x) {
    const double x = verts[q];
    if (!isfinite(x)) {
      atomicOr(err, DEV_ERR_NONFINITE);
      continue;
    }
    // for non-negative doubles the bit patterns order like the values
    atomicMax(out, (unsigned long long)__double_as_longlong(fabs(x)));
  }
}

__global__ void k_seg_labels(Grid g, double h, SegParams sp, int64_t nv, const double* __restrict__ verts,
                             const int32_t* __restrict__ tris, int32_t* __restrict__ lab, int* __restrict__ err) {
  const int64_t total = (int64_t)g.G * g.G * g.G;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(v / ((int64_t)g.G * g.G));
    const int J = (int)((v / g.G) % g.G);
    const int K = (int)(v % g.G);
    const double p[3] = {__dmul_rn((double)(I - g.N), h), __dmul_rn((double)(J - g.N), h),
                         __dmul_rn((double)(K - g.N), h)};
    int label = -1;
    for (int c = 0; c < sp.C && label < 0; ++c) {
      double acc = 0.0;
      for (int64_t t = sp.toff[c]; t < sp.toff[c + 1]; ++t) {
        double A[3], B[3], Cv[3];
        bool ok = true;
        for (int j = 0; j < 3; ++j) {
          const int32_t iv = tris[3 * t + j];
          if (iv < 0 || iv >= nv) {
            ok = false;
            break;
          }
          double* dst = j == 0 ? A : (j == 1 ? B : Cv);
          for (int d = 0; d < 3; ++d) dst[d] = verts[3 * (int64_t)iv + d] - p[d];
        }
        if (!ok) {
          atomicOr(err, DEV_ERR_BAD_INDEX);
          continue;
        }
        const double a = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
        const double b = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        const double cc = sqrt(Cv[0] * Cv[0] + Cv[1] * Cv[1] + Cv[2] * Cv[2]);
        const double num = A[0] * (B[1] * Cv[2] - B[2] * Cv[1]) + A[1] * (B[2] * Cv[0] - B[0] * Cv[2]) +
                           A[2] * (B[0] * Cv[1] - B[1] * Cv[0]);
        const double den = a * b * cc + (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) * cc +
                           (B[0] * Cv[0] + B[1] * Cv[1] + B[2] * Cv[2]) * a +
                           (Cv[0] * A[0] + Cv[1] * A[1] + Cv[2] * A[2]) * b;
        acc += 2.0 * atan2(num, den);
      }
      if (acc / (4.0 * 3.14159265358979323846) >= 0.5) label = c;
    }
    lab[v] = label;
  }
}

// Grid coordinates of the four path vertices of Kuhn tet k of cube (I, J, K).
__device__ __forceinline__ void kuhn_path(int I, int J, int K, int k, int path[4][3]) {
  int p[3] = {I, J, K};
  const int a = c_perm[k][0], b = c_perm[k][1];
  for (int d = 0; d < 3; ++d) path[0][d] = p[d];
  p[a] += 1;
  for (int d = 0; d < 3; ++d) path[1][d] = p[d];
  p[b] += 1;
  for (int d = 0; d < 3; ++d) path[2][d] = p[d];
  path[3][0] = I + 1;
  path[3][1] = J + 1;
  path[3][2] = K + 1;
}

__device__ __forceinline__ int perm_index(int a, int b, int c) {
  for (int k = 0; k < 6; ++k)
    if (c_perm[k][0] == a && c_perm[k][1] == b && c_perm[k][2] == c) return k;
  return 0;
}

__global__ void k_seg_tets(Grid g, SegParams sp, const int32_t* __restrict__ lab, int32_t* __restrict__ keep,
                           int32_t* __restrict__ tlab) {
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    const int I = (int)(q / ((int64_t)g.Gc * g.Gc));
    const int J = (int)((q / g.Gc) % g.Gc);
    const int K = (int)(q % g.Gc);
    int path[4][3];
    kuhn_path(I, J, K, k, path);
    int best = sp.C;
    for (int s = 0; s < 4; ++s) {
      const int l = lab[((int64_t)path[s][0] * g.G + path[s][1]) * g.G + path[s][2]];
      const int r = l < 0 ? sp.C : sp.rank[l];
      best = r < best ? r : best;
    }
    keep[t] = best < sp.C;
    tlab[t] = best < sp.C ? sp.order[best] : -1;
  }
}

__global__ void k_seg_used(Grid g, const int32_t* __restrict__ keep, int32_t* __restrict__ used) {
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[t]) continue;
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    int path[4][3];
    kuhn_path((int)(q / ((int64_t)g.Gc * g.Gc)), (int)((q / g.Gc) % g.Gc), (int)(q % g.Gc), k, path);
    for (int s = 0; s < 4; ++s) used[((int64_t)path[s][0] * g.G + path[s][1]) * g.G + path[s][2]] = 1;
  }
}

__device__ __forceinline__ int seg_kept(const Grid& g, const int32_t* keep, int I, int J, int K, int k) {
  if (I < 0 || J < 0 || K < 0 || I >= g.Gc || J >= g.Gc || K >= g.Gc) return 0;
  return keep[6 * (((int64_t)I * g.Gc + J) * g.Gc + K) + k];
}

// Boundary-face mask of kept candidate tet k of cube (I, J, K), by stored local face.
__device__ __forceinline__ int seg_bmask(const Grid& g, const int32_t* keep, int I, int J, int K, int k) {
  const int a = c_perm[k][0], b = c_perm[k][1], c = c_perm[k][2];
  int nb[4];
  int qa[3] = {I, J, K};
  qa[a] += 1;
  nb[0] = seg_kept(g, keep, qa[0], qa[1], qa[2], perm_index(b, c, a));
  nb[1] = seg_kept(g, keep, I, J, K, perm_index(b, a, c));
  nb[2] = seg_kept(g, keep, I, J, K, perm_index(a, c, b));
  int qc[3] = {I, J, K};
  qc[c] -= 1;
  nb[3] = seg_kept(g, keep, qc[0], qc[1], qc[2], perm_index(c, a, b));
  int m = 0;
  for (int f = 0; f < 4; ++f) {
    const int pv = c_odd[k] ? (f == 2 ? 3 : (f == 3 ? 2 : f)) : f;  // path vertex opposite stored face f
    if (!nb[pv]) m |= 1 << f;
  }
  return m;
}

__global__ void k_seg_out(Grid g, const int32_t* __restrict__ keep, const int32_t* __restrict__ tlab,
                          const int32_t* __restrict__ toff, const int32_t* __restrict__ nid,
                          int32_t* __restrict__ tets, int32_t* __restrict__ labels, int32_t* __restrict__ bcnt) {
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[t]) continue;
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    const int I = (int)(q / ((int64_t)g.Gc * g.Gc));
    const int J = (int)((q / g.Gc) % g.Gc);
    const int K = (int)(q % g.Gc);
    const int64_t o = toff[t];
    if (tets) {
      int path[4][3];
      kuhn_path(I, J, K, k, path);
      int32_t v[4];
      for (int s = 0; s < 4; ++s) v[s] = nid[((int64_t)path[s][0] * g.G + path[s][1]) * g.G + path[s][2]];
      if (c_odd[k]) {
        const int32_t x = v[2];
        v[2] = v[3];
        v[3] = x;
      }
      for (int s = 0; s < 4; ++s) tets[4 * o + s] = v[s];
      labels[o] = tlab[t];
    }
    bcnt[o] = __popc(seg_bmask(g, keep, I, J, K, k));
  }
}

__global__ void k_seg_bfaces(Grid g, const int32_t* __restrict__ keep, const int32_t* __restrict__ toff,
                             const int32_t* __restrict__ boff, const int32_t* __restrict__ tets,
                             int32_t* __restrict__ bfaces) {
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[t]) continue;
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    const int msk = seg_bmask(g, keep, (int)(q / ((int64_t)g.Gc * g.Gc)), (int)((q / g.Gc) % g.Gc),
                              (int)(q % g.Gc), k);
    if (!msk) continue;
    const int64_t o = toff[t];
    int64_t b = boff[o];
    for (int f = 0; f < 4; ++f) {
      if (!(msk >> f & 1)) continue;
      for (int j = 0; j < 3; ++j) bfaces[3 * b + j] = tets[4 * o + c_face[f][j]];
      ++b;
    }
  }
}

}  // namespace
}  // namespace zi

extern "C" int zi_mesh_from_surfaces(double h, int n_surf, const int64_t* tri_offset, const int32_t* priority,
                                     const double* verts, int64_t nv, const int32_t* tris, int64_t* n_nodes,
                                     int64_t* n_tets, int64_t* n_bfaces, double* nodes, int32_t* tets,
                                     int32_t* labels, int32_t* bfaces, cudaStream_t s) {
  if (!n_nodes || !n_tets || !n_bfaces) return set_error(ZI_ERR_ARG, "size outputs must be non-null");
  const int outs = (nodes != nullptr) + (tets != nullptr) + (labels != nullptr) + (bfaces != nullptr);
  if (outs != 0 && outs != 4) return set_error(ZI_ERR_ARG, "pass all four mesh outputs or none");
  if (!(h > 0) || !isfinite(h)) return set_error(ZI_ERR_ARG, "grid step h must be positive and finite");
  if (n_surf < 1 || n_surf > SEG_MAX_SURF) return set_error(ZI_ERR_ARG, "need 1..%d surfaces", SEG_MAX_SURF);
  if (!tri_offset || !priority || !verts || !tris || nv < 3) return set_error(ZI_ERR_ARG, "null or empty surface input");
  SegParams sp;
  sp.C = n_surf;
  if (tri_offset[0] != 0) return set_error(ZI_ERR_ARG, "tri_offset[0] must be 0");
  for (int c = 0; c <= n_surf; ++c) {
    sp.toff[c] = tri_offset[c];
    if (c && !(tri_offset[c] > tri_offset[c - 1])) return set_error(ZI_ERR_ARG, "every surface needs triangles");
  }
  // ranks: order by (priority, index)
  for (int c = 0; c < n_surf; ++c) sp.order[c] = c;
  for (int i = 1; i < n_surf; ++i)
    for (int j = i; j > 0; --j) {
      const int x = sp.order[j - 1], y = sp.order[j];
      if (priority[y] < priority[x] || (priority[y] == priority[x] && y < x)) {
        sp.order[j - 1] = y;
        sp.order[j] = x;
      }
    }
  for (int r = 0; r < n_surf; ++r) sp.rank[sp.order[r]] = r;
  DevTmp<unsigned long long> mx;
  DevTmp<int> err;
  ZI_CHECK(mx.alloc(1, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_seg_maxabs<<<grid_for(3 * nv, 256), 256, 0, s>>>(nv, verts, mx.p, err.p);
  ZI_LAUNCH_CHECK();
  unsigned long long bits = 0;
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  double R;
  memcpy(&R, &bits, sizeof(R));
  const double qd = ceil(R / h);
  if (qd > 300) return set_error(ZI_ERR_ARG, "grid too large (max |coordinate| / h = %g)", qd);
  Grid g;
  g.N = (int)qd + 1;
  g.G = 2 * g.N + 1;
  g.Gc = 2 * g.N;
  const int64_t nvg = (int64_t)g.G * g.G * g.G;
  const int64_t ncand = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  DevTmp<int32_t> lab, keep, tlab, used, nid, toff, bcnt, boff, tets_tmp;
  ZI_CHECK(lab.alloc(nvg, s));
  ZI_CHECK(keep.alloc(ncand, s));
  ZI_CHECK(tlab.alloc(ncand, s));
  ZI_CHECK(used.alloc(nvg, s));
  ZI_CHECK(nid.alloc(nvg + 1, s));
  ZI_CHECK(toff.alloc(ncand + 1, s));
  k_seg_labels<<<grid_for(nvg, 128, 152u * 64u), 128, 0, s>>>(g, h, sp, nv, verts, tris, lab.p, err.p);
  ZI_LAUNCH_CHECK();
  k_seg_tets<<<grid_for(ncand, 256), 256, 0, s>>>(g, sp, lab.p, keep.p, tlab.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaMemsetAsync(used.p, 0, sizeof(int32_t) * nvg, s));
  k_seg_used<<<grid_for(ncand, 256), 256, 0, s>>>(g, keep.p, used.p);
  ZI_LAUNCH_CHECK();
  int64_t n = 0, m = 0, nb = 0;
  ZI_CHECK(exclusive_scan_i32(used.p, nid.p, nvg, &n, s));
  ZI_CHECK(exclusive_scan_i32(keep.p, toff.p, ncand, &m, s));
  if (m > INT32_MAX / 4) return set_error(ZI_ERR_ARG, "mesh too large for int32 indices");
  ZI_CHECK(bcnt.alloc(m, s));
  ZI_CHECK(boff.alloc(m + 1, s));
  // the boundary faces read the tets back, so the counting call keeps its own copy
  int32_t* tets_w = tets;
  int32_t* labels_w = labels;
  DevTmp<int32_t> labels_tmp;
  if (!outs) {
    ZI_CHECK(tets_tmp.alloc(4 * m, s));
    ZI_CHECK(labels_tmp.alloc(m, s));
    tets_w = tets_tmp.p;
    labels_w = labels_tmp.p;
  }
  k_seg_out<<<grid_for(ncand, 256), 256, 0, s>>>(g, keep.p, tlab.p, toff.p, nid.p, tets_w, labels_w, bcnt.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(exclusive_scan_i32(bcnt.p, boff.p, m, &nb, s));
  if (outs && *n_bfaces != nb)
    return set_error(ZI_ERR_ARG, "pass the count of the counting call in n_bfaces");
  if (outs) {
    k_nodes_out<<<grid_for(nvg, 256), 256, 0, s>>>(g, h, used.p, nid.p, nodes);
    ZI_LAUNCH_CHECK();
    k_seg_bfaces<<<grid_for(ncand, 256), 256, 0, s>>>(g, keep.p, toff.p, boff.p, tets, bfaces);
    ZI_LAUNCH_CHECK();
  }
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  *n_nodes = n;
  *n_tets = m;
  *n_bfaces = nb;
  return ZI_OK;
}
