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

// The surface tables live in one small device array of int64 (never in the
// kernel parameters, and read one entry at a time):
//   tab[0 .. C]            triangle offsets (surface c: tab[c] .. tab[c+1]-1)
//   tab[C+1 .. 2C]         rank of compartment c (order by (priority, index))
//   tab[2C+1 .. 3C]        compartment of rank r
__host__ __device__ inline int64_t seg_tab_len(int C) { return 3 * (int64_t)C + 1; }

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

// Node labels by winding numbers.  Each surface's triangle range starts where
// the previous one ended, so only the range ends are read (into shared
// memory, one entry per load).
__global__ void k_seg_labels(Grid g, double h, int C, const int64_t* __restrict__ tab, int64_t nv, int64_t ntri,
                             const double* __restrict__ verts, const int32_t* __restrict__ tris,
                             int32_t* __restrict__ lab, int* __restrict__ err) {
  __shared__ int64_t s_end[SEG_MAX_SURF];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int64_t e = tab[c + 1];
    s_end[c] = (e < 0 || e > ntri) ? ntri : e;
    if (e < 0 || e > ntri) atomicOr(err, DEV_ERR_BAD_INDEX);
  }
  __syncthreads();
  const int64_t total = (int64_t)g.G * g.G * g.G;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(v / ((int64_t)g.G * g.G));
    const int J = (int)((v / g.G) % g.G);
    const int K = (int)(v % g.G);
    const double px = __dmul_rn((double)(I - g.N), h);
    const double py = __dmul_rn((double)(J - g.N), h);
    const double pz = __dmul_rn((double)(K - g.N), h);
    int label = -1;
    int64_t t = 0;
    for (int c = 0; c < C && label < 0; ++c) {
      const int64_t t1 = s_end[c];
      double acc = 0.0;
      for (; t < t1; ++t) {
        const int32_t i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
        if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
          atomicOr(err, DEV_ERR_BAD_INDEX);
          continue;
        }
        const double ax = verts[3 * (int64_t)i0] - px, ay = verts[3 * (int64_t)i0 + 1] - py,
                     az = verts[3 * (int64_t)i0 + 2] - pz;
        const double bx = verts[3 * (int64_t)i1] - px, by = verts[3 * (int64_t)i1 + 1] - py,
                     bz = verts[3 * (int64_t)i1 + 2] - pz;
        const double cx = verts[3 * (int64_t)i2] - px, cy = verts[3 * (int64_t)i2 + 1] - py,
                     cz = verts[3 * (int64_t)i2 + 2] - pz;
        const double a = sqrt(ax * ax + ay * ay + az * az);
        const double b = sqrt(bx * bx + by * by + bz * bz);
        const double cc = sqrt(cx * cx + cy * cy + cz * cz);
        const double num = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
        const double den = a * b * cc + (ax * bx + ay * by + az * bz) * cc + (bx * cx + by * cy + bz * cz) * a +
                           (cx * ax + cy * ay + cz * az) * b;
        acc += 2.0 * atan2(num, den);
      }
      if (acc / (4.0 * 3.14159265358979323846) >= 0.5) label = c;
    }
    lab[v] = label;
  }
}

// The segmentation kernels take the Kuhn permutation of a candidate tet from
// its run-time index k (t mod 6), so they derive its axes by arithmetic
// instead of reading rows of the constant tables at a run-time index.
// Axis order of permutation k in lexicographic order (012, 021, 102, 120,
// 201, 210): a = k / 2, then the smaller (k even) or larger (k odd) of the two
// other axes; odd permutations are 021, 102, 210.
__device__ __forceinline__ void perm_axes(int k, int& a, int& b, int& c) {
  a = k >> 1;
  const int lo = a == 0 ? 1 : 0, hi = a == 2 ? 1 : 2;
  b = (k & 1) ? hi : lo;
  c = 3 - a - b;
}
__device__ __forceinline__ int perm_odd(int k) { return (k + (k >> 1)) & 1; }
__device__ __forceinline__ int perm_index(int a, int b, int c) { return 2 * a + (b > c ? 1 : 0); }

// Path vertex s (0..3) of Kuhn tet k of cube (I, J, K): the cube's first
// corner, then unit steps along axes a, b, c.
__device__ __forceinline__ void kuhn_vertex(int I, int J, int K, int k, int s, int& x, int& y, int& z) {
  int a, b, c;
  perm_axes(k, a, b, c);
  x = I + (s >= 1 && a == 0) + (s >= 2 && b == 0) + (s >= 3 && c == 0);
  y = J + (s >= 1 && a == 1) + (s >= 2 && b == 1) + (s >= 3 && c == 1);
  z = K + (s >= 1 && a == 2) + (s >= 2 && b == 2) + (s >= 3 && c == 2);
}

// Linear index of grid node (x, y, z), or -1 outside the G^3 grid.
__device__ __forceinline__ int64_t seg_node(const Grid& g, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= g.G || y >= g.G || z >= g.G) return -1;
  return ((int64_t)x * g.G + y) * g.G + z;
}

__global__ void k_seg_tets(Grid g, int C, const int64_t* __restrict__ tab, const int32_t* __restrict__ lab,
                           int32_t* __restrict__ keep, int32_t* __restrict__ tlab, int* __restrict__ err) {
  __shared__ int s_rank[SEG_MAX_SURF], s_order[SEG_MAX_SURF];
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int64_t r = tab[C + 1 + c], o = tab[2 * C + 1 + c];
    const bool bad = r < 0 || r >= C || o < 0 || o >= C;
    s_rank[c] = bad ? C : (int)r;
    s_order[c] = bad ? 0 : (int)o;
    if (bad) atomicOr(err, DEV_ERR_BAD_INDEX);
  }
  __syncthreads();
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    const int I = (int)(q / ((int64_t)g.Gc * g.Gc)), J = (int)((q / g.Gc) % g.Gc), K = (int)(q % g.Gc);
    int best = C;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int x, y, z;
      kuhn_vertex(I, J, K, k, s, x, y, z);
      const int64_t lin = seg_node(g, x, y, z);
      if (lin < 0) {
        atomicOr(err, DEV_ERR_BAD_INDEX);
        continue;
      }
      const int l = lab[lin];
      if (l < -1 || l >= C) {
        atomicOr(err, DEV_ERR_BAD_INDEX);
        continue;
      }
      const int r = l < 0 ? C : s_rank[l];
      best = r < best ? r : best;
    }
    keep[t] = best < C;
    tlab[t] = best < C ? s_order[best] : -1;
  }
}

__global__ void k_seg_used(Grid g, const int32_t* __restrict__ keep, int32_t* __restrict__ used,
                           int* __restrict__ err) {
  const int64_t total = 6 * (int64_t)g.Gc * g.Gc * g.Gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[t]) continue;
    const int64_t q = t / 6;
    const int k = (int)(t - 6 * q);
    const int I = (int)(q / ((int64_t)g.Gc * g.Gc)), J = (int)((q / g.Gc) % g.Gc), K = (int)(q % g.Gc);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int x, y, z;
      kuhn_vertex(I, J, K, k, s, x, y, z);
      const int64_t lin = seg_node(g, x, y, z);
      if (lin < 0) {
        atomicOr(err, DEV_ERR_BAD_INDEX);
        continue;
      }
      used[lin] = 1;
    }
  }
}

__device__ __forceinline__ int seg_kept(const Grid& g, const int32_t* keep, int I, int J, int K, int k) {
  if (I < 0 || J < 0 || K < 0 || I >= g.Gc || J >= g.Gc || K >= g.Gc) return 0;
  return keep[6 * (((int64_t)I * g.Gc + J) * g.Gc + K) + k];
}

// Boundary-face mask of kept candidate tet k of cube (I, J, K), by stored
// local face (bit f: face f is on the boundary).  The neighbour across the
// face opposite path vertex 0 is tet (b, c, a) of cube +e_a, opposite path
// vertex 3 tet (c, a, b) of cube -e_c, opposite path vertices 1 and 2 the
// tets (b, a, c) and (a, c, b) of the same cube; for an odd permutation the
// stored faces 2 and 3 are opposite path vertices 3 and 2.
__device__ __forceinline__ int seg_bmask(const Grid& g, const int32_t* keep, int I, int J, int K, int k) {
  int a, b, c;
  perm_axes(k, a, b, c);
  const int n0 = seg_kept(g, keep, I + (a == 0), J + (a == 1), K + (a == 2), perm_index(b, c, a));
  const int n1 = seg_kept(g, keep, I, J, K, perm_index(b, a, c));
  const int n2 = seg_kept(g, keep, I, J, K, perm_index(a, c, b));
  const int n3 = seg_kept(g, keep, I - (c == 0), J - (c == 1), K - (c == 2), perm_index(c, a, b));
  const bool odd = perm_odd(k);
  const int f2 = odd ? n3 : n2, f3 = odd ? n2 : n3;
  return (n0 ? 0 : 1) | (n1 ? 0 : 2) | (f2 ? 0 : 4) | (f3 ? 0 : 8);
}

// Vertices of the outward local face f of a positively oriented tet (face f
// opposite vertex f): {1,2,3}, {0,3,2}, {0,1,3}, {0,2,1}.
__device__ __forceinline__ void tet_face(int f, int& u, int& v, int& w) {
  u = f == 0 ? 1 : 0;
  v = f == 0 ? 2 : (f == 1 ? 3 : (f == 2 ? 1 : 2));
  w = f == 0 ? 3 : (f == 1 ? 2 : (f == 2 ? 3 : 1));
}

// Kept tets with their labels (output call) and boundary-face counts.  toff
// and nid come from scans of keep and used, so o < m and every node id of a
// kept tet is < n; the node index is still checked.
__global__ void k_seg_out(Grid g, const int32_t* __restrict__ keep, const int32_t* __restrict__ tlab,
                          const int32_t* __restrict__ toff, const int32_t* __restrict__ nid,
                          int32_t* __restrict__ tets, int32_t* __restrict__ labels, int32_t* __restrict__ bcnt,
                          int* __restrict__ err) {
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
      int32_t v[4];
      bool ok = true;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        int x, y, z;
        kuhn_vertex(I, J, K, k, s, x, y, z);
        const int64_t lin = seg_node(g, x, y, z);
        ok = ok && lin >= 0;
        v[s] = lin >= 0 ? nid[lin] : -1;
      }
      if (!ok) atomicOr(err, DEV_ERR_BAD_INDEX);
      const bool odd = perm_odd(k);
      tets[4 * o + 0] = v[0];
      tets[4 * o + 1] = v[1];
      tets[4 * o + 2] = odd ? v[3] : v[2];
      tets[4 * o + 3] = odd ? v[2] : v[3];
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
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!(msk >> f & 1)) continue;
      int u, v, w;
      tet_face(f, u, v, w);
      bfaces[3 * b + 0] = tets[4 * o + u];
      bfaces[3 * b + 1] = tets[4 * o + v];
      bfaces[3 * b + 2] = tets[4 * o + w];
      ++b;
    }
  }
}

inline bool misaligned(const void* p, size_t a) { return ((uintptr_t)p % a) != 0; }

}  // namespace
}  // namespace zi

// The mesher is set-up work, so each kernel is followed by a stream
// synchronisation: a device error is then reported at the line of the kernel
// that raised it.
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
  if (nv > INT32_MAX) return set_error(ZI_ERR_ARG, "too many surface vertices for int32 triangle indices");
  if (misaligned(verts, 8) || misaligned(tris, 4) || misaligned(nodes, 8) || misaligned(tets, 4) ||
      misaligned(labels, 4) || misaligned(bfaces, 4))
    return set_error(ZI_ERR_ARG, "arrays must be aligned to their element size");
  if (tri_offset[0] != 0) return set_error(ZI_ERR_ARG, "tri_offset[0] must be 0");
  const int C = n_surf;
  std::vector<int64_t> tab(seg_tab_len(C));
  for (int c = 0; c <= C; ++c) {
    if (c && !(tri_offset[c] > tri_offset[c - 1])) return set_error(ZI_ERR_ARG, "every surface needs triangles");
    tab[c] = tri_offset[c];
  }
  const int64_t ntri = tri_offset[C];
  if (ntri > INT64_MAX / 3) return set_error(ZI_ERR_ARG, "too many triangles");
  // ranks: order by (priority, index)
  std::vector<int> order(C), rank(C);
  for (int c = 0; c < C; ++c) order[c] = c;
  for (int i = 1; i < C; ++i)
    for (int j = i; j > 0; --j) {
      const int x = order[j - 1], y = order[j];
      if (priority[y] < priority[x] || (priority[y] == priority[x] && y < x)) {
        order[j - 1] = y;
        order[j] = x;
      }
    }
  for (int r = 0; r < C; ++r) rank[order[r]] = r;
  for (int c = 0; c < C; ++c) {
    tab[C + 1 + c] = rank[c];
    tab[2 * C + 1 + c] = order[c];
  }
  DevTmp<unsigned long long> mx;
  DevTmp<int> err;
  DevTmp<int64_t> dtab;
  ZI_CHECK(mx.alloc(1, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CHECK(dtab.alloc(tab.size(), s));
  ZI_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  ZI_CUDA(cudaMemcpyAsync(dtab.p, tab.data(), sizeof(int64_t) * tab.size(), cudaMemcpyHostToDevice, s));
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
  k_seg_labels<<<grid_for(nvg, 128, 152u * 64u), 128, 0, s>>>(g, h, C, dtab.p, nv, ntri, verts, tris, lab.p,
                                                                err.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaStreamSynchronize(s));
  k_seg_tets<<<grid_for(ncand, 256), 256, 0, s>>>(g, C, dtab.p, lab.p, keep.p, tlab.p, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CUDA(cudaMemsetAsync(used.p, 0, sizeof(int32_t) * nvg, s));
  k_seg_used<<<grid_for(ncand, 256), 256, 0, s>>>(g, keep.p, used.p, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  int64_t n = 0, m = 0, nb = 0;
  ZI_CHECK(exclusive_scan_i32(used.p, nid.p, nvg, &n, s));
  ZI_CHECK(exclusive_scan_i32(keep.p, toff.p, ncand, &m, s));
  if (m > INT32_MAX / 4) return set_error(ZI_ERR_ARG, "mesh too large for int32 indices");
  // the output call writes into arrays sized by the counting call's counts
  if (outs && (*n_nodes != n || *n_tets != m))
    return set_error(ZI_ERR_ARG, "pass the counts of the counting call in n_nodes and n_tets");
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
  k_seg_out<<<grid_for(ncand, 256), 256, 0, s>>>(g, keep.p, tlab.p, toff.p, nid.p, tets_w, labels_w, bcnt.p,
                                                   err.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(exclusive_scan_i32(bcnt.p, boff.p, m, &nb, s));
  if (outs && *n_bfaces != nb)
    return set_error(ZI_ERR_ARG, "pass the count of the counting call in n_bfaces");
  if (outs) {
    k_nodes_out<<<grid_for(nvg, 256), 256, 0, s>>>(g, h, used.p, nid.p, nodes);
    ZI_LAUNCH_CHECK();
    ZI_CUDA(cudaStreamSynchronize(s));
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
