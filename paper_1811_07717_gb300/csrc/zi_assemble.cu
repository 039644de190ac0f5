// Assembly of the grounded FEM system (App. A.1):
//   a_ij = sum_e vol_e grad(psi_i)^T Sigma_e grad(psi_j)
//        + sum_l 1/z_l int_{e_l} psi_i psi_j,
//   b_il = 1/z_l int_{e_l} psi_i,  c_ll = |e_l| / z_l,
// grounding row and column i'.
//
// The CSR pattern is the mesh graph.  Every contribution to A is an "entry"
// with a unique id: tet entries 16 t + 4 a + b, surface entries of electrode
// patch faces 16 m + 9 f + 3 a + b.  Entries are bucketed by row, each bucket
// is sorted by (column, id), and A's values are segmented sums over that
// order: deterministic, with no floating-point atomics.  The sorted buckets
// (seg, perm) are the element-to-nonzero map reused whenever the conductivity
// changes.
#include <math.h>
#include <string.h>

#include <vector>

#include "zi_internal.cuh"
#include "zi_pcg.cuh"

namespace zi {
namespace {

__constant__ int c_sym[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};

// ---------------------------------------------------------------------------
// element geometry and stiffness
// ---------------------------------------------------------------------------

// grad(lambda_1..3) = (e2 x e3, e3 x e1, e1 x e2) / det with e_k = x_k - x_0,
// grad(lambda_0) = -(sum of the others), vol = det / 6.
__global__ void k_element(int64_t m, const double* __restrict__ X, const int32_t* __restrict__ tets,
                          const double* __restrict__ s6, double* __restrict__ Ke, int* __restrict__ err) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    int4 v = reinterpret_cast<const int4*>(tets)[t];
    double x0[3], e[3][3];
    for (int d = 0; d < 3; ++d) x0[d] = X[3 * (int64_t)v.x + d];
    for (int d = 0; d < 3; ++d) {
      e[0][d] = X[3 * (int64_t)v.y + d] - x0[d];
      e[1][d] = X[3 * (int64_t)v.z + d] - x0[d];
      e[2][d] = X[3 * (int64_t)v.w + d] - x0[d];
    }
    double g[4][3];
    // cross products
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
    const double* sp = s6 + 6 * t;
    double s11 = sp[0], s22 = sp[1], s33 = sp[2], s12 = sp[3], s13 = sp[4], s23 = sp[5];
    bool fin = isfinite(s11) && isfinite(s22) && isfinite(s33) && isfinite(s12) && isfinite(s13) &&
               isfinite(s23);
    if (!fin) atomicOr(err, DEV_ERR_NONFINITE);
    if (!(det > 0) || !isfinite(det)) atomicOr(err, DEV_ERR_BAD_VOLUME);
    double inv = 1.0 / det;
    for (int a = 1; a < 4; ++a)
      for (int d = 0; d < 3; ++d) g[a][d] *= inv;
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    double vol = det / 6.0;
    double sg[4][3];
    for (int a = 0; a < 4; ++a) {
      sg[a][0] = s11 * g[a][0] + s12 * g[a][1] + s13 * g[a][2];
      sg[a][1] = s12 * g[a][0] + s22 * g[a][1] + s23 * g[a][2];
      sg[a][2] = s13 * g[a][0] + s23 * g[a][1] + s33 * g[a][2];
    }
    double* kp = Ke + 10 * t;
    int idx = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = a; b < 4; ++b)
        kp[idx++] = vol * (g[a][0] * sg[b][0] + g[a][1] * sg[b][1] + g[a][2] * sg[b][2]);
  }
}

// ---------------------------------------------------------------------------
// electrodes
// ---------------------------------------------------------------------------

// CEM patch of each boundary face: the electrode whose centre is within
// `radius` of the face centroid ((p0+p1)+p2)/3; squared distance summed x, y, z.
__global__ void k_face_electrode(int64_t nb, const double* __restrict__ X, const int32_t* __restrict__ bf,
                                 int L, const double* __restrict__ cen, double r2,
                                 const double* __restrict__ zinv, int32_t* __restrict__ face_el,
                                 double* __restrict__ face_w, int32_t* __restrict__ el_count,
                                 int* __restrict__ err) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nb;
       f += (int64_t)gridDim.x * blockDim.x) {
    int32_t v0 = bf[3 * f], v1 = bf[3 * f + 1], v2 = bf[3 * f + 2];
    double p[3][3];
    for (int d = 0; d < 3; ++d) {
      p[0][d] = X[3 * (int64_t)v0 + d];
      p[1][d] = X[3 * (int64_t)v1 + d];
      p[2][d] = X[3 * (int64_t)v2 + d];
    }
    double c[3];
    for (int d = 0; d < 3; ++d) c[d] = __ddiv_rn(__dadd_rn(__dadd_rn(p[0][d], p[1][d]), p[2][d]), 3.0);
    int owner = -1, hits = 0;
    for (int l = 0; l < L; ++l) {
      double dx = __dsub_rn(c[0], cen[3 * l + 0]);
      double dy = __dsub_rn(c[1], cen[3 * l + 1]);
      double dz = __dsub_rn(c[2], cen[3 * l + 2]);
      double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      if (d2 < r2) {
        if (owner < 0) owner = l;
        ++hits;
      }
    }
    if (hits > 1) atomicOr(err, DEV_ERR_OVERLAP);
    face_el[f] = owner;
    double w = 0.0;
    if (owner >= 0) {
      double a[3], b[3];
      for (int d = 0; d < 3; ++d) {
        a[d] = p[1][d] - p[0][d];
        b[d] = p[2][d] - p[0][d];
      }
      double cx = a[1] * b[2] - a[2] * b[1];
      double cy = a[2] * b[0] - a[0] * b[2];
      double cz = a[0] * b[1] - a[1] * b[0];
      double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
      w = area * zinv[owner];
      atomicAdd(&el_count[owner], 1);
    }
    face_w[f] = w;
  }
}

__global__ void k_flag_boundary(int64_t nb, const int32_t* __restrict__ bf, const int32_t* __restrict__ face_el,
                                int32_t* __restrict__ bnode, int32_t* __restrict__ pnode) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nb;
       f += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      int32_t v = bf[3 * f + k];
      bnode[v] = 1;
      if (face_el && face_el[f] >= 0) pnode[v] = 1;
    }
  }
}

__global__ void k_ground_cem(int64_t n, const int32_t* __restrict__ bnode, const int32_t* __restrict__ pnode,
                             int32_t* __restrict__ ground) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (bnode[i] && !pnode[i]) atomicMin(ground, (int32_t)i);
}

// Point electrode l: boundary node nearest its centre, lowest index on ties.
__global__ void k_point_nearest(int64_t n, const double* __restrict__ X, const int32_t* __restrict__ bnode,
                                const double* __restrict__ cen, int32_t* __restrict__ el_nodes) {
  const int l = blockIdx.x;
  double px = cen[3 * l], py = cen[3 * l + 1], pz = cen[3 * l + 2];
  double best = INFINITY;
  int64_t bi = INT64_MAX;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (!bnode[i]) continue;
    double dx = __dsub_rn(X[3 * i], px), dy = __dsub_rn(X[3 * i + 1], py), dz = __dsub_rn(X[3 * i + 2], pz);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < best || (d2 == best && i < bi)) {
      best = d2;
      bi = i;
    }
  }
  __shared__ double sb[1024];
  __shared__ int64_t si[1024];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double b2 = sb[threadIdx.x + o];
      int64_t i2 = si[threadIdx.x + o];
      if (b2 < sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) el_nodes[l] = (int32_t)si[0];
}

// ---------------------------------------------------------------------------
// pattern and entry map
// ---------------------------------------------------------------------------

__global__ void k_row_counts(int64_t m, const int32_t* __restrict__ tets, int64_t nb,
                             const int32_t* __restrict__ bf, const int32_t* __restrict__ face_el,
                             int32_t* __restrict__ cnt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m + nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      for (int a = 0; a < 4; ++a) atomicAdd(&cnt[tets[4 * t + a]], 4);
    } else {
      int64_t f = t - m;
      if (face_el && face_el[f] >= 0)
        for (int a = 0; a < 3; ++a) atomicAdd(&cnt[bf[3 * f + a]], 3);
    }
  }
}

__global__ void k_fill_buckets(int64_t m, const int32_t* __restrict__ tets, int64_t nb,
                               const int32_t* __restrict__ bf, const int32_t* __restrict__ face_el,
                               const int32_t* __restrict__ start, int32_t* __restrict__ fill,
                               uint64_t* __restrict__ bucket) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m + nb;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < m) {
      int32_t v[4];
      for (int a = 0; a < 4; ++a) v[a] = tets[4 * t + a];
      for (int a = 0; a < 4; ++a) {
        int32_t r = v[a];
        int32_t slot = atomicAdd(&fill[r], 4);
        for (int b = 0; b < 4; ++b) {
          uint32_t id = (uint32_t)(16 * t + 4 * a + b);
          bucket[(int64_t)start[r] + slot + b] = ((uint64_t)(uint32_t)v[b] << 32) | id;
        }
      }
    } else {
      int64_t f = t - m;
      if (!face_el || face_el[f] < 0) continue;
      int32_t v[3];
      for (int a = 0; a < 3; ++a) v[a] = bf[3 * f + a];
      for (int a = 0; a < 3; ++a) {
        int32_t r = v[a];
        int32_t slot = atomicAdd(&fill[r], 3);
        for (int b = 0; b < 3; ++b) {
          uint32_t id = (uint32_t)(16 * m + 9 * f + 3 * a + b);
          bucket[(int64_t)start[r] + slot + b] = ((uint64_t)(uint32_t)v[b] << 32) | id;
        }
      }
    }
  }
}

constexpr int WARP_SORT_MAX = 256;
constexpr int BLOCK_SORT_MAX = 4096;
constexpr int SORT_WARPS = 8;

// Sorts each row's bucket by (column, id) and counts its distinct columns.
// Rows longer than WARP_SORT_MAX are queued for the block-wide sort.
__global__ void __launch_bounds__(SORT_WARPS * 32) k_sort_rows_warp(
    int64_t n, const int32_t* __restrict__ start, uint64_t* __restrict__ bucket,
    int32_t* __restrict__ ucount, int32_t* __restrict__ big, int32_t* __restrict__ nbig) {
  __shared__ uint64_t sm[SORT_WARPS][WARP_SORT_MAX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* s = sm[w];
  for (int64_t i = (int64_t)blockIdx.x * SORT_WARPS + w; i < n; i += (int64_t)gridDim.x * SORT_WARPS) {
    int64_t b0 = start[i];
    int cnt = start[i + 1] - start[i];
    if (cnt > WARP_SORT_MAX) {
      if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)i;
      continue;
    }
    int S = 1;
    while (S < cnt) S <<= 1;
    for (int k = lane; k < S; k += 32) s[k] = (k < cnt) ? bucket[b0 + k] : ~0ull;
    __syncwarp();
    for (int k = 2; k <= S; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int x = lane; x < S; x += 32) {
          int y = x ^ j;
          if (y > x) {
            uint64_t a = s[x], b = s[y];
            bool up = (x & k) == 0;
            if ((a > b) == up) {
              s[x] = b;
              s[y] = a;
            }
          }
        }
        __syncwarp();
      }
    }
    int u = 0;
    for (int k = lane; k < cnt; k += 32) {
      bucket[b0 + k] = s[k];
      if (k == 0 || (s[k] >> 32) != (s[k - 1] >> 32)) ++u;
    }
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) ucount[i] = u;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_sort_rows_block(const int32_t* __restrict__ big, const int32_t* __restrict__ nbig,
                                                         const int32_t* __restrict__ start, uint64_t* __restrict__ bucket,
                                                         int32_t* __restrict__ ucount, int* __restrict__ err) {
  extern __shared__ uint64_t s[];
  __shared__ int red[256];
  for (int q = blockIdx.x; q < *nbig; q += gridDim.x) {
    int64_t i = big[q];
    int64_t b0 = start[i];
    int cnt = start[i + 1] - start[i];
    if (cnt > BLOCK_SORT_MAX) {
      if (threadIdx.x == 0) {
        atomicOr(err, DEV_ERR_VALENCE);
        ucount[i] = 0;
      }
      continue;
    }
    int S = 1;
    while (S < cnt) S <<= 1;
    for (int k = threadIdx.x; k < S; k += blockDim.x) s[k] = (k < cnt) ? bucket[b0 + k] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= S; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int x = threadIdx.x; x < S; x += blockDim.x) {
          int y = x ^ j;
          if (y > x) {
            uint64_t a = s[x], b = s[y];
            bool up = (x & k) == 0;
            if ((a > b) == up) {
              s[x] = b;
              s[y] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    int u = 0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      bucket[b0 + k] = s[k];
      if (k == 0 || (s[k] >> 32) != (s[k - 1] >> 32)) ++u;
    }
    red[threadIdx.x] = u;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) ucount[i] = red[0];
    __syncthreads();
  }
}

// Writes colind / seg / diagpos for each row and the entry ids (perm).
__global__ void k_emit_pattern(int64_t n, const int32_t* __restrict__ start, const uint64_t* __restrict__ bucket,
                               const int32_t* __restrict__ rowptr, int32_t* __restrict__ colind,
                               int32_t* __restrict__ seg, int32_t* __restrict__ diagpos,
                               int32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int64_t b0 = start[i];
    int cnt = start[i + 1] - start[i];
    int base = rowptr[i];
    int run = 0;  // distinct columns seen before this chunk
    for (int k0 = 0; k0 < cnt; k0 += 32) {
      int k = k0 + lane;
      bool first = false;
      uint64_t e = 0;
      if (k < cnt) {
        e = bucket[b0 + k];
        perm[b0 + k] = (int32_t)(uint32_t)(e & 0xffffffffu);
        first = (k == 0) || ((bucket[b0 + k - 1] >> 32) != (e >> 32));
      }
      unsigned msk = __ballot_sync(0xffffffffu, first);
      if (first) {
        int r = run + __popc(msk & ((1u << lane) - 1u));
        int32_t col = (int32_t)(e >> 32);
        colind[base + r] = col;
        seg[base + r] = (int32_t)(b0 + k);
        if (col == (int32_t)i) diagpos[i] = base + r;
      }
      run += __popc(msk);
    }
  }
}

// ---------------------------------------------------------------------------
// values: segmented sums in (row, column, id) order
// ---------------------------------------------------------------------------

__global__ void k_values(int64_t n, int64_t m, const int32_t* __restrict__ rowptr,
                         const int32_t* __restrict__ colind, const int32_t* __restrict__ seg,
                         const int32_t* __restrict__ perm, const double* __restrict__ Ke,
                         const double* __restrict__ face_w, const int32_t* __restrict__ face_el,
                         double* __restrict__ vals, double* __restrict__ B, int ldb) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t surf0 = 16 * m;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    int r0 = rowptr[i], r1 = rowptr[i + 1];
    for (int k = r0 + lane; k < r1; k += 32) {
      double acc = 0.0;
      bool diag = colind[k] == (int32_t)i;
      for (int q = seg[k]; q < seg[k + 1]; ++q) {
        int64_t id = (uint32_t)perm[q];
        if (id < surf0) {
          int64_t t = id >> 4;
          int a = (id >> 2) & 3, b = id & 3;
          acc += Ke[10 * t + c_sym[a][b]];
        } else {
          int64_t r = id - surf0;
          int64_t f = r / 9;
          int ab = (int)(r % 9);
          int a = ab / 3, b = ab % 3;
          double w = face_w[f];
          acc += (a == b) ? w * (2.0 / 12.0) : w * (1.0 / 12.0);
          if (diag && B) B[i * (int64_t)ldb + face_el[f]] += w * (1.0 / 3.0);
        }
      }
      vals[k] = acc;
    }
  }
}

// Grounding: row and column i' zeroed, a_i'i' = 1, B row i' zeroed.
__global__ void k_pin(int64_t ip, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                      double* __restrict__ vals, double* __restrict__ B, int ldb) {
  int r0 = rowptr[ip], r1 = rowptr[ip + 1];
  for (int k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
    int32_t j = colind[k];
    vals[k] = (j == (int32_t)ip) ? 1.0 : 0.0;
    if (j != (int32_t)ip) {
      int lo = rowptr[j], hi = rowptr[j + 1] - 1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int32_t c = colind[mid];
        if (c == (int32_t)ip) {
          vals[mid] = 0.0;
          break;
        }
        if (c < (int32_t)ip) lo = mid + 1; else hi = mid - 1;
      }
    }
  }
  if (B)
    for (int c = threadIdx.x; c < ldb; c += blockDim.x) B[ip * (int64_t)ldb + c] = 0.0;
}

// c_ll = sum of area/z_l over the patch, summed by one warp in a fixed order.
__global__ void k_cem_C(int64_t nb, int L, const int32_t* __restrict__ face_el, const double* __restrict__ face_w,
                        double* __restrict__ C) {
  const int lane = threadIdx.x & 31;
  for (int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < L; l += gridDim.x * (blockDim.x >> 5)) {
    double s = 0.0;
    for (int64_t f = lane; f < nb; f += 32)
      if (face_el[f] == l) s += face_w[f];
    s = warp_sum(s);
    if (lane == 0) C[l] = s;
  }
}

__global__ void k_point_rhs(int L, const int32_t* __restrict__ el_nodes, double* __restrict__ B, int ldb,
                            int* __restrict__ err) {
  int l = threadIdx.x + 1;
  for (; l < L; l += blockDim.x) {
    B[(int64_t)el_nodes[l] * ldb + (l - 1)] = 1.0;
    for (int k = 0; k < l; ++k)
      if (el_nodes[k] == el_nodes[l]) atomicOr(err, DEV_ERR_DUP_ELECTRODE);
  }
}

__global__ void k_nonzero_rows(int64_t n, const double* __restrict__ B, int ldb, int32_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int f = 0;
    for (int c = 0; c < ldb && !f; ++c) f = B[i * (int64_t)ldb + c] != 0.0;
    flag[i] = f;
  }
}

__global__ void k_compact(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ off,
                          int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) out[off[i]] = (int32_t)i;
}

int read_err(int* derr, cudaStream_t s) {
  int h = 0;
  ZI_CUDA(cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(h);
}

}  // namespace

void system_free(zi_system* S) {
  if (!S) return;
  cudaStream_t s = 0;
  void* ptrs[] = {S->nodes, S->tets, S->bfaces, S->Ke, S->rowptr, S->colind, S->diagpos, S->seg,
                  S->perm, S->vals, S->face_el, S->face_w, S->zinv, S->B, S->C, S->el_nodes,
                  S->patch_nodes, S->T};
  for (void* p : ptrs) dfree(p, s);
}


// Recomputes K_e, the values of A, B, C and the grounding (pattern fixed).
static int assemble_values(zi_system* S, const double* sigma6, cudaStream_t s) {
  DevTmp<int> err;
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  k_element<<<grid_for(S->m, 256), 256, 0, s>>>(S->m, S->nodes, S->tets, sigma6, S->Ke, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(read_err(err.p, s));
  ZI_CUDA(cudaMemsetAsync(S->B, 0, sizeof(double) * S->n * S->n_rhs, s));
  bool cem = S->model == ZI_ELECTRODE_CEM;
  k_values<<<grid_for(S->n * 32, 256, 152u * 64u), 256, 0, s>>>(
      S->n, S->m, S->rowptr, S->colind, S->seg, S->perm, S->Ke, S->face_w, S->face_el, S->vals,
      cem ? S->B : nullptr, S->n_rhs);
  ZI_LAUNCH_CHECK();
  if (cem) {
    k_cem_C<<<(S->n_el + 7) / 8, 256, 0, s>>>(S->nb, S->n_el, S->face_el, S->face_w, S->C);
    ZI_LAUNCH_CHECK();
  } else {
    k_point_rhs<<<1, 256, 0, s>>>(S->n_el, S->el_nodes, S->B, S->n_rhs, err.p);
    ZI_LAUNCH_CHECK();
  }
  k_pin<<<1, 256, 0, s>>>(S->ground, S->rowptr, S->colind, S->vals, S->B, S->n_rhs);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(read_err(err.p, s));
  S->has_T = 0;
  solver_invalidate(S);
  return ZI_OK;
}

static int assemble_impl(const double* nodes, int64_t n, const int32_t* tets, int64_t m,
                         const double* sigma6, const int32_t* bfaces, int64_t nb, const zi_electrodes* el,
                         zi_system* S, cudaStream_t s) {
  S->n = n;
  S->m = m;
  S->nb = nb;
  S->n_el = el->n;
  S->model = el->model;
  S->n_rhs = el->model == ZI_ELECTRODE_CEM ? el->n : el->n - 1;
  S->el_radius = el->radius;
  ZI_CUDA(cudaGetDevice(&S->device));
  ZI_CHECK(dalloc_n(&S->nodes, 3 * n, s));
  ZI_CHECK(dalloc_n(&S->tets, 4 * m, s));
  ZI_CHECK(dalloc_n(&S->bfaces, 3 * nb, s));
  ZI_CUDA(cudaMemcpyAsync(S->nodes, nodes, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  ZI_CUDA(cudaMemcpyAsync(S->tets, tets, sizeof(int32_t) * 4 * m, cudaMemcpyDeviceToDevice, s));
  ZI_CUDA(cudaMemcpyAsync(S->bfaces, bfaces, sizeof(int32_t) * 3 * nb, cudaMemcpyDeviceToDevice, s));
  ZI_CHECK(dalloc_n(&S->Ke, 10 * m, s));
  ZI_CHECK(dalloc_n(&S->face_el, nb, s));
  ZI_CHECK(dalloc_n(&S->face_w, nb, s));
  ZI_CHECK(dalloc_n(&S->zinv, S->n_el, s));
  ZI_CHECK(dalloc_n(&S->C, S->n_el, s));
  ZI_CHECK(dalloc_n(&S->B, n * (int64_t)S->n_rhs, s));
  ZI_CHECK(dalloc_n(&S->el_nodes, S->n_el, s));

  DevTmp<int> err;
  DevTmp<int32_t> bnode, pnode, elcnt, ground;
  ZI_CHECK(err.alloc(1, s));
  ZI_CHECK(bnode.alloc(n, s));
  ZI_CHECK(pnode.alloc(n, s));
  ZI_CHECK(elcnt.alloc(S->n_el, s));
  ZI_CHECK(ground.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  ZI_CUDA(cudaMemsetAsync(bnode.p, 0, sizeof(int32_t) * n, s));
  ZI_CUDA(cudaMemsetAsync(pnode.p, 0, sizeof(int32_t) * n, s));
  ZI_CUDA(cudaMemsetAsync(elcnt.p, 0, sizeof(int32_t) * S->n_el, s));
  ZI_CUDA(cudaMemsetAsync(S->face_w, 0, sizeof(double) * nb, s));

  const bool cem = el->model == ZI_ELECTRODE_CEM;
  std::vector<int32_t> h_el(S->n_el);
  if (cem) {
    // 1 / z_l on the host (z is small), then the patch of every boundary face
    std::vector<double> hz(S->n_el);
    ZI_CUDA(cudaMemcpyAsync(hz.data(), el->z, sizeof(double) * S->n_el, cudaMemcpyDeviceToHost, s));
    ZI_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < S->n_el; ++l) {
      if (!(hz[l] > 0) || !isfinite(hz[l])) return set_error(ZI_ERR_ARG, "contact impedance must be positive");
      hz[l] = 1.0 / hz[l];
    }
    ZI_CUDA(cudaMemcpyAsync(S->zinv, hz.data(), sizeof(double) * S->n_el, cudaMemcpyHostToDevice, s));
    double r2 = el->radius * el->radius;
    k_face_electrode<<<grid_for(nb, 256), 256, 0, s>>>(nb, S->nodes, S->bfaces, S->n_el, el->centres, r2,
                                                       S->zinv, S->face_el, S->face_w, elcnt.p, err.p);
    ZI_LAUNCH_CHECK();
    k_flag_boundary<<<grid_for(nb, 256), 256, 0, s>>>(nb, S->bfaces, S->face_el, bnode.p, pnode.p);
    ZI_LAUNCH_CHECK();
    int32_t big = INT32_MAX;
    ZI_CUDA(cudaMemcpyAsync(ground.p, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_ground_cem<<<grid_for(n, 256), 256, 0, s>>>(n, bnode.p, pnode.p, ground.p);
    ZI_LAUNCH_CHECK();
    int32_t g = 0;
    std::vector<int32_t> cnt(S->n_el);
    ZI_CUDA(cudaMemcpyAsync(&g, ground.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    ZI_CUDA(cudaMemcpyAsync(cnt.data(), elcnt.p, sizeof(int32_t) * S->n_el, cudaMemcpyDeviceToHost, s));
    ZI_CHECK(read_err(err.p, s));
    for (int l = 0; l < S->n_el; ++l)
      if (cnt[l] == 0) return set_error(ZI_ERR_BAD_MESH, "electrode %d covers no boundary triangle", l);
    if (g == INT32_MAX) return set_error(ZI_ERR_BAD_MESH, "no boundary node outside the electrodes");
    S->ground = g;
    int64_t npf = 0;
    for (int l = 0; l < S->n_el; ++l) npf += cnt[l];
    S->n_patch_faces = npf;
  } else {
    ZI_CUDA(cudaMemsetAsync(S->face_el, 0xff, sizeof(int32_t) * nb, s));
    k_flag_boundary<<<grid_for(nb, 256), 256, 0, s>>>(nb, S->bfaces, nullptr, bnode.p, pnode.p);
    ZI_LAUNCH_CHECK();
    k_point_nearest<<<S->n_el, 1024, 0, s>>>(n, S->nodes, bnode.p, el->centres, S->el_nodes);
    ZI_LAUNCH_CHECK();
    ZI_CUDA(cudaMemcpyAsync(h_el.data(), S->el_nodes, sizeof(int32_t) * S->n_el, cudaMemcpyDeviceToHost, s));
    ZI_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < S->n_el; ++a)
      for (int b = 0; b < a; ++b)
        if (h_el[a] == h_el[b]) return set_error(ZI_ERR_BAD_MESH, "point electrodes %d and %d share node %d", b, a, h_el[a]);
    S->ground = h_el[0];
  }

  // --- pattern: bucket entries by row, sort, dedupe
  DevTmp<int32_t> cnt, start, fill, ucount, big, nbig;
  ZI_CHECK(cnt.alloc(n, s));
  ZI_CHECK(start.alloc(n + 1, s));
  ZI_CHECK(fill.alloc(n, s));
  ZI_CHECK(ucount.alloc(n, s));
  ZI_CHECK(big.alloc(n, s));
  ZI_CHECK(nbig.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n, s));
  ZI_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int32_t) * n, s));
  ZI_CUDA(cudaMemsetAsync(nbig.p, 0, sizeof(int32_t), s));
  const int32_t* fe = cem ? S->face_el : nullptr;
  k_row_counts<<<grid_for(m + nb, 256), 256, 0, s>>>(m, S->tets, nb, S->bfaces, fe, cnt.p);
  ZI_LAUNCH_CHECK();
  int64_t E = 0;
  ZI_CHECK(exclusive_scan_i32(cnt.p, start.p, n, &E, s));
  S->n_entries = E;
  DevTmp<uint64_t> bucket;
  ZI_CHECK(bucket.alloc(E, s));
  k_fill_buckets<<<grid_for(m + nb, 256), 256, 0, s>>>(m, S->tets, nb, S->bfaces, fe, start.p, fill.p, bucket.p);
  ZI_LAUNCH_CHECK();
  k_sort_rows_warp<<<grid_for(n, SORT_WARPS, 152u * 16u), SORT_WARPS * 32, 0, s>>>(n, start.p, bucket.p, ucount.p,
                                                                                  big.p, nbig.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaFuncSetAttribute(k_sort_rows_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               BLOCK_SORT_MAX * (int)sizeof(uint64_t)));
  k_sort_rows_block<<<152, 256, BLOCK_SORT_MAX * sizeof(uint64_t), s>>>(big.p, nbig.p, start.p, bucket.p,
                                                                        ucount.p, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(dalloc_n(&S->rowptr, n + 1, s));
  int64_t nnz = 0;
  ZI_CHECK(exclusive_scan_i32(ucount.p, S->rowptr, n, &nnz, s));
  ZI_CHECK(read_err(err.p, s));
  S->nnz = nnz;
  ZI_CHECK(dalloc_n(&S->colind, nnz, s));
  ZI_CHECK(dalloc_n(&S->seg, nnz + 1, s));
  ZI_CHECK(dalloc_n(&S->diagpos, n, s));
  ZI_CHECK(dalloc_n(&S->perm, E, s));
  ZI_CHECK(dalloc_n(&S->vals, nnz, s));
  ZI_CUDA(cudaMemsetAsync(S->diagpos, 0xff, sizeof(int32_t) * n, s));
  k_emit_pattern<<<grid_for(n * 32, 256, 152u * 64u), 256, 0, s>>>(n, start.p, bucket.p, S->rowptr, S->colind,
                                                                  S->seg, S->diagpos, S->perm);
  ZI_LAUNCH_CHECK();
  int32_t Ei = (int32_t)E;
  ZI_CUDA(cudaMemcpyAsync(S->seg + nnz, &Ei, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ZI_CUDA(cudaStreamSynchronize(s));  // Ei lives on this stack frame

  ZI_CHECK(assemble_values(S, sigma6, s));

  // nodes with a nonzero B row (CEM): the rows B^T T needs
  if (cem) {
    DevTmp<int32_t> flag, off;
    ZI_CHECK(flag.alloc(n, s));
    ZI_CHECK(off.alloc(n + 1, s));
    k_nonzero_rows<<<grid_for(n, 256), 256, 0, s>>>(n, S->B, S->n_rhs, flag.p);
    ZI_LAUNCH_CHECK();
    int64_t np_ = 0;
    ZI_CHECK(exclusive_scan_i32(flag.p, off.p, n, &np_, s));
    ZI_CHECK(dalloc_n(&S->patch_nodes, np_, s));
    k_compact<<<grid_for(n, 256), 256, 0, s>>>(n, flag.p, off.p, S->patch_nodes);
    ZI_LAUNCH_CHECK();
    S->n_patch_nodes = np_;
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}

}  // namespace zi

using namespace zi;

extern "C" int zi_assemble(const double* nodes, int64_t n, const int32_t* tets, int64_t m, const double* sigma6,
                           const int32_t* bfaces, int64_t nb, const zi_electrodes* el, zi_system** sys,
                           cudaStream_t s) {
  if (!sys) return set_error(ZI_ERR_ARG, "null output handle");
  *sys = nullptr;
  if (!nodes || !tets || !sigma6 || !bfaces || !el) return set_error(ZI_ERR_ARG, "null input array");
  if (n < 4 || m < 1 || nb < 4) return set_error(ZI_ERR_ARG, "mesh too small (n=%lld m=%lld nb=%lld)",
                                                 (long long)n, (long long)m, (long long)nb);
  if (n > INT32_MAX - 1 || m > INT32_MAX / 16 || 16 * m + 9 * nb > INT32_MAX)
    return set_error(ZI_ERR_ARG, "mesh too large for int32 entry ids");
  if (el->n < 2 || el->n > 4096 || !el->centres) return set_error(ZI_ERR_ARG, "need 2..4096 electrodes with centres");
  if (el->model != ZI_ELECTRODE_POINT && el->model != ZI_ELECTRODE_CEM)
    return set_error(ZI_ERR_ARG, "unknown electrode model %d", el->model);
  if (el->model == ZI_ELECTRODE_CEM && (!el->z || !(el->radius > 0)))
    return set_error(ZI_ERR_ARG, "CEM electrodes need z and a positive radius");
  zi_system* S = new zi_system();
  int st = assemble_impl(nodes, n, tets, m, sigma6, bfaces, nb, el, S, s);
  if (st != ZI_OK) {
    cudaStreamSynchronize(s);
    system_free(S);
    delete S;
    return st;
  }
  *sys = S;
  return ZI_OK;
}

extern "C" int zi_system_set_conductivity(zi_system* S, const double* sigma6, cudaStream_t s) {
  if (!S || !sigma6) return set_error(ZI_ERR_ARG, "null argument");
  ZI_CHECK(assemble_values(S, sigma6, s));
  return ZI_OK;
}

namespace zi {
namespace {
// sigma_e = exp(log_s_e) * base_e, all six tensor entries of element e.
__global__ void k_scale_sigma(int64_t m, const double* __restrict__ base6, const double* __restrict__ log_s,
                              double* __restrict__ out6) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double f = exp(log_s[e]);
    for (int k = 0; k < 6; ++k) out6[6 * e + k] = f * base6[6 * e + k];
  }
}
}  // namespace
}  // namespace zi

extern "C" int zi_system_set_log_conductivity(zi_system* S, const double* sigma_base6, const double* log_s,
                                              cudaStream_t s) {
  if (!S || !sigma_base6 || !log_s) return set_error(ZI_ERR_ARG, "null argument");
  DevTmp<double> s6;
  ZI_CHECK(s6.alloc(6 * (size_t)S->m, s));
  k_scale_sigma<<<grid_for(S->m, 256), 256, 0, s>>>(S->m, sigma_base6, log_s, s6.p);
  ZI_LAUNCH_CHECK();
  ZI_CHECK(assemble_values(S, s6.p, s));
  return ZI_OK;
}

extern "C" int zi_system_get_info(const zi_system* S, zi_system_info* info) {
  if (!S || !info) return set_error(ZI_ERR_ARG, "null argument");
  info->n = S->n;
  info->m = S->m;
  info->nnz = S->nnz;
  info->n_el = S->n_el;
  info->n_rhs = S->n_rhs;
  info->n_rows_L = S->n_rhs;
  info->model = S->model;
  info->ground = S->ground;
  info->n_patch_faces = S->n_patch_faces;
  info->has_T = S->has_T;
  return ZI_OK;
}

extern "C" int zi_system_get_matrix(const zi_system* S, int32_t* rowptr, int32_t* colind, double* values,
                                    double* B, double* C, int32_t* el_nodes, cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (rowptr) ZI_CUDA(cudaMemcpyAsync(rowptr, S->rowptr, sizeof(int32_t) * (S->n + 1), cudaMemcpyDeviceToDevice, s));
  if (colind) ZI_CUDA(cudaMemcpyAsync(colind, S->colind, sizeof(int32_t) * S->nnz, cudaMemcpyDeviceToDevice, s));
  if (values) ZI_CUDA(cudaMemcpyAsync(values, S->vals, sizeof(double) * S->nnz, cudaMemcpyDeviceToDevice, s));
  if (B) ZI_CUDA(cudaMemcpyAsync(B, S->B, sizeof(double) * S->n * S->n_rhs, cudaMemcpyDeviceToDevice, s));
  if (C) {
    if (S->model != ZI_ELECTRODE_CEM) return set_error(ZI_ERR_ARG, "C exists for CEM systems only");
    ZI_CUDA(cudaMemcpyAsync(C, S->C, sizeof(double) * S->n_el, cudaMemcpyDeviceToDevice, s));
  }
  if (el_nodes) {
    if (S->model != ZI_ELECTRODE_POINT) return set_error(ZI_ERR_ARG, "electrode nodes exist for point systems only");
    ZI_CUDA(cudaMemcpyAsync(el_nodes, S->el_nodes, sizeof(int32_t) * S->n_el, cudaMemcpyDeviceToDevice, s));
  }
  ZI_CUDA(cudaStreamSynchronize(s));
  return ZI_OK;
}

extern "C" void zi_system_destroy(zi_system* S) {
  if (!S) return;
  cudaDeviceSynchronize();
  solver_scratch_free(S);
  system_free(S);
  cudaDeviceSynchronize();
  delete S;
}
