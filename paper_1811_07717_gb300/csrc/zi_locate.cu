// Point location on any tetrahedral mesh (the source positions of Sec. 2.5
// placed in the elements that hold them), and the lead field of dipoles given
// by position.
//
// The element holding point x is the one whose smallest barycentric
// coordinate at x is largest (ties to the lowest element index); x lies in
// the mesh when that coordinate is >= -ZI_LOCATE_TOL.  Barycentric
// coordinates come from 3x3 determinants of vertex differences in FP64:
//   D = det(x1-x0, x2-x0, x3-x0), l1 = det(x-x0, x2-x0, x3-x0) / D,
//   l2 = det(x1-x0, x-x0, x3-x0) / D, l3 = det(x1-x0, x2-x0, x-x0) / D,
//   l0 = 1 - l1 - l2 - l3.
// Candidates come from a uniform grid of cells over the nodes' bounding box:
// every element is listed in each cell its bounding box overlaps, and a point
// tests the elements of its own cell.  The selection (largest score, then
// lowest index) does not depend on the order of a cell's list, so the result
// is deterministic although the lists are filled with integer atomics.
#include <math.h>
#include <string.h>

#include "zi_internal.cuh"

namespace zi {
namespace {

constexpr double LOCATE_TOL = 1e-10;
constexpr int64_t LOCATE_MAX_CELLS = 1 << 24;

struct CellGrid {
  double lo[3];
  double inv_h;
  int dim[3];
};

// Order-preserving map of a double to an unsigned 64-bit key (for atomic
// min / max of coordinates).
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
inline double dkey_inv(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double v;
  memcpy(&v, &b, sizeof(v));
  return v;
}

// bounds[0..2] = min keys, bounds[3..5] = max keys: per-thread extremes,
// combined in shared memory, one update per block.
__global__ void __launch_bounds__(256) k_node_bounds(int64_t n, const double* __restrict__ nodes,
                                                     unsigned long long* __restrict__ bounds,
                                                     int* __restrict__ err) {
  __shared__ unsigned long long sk[6][256];
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      const double x = nodes[3 * i + d];
      if (!isfinite(x)) {
        atomicOr(err, DEV_ERR_NONFINITE);
        continue;
      }
      lo[d] = min(lo[d], dkey(x));
      hi[d] = max(hi[d], dkey(x));
    }
  }
  for (int d = 0; d < 3; ++d) {
    sk[d][threadIdx.x] = lo[d];
    sk[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int d = 0; d < 3; ++d) {
        sk[d][threadIdx.x] = min(sk[d][threadIdx.x], sk[d][threadIdx.x + w]);
        sk[3 + d][threadIdx.x] = max(sk[3 + d][threadIdx.x], sk[3 + d][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 3; ++d) {
      atomicMin(bounds + d, sk[d][0]);
      atomicMax(bounds + 3 + d, sk[3 + d][0]);
    }
}

__device__ __forceinline__ int cell_coord(const CellGrid& g, int d, double x) {
  const double f = floor((x - g.lo[d]) * g.inv_h);
  return f < 0.0 ? 0 : (f >= (double)g.dim[d] ? g.dim[d] - 1 : (int)f);
}

// Cell range of element e's bounding box; false for a vertex index outside the mesh.
__device__ __forceinline__ bool elem_cells(const CellGrid& g, int64_t n, const double* nodes, const int32_t* tets,
                                           int64_t e, int (&c0)[3], int (&c1)[3]) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int a = 0; a < 4; ++a) {
    const int32_t v = tets[4 * e + a];
    if (v < 0 || v >= n) return false;
    for (int d = 0; d < 3; ++d) {
      const double x = nodes[3 * (int64_t)v + d];
      lo[d] = fmin(lo[d], x);
      hi[d] = fmax(hi[d], x);
    }
  }
  for (int d = 0; d < 3; ++d) {
    c0[d] = cell_coord(g, d, lo[d]);
    c1[d] = cell_coord(g, d, hi[d]);
  }
  return true;
}

__global__ void k_cell_count(CellGrid g, int64_t n, const double* __restrict__ nodes, int64_t m,
                             const int32_t* __restrict__ tets, int32_t* __restrict__ cnt, int* __restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int c0[3], c1[3];
    if (!elem_cells(g, n, nodes, tets, e, c0, c1)) {
      atomicOr(err, DEV_ERR_BAD_INDEX);
      continue;
    }
    for (int i = c0[0]; i <= c1[0]; ++i)
      for (int j = c0[1]; j <= c1[1]; ++j)
        for (int k = c0[2]; k <= c1[2]; ++k) atomicAdd(cnt + ((int64_t)i * g.dim[1] + j) * g.dim[2] + k, 1);
  }
}

__global__ void k_cell_fill(CellGrid g, int64_t n, const double* __restrict__ nodes, int64_t m,
                            const int32_t* __restrict__ tets, const int32_t* __restrict__ off,
                            int32_t* __restrict__ cur, int32_t* __restrict__ list) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int c0[3], c1[3];
    if (!elem_cells(g, n, nodes, tets, e, c0, c1)) continue;
    for (int i = c0[0]; i <= c1[0]; ++i)
      for (int j = c0[1]; j <= c1[1]; ++j)
        for (int k = c0[2]; k <= c1[2]; ++k) {
          const int64_t c = ((int64_t)i * g.dim[1] + j) * g.dim[2] + k;
          list[off[c] + atomicAdd(cur + c, 1)] = (int32_t)e;
        }
  }
}

__device__ __forceinline__ double det3(double ax, double ay, double az, double bx, double by, double bz, double cx,
                                       double cy, double cz) {
  return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
}

// Smallest barycentric coordinate of point (px, py, pz) in element e.
__device__ __forceinline__ double min_bary(const double* nodes, const int32_t* tets, int64_t e, double px, double py,
                                           double pz) {
  const int32_t* t = tets + 4 * e;
  const double* x0 = nodes + 3 * (int64_t)t[0];
  const double* x1 = nodes + 3 * (int64_t)t[1];
  const double* x2 = nodes + 3 * (int64_t)t[2];
  const double* x3 = nodes + 3 * (int64_t)t[3];
  const double ax = x1[0] - x0[0], ay = x1[1] - x0[1], az = x1[2] - x0[2];
  const double bx = x2[0] - x0[0], by = x2[1] - x0[1], bz = x2[2] - x0[2];
  const double cx = x3[0] - x0[0], cy = x3[1] - x0[1], cz = x3[2] - x0[2];
  const double qx = px - x0[0], qy = py - x0[1], qz = pz - x0[2];
  const double D = det3(ax, ay, az, bx, by, bz, cx, cy, cz);
  if (!(D != 0.0)) return -INFINITY;
  const double l1 = det3(qx, qy, qz, bx, by, bz, cx, cy, cz) / D;
  const double l2 = det3(ax, ay, az, qx, qy, qz, cx, cy, cz) / D;
  const double l3 = det3(ax, ay, az, bx, by, bz, qx, qy, qz) / D;
  const double l0 = 1.0 - l1 - l2 - l3;
  return fmin(fmin(l0, l1), fmin(l2, l3));
}

__global__ void k_locate_points(CellGrid g, const double* __restrict__ nodes, const int32_t* __restrict__ tets,
                                const int32_t* __restrict__ off, const int32_t* __restrict__ list, int64_t P,
                                const double* __restrict__ pos, int32_t* __restrict__ out, int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const double px = pos[3 * p], py = pos[3 * p + 1], pz = pos[3 * p + 2];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) {
      atomicOr(err, DEV_ERR_NONFINITE);
      out[p] = -1;
      continue;
    }
    const int64_t c = ((int64_t)cell_coord(g, 0, px) * g.dim[1] + cell_coord(g, 1, py)) * g.dim[2] +
                      cell_coord(g, 2, pz);
    double best = -INFINITY;
    int32_t be = -1;
    for (int32_t k = off[c]; k < off[c + 1]; ++k) {
      const int32_t e = list[k];
      const double s = min_bary(nodes, tets, e, px, py, pz);
      if (s > best || (s == best && e < be)) {
        best = s;
        be = e;
      }
    }
    if (be < 0 || !(best >= -LOCATE_TOL)) {
      atomicOr(err, DEV_ERR_OUTSIDE);
      be = -1;
    }
    out[p] = be;
  }
}

}  // namespace

int locate_points(const double* nodes, int64_t n, const int32_t* tets, int64_t m, const double* pos, int64_t P,
                  int32_t* out, cudaStream_t s) {
  if (n < 4 || m < 1 || m > INT32_MAX) return set_error(ZI_ERR_ARG, "need a mesh of at least one element");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative point count");
  if (!nodes || !tets || (P > 0 && (!pos || !out))) return set_error(ZI_ERR_ARG, "null mesh, point or output array");
  if (P == 0) return ZI_OK;
  DevTmp<unsigned long long> bounds;
  DevTmp<int> err;
  ZI_CHECK(bounds.alloc(6, s));
  ZI_CHECK(err.alloc(1, s));
  ZI_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  ZI_CUDA(cudaMemsetAsync(bounds.p, 0xff, 3 * sizeof(unsigned long long), s));
  ZI_CUDA(cudaMemsetAsync(bounds.p + 3, 0, 3 * sizeof(unsigned long long), s));
  k_node_bounds<<<grid_for(n, 256), 256, 0, s>>>(n, nodes, bounds.p, err.p);
  ZI_LAUNCH_CHECK();
  unsigned long long hb[6];
  int herr = 0;
  ZI_CUDA(cudaMemcpyAsync(hb, bounds.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  CellGrid g;
  double ext[3], vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    g.lo[d] = dkey_inv(hb[d]);
    ext[d] = dkey_inv(hb[3 + d]) - g.lo[d];
    vol *= ext[d] > 0 ? ext[d] : 1.0;
  }
  // about two elements per cell
  double h = cbrt(2.0 * vol / (double)m);
  if (!(h > 0) || !isfinite(h)) h = 1.0;
  for (;;) {
    int64_t cells = 1;
    for (int d = 0; d < 3; ++d) {
      const double q = ceil(ext[d] / h);
      g.dim[d] = q < 1 ? 1 : (int)fmin(q, 4096.0);
      cells *= g.dim[d];
    }
    if (cells <= LOCATE_MAX_CELLS) break;
    h *= 1.25;
  }
  g.inv_h = 1.0 / h;
  const int64_t ncell = (int64_t)g.dim[0] * g.dim[1] * g.dim[2];
  DevTmp<int32_t> cnt, off, list;
  ZI_CHECK(cnt.alloc(ncell, s));
  ZI_CHECK(off.alloc(ncell + 1, s));
  ZI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * ncell, s));
  k_cell_count<<<grid_for(m, 256), 256, 0, s>>>(g, n, nodes, m, tets, cnt.p, err.p);
  ZI_LAUNCH_CHECK();
  int64_t total = 0;
  ZI_CHECK(exclusive_scan_i32(cnt.p, off.p, ncell, &total, s));
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  ZI_CHECK(device_error_to_status(herr));
  ZI_CHECK(list.alloc(total, s));
  ZI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * ncell, s));  // reused as the fill cursor
  k_cell_fill<<<grid_for(m, 256), 256, 0, s>>>(g, n, nodes, m, tets, off.p, cnt.p, list.p);
  ZI_LAUNCH_CHECK();
  k_locate_points<<<grid_for(P, 128), 128, 0, s>>>(g, nodes, tets, off.p, list.p, P, pos, out, err.p);
  ZI_LAUNCH_CHECK();
  ZI_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  ZI_CUDA(cudaStreamSynchronize(s));
  return device_error_to_status(herr);
}

}  // namespace zi

using namespace zi;

extern "C" int zi_locate_points(const double* nodes, int64_t n, const int32_t* tets, int64_t m, const double* pos,
                                int64_t P, int32_t* tet_out, cudaStream_t s) {
  return locate_points(nodes, n, tets, m, pos, P, tet_out, s);
}

extern "C" int zi_leadfield_at(zi_system* S, const double* pos, int64_t P, const zi_solver_opts* o, double* L,
                               cudaStream_t s) {
  if (!S) return set_error(ZI_ERR_ARG, "null system");
  if (P < 0) return set_error(ZI_ERR_ARG, "negative dipole count");
  if (P > 0 && (!pos || !L)) return set_error(ZI_ERR_ARG, "null dipole or output array");
  DevTmp<int32_t> tet;
  if (P > 0) {
    ZI_CHECK(tet.alloc(P, s));
    ZI_CHECK(locate_points(S->nodes, S->n, S->tets, S->m, pos, P, tet.p, s));
  }
  return zi_leadfield(S, tet.p, P, o, L, s);
}
