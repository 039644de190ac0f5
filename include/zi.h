/*
 * zi.h -- C ABI of libzi, a GB300 (sm_103a) implementation of the finite-element
 * lead-field (LF) build of the Zeffiro Interface paper (arXiv 1811.07717):
 * tetrahedral P1 stiffness assembly with per-element conductivity tensors,
 * complete-electrode-model (CEM) terms, the transfer matrix T = A^-1 B by
 * multi-right-hand-side preconditioned conjugate gradients, the EEG lead field
 * L = R (C - B^T T)^-1 T^T F and the linearised-EIT Jacobian.
 *
 * Conventions for every entry point
 *   - Plain C: no exceptions cross this boundary; every call returns a zi_status
 *     (0 = ZI_OK).  zi_last_error() gives the message of the last failure of the
 *     calling thread.
 *   - Arrays are row-major, indices are 0-based int32, sizes int64.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary host memory.  The caller owns every buffer it
 *     passes; outputs are written, never reallocated.  A zi_system handle owns
 *     only library-internal memory and is released by zi_system_destroy().
 *   - Every call that launches GPU work takes a cudaStream_t (0 = legacy default
 *     stream) and is stream-ordered: device outputs are valid once that stream
 *     reaches the point of the call.  Calls that return a size or a status read
 *     back from the device synchronise the stream before returning.
 *   - Units: SI (m, S/m, Ohm*m^2).  Any consistent length unit works for the
 *     mesh calls; conductivity and contact impedance scale as usual.
 *
 * Error behaviour: ZI_ERR_ARG for null pointers, negative or inconsistent sizes
 * and unsupported options; ZI_ERR_BAD_MESH for a non-positive element volume, an
 * electrode with no surface patch, overlapping patches, two point electrodes on
 * one node or a dipole outside the mesh; ZI_ERR_NONFINITE for NaN/Inf inputs;
 * ZI_ERR_NOT_CONVERGED when a column misses its tolerance within maxit (outputs
 * are still written; per-column iteration counts and residuals say which);
 * ZI_ERR_TIMEOUT when a device-side wait exceeded its bound; ZI_ERR_CUDA for a
 * CUDA runtime failure; ZI_ERR_NOMEM when device memory runs out.
 */
#ifndef ZI_H
#define ZI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#ifndef __CUDA_RUNTIME_H__
typedef struct CUstream_st* cudaStream_t;
#endif

typedef enum zi_status {
  ZI_OK = 0,
  ZI_ERR_ARG = 1,
  ZI_ERR_BAD_MESH = 2,
  ZI_ERR_NONFINITE = 3,
  ZI_ERR_NOT_CONVERGED = 4,
  ZI_ERR_TIMEOUT = 5,
  ZI_ERR_CUDA = 6,
  ZI_ERR_NOMEM = 7
} zi_status;

/* Electrode models. */
enum { ZI_ELECTRODE_POINT = 0, ZI_ELECTRODE_CEM = 1 };
/* Diagonal preconditioners (Sec. 2.3.1): Jacobi 1/a_ii, or the paper's lumped
 * diagonal preconditioner 1/sum_j |a_ij|. */
enum { ZI_PRECOND_JACOBI = 0, ZI_PRECOND_LDP = 1 };
/* Solver precision: FP64 throughout, or FP32 inner PCG inside FP64 iterative
 * refinement (FP64 residual b - A x and solution update).  The FP32 solve
 * works on the unscaled matrix in difference form, c_i p_i + sum_j a_ij
 * (p_j - p_i) with c_i the row sum, which avoids the cancellation of the plain
 * stencil on smooth vectors; it stores its search directions and residuals in
 * FP16 (round to nearest, saturating) and computes in FP32, with x and A p in
 * FP32.  The FP64 refinement decides the accuracy in both precisions.  Both
 * omit couplings at assembly rounding level (|a_ij| <= 2^-40 sqrt(a_ii a_jj);
 * FP32: <= 2^-24). */
enum { ZI_FP64 = 0, ZI_MIXED = 1 };
/* EIT output modes. */
enum { ZI_EIT_FULL = 0, ZI_EIT_VJP = 1 };
/* IAS hypermodels (App. B): gamma (G) and inverse gamma (IG). */
enum { ZI_HYPER_G = 0, ZI_HYPER_IG = 1 };

typedef struct zi_system zi_system;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int zi_version(void);

/* Copies the message of the calling thread's last error (NUL-terminated,
 * truncated to len) into buf; returns the status of that error. */
int zi_last_error(char* buf, size_t len);

/* Short name of a status code ("ZI_OK", ...). Static storage. */
const char* zi_status_string(int status);

/* ------------------------------------------------------------------------ */
/* Mesh (stand-in for the paper's mesh tool, Sec. 2.5; the mesh fields are    */
/* the zef.nodes / zef.tetra arrays of Sec. 2.5)                              */
/* ------------------------------------------------------------------------ */

/* Regular-grid Kuhn mesh of the ball r < radii[n_shells-1].
 *   Grid indices run over [-N, N] per axis, N = ceil(R_out/h) + 1.  Cube
 *   (i,j,k) spans [i,i+1]h x [j,j+1]h x [k,k+1]h and is kept when
 *   (2i+1)^2 + (2j+1)^2 + (2k+1)^2 < (2R_out/h)^2 (its centre is inside); its
 *   label is the first shell s with the same test against radii[s] true.
 *   Nodes: corners of kept cubes, ordered by grid linear index; coordinates
 *   (i*h, j*h, k*h) in FP64.  Tets: kept cubes in grid order, six Kuhn tets per
 *   cube for the axis permutations in lexicographic order, path
 *   v0 -> v0+e_a -> v0+e_a+e_b -> v0+(1,1,1), last two vertices swapped when
 *   that path is negatively oriented.  Boundary faces: faces of exactly one
 *   tet, in (tet, local face) order, outward vertex order
 *   (1,2,3), (0,3,2), (0,1,3), (0,2,1) for local faces 0..3.
 * Arguments:
 *   h > 0, n_shells >= 1, radii: host, n_shells ascending positive values.
 *   n_nodes, n_tets, n_bfaces: host out, always written.
 *   nodes (n x 3 f64), tets (m x 4 i32), labels (m i32), bfaces (nb x 3 i32):
 *   device out.  Pass all four as NULL to query the sizes only (two-call
 *   pattern); otherwise all four must be non-NULL and sized from the query.
 * Synchronises the stream (sizes are read back). */
int zi_mesh_from_grid(double h, int n_shells, const double* radii,
                      int64_t* n_nodes, int64_t* n_tets, int64_t* n_bfaces,
                      double* nodes, int32_t* tets, int32_t* labels, int32_t* bfaces,
                      cudaStream_t stream);

/* Mesh from a surface segmentation (Sec. 2.5, mesh tool): the Kuhn grid of
 * zi_mesh_from_grid over [-N h, N h]^3, N = ceil(max |vertex coordinate| / h) + 1,
 * labelled from closed, outward-oriented triangle surfaces, one per
 * compartment, innermost first.
 *   node label: the first surface whose winding number at the node is >= 1/2
 *     (the sum of its triangles' solid angles over 4 pi, Van Oosterom-Strackee);
 *   tet label: among its four node labels, the compartment with the lowest
 *     priority value (ties to the inner compartment); a tet with no node
 *     inside any surface is dropped;
 *   nodes (vertices of kept tets) in grid order, tets in (cube, permutation)
 *   order, positively oriented; bfaces: faces of exactly one kept tet, in
 *   (tet, local face) order, outward.
 *   tri_offset: host, n_surf + 1 i64, triangles of surface c are
 *     tri_offset[c] .. tri_offset[c+1] - 1 (tri_offset[0] = 0, each non-empty);
 *   priority: host, n_surf i32; verts: device nv x 3 f64; tris: device nt x 3
 *     i32 indices into verts.  1 <= n_surf <= 64, N <= 301.
 * Two calls: first with the four outputs NULL to get the counts, then with
 * all four allocated from them and *n_nodes, *n_tets, *n_bfaces still holding
 * those counts (the call checks them before writing).  ZI_ERR_NONFINITE for a
 * non-finite vertex, ZI_ERR_ARG for a triangle index outside verts.  A node
 * lying on a surface gets the winding number's rounding (about 1/2): keep
 * surfaces off the grid nodes where labels must be exact.  Synchronises. */
int zi_mesh_from_surfaces(double h, int n_surf, const int64_t* tri_offset, const int32_t* priority,
                          const double* verts, int64_t nv, const int32_t* tris,
                          int64_t* n_nodes, int64_t* n_tets, int64_t* n_bfaces,
                          double* nodes, int32_t* tets, int32_t* labels, int32_t* bfaces,
                          cudaStream_t stream);

/* Source interpolation (Sec. 2.5's index array linking mesh nodes to DOFs;
 * Sec. 3.2's grouping of DOFs around random centres): out[i] = the index of the
 * source nearest to point i, ties to the lowest index, distances compared as
 * FP64 (dx*dx + dy*dy) + dz*dz with every operation rounded once.
 *   points: device n x 3 f64; sources: device P x 3 f64 (1 <= P < 2^31);
 *   out: device n i32.  ZI_ERR_NONFINITE for a non-finite coordinate.
 * Synchronises. */
int zi_nearest_source(const double* points, int64_t n, const double* sources, int64_t P, int32_t* out,
                      cudaStream_t stream);

/* Element of any tetrahedral mesh that holds each point (Sec. 2.5: source
 * positions placed in the mesh): the element whose smallest barycentric
 * coordinate at the point is largest, ties to the lowest element index; the
 * point lies in the mesh when that coordinate is >= -1e-10.  Barycentric
 * coordinates in FP64 from 3x3 determinants of vertex differences:
 * D = det(x1-x0, x2-x0, x3-x0), l1 = det(x-x0, x2-x0, x3-x0)/D,
 * l2 = det(x1-x0, x-x0, x3-x0)/D, l3 = det(x1-x0, x2-x0, x-x0)/D,
 * l0 = 1 - l1 - l2 - l3.  Candidates come from a uniform grid of cells over
 * the nodes' bounding box (each element listed in every cell its bounding box
 * overlaps); the result does not depend on the order of those lists.
 *   nodes: device n x 3 f64; tets: device m x 4 i32; pos: device P x 3 f64;
 *   tet_out: device out, P i32 (-1 for a point outside the mesh).
 * ZI_ERR_BAD_MESH if a point lies outside the mesh, ZI_ERR_NONFINITE for a
 * non-finite coordinate, ZI_ERR_ARG for an element vertex outside the nodes.
 * Synchronises. */
int zi_locate_points(const double* nodes, int64_t n, const int32_t* tets, int64_t m,
                     const double* pos, int64_t P, int32_t* tet_out, cudaStream_t stream);

/* Element of a zi_mesh_from_grid mesh (same h, radii) that holds each point:
 * cube = floor(x/h) per axis, then the Kuhn tet whose axis order sorts the
 * fractional coordinates in descending order (first permutation on ties).
 *   pos: device P x 3 f64.  dip_tet: device out, P i32.
 * Returns ZI_ERR_BAD_MESH if a point lies in no kept cube (synchronises). */
int zi_locate_dipoles_grid(double h, int n_shells, const double* radii,
                           const double* pos, int64_t P, int32_t* dip_tet,
                           cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Assembly (App. A.1)                                                        */
/* ------------------------------------------------------------------------ */

typedef struct zi_electrodes {
  int32_t model;          /* ZI_ELECTRODE_POINT or ZI_ELECTRODE_CEM */
  int32_t n;              /* number of electrodes L >= 2 */
  const double* centres;  /* device, L x 3: electrode centre points */
  const double* z;        /* device, L: CEM contact impedance z_l = Z_l*|e_l| (Ohm m^2); NULL for point */
  double radius;          /* CEM: boundary triangles whose centroid is within this distance of a centre */
} zi_electrodes;

/* Builds the grounded FEM system of one head:
 *   A = sum_e K_e + sum_l 1/z_l int_{e_l} psi_i psi_j   (App. A.1, a_ij),
 *   K_e = vol_e grad(lambda)^T Sigma_e grad(lambda), Sigma_e from the 6-tuple
 *   (s11, s22, s33, s12, s13, s23) of element e (Sec. 2.1.2), on the mesh-graph
 *   CSR pattern, summed in a fixed order (no floating-point atomics);
 *   CEM: b_il = 1/z_l int psi_i, c_ll = |e_l|/z_l; grounding node i' = the
 *   lowest-index boundary node outside every patch, row and column i' of A
 *   zeroed with a_i'i' = 1 (App. A.1).
 *   Point electrodes: electrode l sits on the boundary node nearest its centre
 *   (lowest index on ties); i' = electrode 0's node, and the L-1 right-hand
 *   sides are the unit vectors of electrodes 1..L-1 (electrode 0 is the
 *   reference).
 * Arguments: nodes device n x 3; tets device m x 4; sigma6 device m x 6;
 *   bfaces device nb x 3 (boundary faces as from zi_mesh_from_grid); el host
 *   struct with device arrays.  *sys receives a new handle (caller destroys).
 *   The handle keeps its own copies of nodes and tets.
 * Synchronises the stream. */
int zi_assemble(const double* nodes, int64_t n, const int32_t* tets, int64_t m,
                const double* sigma6, const int32_t* bfaces, int64_t nb,
                const zi_electrodes* el, zi_system** sys, cudaStream_t stream);

/* Re-assembles the values of A for new element conductivities (same mesh,
 * electrodes and pattern); invalidates a previously computed T. */
int zi_system_set_conductivity(zi_system* sys, const double* sigma6, cudaStream_t stream);

/* The same for the log-conductivity parametrisation of the linearised EIT
 * (App. A.3): element e's tensor is exp(log_s[e]) times its base tensor,
 * formed on the device (sigma_base6: device m x 6 f64; log_s: device m f64). */
int zi_system_set_log_conductivity(zi_system* sys, const double* sigma_base6, const double* log_s,
                                   cudaStream_t stream);

typedef struct zi_system_info {
  int64_t n;          /* nodes */
  int64_t m;          /* tets */
  int64_t nnz;        /* CSR nonzeros of A (mesh-graph pattern) */
  int32_t n_el;       /* electrodes L */
  int32_t n_rhs;      /* right-hand sides / columns of T: L (CEM) or L-1 (point) */
  int32_t n_rows_L;   /* rows of the lead field: L (CEM) or L-1 (point) */
  int32_t model;      /* electrode model */
  int64_t ground;     /* grounding node i' */
  int64_t n_patch_faces; /* CEM boundary triangles under electrodes */
  int32_t has_T;      /* 1 once zi_transfer has run for the current values */
} zi_system_info;

int zi_system_get_info(const zi_system* sys, zi_system_info* info);

/* Copies the grounded CSR matrix A (rowptr n+1, colind nnz, values nnz; device
 * out, any may be NULL), the right-hand sides B (device n x n_rhs, NULL to
 * skip), C (device L, CEM only, NULL to skip) and the electrode node of each
 * point electrode (device L i32, point model only, NULL to skip). */
int zi_system_get_matrix(const zi_system* sys, int32_t* rowptr, int32_t* colind, double* values,
                         double* B, double* C, int32_t* el_nodes, cudaStream_t stream);

void zi_system_destroy(zi_system* sys);

/* ------------------------------------------------------------------------ */
/* Transfer matrix (App. A.4) by multi-RHS PCG (Sec. 2.3.1)                    */
/* ------------------------------------------------------------------------ */

typedef struct zi_solver_opts {
  double tol;         /* stop column c when ||b_c - A t_c||_2 <= tol ||b_c||_2 (true FP64 residual) */
  int32_t maxit;      /* bound on inner CG iterations in total per solve */
  int32_t precond;    /* ZI_PRECOND_JACOBI or ZI_PRECOND_LDP */
  int32_t precision;  /* ZI_FP64 or ZI_MIXED */
  double inner_tol;   /* ZI_MIXED: FP32 residual reduction between FP64 reliable updates (0 = default 0.05) */
  int32_t max_outer;  /* ZI_MIXED: bound on refinement steps (0 = default 30) */
  int32_t check_every;/* iterations between convergence read-backs (0 = default) */
} zi_solver_opts;

/* Fills opts with the defaults: tol 1e-10, maxit 100000, Jacobi, FP64. */
void zi_solver_opts_default(zi_solver_opts* opts);

/* T = A^-1 B: one preconditioned CG recurrence per right-hand side, all
 * columns sharing each sparse matrix product.  The handle keeps T for
 * zi_leadfield / zi_eit_*.
 *   T: device out, n x n_rhs f64 (NULL: keep it in the handle only).
 *   iters (n_rhs i32) and relres (n_rhs f64): host out, may be NULL; relres is
 *   the true relative residual recomputed in FP64 after the solve.
 * Returns ZI_ERR_NOT_CONVERGED if any column misses tol. Synchronises. */
int zi_transfer(zi_system* sys, const zi_solver_opts* opts, double* T,
                int32_t* iters, double* relres, cudaStream_t stream);

/* Batched transfer: the systems of nb heads (any sizes, any electrode counts)
 * solved in the schedule of zi_batch_tune (tuned on the first call of a batch
 * signature, cached after): the heads of its persistent set together in one
 * persistent launch per iteration chunk, replayed as a CUDA graph, the others
 * on their own iteration graphs.  T[b] may be NULL.  Per-head iteration counts
 * go to iters[b] (host arrays of n_rhs each, may be NULL). */
int zi_transfer_batched(zi_system* const* sys, int nb, const zi_solver_opts* opts,
                        double* const* T, int32_t* const* iters, cudaStream_t stream);

/* The batch schedule chosen by the library's autotuner for zi_transfer_batched.
 * Heads of the persistent set are solved together in one cooperative launch
 * per chunk of 16 iterations (replayed from a CUDA graph); the others one after
 * another on their own captured iteration graphs (zi_transfer's path).  The
 * tuner ranks the heads by per-iteration work (nodes x padded right-hand
 * sides) and times, from every head's initial state, a window of the solve
 * (the first CG phase, at most 64 iterations): every head alone, and the
 * persistent launch of the k smallest heads for k in {2, nb/4, nb/2, 3nb/4, nb};
 * it keeps the k with the least estimated window time of the whole batch,
 * t(k smallest together) + sum of the other heads' times alone (k = 0: every
 * head alone).  The result is cached per batch signature (device, precision,
 * preconditioner, each head's n, nnz and n_rhs in call order): only the first
 * call of a signature pays for the timing.  Every head is reset to its
 * initial state afterwards; T is untouched. */
enum { ZI_BATCH_TUNED = 1, ZI_BATCH_CACHED = 2 };

typedef struct zi_batch_schedule {
  int32_t source;                         /* ZI_BATCH_TUNED (timed in this call) or ZI_BATCH_CACHED */
  double est_window_ms;            /* estimated ms of the tuning window: the chosen schedule */
  double est_window_ms_per_head;   /* every head alone */
  double est_window_ms_persistent; /* every head in the persistent launch */
} zi_batch_schedule;

/* Runs (or looks up) the autotuner: persistent (host out, nb i32) gets 1 for the
 * heads of the persistent launch.  info (host out) may be NULL.  Synchronises. */
int zi_batch_tune(zi_system* const* sys, int nb, const zi_solver_opts* opts, int32_t* persistent,
                  zi_batch_schedule* info, cudaStream_t stream);

/* zi_transfer_batched with a given schedule: persistent (host in, nb i32) marks
 * the heads of the persistent launch; chunk = iterations per launch (0: opts'
 * check_every, else 25).  Results are bitwise reproducible for a fixed
 * schedule. */
int zi_transfer_batched_schedule(zi_system* const* sys, int nb, const zi_solver_opts* opts, double* const* T,
                                 int32_t* const* iters, const int32_t* persistent, int chunk,
                                 cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Lead field (App. A.2, Eq. aku)                                              */
/* ------------------------------------------------------------------------ */

/* L for dipoles at tets dip_tet (device P i32, from zi_locate_dipoles_grid or
 * the caller's own point location), three Cartesian orientations each, columns
 * 3p + d (Sec. 2.5 ordering).  Partial-integration source model: the load of
 * dipole q in tet e is f_i = q . grad psi_i on e's four nodes (the paper's
 * G = -F).  CEM: L = R (C - B^T T)^-1 T^T F, L rows average-referenced
 * (r_jj = 1 - 1/L, r_ij = -1/L); point electrodes: L = T^T F, rows for
 * electrodes 1..L-1 referenced to electrode 0.
 *   L: device out, n_rows_L x 3P f64.  Runs zi_transfer with opts first if
 *   the handle holds no T.  Synchronises. */
int zi_leadfield(zi_system* sys, const int32_t* dip_tet, int64_t P,
                 const zi_solver_opts* opts, double* L, cudaStream_t stream);

/* The same lead field for dipoles given by position (device P x 3 f64): each
 * is placed in its element of the system's own mesh by zi_locate_points, then
 * as zi_leadfield.  ZI_ERR_BAD_MESH if a dipole lies outside the mesh. */
int zi_leadfield_at(zi_system* sys, const double* dip_pos, int64_t P,
                    const zi_solver_opts* opts, double* L, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* H(div) sources (Sec. 2.1, primary current model)                            */
/* ------------------------------------------------------------------------ */

/* Source stencils: the four face functions of the holding tet (Whitney), or
 * those plus its six edge functions (the 10-source stencil). */
enum { ZI_SOURCE_WHITNEY4 = 0, ZI_SOURCE_PBO10 = 1 };
#define ZI_STENCIL_WIDTH 8          /* entries per source-matrix column */
#define ZI_PBO_LAMBDA_DEFAULT 1e-2  /* Tikhonov weight of the PBO fit */

/* Columns of the source matrix F for Cartesian H(div) sources at positions
 * pos (device P x 3 f64, m) in tets dip_tet (device P i32).  Column 3p + j
 * (orientation e_j, Sec. 2.5 ordering) is sum_k w_k f_k over the stencil of
 * tet t = dip_tet[p]:
 *   face source k: the lowest-order Raviart-Thomas function of the face
 *     opposite vertex v_k with unit flux into the neighbour N_k; load
 *     (e_{o_k} - e_{v_k})/4 (o_k: N_k's vertex off the face), moment
 *     (x_{o_k} - x_{v_k})/4 at the face centroid; absent on the mesh boundary;
 *   edge source (a, b) (ZI_SOURCE_PBO10): load e_{v_b} - e_{v_a}, moment
 *     x_{v_b} - x_{v_a} at the edge midpoint.
 * Position-based optimisation: w minimises the first moment of the combined
 * source about x0, |sum_k w_k d_k (c_k - x0)^T / s|_F^2, plus
 * lambda sum_k (1 + |c_k - x0|^2/s^2) |d_k|^2 w_k^2 (s: mean edge length of t),
 * subject to sum_k w_k d_k = e_j (the dipole moment exactly).
 *   lambda: > 0, or 0 for ZI_PBO_LAMBDA_DEFAULT.
 *   F_nodes: device out, 3P x ZI_STENCIL_WIDTH i32: t's four vertices, then
 *     the vertex across each face (t's own vertex where the face is on the
 *     boundary, with weight 0).
 *   F_w: device out, 3P x ZI_STENCIL_WIDTH f64, the loads at those nodes.
 * Feed both to zi_leadfield_sparse.  Scratch: a node -> tet incidence list
 * (4m + n + 1 int32).  ZI_ERR_BAD_MESH for a tet index outside the mesh, a face
 * shared by more than two tets, or a stencil whose moments do not span R^3
 * (a Whitney stencil with two boundary faces); that column's weights are 0.
 * Synchronises. */
int zi_source_stencil(zi_system* sys, const double* pos, const int32_t* dip_tet, int64_t P, int model,
                      double lambda, int32_t* F_nodes, double* F_w, cudaStream_t stream);

/* L for a source matrix F given column by column: column c has the load
 * F_w[c*K + j] at node F_nodes[c*K + j], j < K (repeated nodes add up).
 * L = R (C - B^T T)^-1 T^T F (CEM) or T^T F (point electrodes), as in
 * zi_leadfield, with ncols columns.
 *   F_nodes: device in, ncols x K i32; F_w: device in, ncols x K f64; 1 <= K <= 32.
 *   L: device out, n_rows_L x ncols f64.
 * ZI_ERR_ARG for a node index outside the mesh or a non-finite weight (L is
 * not written).  Runs zi_transfer with opts first if the handle holds no T.
 * Synchronises. */
int zi_leadfield_sparse(zi_system* sys, const int32_t* F_nodes, const double* F_w, int64_t ncols, int K,
                        const zi_solver_opts* opts, double* L, cudaStream_t stream);

/* Partial-integration source columns in the form zi_leadfield_sparse and
 * zi_meg_leadfield take: column 3p + d holds d psi_a / d x_d at the four
 * vertices a of tet dip_tet[p] (the same F as zi_leadfield).
 *   F_nodes: device out, 3P x 4 i32; F_w: device out, 3P x 4 f64.
 * ZI_ERR_BAD_MESH for a tet index outside the mesh.  Synchronises. */
int zi_source_pi(zi_system* sys, const int32_t* dip_tet, int64_t P, int32_t* F_nodes, double* F_w,
                 cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* MEG lead field (App. A.2: the Biot-Savart formula)                          */
/* ------------------------------------------------------------------------ */

/* Magnetometers at sens_pos (device Ns x 3 f64, outside the head) reading the
 * field along unit orientations sens_dir (device Ns x 3 f64).  The field of
 * the total current J^p - sigma grad u (Sec. 2.1) by Biot-Savart is the
 * primary dipole's field plus Bm^T u, with
 *   Bm[i][s] = -mu0/(4 pi) sum_{e containing i} grad psi_i|_e . sigma_e (G_e(r_s) x n_s),
 *   G_e(r) = int_e (r - r')/|r - r'|^3 dV' by the 4-point degree-2 rule
 *   (barycentric points (a, b, b, b), a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20),
 * mu0/(4 pi) = 1e-7 T m/A, row i' (the grounding node) zero.  u solves the
 * system's own A (with whatever electrode terms it was assembled with).
 * sigma6: device m x 6 f64, the conductivity the system was assembled with. */

/* Bm: device out, n x Ns f64.  Bitwise reproducible (per-node sums in tet
 * order).  ZI_ERR_NONFINITE if a sensor sits on a quadrature point.
 * Synchronises. */
int zi_meg_rhs(zi_system* sys, const double* sigma6, const double* sens_pos, const double* sens_dir, int Ns,
               double* Bm, cudaStream_t stream);

/* T_meg = A^-1 Bm, one PCG recurrence per sensor (the solver of zi_transfer,
 * with opts).  T_meg: device out, n x Ns f64; iters (Ns i32) and relres (Ns
 * f64): host out, may be NULL.  The handle's own T is untouched.
 * ZI_ERR_NOT_CONVERGED as in zi_transfer.  Synchronises the device. */
int zi_meg_transfer(zi_system* sys, const double* sigma6, const double* sens_pos, const double* sens_dir, int Ns,
                    const zi_solver_opts* opts, double* T_meg, int32_t* iters, double* relres,
                    cudaStream_t stream);

/* MEG lead field of Cartesian sources: L[s][3p + d] = mu0/(4 pi) e_d . ((r_s -
 * x_p) x n_s) / |r_s - x_p|^3 + (T_meg^T F)[s][3p + d], with F given column by
 * column (3P x K node indices and loads, 1 <= K <= 32: zi_source_pi or
 * zi_source_stencil).  pos: device P x 3 f64; T_meg: device n x Ns f64 from
 * zi_meg_transfer; L: device out, Ns x 3P f64.  ZI_ERR_ARG for a node index
 * outside the mesh or a non-finite weight.  Synchronises. */
int zi_meg_leadfield(zi_system* sys, const double* T_meg, const double* sens_pos, const double* sens_dir, int Ns,
                     const double* pos, int64_t P, const int32_t* F_nodes, const double* F_w, int K, double* L,
                     cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Linearised EIT (App. A.3)                                                   */
/* ------------------------------------------------------------------------ */

/* CEM systems only.  Current patterns I (device np x L f64).  Writes
 *   y (device np x L, may be NULL): y_p = R M^-1 I_p, M = C - B^T A^-1 B;
 *   mode ZI_EIT_FULL: out (device m x np x L): out[m][p][k] = dy_{p,k}/dlog s_m
 *       = -u_p^T K_m w_k, u_p = T M^-1 I_p, w_k = T M^-1 R e_k;
 *   mode ZI_EIT_VJP: out (device m): sum_{p,k} grad_y[p][k] dy_{p,k}/dlog s_m,
 *       grad_y device np x L.
 * Runs zi_transfer with opts first if the handle holds no T. Synchronises. */
int zi_eit_jacobian(zi_system* sys, const double* I, int np, int mode,
                    const double* grad_y, double* out, double* y,
                    const zi_solver_opts* opts, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Lead field without device allocation (no counterpart in the paper)         */
/* ------------------------------------------------------------------------ */

/* Size of the fixed device scratch used by zi_leadfield_noalloc: 8 MiB, of
 * which the first 256 bytes hold an error word and the rest doubles. */
#define ZI_NOALLOC_SCRATCH_BYTES (8u << 20)

/* The same lead field as zi_leadfield, for callers that cannot allocate
 * device memory while it runs: applications that hand the whole GPU to their
 * own allocator up front (a library allocation would fail or fragment it),
 * and code that must not allocate inside a latency-critical loop.  It calls no
 * cudaMalloc, cudaFree or allocating routine; its scratch is one fixed array in
 * the library's device memory (ZI_NOALLOC_SCRATCH_BYTES on every GPU that
 * loads the library, held until the process exits).  Its device address is
 * looked up once per device and kept for the life of the process: this
 * assumes the device's primary context lives as long as the process (after a
 * cudaDeviceReset, or a context destroyed and created again, the kept address
 * is stale; do not call this entry point after either).
 *   The system must already hold T (zi_transfer has run; otherwise ZI_ERR_ARG,
 *   since solving would allocate).  dip_tet: device P i32; L: device out,
 *   n_rows_L x 3P f64, as in zi_leadfield.
 *   Scratch need: 3*P*n_rows_L doubles, plus 2*L*L for CEM systems; a call
 *   needing more than (ZI_NOALLOC_SCRATCH_BYTES - 256) / 8 doubles returns
 *   ZI_ERR_ARG with the limit in the message.
 *   The first call on a device looks up the scratch address
 *   (cudaGetSymbolAddress), so make that first call before any stream capture.
 *   All calls share the one array: calls that overlap on the GPU (other
 *   streams, other threads) race and must be serialised by the caller.
 * Synchronises the stream. */
int zi_leadfield_noalloc(zi_system* sys, const int32_t* dip_tet, int64_t P, double* L,
                         cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* IAS MAP inversion (App. B)                                                  */
/* ------------------------------------------------------------------------ */

/* Iterative alternating sequential MAP estimates for T data vectors, each
 * inverted on its own: theta = theta0 for every source, then `iters` rounds of
 *   x     = D L^T (L D L^T + nu^2 I)^-1 y,   D = diag(theta)   (App. B, Eq. ias_matrix;
 *           the paper's D^{1/2} L_k^T with L_k = L D^{1/2}, theta > 0)
 *   theta = theta0/2 (eta + sqrt(eta^2 + 2 x^2/theta0)), eta = beta - 3/2    (ZI_HYPER_G)
 *         or (theta0 + x^2/2) / (beta + 3/2)                                (ZI_HYPER_IG)
 * elementwise.  L D L^T is an FP64 product over the sources split across the
 * GPU; the Le x Le systems are solved by Cholesky.
 *   L:     device in, Le x n f64 row-major (a lead field, e.g. from zi_leadfield); 1 <= Le <= 256.
 *   Y:     device in, T x Le f64 (data vector t in row t).
 *   X:     device out, T x n f64 (the estimate of data vector t in row t).
 *   Theta: device out, T x n f64 (the final hyperparameters).
 * nu > 0 (noise standard deviation), theta0 > 0; IG needs beta > -3/2.  With
 * G and beta <= 3/2 a source whose estimate reaches zero stays at zero.
 * ZI_ERR_ARG for bad sizes or parameters.  Scratch comes from the library's
 * pool.  Synchronises. */
int zi_ias_map(const double* L, int32_t Le, int64_t n, const double* Y, int32_t T, double nu, double theta0,
               double beta, int32_t hypermodel, int32_t iters, double* X, double* Theta, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics (no counterpart in the paper: measurement support)             */
/* ------------------------------------------------------------------------ */

/* Times the solver's sparse matrix product (the multi-RHS SpMM fused with the
 * column dots, the kernel of each CG iteration) on the system's current
 * solver matrix and work vectors: `reps` launches on the library's stream,
 * each bracketed by CUDA events, with a write of a 256 MB buffer between
 * launches so the next one starts with a cold L2.  precision: ZI_FP64 or
 * ZI_MIXED (FP32 product).  Requires a prior zi_transfer with the same
 * precision.  Writes the mean launch time in ms to *ms_per_launch and the
 * kernel's algorithmic bytes per launch (matrix values, column indices, row
 * pointers, one read of P and one write of Q; for ZI_MIXED, P is read in FP16
 * and Q written in FP32) to *bytes_per_launch. */
int zi_time_spmm(zi_system* sys, int precision, int reps, double* ms_per_launch,
                 double* bytes_per_launch, cudaStream_t stream);

/* Times the source application of zi_leadfield_sparse (H^T = F^T T, the
 * kernel that reads the transfer matrix at the source columns' nodes): `reps`
 * launches on `stream`, each after a 256 MB write that evicts the L2 and
 * bracketed by CUDA events.  The system must hold T.  Writes the mean launch
 * time in ms and the algorithmic bytes per launch: the F entries (12 B each),
 * one read of every distinct T row per group of three columns (one Cartesian
 * source; per column when ncols is not a multiple of 3), and the write of
 * H^T (ncols x n_rhs f64). */
int zi_time_source_apply(zi_system* sys, const int32_t* F_nodes, const double* F_w, int64_t ncols, int K,
                         int reps, double* ms_per_launch, double* bytes_per_launch, cudaStream_t stream);

/* Applies the solver's own sparse operator, with the same kernel and the same
 * fused column reduction that every CG iteration runs (Sec. 2.3.1, the
 * product of A (App. A.1) with the search directions of all right-hand sides):
 *   opts->precision == ZI_FP64: Y = S A~ S X, the FP64 CG's operator: A~ is A
 *     without its rounding-noise entries (|a_ij| <= 2^-40 sqrt(|a_ii a_jj|)),
 *     S = D^-1/2 with D the diagonal of opts->precond (a_ii for Jacobi,
 *     sum_j |a_ij| for LDP);
 *   ZI_MIXED: Y = A X by the inner FP32 operator: X rounded to FP16 (round to
 *     nearest even, saturating at +-65504: the storage of the FP32 path's
 *     search directions), A in difference form (A x)_i = c_i x_i +
 *     sum_{j != i} a_ij (x_j - x_i) with c_i the FP64 row sum, entries below
 *     2^-24 of the scaled diagonal left to c_i; FP32 arithmetic.
 *   X: device n x n_rhs f64 (node-major, like T); Y: device out, n x n_rhs f64.
 *   dots: device out, n_rhs f64, or NULL: the column dots sum_i x_ic y_ic as the
 *     CG forms its p.q (per-thread partials, then per-block and per-cluster
 *     sums in a fixed order).
 * Builds the solver's matrix copies when needed and overwrites the solver's
 * work vectors (the next zi_transfer starts afresh); T is kept.  A diagnostic:
 * it lets a test check the operator and its reduction row by row.
 * Synchronises. */
int zi_apply_operator(zi_system* sys, const zi_solver_opts* opts, const double* X, double* Y, double* dots,
                      cudaStream_t stream);

/* Layout of the FP32 sparse product (zi_solver_info.spmm32). */
enum {
  ZI_SPMM32_NONE = 0,          /* the FP32 copy has not been built yet */
  ZI_SPMM32_ELL = 1,           /* 8 slots per row, longer rows continue in a CSR tail */
  ZI_SPMM32_ELL_OVERFLOW = 2   /* as 1, with eight more slots per row staged with the row (many long rows) */
};

typedef struct zi_solver_info {
  int32_t ld;                   /* columns of the solver's vectors (n_rhs padded) */
  int32_t threads_per_row64;    /* FP64 kernels: threads per row, 16-byte vectors per thread */
  int32_t vectors_per_thread64;
  int32_t threads_per_row32;    /* FP32 kernels */
  int32_t vectors_per_thread32;
  int32_t spmm32;               /* ZI_SPMM32_* */
  int64_t nnz64;                /* entries of the FP64 solver copy (0 until built) */
  int64_t nnz32;                /* entries of the FP32 copy (0 until built) */
  int64_t tail_rows;            /* rows of the FP32 copy with more than 8 entries */
  int64_t tail_entries;         /* entries beyond the first 8 of those rows */
  int32_t ell_tiled;            /* 1: the FP32 copy stores its rows in tile columns (nodes on a grid), 0: in
                                   row order; the product is the same either way */
} zi_solver_info;

/* The solver's layout for this system: vector width and row split, and the
 * sizes and FP32 product layout of the matrix copies built by the last
 * zi_transfer or zi_apply_operator.  Host only; never synchronises. */
int zi_solver_get_info(const zi_system* sys, zi_solver_info* info);

/* Device memory of the library's private pool on the current device (every
 * library allocation comes from it): bytes in use now and the high-water mark
 * since the last reset (reset_high != 0 sets the mark to zero after reading).
 * A diagnostic: a test reads it around calls that must not allocate. */
int zi_memory_stats(int64_t* used_now, int64_t* used_high, int reset_high);

/* Number of libzi kernels launched by this process so far (graph replays
 * count each kernel node). */
int64_t zi_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* ZI_H */
