/*
 * lfem.h -- C ABI of the GB300 (sm_103a) isoparametric finite-element assembly library.
 *
 * The library assembles, for Lagrange elements of order 1 to 4 on curves and
 * surfaces (d = 1, 2 in R^{d+1}) and in bulk domains (d = n = 2, 3):
 *   mass                    M_ij  = int phi_i phi_j                  (Sec. 2.2; Eq. M matrix)
 *   stiffness               A_ij  = int grad_G phi_i . grad_G phi_j   (Sec. 2.2; Eq. A matrix)
 *   coefficient-weighted    MC_ij = int c phi_i phi_j, c given at quadrature points
 *                                   (the quadrature-point weighting of Sec. 5.2)
 * element by element with a quadrature rule (Eqs. reference_quadrature_mass,
 * reference_quadrature_stiffness), summed into a CSR matrix whose pattern is
 * every structural pair (E[e,a], E[e,b]) (the index set sparse(I,J,V) builds,
 * Sec. 3.3/3.4; "precomputing the sparsity structure", Sec. 3.3).
 *
 * Conventions shared by every entry point
 *  - Node coordinates  coords: double [n_nodes][ambient], row-major (Sec. 4: array N).
 *  - Connectivity      conn:   int32  [n_elem][ref], ref = C(order+dim, dim), 0-based,
 *                              corners first then edge nodes (Sec. 4.1: array E).
 *                              Edge-node order: segment (0,1); triangle (0,1),(1,2),(2,0);
 *                              tetrahedron (0,1),(1,2),(2,0),(0,3),(1,3),(2,3).
 *  - Supported (dim, ambient): (1,1) (1,2) (1,3) (2,2) (2,3) (3,3); order 1 or 2
 *    (Table ellFEM_overview); orders 3 and 4 for lfem_pattern and lfem_assemble
 *    (every (dim, ambient)), and on curves and triangles also for the vector
 *    assemblies (not for the adjoint, the stage entry points, batches or
 *    lfem_pattern_csr_noalloc).
 *    Order-p node order (p = 3, 4): corners; then per edge (i, j) in the order
 *    above the p - 1 nodes at barycentric ((p-k) e_i + k e_j) / p, k = 1..p-1;
 *    then the triangle's interior nodes alpha / p (every alpha_i >= 1) in
 *    increasing (alpha_1, alpha_2); for tetrahedra instead the face nodes,
 *    face by face in the order (0,1,2), (0,1,3), (0,2,3), (1,2,3), each face
 *    (i, j, l) with alpha_i, alpha_j, alpha_l >= 1 by increasing (alpha_j,
 *    alpha_l), then the interior nodes (all four >= 1) by increasing
 *    (alpha_1, alpha_2, alpha_3).  Anything else: LFEM_E_UNSUPPORTED.
 *  - Quadrature rules are host arrays on the reference simplex (interval [0,1],
 *    triangle conv{0,e1,e2}, tetrahedron conv{0,e1,e2,e3}); weights sum to its
 *    measure.  n_pts <= LFEM_MAX_QPTS.  For order-1 elements quad may be NULL
 *    in lfem_assemble, lfem_autotune, the adjoints, the vector assemblies,
 *    lfem_mcf_step and batch items: M and A are then the exact ones of the
 *    paper's P1 precomputation (exact reference mass matrix and stiffness
 *    building blocks, Sec. 4.2), computed with the element's degree-2 rule
 *    (3-point Gauss on [0,1]; the interior 3-point triangle rule; the 4-point
 *    tet rule), which integrates every order-1 mass and stiffness integrand
 *    exactly on affine elements.  LFEM_CMASS and coefficient gradients need
 *    an explicit rule (LFEM_E_ARG).
 *  - Device pointers are caller-owned unless stated.  Outputs are overwritten,
 *    never accumulated into.
 *  - All work is enqueued on the given CUDA stream (NULL = legacy default
 *    stream) and is asynchronous, except where an entry point says it
 *    synchronises.  A pattern may be used by one stream at a time.
 *  - Errors that the host can see are returned at once.  Errors found on the
 *    device (node index out of range, zero or non-finite |det DF|) are
 *    recorded in the pattern's status word and returned by lfem_sync_status.
 *    lfem_last_error() gives a thread-local message for the last failure.
 */
#ifndef LFEM_H
#define LFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LFEM_MAX_QPTS 64

typedef struct lfem_pattern_s* lfem_pattern_t;
typedef struct lfem_batch_s* lfem_batch_t;

typedef enum {
  LFEM_OK = 0,
  LFEM_E_ARG = 1,          /* null pointer, negative size, bad flag */
  LFEM_E_INDEX = 2,        /* node index outside [0, n_nodes) */
  LFEM_E_UNSUPPORTED = 3,  /* (dim, ambient, order) not supported, or too many quadrature points */
  LFEM_E_TOO_LARGE = 4,    /* a size limit below is exceeded */
  LFEM_E_NOMEM = 5,        /* a device or host allocation failed */
  LFEM_E_CUDA = 6,         /* a CUDA runtime call failed (message in lfem_last_error) */
  LFEM_E_DEGENERATE = 7,   /* |det DF| zero or non-finite at a quadrature point (values still written) */
  LFEM_E_TIMEOUT = 8       /* a bounded device wait gave up */
} lfem_status;

typedef enum {
  LFEM_FP64 = 0,  /* every step in double; outputs double */
  LFEM_MIXED = 1  /* geometry and local matrices in float (Jacobian from double
                     coordinate differences), elements with an ill-conditioned
                     metric redone in double, compensated (two-float) sums;
                     outputs float */
} lfem_precision;

enum { LFEM_MASS = 1, LFEM_STIFF = 2, LFEM_CMASS = 4 };

/* Quadrature rule, host arrays: xi [n_pts][dim], w [n_pts]. */
typedef struct {
  int n_pts;
  const double* xi;
  const double* w;
} lfem_quad;

/* ---------------------------------------------------------------------------
 * Pattern (once per topology).
 *
 * lfem_pattern builds, on the device, the CSR pattern of all pairs
 * (conn[e][a], conn[e][b]) (rows ascending, columns ascending within a row,
 * duplicates merged; rows of unreferenced nodes are empty) and the maps the
 * assembly kernels use.  conn is a device pointer; it is copied, so the caller
 * may free it afterwards.  The call synchronises the stream once (to size the
 * column array) and returns LFEM_E_INDEX if any node index is outside
 * [0, n_nodes).
 * Limits: n_elem * ref < 2^31 (order-3/4 tets: n_elem < 2^25 and n_elem * ref^2
 * < 2^31); every CSR row shorter than the tile capacity (default 4096 slots);
 * at most 2048 elements meet at one node; nnz < 2^31.  Order-3/4 tets (more
 * than 16 nodes) get no row tiles.
 * Ownership: *out owns all of its device memory until lfem_pattern_destroy.
 */
lfem_status lfem_pattern(const int32_t* conn, int64_t n_elem, int32_t n_nodes, int dim, int order,
                         void* cuda_stream, lfem_pattern_t* out);

/* Read-only views of the pattern's CSR arrays (device pointers owned by the pattern). */
lfem_status lfem_pattern_csr(lfem_pattern_t p, int64_t* n_rows, int64_t* nnz, const int64_t** row_ptr,
                             const int32_t** col_idx);

/* Copy the CSR arrays into caller buffers (device pointers: row_ptr int64 [n_rows+1],
 * col_idx int32 [nnz]); asynchronous on the stream. */
lfem_status lfem_pattern_copy_csr(lfem_pattern_t p, int64_t* row_ptr, int32_t* col_idx, void* cuda_stream);

/* Pattern statistics: tiles, elements computed per tile pass (halo recompute
 * factor x 1000), maximum row length.  Host values; no synchronisation. */
lfem_status lfem_pattern_info(lfem_pattern_t p, int64_t* n_tiles, int64_t* recompute_x1000, int32_t* max_row,
                              int32_t* tile_slots);

/* Rebuild the row tiles with a different capacity (slots per tile, 256..16384).
 * LFEM_E_UNSUPPORTED for elements of more than 16 nodes (order-3/4 tets). */
lfem_status lfem_pattern_retile(lfem_pattern_t p, int32_t tile_slots, void* cuda_stream);

void lfem_pattern_destroy(lfem_pattern_t p);

/* ---------------------------------------------------------------------------
 * Assembly: fills the CSR values of the requested matrices.
 *   which:  bitmask of LFEM_MASS / LFEM_STIFF / LFEM_CMASS.
 *   coef:   [n_elem][n_pts] quadrature-point coefficient for LFEM_CMASS, double,
 *           or float when coef_is_fp32 != 0 (the value at the physical point
 *           F_E(xi_q), see lfem_eval_points).  NULL only if LFEM_CMASS is not requested.
 *   M, A, MC: [nnz] outputs, double for LFEM_FP64 and float for LFEM_MIXED;
 *           a matrix not requested may be NULL.
 * Work per CSR slot is summed in a fixed order; the result does not depend on
 * scheduling (bit-identical reruns).  No atomics are used.
 * Surfaces, curves and bulk triangles of order 1, 2 run on row tiles;
 * tetrahedra and orders 3, 4 compute every element once into a local-matrix
 * buffer owned by the pattern ([n_elem][matrices][U], allocated on first use
 * or when a call needs more; that call allocates device memory, so make it
 * before any stream capture).  Order-3/4 tets take one warp per element and
 * tabulate the basis on the device (the buffer also holds those tables and,
 * for LFEM_MIXED, the list of elements redone in double: an element whose
 * metric fails the conditioning test at any point is redone whole).
 */
lfem_status lfem_assemble(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                          const void* coef, int coef_is_fp32, unsigned which, lfem_precision prec, void* M,
                          void* A, void* MC, void* cuda_stream);

/* Launch configuration of the assembly kernels (elements per chunk, threads
 * per block); 0 keeps the current value.  Used by the autotuner. */
lfem_status lfem_set_launch(lfem_pattern_t p, int32_t elems_per_chunk, int32_t threads);

/* Conditioning threshold of LFEM_MIXED (the precision split of the method's
 * FP32 geometry, with FP64 kept for thin elements).  The stiffness of an
 * element of dimension d = 2, 3 is redone in double when, at some quadrature
 * point, its metric G = J^T J may have condition number above kappa_max (the
 * mass-type matrices need |det DF| only and stay in FP32).  The test needs no
 * eigenvalues: with q = det G / (tr G / d)^d, q >= 4 k / (1 + k)^2 implies
 * cond(G) <= k for d = 2 (equality) and d = 3 (the bound is reached when the
 * middle eigenvalue is the mean of the outer two), so elements with q below
 * that bound are redone; the test is conservative for d = 3.  Curves have a
 * scalar metric and are redone only for the degenerate / non-finite checks,
 * which apply for every kappa_max.  kappa_max >= 1 (INFINITY: never for
 * conditioning); default 64 (q = 256/4225).  A batch uses the
 * strictest threshold of its patterns, read when it is created.
 * LFEM_E_ARG for kappa_max < 1 or NaN. */
lfem_status lfem_set_mixed_kappa(lfem_pattern_t p, double kappa_max);

/* Autotuner: times lfem_assemble (CUDA events, after one warm-up) for each
 * candidate tile capacity (slots per tile: 512..8192, those whose shared
 * memory fits), keeps the fastest and retiles p with it.  M/A/MC are scratch
 * outputs sized as for lfem_assemble (overwritten).  If cache_path is not
 * NULL, results are read from / appended to that text file, keyed by
 * (dim, ambient, order, quadrature points, precision, which, element-count
 * bucket, GPU name).  Synchronises the stream; *best_slots may be NULL. */
lfem_status lfem_autotune(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad, const void* coef,
                          int coef_is_fp32, unsigned which, lfem_precision prec, void* M, void* A, void* MC,
                          const char* cache_path, void* cuda_stream, int32_t* best_slots);

/* Failure-path test knob (not for production use): with starve != 0 the first
 * CTA of the next assemblies on p skips its first metadata copy, so its bounded
 * wait (2 s) runs out; lfem_sync_status then returns LFEM_E_TIMEOUT and the
 * values of that CTA's tiles are left unwritten.  The CUDA context stays usable. */
lfem_status lfem_debug_starve_wait(lfem_pattern_t p, int starve);

/* Test knob: with wide != 0 the pattern's tile blocks store their slot
 * entries in 32 bits even when 16 would do (batches widen them that way when
 * a mesh needs it); the tiles are rebuilt on the stream.  Results do not
 * depend on the width. */
lfem_status lfem_debug_wide_entries(lfem_pattern_t p, int wide, void* cuda_stream);

/* Test knob: the number of device allocations (cudaMalloc) the library has
 * made successfully in this process, across all devices and threads.  Used to
 * check that an entry point allocates nothing; it never resets. */
long long lfem_debug_alloc_count(void);

/* ---------------------------------------------------------------------------
 * Batches: many meshes of uneven sizes and different element types assembled
 * by persistent launches over all their row tiles, one launch per element
 * family (the work list is sorted by family; each launch is the single-type
 * kernel of that family), mixed precision only; curves and triangles:
 * (dim, ambient) in (1,2) (2,2) (2,3).  Items of order 3 or 4 run their
 * element-major path on the same stream after those launches (inside the same
 * graph); their rule and element buffer are registered at creation, their
 * status is read by lfem_batch_sync_status.
 * Motivated by the paper's batchwise processing of large meshes (Remark
 * "Batch computations", Sec. 3.3; Sec. 5.1).
 *
 * Every pointer of an item is fixed at creation: later calls read the current
 * contents of coords / coef and overwrite M / A / MC (float [nnz] of the
 * item's pattern).  The batch keeps its own status word.
 */
typedef struct {
  lfem_pattern_t pattern;  /* topology (not owned) */
  const double* coords;    /* device [n_nodes][ambient] */
  int ambient;
  const lfem_quad* quad;   /* host rule; tables are registered at creation */
  const void* coef;        /* device [n_elem][n_pts] (float if coef_is_fp32) or NULL */
  void* M;
  void* A;
  void* MC;
} lfem_batch_item;

lfem_status lfem_batch_create(const lfem_batch_item* items, int n_items, unsigned which, int coef_is_fp32,
                              void* cuda_stream, lfem_batch_t* out);
/* The batch's persistent launches, one per element family (asynchronous). */
lfem_status lfem_batch_assemble(lfem_batch_t b, void* cuda_stream);
/* The same launch as a CUDA graph: captured on the first call, replayed after. */
lfem_status lfem_batch_graph_launch(lfem_batch_t b, void* cuda_stream);
/* Synchronises; returns and clears the batch status (LFEM_E_DEGENERATE, LFEM_E_TIMEOUT). */
lfem_status lfem_batch_sync_status(lfem_batch_t b, void* cuda_stream);
/* Work items, elements computed and the largest tile of the batch (host values). */
lfem_status lfem_batch_info(lfem_batch_t b, int64_t* n_work_items, int64_t* n_elements, int32_t* cap_elements);
void lfem_batch_destroy(lfem_batch_t b);

/* Tile capacity of a batch's meshes, per element family (dim, order): the
 * batch (the same items, which and coef_is_fp32 as lfem_batch_create) is
 * launched with each candidate capacity of the P2 triangle meshes, then of the
 * P1 triangles, the P2 curves and the P1 curves (each family's patterns
 * retiled together, the others held), and every pattern is left at its
 * family's fastest (the paper's batchwise processing, Remark "Batch
 * computations", Sec. 3.3; tuned here by measurement).  best_slots (host
 * int32[4], may be NULL): capacities of P1 curves, P2 curves, P1 triangles,
 * P2 triangles (0 for a family the batch does not hold).  If cache_path is not NULL, the
 * result is read from / appended to that text file, keyed by which, the
 * (dim, ambient, order) counts, the element-count bucket and the GPU name.
 * Create the batch after this call (a batch keeps the tile blocks it was
 * created with); the outputs of the items are overwritten.  Synchronises the
 * stream.  Errors: as lfem_batch_create; LFEM_E_TOO_LARGE if no candidate
 * fits. */
lfem_status lfem_batch_autotune(const lfem_batch_item* items, int n_items, unsigned which, int coef_is_fp32,
                                const char* cache_path, void* cuda_stream, int32_t* best_slots);

/* ---------------------------------------------------------------------------
 * Vector assembly on the pattern's node incidences, FP64, deterministic (each
 * element's local vector once, then every node sums its incidences in
 * ascending element order; no atomics).  coords as for lfem_assemble; the
 * local-vector scratch ([n_elem][ref][nc] doubles) is allocated by the
 * pattern on first use and kept.
 *
 * Load vector of the Poisson problem (Sec. 2): b_j = integral over Gamma_h of
 * f_h phi_j, f_h = sum_i f_i phi_i the interpolant of the nodal values, so
 * b = M f.  f: [n_nodes] doubles; b: [n_nodes] doubles, overwritten.  Every
 * (dim, ambient, order) lfem_assemble supports except order-3/4 tetrahedra
 * (LFEM_E_UNSUPPORTED).
 */
lfem_status lfem_assemble_load(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                               const double* f, double* b, void* cuda_stream);

/* Non-linear vectors of the mean curvature flow system (Sec. 5.1): with
 * u = (nu, H) at the nodes ([n_nodes][4] doubles: normal components, then
 * mean curvature), nu_h, H_h their interpolants and alpha^2 =
 * |grad_Gamma_h nu_h|^2 (Frobenius norm of the tangential gradient),
 *   out[k * n_nodes + j]     = integral of alpha^2 (nu_h)_k phi_j  (k = 0, 1, 2)
 *   out[3 * n_nodes + j]     = integral of alpha^2 H_h phi_j.
 * out: [4][n_nodes] doubles, overwritten.  Surfaces only (dim 2, ambient 3):
 * LFEM_E_UNSUPPORTED otherwise. */
lfem_status lfem_assemble_mcf_nonlinear(lfem_pattern_t p, const double* coords, const lfem_quad* quad,
                                        const double* u, double* out, void* cuda_stream);

/* One step of Dziuk's scheme for mean curvature flow, the classical method the
 * paper's flow example builds on (Sec. 5.1):
 *   (M(x0) + tau A(x0)) x1 = M(x0) x0      (one system per coordinate),
 * M and A assembled in FP64 on the pattern, the systems solved together by a
 * Jacobi-preconditioned conjugate gradient (hand-written kernels, reductions
 * in a fixed order: bit-reproducible), started from x0, stopped when every
 * column's residual satisfies |r| <= rtol |M x0| (checked every 8
 * iterations) or after max_iter iterations.  Curves in R^2 and surfaces in R^3
 * (ambient = dim + 1), else LFEM_E_UNSUPPORTED.  A CG iteration is three
 * kernels (K p with <p, q>; x, r, z with <r, z>; p), each block reducing the
 * previous kernel's per-block partials itself in one fixed order; on a stream
 * other than the legacy default one the 8 iterations between two checks are a
 * CUDA graph, captured on first use and kept by the pattern.
 *   coords:     x0 [n_nodes][ambient] device doubles.
 *   coords_out: x1 [n_nodes][ambient] device doubles (may equal coords).
 *   iterations: host int, the CG iterations done (== max_iter: not converged).
 * Synchronises the stream (convergence checks); scratch (3 nnz + 6 n_nodes x
 * ambient doubles and 7,296 for the partial sums) is allocated by the pattern
 * on first use and kept. */
lfem_status lfem_mcf_step(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad, double tau,
                          double rtol, int max_iter, double* coords_out, int* iterations, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Adjoint: for L = gM.M + gA.A + gMC.MC (dot products over the CSR values),
 * g_coords [n_nodes][ambient] = dL/d coords (overwritten) and, when g_coef is
 * not NULL, g_coef [n_elem][n_pts] = dL/d coef.  FP64 throughout.  gM, gA,
 * gMC are [nnz] doubles; any may be NULL (treated as zero).  Geometry is
 * recomputed, not stored.  Orders 1, 2: one thread per element in the
 * pattern's row tiles.  Orders 3, 4 (curves, triangles, tets): one warp per
 * element, the element node gradients in the pattern's element buffer (grown
 * on demand, n_elem x ref x ambient doubles), then summed per node over its
 * incidences in ascending element order.  (Not in the paper: the derivative
 * of its local matrices, Eqs. reference_quadrature_mass / _stiffness, with
 * respect to the node positions.)
 */
lfem_status lfem_assemble_adjoint(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                  const double* coef, const double* gM, const double* gA, const double* gMC,
                                  double* g_coords, double* g_coef, void* cuda_stream);

/* The same adjoint with FP32 geometry and per-point algebra (coordinates split
 * into exact float pairs as in LFEM_MIXED), the element's node gradients summed
 * per node in double, and a double recomputation of every element whose
 * metric may have cond(G) > sqrt(kappa_max) (G^{-1} enters the derivative
 * twice; kappa_max from lfem_set_mixed_kappa) or fails the finiteness test;
 * the count is reported by lfem_mixed_fallback_count.  Orders 3, 4 run the
 * double path for every element (each counted as recomputed).
 * Arguments and outputs as for lfem_assemble_adjoint (double). */
lfem_status lfem_assemble_adjoint_mixed(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                        const double* coef, const double* gM, const double* gA, const double* gMC,
                                        double* g_coords, double* g_coef, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Element-level stages (no global scatter).  Useful on their own (matrix-free
 * use, coefficient evaluation) and to test each stage.
 *
 * lfem_eval_points: x_q = F_E(xi_q) = sum_a x_a phi_a(xi_q) (Eq. F_map),
 *   out double [n_elem][n_pts][ambient].
 * lfem_geometry: per quadrature point, J = DF (Eq. jacobian_inv's rows) as
 *   double [n_elem][n_pts][ambient][dim], s = |det DF| (surface: |d1F x d2F|)
 *   [n_elem][n_pts], and G^{-1} with G = J^T J, [n_elem][n_pts][dim][dim];
 *   any output may be NULL.
 * lfem_local: element matrices by quadrature, upper triangle (a <= b, row-major
 *   order (0,0),(0,1)..(0,ref-1),(1,1)..), double [n_elem][ref(ref+1)/2] each.
 * conn and coords are device pointers; these calls are asynchronous and set
 * no status word (non-finite results are written as computed).  Orders 1-4
 * on curves and triangles, orders 1-2 on tets; order-3/4 tets return
 * LFEM_E_UNSUPPORTED (their basis tables live on the device, not in the
 * constant bank these kernels read).
 */
lfem_status lfem_eval_points(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords,
                             int ambient, const lfem_quad* quad, double* out, void* cuda_stream);
lfem_status lfem_geometry(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords,
                          int ambient, const lfem_quad* quad, double* J, double* s, double* Ginv,
                          void* cuda_stream);
lfem_status lfem_local(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords, int ambient,
                       const lfem_quad* quad, const double* coef, double* Mloc, double* Aloc, double* MCloc,
                       void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Status word: synchronises the stream, returns and clears the device status
 * of pattern p (LFEM_OK, LFEM_E_DEGENERATE, LFEM_E_INDEX), and reports how
 * many elements the last LFEM_MIXED assembly redid in double.
 */
lfem_status lfem_sync_status(lfem_pattern_t p, void* cuda_stream);  /* also LFEM_E_TIMEOUT, and
  LFEM_E_UNSUPPORTED if a tile met a kernel without a variant for its element type */
lfem_status lfem_mixed_fallback_count(lfem_pattern_t p, void* cuda_stream, int64_t* n_fp64_elements);

const char* lfem_last_error(void);
const char* lfem_status_string(lfem_status s);

/* Order-p nodes from an order-1 curve, triangle or tetrahedron mesh (the node
 * generation of the paper's preprocessing, Sec. 4; orders 2..4).  p1 is the
 * order-1 pattern of the mesh; its edges are the upper slots (i < j) of the
 * pattern's rows, numbered in CSR order.  Output numbering: the P1 vertices
 * keep their numbers; then p - 1 nodes per edge, from its lower to its higher
 * vertex number, at the straight positions x_lo (1 - k/p) + x_hi k/p; then
 * each triangle's interior nodes at alpha / p in barycentrics; for
 * tetrahedra instead the (p-1)(p-2)/2 nodes of every face (faces in
 * lexicographic order of their sorted vertex triples (g0 < g1 < g2), nodes
 * sum_k (a_k / p) x_{g_k} by increasing (a_1, a_2), shared by the face's two
 * tets), then each tet's interior nodes (order 4: one, at the centroid).
 * Local order: that of the conventions above.  Positions are rounded in a
 * fixed order (products, then sums left to right), so any implementation
 * that evaluates the same expressions that way gets the same bits.
 *   coords:      [n_vertices][ambient] device doubles (the P1 nodes).
 *   conn_out:    [n_elem][C(order+dim, dim)] device int32, or NULL.
 *   coords_out:  [n_nodes_out][ambient] device doubles, or NULL.
 *   n_nodes_out: host; always written.  With both outputs NULL only the size
 *                is computed.  Synchronises the stream.
 * Curved geometry: move the generated nodes afterwards (e.g. project them). */
lfem_status lfem_lift_order(lfem_pattern_t p1, const double* coords, int ambient, int order, int32_t* conn_out,
                            double* coords_out, int64_t* n_nodes_out, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * CSR pattern without any device allocation.  (The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * run time -- programs whose memory arena or pool owns the device up front, or
 * loops that forbid cudaMalloc after start-up.)
 *
 * Same pattern as lfem_pattern (rows and columns ascending, duplicates merged,
 * bit-identical output) but only the CSR arrays, no assembly maps.  The caller
 * passes row_ptr (device int64 [n_nodes+1]) and col_idx (device int32
 * [col_capacity]); *nnz receives the pattern size.  Scratch lives in a 16 MiB
 * array inside the library that every GPU loading the library keeps until the
 * process exits; the mesh must fit it:
 *   ~ n_elem*ref*(ref+2) + 4*n_nodes int32 words <= 4 Mi words
 * (for example about 100k six-node triangles), else LFEM_E_TOO_LARGE and
 * nothing is written.  If nnz > col_capacity the call writes row_ptr, sets *nnz
 * and returns LFEM_E_TOO_LARGE.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset (or
 * anything else that destroys the device's primary context) it is stale and
 * the entry point must not be called again on that device.
 * The call synchronises the stream.  All calls share the one array: calls that
 * overlap on the GPU race, so issue them one at a time.
 */
lfem_status lfem_pattern_csr_noalloc(const int32_t* conn, int64_t n_elem, int32_t n_nodes, int dim, int order,
                                     int64_t* row_ptr, int32_t* col_idx, int64_t col_capacity, int64_t* nnz,
                                     void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LFEM_H */
