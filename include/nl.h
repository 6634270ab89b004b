/* nl.h -- C ABI of the GB300 library for finite-element assembly of the mollified
 * nonlocal diffusion operator of Aulisa, Capodaglio, Chierici, D'Elia, "Efficient
 * quadrature rules for finite element discretizations of nonlocal equations"
 * (arXiv 2101.08825), and for the volume-constrained Poisson problem built on it.
 *
 * Problem (Sec. 2, eqs. L, poisson, A-F): Omega open and bounded, Gamma the interaction
 * layer of points within delta of Omega, gamma(x,y) = C eta(|x-y|) 1(|x-y| <= delta)
 * (eq. gamma).  Sec. 3 (eqs. approx-kernel, mollifier) replaces the indicator by the
 * C^4 mollifier mu_{delta,eps}(r) = 1 (r < delta-eps), xi((delta-r)/eps) (band),
 * 0 (r > delta+eps).  Sec. 4 (eq. Aij-support2) defines the P1 stiffness matrix
 * A_ij = int int (phi_i(x)-phi_i(y))(phi_j(x)-phi_j(y)) gamma_eps(x,y) dy dx, which
 * Sec. 5 (Corollary 1, eqs. J21Nr, J22Nr) computes as 2 A^21 + 2 A^22: an inner
 * Gauss rule on element m (rows: the nodes of m) and an outer rule on element l that
 * Algorithm 1 refines adaptively per (l, m) pair with the box distances of Sec. 5.1.
 *
 * Conventions for every entry point:
 *   - the return value is an nl_status; nothing aborts or throws across the ABI, and on
 *     failure nl_last_error() returns a message for the calling thread;
 *   - handles are opaque and owned by the library; destroy them with their *_destroy;
 *   - host arrays passed in are owned by the caller and are copied before return;
 *     host arrays passed out are caller-allocated with the documented size;
 *   - every handle binds the CUDA stream given at mesh creation (NULL = legacy default
 *     stream); work is enqueued on it and the calls that return host data synchronise it;
 *   - device memory comes from the allocator installed by nl_set_allocator
 *     (default: cudaMallocAsync / cudaFreeAsync on the handle's stream).
 */
#ifndef NL_H
#define NL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NL_OK = 0,
  NL_EINVAL = 1,     /* invalid argument (message in nl_last_error) */
  NL_ENOMEM = 2,     /* a device or host allocation failed */
  NL_ECUDA = 3,      /* a CUDA runtime call failed */
  NL_ENOTCONV = 4,   /* the iterative solver hit max_iter before rtol */
  NL_ETIMEOUT = 5,   /* a bounded wait ran out */
  NL_EBUSY = 6,      /* the result is not ready yet (nl_serve_poll) */
  NL_EINTERNAL = 7   /* a device-side capacity or consistency check failed */
} nl_status;

typedef enum {
  NL_KERNEL_CONST = 0,      /* eta = 1 (Sec. 6) */
  NL_KERNEL_TRUNC_GAUSS = 1 /* eta = exp(-r^2/delta^2) */
} nl_kernel_kind;

typedef enum {
  NL_PREC_FP64 = 0,       /* every point pair and every accumulation in FP64 */
  NL_PREC_MIXED_TF32 = 1, /* the NL_PREC_FP32 path with the per-pair contraction over the
                             outer points, H_c(y) = sum_x gamma_eps(x,y) w_x phi^l_c(x), on the
                             tensor cores (mma.sync m16n8k8 TF32, FP32 accumulation); both
                             operands split into two TF32 parts (about 22 significant bits)
                             and the cross products summed; self blocks, scatter and
                             decisions as in NL_PREC_FP32 */
  NL_PREC_MIXED_BF16 = 2, /* as MIXED_TF32 with mma.sync m16n8k16 BF16 and two BF16 parts per
                             operand (about 16 significant bits) */
  NL_PREC_FP32 = 3        /* gamma_eps and the per-pair local sums in FP32 on the ALUs
                             (packed FP32x2 arithmetic), decisions and scatter exact/FP64 */
} nl_precision;
/* nl_assemble runs each precision as named.  nl_assemble_noalloc and batched plans run the
 * MIXED precisions with the NL_PREC_FP32 arithmetic; every assembly reports the arithmetic
 * that ran in nl_assemble_stats.precision_run. */

/* Kernel gamma_eps = C eta mu_{delta,eps}.  Requires 0 < eps < delta (Sec. 3).
 * C_override = 0 selects C_{delta,eps}: for NL_KERNEL_CONST the closed form of Sec. 6
 * with kappa = 1, otherwise the value that makes int z_1^2 gamma_eps dz = 1 (so that
 * L_eps u = Laplace(u) for quadratic u, the property Sec. 6 uses to fix the constant). */
typedef struct {
  double delta, eps;
  double kappa;      /* multiplies C; 0 is read as 1 */
  int kernel;        /* nl_kernel_kind */
  double C_override; /* > 0: use this C instead */
} nl_kernel_params;

/* Algorithm 1 levels, 1 <= L_min <= L_max <= 12 (2D) or 9 (3D).  rule: 0 = the degree-5
 * 7-point triangle rule (Sec. 6) and the degree-5 14-point tetrahedral rule, optionally OR
 *   NL_QUAD_COUNT_BAND  count the point pairs in the mollifier band (a measurement aid; it
 *                       adds an integer add per evaluated point pair);
 *   NL_QUAD_MINDIST_L2  Algorithm 1's refinement test uses the Euclidean approximate minimum
 *                       distance sqrt(sum_k max(0, d1^k, d2^k)^2) that Sec. 5.1 gives after
 *                       eq. mindistin (valid for kernels supported on a Euclidean ball, as
 *                       both kernels here are) instead of eq. mindist.  It drops sub-elements
 *                       and pairs whose every point pair lies beyond delta + eps, so the
 *                       matrix is unchanged (their contributions are exactly zero) while the
 *                       work counters shrink; the element pairs and the pattern (eq. k_l)
 *                       keep eq. mindist. */
#define NL_QUAD_COUNT_BAND 0x100
#define NL_QUAD_MINDIST_L2 0x200
typedef struct {
  int L_min, L_max;
  int rule;
} nl_quad_params;

/* Work counters of one assembly. */
typedef struct {
  int64_t n_pairs;        /* element pairs |J| */
  int64_t n_point_pairs;  /* (outer, inner) point pairs of Algorithm 1 */
  int64_t n_items;        /* (sub-element, m) integrations of Algorithm 1 */
  int64_t n_exact_checks; /* classifications decided by the FP64 fallback */
  double ms_assemble;     /* device time of the assembly kernels (CUDA events) */
  int64_t n_eval_point_pairs; /* point pairs evaluated one by one; the others belong to
                                 sub-elements beyond delta+eps (mu = 0) or, with the
                                 constant kernel, to sub-elements with mu = 1, whose outer
                                 sums have the closed form C |E'| [1, lambda(centroid)] */
  int64_t n_closed_items;     /* sub-elements summed in closed form (mu = 1, constant kernel) */
  int64_t n_band_point_pairs; /* evaluated point pairs with delta-eps <= r <= delta+eps, when
                                 NL_QUAD_COUNT_BAND was given; -1 otherwise */
  int32_t precision_run;      /* the nl_precision whose arithmetic ran */
  int32_t n_quad_launches;    /* launches of the point-pair kernel (the pairs are processed in
                                 batches that bound the block buffer) */
  double ms_quad;             /* device time of those launches (CUDA events; 0 in
                                 nl_assemble_noalloc and nl_plan_sync) */
  double ms_scatter;          /* device time of the scatter launches (as ms_quad) */
} nl_assemble_stats;

typedef struct nl_mesh nl_mesh;
typedef struct nl_pairs nl_pairs;
typedef struct nl_matrix nl_matrix;
typedef struct nl_vector nl_vector;
typedef struct nl_server nl_server;

/* Allocator hooks: alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, bytes, stream, ctx).  Pass NULLs to restore the default.  Not thread-safe
 * against concurrent calls; install it before creating handles. */
typedef void* (*nl_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*nl_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
nl_status nl_set_allocator(nl_alloc_fn alloc, nl_free_fn free_fn, void* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* nl_last_error(void);
/* Library version string. */
const char* nl_version(void);
/* Number of CUDA kernels this library has launched in this process (all threads). */
int64_t nl_launch_count(void);

/* Mesh of Omega U Gamma (Sec. 4: a triangulation T_h, here P1 triangles (dim 2) or
 * tetrahedra (dim 3)).
 *   coords        host, SoA: coords[k*n_vert + v], k < dim (FP64)
 *   conn          host, (dim+1)*n_elem vertex indices, element-major
 *   elem_in_omega host, n_elem flags: 1 = element of Omega, 0 = of Gamma
 *   node_free     host, n_vert flags: 1 = degree of freedom (inside Omega), 0 = value
 *                 prescribed by the volume constraint u = g (eq. poisson)
 * Errors: NL_EINVAL for dim not 2/3, empty or >2^31-1 vertices, an index out of range,
 * a non-finite coordinate or a degenerate element (zero volume). */
nl_status nl_mesh_create(int dim, int64_t n_vert, const double* coords, int64_t n_elem,
                         const int32_t* conn, const uint8_t* elem_in_omega,
                         const uint8_t* node_free, void* cuda_stream, nl_mesh** out);

/* Structured mesh of Omega = prod_k [lo_k, lo_k + cells_k h] with `layer` cells of Gamma on
 * every side.  Vertices are numbered lexicographically (x fastest) over the grid lines
 * counted from the outer corner; cells likewise.  Each square (v00 v10 v01 v11) becomes the
 * triangles (v00, v10, v11), (v00, v11, v01); each cube the 6 Kuhn tetrahedra
 * (v000, v000+e_a, v000+e_a+e_b, v111) for the axis permutations (a, b, c) in
 * lexicographic order.  Vertices off the boundary of Omega and off the outer boundary move
 * by (jitter*h)*(2u-1) per axis, u = splitmix64 output at counter 4*vertex+axis for the
 * given seed, mapped to [0,1) by its top 53 bits.  cells and lo have dim entries. */
nl_status nl_mesh_create_box(int dim, const int32_t* cells, double h, const double* lo,
                             int32_t layer, double jitter, uint64_t seed, void* cuda_stream,
                             nl_mesh** out);
/* Mesh of quadratic (P2) Lagrange simplices (Sec. 6, Tables 1-3, the quadratic columns):
 * the arguments of nl_mesh_create; dim = 2: six nodes per element in conn, ordered
 * (v0, v1, v2, m01, m12, m02): the three vertices, then the nodes at the midpoints of the
 * edges (v0,v1), (v1,v2), (v0,v2); dim = 3: ten nodes, the four vertices, then the midpoints
 * of the edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  n_vert counts every node (vertices
 * and edge nodes); node_free flags every node.  The elements are straight-sided: each edge node must lie at
 * the midpoint of its edge.  The basis on an element with barycentric coordinates lambda is
 * lambda_a (2 lambda_a - 1) at the vertices and 4 lambda_a lambda_b at the edge nodes.
 * Pairs, pattern, nl_assemble (FP64 and FP32; the MIXED precisions run the FP32 path and
 * report it in stats->precision_run), nl_rhs and nl_solve accept it; the batched plans and
 * nl_assemble_noalloc take P1 meshes only.
 * Errors: those of nl_mesh_create, and NL_EINVAL for an edge node off the midpoint of its
 * edge (by more than 1e-9 of the edge's length). */
nl_status nl_mesh_create_p2(int dim, int64_t n_vert, const double* coords, int64_t n_elem,
                            const int32_t* conn, const uint8_t* elem_in_omega,
                            const uint8_t* node_free, void* cuda_stream, nl_mesh** out);
/* Mesh of quadrilaterals (Sec. 6: the QUAD meshes; Gauss-Legendre 3x3 product rule for the
 * inner and the outer integral): dim 2, each element the bilinear image of the unit square,
 * vertices v0..v3 counterclockwise (the images of (0,0), (1,0), (1,1), (0,1)).  order 1: Q1,
 * conn holds the 4 vertices per element; order 2: Q2 (biquadratic Lagrange), 9 nodes per
 * element: the vertices, the nodes at the midpoints of the edges (0,1), (1,2), (2,3), (3,0),
 * then the node at the image of the square's centre (the mean of the vertices); order 3: the
 * 8-node serendipity element, the Q2 nodes without the centre.  Algorithm
 * 1's midpoint refinement splits the square into its four half-size sub-squares (physical
 * vertices: the parent's vertices, edge midpoints (a+b)*0.5 and the centre as the midpoint
 * of the midpoints of the edges (0,1) and (2,3)).  Other arguments as nl_mesh_create.  Pairs,
 * pattern, nl_assemble (FP64, FP32; the MIXED precisions run the FP32 path and report it),
 * nl_rhs and nl_solve accept it; plans and nl_assemble_noalloc take P1 meshes only.
 * Errors: those of nl_mesh_create; NL_EINVAL for order not 1/2/3, an element that is not a
 * convex counterclockwise quadrilateral, or a Q2 node off its position (by more than 1e-9
 * of the element's diagonal). */
nl_status nl_mesh_create_quad(int order, int64_t n_vert, const double* coords, int64_t n_elem,
                              const int32_t* conn, const uint8_t* elem_in_omega,
                              const uint8_t* node_free, void* cuda_stream, nl_mesh** out);
/* Mesh of hexahedra (Sec. 6: the HEX meshes of the 3D tests; Q1 trilinear, Q2 triquadratic
 * or 20-node serendipity elements, the Gauss-Legendre 3x3x3 product rule for the inner and the outer integral): dim
 * 3, each element the trilinear image of the unit cube of its first 8 nodes, the images of the
 * corners (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1).  order 1:
 * conn holds those 8 vertices per element; order 2: 27 nodes per element, the 8 vertices,
 * then the images of the cube's lattice of half steps (i, j, k)/2 that are not corners: the
 * twelve edge midpoints, the six face centres and the centre, each group ordered by
 * i + 3 j + 9 k; the basis is the products of the 1D quadratic Lagrange functions on
 * {0, 1/2, 1}; order 3: the 20-node serendipity element, the first 20 of those nodes (the
 * vertices and the edge midpoints; the quadratic FE of Sec. 6's 3D tests, whose mesh figure
 * counts vertices and edge midpoints).  Algorithm 1's midpoint refinement splits the cube into its eight half-size
 * sub-cubes; their physical vertices lie on the lattice of half steps, a lattice point with a
 * middle index being the midpoint (a+b)*0.5 of its two neighbours along the first such axis
 * (x, then y, then z).  Other arguments as nl_mesh_create; pairs, pattern, nl_assemble
 * (FP64, FP32; MIXED runs FP32), nl_rhs and nl_solve accept it; plans and
 * nl_assemble_noalloc take P1 meshes only.
 * Errors: those of nl_mesh_create; NL_EINVAL for order not 1, 2 or 3, an element whose
 * trilinear map has a non-positive Jacobian determinant at a corner, or a node off the image
 * of its lattice point (by more than 1e-9 of the element's diagonal). */
nl_status nl_mesh_create_hex(int order, int64_t n_vert, const double* coords, int64_t n_elem,
                             const int32_t* conn, const uint8_t* elem_in_omega,
                             const uint8_t* node_free, void* cuda_stream, nl_mesh** out);
nl_status nl_mesh_info(const nl_mesh* mesh, int* dim, int64_t* n_vert, int64_t* n_elem);
/* Polynomial order of the mesh's elements (1: P1 / Q1, 2: P2 / Q2, 3: serendipity
 * quadrilaterals) and nodes per element (simplices dim+1, 6 or 10, quadrilaterals 4, 8 or 9,
 * hexahedra 8, 27 or 20 (serendipity, order 3)); either pointer may be NULL. */
nl_status nl_mesh_order(const nl_mesh* mesh, int* order, int* nodes_per_elem);
/* Copies the mesh back (host buffers of the sizes of nl_mesh_create, conn of
 * nodes_per_elem*n_elem entries; any may be NULL). */
nl_status nl_mesh_export(const nl_mesh* mesh, double* coords, int32_t* conn,
                         uint8_t* elem_in_omega, uint8_t* node_free);
void nl_mesh_destroy(nl_mesh* mesh);

/* Element pairs and sparsity pattern (Sec. 5, eq. k_l; Sec. 5.1 eq. mindist):
 *   J = {(m, l) : aprx-min-dist(E_l, E_m) < delta + eps}, bounding boxes of the vertices,
 * stored m-major with l ascending, and the CSR pattern of A: row i (every node) holds the
 * nodes of every l with (m, l) in J and i a node of m, columns ascending.  The distance test
 * runs in FP32 on boxes rounded outwards and is repeated in FP64 within a margin of the
 * threshold that bounds the FP32 rounding, so J is exactly that of the FP64 test.
 * Errors: NL_EINVAL unless 0 < eps < delta; NL_EINTERNAL if a neighbourhood exceeds the
 * builder's shared-memory capacity (more than 49152 pairs for one element or 8192
 * columns in one row). */
nl_status nl_pairs_build(nl_mesh* mesh, double delta, double eps, nl_pairs** out);
nl_status nl_pairs_info(const nl_pairs* pairs, int64_t* n_pairs, int64_t* nnz);
/* Host copies: pair_off[n_elem+1], pair_l[n_pairs], row_ptr[n_vert+1], col[nnz]; any may
 * be NULL. */
nl_status nl_pairs_export(const nl_pairs* pairs, int64_t* pair_off, int32_t* pair_l,
                          int64_t* row_ptr, int32_t* col);
void nl_pairs_destroy(nl_pairs* pairs);

/* Stiffness matrix values on the pattern of `pairs` (Sec. 5: Corollary 1, eqs. J21Nr and
 * J22Nr with Algorithm 1), computed in the given precision.  The int/ref/drop decisions
 * of Algorithm 1 are bit-identical to a plain FP64 evaluation of eqs. maxdist/mindist on
 * the sub-element vertices obtained by repeated (a+b)*0.5 midpoints (triangles: corner
 * children then the middle one; tetrahedra: Bey's rule with the x02-x13 diagonal), in
 * every precision.  stats may be NULL.  *A is created (or, if *A is a matrix of the same
 * pattern, overwritten). */
nl_status nl_assemble(nl_mesh* mesh, nl_pairs* pairs, const nl_kernel_params* kp,
                      const nl_quad_params* qp, nl_precision precision, nl_matrix** A,
                      nl_assemble_stats* stats);
/* Assembly that allocates no device memory.  The paper has no counterpart: this is an
 * interface for callers that cannot call cudaMalloc while they assemble -- a process that
 * reserves all of its device memory at start-up (a fixed pool it must not grow, where a new
 * allocation would fail), or code that must not stall other streams on an allocation.
 * It computes the same matrix as nl_assemble (same kernels; the cross blocks are added to
 * the values directly) into `values`, a device array of nnz doubles (nl_pairs_info) that the
 * caller owns.  Its scratch (work counter, counters, error word, per-element self blocks)
 * lives in a fixed 16 MiB device array that the library holds on every GPU that loads it
 * until the process exits, so the mesh may have at most (16 MiB - 256 B) / (8 (dim+1)^2 B)
 * elements (233,013 triangles or 131,070 tetrahedra); larger meshes return NL_EINVAL.
 * Every call looks up that array's device address in the current context
 * (cudaGetSymbolAddress); the first lookup in a context may load the library's device code,
 * so make the first call before any stream capture.  Every call clears the scratch it uses
 * and leaves its contents behind; all calls share the one array, so calls that overlap on
 * the GPU (other streams or threads) race and must be serialised by the caller.
 * stats may be NULL; stats->ms_assemble is 0. */
nl_status nl_assemble_noalloc(nl_mesh* mesh, nl_pairs* pairs, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision precision, double* values,
                              nl_assemble_stats* stats);
/* Host copy of the nnz values (CSR order of the pattern). */
nl_status nl_matrix_export(const nl_matrix* A, double* values);
/* y = A x over every row, in FP64: the discrete operator of Sec. 2 (eq. A-F) applied to the
 * nodal vector x.  x and y are device arrays of n_vert doubles owned by the caller (x is read
 * through the pattern's columns, y written).  Enqueued on the matrix's stream; returns without
 * waiting.  Errors: NL_EINVAL for NULL arguments or x == y. */
nl_status nl_matrix_apply(const nl_matrix* A, const double* x, double* y);
/* Device pointer to the values (valid until nl_matrix_destroy). */
nl_status nl_matrix_device_values(const nl_matrix* A, double** values);
void nl_matrix_destroy(nl_matrix* A);

/* Right-hand side with lifting (Sec. 2, eqs. A-F and weak-homo):
 *   F_i = int_Omega f phi_i for free i, f = f_const + the interpolant of f_nodes in the
 *         mesh's element space (P1 or P2; f_nodes may be NULL), integrated with the
 *         degree-5 rule per element of Omega;
 *   F~_i = F_i - sum_{k not free} A_ik g_k;  F~_i = 0 for constrained i.
 * f_nodes, g_nodes: host, n_vert values (g_nodes is read at constrained nodes only). */
nl_status nl_rhs(nl_mesh* mesh, nl_matrix* A, const double* f_nodes, double f_const,
                 const double* g_nodes, nl_vector** rhs);
nl_status nl_vector_export(const nl_vector* v, double* values);
void nl_vector_destroy(nl_vector* v);

/* Solves A_{free,free} W = F~_free (A is nonsymmetric at quadrature-error level when
 * L_max > 1, Sec. 5): solver 0 = CG, 1 = BiCGStab.  precision NL_PREC_FP64 runs the Krylov
 * method in FP64; any other value runs it in FP32 inside FP64 iterative refinement
 * (residuals r = F~ - A u in FP64; each inner FP32 solve stops at 1e-5 of its right-hand
 * side while the remaining factor q = rtol ||F~|| / ||r|| is below 1e-6, else at q / 2
 * clamped to [1e-6, 1e-3]).  Stops when ||F~ - A u|| <= rtol ||F~|| (free rows)
 * or after max_iter iterations (total inner iterations).  u_out: host, n_vert values (free
 * nodes: W; constrained nodes: g).  iters, final_rel_res may be NULL.  The solve runs on the
 * stream of the matrix's mesh; when that stream can be captured (any stream but the legacy
 * default stream), every batch of 8 iterations after the first is replayed from a CUDA graph.
 * Errors: NL_ENOTCONV when max_iter ran out (u_out still written). */
nl_status nl_solve(nl_matrix* A, const nl_vector* rhs, const double* g_nodes, int solver,
                   double rtol, int max_iter, nl_precision precision, double* u_out,
                   int* iters, double* final_rel_res);

/* ---- batched assembly: many problems in one launch -----------------------------------
 * The paper assembles one problem at a time; a plan is this library's way to keep the GPU
 * full with many small or uneven ones.  A plan assembles n problems (mesh, pairs, kernel,
 * Algorithm 1 levels) of one dimension in one precision: a single persistent launch of the
 * assembly kernel runs over the concatenated pair lists (every warp takes chunks of pairs
 * from one counter, so pairs of different refinement depth and problems of different sizes
 * share the grid until the last chunk), then one scatter launch and, for the FP32 paths, one
 * diagonal launch cover all problems.  Problem k's values equal those of nl_assemble with the
 * same arguments up to the order of FP64 additions.  Kernels, delta, eps and levels may
 * differ between problems.  flags:
 *   NL_PLAN_AUTOTUNE  time candidate launch shapes of the assembly kernel (warps per CTA,
 *                     CTAs per SM, pairs per grab of the counter) on the plan's problems at
 *                     creation and keep the fastest (nl_plan_shape reports it);
 *   NL_PLAN_GRAPH     capture one execution (clears and kernels) into a CUDA graph at
 *                     creation; every nl_plan_execute replays it.
 * cuda_stream: the stream the plan runs on (NULL: the plan creates its own non-blocking
 * stream).  The plan holds references to the pairs (and through them the meshes), owns the
 * values of all problems, its block buffer ((D+1)^2 values per pair of all problems, FP32 or
 * FP64) and its counters, and allocates only in nl_plan_create.
 * Errors: NL_EINVAL for NULL arguments, n < 1, mixed dimensions, pairs of another mesh,
 * delta/eps that differ from the pairs', or invalid kernel/levels/precision (as nl_assemble);
 * NL_ENOMEM if the block buffer exceeds half of the free device memory. */
typedef struct nl_plan nl_plan;
#define NL_PLAN_AUTOTUNE 1
#define NL_PLAN_GRAPH 2
nl_status nl_plan_create(int n, nl_mesh* const* meshes, nl_pairs* const* pairs,
                         const nl_kernel_params* kps, const nl_quad_params* qps,
                         nl_precision precision, int flags, void* cuda_stream, nl_plan** out);
/* Enqueues one execution on the plan's stream and returns (asynchronous). */
nl_status nl_plan_execute(nl_plan* plan);
/* Waits for the last execution and checks its device error word (NL_EINTERNAL as in
 * nl_assemble).  stats: NULL or n entries; ms_assemble is the GPU time of the whole last
 * execution (all problems). */
nl_status nl_plan_sync(nl_plan* plan, nl_assemble_stats* stats);
/* Problem k's values: device pointer (valid until nl_plan_destroy) and count. */
nl_status nl_plan_values(const nl_plan* plan, int k, double** values, int64_t* nnz);
/* Host copy of problem k's nnz values (waits for the plan's stream). */
nl_status nl_plan_export(const nl_plan* plan, int k, double* values);
/* A matrix handle with a copy of problem k's values, for nl_rhs / nl_solve (*A is created,
 * or overwritten if it is a matrix of the same pattern). */
nl_status nl_plan_matrix(const nl_plan* plan, int k, nl_matrix** A);
/* The launch shape in use (0 = default), the tuned kernel time (0 if not tuned) and whether
 * executions replay a CUDA graph; any pointer may be NULL. */
nl_status nl_plan_shape(const nl_plan* plan, int* warps, int* ctas_per_sm, int* chunk,
                        double* tuned_ms, int* graph);
void nl_plan_destroy(nl_plan* plan);

/* ---- serving: continuous batching of assemble + solve requests ----------------------
 * A request is one volume-constrained Poisson problem (Sec. 2) on a structured box mesh,
 * assembled (Sec. 5) and solved as above, with the manufactured solution u = g on Gamma and
 * f = -Laplace(u) (= -L_eps u for these polynomials, Sec. 6). */
typedef struct {
  int dim;
  int32_t cells[3];  /* structured box mesh as in nl_mesh_create_box */
  double h, lo[3];
  int32_t layer;
  double jitter;
  uint64_t seed;
  nl_kernel_params kernel;
  nl_quad_params quad;
  nl_precision precision;
  int ms;            /* manufactured solution: 0 = 1+sum x, 1 = sum x^2, 2 = sum x^3 */
  int solver;        /* 0 CG, 1 BiCGStab */
  double rtol;
  int max_iter;
  double* u_out;     /* nullable host array of n_vert values that receives u_h; it must stay
                        valid until the result has been taken */
} nl_request;

typedef struct {
  nl_status status;
  int iters;
  double rel_res;
  double l2_err_omega;   /* ||u - u_h|| over Omega (degree-5 rule per element) */
  int64_t n_pairs, n_point_pairs, nnz, n_vert;
  double t_submit_ms, t_start_ms, t_done_ms; /* host clock since nl_serve_create */
  char message[160];     /* error message when status != NL_OK, "" otherwise */
  int32_t group;         /* batched group the request was assembled in (-1: alone) */
} nl_result;

/* device_mem_budget: bytes the server may hold at once (>= 64 MiB); max_slots (1..64):
 * worker threads, each with its own CUDA stream of the device that is current at creation.
 * A request is admitted when a slot is free and its estimated footprint fits in the budget
 * left by the requests in flight (a request larger than the whole budget runs when nothing
 * else does); requests wait in arrival order.  Continuous batching: when a slot admits a
 * small request (at most about 4e6 element pairs), later small requests of the same dimension
 * and precision class (FP64 or not) that are waiting and fit the budget join it, up to 16:
 * their meshes and patterns are built, one batched plan (nl_plan_*) assembles all of them in a
 * single launch, and each is solved and completed on its own; the result's `group` says which
 * requests shared a launch.  Requests on different slots run concurrently on the device; each
 * keeps its mesh, pattern, matrix and Krylov vectors on the device while it runs.
 * nl_serve_destroy lets running requests finish and drops the ones still waiting. */
nl_status nl_serve_create(size_t device_mem_budget, int max_slots, nl_server** out);
nl_status nl_serve_submit(nl_server* s, const nl_request* req, uint64_t* ticket);
/* NL_EBUSY while the request is not finished; otherwise the result (once). */
nl_status nl_serve_poll(nl_server* s, uint64_t ticket, nl_result* out);
/* Waits at most timeout_ms (NL_ETIMEOUT after that). */
nl_status nl_serve_wait(nl_server* s, uint64_t ticket, double timeout_ms, nl_result* out);
nl_status nl_serve_stats(nl_server* s, double* p50_ms, double* p99_ms, double* solves_per_s);
void nl_serve_destroy(nl_server* s);

/* ---- host-side tables (no device work; usable without a GPU) ------------------------- */
/* The degree-5 simplex rule used by the kernels: bary[npts*(dim+1)], w[npts] (sum 1).
 * Returns the number of points, or -1. */
int nl_quad_rule(int dim, double* bary, double* w);
/* C_{delta,eps} as nl_assemble uses it (kappa = 1, no override). */
double nl_kernel_constant(int dim, int kernel, double delta, double eps);

#ifdef __cplusplus
}
#endif
#endif
