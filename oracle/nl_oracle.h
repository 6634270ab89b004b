/* nl_oracle.h -- plain FP64 CPU oracle for the mollified nonlocal FE assembly of
 * Aulisa, Capodaglio, Chierici, D'Elia, "Efficient quadrature rules for finite
 * element discretizations of nonlocal equations" (arXiv 2101.08825).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or constant generator with the CUDA library; the only
 * thing the two sides have in common are the seeded input meshes.
 *
 * Conventions
 *   coords : SoA, coords[k*n_vert + v] = k-th coordinate of vertex v (k < dim)
 *   conn   : element-major, conn[e*npe + a] = a-th node of element e (npe nodes per
 *            element: P1 simplices dim+1, P2 triangles 6, quadrilaterals 4 (Q1) or 9 (Q2))
 *   pairs  : m-major lists, pair_off[m]..pair_off[m+1] index pair_l, l ascending
 *   CSR    : row_ptr[n_vert+1] (int64), col (int32), columns sorted ascending
 */
#ifndef NL_ORACLE_H
#define NL_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define OR_KERNEL_CONST 0 /* eta = 1                       (Sec. 6)   */
#define OR_KERNEL_GAUSS 1 /* eta = exp(-r^2/delta^2)        (workload) */

#define OR_MS_LINEAR 0    /* u = 1 + sum_k x_k              (Sec. 6, consistency) */
#define OR_MS_QUADRATIC 1 /* u = sum_k x_k^2                                     */
#define OR_MS_CUBIC 2     /* u = sum_k x_k^3                (Table 2)            */
#define OR_MS_QUARTIC 3   /* u = sum_k x_k^4                (Table 3)            */

typedef struct {
  int dim;
  int64_t n_vert, n_elem;       /* n_vert: all nodes (P2: vertices and edge midpoints) */
  const double* coords;
  const int32_t* conn;          /* npe nodes per element: P1 dim+1; P2 triangles 6 */
  const uint8_t* elem_in_omega; /* 1 = element of Omega, 0 = of the layer Gamma */
  const uint8_t* node_free;     /* 1 = degree of freedom (node inside open Omega) */
  int order;                    /* 1 (or 0): P1; 2: P2 Lagrange triangles (vertices, then the
                                   midpoints of the edges (0,1), (1,2), (0,2)) */
  int cell;                     /* 0: simplices; 1: quadrilaterals (dim 2), vertices v0..v3
                                   counterclockwise, the images of the unit square's corners
                                   (0,0), (1,0), (1,1), (0,1) under the bilinear map; order 1:
                                   Q1 (the four vertices), order 2: Q2 (the vertices, the
                                   midpoints of the edges (0,1), (1,2), (2,3), (3,0), then the
                                   image of the square's centre), order 3: the 8-node
                                   serendipity element (the Q2 nodes without the centre);
                                   2: hexahedra (dim 3), vertices the images of the unit cube's
                                   corners (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1),
                                   (1,1,1), (0,1,1); order 1: Q1 (trilinear), order 2: Q2 (27
                                   nodes on the lattice of half steps: the vertices, the edge
                                   midpoints, the face centres, the centre) */
} or_mesh;

/* or_params.flags: the refinement test of Algorithm 1 uses the Euclidean variant of the
 * approximate minimum distance that Sec. 5.1 gives after eq. (mindistin) instead of eq.
 * (mindist).  The element pairs (eq. k_l) keep eq. (mindist). */
#define OR_MINDIST_L2 1

typedef struct {
  double delta, eps, C; /* horizon, mollifier half-width, kernel constant C_{delta,eps} */
  int kernel;           /* OR_KERNEL_* */
  int L_min, L_max;     /* Algorithm 1 refinement levels */
  int flags;            /* OR_MINDIST_L2 or 0 */
} or_params;

typedef struct {
  int64_t n_point_pairs;  /* (outer point, inner point) evaluations of gamma_eps */
  int64_t n_band_pairs;   /* of which delta-eps <= r <= delta+eps */
  int64_t n_integrations; /* (sub-element, m) integrations */
} or_stats;

/* Sec. 3, eq. (mollifier): the polynomial xi and the mollifier mu_{delta,eps}(r). */
double or_xi(double s);
double or_mu(double r, double delta, double eps);
/* Sec. 3, eq. (gamma): radial factor eta. */
double or_eta(int kernel, double r, double delta);
/* Sec. 6: C_{delta,eps}.  Constant kernel: the printed closed form.  Other kernels:
 * the value that makes L_eps u = Laplace(u) for quadratics, n / int |z|^2 eta mu dz. */
double or_kernel_constant(int dim, int kernel, double delta, double eps);
/* int z_1^p gamma_eps(|z|) dz over R^n for p = 2 or 4 with constant C (radial quadrature). */
double or_kernel_moment(int dim, int kernel, double delta, double eps, double C, int p);
/* n-point Gauss-Legendre rule on [-1, 1]; returns 0 on success. */
int or_gauss_legendre(int n, double* x, double* w);

/* Symmetric simplex rules of degree 5: 7 points (dim 2), 14 points (dim 3), solved from
 * their moment equations.  bary[q*(dim+1)+v], weights sum to 1.  Returns the number of
 * points, or -1 if Newton's method did not converge. */
int or_quad_rule(int dim, double* bary, double* w);

/* Sec. 5.1, eqs. (maxdist), (mindist) on axis-aligned boxes lo/hi of two point sets. */
double or_aprx_max_dist(int dim, const double* lo1, const double* hi1, const double* lo2,
                        const double* hi2);
double or_aprx_min_dist(int dim, const double* lo1, const double* hi1, const double* lo2,
                        const double* hi2);
/* Sec. 5.1, the Euclidean variant after eq. (mindistin): sqrt(sum_k max(0, d1^k, d2^k)^2). */
double or_aprx_min_dist_l2(int dim, const double* lo1, const double* hi1, const double* lo2,
                           const double* hi2);

/* Eq. (k_l): J = {(m, l) : aprx-min-dist(E_l, E_m) < delta + eps}, m-major, l ascending.
 * pair_off has n_elem+1 entries; pair_l has room for cap entries.  m_mask (nullable) keeps
 * only the lists of the selected m (the others are empty).  Returns the number of pairs
 * (which may exceed cap: then call again with a larger buffer), or -1 on error. */
int64_t or_pairs(const or_mesh* M, double delta, double eps, int64_t* pair_off, int32_t* pair_l,
                 int64_t cap, const uint8_t* m_mask);

/* Sparsity of A: row i holds the nodes of every l with (m, l) in J and i a node of m.
 * Returns nnz (row_ptr filled; col filled when cap >= nnz), or -1 on error. */
int64_t or_csr(const or_mesh* M, const int64_t* pair_off, const int32_t* pair_l, int64_t* row_ptr,
               int32_t* col, int64_t cap);

/* Sec. 5: A = 2 A^21 + 2 A^22 (Corollary 1, eqs. J21Nr, J22Nr) with Algorithm 1 on the outer
 * element.  values (nnz, zeroed here) follows row_ptr/col.  m_mask (nullable) restricts the
 * inner elements m: rows whose every element is selected are then complete.  Returns 0. */
int or_assemble(const or_mesh* M, const int64_t* pair_off, const int32_t* pair_l,
                const or_params* P, const int64_t* row_ptr, const int32_t* col, double* values,
                const uint8_t* m_mask, or_stats* stats);

/* Manufactured solution u and forcing f = -L_eps u (Sec. 2, eq. L). */
double or_ms_u(int ms, int dim, const double* x);
double or_ms_f(int ms, int dim, const double* x, int kernel, double delta, double eps, double C);

/* Sec. 2, eqs. (A-F), (weak-homo): F~_i = int_Omega f phi_i - sum_{k constrained} A_ik u(x_k)
 * for free i, 0 otherwise. */
int or_rhs(const or_mesh* M, const int64_t* row_ptr, const int32_t* col, const double* values,
           int ms, int kernel, double delta, double eps, double C, double* F);

/* Solves A_{free,free} W = F_free by dense Gaussian elimination with partial pivoting and
 * returns the nodal solution u_h (free nodes: W, constrained nodes: u(x_k)).  n_free <= 20000. */
int or_solve_dense(const or_mesh* M, const int64_t* row_ptr, const int32_t* col,
                   const double* values, const double* F, int ms, double* u_h);

/* L2 error of u_h against u over Omega (omega_only = 1) or Omega U Gamma (0). */
double or_l2_error(const or_mesh* M, const double* u_h, int ms, int omega_only);

#ifdef __cplusplus
}
#endif
#endif
