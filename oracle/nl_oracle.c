/* nl_oracle.c -- plain FP64 CPU oracle for the mollified nonlocal FE assembly of
 * Aulisa, Capodaglio, Chierici, D'Elia, "Efficient quadrature rules for finite
 * element discretizations of nonlocal equations" (arXiv 2101.08825).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library; the product path
 * never does.  It is deliberately slow and literal: every step follows the paper's
 * definitions in the paper's order and notation, in FP64, compiled with
 * -ffp-contract=off.  It shares no code with the CUDA library.
 *
 * Pins (tests/test_oracle_*.py): xi and mu against their closed-form properties,
 * C_{delta,eps} against an independent radial quadrature, the simplex rules against
 * exact monomial integrals, the box distances against exact point-set distances,
 * fully-interior pairs against closed-form local matrices, transition pairs against
 * brute-force uniform quadrature, zero row sums, exact symmetry at L_max = 1,
 * L_eps u = Laplace(u) on quadratics, and the printed Table 2 (TRI, linear) errors.
 * The other element families (P2 triangles and tetrahedra, Q1/Q2/serendipity
 * quadrilaterals and hexahedra with Gauss-Legendre product rules) are pinned the same
 * way, with their bases written out independently in the tests, and against the printed
 * TRI and QUAD columns of Tables 1-3 and the HEX linear column of Table 7.
 */
#include "nl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------
 * Sec. 3, eq. (mollifier).  The printed argument of xi reads ((delta-eps) - r)/eps,
 * which gives mu = xi(-1) = 0 at r = delta-eps and a negative second moment; the
 * reading used here is (delta - r)/eps, for which mu is C^4, equals 1 at r = delta-eps
 * and 0 at r = delta+eps, and reproduces the printed C_{delta,eps} of Sec. 6. */
double or_xi(double s) {
  double s2 = s * s;
  double s3 = s2 * s;
  double s5 = s3 * s2;
  double s7 = s5 * s2;
  double s9 = s7 * s2;
  return (128.0 + 315.0 * s - 420.0 * s3 + 378.0 * s5 - 180.0 * s7 + 35.0 * s9) / 256.0;
}

double or_mu(double r, double delta, double eps) {
  if (r < delta - eps) return 1.0;
  if (r > delta + eps) return 0.0;
  return or_xi((delta - r) / eps);
}

/* Sec. 3, eq. (gamma): gamma = C eta(|x-y|) 1(y in B_delta(x)).  eta = 1 in every test of
 * the paper (Sec. 6); the truncated Gaussian exp(-r^2/delta^2) is the second radial
 * profile of the workloads. */
double or_eta(int kernel, double r, double delta) {
  if (kernel == OR_KERNEL_GAUSS) return exp(-(r * r) / (delta * delta));
  return 1.0;
}

/* n-point Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's method on
 * the three-term recurrence, w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2). */
int or_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; i++) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* int_a^b r^q eta(r) mu(r) dr by 60-point Gauss-Legendre on [0, delta-eps] (mu = 1) and
 * [delta-eps, delta+eps] (mu = xi), where the integrand is smooth. */
static double radial_integral(int q, int kernel, double delta, double eps) {
  enum { NG = 60 };
  double gx[NG], gw[NG];
  or_gauss_legendre(NG, gx, gw);
  double pieces[3] = {0.0, delta - eps, delta + eps};
  double total = 0.0;
  for (int s = 0; s < 2; s++) {
    double a = pieces[s], b = pieces[s + 1];
    double half = 0.5 * (b - a), mid = 0.5 * (b + a);
    for (int i = 0; i < NG; i++) {
      double r = mid + half * gx[i];
      double rq = 1.0;
      for (int k = 0; k < q; k++) rq *= r;
      total += half * gw[i] * rq * or_eta(kernel, r, delta) * or_mu(r, delta, eps);
    }
  }
  return total;
}

/* int_{R^n} z_1^p gamma_eps(|z|) dz, p in {2, 4}, for gamma_eps = C eta mu (Sec. 3, eq.
 * approx-kernel).  In polar form: int z_1^2 f = (1/n) |S^{n-1}| int r^{n+1} f dr and
 * int z_1^4 f = 3/(n(n+2)) |S^{n-1}| int r^{n+3} f dr, |S^1| = 2 pi, |S^2| = 4 pi. */
double or_kernel_moment(int dim, int kernel, double delta, double eps, double C, int p) {
  double sphere = (dim == 2) ? 2.0 * OR_PI : 4.0 * OR_PI;
  if (p == 2) return C * sphere / dim * radial_integral(dim + 1, kernel, delta, eps);
  if (p == 4) return C * sphere * 3.0 / (dim * (dim + 2.0)) * radial_integral(dim + 3, kernel, delta, eps);
  return NAN;
}

/* Sec. 6: the scaling constants.  kappa (undefined in the paper) is read as 1. */
double or_kernel_constant(int dim, int kernel, double delta, double eps) {
  if (kernel == OR_KERNEL_CONST) {
    double t = eps / delta;
    double t2 = t * t;
    double t4 = t2 * t2;
    if (dim == 2) {
      double c_delta = 4.0 / (OR_PI * delta * delta * delta * delta);
      return c_delta / (1.0 + 6.0 / 11.0 * t2 + 3.0 / 143.0 * t4);
    }
    double c_delta = 15.0 / (4.0 * OR_PI * delta * delta * delta * delta * delta);
    return c_delta / (1.0 + 10.0 / 11.0 * t2 + 15.0 / 143.0 * t4);
  }
  /* L_eps u = Laplace(u) for quadratic u  <=>  int z_1^2 gamma_eps dz = 1. */
  return 1.0 / or_kernel_moment(dim, kernel, delta, eps, 1.0, 2);
}

/* ------------------------------------------------------------------------------------
 * Degree-5 symmetric simplex rules (Sec. 6: the 7-point rule for triangles; the
 * 14-point tetrahedral rule of the 3D workloads).  Each rule is a union of symmetry
 * orbits of barycentric points; the unknowns (orbit weights and parameters) solve the
 * moment equations sum_q w_q lambda^alpha(q) = n! alpha! / (|alpha| + n)! for a set of
 * monomials spanning the symmetric polynomials of degree <= 5. */

/* The moment equations are solved in long double (80-bit on x86-64, 128-bit on
 * aarch64) and the result is rounded to double, so the tables are correct to the last
 * bit or so on both machines. */
typedef long double ld;

/* Fills the distinct permutations of an orbit; returns how many. */
static int orbit_points(int dim, int type, ld a, ld pts[][4]) {
  if (dim == 2) {
    if (type == 0) { /* centroid */
      pts[0][0] = pts[0][1] = pts[0][2] = 1.0L / 3.0L;
      return 1;
    }
    ld b = 1.0L - 2.0L * a; /* (a, a, b) */
    ld base[3][3] = {{a, a, b}, {a, b, a}, {b, a, a}};
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) pts[i][k] = base[i][k];
    return 3;
  }
  if (type == 1) { /* (a, a, a, 1-3a) */
    ld b = 1.0L - 3.0L * a;
    for (int i = 0; i < 4; i++)
      for (int k = 0; k < 4; k++) pts[i][k] = (k == 3 - i) ? b : a;
    return 4;
  }
  /* type 2: (a, a, 1/2-a, 1/2-a) */
  ld b = 0.5L - a;
  int n = 0;
  for (int i = 0; i < 4; i++)
    for (int j = i + 1; j < 4; j++) {
      for (int k = 0; k < 4; k++) pts[n][k] = (k == i || k == j) ? a : b;
      n++;
    }
  return 6;
}

static ld factorial(int n) {
  ld f = 1.0L;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}

/* Moment test functions: lambda_1^k (k = 0, 2, 3, 4, 5) and, in 3D, lambda_1^2 lambda_2^2. */
static const int tri_alpha[5][3] = {{0, 0, 0}, {2, 0, 0}, {3, 0, 0}, {4, 0, 0}, {5, 0, 0}};
static const int tet_alpha[6][4] = {{0, 0, 0, 0}, {2, 0, 0, 0}, {3, 0, 0, 0},
                                    {4, 0, 0, 0}, {5, 0, 0, 0}, {2, 2, 0, 0}};

static ld mono(int dim, const int* alpha, const ld* lam) {
  ld v = 1.0L;
  for (int k = 0; k <= dim; k++)
    for (int e = 0; e < alpha[k]; e++) v *= lam[k];
  return v;
}

static ld mono_exact(int dim, const int* alpha) {
  int s = 0;
  ld num = factorial(dim);
  for (int k = 0; k <= dim; k++) {
    s += alpha[k];
    num *= factorial(alpha[k]);
  }
  return num / factorial(s + dim);
}

/* Rule layout: 2D unknowns u = (w0, w1, a1, w2, a2) for orbits (centroid, S21(a1),
 * S21(a2)); 3D u = (w1, a, w2, b, w3, c) for orbits (S31(a), S31(b), S22(c)). */
static int rule_points(int dim, const ld* u, ld pts[][4], ld* w) {
  ld tmp[8][4];
  int n = 0;
  for (int o = 0; o < 3; o++) {
    int type;
    ld wt, par;
    if (dim == 2) {
      type = (o == 0) ? 0 : 1;
      wt = (o == 0) ? u[0] : u[2 * o - 1];
      par = (o == 0) ? 0.0L : u[2 * o];
    } else {
      type = (o < 2) ? 1 : 2;
      wt = u[2 * o];
      par = u[2 * o + 1];
    }
    int c = orbit_points(dim, type, par, tmp);
    for (int i = 0; i < c; i++) {
      for (int k = 0; k < 4; k++) pts[n][k] = tmp[i][k];
      w[n] = wt;
      n++;
    }
  }
  return n;
}

static void rule_residual(int dim, const ld* u, ld* res) {
  ld pts[16][4], w[16];
  int n = rule_points(dim, u, pts, w);
  int neq = (dim == 2) ? 5 : 6;
  for (int j = 0; j < neq; j++) {
    const int* alpha = (dim == 2) ? tri_alpha[j] : tet_alpha[j];
    ld s = 0.0L;
    for (int q = 0; q < n; q++) s += w[q] * mono(dim, alpha, pts[q]);
    res[j] = s - mono_exact(dim, alpha);
  }
}

static int dense_solve_ld(int n, ld* A, ld* b) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    for (int i = k + 1; i < n; i++)
      if (fabsl(A[i * n + k]) > fabsl(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0L) return -1;
    for (int j = 0; j < n; j++) {
      ld t = A[k * n + j];
      A[k * n + j] = A[piv * n + j];
      A[piv * n + j] = t;
    }
    ld t = b[k];
    b[k] = b[piv];
    b[piv] = t;
    for (int i = k + 1; i < n; i++) {
      ld f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    ld s = b[i];
    for (int j = i + 1; j < n; j++) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return 0;
}

int or_quad_rule(int dim, double* bary, double* w) {
  /* Starting points near the positive interior solution; Newton's method with a
   * central-difference Jacobian then solves the moment equations. */
  ld u[6];
  int nu;
  if (dim == 2) {
    ld u0[5] = {0.22L, 0.13L, 0.10L, 0.13L, 0.47L};
    memcpy(u, u0, sizeof u0);
    nu = 5;
  } else if (dim == 3) {
    ld u0[6] = {0.07L, 0.09L, 0.11L, 0.31L, 0.04L, 0.045L};
    memcpy(u, u0, sizeof u0);
    nu = 6;
  } else {
    return -1;
  }
  ld res[6], rp[6], rm[6], J[36];
  for (int it = 0; it < 60; it++) {
    rule_residual(dim, u, res);
    for (int c = 0; c < nu; c++) {
      ld save = u[c], hstep = 1e-9L;
      u[c] = save + hstep;
      rule_residual(dim, u, rp);
      u[c] = save - hstep;
      rule_residual(dim, u, rm);
      u[c] = save;
      for (int j = 0; j < nu; j++) J[j * nu + c] = (rp[j] - rm[j]) / (2.0L * hstep);
    }
    for (int j = 0; j < nu; j++) res[j] = -res[j];
    if (dense_solve_ld(nu, J, res) != 0) return -1;
    for (int c = 0; c < nu; c++) u[c] += res[c];
  }
  rule_residual(dim, u, res);
  ld nr = 0.0L;
  for (int j = 0; j < nu; j++) nr += fabsl(res[j]);
  if (!(nr < 1e-17L)) return -1;
  ld pts[16][4], ww[16];
  int n = rule_points(dim, u, pts, ww);
  for (int q = 0; q < n; q++) {
    if (!(ww[q] > 0.0L)) return -1;
    for (int k = 0; k <= dim; k++) {
      if (!(pts[q][k] > 0.0L && pts[q][k] < 1.0L)) return -1;
      bary[q * (dim + 1) + k] = (double)pts[q][k];
    }
    w[q] = (double)ww[q];
  }
  return n;
}

/* Dense Gaussian elimination with partial pivoting; solves A x = b in place (b -> x). */
static int dense_solve(int n, double* A, double* b) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    for (int i = k + 1; i < n; i++)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
    if (A[(size_t)piv * n + k] == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; j++) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)piv * n + j];
        A[(size_t)piv * n + j] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int i = k + 1; i < n; i++) {
      double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = b[i];
    for (int j = i + 1; j < n; j++) s -= A[(size_t)i * n + j] * b[j];
    b[i] = s / A[(size_t)i * n + i];
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Sec. 5.1: approximate distances between the bounding boxes of E_l (lo1, hi1) and
 * E_m (lo2, hi2): d1^k = x^k_min - y^k_max, d2^k = y^k_min - x^k_max. */
double or_aprx_max_dist(int dim, const double* lo1, const double* hi1, const double* lo2,
                        const double* hi2) {
  double s = 0.0;
  for (int k = 0; k < dim; k++) { /* eq. (maxdist) */
    double d1 = lo1[k] - hi2[k];
    double d2 = lo2[k] - hi1[k];
    double a = d1 * d1, b = d2 * d2;
    s += (a > b) ? a : b;
  }
  return sqrt(s);
}

double or_aprx_min_dist(int dim, const double* lo1, const double* hi1, const double* lo2,
                        const double* hi2) {
  double m = 0.0;
  for (int k = 0; k < dim; k++) { /* eq. (mindist) */
    double d1 = lo1[k] - hi2[k];
    double d2 = lo2[k] - hi1[k];
    double t = (d1 > d2) ? d1 : d2;
    if (t > m) m = t;
  }
  return m;
}

/* The sharper variant that Sec. 5.1 states after eq. (mindistin) for kernels supported on a
 * Euclidean ball: the length of the vector of per-axis gaps max(0, d1^k, d2^k). */
double or_aprx_min_dist_l2(int dim, const double* lo1, const double* hi1, const double* lo2,
                           const double* hi2) {
  double s = 0.0;
  for (int k = 0; k < dim; k++) {
    double d1 = lo1[k] - hi2[k];
    double d2 = lo2[k] - hi1[k];
    double t = (d1 > d2) ? d1 : d2;
    if (t < 0.0) t = 0.0;
    s += t * t;
  }
  return sqrt(s);
}

/* ------------------------------------------------------------------------------------
 * Mesh helpers. */
/* Nodes per element: P1 simplices dim+1; P2 triangles 6 (the vertices, then the midpoints of
 * the edges (0,1), (1,2), (0,2)); P2 tetrahedra 10 (the vertices, then the midpoints of the
 * edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3)). */
static int npe(const or_mesh* M) {
  if (M->cell == 2) return (M->order == 2) ? 27 : (M->order == 3) ? 20 : 8;
  if (M->cell == 1) return (M->order == 2) ? 9 : (M->order == 3) ? 8 : 4;
  if (M->order == 2) return M->dim == 2 ? 6 : 10;
  return M->dim + 1;
}
/* Vertices per element: simplices dim+1, quadrilaterals 4 (hexahedra 8: hex_verts). */
static int nverts(const or_mesh* M) { return (M->cell == 1) ? 4 : M->dim + 1; }

/* The 8 vertices of hexahedron e (its first 8 nodes) and their box. */
static void hex_verts(const or_mesh* M, int64_t e, double V[8][3]) {
  int nb = npe(M);
  for (int a = 0; a < 8; a++) {
    int64_t v = M->conn[e * nb + a];
    for (int k = 0; k < 3; k++) V[a][k] = M->coords[k * M->n_vert + v];
  }
}
static void hex_bbox(const double V[8][3], double* lo, double* hi) {
  for (int k = 0; k < 3; k++) {
    lo[k] = V[0][k];
    hi[k] = V[0][k];
    for (int a = 1; a < 8; a++) {
      if (V[a][k] < lo[k]) lo[k] = V[a][k];
      if (V[a][k] > hi[k]) hi[k] = V[a][k];
    }
  }
}

/* The box of element e (any cell kind). */
static void elem_box(const or_mesh* M, int64_t e, double* lo, double* hi);

/* The element's Lagrange basis at the point with barycentric coordinates lam: P1 the
 * barycentric coordinates; P2 lam_a (2 lam_a - 1) at the vertices and 4 lam_a lam_b at the
 * edge midpoints, in the node order of npe(). */
static void basis(const or_mesh* M, const double* lam, double* phi) {
  if (M->order != 2) {
    for (int a = 0; a <= M->dim; a++) phi[a] = lam[a];
    return;
  }
  static const int e2[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  static const int e3[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
  int nv = M->dim + 1, ne = M->dim == 2 ? 3 : 6;
  for (int a = 0; a < nv; a++) phi[a] = lam[a] * (2.0 * lam[a] - 1.0);
  for (int j = 0; j < ne; j++) {
    const int* e = M->dim == 2 ? e2[j] : e3[j];
    phi[nv + j] = 4.0 * lam[e[0]] * lam[e[1]];
  }
}

/* The vertices of element e (the first nverts of its nodes). */
static void elem_verts(const or_mesh* M, int64_t e, double V[4][3]) {
  int nv = nverts(M), nb = npe(M);
  for (int a = 0; a < nv; a++) {
    int64_t v = M->conn[e * nb + a];
    for (int k = 0; k < 3; k++) V[a][k] = (k < M->dim) ? M->coords[k * M->n_vert + v] : 0.0;
  }
}

/* Box of the first nvx vertices of V. */
static void verts_bbox(int dim, int nvx, const double V[4][3], double* lo, double* hi) {
  for (int k = 0; k < dim; k++) {
    lo[k] = V[0][k];
    hi[k] = V[0][k];
    for (int a = 1; a < nvx; a++) {
      if (V[a][k] < lo[k]) lo[k] = V[a][k];
      if (V[a][k] > hi[k]) hi[k] = V[a][k];
    }
  }
}

static void elem_box(const or_mesh* M, int64_t e, double* lo, double* hi) {
  if (M->cell == 2) {
    double H[8][3];
    hex_verts(M, e, H);
    hex_bbox(H, lo, hi);
    return;
  }
  double V[4][3];
  elem_verts(M, e, V);
  verts_bbox(M->dim, nverts(M), V, lo, hi);
}

/* |det[v1-v0, ..., vn-v0]| / n! */
static double simplex_volume(int dim, const double V[4][3]) {
  if (dim == 2) {
    double a = V[1][0] - V[0][0], b = V[2][0] - V[0][0];
    double c = V[1][1] - V[0][1], d = V[2][1] - V[0][1];
    return fabs(a * d - b * c) / 2.0;
  }
  double m[3][3];
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) m[k][i] = V[i + 1][k] - V[0][k];
  double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
               m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
               m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
  return fabs(det) / 6.0;
}

/* P1 basis of the simplex V at x: the barycentric coordinates, from Cramer's rule on
 * sum_{a>=1} lambda_a (v_a - v_0) = x - v_0. */
static void barycentric(int dim, const double V[4][3], const double* x, double* lam) {
  if (dim == 2) {
    double a = V[1][0] - V[0][0], b = V[2][0] - V[0][0];
    double c = V[1][1] - V[0][1], d = V[2][1] - V[0][1];
    double rx = x[0] - V[0][0], ry = x[1] - V[0][1];
    double det = a * d - b * c;
    lam[1] = (rx * d - b * ry) / det;
    lam[2] = (a * ry - rx * c) / det;
    lam[0] = 1.0 - lam[1] - lam[2];
    return;
  }
  double m[3][3], r[3];
  for (int i = 0; i < 3; i++) {
    for (int k = 0; k < 3; k++) m[k][i] = V[i + 1][k] - V[0][k];
    r[i] = x[i] - V[0][i];
  }
  double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
               m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
               m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
  for (int c = 0; c < 3; c++) {
    double mc[3][3];
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) mc[i][k] = (k == c) ? r[i] : m[i][k];
    double dc = mc[0][0] * (mc[1][1] * mc[2][2] - mc[1][2] * mc[2][1]) -
                mc[0][1] * (mc[1][0] * mc[2][2] - mc[1][2] * mc[2][0]) +
                mc[0][2] * (mc[1][0] * mc[2][1] - mc[1][1] * mc[2][0]);
    lam[c + 1] = dc / det;
  }
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

static void midpoint(const double* a, const double* b, double* out) {
  for (int k = 0; k < 3; k++) out[k] = (a[k] + b[k]) * 0.5;
}

/* Midpoint refinement into 2^N children (Sec. 5).  Triangle: the three corner triangles
 * and the middle one.  Tetrahedron: Bey's rule, interior octahedron cut along the
 * diagonal x02-x13. */
static void split(int dim, const double V[4][3], double C[8][4][3]) {
  if (dim == 2) {
    double m01[3], m02[3], m12[3];
    midpoint(V[0], V[1], m01);
    midpoint(V[0], V[2], m02);
    midpoint(V[1], V[2], m12);
    const double* ch[4][3] = {{V[0], m01, m02}, {m01, V[1], m12}, {m02, m12, V[2]}, {m01, m12, m02}};
    for (int c = 0; c < 4; c++)
      for (int a = 0; a < 3; a++)
        for (int k = 0; k < 3; k++) C[c][a][k] = ch[c][a][k];
    return;
  }
  double x01[3], x02[3], x03[3], x12[3], x13[3], x23[3];
  midpoint(V[0], V[1], x01);
  midpoint(V[0], V[2], x02);
  midpoint(V[0], V[3], x03);
  midpoint(V[1], V[2], x12);
  midpoint(V[1], V[3], x13);
  midpoint(V[2], V[3], x23);
  const double* ch[8][4] = {{V[0], x01, x02, x03}, {x01, V[1], x12, x13}, {x02, x12, V[2], x23},
                            {x03, x13, x23, V[3]}, {x01, x02, x03, x13}, {x01, x02, x12, x13},
                            {x02, x03, x13, x23},  {x02, x12, x13, x23}};
  for (int c = 0; c < 8; c++)
    for (int a = 0; a < 4; a++)
      for (int k = 0; k < 3; k++) C[c][a][k] = ch[c][a][k];
}

/* ------------------------------------------------------------------------------------
 * Eq. (k_l): the element pairs. */
int64_t or_pairs(const or_mesh* M, double delta, double eps, int64_t* pair_off, int32_t* pair_l,
                 int64_t cap, const uint8_t* m_mask) {
  int dim = M->dim;
  int64_t n = M->n_elem;
  double* lo = (double*)malloc(sizeof(double) * 3 * n);
  double* hi = (double*)malloc(sizeof(double) * 3 * n);
  if (!lo || !hi) {
    free(lo);
    free(hi);
    return -1;
  }
  for (int64_t e = 0; e < n; e++) elem_box(M, e, lo + 3 * e, hi + 3 * e);
  double reach = delta + eps;
  int64_t cnt = 0;
  for (int64_t m = 0; m < n; m++) {
    pair_off[m] = cnt;
    if (m_mask && !m_mask[m]) continue;
    for (int64_t l = 0; l < n; l++) {
      if (or_aprx_min_dist(dim, lo + 3 * l, hi + 3 * l, lo + 3 * m, hi + 3 * m) < reach) {
        if (cnt < cap) pair_l[cnt] = (int32_t)l;
        cnt++;
      }
    }
  }
  pair_off[n] = cnt;
  free(lo);
  free(hi);
  return cnt;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* The entries (i, j) that Eqs. (J21Nr), (J22Nr) can touch: i a node of m, j a node of m or
 * of l, (m, l) in J (l = m is in J, so the nodes of m are included). */
int64_t or_csr(const or_mesh* M, const int64_t* pair_off, const int32_t* pair_l, int64_t* row_ptr,
               int32_t* col, int64_t cap) {
  int nv = npe(M);
  int64_t nV = M->n_vert, nE = M->n_elem;
  /* node -> elements */
  int64_t* deg = (int64_t*)calloc(nV + 1, sizeof(int64_t));
  int64_t* n2e = (int64_t*)malloc(sizeof(int64_t) * nE * nv + 1);
  int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (nV + 1));
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * nV);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * nV);
  if (!deg || !n2e || !fillp || !mark || !buf) {
    free(deg), free(n2e), free(fillp), free(mark), free(buf);
    return -1;
  }
  for (int64_t e = 0; e < nE; e++)
    for (int a = 0; a < nv; a++) deg[M->conn[e * nv + a] + 1]++;
  for (int64_t v = 0; v < nV; v++) deg[v + 1] += deg[v];
  for (int64_t v = 0; v <= nV; v++) fillp[v] = deg[v];
  for (int64_t e = 0; e < nE; e++)
    for (int a = 0; a < nv; a++) n2e[fillp[M->conn[e * nv + a]]++] = e;
  for (int64_t v = 0; v < nV; v++) mark[v] = -1;
  int64_t nnz = 0;
  for (int64_t i = 0; i < nV; i++) {
    row_ptr[i] = nnz;
    int64_t cnt = 0;
    for (int64_t t = deg[i]; t < deg[i + 1]; t++) {
      int64_t m = n2e[t];
      for (int64_t p = pair_off[m]; p < pair_off[m + 1]; p++) {
        int64_t l = pair_l[p];
        for (int c = 0; c < nv; c++) {
          int32_t j = M->conn[l * nv + c];
          if (mark[j] != i) {
            mark[j] = i;
            buf[cnt++] = j;
          }
        }
      }
    }
    qsort(buf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    if (col && nnz + cnt <= cap) memcpy(col + nnz, buf, sizeof(int32_t) * cnt);
    nnz += cnt;
  }
  row_ptr[nV] = nnz;
  free(deg), free(n2e), free(fillp), free(mark), free(buf);
  return nnz;
}

static double* csr_entry(const int64_t* row_ptr, const int32_t* col, double* values, int64_t i,
                         int32_t j) {
  int64_t lo = row_ptr[i], hi = row_ptr[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] == j) return values + mid;
    if (col[mid] < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return NULL;
}

/* ------------------------------------------------------------------------------------
 * Sec. 5: Algorithm 1 and the element sums (J21Nr), (J22Nr). */
typedef struct {
  const or_mesh* M;
  const or_params* P;
  int dim, nv, nq, nb; /* nv: vertices (dim+1); nb: nodes (basis functions) per element */
  double qb[16][4], qw[16];
  const double* lo; /* element boxes (3 per element) */
  const double* hi;
  int64_t l;
  double Vl[4][3];
  const int64_t* row_ptr;
  const int32_t* col;
  double* values;
  or_stats* st;
  int error;
} actx;

/* Integration(E', J'): for every m in J', Q2 on the sub-element E' (outer variable x, test
 * functions of l) and Q1 on E_m (inner variable y).  Adds
 *   2 A^22_ij : 2 sum w_x w_y gamma_eps(x,y) phi^m_i(y) phi^m_j(y)     (eq. J22Nr)
 *   2 A^21_ij : -2 sum w_x w_y gamma_eps(x,y) phi^m_i(y) phi^l_j(x)    (eq. J21Nr; the minus
 *              sign of eq. J21 is restored, it is missing in the discrete version)
 * The finite sum over (x, m, y) is accumulated per m into the local blocks S (i, j in m)
 * and X (i in m, j in l) before it is added to A. */
static void integration(actx* c, const double E[4][3], const int32_t* J, int64_t nJ) {
  int dim = c->dim, nv = c->nv, nq = c->nq, nb = c->nb;
  const or_params* P = c->P;
  double vol = simplex_volume(dim, E);
  double xq[16][3], wx[16], phil[16][10], phim[16][10];
  for (int q = 0; q < nq; q++) {
    for (int k = 0; k < 3; k++) {
      double s = 0.0;
      for (int v = 0; v < nv; v++) s += c->qb[q][v] * E[v][k];
      xq[q][k] = s;
    }
    wx[q] = c->qw[q] * vol;
    double lam[4];
    barycentric(dim, c->Vl, xq[q], lam);
    basis(c->M, lam, phil[q]);     /* basis of l at the outer point */
    basis(c->M, c->qb[q], phim[q]); /* basis of m at its inner point q */
  }
  for (int64_t t = 0; t < nJ; t++) {
    int64_t m = J[t];
    double Vm[4][3];
    elem_verts(c->M, m, Vm);
    double volm = simplex_volume(dim, Vm);
    double S[10][10] = {{0}}, X[10][10] = {{0}};
    for (int q = 0; q < nq; q++) {
      for (int p = 0; p < nq; p++) {
        double y[3];
        for (int k = 0; k < 3; k++) {
          double s = 0.0;
          for (int v = 0; v < nv; v++) s += c->qb[p][v] * Vm[v][k];
          y[k] = s;
        }
        double wy = c->qw[p] * volm;
        double r2 = 0.0;
        for (int k = 0; k < dim; k++) r2 += (xq[q][k] - y[k]) * (xq[q][k] - y[k]);
        double r = sqrt(r2);
        double G = wx[q] * wy * P->C * or_eta(P->kernel, r, P->delta) * or_mu(r, P->delta, P->eps);
        c->st->n_point_pairs++;
        if (r >= P->delta - P->eps && r <= P->delta + P->eps) c->st->n_band_pairs++;
        for (int a = 0; a < nb; a++) {
          double phia = phim[p][a]; /* phi^m_a(y_p) */
          for (int b = 0; b < nb; b++) S[a][b] += G * phia * phim[p][b];
          for (int d = 0; d < nb; d++) X[a][d] += G * phia * phil[q][d];
        }
      }
    }
    c->st->n_integrations++;
    for (int a = 0; a < nb; a++) {
      int64_t i = c->M->conn[m * nb + a];
      for (int b = 0; b < nb; b++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[m * nb + b]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e += 2.0 * S[a][b];
      }
      for (int d = 0; d < nb; d++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[c->l * nb + d]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e -= 2.0 * X[a][d];
      }
    }
  }
}

/* Algorithm 1, Adaptive Integration(L_min, L_max, L_cur, E_l, J_l). */
static void adaptive_integration(actx* c, int L_cur, const double E[4][3], const int32_t* J,
                                 int64_t nJ) {
  const or_params* P = c->P;
  int dim = c->dim;
  int nchild = (dim == 2) ? 4 : 8;
  if (L_cur < P->L_min) {
    double C[8][4][3];
    split(dim, E, C);
    for (int i = 0; i < nchild; i++) adaptive_integration(c, L_cur + 1, C[i], J, nJ);
    return;
  }
  if (L_cur == P->L_max) {
    integration(c, E, J, nJ);
    return;
  }
  int32_t* Jint = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  int32_t* Jref = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  if (!Jint || !Jref) {
    free(Jint), free(Jref);
    c->error = 1;
    return;
  }
  int64_t nint = 0, nref = 0;
  double lo[3], hi[3];
  verts_bbox(dim, dim + 1, E, lo, hi);
  for (int64_t t = 0; t < nJ; t++) {
    int64_t m = J[t];
    double amin = (P->flags & OR_MINDIST_L2)
                      ? or_aprx_min_dist_l2(dim, lo, hi, c->lo + 3 * m, c->hi + 3 * m)
                      : or_aprx_min_dist(dim, lo, hi, c->lo + 3 * m, c->hi + 3 * m);
    if (or_aprx_max_dist(dim, lo, hi, c->lo + 3 * m, c->hi + 3 * m) < P->delta - P->eps)
      Jint[nint++] = (int32_t)m;
    else if (amin < P->delta + P->eps)
      Jref[nref++] = (int32_t)m;
  }
  if (nint > 0) integration(c, E, Jint, nint);
  if (nref > 0) {
    double C[8][4][3];
    split(dim, E, C);
    for (int i = 0; i < nchild; i++) adaptive_integration(c, L_cur + 1, C[i], Jref, nref);
  }
  free(Jint);
  free(Jref);
}

/* ------------------------------------------------------------------------------------
 * Quadrilateral elements (Sec. 6: the QUAD meshes, the Gauss-Legendre 3x3 product rule for
 * both the inner and the outer integral).  An element is the image of the unit square
 * under the bilinear map F(s,t) = (1-s)(1-t) v0 + s(1-t) v1 + s t v2 + (1-s) t v3.  A
 * sub-element of Algorithm 1 is the image of a sub-square [s0, s0+len] x [t0, t0+len] of
 * l's unit square; its physical vertices (for the box distances of Sec. 5.1) come from the
 * parent's by midpoints, the centre as the midpoint of the midpoints of the edges (0,1) and
 * (2,3). */
typedef struct {
  double V[4][3];      /* physical vertices */
  double s0, t0, len;  /* the sub-square of l's unit square */
} qsub;

/* 1D Lagrange basis of degree 1 or 2 at s (nodes 0, 1 or 0, 1/2, 1). */
static void lagrange1d(int order, double s, double* L) {
  if (order == 2) {
    L[0] = 2.0 * (s - 0.5) * (s - 1.0);
    L[1] = 4.0 * s * (1.0 - s);
    L[2] = 2.0 * s * (s - 0.5);
  } else {
    L[0] = 1.0 - s;
    L[1] = s;
  }
}

/* Q1 / Q2 basis at (s, t), nodes in the mesh's order: Q1 the vertices (0,0), (1,0), (1,1),
 * (0,1); Q2 the vertices, the midpoints of the edges (0,1), (1,2), (2,3), (3,0), the centre.
 * Order 3, the serendipity element (the Q2 nodes without the centre): with xi = 2s - 1,
 * eta = 2t - 1 and a node at (xi_a, eta_a), the corner functions
 * (1 + xi xi_a)(1 + eta eta_a)(xi xi_a + eta eta_a - 1)/4 and the edge functions
 * (1 - xi^2)(1 + eta eta_a)/2 (xi_a = 0) or (1 + xi xi_a)(1 - eta^2)/2 (eta_a = 0). */
static void quad_basis(int order, double s, double t, double* phi) {
  if (order == 3) {
    static const double nd[8][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}, {0, -1}, {1, 0}, {0, 1}, {-1, 0}};
    double xi = 2.0 * s - 1.0, eta = 2.0 * t - 1.0;
    for (int a = 0; a < 8; a++) {
      double xa = nd[a][0], ya = nd[a][1];
      if (a < 4)
        phi[a] = 0.25 * (1.0 + xi * xa) * (1.0 + eta * ya) * (xi * xa + eta * ya - 1.0);
      else if (xa == 0.0)
        phi[a] = 0.5 * (1.0 - xi * xi) * (1.0 + eta * ya);
      else
        phi[a] = 0.5 * (1.0 + xi * xa) * (1.0 - eta * eta);
    }
    return;
  }
  double Ls[3], Lt[3];
  lagrange1d(order, s, Ls);
  lagrange1d(order, t, Lt);
  if (order != 2) {
    phi[0] = Ls[0] * Lt[0];
    phi[1] = Ls[1] * Lt[0];
    phi[2] = Ls[1] * Lt[1];
    phi[3] = Ls[0] * Lt[1];
    return;
  }
  static const int ij[9][2] = {{0, 0}, {2, 0}, {2, 2}, {0, 2}, {1, 0}, {2, 1}, {1, 2}, {0, 1}, {1, 1}};
  for (int a = 0; a < 9; a++) phi[a] = Ls[ij[a][0]] * Lt[ij[a][1]];
}

/* x = F(s,t) for the quadrilateral V and |det DF(s,t)|. */
static void quad_map(const double V[4][3], double s, double t, double* x, double* detJ) {
  double N[4] = {(1.0 - s) * (1.0 - t), s * (1.0 - t), s * t, (1.0 - s) * t};
  double xs[2], xt[2];
  for (int k = 0; k < 3; k++) x[k] = N[0] * V[0][k] + N[1] * V[1][k] + N[2] * V[2][k] + N[3] * V[3][k];
  for (int k = 0; k < 2; k++) {
    xs[k] = (1.0 - t) * (V[1][k] - V[0][k]) + t * (V[2][k] - V[3][k]);
    xt[k] = (1.0 - s) * (V[3][k] - V[0][k]) + s * (V[2][k] - V[1][k]);
  }
  *detJ = fabs(xs[0] * xt[1] - xs[1] * xt[0]);
}

/* Gauss-Legendre 3x3 on the unit square: points (g[i], g[j]), weights gw[i] gw[j]. */
static void gl3_unit(double* g, double* gw) {
  double x[3], w[3];
  or_gauss_legendre(3, x, w);
  for (int i = 0; i < 3; i++) {
    g[i] = 0.5 * (x[i] + 1.0);
    gw[i] = 0.5 * w[i];
  }
}

/* The four children of a quadrilateral sub-element (Sec. 5, midpoint refinement). */
static void quad_split(const qsub* E, qsub C[4]) {
  double m01[3], m12[3], m23[3], m30[3], ce[3];
  midpoint(E->V[0], E->V[1], m01);
  midpoint(E->V[1], E->V[2], m12);
  midpoint(E->V[2], E->V[3], m23);
  midpoint(E->V[3], E->V[0], m30);
  midpoint(m01, m23, ce);
  const double* ch[4][4] = {{E->V[0], m01, ce, m30}, {m01, E->V[1], m12, ce},
                            {ce, m12, E->V[2], m23}, {m30, ce, m23, E->V[3]}};
  const double h = 0.5 * E->len;
  const double org[4][2] = {{0.0, 0.0}, {h, 0.0}, {h, h}, {0.0, h}};
  for (int c = 0; c < 4; c++) {
    for (int a = 0; a < 4; a++)
      for (int k = 0; k < 3; k++) C[c].V[a][k] = ch[c][a][k];
    C[c].s0 = E->s0 + org[c][0];
    C[c].t0 = E->t0 + org[c][1];
    C[c].len = h;
  }
}

/* Integration(E', J') on a quadrilateral sub-element: the sums of integration() with the
 * outer points x = F_l(s0 + len g_i, t0 + len g_j), weights w_i w_j len^2 |det DF_l|, the
 * basis of l at those reference points, and the inner points y = F_m(g_i, g_j) with weights
 * w_i w_j |det DF_m| and the basis of m there. */
static void integration_quad(actx* c, const qsub* E, const int32_t* J, int64_t nJ) {
  const or_params* P = c->P;
  int nb = c->nb, order = c->M->order;
  double g[3], gw[3];
  gl3_unit(g, gw);
  double xq[9][3], wx[9], phil[9][9], phim[9][9], gq[9][2], gwq[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      int q = 3 * i + j;
      gq[q][0] = g[i];
      gq[q][1] = g[j];
      gwq[q] = gw[i] * gw[j];
      double s = E->s0 + E->len * g[i], t = E->t0 + E->len * g[j], det;
      quad_map(c->Vl, s, t, xq[q], &det);
      wx[q] = gwq[q] * E->len * E->len * det;
      quad_basis(order, s, t, phil[q]);
      quad_basis(order, g[i], g[j], phim[q]);
    }
  for (int64_t tt = 0; tt < nJ; tt++) {
    int64_t m = J[tt];
    double Vm[4][3];
    elem_verts(c->M, m, Vm);
    double S[9][9] = {{0}}, X[9][9] = {{0}};
    for (int q = 0; q < 9; q++) {
      for (int p = 0; p < 9; p++) {
        double y[3], detm;
        quad_map(Vm, gq[p][0], gq[p][1], y, &detm);
        double wy = gwq[p] * detm;
        double r2 = 0.0;
        for (int k = 0; k < 2; k++) r2 += (xq[q][k] - y[k]) * (xq[q][k] - y[k]);
        double r = sqrt(r2);
        double G = wx[q] * wy * P->C * or_eta(P->kernel, r, P->delta) * or_mu(r, P->delta, P->eps);
        c->st->n_point_pairs++;
        if (r >= P->delta - P->eps && r <= P->delta + P->eps) c->st->n_band_pairs++;
        for (int a = 0; a < nb; a++) {
          double phia = phim[p][a];
          for (int b = 0; b < nb; b++) S[a][b] += G * phia * phim[p][b];
          for (int d = 0; d < nb; d++) X[a][d] += G * phia * phil[q][d];
        }
      }
    }
    c->st->n_integrations++;
    for (int a = 0; a < nb; a++) {
      int64_t i = c->M->conn[m * nb + a];
      for (int b = 0; b < nb; b++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[m * nb + b]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e += 2.0 * S[a][b];
      }
      for (int d = 0; d < nb; d++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[c->l * nb + d]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e -= 2.0 * X[a][d];
      }
    }
  }
}

/* Algorithm 1 on a quadrilateral sub-element (the three branches of adaptive_integration). */
static void adaptive_integration_quad(actx* c, int L_cur, const qsub* E, const int32_t* J,
                                      int64_t nJ) {
  const or_params* P = c->P;
  if (L_cur < P->L_min) {
    qsub C[4];
    quad_split(E, C);
    for (int i = 0; i < 4; i++) adaptive_integration_quad(c, L_cur + 1, &C[i], J, nJ);
    return;
  }
  if (L_cur == P->L_max) {
    integration_quad(c, E, J, nJ);
    return;
  }
  int32_t* Jint = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  int32_t* Jref = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  if (!Jint || !Jref) {
    free(Jint), free(Jref);
    c->error = 1;
    return;
  }
  int64_t nint = 0, nref = 0;
  double lo[3], hi[3];
  verts_bbox(2, 4, E->V, lo, hi);
  for (int64_t t = 0; t < nJ; t++) {
    int64_t m = J[t];
    double amin = (P->flags & OR_MINDIST_L2)
                      ? or_aprx_min_dist_l2(2, lo, hi, c->lo + 3 * m, c->hi + 3 * m)
                      : or_aprx_min_dist(2, lo, hi, c->lo + 3 * m, c->hi + 3 * m);
    if (or_aprx_max_dist(2, lo, hi, c->lo + 3 * m, c->hi + 3 * m) < P->delta - P->eps)
      Jint[nint++] = (int32_t)m;
    else if (amin < P->delta + P->eps)
      Jref[nref++] = (int32_t)m;
  }
  if (nint > 0) integration_quad(c, E, Jint, nint);
  if (nref > 0) {
    qsub C[4];
    quad_split(E, C);
    for (int i = 0; i < 4; i++) adaptive_integration_quad(c, L_cur + 1, &C[i], Jref, nref);
  }
  free(Jint);
  free(Jref);
}

/* ------------------------------------------------------------------------------------
 * Hexahedra (Sec. 6: the HEX meshes of the three-dimensional tests; the Gauss-Legendre
 * 3x3x3 product rule for both integrals; Q1 trilinear elements).  An element is the image
 * of the unit cube under the trilinear map F(s,t,u) = sum_a N_a(s,t,u) v_a; a sub-element of
 * Algorithm 1 is the image of a sub-cube [s0, s0+len] x [t0, t0+len] x [u0, u0+len].  The
 * physical vertices of the eight children come from the parent's by midpoints on the lattice
 * of half-steps: a lattice point with a middle index is the midpoint of its two neighbours
 * along the first such axis (x, then y, then z), so edge midpoints are (a+b)*0.5 of two
 * vertices, face centres the midpoints of two edge midpoints, the centre the midpoint of
 * two face centres. */
typedef struct {
  double V[8][3];
  double s0, t0, u0, len;
} hsub;

static const int hex_corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                     {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

/* Trilinear basis N_a(s,t,u) and x = F(s,t,u), |det DF(s,t,u)|. */
static void hex_map(const double V[8][3], double s, double t, double u, double* x, double* detJ,
                    double* N) {
  double J[3][3] = {{0}};
  for (int k = 0; k < 3; k++) x[k] = 0.0;
  for (int a = 0; a < 8; a++) {
    const int* c = hex_corner[a];
    double fs = c[0] ? s : 1.0 - s, ft = c[1] ? t : 1.0 - t, fu = c[2] ? u : 1.0 - u;
    double ds = c[0] ? 1.0 : -1.0, dt = c[1] ? 1.0 : -1.0, du = c[2] ? 1.0 : -1.0;
    N[a] = fs * ft * fu;
    for (int k = 0; k < 3; k++) {
      x[k] += N[a] * V[a][k];
      J[k][0] += ds * ft * fu * V[a][k];
      J[k][1] += fs * dt * fu * V[a][k];
      J[k][2] += fs * ft * du * V[a][k];
    }
  }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  *detJ = fabs(det);
}

/* The 27 nodes of the Q2 hexahedron as points (i, j, k) of the lattice of half steps: the
 * eight vertices in the Q1 order, then the twelve edge midpoints, the six face centres and
 * the centre, each group in the order of (k, j, i) (z slowest, x fastest). */
static const int hex27[27][3] = {
    {0, 0, 0}, {2, 0, 0}, {2, 2, 0}, {0, 2, 0}, {0, 0, 2}, {2, 0, 2}, {2, 2, 2}, {0, 2, 2},
    {1, 0, 0}, {0, 1, 0}, {2, 1, 0}, {1, 2, 0}, {0, 0, 1}, {2, 0, 1}, {0, 2, 1}, {2, 2, 1},
    {1, 0, 2}, {0, 1, 2}, {2, 1, 2}, {1, 2, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {2, 1, 1},
    {1, 2, 1}, {1, 1, 2}, {1, 1, 1}};

/* Basis of a hexahedron at (s, t, u): Q1 the trilinear functions (as hex_map); Q2 the
 * products L_i(s) L_j(t) L_k(u) of the 1D quadratic Lagrange functions on {0, 1/2, 1} for
 * the node at lattice point (i, j, k); order 3 the 20-node serendipity element (the Q2 nodes
 * without the face centres and the centre, i.e. the first 20 of hex27), written on
 * (xi, eta, zeta) = (2s-1, 2t-1, 2u-1) with node a at (xi_a, eta_a, zeta_a) = (i-1, j-1, k-1):
 * a corner has (1/8)(1 + xi xi_a)(1 + eta eta_a)(1 + zeta zeta_a)(xi xi_a + eta eta_a +
 * zeta zeta_a - 2), an edge node with xi_a = 0 has (1/4)(1 - xi^2)(1 + eta eta_a)(1 + zeta
 * zeta_a), and likewise along eta and zeta. */
static void hex_basis(int order, double s, double t, double u, double* phi) {
  if (order == 3) {
    double c[3] = {2.0 * s - 1.0, 2.0 * t - 1.0, 2.0 * u - 1.0};
    for (int a = 0; a < 20; a++) {
      double f[3], p = 1.0;
      int mid = -1;
      for (int k = 0; k < 3; k++) {
        f[k] = (double)(hex27[a][k] - 1);
        if (f[k] == 0.0) mid = k;
      }
      if (mid < 0) {
        for (int k = 0; k < 3; k++) p *= 1.0 + c[k] * f[k];
        phi[a] = 0.125 * p * (c[0] * f[0] + c[1] * f[1] + c[2] * f[2] - 2.0);
      } else {
        for (int k = 0; k < 3; k++) p *= (k == mid) ? 1.0 - c[k] * c[k] : 1.0 + c[k] * f[k];
        phi[a] = 0.25 * p;
      }
    }
    return;
  }
  if (order != 2) {
    for (int a = 0; a < 8; a++)
      phi[a] = (hex_corner[a][0] ? s : 1.0 - s) * (hex_corner[a][1] ? t : 1.0 - t) *
               (hex_corner[a][2] ? u : 1.0 - u);
    return;
  }
  double L[3][3];
  lagrange1d(2, s, L[0]);
  lagrange1d(2, t, L[1]);
  lagrange1d(2, u, L[2]);
  for (int a = 0; a < 27; a++) phi[a] = L[0][hex27[a][0]] * L[1][hex27[a][1]] * L[2][hex27[a][2]];
}

/* The lattice point (i, j, k) in {0, 1, 2}^3 of the hexahedron V (see above). */
static void hex_lattice(const double V[8][3], int i, int j, int k, double* out) {
  double a[3], b[3];
  if (i == 1) {
    hex_lattice(V, 0, j, k, a);
    hex_lattice(V, 2, j, k, b);
    midpoint(a, b, out);
  } else if (j == 1) {
    hex_lattice(V, i, 0, k, a);
    hex_lattice(V, i, 2, k, b);
    midpoint(a, b, out);
  } else if (k == 1) {
    hex_lattice(V, i, j, 0, a);
    hex_lattice(V, i, j, 2, b);
    midpoint(a, b, out);
  } else {
    for (int v = 0; v < 8; v++)
      if (2 * hex_corner[v][0] == i && 2 * hex_corner[v][1] == j && 2 * hex_corner[v][2] == k)
        for (int q = 0; q < 3; q++) out[q] = V[v][q];
  }
}

/* The eight children (sub-cubes (cx, cy, cz), child index cx + 2 cy + 4 cz). */
static void hex_split(const hsub* E, hsub C[8]) {
  double L[3][3][3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++) hex_lattice(E->V, i, j, k, L[i][j][k]);
  const double h = 0.5 * E->len;
  for (int c = 0; c < 8; c++) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    for (int a = 0; a < 8; a++)
      for (int q = 0; q < 3; q++)
        C[c].V[a][q] = L[cx + hex_corner[a][0]][cy + hex_corner[a][1]][cz + hex_corner[a][2]][q];
    C[c].s0 = E->s0 + cx * h;
    C[c].t0 = E->t0 + cy * h;
    C[c].u0 = E->u0 + cz * h;
    C[c].len = h;
  }
}

/* Integration(E', J') on a hexahedral sub-element (the sums of integration() with the 3x3x3
 * rule on the sub-cube of l's cube and on m's cube). */
static void integration_hex(actx* c, const hsub* E, const int32_t* J, int64_t nJ,
                            const double Vl[8][3]) {
  const or_params* P = c->P;
  double g[3], gw[3];
  gl3_unit(g, gw);
  int nb = c->nb, order = c->M->order;
  double xq[27][3], wx[27], phil[27][27], gq[27][3], gwq[27];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++) {
        int q = 9 * i + 3 * j + k;
        gq[q][0] = g[i];
        gq[q][1] = g[j];
        gq[q][2] = g[k];
        gwq[q] = gw[i] * gw[j] * gw[k];
        double det, N[8];
        double s = E->s0 + E->len * g[i], t = E->t0 + E->len * g[j], u = E->u0 + E->len * g[k];
        hex_map(Vl, s, t, u, xq[q], &det, N);
        hex_basis(order, s, t, u, phil[q]);
        wx[q] = gwq[q] * E->len * E->len * E->len * det;
      }
  for (int64_t tt = 0; tt < nJ; tt++) {
    int64_t m = J[tt];
    double Vm[8][3];
    hex_verts(c->M, m, Vm);
    double S[27][27] = {{0}}, X[27][27] = {{0}};
    for (int p = 0; p < 27; p++) {
      double y[3], detm, N[8], phim[27];
      hex_map(Vm, gq[p][0], gq[p][1], gq[p][2], y, &detm, N);
      hex_basis(order, gq[p][0], gq[p][1], gq[p][2], phim);
      double wy = gwq[p] * detm;
      for (int q = 0; q < 27; q++) {
        double r2 = 0.0;
        for (int k = 0; k < 3; k++) r2 += (xq[q][k] - y[k]) * (xq[q][k] - y[k]);
        double r = sqrt(r2);
        double G = wx[q] * wy * P->C * or_eta(P->kernel, r, P->delta) * or_mu(r, P->delta, P->eps);
        c->st->n_point_pairs++;
        if (r >= P->delta - P->eps && r <= P->delta + P->eps) c->st->n_band_pairs++;
        for (int a = 0; a < nb; a++) {
          for (int b = 0; b < nb; b++) S[a][b] += G * phim[a] * phim[b];
          for (int d = 0; d < nb; d++) X[a][d] += G * phim[a] * phil[q][d];
        }
      }
    }
    c->st->n_integrations++;
    for (int a = 0; a < nb; a++) {
      int64_t i = c->M->conn[m * nb + a];
      for (int b = 0; b < nb; b++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[m * nb + b]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e += 2.0 * S[a][b];
      }
      for (int d = 0; d < nb; d++) {
        double* e = csr_entry(c->row_ptr, c->col, c->values, i, c->M->conn[c->l * nb + d]);
        if (!e) {
          c->error = 1;
          continue;
        }
        *e -= 2.0 * X[a][d];
      }
    }
  }
}

/* Algorithm 1 on a hexahedral sub-element. */
static void adaptive_integration_hex(actx* c, int L_cur, const hsub* E, const int32_t* J,
                                     int64_t nJ, const double Vl[8][3]) {
  const or_params* P = c->P;
  if (L_cur < P->L_min) {
    hsub C[8];
    hex_split(E, C);
    for (int i = 0; i < 8; i++) adaptive_integration_hex(c, L_cur + 1, &C[i], J, nJ, Vl);
    return;
  }
  if (L_cur == P->L_max) {
    integration_hex(c, E, J, nJ, Vl);
    return;
  }
  int32_t* Jint = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  int32_t* Jref = (int32_t*)malloc(sizeof(int32_t) * (nJ + 1));
  if (!Jint || !Jref) {
    free(Jint), free(Jref);
    c->error = 1;
    return;
  }
  int64_t nint = 0, nref = 0;
  double lo[3], hi[3];
  hex_bbox(E->V, lo, hi);
  for (int64_t t = 0; t < nJ; t++) {
    int64_t m = J[t];
    double amin = (P->flags & OR_MINDIST_L2)
                      ? or_aprx_min_dist_l2(3, lo, hi, c->lo + 3 * m, c->hi + 3 * m)
                      : or_aprx_min_dist(3, lo, hi, c->lo + 3 * m, c->hi + 3 * m);
    if (or_aprx_max_dist(3, lo, hi, c->lo + 3 * m, c->hi + 3 * m) < P->delta - P->eps)
      Jint[nint++] = (int32_t)m;
    else if (amin < P->delta + P->eps)
      Jref[nref++] = (int32_t)m;
  }
  if (nint > 0) integration_hex(c, E, Jint, nint, Vl);
  if (nref > 0) {
    hsub C[8];
    hex_split(E, C);
    for (int i = 0; i < 8; i++) adaptive_integration_hex(c, L_cur + 1, &C[i], Jref, nref, Vl);
  }
  free(Jint);
  free(Jref);
}

int or_assemble(const or_mesh* M, const int64_t* pair_off, const int32_t* pair_l,
                const or_params* P, const int64_t* row_ptr, const int32_t* col, double* values,
                const uint8_t* m_mask, or_stats* stats) {
  int dim = M->dim, nv = dim + 1;
  int64_t nE = M->n_elem, nV = M->n_vert;
  if (dim != 2 && dim != 3) return -1;
  if (M->cell == 1 && dim != 2) return -1; /* quadrilaterals: dim 2 */
  if (M->cell == 2 && dim != 3) return -1; /* hexahedra: dim 3 */
  if (!(P->eps > 0.0 && P->eps < P->delta) || P->L_min < 1 || P->L_max < P->L_min) return -1;
  actx c;
  memset(&c, 0, sizeof c);
  c.M = M;
  c.P = P;
  c.dim = dim;
  c.nv = nv;
  c.nb = npe(M);

  double bary[64], w[16];
  c.nq = or_quad_rule(dim, bary, w);
  if (c.nq <= 0) return -1;
  for (int q = 0; q < c.nq; q++) {
    for (int v = 0; v < nv; v++) c.qb[q][v] = bary[q * nv + v];
    c.qw[q] = w[q];
  }
  double* lo = (double*)malloc(sizeof(double) * 3 * nE);
  double* hi = (double*)malloc(sizeof(double) * 3 * nE);
  /* J_l: the transpose of the m-major pair lists, restricted to the selected m. */
  int64_t* toff = (int64_t*)calloc(nE + 1, sizeof(int64_t));
  int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (nE + 1));
  int64_t np = pair_off[nE];
  int32_t* tm = (int32_t*)malloc(sizeof(int32_t) * (np + 1));
  if (!lo || !hi || !toff || !fillp || !tm) {
    free(lo), free(hi), free(toff), free(fillp), free(tm);
    return -1;
  }
  for (int64_t e = 0; e < nE; e++) elem_box(M, e, lo + 3 * e, hi + 3 * e);
  for (int64_t m = 0; m < nE; m++) {
    if (m_mask && !m_mask[m]) continue;
    for (int64_t p = pair_off[m]; p < pair_off[m + 1]; p++) toff[pair_l[p] + 1]++;
  }
  for (int64_t l = 0; l < nE; l++) toff[l + 1] += toff[l];
  for (int64_t l = 0; l <= nE; l++) fillp[l] = toff[l];
  for (int64_t m = 0; m < nE; m++) { /* m ascending, so every J_l is sorted */
    if (m_mask && !m_mask[m]) continue;
    for (int64_t p = pair_off[m]; p < pair_off[m + 1]; p++) tm[fillp[pair_l[p]]++] = (int32_t)m;
  }
  c.lo = lo;
  c.hi = hi;
  c.row_ptr = row_ptr;
  c.col = col;
  c.values = values;
  or_stats local;
  memset(&local, 0, sizeof local);
  c.st = &local;
  memset(values, 0, sizeof(double) * row_ptr[nV]);
  for (int64_t l = 0; l < nE; l++) {
    int64_t nJ = toff[l + 1] - toff[l];
    if (nJ == 0) continue;
    c.l = l;
    if (M->cell == 2) {
      hsub root;
      hex_verts(M, l, root.V);
      root.s0 = root.t0 = root.u0 = 0.0;
      root.len = 1.0;
      adaptive_integration_hex(&c, 1, &root, tm + toff[l], nJ, root.V);
      continue;
    }
    elem_verts(M, l, c.Vl);
    if (M->cell == 1) {
      qsub root;
      memcpy(root.V, c.Vl, sizeof root.V);
      root.s0 = 0.0;
      root.t0 = 0.0;
      root.len = 1.0;
      adaptive_integration_quad(&c, 1, &root, tm + toff[l], nJ);
    } else {
      adaptive_integration(&c, 1, c.Vl, tm + toff[l], nJ);
    }
  }
  if (stats) *stats = local;
  free(lo), free(hi), free(toff), free(fillp), free(tm);
  return c.error ? -2 : 0;
}

/* ------------------------------------------------------------------------------------
 * Manufactured solutions (Sec. 6) and f = -L_eps u (Sec. 2, eq. L).  For u = sum_k p(x_k),
 * a Taylor expansion of p(x_k + z_k) - p(x_k) and the radial symmetry of gamma_eps (odd
 * moments vanish) give L_eps u = sum_k [p''(x_k) M2 + p''''(x_k) M4 / 12] with
 * M2 = int z_1^2 gamma_eps, M4 = int z_1^4 gamma_eps, wherever B_{delta+eps}(x) lies
 * inside the mesh. */
double or_ms_u(int ms, int dim, const double* x) {
  double s = (ms == OR_MS_LINEAR) ? 1.0 : 0.0;
  for (int k = 0; k < dim; k++) {
    double t = x[k];
    switch (ms) {
      case OR_MS_LINEAR: s += t; break;
      case OR_MS_QUADRATIC: s += t * t; break;
      case OR_MS_CUBIC: s += t * t * t; break;
      case OR_MS_QUARTIC: s += t * t * t * t; break;
      default: return NAN;
    }
  }
  return s;
}

double or_ms_f(int ms, int dim, const double* x, int kernel, double delta, double eps, double C) {
  double M2 = or_kernel_moment(dim, kernel, delta, eps, C, 2);
  double M4 = or_kernel_moment(dim, kernel, delta, eps, C, 4);
  double Lu = 0.0;
  for (int k = 0; k < dim; k++) {
    double t = x[k], p2 = 0.0, p4 = 0.0;
    switch (ms) {
      case OR_MS_LINEAR: break;
      case OR_MS_QUADRATIC: p2 = 2.0; break;
      case OR_MS_CUBIC: p2 = 6.0 * t; break;
      case OR_MS_QUARTIC: p2 = 12.0 * t * t; p4 = 24.0; break;
      default: return NAN;
    }
    Lu += p2 * M2 + p4 * M4 / 12.0;
  }
  return -Lu;
}

/* Sec. 2, eqs. (A-F) and (weak-homo), Sec. 4: F_i = int_Omega f phi_i (degree-5 rule on
 * every element of Omega), then the lifting u = w + g~ moves the constrained columns to
 * the right-hand side: F~_i = F_i - sum_{k not free} A_ik g(x_k). */
int or_rhs(const or_mesh* M, const int64_t* row_ptr, const int32_t* col, const double* values,
           int ms, int kernel, double delta, double eps, double C, double* F) {
  int dim = M->dim, nv = dim + 1, nb = npe(M);
  double bary[64], w[16];
  int nq = or_quad_rule(dim, bary, w);
  if (nq <= 0) return -1;
  for (int64_t i = 0; i < M->n_vert; i++) F[i] = 0.0;
  for (int64_t e = 0; e < M->n_elem; e++) {
    if (!M->elem_in_omega[e]) continue;
    if (M->cell == 2) { /* Gauss-Legendre 3x3x3 on the image of the unit cube */
      double H[8][3], g[3], gw[3];
      hex_verts(M, e, H);
      gl3_unit(g, gw);
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
          for (int k = 0; k < 3; k++) {
            double x[3], det, N[8], phi[27];
            hex_map(H, g[i], g[j], g[k], x, &det, N);
            hex_basis(M->order, g[i], g[j], g[k], phi);
            double f = or_ms_f(ms, dim, x, kernel, delta, eps, C);
            for (int a = 0; a < nb; a++) {
              int64_t n = M->conn[e * nb + a];
              if (M->node_free[n]) F[n] += gw[i] * gw[j] * gw[k] * det * f * phi[a];
            }
          }
      continue;
    }
    double V[4][3];
    elem_verts(M, e, V);
    if (M->cell == 1) { /* Gauss-Legendre 3x3 on the image of the unit square */
      double g[3], gw[3];
      gl3_unit(g, gw);
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
          double x[3], det, phi[9];
          quad_map(V, g[i], g[j], x, &det);
          double f = or_ms_f(ms, dim, x, kernel, delta, eps, C);
          quad_basis(M->order, g[i], g[j], phi);
          for (int a = 0; a < nb; a++) {
            int64_t n = M->conn[e * nb + a];
            if (M->node_free[n]) F[n] += gw[i] * gw[j] * det * f * phi[a];
          }
        }
      continue;
    }
    double vol = simplex_volume(dim, V);
    for (int q = 0; q < nq; q++) {
      double x[3];
      for (int k = 0; k < 3; k++) {
        double s = 0.0;
        for (int v = 0; v < nv; v++) s += bary[q * nv + v] * V[v][k];
        x[k] = s;
      }
      double f = or_ms_f(ms, dim, x, kernel, delta, eps, C);
      double phi[10];
      basis(M, bary + q * nv, phi);
      for (int a = 0; a < nb; a++) {
        int64_t i = M->conn[e * nb + a];
        if (M->node_free[i]) F[i] += w[q] * vol * f * phi[a];
      }
    }
  }
  for (int64_t i = 0; i < M->n_vert; i++) {
    if (!M->node_free[i]) continue;
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; t++) {
      int64_t j = col[t];
      if (M->node_free[j]) continue;
      double xj[3] = {0, 0, 0};
      for (int k = 0; k < dim; k++) xj[k] = M->coords[k * M->n_vert + j];
      F[i] -= values[t] * or_ms_u(ms, dim, xj);
    }
  }
  return 0;
}

int or_solve_dense(const or_mesh* M, const int64_t* row_ptr, const int32_t* col,
                   const double* values, const double* F, int ms, double* u_h) {
  int64_t nV = M->n_vert;
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * nV);
  if (!idx) return -1;
  int64_t nf = 0;
  for (int64_t i = 0; i < nV; i++) idx[i] = M->node_free[i] ? nf++ : -1;
  if (nf > 20000) {
    free(idx);
    return -1;
  }
  double* A = (double*)calloc((size_t)(nf * nf + 1), sizeof(double));
  double* b = (double*)malloc(sizeof(double) * (nf + 1));
  if (!A || !b) {
    free(idx), free(A), free(b);
    return -1;
  }
  for (int64_t i = 0; i < nV; i++) {
    if (idx[i] < 0) continue;
    b[idx[i]] = F[i];
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; t++)
      if (idx[col[t]] >= 0) A[idx[i] * nf + idx[col[t]]] = values[t];
  }
  int rc = dense_solve((int)nf, A, b);
  for (int64_t i = 0; i < nV; i++) {
    if (idx[i] >= 0) {
      u_h[i] = b[idx[i]];
    } else {
      double x[3] = {0, 0, 0};
      for (int k = 0; k < M->dim; k++) x[k] = M->coords[k * nV + i];
      u_h[i] = or_ms_u(ms, M->dim, x);
    }
  }
  free(idx), free(A), free(b);
  return rc;
}

/* ||u - u_h||_{L2}: each element is split twice by midpoints and the degree-5 rule is
 * applied on every piece. */
static double err_on(const or_mesh* M, const double V[4][3], const double* nodal,
                     const double bary[][4], const double* w, int nq, int ms,
                     const double Vroot[4][3], int depth) {
  int dim = M->dim;
  if (depth > 0) {
    double C[8][4][3];
    split(dim, V, C);
    double s = 0.0;
    for (int i = 0; i < ((dim == 2) ? 4 : 8); i++)
      s += err_on(M, C[i], nodal, bary, w, nq, ms, Vroot, depth - 1);
    return s;
  }
  double vol = simplex_volume(dim, V), s = 0.0;
  for (int q = 0; q < nq; q++) {
    double x[3];
    for (int k = 0; k < 3; k++) {
      double t = 0.0;
      for (int v = 0; v <= dim; v++) t += bary[q][v] * V[v][k];
      x[k] = t;
    }
    double lam[4], phi[10];
    barycentric(dim, Vroot, x, lam);
    basis(M, lam, phi);
    double uh = 0.0;
    for (int a = 0; a < npe(M); a++) uh += phi[a] * nodal[a];
    double d = or_ms_u(ms, dim, x) - uh;
    s += w[q] * vol * d * d;
  }
  return s;
}

/* The same on a quadrilateral: Gauss-Legendre 3x3 on each of the 4 x 4 sub-squares of the
 * unit square, mapped by the element's bilinear map. */
static double err_on_quad(const or_mesh* M, const double V[4][3], const double* nodal, int ms) {
  double g[3], gw[3], s = 0.0;
  gl3_unit(g, gw);
  for (int bi = 0; bi < 4; bi++)
    for (int bj = 0; bj < 4; bj++)
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
          double u = 0.25 * (bi + g[i]), v = 0.25 * (bj + g[j]), x[3], det, phi[9];
          quad_map(V, u, v, x, &det);
          quad_basis(M->order, u, v, phi);
          double uh = 0.0;
          for (int a = 0; a < npe(M); a++) uh += phi[a] * nodal[a];
          double d = or_ms_u(ms, M->dim, x) - uh;
          s += 0.0625 * gw[i] * gw[j] * det * d * d;
        }
  return s;
}

/* The same on a hexahedron: Gauss-Legendre 3x3x3 on each of the 2 x 2 x 2 sub-cubes of the
 * unit cube, mapped by the element's trilinear map. */
static double err_on_hex(const or_mesh* M, const double V[8][3], const double* nodal, int ms) {
  double g[3], gw[3], s = 0.0;
  gl3_unit(g, gw);
  for (int b = 0; b < 8; b++)
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) {
          double u = 0.5 * ((b & 1) + g[i]), v = 0.5 * (((b >> 1) & 1) + g[j]);
          double w = 0.5 * (((b >> 2) & 1) + g[k]), x[3], det, N[8], phi[27];
          hex_map(V, u, v, w, x, &det, N);
          hex_basis(M->order, u, v, w, phi);
          double uh = 0.0;
          for (int a = 0; a < npe(M); a++) uh += phi[a] * nodal[a];
          double d = or_ms_u(ms, M->dim, x) - uh;
          s += 0.125 * gw[i] * gw[j] * gw[k] * det * d * d;
        }
  return s;
}

double or_l2_error(const or_mesh* M, const double* u_h, int ms, int omega_only) {
  int dim = M->dim, nv = dim + 1;
  double b[64], w[16], bary[16][4];
  int nq = or_quad_rule(dim, b, w);
  if (nq <= 0) return NAN;
  for (int q = 0; q < nq; q++)
    for (int v = 0; v < nv; v++) bary[q][v] = b[q * nv + v];
  double s = 0.0;
  for (int64_t e = 0; e < M->n_elem; e++) {
    if (omega_only && !M->elem_in_omega[e]) continue;
    if (M->cell == 2) {
      double H[8][3], hn[27];
      hex_verts(M, e, H);
      for (int a = 0; a < npe(M); a++) hn[a] = u_h[M->conn[e * npe(M) + a]];
      s += err_on_hex(M, H, hn, ms);
      continue;
    }
    double V[4][3], nodal[10];
    elem_verts(M, e, V);
    for (int a = 0; a < npe(M); a++) nodal[a] = u_h[M->conn[e * npe(M) + a]];
    if (M->cell == 1) s += err_on_quad(M, V, nodal, ms);
    else s += err_on(M, V, nodal, (const double(*)[4])bary, w, nq, ms, V, 2);
  }
  return sqrt(s);
}
