// nl_host.cu -- C ABI entry points, handles, allocator, host-side tables, mesh set-up.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <vector>

#include "nl_internal.h"

namespace nlx {

// ---- errors ------------------------------------------------------------------------------
static thread_local std::string g_err;

nl_status fail(nl_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

nl_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // a failed call also sets the thread's last error; later checks start clean
  return fail(e == cudaErrorMemoryAllocation ? NL_ENOMEM : NL_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

// ---- launch counter ---------------------------------------------------------------------
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---- allocator ---------------------------------------------------------------------------
static nl_alloc_fn g_alloc = nullptr;
static nl_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) return nullptr;
  if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, bytes, s, g_alloc_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// ---- quadrature rules ------------------------------------------------------------------------
// Triangle: Radon's 7-point degree-5 rule in closed form (centroid; two orbits (a, a, 1-2a)
// with a = (6 -+ sqrt 15)/21, weights 9/40 and (155 -+ sqrt 15)/1200).
// Tetrahedron: the 14-point degree-5 rule with orbits (a,a,a,1-3a), (b,b,b,1-3b),
// (c,c,1/2-c,1/2-c), obtained here by Newton's method with the analytic Jacobian on the
// equations for the orbit-invariant power sums p_k = sum_i lambda_i^k (k = 2..5) and p_2^2,
// whose averages over the tetrahedron follow from int lambda^alpha = 3! alpha!/(|alpha|+3)!.
typedef long double ld;

static void tet_eqs(const ld u[6], ld F[6], ld J[6][6]) {
  // u = (wa, a, wb, b, wc, c); orbit sizes 4, 4, 6
  const ld exact[6] = {1.0L,
                       4.0L * 6.0L * 2.0L / 120.0L,      // p2: 4 * 3! 2!/5!
                       4.0L * 6.0L * 6.0L / 720.0L,      // p3: 4 * 3! 3!/6!
                       4.0L * 6.0L * 24.0L / 5040.0L,    // p4: 4 * 3! 4!/7!
                       4.0L * 6.0L * 120.0L / 40320.0L,  // p5: 4 * 3! 5!/8!
                       (4.0L * 6.0L * 24.0L + 12.0L * 6.0L * 4.0L) / 5040.0L};  // p2^2
  for (int j = 0; j < 6; j++) {
    F[j] = -exact[j];
    for (int c = 0; c < 6; c++) J[j][c] = 0.0L;
  }
  for (int o = 0; o < 3; o++) {
    ld w = u[2 * o], t = u[2 * o + 1];
    ld nsz = (o < 2) ? 4.0L : 6.0L;
    // representative coordinates: (t, t, t, 1-3t) or (t, t, 1/2-t, 1/2-t)
    ld q = (o < 2) ? 1.0L - 3.0L * t : 0.5L - t;
    ld mt = (o < 2) ? 3.0L : 2.0L, mq = (o < 2) ? 1.0L : 2.0L;  // multiplicities of t and q
    ld dq = (o < 2) ? -3.0L : -1.0L;                            // dq/dt
    ld p[6], dp[6];
    p[0] = 1.0L;
    dp[0] = 0.0L;
    for (int k = 2; k <= 5; k++) {
      ld tk = 1.0L, qk = 1.0L;
      for (int e = 0; e < k - 1; e++) {
        tk *= t;
        qk *= q;
      }
      p[k - 1] = mt * tk * t + mq * qk * q;
      dp[k - 1] = mt * k * tk + mq * k * qk * dq;
    }
    p[5] = p[1] * p[1];
    dp[5] = 2.0L * p[1] * dp[1];
    for (int j = 0; j < 6; j++) {
      F[j] += nsz * w * p[j];
      J[j][2 * o] = nsz * p[j];
      J[j][2 * o + 1] = nsz * w * dp[j];
    }
  }
}

static bool solve6(ld A[6][6], ld b[6]) {
  for (int k = 0; k < 6; k++) {
    int piv = k;
    for (int i = k + 1; i < 6; i++)
      if (fabsl(A[i][k]) > fabsl(A[piv][k])) piv = i;
    if (A[piv][k] == 0.0L) return false;
    for (int j = 0; j < 6; j++) std::swap(A[k][j], A[piv][j]);
    std::swap(b[k], b[piv]);
    for (int i = k + 1; i < 6; i++) {
      ld f = A[i][k] / A[k][k];
      for (int j = k; j < 6; j++) A[i][j] -= f * A[k][j];
      b[i] -= f * b[k];
    }
  }
  for (int i = 5; i >= 0; i--) {
    ld s = b[i];
    for (int j = i + 1; j < 6; j++) s -= A[i][j] * b[j];
    b[i] = s / A[i][i];
  }
  return true;
}

static Rule make_tri_rule() {
  Rule r;
  double s15 = std::sqrt(15.0);
  double a[2] = {(6.0 - s15) / 21.0, (6.0 + s15) / 21.0};
  double w[2] = {(155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0};
  r.n = 7;
  r.bary[0][0] = r.bary[0][1] = r.bary[0][2] = 1.0 / 3.0;
  r.w[0] = 9.0 / 40.0;
  int q = 1;
  for (int o = 0; o < 2; o++)
    for (int k = 0; k < 3; k++) {
      for (int v = 0; v < 3; v++) r.bary[q][v] = (v == k) ? 1.0 - 2.0 * a[o] : a[o];
      r.w[q] = w[o];
      q++;
    }
  return r;
}

static Rule make_tet_rule() {
  Rule r;
  ld u[6] = {0.0735L, 0.0927L, 0.1127L, 0.3109L, 0.0425L, 0.0455L};
  for (int it = 0; it < 80; it++) {
    ld F[6], J[6][6];
    tet_eqs(u, F, J);
    for (int j = 0; j < 6; j++) F[j] = -F[j];
    if (!solve6(J, F)) return r;
    for (int c = 0; c < 6; c++) u[c] += F[c];
  }
  int q = 0;
  for (int o = 0; o < 2; o++) {
    ld t = u[2 * o + 1];
    for (int k = 0; k < 4; k++) {
      for (int v = 0; v < 4; v++) r.bary[q][v] = (double)((v == k) ? 1.0L - 3.0L * t : t);
      r.w[q] = (double)u[2 * o];
      q++;
    }
  }
  ld c = u[5];
  for (int i = 0; i < 4; i++)
    for (int j = i + 1; j < 4; j++) {
      for (int v = 0; v < 4; v++) r.bary[q][v] = (double)((v == i || v == j) ? c : 0.5L - c);
      r.w[q] = (double)u[4];
      q++;
    }
  r.n = q;
  return r;
}

const Rule& rule(int dim) {
  static Rule tri = make_tri_rule();
  static Rule tet = make_tet_rule();
  return dim == 2 ? tri : tet;
}

// Gauss-Legendre with 3 points on [0, 1]: the roots of the Legendre polynomial P_3,
// 0 and +-sqrt(3/5) on [-1, 1], with weights 8/9 and 5/9, mapped by s = (x + 1)/2.
const GL3& gl3() {
  static const GL3 r = [] {
    GL3 t;
    const double a = std::sqrt(0.6);
    t.g[0] = 0.5 * (1.0 - a);
    t.g[1] = 0.5;
    t.g[2] = 0.5 * (1.0 + a);
    t.w[0] = 5.0 / 18.0;
    t.w[1] = 8.0 / 18.0;
    t.w[2] = 5.0 / 18.0;
    return t;
  }();
  return r;
}

// ---- kernel constants ------------------------------------------------------------------------
static double xi_host(double s) {
  double t = s * s;
  double p = 35.0;
  p = p * t - 180.0;
  p = p * t + 378.0;
  p = p * t - 420.0;
  p = p * t + 315.0;
  return 0.5 + s * p / 256.0;
}

static double mu_host(double r, double delta, double eps) {
  if (r <= delta - eps) return 1.0;
  if (r >= delta + eps) return 0.0;
  return xi_host((delta - r) / eps);
}

// int_a^b f by composite 5-point Gauss-Legendre on n panels (closed-form nodes).
template <typename F>
static double gl5(F f, double a, double b, int n) {
  const double x1 = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double x2 = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
  const double w0 = 128.0 / 225.0;
  const double w1 = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0;
  const double w2 = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
  const double xs[5] = {-x2, -x1, 0.0, x1, x2};
  const double ws[5] = {w2, w1, w0, w1, w2};
  double h = (b - a) / n, s = 0.0;
  for (int i = 0; i < n; i++) {
    double c = a + (i + 0.5) * h;
    for (int k = 0; k < 5; k++) s += 0.5 * h * ws[k] * f(c + 0.5 * h * xs[k]);
  }
  return s;
}

}  // namespace nlx

double nl_kernel_constant(int dim, int kernel, double delta, double eps) {
  using namespace nlx;
  if (!(dim == 2 || dim == 3) || !(eps > 0.0 && eps < delta)) return NAN;
  double t2 = (eps / delta) * (eps / delta);
  if (kernel == NL_KERNEL_CONST) {
    // Sec. 6: C_delta = 4/(pi delta^4) (2D), 15/(4 pi delta^5) (3D), kappa = 1
    if (dim == 2) return 4.0 / (M_PI * std::pow(delta, 4)) / (1.0 + 6.0 / 11.0 * t2 + 3.0 / 143.0 * t2 * t2);
    return 15.0 / (4.0 * M_PI * std::pow(delta, 5)) / (1.0 + 10.0 / 11.0 * t2 + 15.0 / 143.0 * t2 * t2);
  }
  // int z_1^2 gamma_eps dz = |S^{n-1}|/n int_0^{delta+eps} r^{n+1} eta(r) mu(r) dr = 1
  auto f = [&](double r) {
    double e = std::exp(-(r * r) / (delta * delta));
    return std::pow(r, dim + 1) * e * mu_host(r, delta, eps);
  };
  double I = gl5(f, 0.0, delta - eps, 64) + gl5(f, delta - eps, delta + eps, 64);
  double sphere = (dim == 2) ? 2.0 * M_PI : 4.0 * M_PI;
  return dim / (sphere * I);
}

double nlx::kernel_constant(int dim, int kernel, double delta, double eps) {
  return nl_kernel_constant(dim, kernel, delta, eps);
}

int nl_quad_rule(int dim, double* bary, double* w) {
  if (dim != 2 && dim != 3) return -1;
  const nlx::Rule& r = nlx::rule(dim);
  if (r.n <= 0) return -1;
  for (int q = 0; q < r.n; q++) {
    if (bary)
      for (int v = 0; v <= dim; v++) bary[q * (dim + 1) + v] = r.bary[q][v];
    if (w) w[q] = r.w[q];
  }
  return r.n;
}

// ---- mesh ------------------------------------------------------------------------------------
namespace {

// Per-element geometry from the first D+1 nodes of each element (its vertices; a P2 element
// lists its edge nodes after them): nb nodes per element in conn.
template <int D>
__global__ void k_mesh_elements(int64_t n_elem, int64_t n_vert, const double* __restrict__ coords,
                                const int32_t* __restrict__ conn, int nb, double* __restrict__ evert,
                                double* __restrict__ blo, double* __restrict__ bhi,
                                double* __restrict__ vol, double* __restrict__ jinv,
                                float* __restrict__ ef) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  double V[D + 1][D];
  for (int a = 0; a <= D; a++) {
    int32_t v = conn[e * nb + a];
    for (int k = 0; k < D; k++) {
      V[a][k] = coords[k * n_vert + v];
      evert[(e * (D + 1) + a) * D + k] = V[a][k];
    }
  }
  for (int k = 0; k < D; k++) {
    double lo = V[0][k], hi = V[0][k];
    for (int a = 1; a <= D; a++) {
      lo = fmin(lo, V[a][k]);
      hi = fmax(hi, V[a][k]);
    }
    blo[e * D + k] = lo;
    bhi[e * D + k] = hi;
  }
  // T = [v1-v0, ..., vD-v0] (columns); lambda_{1..D}(x) = T^{-1} (x - v0)
  double T[D][D];
  for (int c = 0; c < D; c++)
    for (int k = 0; k < D; k++) T[k][c] = V[c + 1][k] - V[0][k];
  double inv[D][D];
  double det;
  if (D == 2) {
    det = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    inv[0][0] = T[1][1] / det;
    inv[0][1] = -T[0][1] / det;
    inv[1][0] = -T[1][0] / det;
    inv[1][1] = T[0][0] / det;
    vol[e] = fabs(det) / 2.0;
  } else {
    double c00 = T[1][1] * T[2][2] - T[1][2] * T[2][1];
    double c01 = T[1][2] * T[2][0] - T[1][0] * T[2][2];
    double c02 = T[1][0] * T[2][1] - T[1][1] * T[2][0];
    det = T[0][0] * c00 + T[0][1] * c01 + T[0][2] * c02;
    double id = 1.0 / det;
    double (*I)[3] = reinterpret_cast<double (*)[3]>(&inv[0][0]);
    I[0][0] = c00 * id;
    I[1][0] = c01 * id;
    I[2][0] = c02 * id;
    I[0][1] = (T[0][2] * T[2][1] - T[0][1] * T[2][2]) * id;
    I[1][1] = (T[0][0] * T[2][2] - T[0][2] * T[2][0]) * id;
    I[2][1] = (T[0][1] * T[2][0] - T[0][0] * T[2][1]) * id;
    I[0][2] = (T[0][1] * T[1][2] - T[0][2] * T[1][1]) * id;
    I[1][2] = (T[0][2] * T[1][0] - T[0][0] * T[1][2]) * id;
    I[2][2] = (T[0][0] * T[1][1] - T[0][1] * T[1][0]) * id;
    vol[e] = fabs(det) / 6.0;
  }
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) jinv[(e * D + r) * D + c] = inv[r][c];
  float* f = ef + e * NL_EF_STRIDE(D);
  for (int a = 1; a <= D; a++)
    for (int k = 0; k < D; k++) f[(a - 1) * D + k] = (float)(V[a][k] - V[0][k]);
  for (int r = 0; r < D; r++)
    for (int c = 0; c < D; c++) f[D * D + r * D + c] = (float)inv[r][c];
  f[2 * D * D] = (float)vol[e];
  for (int t = 2 * D * D + 1; t < NL_EF_STRIDE(D); t++) f[t] = 0.f;
  for (int k = 0; k < D; k++) {
    const float hi = (float)V[0][k];
    f[NL_EF_V0HI(D) + k] = hi;
    f[NL_EF_V0LO(D) + k] = (float)(V[0][k] - (double)hi);
  }
}

// Quadrilaterals (the bilinear image of the unit square, vertices v0..v3 counterclockwise,
// the first four of an element's nb nodes): the four vertices, the box, the area
// |(v2 - v0) x (v3 - v1)| / 2, no inverse Jacobian (zeros), and an FP32 record with the
// offsets v_a - v_0 (a = 1..3) at [0, 6), the area at [8] and v_0 as a float-float pair at
// the positions of the P1 record.
__global__ void k_mesh_quads(int64_t n_elem, int64_t n_vert, const double* __restrict__ coords,
                             const int32_t* __restrict__ conn, int nb, double* __restrict__ evert,
                             double* __restrict__ blo, double* __restrict__ bhi,
                             double* __restrict__ vol, double* __restrict__ jinv,
                             float* __restrict__ ef) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  double V[4][2];
  for (int a = 0; a < 4; a++) {
    int32_t v = conn[e * nb + a];
    for (int k = 0; k < 2; k++) {
      V[a][k] = coords[k * n_vert + v];
      evert[(e * 4 + a) * 2 + k] = V[a][k];
    }
  }
  for (int k = 0; k < 2; k++) {
    double lo = V[0][k], hi = V[0][k];
    for (int a = 1; a < 4; a++) {
      lo = fmin(lo, V[a][k]);
      hi = fmax(hi, V[a][k]);
    }
    blo[e * 2 + k] = lo;
    bhi[e * 2 + k] = hi;
  }
  const double d1x = V[2][0] - V[0][0], d1y = V[2][1] - V[0][1];
  const double d2x = V[3][0] - V[1][0], d2y = V[3][1] - V[1][1];
  vol[e] = fabs(d1x * d2y - d1y * d2x) / 2.0;
  for (int t = 0; t < 4; t++) jinv[e * 4 + t] = 0.0;
  float* f = ef + e * NL_EF_STRIDE(2);
  for (int a = 1; a < 4; a++)
    for (int k = 0; k < 2; k++) f[(a - 1) * 2 + k] = (float)(V[a][k] - V[0][k]);
  f[6] = f[7] = 0.f;
  f[8] = (float)vol[e];
  for (int t = 9; t < NL_EF_STRIDE(2); t++) f[t] = 0.f;
  for (int k = 0; k < 2; k++) {
    const float hi = (float)V[0][k];
    f[NL_EF_V0HI(2) + k] = hi;
    f[NL_EF_V0LO(2) + k] = (float)(V[0][k] - (double)hi);
  }
}

// Hexahedra (the trilinear image of the unit cube, vertices in the order (0,0,0), (1,0,0),
// (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1), the first 8 of the nb nodes of an
// element in conn): the eight vertices, the box, the
// volume (Gauss-Legendre 2x2x2 of |det DF|, exact: the determinant is of degree <= 2 in each
// variable), no inverse Jacobian, and an FP32 record of its own layout: the offsets v_a - v_0
// (a = 1..7) at [0, 21), v_0 as a float-float pair at [21, 24) and [24, 27), the volume at
// [27].
__global__ void k_mesh_hexes(int64_t n_elem, int64_t n_vert, const double* __restrict__ coords,
                             const int32_t* __restrict__ conn, int nb, double* __restrict__ evert,
                             double* __restrict__ blo, double* __restrict__ bhi,
                             double* __restrict__ vol, double* __restrict__ jinv,
                             float* __restrict__ ef) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  double V[8][3];
  for (int a = 0; a < 8; a++) {
    int32_t v = conn[e * nb + a];
    for (int k = 0; k < 3; k++) {
      V[a][k] = coords[k * n_vert + v];
      evert[(e * 8 + a) * 3 + k] = V[a][k];
    }
  }
  for (int k = 0; k < 3; k++) {
    double lo = V[0][k], hi = V[0][k];
    for (int a = 1; a < 8; a++) {
      lo = fmin(lo, V[a][k]);
      hi = fmax(hi, V[a][k]);
    }
    blo[e * 3 + k] = lo;
    bhi[e * 3 + k] = hi;
  }
  const int cc[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
  double v = 0.0;
  for (int p = 0; p < 8; p++) {
    const double s = (p & 1) ? g1 : g0, t = (p & 2) ? g1 : g0, u = (p & 4) ? g1 : g0;
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 8; a++) {
      const double fs = cc[a][0] ? s : 1.0 - s, ft = cc[a][1] ? t : 1.0 - t, fu = cc[a][2] ? u : 1.0 - u;
      const double ds = cc[a][0] ? 1.0 : -1.0, dt = cc[a][1] ? 1.0 : -1.0, du = cc[a][2] ? 1.0 : -1.0;
      for (int k = 0; k < 3; k++) {
        J[k][0] += ds * ft * fu * V[a][k];
        J[k][1] += fs * dt * fu * V[a][k];
        J[k][2] += fs * ft * du * V[a][k];
      }
    }
    const double d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    v += 0.125 * fabs(d);
  }
  vol[e] = v;
  for (int t = 0; t < 9; t++) jinv[e * 9 + t] = 0.0;
  float* f = ef + e * NL_EF_STRIDE(3);
  for (int a = 1; a < 8; a++)
    for (int k = 0; k < 3; k++) f[(a - 1) * 3 + k] = (float)(V[a][k] - V[0][k]);
  for (int k = 0; k < 3; k++) {
    const float hi = (float)V[0][k];
    f[21 + k] = hi;
    f[24 + k] = (float)(V[0][k] - (double)hi);
  }
  f[27] = (float)v;
  for (int t = 28; t < NL_EF_STRIDE(3); t++) f[t] = 0.f;
}

__global__ void k_count_n2e(int64_t n_entries, const int32_t* __restrict__ conn,
                            int32_t* __restrict__ cnt) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n_entries) atomicAdd(&cnt[conn[t]], 1);
}

__global__ void k_fill_n2e(int64_t n_entries, int nv, const int32_t* __restrict__ conn,
                           const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ n2e) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_entries) return;
  int32_t v = conn[t];
  int32_t pos = atomicAdd(&cursor[v], 1);
  n2e[off[v] + pos] = (int32_t)(t / nv);
}

}  // namespace

void nlx::mesh_release(nl_mesh* m) {
  if (!m) return;
  if (m->refs.fetch_sub(1) != 1) return;
  cudaStream_t s = m->stream;
  dev_free(m->coords, 0, s);
  dev_free(m->conn, 0, s);
  dev_free(m->elem_in_omega, 0, s);
  dev_free(m->node_free, 0, s);
  dev_free(m->evert, 0, s);
  dev_free(m->blo, 0, s);
  dev_free(m->bhi, 0, s);
  dev_free(m->vol, 0, s);
  dev_free(m->jinv, 0, s);
  dev_free(m->ef, 0, s);
  dev_free(m->n2e_off, 0, s);
  dev_free(m->n2e, 0, s);
  cudaStreamSynchronize(s);
  delete m;
}

// cell 0, order 1: P1 simplices (dim+1 nodes per element); cell 0, order 2: P2 triangles (6
// nodes: the vertices, then the midpoints of the edges (0,1), (1,2), (0,2)); cell 1:
// quadrilaterals (dim 2), order 1 Q1 (the 4 vertices, counterclockwise), order 2 Q2 (the
// vertices, the midpoints of the edges (0,1), (1,2), (2,3), (3,0), the centre).
static nl_status mesh_create_impl(int dim, int order, int cell, int64_t n_vert,
                                  const double* coords, int64_t n_elem, const int32_t* conn,
                                  const uint8_t* eio, const uint8_t* nf, void* cuda_stream,
                                  nl_mesh** out) {
  using namespace nlx;
  if (!out) return fail(NL_EINVAL, "nl_mesh_create: out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(NL_EINVAL, "nl_mesh_create: dim must be 2 or 3");
  if (order != 1 && order != 2 && !(order == 3 && cell != 0))
    return fail(NL_EINVAL, "nl_mesh_create: unknown element order %d", order);
  if (cell == 1 && dim != 2) return fail(NL_EINVAL, "nl_mesh_create_quad: quadrilaterals are 2D");
  if (cell == 2 && dim != 3) return fail(NL_EINVAL, "nl_mesh_create_hex: hexahedra are 3D");
  if (n_vert <= 0 || n_vert > INT32_MAX || n_elem <= 0 || n_elem > INT32_MAX)
    return fail(NL_EINVAL, "nl_mesh_create: bad sizes n_vert=%lld n_elem=%lld",
                (long long)n_vert, (long long)n_elem);
  if (!coords || !conn || !eio || !nf) return fail(NL_EINVAL, "nl_mesh_create: NULL array");
  const int nv = cell == 1 ? 4 : (cell == 2 ? 8 : dim + 1);
  const int nb = cell == 2 ? (order == 2 ? 27 : (order == 3 ? 20 : 8))
                 : cell == 1 ? (order == 2 ? 9 : (order == 3 ? 8 : 4))
                             : (order == 2 ? (dim == 2 ? 6 : 10) : nv);
  for (int64_t i = 0; i < (int64_t)dim * n_vert; i++)
    if (!std::isfinite(coords[i])) return fail(NL_EINVAL, "nl_mesh_create: non-finite coordinate");
  double bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
  double max_ext = 0.0;
  for (int64_t e = 0; e < n_elem; e++) {
    double V[8][3];
    for (int a = 0; a < nb; a++) {
      int32_t v = conn[e * nb + a];
      if (v < 0 || v >= n_vert) return fail(NL_EINVAL, "nl_mesh_create: vertex index out of range");
      if (a < nv)
        for (int k = 0; k < dim; k++) V[a][k] = coords[k * n_vert + v];
    }
    if (cell == 1) {
      // a convex, counterclockwise quadrilateral: the cross product at every corner is
      // positive (the bilinear map's Jacobian is then positive everywhere)
      for (int a = 0; a < 4; a++) {
        const double* p = V[a];
        const double* q = V[(a + 1) & 3];
        const double* r = V[(a + 3) & 3];
        const double cr = (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0]);
        if (!(cr > 0.0))
          return fail(NL_EINVAL, "nl_mesh_create_quad: element %lld is not a convex counterclockwise quadrilateral",
                      (long long)e);
      }
      if (order >= 2) {
        // Q2 / serendipity: edge node 4 + j at the midpoint of edge j = (0,1), (1,2), (2,3),
        // (3,0); Q2 node 8 at the image of the square's centre, the mean of the four vertices
        for (int j = 0; j < nb - 4; j++) {
          const int32_t v = conn[e * nb + 4 + j];
          double d2 = 0.0, l2 = 0.0;
          for (int k = 0; k < 2; k++) {
            const double mid = j < 4 ? (V[j][k] + V[(j + 1) & 3][k]) * 0.5
                                     : (V[0][k] + V[1][k] + V[2][k] + V[3][k]) * 0.25;
            const double d = coords[k * n_vert + v] - mid, ed = V[2][k] - V[0][k];
            d2 += d * d;
            l2 += ed * ed;
          }
          if (!(d2 <= 1e-18 * l2))
            return fail(NL_EINVAL, "nl_mesh_create_quad: node %d of element %lld is off its position",
                        4 + j, (long long)e);
        }
      }
    } else if (order == 2 && cell == 0) {
      // straight-sided P2: edge node nv + j at the midpoint of edge j = (0,1), (1,2), (0,2)
      // (and for tetrahedra (0,3), (1,3), (2,3))
      static const int ea[6] = {0, 1, 0, 0, 1, 2}, eb[6] = {1, 2, 2, 3, 3, 3};
      for (int j = 0; j < nb - nv; j++) {
        const int32_t v = conn[e * nb + nv + j];
        double d2 = 0.0, l2 = 0.0;
        for (int k = 0; k < dim; k++) {
          const double mid = (V[ea[j]][k] + V[eb[j]][k]) * 0.5;
          const double d = coords[k * n_vert + v] - mid, ed = V[eb[j]][k] - V[ea[j]][k];
          d2 += d * d;
          l2 += ed * ed;
        }
        if (!(d2 <= 1e-18 * l2))
          return fail(NL_EINVAL, "nl_mesh_create_p2: edge node %d of element %lld is not at its edge's midpoint",
                      nv + j, (long long)e);
      }
    }
    double det;
    if (cell == 2) {
      // the trilinear map keeps its orientation at every corner: the Jacobian there, the
      // edges from the corner along s, t, u, has a positive determinant
      static const int cc[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                   {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
      auto idx = [](int i, int j, int k) {
        for (int a = 0; a < 8; a++)
          if (cc[a][0] == i && cc[a][1] == j && cc[a][2] == k) return a;
        return 0;
      };
      det = 1.0;
      for (int a = 0; a < 8; a++) {
        const int i = cc[a][0], j = cc[a][1], k = cc[a][2];
        double E[3][3];
        for (int q = 0; q < 3; q++) {
          E[0][q] = V[idx(1, j, k)][q] - V[idx(0, j, k)][q];
          E[1][q] = V[idx(i, 1, k)][q] - V[idx(i, 0, k)][q];
          E[2][q] = V[idx(i, j, 1)][q] - V[idx(i, j, 0)][q];
        }
        const double d = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                         E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                         E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
        if (!(d > 0.0))
          return fail(NL_EINVAL, "nl_mesh_create_hex: element %lld is inverted or degenerate at corner %d",
                      (long long)e, a);
      }
      // Q2, serendipity: node a >= 8 at the trilinear image of its lattice point (i, j, k) / 2
      for (int a = 8; a < nb; a++) {
        const int c = hex27_code(a);
        double w[8];
        hex_basis<8, double>(0.5 * (c % 3), 0.5 * ((c / 3) % 3), 0.5 * (c / 9), 1.0, w);
        const int32_t v = conn[e * nb + a];
        double d2 = 0.0, l2 = 0.0;
        for (int q = 0; q < 3; q++) {
          double x = 0.0;
          for (int b = 0; b < 8; b++) x += w[b] * V[b][q];
          const double d = coords[q * n_vert + v] - x, ed = V[6][q] - V[0][q];
          d2 += d * d;
          l2 += ed * ed;
        }
        if (!(d2 <= 1e-18 * l2))
          return fail(NL_EINVAL, "nl_mesh_create_hex: node %d of element %lld is off its position",
                      a, (long long)e);
      }
    } else if (dim == 2) {
      det = (V[1][0] - V[0][0]) * (V[2][1] - V[0][1]) - (V[2][0] - V[0][0]) * (V[1][1] - V[0][1]);
    } else {
      double a[3], b[3], c[3];
      for (int k = 0; k < 3; k++) {
        a[k] = V[1][k] - V[0][k];
        b[k] = V[2][k] - V[0][k];
        c[k] = V[3][k] - V[0][k];
      }
      det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
            a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(std::fabs(det) > 0.0)) return fail(NL_EINVAL, "nl_mesh_create: degenerate element %lld", (long long)e);
    for (int k = 0; k < dim; k++) {
      double lo = V[0][k], hi = V[0][k];
      for (int a = 1; a < nv; a++) {
        lo = std::fmin(lo, V[a][k]);
        hi = std::fmax(hi, V[a][k]);
      }
      bl[k] = std::fmin(bl[k], lo);
      bh[k] = std::fmax(bh[k], hi);
      max_ext = std::fmax(max_ext, hi - lo);
    }
  }
  NL_TRY(ensure_device_tables());
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  nl_mesh* m = new nl_mesh();
  m->dim = dim;
  m->order = order;
  m->cell = cell;
  m->nb = nb;
  m->n_vert = n_vert;
  m->n_elem = n_elem;
  m->stream = s;
  m->max_ext = max_ext;
  for (int k = 0; k < 3; k++) {
    m->bb_lo[k] = k < dim ? bl[k] : 0.0;
    m->bb_hi[k] = k < dim ? bh[k] : 0.0;
  }
  DevBuf<double> dc, ev, lo, hi, vol, jinv;
  DevBuf<float> efb;
  DevBuf<int32_t> dconn, n2e, cnt;
  DevBuf<uint8_t> deio, dnf;
  DevBuf<int64_t> off;
  nl_status st = NL_OK;
  do {
    if ((st = dc.alloc(dim * n_vert, s)) != NL_OK) break;
    if ((st = dconn.alloc(nb * n_elem, s)) != NL_OK) break;
    if ((st = deio.alloc(n_elem, s)) != NL_OK) break;
    if ((st = dnf.alloc(n_vert, s)) != NL_OK) break;
    if ((st = ev.alloc((int64_t)nv * dim * n_elem, s)) != NL_OK) break;
    if ((st = lo.alloc(dim * n_elem, s)) != NL_OK) break;
    if ((st = hi.alloc(dim * n_elem, s)) != NL_OK) break;
    if ((st = vol.alloc(n_elem, s)) != NL_OK) break;
    if ((st = jinv.alloc(dim * dim * n_elem, s)) != NL_OK) break;
    if ((st = efb.alloc((size_t)NL_EF_STRIDE(dim) * n_elem, s)) != NL_OK) break;
    if ((st = n2e.alloc(nb * n_elem, s)) != NL_OK) break;
    if ((st = cnt.alloc(n_vert, s)) != NL_OK) break;
    if ((st = off.alloc(n_vert + 1, s)) != NL_OK) break;
  } while (0);
  if (st != NL_OK) {
    delete m;
    return st;
  }
  auto cleanup = [&](nl_status e) {
    delete m;
    return e;
  };
  cudaError_t ce;
  if ((ce = cudaMemcpyAsync(dc.p, coords, sizeof(double) * dim * n_vert, cudaMemcpyHostToDevice, s)) ||
      (ce = cudaMemcpyAsync(dconn.p, conn, sizeof(int32_t) * nb * n_elem, cudaMemcpyHostToDevice, s)) ||
      (ce = cudaMemcpyAsync(deio.p, eio, n_elem, cudaMemcpyHostToDevice, s)) ||
      (ce = cudaMemcpyAsync(dnf.p, nf, n_vert, cudaMemcpyHostToDevice, s)) ||
      (ce = cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n_vert, s)))
    return cleanup(cuda_fail(ce, "nl_mesh_create upload"));
  int tb = 256;
  int64_t gb = (n_elem + tb - 1) / tb;
  if (cell == 2)
    k_mesh_hexes<<<NL_CNT((unsigned)gb), tb, 0, s>>>(n_elem, n_vert, dc.p, dconn.p, nb, ev.p, lo.p, hi.p, vol.p, jinv.p, efb.p);
  else if (cell == 1)
    k_mesh_quads<<<NL_CNT((unsigned)gb), tb, 0, s>>>(n_elem, n_vert, dc.p, dconn.p, nb, ev.p, lo.p, hi.p, vol.p, jinv.p, efb.p);
  else if (dim == 2)
    k_mesh_elements<2><<<NL_CNT((unsigned)gb), tb, 0, s>>>(n_elem, n_vert, dc.p, dconn.p, nb, ev.p, lo.p, hi.p, vol.p, jinv.p, efb.p);
  else
    k_mesh_elements<3><<<NL_CNT((unsigned)gb), tb, 0, s>>>(n_elem, n_vert, dc.p, dconn.p, nb, ev.p, lo.p, hi.p, vol.p, jinv.p, efb.p);
  int64_t ne = (int64_t)nb * n_elem;
  k_count_n2e<<<NL_CNT((unsigned)((ne + tb - 1) / tb)), tb, 0, s>>>(ne, dconn.p, cnt.p);
  st = exclusive_scan_i32_to_i64(cnt.p, off.p, n_vert, s);
  if (st != NL_OK) return cleanup(st);
  if ((ce = cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n_vert, s))) return cleanup(cuda_fail(ce, "memset"));
  k_fill_n2e<<<NL_CNT((unsigned)((ne + tb - 1) / tb)), tb, 0, s>>>(ne, nb, dconn.p, off.p, cnt.p, n2e.p);
  if ((ce = cudaGetLastError())) return cleanup(cuda_fail(ce, "nl_mesh_create kernels"));
  if ((ce = cudaStreamSynchronize(s))) return cleanup(cuda_fail(ce, "nl_mesh_create sync"));
  m->coords = dc.release_ownership();
  m->conn = dconn.release_ownership();
  m->elem_in_omega = deio.release_ownership();
  m->node_free = dnf.release_ownership();
  m->evert = ev.release_ownership();
  m->blo = lo.release_ownership();
  m->bhi = hi.release_ownership();
  m->vol = vol.release_ownership();
  m->jinv = jinv.release_ownership();
  m->ef = efb.release_ownership();
  m->n2e = n2e.release_ownership();
  m->n2e_off = off.release_ownership();
  *out = m;
  return NL_OK;
}

// ---- structured box meshes ---------------------------------------------------------------------
static uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

extern "C" nl_status nl_mesh_create_box(int dim, const int32_t* cells, double h, const double* lo,
                                        int32_t layer, double jitter, uint64_t seed,
                                        void* cuda_stream, nl_mesh** out) {
  using namespace nlx;
  clear_error();
  if (dim != 2 && dim != 3) return fail(NL_EINVAL, "nl_mesh_create_box: dim must be 2 or 3");
  if (!cells || !lo || !(h > 0.0) || layer < 0 || !(jitter >= 0.0 && jitter < 0.5))
    return fail(NL_EINVAL, "nl_mesh_create_box: bad arguments");
  int64_t nc[3] = {1, 1, 1}, nl[3] = {1, 1, 1};
  int64_t n_vert = 1, n_cells = 1;
  for (int k = 0; k < dim; k++) {
    if (cells[k] < 1) return fail(NL_EINVAL, "nl_mesh_create_box: cells must be >= 1");
    nc[k] = cells[k] + 2 * (int64_t)layer;
    nl[k] = nc[k] + 1;
    n_vert *= nl[k];
    n_cells *= nc[k];
  }
  int per_cell = dim == 2 ? 2 : 6;
  int64_t n_elem = n_cells * per_cell;
  if (n_vert > INT32_MAX || n_elem > INT32_MAX) return fail(NL_EINVAL, "nl_mesh_create_box: mesh too large");
  std::vector<double> coords(dim * n_vert);
  std::vector<uint8_t> nf(n_vert), eio(n_elem);
  std::vector<int32_t> conn(n_elem * (dim + 1));
  for (int64_t v = 0; v < n_vert; v++) {
    int64_t idx[3], r = v;
    for (int k = 0; k < dim; k++) {
      idx[k] = r % nl[k];
      r /= nl[k];
    }
    bool on_face = false, inside = true;
    for (int k = 0; k < dim; k++) {
      on_face |= idx[k] == 0 || idx[k] == layer || idx[k] == layer + cells[k] || idx[k] == nc[k];
      inside &= idx[k] > layer && idx[k] < layer + cells[k];
    }
    nf[v] = inside ? 1 : 0;
    for (int k = 0; k < dim; k++) {
      double c = lo[k] + (double)(idx[k] - layer) * h;
      if (jitter != 0.0 && !on_face) {
        uint64_t z = splitmix64_at(seed, (uint64_t)v * 4 + k);
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        double off = (jitter * h) * (2.0 * u - 1.0);
        c = c + off;
      }
      coords[k * n_vert + v] = c;
    }
  }
  int64_t stride[3] = {1, nl[0], nl[0] * nl[1]};
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int64_t c = 0; c < n_cells; c++) {
    int64_t idx[3], r = c;
    bool in_omega = true;
    for (int k = 0; k < dim; k++) {
      idx[k] = r % nc[k];
      r /= nc[k];
      in_omega &= idx[k] >= layer && idx[k] < layer + cells[k];
    }
    int64_t base = 0;
    for (int k = 0; k < dim; k++) base += idx[k] * stride[k];
    for (int t = 0; t < per_cell; t++) eio[c * per_cell + t] = in_omega ? 1 : 0;
    if (dim == 2) {
      int32_t v00 = (int32_t)base, v10 = (int32_t)(base + stride[0]), v01 = (int32_t)(base + stride[1]),
              v11 = (int32_t)(base + stride[0] + stride[1]);
      int32_t* e0 = &conn[(c * 2) * 3];
      e0[0] = v00, e0[1] = v10, e0[2] = v11;
      e0[3] = v00, e0[4] = v11, e0[5] = v01;
    } else {
      for (int t = 0; t < 6; t++) {
        int64_t a = base + stride[perms[t][0]];
        int64_t b = a + stride[perms[t][1]];
        int32_t* e = &conn[(c * 6 + t) * 4];
        e[0] = (int32_t)base;
        e[1] = (int32_t)a;
        e[2] = (int32_t)b;
        e[3] = (int32_t)(base + stride[0] + stride[1] + stride[2]);
      }
    }
  }
  return mesh_create_impl(dim, 1, 0, n_vert, coords.data(), n_elem, conn.data(), eio.data(), nf.data(),
                          cuda_stream, out);
}

// ---- C ABI -------------------------------------------------------------------------------------
extern "C" {

nl_status nl_set_allocator(nl_alloc_fn alloc, nl_free_fn free_fn, void* ctx) {
  nlx::clear_error();
  if ((alloc == nullptr) != (free_fn == nullptr))
    return nlx::fail(NL_EINVAL, "nl_set_allocator: give both functions or neither");
  nlx::g_alloc = alloc;
  nlx::g_free = free_fn;
  nlx::g_alloc_ctx = ctx;
  return NL_OK;
}

const char* nl_last_error(void) { return nlx::g_err.c_str(); }

const char* nl_version(void) { return "nlquad-gb300 0.1 (sm_103a)"; }

int64_t nl_launch_count(void) { return nlx::launch_count(); }

nl_status nl_mesh_create(int dim, int64_t n_vert, const double* coords, int64_t n_elem,
                         const int32_t* conn, const uint8_t* elem_in_omega,
                         const uint8_t* node_free, void* cuda_stream, nl_mesh** out) {
  nlx::clear_error();
  return mesh_create_impl(dim, 1, 0, n_vert, coords, n_elem, conn, elem_in_omega, node_free,
                          cuda_stream, out);
}

nl_status nl_mesh_create_p2(int dim, int64_t n_vert, const double* coords, int64_t n_elem,
                            const int32_t* conn, const uint8_t* elem_in_omega,
                            const uint8_t* node_free, void* cuda_stream, nl_mesh** out) {
  nlx::clear_error();
  return mesh_create_impl(dim, 2, 0, n_vert, coords, n_elem, conn, elem_in_omega, node_free,
                          cuda_stream, out);
}

nl_status nl_mesh_create_hex(int order, int64_t n_vert, const double* coords, int64_t n_elem,
                             const int32_t* conn, const uint8_t* elem_in_omega,
                             const uint8_t* node_free, void* cuda_stream, nl_mesh** out) {
  nlx::clear_error();
  if (order < 1 || order > 3) return nlx::fail(NL_EINVAL, "nl_mesh_create_hex: order must be 1, 2 or 3");
  return mesh_create_impl(3, order, 2, n_vert, coords, n_elem, conn, elem_in_omega, node_free,
                          cuda_stream, out);
}

nl_status nl_mesh_create_quad(int order, int64_t n_vert, const double* coords, int64_t n_elem,
                              const int32_t* conn, const uint8_t* elem_in_omega,
                              const uint8_t* node_free, void* cuda_stream, nl_mesh** out) {
  nlx::clear_error();
  if (order < 1 || order > 3) return nlx::fail(NL_EINVAL, "nl_mesh_create_quad: order must be 1, 2 or 3");
  return mesh_create_impl(2, order, 1, n_vert, coords, n_elem, conn, elem_in_omega, node_free,
                          cuda_stream, out);
}

nl_status nl_mesh_order(const nl_mesh* m, int* order, int* nodes_per_elem) {
  nlx::clear_error();
  if (!m) return nlx::fail(NL_EINVAL, "nl_mesh_order: NULL mesh");
  if (order) *order = m->order;
  if (nodes_per_elem) *nodes_per_elem = m->nb;
  return NL_OK;
}

nl_status nl_mesh_info(const nl_mesh* m, int* dim, int64_t* n_vert, int64_t* n_elem) {
  nlx::clear_error();
  if (!m) return nlx::fail(NL_EINVAL, "nl_mesh_info: NULL mesh");
  if (dim) *dim = m->dim;
  if (n_vert) *n_vert = m->n_vert;
  if (n_elem) *n_elem = m->n_elem;
  return NL_OK;
}

nl_status nl_mesh_export(const nl_mesh* m, double* coords, int32_t* conn, uint8_t* eio,
                         uint8_t* nf) {
  nlx::clear_error();
  if (!m) return nlx::fail(NL_EINVAL, "nl_mesh_export: NULL mesh");
  cudaStream_t s = m->stream;
  if (coords) NL_CUDA(cudaMemcpyAsync(coords, m->coords, sizeof(double) * m->dim * m->n_vert, cudaMemcpyDeviceToHost, s));
  if (conn) NL_CUDA(cudaMemcpyAsync(conn, m->conn, sizeof(int32_t) * m->nb * m->n_elem, cudaMemcpyDeviceToHost, s));
  if (eio) NL_CUDA(cudaMemcpyAsync(eio, m->elem_in_omega, m->n_elem, cudaMemcpyDeviceToHost, s));
  if (nf) NL_CUDA(cudaMemcpyAsync(nf, m->node_free, m->n_vert, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  return NL_OK;
}

void nl_mesh_destroy(nl_mesh* m) { nlx::mesh_release(m); }

nl_status nl_pairs_build(nl_mesh* mesh, double delta, double eps, nl_pairs** out) {
  nlx::clear_error();
  if (!mesh || !out) return nlx::fail(NL_EINVAL, "nl_pairs_build: NULL argument");
  *out = nullptr;
  if (!(std::isfinite(delta) && std::isfinite(eps) && eps > 0.0 && eps < delta))
    return nlx::fail(NL_EINVAL, "nl_pairs_build: need 0 < eps < delta (Sec. 3)");
  nl_pairs* p = new nl_pairs();
  nl_status st = nlx::build_pairs(mesh, delta, eps, p);
  if (st != NL_OK) {
    nlx::pairs_release(p);
    return st;
  }
  *out = p;
  return NL_OK;
}

nl_status nl_pairs_info(const nl_pairs* p, int64_t* n_pairs, int64_t* nnz) {
  nlx::clear_error();
  if (!p) return nlx::fail(NL_EINVAL, "nl_pairs_info: NULL pairs");
  if (n_pairs) *n_pairs = p->n_pairs;
  if (nnz) *nnz = p->nnz;
  return NL_OK;
}

nl_status nl_pairs_export(const nl_pairs* p, int64_t* pair_off, int32_t* pair_l, int64_t* row_ptr,
                          int32_t* col) {
  nlx::clear_error();
  if (!p) return nlx::fail(NL_EINVAL, "nl_pairs_export: NULL pairs");
  cudaStream_t s = p->mesh->stream;
  if (pair_off) NL_CUDA(cudaMemcpyAsync(pair_off, p->pair_off, sizeof(int64_t) * (p->mesh->n_elem + 1), cudaMemcpyDeviceToHost, s));
  if (pair_l && p->n_pairs) NL_CUDA(cudaMemcpyAsync(pair_l, p->pair_l, sizeof(int32_t) * p->n_pairs, cudaMemcpyDeviceToHost, s));
  if (row_ptr) NL_CUDA(cudaMemcpyAsync(row_ptr, p->row_ptr, sizeof(int64_t) * (p->mesh->n_vert + 1), cudaMemcpyDeviceToHost, s));
  if (col && p->nnz) NL_CUDA(cudaMemcpyAsync(col, p->col, sizeof(int32_t) * p->nnz, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  return NL_OK;
}

void nl_pairs_destroy(nl_pairs* p) { nlx::pairs_release(p); }

nl_status nl_assemble(nl_mesh* mesh, nl_pairs* pairs, const nl_kernel_params* kp,
                      const nl_quad_params* qp, nl_precision precision, nl_matrix** A,
                      nl_assemble_stats* stats) {
  using namespace nlx;
  clear_error();
  if (!mesh || !pairs || !kp || !qp || !A) return fail(NL_EINVAL, "nl_assemble: NULL argument");
  if (pairs->mesh != mesh) return fail(NL_EINVAL, "nl_assemble: pairs were built on another mesh");
  if (kp->delta != pairs->delta || kp->eps != pairs->eps)
    return fail(NL_EINVAL, "nl_assemble: delta/eps differ from those of the pairs");
  nl_matrix* M = *A;
  bool fresh = false;
  if (M && M->pairs != pairs) return fail(NL_EINVAL, "nl_assemble: *A has another pattern");
  if (!M) {
    M = new nl_matrix();
    M->pairs = pairs;
    M->stream = mesh->stream;
    pairs->refs.fetch_add(1);
    mesh->refs.fetch_add(0);
    M->values = static_cast<double*>(dev_alloc(sizeof(double) * (pairs->nnz ? pairs->nnz : 1), mesh->stream));
    if (!M->values) {
      pairs_release(pairs);
      delete M;
      return fail(NL_ENOMEM, "nl_assemble: cannot allocate %lld values", (long long)pairs->nnz);
    }
    fresh = true;
  }
  nl_status st = assemble_values(mesh, pairs, kp, qp, precision, M->values, stats);
  if (st != NL_OK) {
    if (fresh) nl_matrix_destroy(M);
    return st;
  }
  *A = M;
  return NL_OK;
}

nl_status nl_matrix_apply(const nl_matrix* A, const double* x, double* y) {
  nlx::clear_error();
  if (!A || !x || !y) return nlx::fail(NL_EINVAL, "nl_matrix_apply: NULL argument");
  if (x == y) return nlx::fail(NL_EINVAL, "nl_matrix_apply: x and y must not alias");
  return nlx::apply_matrix(A, x, y);
}

nl_status nl_matrix_export(const nl_matrix* A, double* values) {
  nlx::clear_error();
  if (!A || !values) return nlx::fail(NL_EINVAL, "nl_matrix_export: NULL argument");
  if (A->pairs->nnz)
    NL_CUDA(cudaMemcpyAsync(values, A->values, sizeof(double) * A->pairs->nnz, cudaMemcpyDeviceToHost, A->stream));
  NL_CUDA(cudaStreamSynchronize(A->stream));
  return NL_OK;
}

nl_status nl_matrix_device_values(const nl_matrix* A, double** values) {
  nlx::clear_error();
  if (!A || !values) return nlx::fail(NL_EINVAL, "nl_matrix_device_values: NULL argument");
  *values = A->values;
  return NL_OK;
}

void nl_matrix_destroy(nl_matrix* A) {
  if (!A) return;
  nlx::dev_free(A->values, 0, A->stream);
  cudaStreamSynchronize(A->stream);
  nlx::pairs_release(A->pairs);
  delete A;
}

nl_status nl_rhs(nl_mesh* mesh, nl_matrix* A, const double* f_nodes, double f_const,
                 const double* g_nodes, nl_vector** rhs) {
  using namespace nlx;
  clear_error();
  if (!mesh || !A || !g_nodes || !rhs) return fail(NL_EINVAL, "nl_rhs: NULL argument");
  if (A->pairs->mesh != mesh) return fail(NL_EINVAL, "nl_rhs: matrix of another mesh");
  nl_vector* v = new nl_vector();
  v->mesh = mesh;
  mesh->refs.fetch_add(1);
  v->n = mesh->n_vert;
  v->stream = mesh->stream;
  v->v = static_cast<double*>(dev_alloc(sizeof(double) * v->n, v->stream));
  if (!v->v) {
    nl_vector_destroy(v);
    return fail(NL_ENOMEM, "nl_rhs: allocation failed");
  }
  nl_status st = rhs_values(mesh, A, f_nodes, f_const, g_nodes, v->v);
  if (st != NL_OK) {
    nl_vector_destroy(v);
    return st;
  }
  *rhs = v;
  return NL_OK;
}

nl_status nl_vector_export(const nl_vector* v, double* values) {
  nlx::clear_error();
  if (!v || !values) return nlx::fail(NL_EINVAL, "nl_vector_export: NULL argument");
  NL_CUDA(cudaMemcpyAsync(values, v->v, sizeof(double) * v->n, cudaMemcpyDeviceToHost, v->stream));
  NL_CUDA(cudaStreamSynchronize(v->stream));
  return NL_OK;
}

void nl_vector_destroy(nl_vector* v) {
  if (!v) return;
  nlx::dev_free(v->v, 0, v->stream);
  cudaStreamSynchronize(v->stream);
  nlx::mesh_release(v->mesh);
  delete v;
}

nl_status nl_solve(nl_matrix* A, const nl_vector* rhs, const double* g_nodes, int solver,
                   double rtol, int max_iter, nl_precision precision, double* u_out, int* iters,
                   double* final_rel_res) {
  using namespace nlx;
  clear_error();
  if (!A || !rhs || !g_nodes || !u_out) return fail(NL_EINVAL, "nl_solve: NULL argument");
  if (rhs->mesh != A->pairs->mesh) return fail(NL_EINVAL, "nl_solve: rhs of another mesh");
  if (solver != 0 && solver != 1) return fail(NL_EINVAL, "nl_solve: solver must be 0 (CG) or 1 (BiCGStab)");
  if (!(rtol > 0.0) || max_iter < 1) return fail(NL_EINVAL, "nl_solve: need rtol > 0 and max_iter >= 1");
  return solve_system(A, rhs, g_nodes, solver, rtol, max_iter, precision, u_out, iters, final_rel_res);
}

}  // extern "C"
