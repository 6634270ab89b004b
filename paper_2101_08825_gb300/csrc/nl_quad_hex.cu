// nl_quad_hex.cu -- nl_assemble on meshes of hexahedra (Sec. 6: the HEX meshes of the 3D
// tests, Q1 trilinear, Q2 triquadratic or 20-node serendipity elements, the Gauss-Legendre
// 3x3x3 product rule for the inner and the outer integral).
//
// What is computed (Sec. 5, Corollary 1, eqs. J21Nr and J22Nr): for every element pair
// (m, l) of J, with the 3x3x3 rule on E_m (points y = F_m(g), weights w_y |det DF_m|, rows =
// the NN nodes of m) and on the sub-elements E' of E_l that Algorithm 1 selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_d] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_d(x).
// An element is the trilinear image F of the unit cube (its 8 vertices; the other nodes of a
// Q2 or serendipity element sit at the images of the lattice of half steps); a sub-element
// is the image of a sub-cube of l's cube, its outer points x = F_l(s0 + len g_i, t0 + len g_j,
// u0 + len g_k) with weights w_i w_j w_k len^3 |det DF_l| and the basis of l at those
// reference points.
// Algorithm 1 splits a cube into its eight half-size sub-cubes and decides on the box of the
// sub-element's physical vertices, which lie on the lattice of half steps: a lattice point
// with a middle index is the midpoint (a+b)*0.5 of its two neighbours along the first such
// axis (x, then y, then z).
//
// How (k_quad_h): the structure of the other assembly kernels -- a persistent grid, chunks of
// consecutive m-major pairs per warp, Algorithm 1 as a warp LIFO (4 parents x 8 children per
// round), decisions in FP64 (FP64 path) or by the FP32 screen with an FP64 re-decision inside
// the margin (FP32 path), buffered sub-elements integrated by the whole warp.
//  Q1 (NN = 8): the warp is four groups of eight lanes: a pass takes 8 outer points, one per
// lane of a group, and the groups hold inner points 0-6, 7-13, 14-20 and 21-26 of m (56 sums
// H_d(y) = sum_x w_x C eta mu phi^l_d(x) per lane).  The end of a pair sums H over the 8 lanes
// of each group through shared memory, writes the cross block -2 sum_y w_y |det DF_m|
// phi^m_a(y) H_d(y) and keeps g(y) = sum_d H_d(y) for m's self block.  With the constant
// kernel an INT sub-element adds sum_x w_x C phi^l_d(x), independent of y, to every inner
// point without evaluating point pairs.
//  Q2 and serendipity (NN = 27, 20; the wide layout): lane q < 27 holds inner point q and its
// NN sums H_d(y_q).  A pass stages 32 outer points in shared memory (one per lane: x, the
// item's kind and w_x phi^l_d(x) for the NN d), then every lane runs over the staged points
// (the same point on every lane, so the mollifier's branch is uniform).  A constant-kernel
// INT sub-element's points are not paired: lane d sums their w_x C phi^l_d(x).  At the end of
// a pair the H table is transposed through shared memory so that lane d computes column d of
// the cross block (NN x 27 products with the broadcast rows w_y phi^m_a(y)).
#include <cuda_runtime.h>

#include "nl_quad_kernel.cuh"

namespace nlx {
namespace {

constexpr int HX_NQ = 27;      // Gauss-Legendre 3x3x3 points
constexpr int HX_IMAX = 64;    // buffered sub-elements
constexpr int HX_RS = 9;       // row stride of the Q1 reduction scratch
constexpr int HX_REC = 28;     // LIFO record: 8 vertices x 3, s0, t0, u0, pad
constexpr int HX_WARPS = 4;
constexpr int HX_SR = 32;      // wide layout: staged outer point: x, y, z, kind, w_x phi^l_d, pad
constexpr int HX_WP = 28;      // wide layout: row stride of the tables over the points or nodes

// item kinds
constexpr int HK_INT = 0, HK_FINAL = 1, HK_CLOSED = 2;

// per-lane layout of the inner points: NYL points per lane, XPI outer points per pass
template <int NN>
struct HxLay {
  static constexpr int NYL = NN == 8 ? 7 : 1;
  static constexpr int XPI = NN == 8 ? 8 : 32;
  static constexpr int NBLK = NN * NN;
};

// hexahedron corner a = (x, y, z) bits of the unit cube
__host__ __device__ constexpr int hx_c(int a, int k) {
  return k == 0 ? ((a == 1 || a == 2 || a == 5 || a == 6) ? 1 : 0)
                : k == 1 ? ((a == 2 || a == 3 || a == 6 || a == 7) ? 1 : 0) : (a >= 4 ? 1 : 0);
}

// FP32 element record of a hexahedron (k_mesh_hexes): offsets v_a - v_0 at [0, 21), v_0 high
// and low parts at [21, 24) and [24, 27)
constexpr int HX_EF_V0HI = 21, HX_EF_V0LO = 24;

// block tables: the rule (s, t, u, w) in FP64 and R, the basis at the rule's points in FP64
template <typename R, int NN>
__host__ __device__ constexpr size_t hx_table_bytes() {
  return (sizeof(double) * (HX_NQ * 4 + HX_NQ * NN) + sizeof(R) * (HX_NQ * 4) + 15) & ~size_t(15);
}

template <typename R, int NN>
struct HMem {
  // Q1: wpm [8][27], red [8 * 27][RS] + hs [8 * 27 + 8];
  // wide: wpm [NN][WP], red = the staged outer points [32][SR], at the end of a pair the
  //       transposed H table [27][WP]
  static constexpr size_t WPM_N = NN == 8 ? 8 * HX_NQ : 27 * HX_WP;
  static constexpr size_t RED_N = NN == 8 ? (size_t)8 * HX_NQ * HX_RS + 8 * HX_NQ + 8 : 32 * HX_SR;
  R* sv;         // [scap][REC]
  uint32_t* sc;  // [scap]
  R* it;         // [IMAX][8]: s0, t0, u0, len, kind
  R* wpm;        // w_y |det DF_m(y)| phi^m_a(y)
  R* vl;         // [32]: E_l's 8 vertices in the frame of the inner points
  double* wd;    // [28]
  R* red;
  R* hs;
  double* sd;    // [28]
  static __host__ __device__ size_t bytes(int scap) {
    size_t b = sizeof(R) * HX_REC * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * ((size_t)HX_IMAX * 8 + WPM_N + 32);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * 28;
    b += sizeof(R) * RED_N;
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * 28;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    sv = reinterpret_cast<R*>(base);
    sc = reinterpret_cast<uint32_t*>(sv + HX_REC * (size_t)scap);
    size_t off = sizeof(R) * HX_REC * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    off = (off + 15) & ~size_t(15);
    it = reinterpret_cast<R*>(base + off);
    wpm = it + (size_t)HX_IMAX * 8;
    vl = wpm + WPM_N;
    off += sizeof(R) * ((size_t)HX_IMAX * 8 + WPM_N + 32);
    off = (off + 15) & ~size_t(15);
    wd = reinterpret_cast<double*>(base + off);
    off += sizeof(double) * 28;
    red = reinterpret_cast<R*>(base + off);  // 16-byte aligned: 28 doubles after an aligned offset
    hs = red + (size_t)8 * HX_NQ * HX_RS;    // Q1 only
    off += sizeof(R) * RED_N;
    off = (off + 15) & ~size_t(15);
    sd = reinterpret_cast<double*>(base + off);
  }
};

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = b.x;
  o[3] = b.y;
}

// x = F(s, t, u) of the hexahedron V (8 vertices, x y z each), |det DF(s, t, u)| and the
// trilinear basis N
template <typename R>
__device__ __forceinline__ void hmap(const R* V, R s, R t, R u, R (&x)[3], R& det, R (&N)[8]) {
  R J[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    x[k] = 0;
    J[k][0] = J[k][1] = J[k][2] = 0;
  }
#pragma unroll
  for (int a = 0; a < 8; a++) {
    const R fs = hx_c(a, 0) ? s : (R)1 - s, ft = hx_c(a, 1) ? t : (R)1 - t;
    const R fu = hx_c(a, 2) ? u : (R)1 - u;
    const R ds = hx_c(a, 0) ? (R)1 : (R)-1, dt = hx_c(a, 1) ? (R)1 : (R)-1;
    const R du = hx_c(a, 2) ? (R)1 : (R)-1;
    N[a] = fs * ft * fu;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const R v = V[a * 3 + k];
      x[k] += N[a] * v;
      J[k][0] += ds * ft * fu * v;
      J[k][1] += fs * dt * fu * v;
      J[k][2] += fs * ft * du * v;
    }
  }
  const R d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
              J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  det = d < (R)0 ? -d : d;
}

// Child c (bits x, y, z of the sub-cube) of the hexahedron P: its vertices on the lattice of
// half steps (see the file's header), computed per coordinate with compile-time indices.
template <typename R>
__device__ __forceinline__ void hchild(const R* P, int c, R (&V)[8][3]) {
  const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
#pragma unroll
  for (int q = 0; q < 3; q++) {
    R L[3][3][3];
#pragma unroll
    for (int a = 0; a < 8; a++) L[2 * hx_c(a, 0)][2 * hx_c(a, 1)][2 * hx_c(a, 2)] = P[a * 3 + q];
#pragma unroll
    for (int i = 0; i < 3; i += 2) {
#pragma unroll
      for (int j = 0; j < 3; j += 2) L[i][j][1] = midp(L[i][j][0], L[i][j][2]);
#pragma unroll
      for (int k = 0; k < 3; k++) L[i][1][k] = midp(L[i][0][k], L[i][2][k]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
      for (int k = 0; k < 3; k++) L[1][j][k] = midp(L[0][j][k], L[2][j][k]);
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int ax = hx_c(a, 0), ay = hx_c(a, 1), az = hx_c(a, 2);
      const R v0 = cz ? L[ax][ay][az + 1] : L[ax][ay][az];
      const R v1 = cz ? L[ax][ay + 1][az + 1] : L[ax][ay + 1][az];
      const R v2 = cz ? L[ax + 1][ay][az + 1] : L[ax + 1][ay][az];
      const R v3 = cz ? L[ax + 1][ay + 1][az + 1] : L[ax + 1][ay + 1][az];
      const R w0 = cy ? v1 : v0, w1 = cy ? v3 : v2;
      V[a][q] = cx ? w1 : w0;
    }
  }
}

// Box distances of Sec. 5.1 between the box of the 8 vertices V and (lo2, hi2), FP64 in the
// order of a plain evaluation.
__device__ void hexact_dists(const double (&V)[8][3], const double* lo2, const double* hi2,
                             double& amax, double& amin, bool l2) {
  double s = 0.0, mn = 0.0, e = 0.0;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    double lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a < 8; a++) {
      lo = V[a][k] < lo ? V[a][k] : lo;
      hi = V[a][k] > hi ? V[a][k] : hi;
    }
    double d1 = __dsub_rn(lo, hi2[k]);
    double d2 = __dsub_rn(lo2[k], hi);
    double p = __dmul_rn(d1, d1), q = __dmul_rn(d2, d2);
    s = __dadd_rn(s, p > q ? p : q);
    double t = d1 > d2 ? d1 : d2;
    mn = t > mn ? t : mn;
    const double u = t < 0.0 ? 0.0 : t;
    e = __dadd_rn(e, __dmul_rn(u, u));
  }
  amax = __dsqrt_rn(s);
  amin = l2 ? __dsqrt_rn(e) : mn;
}

__device__ __forceinline__ void hscreen_dists(const float (&V)[8][3], const float* lo2,
                                              const float* hi2, float& amax, float& amin,
                                              float& amin2) {
  float s = 0.f, mn = 0.f, e = 0.f;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    float lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a < 8; a++) {
      lo = fminf(lo, V[a][k]);
      hi = fmaxf(hi, V[a][k]);
    }
    float d1 = lo - hi2[k], d2 = lo2[k] - hi;
    s += fmaxf(d1 * d1, d2 * d2);
    const float t = fmaxf(d1, d2);
    mn = fmaxf(mn, t);
    const float u = fmaxf(t, 0.f);
    e = fmaf(u, u, e);
  }
  amax = s;
  amin = mn;
  amin2 = e;
}

// FP64 decision below L_max for the sub-element with path `code` (3 bits per level), its
// vertices rebuilt from E_l's by the same lattice midpoints.
__device__ __noinline__ int hexact_classify(const double* __restrict__ evert_l,
                                            const double* __restrict__ lo_m,
                                            const double* __restrict__ hi_m, uint32_t code,
                                            double dme, double dpe, bool l2) {
  double V[8][3], lo2[3], hi2[3];
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int k = 0; k < 3; k++) V[a][k] = evert_l[a * 3 + k];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    lo2[k] = lo_m[k];
    hi2[k] = hi_m[k];
  }
  const int level = code >> LEVEL_SHIFT;
  for (int lv = 2; lv <= level; lv++) {
    const int c = (code >> (3 * (lv - 2))) & 7;
    double P[24];
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
      for (int k = 0; k < 3; k++) P[a * 3 + k] = V[a][k];
    hchild<double>(P, c, V);
  }
  double amax, amin;
  hexact_dists(V, lo2, hi2, amax, amin, l2);
  if (amax < dme) return ACT_INT;
  if (amin < dpe) return ACT_REFINE;
  return ACT_DROP;
}

template <typename R, int KERN, int NN>
__global__ void __launch_bounds__(HX_WARPS * 32,
                                  std::is_same<R, float>::value ? (NN == 8 ? 2 : 3) : 1)
    k_quad_h(const QParams P) {
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr bool WIDE = NN != 8;  // Q2 or serendipity: one inner point per lane
  constexpr int NYL = HxLay<NN>::NYL, XPI = HxLay<NN>::XPI, NBLK = HxLay<NN>::NBLK;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) char smem_raw[];
  double* tS = reinterpret_cast<double*>(smem_raw);  // [27][4]: s, t, u, w
  double* tB = tS + HX_NQ * 4;                        // [27][NN]: the basis at point q
  R* rS = reinterpret_cast<R*>(tB + HX_NQ * NN);
  for (int q = threadIdx.x; q < HX_NQ; q += blockDim.x) {
    const int i = q / 9, j = (q / 3) % 3, k = q % 3;
    const double s = P.B[i][0], t = P.B[j][0], u = P.B[k][0];  // the 3-point rule (host-filled)
    tS[q * 4] = s;
    tS[q * 4 + 1] = t;
    tS[q * 4 + 2] = u;
    tS[q * 4 + 3] = P.W[i] * P.W[j] * P.W[k];
    hex_basis<NN, double>(s, t, u, 1.0, tB + q * NN);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < HX_NQ * 4; t += blockDim.x) rS[t] = (R)tS[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // Q1: first inner point of this lane's group and its outer point slot; wide: inner point q
  const int ybase = WIDE ? lane : (lane >> 3) * NYL;
  const int xl = WIDE ? lane : lane & 7;
  HMem<R, NN> wm;
  wm.carve(smem_raw + hx_table_bytes<R, NN>() + (size_t)wid * HMem<R, NN>::bytes(P.scap), P.scap);

  unsigned st_items = 0, st_exact = 0, st_eval = 0, st_closed = 0, st_band = 0;
  int err = 0;
  int64_t cur_m = -1;
  double v0m[3] = {0.0, 0.0, 0.0}, mlo[3] = {0.0, 0.0, 0.0}, mhi[3] = {0.0, 0.0, 0.0};
  float v0h[3] = {0.f, 0.f, 0.f}, v0l[3] = {0.f, 0.f, 0.f}, flo[3] = {0.f, 0.f, 0.f};
  float fhi[3] = {0.f, 0.f, 0.f};
  R y[NYL][3];
  R gsh = 0, gsl = 0;  // lane q < 27: sum of g(y_q) over the current m-run

  // m's self block from g(y_q) summed over the m-run: 2 sum_q w_q phi_a(y_q) phi_b(y_q) g(y_q),
  // symmetric, so only the NN (NN + 1) / 2 entries a <= b are summed, then mirrored
  auto flush_self = [&]() {
    if (lane < HX_NQ) wm.sd[lane] = ((double)gsh + (double)gsl) * wm.wd[lane];
    gsh = gsl = 0;
    __syncwarp();
    constexpr int NTRI = NN * (NN + 1) / 2;
    for (int t = lane; t < NTRI; t += 32) {
      int a = 0, r = t;
      while (r >= NN - a) {  // row a of the upper triangle holds NN - a entries
        r -= NN - a;
        a++;
      }
      const int b = a + r;
      double s = 0.0;
      for (int q = 0; q < HX_NQ; q++) s = fma(tB[q * NN + a] * tB[q * NN + b], wm.sd[q], s);
      atomicAdd(&P.selfblk[cur_m * NBLK + a * NN + b], 2.0 * s);
      if (b != a) atomicAdd(&P.selfblk[cur_m * NBLK + b * NN + a], 2.0 * s);
    }
    __syncwarp();
  };
  auto flush_stats = [&]() {
    for (int o = 16; o > 0; o >>= 1) {
      st_items += __shfl_xor_sync(FULL, st_items, o);
      st_exact += __shfl_xor_sync(FULL, st_exact, o);
      st_closed += __shfl_xor_sync(FULL, st_closed, o);
      st_band += __shfl_xor_sync(FULL, st_band, o);
      err |= __shfl_xor_sync(FULL, err, o);
    }
    if (lane == 0) {
      if (st_items) atomicAdd(&P.stats[0], (unsigned long long)st_items);
      if (st_exact) atomicAdd(&P.stats[2], (unsigned long long)st_exact);
      if (st_eval) atomicAdd(&P.stats[3], (unsigned long long)st_eval);  // alike on every lane
      if (st_closed) atomicAdd(&P.stats[4], (unsigned long long)st_closed);
      if (st_band) atomicAdd(&P.stats[5], (unsigned long long)st_band);
      if (err) atomicOr(P.err, err);
    }
    st_items = st_exact = st_eval = st_closed = st_band = 0;
    err = 0;
    __syncwarp();
  };

  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(P.counter, (unsigned long long)P.chunk);
    start = __shfl_sync(FULL, start, 0);
    const int64_t g0 = P.p_begin + (int64_t)start;
    if (g0 >= P.p_end) break;
    const int64_t g1 = min(g0 + (int64_t)P.chunk, P.p_end);
    int64_t m;
    if (cur_m >= 0 && P.pair_off[cur_m] <= g0 && g0 < P.pair_off[cur_m + 1]) {
      m = cur_m;
    } else {
      int64_t lo = 0, hi = P.n_elem;
      while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t idx = lo + (int64_t)lane * step;
        const bool le = idx < hi && P.pair_off[idx] <= g0;
        const unsigned bal = __ballot_sync(FULL, le);
        const int last = 31 - __clz(bal);  // lane 0 probes lo itself, so bal != 0
        const int64_t nlo = lo + (int64_t)last * step;
        hi = min(hi, nlo + step);
        lo = nlo;
      }
      m = lo;
    }
    int64_t m_end = P.pair_off[m + 1];
    for (int64_t p = g0; p < g1; p++) {
      while (p >= m_end) {
        m++;
        m_end = P.pair_off[m + 1];
      }
      if (m != cur_m) {
        if (cur_m >= 0) flush_self();
        cur_m = m;
        double Vmr[24];  // m's vertices relative to its first one
#pragma unroll
        for (int k = 0; k < 3; k++) {
          v0m[k] = P.evert[(m * 8) * 3 + k];
          mlo[k] = P.blo[m * 3 + k];
          mhi[k] = P.bhi[m * 3 + k];
        }
#pragma unroll
        for (int a = 0; a < 8; a++)
#pragma unroll
          for (int k = 0; k < 3; k++) Vmr[a * 3 + k] = P.evert[(m * 8 + a) * 3 + k] - v0m[k];
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          const int q = min(ybase + i, HX_NQ - 1);
          double x[3], det, N[8];
          hmap<double>(Vmr, tS[q * 4], tS[q * 4 + 1], tS[q * 4 + 2], x, det, N);
#pragma unroll
          for (int k = 0; k < 3; k++) y[i][k] = (R)x[k];
        }
        if (lane < HX_NQ) {
          double x[3], det, N[8];
          hmap<double>(Vmr, tS[lane * 4], tS[lane * 4 + 1], tS[lane * 4 + 2], x, det, N);
          const double wy = tS[lane * 4 + 3] * det;
          wm.wd[lane] = wy;
          if constexpr (WIDE) {
#pragma unroll 1
            for (int a = 0; a < NN; a++) wm.wpm[a * HX_WP + lane] = (R)(wy * tB[lane * NN + a]);
          } else {
#pragma unroll
            for (int a = 0; a < 8; a++) wm.wpm[a * HX_NQ + lane] = (R)(wy * N[a]);
          }
        } else if (WIDE && lane == HX_NQ) {
          for (int a = 0; a < NN; a++) wm.wpm[a * HX_WP + HX_NQ] = (R)0;  // the rows' pad
        }
        if constexpr (F32) {
          const float* ef = P.ef + m * NL_EF_STRIDE(3);
#pragma unroll
          for (int k = 0; k < 3; k++) {
            v0h[k] = ef[HX_EF_V0HI + k];
            v0l[k] = ef[HX_EF_V0LO + k];
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int a = 1; a < 8; a++) {
              const float v = ef[(a - 1) * 3 + k];
              lo = v < lo ? v : lo;
              hi = v > hi ? v : hi;
            }
            flo[k] = lo;
            fhi[k] = hi;
          }
        }
        __syncwarp();
      }
      const int32_t l = P.pair_l[p];
      // E_l's vertices: R = float in the local FP32 frame (the screen's), R = double global (the
      // decisions); in shared memory in the frame of the inner points (the integration)
      const R wl = F32 ? (R)P.fC : (R)P.C;
      if (lane < 24) {
        const int a = lane / 3, k = lane % 3;
        R v;
        if constexpr (F32) {
          const float* ef = P.ef + (int64_t)l * NL_EF_STRIDE(3);
          const float o = (ef[HX_EF_V0HI + k] - v0h[k]) + (ef[HX_EF_V0LO + k] - v0l[k]);
          v = a == 0 ? o : o + ef[(a - 1) * 3 + k];
        } else {
          v = P.evert[((int64_t)l * 8 + a) * 3 + k] - v0m[k];
        }
        wm.vl[lane] = v;
      }
      __syncwarp();
      const R* VL = wm.vl;
      R H[NN][NYL];
#pragma unroll
      for (int d = 0; d < NN; d++)
#pragma unroll
        for (int i = 0; i < NYL; i++) H[d][i] = 0;
      // Q1: the closed forms' sums per node d; wide: lane d's sum for node d
      R U[WIDE ? 1 : NN];
#pragma unroll
      for (int d = 0; d < (WIDE ? 1 : NN); d++) U[d] = 0;
      bool contrib = false, has_u = false;

      auto classify = [&](const R (&V)[8][3], uint32_t code, bool count_exact) -> int {
        const int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        const bool last = level == P.L_max;
        const bool l2 = P.mindist_l2 != 0;
        if constexpr (F32) {
          float fam, fan, fe2;
          hscreen_dists(V, flo, fhi, fam, fan, fe2);
          const bool c_int = fam < P.fint2;
          const bool c_notint = fam > P.fnotint2;
          const bool c_ref = l2 ? fe2 < P.fref2 : fan < P.fdpe - P.margin;
          const bool c_out = l2 ? fe2 > P.fout2 : fan > P.fdpe + P.margin;
          if (last) return c_int ? ACT_INT : (c_out ? ACT_ZERO : ACT_FINAL);
          if (c_int) return ACT_INT;
          if (c_notint && c_ref) return ACT_REFINE;
          if (c_notint && c_out) return ACT_DROP;
          st_exact += count_exact ? 1 : 0;
          return hexact_classify(P.evert + (int64_t)l * 24, P.blo + cur_m * 3, P.bhi + cur_m * 3,
                                 code, P.dme, P.dpe, l2);
        } else {
          double amax, amin;
          hexact_dists(V, mlo, mhi, amax, amin, l2);
          if (last) return amax < P.dme ? ACT_INT : (amin > P.dpe ? ACT_ZERO : ACT_FINAL);
          if (amax < P.dme) return ACT_INT;
          if (amin < P.dpe) return ACT_REFINE;
          return ACT_DROP;
        }
      };
      // Q1: closed form of an INT sub-element (constant kernel): sum_x w_x C phi^l_d(x) over
      // the sub-cube, the same at every inner point (summed over the warp at the end of the pair)
      auto closed_int = [&](R s0, R t0, R u0, R len) {
        if constexpr (!WIDE) {
#pragma unroll 1
          for (int q = 0; q < HX_NQ; q++) {  // not unrolled: rare, keeps the code small
            R x[3], det, N[8];
            hmap<R>(VL, s0 + len * rS[q * 4], t0 + len * rS[q * 4 + 1], u0 + len * rS[q * 4 + 2], x, det, N);
            const R w = rS[q * 4 + 3] * det * (wl * len * len * len);
#pragma unroll
            for (int d = 0; d < NN; d++) U[d] += w * N[d];
          }
          has_u = true;
          st_closed++;
          contrib = true;
        }
      };
      auto put_item = [&](int slot, R s0, R t0, R u0, int level, int kind) {
        R* r = wm.it + slot * 8;
        r[0] = s0;
        r[1] = t0;
        r[2] = u0;
        r[3] = pow2m(R(0), level - 1);  // the sub-cube's side, a power of two
        r[4] = (R)kind;
      };
      auto push = [&](int slot, const R (&V)[8][3], R s0, R t0, R u0, uint32_t code) {
        R* r = wm.sv + slot * HX_REC;
#pragma unroll
        for (int a = 0; a < 8; a++)
#pragma unroll
          for (int k = 0; k < 3; k++) r[a * 3 + k] = V[a][k];
        r[24] = s0;
        r[25] = t0;
        r[26] = u0;
        wm.sc[slot] = code;
      };
      // Q1: 8 outer points per pass, each paired with the 7 inner points of the lane's group
      auto integrate1 = [&](int n_it) {
        const int n_x = n_it * HX_NQ;
        st_eval += (unsigned)(n_x * HX_NQ);
        contrib = true;
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        for (int base = 0; base < n_x; base += XPI) {
          const int o = base + xl;
          const bool valid = o < n_x;
          const int itx = valid ? o / HX_NQ : 0;
          const int q = valid ? o - itx * HX_NQ : 0;
          const R* r = wm.it + itx * 8;
          const R len = r[3];
          const bool fin = r[4] == (R)HK_FINAL;
          R x[3], det, N[8];
          hmap<R>(VL, r[0] + len * rS[q * 4], r[1] + len * rS[q * 4 + 1], r[2] + len * rS[q * 4 + 2], x, det, N);
          const R wx = valid ? rS[q * 4 + 3] * (wl * len * len * len) * det : (R)0;
          R bw[8];
#pragma unroll
          for (int d = 0; d < 8; d++) bw[d] = wx * N[d];
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            const bool yv = ybase + i < HX_NQ;
            const R d0 = x[0] - y[i][0], d1 = x[1] - y[i][1], d2 = x[2] - y[i][2];
            const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
            R g = 1;
            if constexpr (F32) {
              const float mu = mollifier_bf(MK, r2);
              g = fin ? mu : 1.f;
              if (P.count_band) st_band += (valid && yv && fin && r2 >= P.fdme2 && r2 <= P.fdpe2) ? 1 : 0;
            } else {
              if (fin) g = mollifier(P, r2);
              if (P.count_band)
                st_band += (valid && yv && fin && r2 >= P.dme * P.dme && r2 <= P.dpe * P.dpe) ? 1 : 0;
            }
            if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= eta_gauss<R>(P, r2);
#pragma unroll
            for (int d = 0; d < (WIDE ? 1 : NN); d++) H[d][i] += g * bw[d];
          }
        }
      };
      // wide layout: 32 outer points staged per pass; every lane runs over the staged points
      auto integrate2 = [&](int n_it) {
        const int n_x = n_it * HX_NQ;
        contrib = true;
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        for (int base = 0; base < n_x; base += XPI) {
          const int o = base + lane;
          const bool valid = o < n_x;
          const int itx = valid ? o / HX_NQ : 0;
          const int q = valid ? o - itx * HX_NQ : 0;
          const R* r = wm.it + itx * 8;
          const R len = r[3];
          const R kind = r[4];
          const R s = r[0] + len * rS[q * 4], t = r[1] + len * rS[q * 4 + 1], u = r[2] + len * rS[q * 4 + 2];
          R x[3], det, N[8];
          hmap<R>(VL, s, t, u, x, det, N);
          const R wx = valid ? rS[q * 4 + 3] * (wl * len * len * len) * det : (R)0;
          R* sp = wm.red + lane * HX_SR;
          sp[0] = x[0];
          sp[1] = x[1];
          sp[2] = x[2];
          sp[3] = kind;
          hex_basis<NN, R>(s, t, u, wx, sp + 4);
          sp[31] = (R)0;
          __syncwarp();
          const unsigned vm = __ballot_sync(FULL, valid);
          const unsigned cm = __ballot_sync(FULL, valid && kind == (R)HK_CLOSED);
          if (cm != 0u && lane < NN) {
            unsigned c = cm;
            while (c) {
              const int oo = __ffs(c) - 1;
              c &= c - 1u;
              U[0] += wm.red[oo * HX_SR + 4 + lane];
            }
          }
          unsigned em = vm & ~cm;
          st_eval += (unsigned)(__popc(em) * HX_NQ);
          while (em) {
            const int oo = __ffs(em) - 1;
            em &= em - 1u;
            const R* op = wm.red + oo * HX_SR;
            R hd[4];
            ld4(op, hd);
            const R d0 = hd[0] - y[0][0], d1 = hd[1] - y[0][1], d2 = hd[2] - y[0][2];
            const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
            R g = 1;
            if (hd[3] == (R)HK_FINAL) {  // the same staged point on every lane: a uniform branch
              if constexpr (F32) {
                g = mollifier_bf(MK, r2);
                if (P.count_band) st_band += (lane < HX_NQ && r2 >= P.fdme2 && r2 <= P.fdpe2) ? 1 : 0;
              } else {
                g = mollifier(P, r2);
                if (P.count_band) st_band += (lane < HX_NQ && r2 >= P.dme * P.dme && r2 <= P.dpe * P.dpe) ? 1 : 0;
              }
            }
            if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= eta_gauss<R>(P, r2);
#pragma unroll
            for (int j = 0; j < 7; j++) {
              R b[4];
              ld4(op + 4 + 4 * j, b);
#pragma unroll
              for (int v = 0; v < 4; v++)
                if (4 * j + v < NN) H[(4 * j + v) % NN][0] += g * b[v];
            }
          }
          __syncwarp();  // the staged points are read before the next pass writes them
        }
      };
      auto integrate = [&](int n_it) {
        if constexpr (WIDE) integrate2(n_it);
        else integrate1(n_it);
      };
      // the kind of a buffered INT or FINAL sub-element
      auto item_kind = [&](int act) -> int {
        return act == ACT_FINAL ? HK_FINAL : ((WIDE && KERN == NL_KERNEL_CONST) ? HK_CLOSED : HK_INT);
      };

      // ---- Algorithm 1 for this pair ------------------------------------------------------
      {
        int sp = 0, n_it = 0;
        const uint32_t code0 = 1u << LEVEL_SHIFT;
        int act0;
        {
          R Vl[8][3];  // E_l in the classification frame
#pragma unroll
          for (int a = 0; a < 8; a++)
#pragma unroll
            for (int k = 0; k < 3; k++)
              Vl[a][k] = F32 ? VL[a * 3 + k] : (R)P.evert[((int64_t)l * 8 + a) * 3 + k];
          act0 = classify(Vl, code0, lane == 0);
          if (act0 == ACT_REFINE && lane == 0) push(0, Vl, (R)0, (R)0, (R)0, code0);
        }
        if (act0 == ACT_INT || act0 == ACT_FINAL || act0 == ACT_ZERO) st_items += (lane == 0);
        if (KERN == NL_KERNEL_CONST && act0 == ACT_INT) {
          if constexpr (WIDE) {
            st_closed += (lane == 0);
          } else {
            if (lane == 0) closed_int((R)0, (R)0, (R)0, (R)1);
            act0 = ACT_DROP;
          }
        }
        if (act0 == ACT_INT || act0 == ACT_FINAL) {
          if (lane == 0) put_item(0, (R)0, (R)0, (R)0, 1, item_kind(act0));
          n_it = 1;
        } else if (act0 == ACT_REFINE) {
          sp = 1;  // pushed above
        }
        __syncwarp();
        while (sp > 0) {
          if (n_it > HX_IMAX - 32) {
            integrate(n_it);
            n_it = 0;
          }
          const int np = min(4, sp);
          const int base = sp - np;
          const int par = lane >> 3, c = lane & 7;
          const bool active = par < np;
          R V[8][3], s0 = 0, t0 = 0, u0 = 0;
          uint32_t code = 0;
          if (active) {
            const R* pv = wm.sv + (base + par) * HX_REC;
            const uint32_t pcode = wm.sc[base + par];
            const int plevel = pcode >> LEVEL_SHIFT;
            code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) | (pcode & ((1u << LEVEL_SHIFT) - 1)) |
                   ((uint32_t)c << (3 * (plevel - 1)));
            hchild<R>(pv, c, V);
            const R h = pow2m(R(0), plevel);  // side of the child's sub-cube
            s0 = pv[24] + ((c & 1) ? h : (R)0);
            t0 = pv[25] + ((c & 2) ? h : (R)0);
            u0 = pv[26] + ((c & 4) ? h : (R)0);
          }
          __syncwarp();  // parents are read before children overwrite their slots
          int act = active ? classify(V, code, true) : ACT_DROP;
          const int level = code >> LEVEL_SHIFT;
          if (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO) st_items++;
          if (KERN == NL_KERNEL_CONST && act == ACT_INT) {
            if constexpr (WIDE) {
              st_closed++;
            } else {
              closed_int(s0, t0, u0, pow2m(R(0), level - 1));
              act = ACT_DROP;
            }
          }
          const unsigned m_it = __ballot_sync(FULL, act == ACT_INT || act == ACT_FINAL);
          const unsigned m_ref = __ballot_sync(FULL, act == ACT_REFINE);
          const unsigned below = (1u << lane) - 1u;
          if (act == ACT_INT || act == ACT_FINAL)
            put_item(n_it + __popc(m_it & below), s0, t0, u0, level, item_kind(act));
          const int nref = __popc(m_ref);
          const bool overflow = base + nref > P.scap;
          if (overflow) err |= ERR_STACK;
          else if (act == ACT_REFINE) push(base + __popc(m_ref & below), V, s0, t0, u0, code);
          sp = overflow ? base : base + nref;
          n_it += __popc(m_it);
          __syncwarp();  // records and items of this LIFO step are visible to every lane
        }
        if (n_it > 0) integrate(n_it);
      }

      // ---- end of pair ---------------------------------------------------------------------
      R* bp = reinterpret_cast<R*>(P.blk) + (p - P.p_begin) * NBLK;
      if (!__any_sync(FULL, contrib)) {
        for (int e = lane; e < NBLK; e += 32) bp[e] = (R)0;
        __syncwarp();
        continue;
      }
      if constexpr (WIDE) {
        // lane q writes row q of the H table; lane d then holds column d (+ its closed sum)
        R usum = U[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) usum += __shfl_xor_sync(FULL, usum, o);
        if (lane < HX_NQ) {
          R* row = wm.red + lane * HX_WP;
#pragma unroll
          for (int d = 0; d < NN; d++) row[d] = H[d][0];
          row[HX_NQ] = (R)0;
        }
        __syncwarp();
        if (lane < NN) {
          R col[HX_WP];
#pragma unroll
          for (int q = 0; q < HX_NQ; q++) col[q] = wm.red[q * HX_WP + lane] + U[0];
          col[HX_NQ] = (R)0;
#pragma unroll 1
          for (int a = 0; a < NN; a++) {
            const R* wr = wm.wpm + a * HX_WP;
            R s = 0;
#pragma unroll
            for (int j = 0; j < 7; j++) {
              R w4[4];
              ld4(wr + 4 * j, w4);
#pragma unroll
              for (int v = 0; v < 4; v++) s += w4[v] * col[4 * j + v];
            }
            bp[a * NN + lane] = (R)(-2) * s;
          }
        }
        if (lane < HX_NQ) {
          R g = usum;
#pragma unroll
          for (int d = 0; d < NN; d++) g += H[d][0];
          two_sum_add(gsh, gsl, g);
        }
      } else {
        if (__any_sync(FULL, has_u)) {
#pragma unroll
          for (int d = 0; d < NN; d++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) U[d] += __shfl_xor_sync(FULL, U[d], o);
        }
#pragma unroll
        for (int d = 0; d < NN; d++)
#pragma unroll
          for (int i = 0; i < NYL; i++)
            if (ybase + i < HX_NQ) wm.red[(d * HX_NQ + ybase + i) * HX_RS + xl] = H[d][i];
        __syncwarp();
        for (int j = lane; j < NN * HX_NQ; j += 32) {
          R s = 0;
#pragma unroll
          for (int t = 0; t < XPI; t++) s += wm.red[j * HX_RS + t];
          wm.hs[j] = s + U[j / HX_NQ];
        }
        __syncwarp();
        for (int e = lane; e < NBLK; e += 32) {
          const int a = e / NN, d = e % NN;
          R s = 0;
          for (int q = 0; q < HX_NQ; q++) s += wm.wpm[a * HX_NQ + q] * wm.hs[d * HX_NQ + q];
          bp[e] = (R)(-2) * s;
        }
        if (lane < HX_NQ) {
          R g = 0;
#pragma unroll
          for (int d = 0; d < NN; d++) g += wm.hs[d * HX_NQ + lane];
          two_sum_add(gsh, gsl, g);
        }
      }
      __syncwarp();  // the scratch and E_l's vertices are read before the next pair writes them
    }
    flush_stats();
  }
  if (cur_m >= 0) flush_self();
}

template <typename R, int KERN, int NN>
nl_status launch_quad_h(const QParams& P, cudaStream_t s) {
  int dev = 0, nsm = 0;
  NL_CUDA(cudaGetDevice(&dev));
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t per_warp = HMem<R, NN>::bytes(P.scap);
  int warps = HX_WARPS;
  while (warps > 1 && hx_table_bytes<R, NN>() + warps * per_warp > (size_t)200 * 1024) warps >>= 1;
  const size_t smem = hx_table_bytes<R, NN>() + warps * per_warp;
  if (smem > (size_t)220 * 1024)
    return fail(NL_EINTERNAL, "hexahedral assembly kernel needs %zu bytes of shared memory", smem);
  auto kern = k_quad_h<R, KERN, NN>;
  NL_TRY(allow_smem(kern, smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "hexahedral assembly kernel does not fit on an SM (smem %zu)", smem);
  kern<<<NL_CNT(nsm * per_sm), warps * 32, smem, s>>>(P);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

template <typename R, int KERN, int NN>
nl_status run_assembly_h(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s,
                         unsigned long long* scratch, int* err, PhaseTimer& T) {
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
  if (g_block_budget) budget = std::min(budget, g_block_budget);
  constexpr int NBLK = HxLay<NN>::NBLK;
  int64_t batch = std::max<int64_t>(1 << 20, (int64_t)(budget / (sizeof(R) * NBLK)));
  batch = std::min<int64_t>(batch, p->n_pairs);
  DevBuf<R> blk;
  DevBuf<double> selfblk;
  NL_TRY(blk.alloc((size_t)batch * NBLK, s));
  NL_TRY(selfblk.alloc((size_t)m->n_elem * NBLK, s));
  NL_CUDA(cudaMemsetAsync(selfblk.p, 0, sizeof(double) * m->n_elem * NBLK, s));
  std::vector<int64_t> h_off(m->n_elem + 1);
  NL_CUDA(cudaMemcpyAsync(h_off.data(), p->pair_off, sizeof(int64_t) * (m->n_elem + 1),
                          cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  P.blk = blk.p;
  P.selfblk = selfblk.p;
  for (int64_t b0 = 0; b0 < p->n_pairs; b0 += batch) {
    const int64_t b1 = std::min(p->n_pairs, b0 + batch);
    P.p_begin = b0;
    P.p_end = b1;
    NL_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s));  // work counter
    NL_TRY(T.mark(0, s));
    NL_TRY((launch_quad_h<R, KERN, NN>(P, s)));
    NL_TRY(T.mark(0, s));
    NL_TRY(T.mark(1, s));
    NL_TRY((launch_scatter<3, R, NN>(m, p, b0, b1, blk.p, nullptr, 0, values, err, s, h_off.data())));
    NL_TRY(T.mark(1, s));
  }
  NL_TRY(T.mark(1, s));
  NL_TRY((launch_scatter<3, R, NN>(m, p, 0, 0, blk.p, selfblk.p, 1, values, err, s, h_off.data())));
  NL_TRY(T.mark(1, s));
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}

}  // namespace

nl_status assemble_values_hex(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st) {
  if (m->dim != 3 || m->cell != 2) return fail(NL_EINVAL, "nl_assemble: not a mesh of hexahedra");
  QParams P;
  NL_TRY(fill_qparams("nl_assemble", m, p, kp, qp, prec, &P));
  // the kernel reads the 3-point Gauss-Legendre rule from the rule slots: B[i][0] = g_i, W[i]
  const GL3& g = gl3();
  for (int i = 0; i < 3; i++) {
    for (int a = 0; a < 4; a++) P.B[i][a] = a == 0 ? g.g[i] : 0.0;
    P.W[i] = g.w[i];
  }
  cudaStream_t s = m->stream;
  DevBuf<unsigned long long> scratch;
  DevBuf<int> err;
  NL_TRY(scratch.alloc(8, s));
  NL_TRY(err.alloc(1, s));
  NL_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(unsigned long long) * 8, s));
  NL_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  NL_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (p->nnz ? p->nnz : 1), s));
  P.counter = scratch.p;
  P.stats = scratch.p + 1;
  P.err = err.p;
  cudaEvent_t e0, e1;
  NL_CUDA(cudaEventCreate(&e0));
  NL_CUDA(cudaEventCreate(&e1));
  NL_CUDA(cudaEventRecord(e0, s));
  nl_status rc = NL_OK;
  const bool f32 = prec != NL_PREC_FP64;
  const bool gauss = kp->kernel == NL_KERNEL_TRUNC_GAUSS;
  PhaseTimer T;
  if (p->n_pairs > 0) {
    if (m->nb == 27) {
      if (f32) rc = gauss ? run_assembly_h<float, 1, 27>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly_h<float, 0, 27>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly_h<double, 1, 27>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly_h<double, 0, 27>(m, p, P, values, s, scratch.p, err.p, T);
    } else if (m->nb == 20) {
      if (f32) rc = gauss ? run_assembly_h<float, 1, 20>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly_h<float, 0, 20>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly_h<double, 1, 20>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly_h<double, 0, 20>(m, p, P, values, s, scratch.p, err.p, T);
    } else {
      if (f32) rc = gauss ? run_assembly_h<float, 1, 8>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly_h<float, 0, 8>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly_h<double, 1, 8>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly_h<double, 0, 8>(m, p, P, values, s, scratch.p, err.p, T);
    }
  }
  cudaEventRecord(e1, s);
  unsigned long long hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int herr = 0;
  cudaMemcpyAsync(hs, scratch.p, sizeof hs, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NL_OK) return rc;
  if (ce != cudaSuccess) return cuda_fail(ce, "nl_assemble");
  if (herr) {
    return fail(NL_EINTERNAL, "nl_assemble: device check failed (code %d: %s)", herr,
                (herr & ERR_STACK) ? "refinement stack capacity exceeded" : "CSR entry missing");
  }
  if (st) {
    st->n_pairs = p->n_pairs;
    st->n_items = (int64_t)hs[1];
    st->n_point_pairs = (int64_t)hs[1] * HX_NQ * HX_NQ;
    st->n_exact_checks = (int64_t)hs[3];
    st->ms_assemble = ms;
    st->n_eval_point_pairs = (int64_t)hs[4];
    st->n_closed_items = (int64_t)hs[5];
    st->n_band_point_pairs = P.count_band ? (int64_t)hs[6] : -1;
    st->precision_run = f32 ? NL_PREC_FP32 : NL_PREC_FP64;
    st->n_quad_launches = T.launches(0);
    st->ms_quad = T.ms(0);
    st->ms_scatter = T.ms(1);
  }
  return NL_OK;
}

}  // namespace nlx
