// nl_quad_quad.cu -- nl_assemble on meshes of quadrilaterals (Sec. 6: the QUAD meshes, Q1
// bilinear and Q2 biquadratic Lagrange elements, the Gauss-Legendre 3x3 product rule for the
// inner and the outer integral).
//
// What is computed (Sec. 5, Corollary 1, eqs. J21Nr and J22Nr): for every element pair
// (m, l) of J, with the 3x3 rule on E_m (points y = F_m(g), weights w_y |det DF_m|, rows = the
// nodes of m) and on the sub-elements E' of E_l that Algorithm 1 selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_d] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_d(x).
// An element is the bilinear image F of the unit square; a sub-element is the image of a
// sub-square [s0, s0+len] x [t0, t0+len] of l's square, its outer points x = F_l(s0 + len g_i,
// t0 + len g_j) with weights w_i w_j len^2 |det DF_l| and the basis of l at those reference
// points.  Algorithm 1 splits a square into its four half-size sub-squares and decides on the
// box of the sub-element's physical vertices (the parent's vertices, the edge midpoints
// (a+b)*0.5, the centre as the midpoint of the midpoints of the edges (0,1) and (2,3)).
//
// How (k_quad_q): the structure of the triangle kernels -- a persistent grid, chunks of
// consecutive m-major pairs per warp, Algorithm 1 as a warp LIFO (8 parents x 4 children per
// round), decisions in FP64 (FP64 path) or by the FP32 screen with an FP64 re-decision inside
// the margin (FP32 path), buffered sub-elements integrated by the whole warp.  Q1: each lane
// owns one outer point per pass and m's 9 inner points (36 sums H_d(y) = sum_x w_x C eta mu
// phi^l_d(x)); Q2 and the 8-node serendipity element: the two half-warps share the outer
// points and take inner points 0-4 and 5-8 (45 / 40 sums per lane).  The end of a pair sums H over the lanes through shared memory,
// writes the cross block -2 sum_y w_y |det DF_m| phi^m_a(y) H_d(y) and keeps g(y) = sum_d
// H_d(y) (the basis sums to one) for m's self block.  With the constant kernel an INT
// sub-element (mu = 1 at every point pair) adds sum_x w_x C phi^l_d(x), which does not depend
// on y, to every inner point without evaluating point pairs; in Q1 so does a FINAL one whose
// ball clears delta - eps or delta + eps at each inner point (mu exactly 1 or 0 there).
#include <cuda_runtime.h>

#include "nl_quad_kernel.cuh"

namespace nlx {
namespace {

constexpr int QQ_NQ = 9;       // Gauss-Legendre 3x3 points
constexpr int QQ_IMAX = 64;    // buffered sub-elements
constexpr int QQ_RS = 33;      // row stride of the reduction scratch
constexpr int QQ_WARPS = 4;

// ORD 1: Q1, 2: Q2, 3: the 8-node serendipity element
template <int ORD>
struct QGeo {
  static constexpr int NN = ORD == 2 ? 9 : (ORD == 3 ? 8 : 4);  // nodes per element
  static constexpr int NYL = ORD == 1 ? 9 : 5;                  // inner points per lane
  static constexpr int XPI = ORD == 1 ? 32 : 16;                // outer points per warp pass
  static constexpr int NH = NN * QQ_NQ;             // H_d(y) per pair
  static constexpr int NBLK = NN * NN;
};

// Block tables: the 3x3 rule (s, t, weight) and the basis at its points, in FP64 and R.
template <typename R>
__host__ __device__ constexpr size_t qq_table_bytes() {
  return (sizeof(double) * (27 + 81) + sizeof(R) * (27 + 81) + 15) & ~size_t(15);
}

// Per-warp shared memory: the LIFO (4 vertices, the sub-square's corner, path codes), the
// item buffer (corner, side, kind), m's weighted basis table, the reduction scratch.
template <typename R, int ORD>
struct QMem {
  R* sv;         // [scap][10]: 4 vertices (x, y), then s0, t0
  uint32_t* sc;  // [scap]
  R* it;         // [IMAX][4]: s0, t0, len, kind (1 = FINAL)
  R* wpm;        // [NN][9]: w_y |det DF_m(y)| phi^m_a(y)
  double* wd;    // [9]: w_y |det DF_m(y)| (FP64, self blocks)
  R* red;        // [NH][RS]
  R* hs;         // [NH + 3]
  double* sd;    // [9 + 3]
  static __host__ __device__ size_t bytes(int scap) {
    using G = QGeo<ORD>;
    size_t b = sizeof(R) * 10 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * ((size_t)QQ_IMAX * 4 + G::NN * 9);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * 12;
    b += sizeof(R) * ((size_t)G::NH * QQ_RS + G::NH + 3);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * 12;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    using G = QGeo<ORD>;
    sv = reinterpret_cast<R*>(base);
    sc = reinterpret_cast<uint32_t*>(sv + 10 * (size_t)scap);
    size_t off = sizeof(R) * 10 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    off = (off + 15) & ~size_t(15);
    it = reinterpret_cast<R*>(base + off);
    wpm = it + (size_t)QQ_IMAX * 4;
    off += sizeof(R) * ((size_t)QQ_IMAX * 4 + G::NN * 9);
    off = (off + 15) & ~size_t(15);
    wd = reinterpret_cast<double*>(base + off);
    off += sizeof(double) * 12;
    red = reinterpret_cast<R*>(base + off);
    hs = red + (size_t)G::NH * QQ_RS;
    off += sizeof(R) * ((size_t)G::NH * QQ_RS + G::NH + 3);
    off = (off + 15) & ~size_t(15);
    sd = reinterpret_cast<double*>(base + off);
  }
};

// x = F(s, t) of the quadrilateral V (4 vertices) and |det DF(s, t)|
template <typename R>
__device__ __forceinline__ void qmap(const R (&V)[4][2], R s, R t, R& x0, R& x1, R& det) {
  const R n0 = ((R)1 - s) * ((R)1 - t), n1 = s * ((R)1 - t), n2 = s * t, n3 = ((R)1 - s) * t;
  x0 = n0 * V[0][0] + n1 * V[1][0] + n2 * V[2][0] + n3 * V[3][0];
  x1 = n0 * V[0][1] + n1 * V[1][1] + n2 * V[2][1] + n3 * V[3][1];
  const R xs0 = ((R)1 - t) * (V[1][0] - V[0][0]) + t * (V[2][0] - V[3][0]);
  const R xs1 = ((R)1 - t) * (V[1][1] - V[0][1]) + t * (V[2][1] - V[3][1]);
  const R xt0 = ((R)1 - s) * (V[3][0] - V[0][0]) + s * (V[2][0] - V[1][0]);
  const R xt1 = ((R)1 - s) * (V[3][1] - V[0][1]) + s * (V[2][1] - V[1][1]);
  const R d = xs0 * xt1 - xs1 * xt0;
  det = d < (R)0 ? -d : d;
}

// Child c (0..3: lower-left, lower-right, upper-right, upper-left sub-square) of the
// quadrilateral P by midpoints.
template <typename R>
__device__ __forceinline__ void qchild(const R (&P)[4][2], int c, R (&V)[4][2]) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const R m01 = midp(P[0][k], P[1][k]), m12 = midp(P[1][k], P[2][k]);
    const R m23 = midp(P[2][k], P[3][k]), m30 = midp(P[3][k], P[0][k]);
    const R ce = midp(m01, m23);
    V[0][k] = c == 0 ? P[0][k] : (c == 1 ? m01 : (c == 2 ? ce : m30));
    V[1][k] = c == 0 ? m01 : (c == 1 ? P[1][k] : (c == 2 ? m12 : ce));
    V[2][k] = c == 0 ? ce : (c == 1 ? m12 : (c == 2 ? P[2][k] : m23));
    V[3][k] = c == 0 ? m30 : (c == 1 ? ce : (c == 2 ? m23 : P[3][k]));
  }
}

// Box distances of Sec. 5.1 (eqs. maxdist, mindist; with l2 the Euclidean variant) between the
// box of the 4 vertices V and the box (lo2, hi2), in FP64 in the order of a plain evaluation.
__device__ void qexact_dists(const double (&V)[4][2], const double* lo2, const double* hi2,
                             double& amax, double& amin, bool l2) {
  double s = 0.0, mn = 0.0, e = 0.0;
#pragma unroll
  for (int k = 0; k < 2; k++) {
    double lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a < 4; a++) {
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

// FP32 screen of the same distances (amax squared, amin, the Euclidean amin squared).
__device__ __forceinline__ void qscreen_dists(const float (&V)[4][2], const float* lo2,
                                              const float* hi2, float& amax, float& amin,
                                              float& amin2) {
  float s = 0.f, mn = 0.f, e = 0.f;
#pragma unroll
  for (int k = 0; k < 2; k++) {
    float lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a < 4; a++) {
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

// FP64 decision of Algorithm 1 below L_max for the sub-element with path `code` (2 bits per
// level), its vertices rebuilt from E_l's by the same midpoints: ACT_INT, ACT_REFINE or
// ACT_DROP.
__device__ __noinline__ int qexact_classify(const double* __restrict__ evert_l,
                                            const double* __restrict__ lo_m,
                                            const double* __restrict__ hi_m, uint32_t code,
                                            double dme, double dpe, bool l2) {
  double V[4][2], lo2[2], hi2[2];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int k = 0; k < 2; k++) V[a][k] = evert_l[a * 2 + k];
#pragma unroll
  for (int k = 0; k < 2; k++) {
    lo2[k] = lo_m[k];
    hi2[k] = hi_m[k];
  }
  const int level = code >> LEVEL_SHIFT;
  for (int lv = 2; lv <= level; lv++) {
    const int c = (code >> (2 * (lv - 2))) & 3;
    double P[4][2];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int k = 0; k < 2; k++) P[a][k] = V[a][k];
    qchild<double>(P, c, V);
  }
  double amax, amin;
  qexact_dists(V, lo2, hi2, amax, amin, l2);
  if (amax < dme) return ACT_INT;
  if (amin < dpe) return ACT_REFINE;
  return ACT_DROP;
}

// FP32: 3 CTAs of 4 warps per SM (168 registers; measured on GB300 at the 2D workload's grid,
// Q1 56.5 / Q2 72.8 ms per assembly kernel against 61.7 / 84.8 ms with 2 CTAs and 222 / 242
// registers, and 61.9 / 83.9 ms with 4 CTAs at 128 registers); FP64 1.
template <typename R, int KERN, int ORD>
__global__ void __launch_bounds__(QQ_WARPS * 32, std::is_same<R, float>::value ? 3 : 1)
    k_quad_q(const QParams P) {
  using G = QGeo<ORD>;
  constexpr int NN = G::NN, NYL = G::NYL, XPI = G::XPI, NH = G::NH, NBLK = G::NBLK;
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) char smem_raw[];
  double* tS = reinterpret_cast<double*>(smem_raw);  // [9][3]: s, t, w
  double* tB = tS + 27;                               // [9][9]: phi_a at point q
  R* rS = reinterpret_cast<R*>(tB + 81);
  R* rB = rS + 27;
  for (int t = threadIdx.x; t < QQ_NQ; t += blockDim.x) {
    const int i = t / 3, j = t % 3;
    const double gi = P.B[i][0], gj = P.B[j][0];  // the 3 points and weights (host-filled)
    tS[t * 3] = gi;
    tS[t * 3 + 1] = gj;
    tS[t * 3 + 2] = P.W[i] * P.W[j];
    double phi[9];
    quad_basis<double>(ORD, gi, gj, phi);
    for (int a = 0; a < 9; a++) tB[t * 9 + a] = a < NN ? phi[a] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 27; t += blockDim.x) rS[t] = (R)tS[t];
  for (int t = threadIdx.x; t < 81; t += blockDim.x) rB[t] = (R)tB[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ybase = (ORD != 1 && lane >= 16) ? 5 : 0;  // first inner point of this lane
  const int xl = ORD != 1 ? (lane & 15) : lane;        // outer point slot of this lane
  QMem<R, ORD> wm;
  wm.carve(smem_raw + qq_table_bytes<R>() + (size_t)wid * QMem<R, ORD>::bytes(P.scap), P.scap);

  unsigned st_items = 0, st_exact = 0, st_eval = 0, st_closed = 0, st_band = 0;
  int err = 0;
  int64_t cur_m = -1;
  double v0m[2] = {0.0, 0.0}, mlo[2] = {0.0, 0.0}, mhi[2] = {0.0, 0.0};
  float v0h[2] = {0.f, 0.f}, v0l[2] = {0.f, 0.f}, flo[2] = {0.f, 0.f}, fhi[2] = {0.f, 0.f};
  R y[NYL][2];   // this lane's inner points of m, relative to m's first vertex
  R gsh = 0, gsl = 0;  // lane q < 9: sum of g(y_q) over the current m-run

  auto flush_self = [&]() {
    if (lane < QQ_NQ) wm.sd[lane] = (double)gsh + (double)gsl;
    gsh = gsl = 0;
    __syncwarp();
    for (int e = lane; e < NBLK; e += 32) {
      const int a = e / NN, b = e % NN;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < QQ_NQ; q++) s += wm.wd[q] * tB[q * 9 + a] * tB[q * 9 + b] * wm.sd[q];
      atomicAdd(&P.selfblk[cur_m * NBLK + e], 2.0 * s);
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
      // the last m with pair_off[m] <= g0, every lane probing one position per round
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
        double Vm[4][2];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) Vm[a][k] = P.evert[(m * 4 + a) * 2 + k];
#pragma unroll
        for (int k = 0; k < 2; k++) {
          v0m[k] = Vm[0][k];
          mlo[k] = P.blo[m * 2 + k];
          mhi[k] = P.bhi[m * 2 + k];
        }
        double Vmr[4][2];  // relative to the first vertex
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) Vmr[a][k] = Vm[a][k] - v0m[k];
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          const int q = min(ybase + i, QQ_NQ - 1);
          double x0, x1, det;
          qmap<double>(Vmr, tS[q * 3], tS[q * 3 + 1], x0, x1, det);
          y[i][0] = (R)x0;
          y[i][1] = (R)x1;
        }
        // m's weights w_y |det DF_m| and weighted basis (one lane per inner point)
        if (lane < QQ_NQ) {
          double x0, x1, det;
          qmap<double>(Vmr, tS[lane * 3], tS[lane * 3 + 1], x0, x1, det);
          const double wy = tS[lane * 3 + 2] * det;
          wm.wd[lane] = wy;
#pragma unroll
          for (int a = 0; a < NN; a++) wm.wpm[a * 9 + lane] = (R)(wy * tB[lane * 9 + a]);
        }
        if constexpr (F32) {
          const float* ef = P.ef + m * NL_EF_STRIDE(2);
#pragma unroll
          for (int k = 0; k < 2; k++) {
            v0h[k] = ef[NL_EF_V0HI(2) + k];
            v0l[k] = ef[NL_EF_V0LO(2) + k];
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int a = 1; a < 4; a++) {
              const float v = ef[(a - 1) * 2 + k];
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
      // E_l: R = float in the local FP32 frame, R = double in global FP64 coordinates; VL in
      // the frame of y in both
      R Vl[4][2], VL[4][2], wl;
      if constexpr (F32) {
        const float* ef = P.ef + (int64_t)l * NL_EF_STRIDE(2);
        float o[2];
#pragma unroll
        for (int k = 0; k < 2; k++) o[k] = (ef[NL_EF_V0HI(2) + k] - v0h[k]) + (ef[NL_EF_V0LO(2) + k] - v0l[k]);
#pragma unroll
        for (int k = 0; k < 2; k++) {
          Vl[0][k] = o[k];
#pragma unroll
          for (int a = 1; a < 4; a++) Vl[a][k] = o[k] + ef[(a - 1) * 2 + k];
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) VL[a][k] = Vl[a][k];
        wl = P.fC;
      } else {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) {
            Vl[a][k] = P.evert[((int64_t)l * 4 + a) * 2 + k];
            VL[a][k] = Vl[a][k] - v0m[k];
          }
        wl = P.C;
      }
      R H[NN][NYL];
#pragma unroll
      for (int d = 0; d < NN; d++)
#pragma unroll
        for (int i = 0; i < NYL; i++) H[d][i] = 0;
      R U[NN];  // the closed forms' sums that every inner point receives (Q2)
#pragma unroll
      for (int d = 0; d < NN; d++) U[d] = 0;
      bool contrib = false;
      bool has_u = false;

      // Algorithm 1 decision (as in the triangle kernels)
      auto classify = [&](const R (&V)[4][2], uint32_t code, bool count_exact) -> int {
        const int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        const bool last = level == P.L_max;
        const bool l2 = P.mindist_l2 != 0;
        if constexpr (F32) {
          float fam, fan, fe2;
          qscreen_dists(V, flo, fhi, fam, fan, fe2);
          const bool c_int = fam < P.fint2;
          const bool c_notint = fam > P.fnotint2;
          const bool c_ref = l2 ? fe2 < P.fref2 : fan < P.fdpe - P.margin;
          const bool c_out = l2 ? fe2 > P.fout2 : fan > P.fdpe + P.margin;
          if (last) return c_int ? ACT_INT : (c_out ? ACT_ZERO : ACT_FINAL);
          if (c_int) return ACT_INT;
          if (c_notint && c_ref) return ACT_REFINE;
          if (c_notint && c_out) return ACT_DROP;
          st_exact += count_exact ? 1 : 0;
          return qexact_classify(P.evert + (int64_t)l * 8, P.blo + cur_m * 2, P.bhi + cur_m * 2,
                                 code, P.dme, P.dpe, l2);
        } else {
          double amax, amin;
          qexact_dists(V, mlo, mhi, amax, amin, l2);
          if (last) return amax < P.dme ? ACT_INT : (amin > P.dpe ? ACT_ZERO : ACT_FINAL);
          if (amax < P.dme) return ACT_INT;
          if (amin < P.dpe) return ACT_REFINE;
          return ACT_DROP;
        }
      };
      // sum_x w_x C phi^l_d(x) over the sub-square (s0, t0, len) of l's square
      auto outer_sum = [&](R s0, R t0, R len, R (&S)[NN]) {
#pragma unroll
        for (int d = 0; d < NN; d++) S[d] = 0;
#pragma unroll 1
        for (int q = 0; q < QQ_NQ; q++) {  // not unrolled: rare, keeps the code small
          const R s = s0 + len * rS[q * 3], t = t0 + len * rS[q * 3 + 1];
          R x0, x1, det;
          qmap<R>(VL, s, t, x0, x1, det);
          R phi[9];
          quad_basis<R>(ORD, s, t, phi);
          const R w = rS[q * 3 + 2] * det;
#pragma unroll
          for (int d = 0; d < NN; d++) S[d] += w * phi[d];
        }
        const R wv = wl * len * len;
#pragma unroll
        for (int d = 0; d < NN; d++) S[d] *= wv;
      };
      // Closed forms (constant kernel; the lane that classified the sub-element adds them)
      auto closed_int = [&](R s0, R t0, R len) {
        R S[NN];
        outer_sum(s0, t0, len, S);
#pragma unroll
        for (int d = 0; d < NN; d++) U[d] += S[d];
        has_u = true;
        st_closed++;
        contrib = true;
      };
      // Q1: a FINAL sub-element whose ball (the vertices' mean c, radius max |v - c|) clears
      // delta - eps - margin or delta + eps + margin at every inner point
      auto closed_final = [&](const R (&V)[4][2], R s0, R t0, R len) -> bool {
        if (ORD != 1) return false;
        R c[2], r2 = 0;
#pragma unroll
        for (int k = 0; k < 2; k++)
          c[k] = (V[0][k] + V[1][k] + V[2][k] + V[3][k]) * (R)0.25 - (F32 ? (R)0 : (R)v0m[k]);
#pragma unroll
        for (int a = 0; a < 4; a++) {
          const R d0 = V[a][0] - (F32 ? (R)0 : (R)v0m[0]) - c[0];
          const R d1 = V[a][1] - (F32 ? (R)0 : (R)v0m[1]) - c[1];
          const R d2 = d0 * d0 + d1 * d1;
          r2 = d2 > r2 ? d2 : r2;
        }
        const R rad = sqrt(r2);
        const R lo = (R)P.fdme - rad - (R)P.margin, hi = (R)P.fdpe + rad + (R)P.margin;
        const R lo2 = lo > 0 ? lo * lo : (R)-1, hi2 = hi * hi;
        unsigned in_mask = 0;
        bool decided = true;
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          const R d0 = c[0] - y[i][0], d1 = c[1] - y[i][1];
          const R d2 = d0 * d0 + d1 * d1;
          const bool in = d2 < lo2, out = d2 > hi2;
          in_mask |= in ? (1u << i) : 0u;
          decided = decided && (in || out);
        }
        if (!decided) return false;
        R S[NN];
        outer_sum(s0, t0, len, S);
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          const R wi = (in_mask >> i) & 1u ? (R)1 : (R)0;
#pragma unroll
          for (int d = 0; d < NN; d++) H[d][i] += wi * S[d];
        }
        st_closed++;
        contrib = true;
        return true;
      };
      auto put_item = [&](int slot, R s0, R t0, int level, int fin) {
        R* r = wm.it + slot * 4;
        r[0] = s0;
        r[1] = t0;
        r[2] = pow2m(R(0), level - 1);  // the sub-square's side, a power of two
        r[3] = fin ? (R)1 : (R)0;
      };
      auto push = [&](int slot, const R (&V)[4][2], R s0, R t0, uint32_t code) {
        R* r = wm.sv + slot * 10;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) r[a * 2 + k] = V[a][k];
        r[8] = s0;
        r[9] = t0;
        wm.sc[slot] = code;
      };
      // the buffered items (warp-collective): one outer point per lane (Q1) or per half-warp
      // lane (Q2) and pass
      auto integrate = [&](int n_it) {
        const int n_x = n_it * QQ_NQ;
        st_eval += (unsigned)(n_x * QQ_NQ);
        contrib = true;
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        for (int base = 0; base < n_x; base += XPI) {
          const int o = base + xl;
          const bool valid = o < n_x;
          const int itx = valid ? o / QQ_NQ : 0;
          const int q = valid ? o - itx * QQ_NQ : 0;
          const R* r = wm.it + itx * 4;
          const R len = r[2];
          const R s = r[0] + len * rS[q * 3], t = r[1] + len * rS[q * 3 + 1];
          const bool fin = r[3] != (R)0;
          R x0, x1, det;
          qmap<R>(VL, s, t, x0, x1, det);
          const R wx = valid ? rS[q * 3 + 2] * (wl * len * len) * det : (R)0;
          R phi[9];
          quad_basis<R>(ORD, s, t, phi);
          R bw[NN];
#pragma unroll
          for (int d = 0; d < NN; d++) bw[d] = wx * phi[d];
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            const bool yv = ybase + i < QQ_NQ;
            const R d0 = x0 - y[i][0], d1 = x1 - y[i][1];
            const R r2 = d0 * d0 + d1 * d1;
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
            for (int d = 0; d < NN; d++) H[d][i] += g * bw[d];
          }
        }
      };

      // ---- Algorithm 1 for this pair ------------------------------------------------------
      {
        int sp = 0, n_it = 0;
        const uint32_t code0 = 1u << LEVEL_SHIFT;
        int act0 = classify(Vl, code0, lane == 0);
        if (act0 == ACT_INT || act0 == ACT_FINAL || act0 == ACT_ZERO) st_items += (lane == 0);
        if (KERN == NL_KERNEL_CONST && act0 == ACT_INT) {
          if (lane == 0) closed_int((R)0, (R)0, (R)1);
          act0 = ACT_DROP;
        }
        if (act0 == ACT_INT || act0 == ACT_FINAL) {
          if (lane == 0) put_item(0, (R)0, (R)0, 1, act0 == ACT_FINAL);
          n_it = 1;
        } else if (act0 == ACT_REFINE) {
          if (lane == 0) push(0, Vl, (R)0, (R)0, code0);
          sp = 1;
        }
        __syncwarp();
        while (sp > 0) {
          if (n_it > QQ_IMAX - 32) {
            integrate(n_it);
            n_it = 0;
          }
          const int np = min(8, sp);
          const int base = sp - np;
          const int par = lane >> 2, c = lane & 3;
          const bool active = par < np;
          R V[4][2], s0 = 0, t0 = 0;
          uint32_t code = 0;
          if (active) {
            const R* pv = wm.sv + (base + par) * 10;
            const uint32_t pcode = wm.sc[base + par];
            const int plevel = pcode >> LEVEL_SHIFT;
            code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) | (pcode & ((1u << LEVEL_SHIFT) - 1)) |
                   ((uint32_t)c << (2 * (plevel - 1)));
            R Pv[4][2];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
              for (int k = 0; k < 2; k++) Pv[a][k] = pv[a * 2 + k];
            qchild<R>(Pv, c, V);
            const R h = pow2m(R(0), plevel);  // side of the child's sub-square
            s0 = pv[8] + ((c == 1 || c == 2) ? h : (R)0);
            t0 = pv[9] + (c >= 2 ? h : (R)0);
          }
          __syncwarp();  // parents are read before children overwrite their slots
          int act = active ? classify(V, code, true) : ACT_DROP;
          const int level = code >> LEVEL_SHIFT;
          if (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO) st_items++;
          if (KERN == NL_KERNEL_CONST) {
            const R len = pow2m(R(0), level - 1);
            if (act == ACT_INT) {
              closed_int(s0, t0, len);
              act = ACT_DROP;
            } else if (act == ACT_FINAL && closed_final(V, s0, t0, len)) {
              act = ACT_DROP;
            }
          }
          const unsigned m_it = __ballot_sync(FULL, act == ACT_INT || act == ACT_FINAL);
          const unsigned m_ref = __ballot_sync(FULL, act == ACT_REFINE);
          const unsigned below = (1u << lane) - 1u;
          if (act == ACT_INT || act == ACT_FINAL)
            put_item(n_it + __popc(m_it & below), s0, t0, level, act == ACT_FINAL);
          const int nref = __popc(m_ref);
          const bool overflow = base + nref > P.scap;
          if (overflow) err |= ERR_STACK;
          else if (act == ACT_REFINE) push(base + __popc(m_ref & below), V, s0, t0, code);
          sp = overflow ? base : base + nref;
          n_it += __popc(m_it);
          __syncwarp();  // records and items of this LIFO step are visible to every lane
        }
        if (n_it > 0) integrate(n_it);
      }

      // ---- end of pair: sums over the lanes, cross block, self sums ---------------------------
      R* bp = reinterpret_cast<R*>(P.blk) + (p - P.p_begin) * NBLK;
      if (!__any_sync(FULL, contrib)) {  // every sub-element dropped or beyond delta + eps
        for (int e = lane; e < NBLK; e += 32) bp[e] = (R)0;
        __syncwarp();
        continue;
      }
      // the closed forms' uniform sums, totalled over the warp
      if (__any_sync(FULL, has_u)) {
#pragma unroll
        for (int d = 0; d < NN; d++)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) U[d] += __shfl_xor_sync(FULL, U[d], o);
      }
      // rows (d, q) of the scratch: Q1 every lane writes column `lane` of all rows; Q2 a
      // half-warp writes columns 0-15 of the rows of its inner points
#pragma unroll
      for (int d = 0; d < NN; d++)
#pragma unroll
        for (int i = 0; i < NYL; i++)
          if (ybase + i < QQ_NQ) wm.red[(d * QQ_NQ + ybase + i) * QQ_RS + xl] = H[d][i];
      __syncwarp();
      for (int j = lane; j < NH; j += 32) {
        R s = 0;
        for (int t = 0; t < XPI; t++) s += wm.red[j * QQ_RS + t];
        wm.hs[j] = s + U[j / QQ_NQ];
      }
      __syncwarp();
      for (int e = lane; e < NBLK; e += 32) {
        const int a = e / NN, d = e % NN;
        R s = 0;
#pragma unroll
        for (int i = 0; i < QQ_NQ; i++) s += wm.wpm[a * 9 + i] * wm.hs[d * QQ_NQ + i];
        bp[e] = (R)(-2) * s;
      }
      if (lane < QQ_NQ) {
        R g = 0;
#pragma unroll
        for (int d = 0; d < NN; d++) g += wm.hs[d * QQ_NQ + lane];
        two_sum_add(gsh, gsl, g);
      }
      __syncwarp();  // the scratch is read before the next pair writes it
    }
    flush_stats();
  }
  if (cur_m >= 0) flush_self();
}

template <typename R, int KERN, int ORD>
nl_status launch_quad_q(const QParams& P, cudaStream_t s) {
  int dev = 0, nsm = 0;
  NL_CUDA(cudaGetDevice(&dev));
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t per_warp = QMem<R, ORD>::bytes(P.scap);
  int warps = QQ_WARPS;
  while (warps > 1 && qq_table_bytes<R>() + warps * per_warp > (size_t)200 * 1024) warps >>= 1;
  const size_t smem = qq_table_bytes<R>() + warps * per_warp;
  if (smem > (size_t)220 * 1024)
    return fail(NL_EINTERNAL, "quadrilateral assembly kernel needs %zu bytes of shared memory", smem);
  auto kern = k_quad_q<R, KERN, ORD>;
  NL_TRY(allow_smem(kern, smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "quadrilateral assembly kernel does not fit on an SM (smem %zu)", smem);
  kern<<<NL_CNT(nsm * per_sm), warps * 32, smem, s>>>(P);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

template <typename R, int KERN, int ORD>
nl_status run_assembly_q(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s,
                         unsigned long long* scratch, int* err, PhaseTimer& T) {
  constexpr int NN = QGeo<ORD>::NN, NBLK = QGeo<ORD>::NBLK;
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
  if (g_block_budget) budget = std::min(budget, g_block_budget);
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
    NL_TRY((launch_quad_q<R, KERN, ORD>(P, s)));
    NL_TRY(T.mark(0, s));
    NL_TRY(T.mark(1, s));
    NL_TRY((launch_scatter<2, R, NN>(m, p, b0, b1, blk.p, nullptr, 0, values, err, s, h_off.data())));
    NL_TRY(T.mark(1, s));
  }
  NL_TRY(T.mark(1, s));
  NL_TRY((launch_scatter<2, R, NN>(m, p, 0, 0, blk.p, selfblk.p, 1, values, err, s, h_off.data())));
  NL_TRY(T.mark(1, s));
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}

template <int ORD>
nl_status run_q(nl_mesh* m, nl_pairs* p, const QParams& P, double* values, cudaStream_t s,
                unsigned long long* scratch, int* err, PhaseTimer& T, bool f32, bool gauss) {
  if (f32) return gauss ? run_assembly_q<float, 1, ORD>(m, p, P, values, s, scratch, err, T)
                        : run_assembly_q<float, 0, ORD>(m, p, P, values, s, scratch, err, T);
  return gauss ? run_assembly_q<double, 1, ORD>(m, p, P, values, s, scratch, err, T)
               : run_assembly_q<double, 0, ORD>(m, p, P, values, s, scratch, err, T);
}

}  // namespace

nl_status assemble_values_quad(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                               const nl_quad_params* qp, nl_precision prec, double* values,
                               nl_assemble_stats* st) {
  if (m->dim != 2 || m->cell != 1) return fail(NL_EINVAL, "nl_assemble: not a mesh of quadrilaterals");
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
    rc = m->order == 2   ? run_q<2>(m, p, P, values, s, scratch.p, err.p, T, f32, gauss)
         : m->order == 3 ? run_q<3>(m, p, P, values, s, scratch.p, err.p, T, f32, gauss)
                         : run_q<1>(m, p, P, values, s, scratch.p, err.p, T, f32, gauss);
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
    st->n_point_pairs = (int64_t)hs[1] * QQ_NQ * QQ_NQ;
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
