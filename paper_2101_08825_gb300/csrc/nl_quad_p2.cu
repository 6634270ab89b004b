// nl_quad_p2.cu -- nl_assemble on meshes of quadratic (P2) Lagrange triangles (Sec. 6, the
// quadratic columns of Tables 1-3).
//
// What is computed is the P1 computation of nl_quad_kernel.cuh with the P2 basis (Sec. 5,
// Corollary 1, eqs. J21Nr and J22Nr): for every element pair (m, l) of J, the inner degree-5
// rule on E_m (points y, rows = the six nodes of m) and the outer rule on the sub-elements E' of
// E_l that Algorithm 1 selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_d] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_d(x),
// phi the P2 basis: lambda_a (2 lambda_a - 1) at the vertices, 4 lambda_a lambda_b at the
// nodes of the edges (0,1), (1,2), (0,2).  Algorithm 1 only looks at the vertices of the
// sub-elements, so it decides exactly as for P1.
//
// How (k_quad_p2): a persistent grid; each warp takes chunks of consecutive pairs (m-major)
// from a global counter.  Per pair the warp runs Algorithm 1 as a LIFO of refined sub-elements
// in shared memory: a round pops up to 8 parents and each lane builds and classifies one of
// their 4 midpoint children, with the decisions of the P1 kernel (FP64 in the FP64 path; in the
// FP32 path the FP32 screen with its proven margin and the FP64 decision inside the margin).
// Sub-elements to integrate are buffered with their vertices relative to the first vertex of
// m; a full buffer is integrated by the whole warp, one outer point x per lane and the 7 inner
// points y of m in registers: per y the lane accumulates H_d(y) = sum_x w_x C eta mu
// phi^l_d(x) for the six nodes d of l (42 sums; mu is 1 on a sub-element whose max-dist is
// below delta - eps; FP32: inner points 0-5 in packed f32x2 pairs).  At the end of the pair the warp
// sums the 42 H_d(y) over its lanes through shared memory, writes the cross block
// -2 |E_m| sum_y w_y phi^m_a(y) H_d(y), and keeps g(y) = sum_d H_d(y) (the basis sums to one)
// summed over the consecutive pairs of m for the self block 2 |E_m| sum_y w_y phi_a phi_b g,
// which is added to a per-element block once per run of m.  k_scatter<2, R, 6> then adds the
// 6 x 6 blocks to the CSR values.
//
// Precision: R = double classifies and evaluates in FP64 (global coordinates for the
// decisions, coordinates relative to the first vertex of m for the point pairs).  R = float
// works in the P1 kernel's local FP32 frame (origin m's first vertex as a float-float pair,
// vertex offsets from the FP32 element records): the decisions are those of a plain FP64
// evaluation, the point pairs, the basis, the sums and the cross blocks are FP32; the inner
// points are formed in FP64 and rounded once.
#include <cuda_runtime.h>

#include "nl_quad_kernel.cuh"

namespace nlx {
namespace {

constexpr int P2_NN = 6;                  // nodes per element
constexpr int P2_NQ = 7;                  // points of the degree-5 triangle rule
constexpr int P2_NH = P2_NN * P2_NQ;      // H_d(y) per pair
constexpr int P2_NBLK = P2_NN * P2_NN;    // entries of a local block
constexpr int P2_IMAX = 64;               // buffered sub-elements
constexpr int P2_RS = 33;                 // row stride of the reduction scratch
constexpr int P2_WARPS = 4;

// P2 basis function a at barycentric coordinates lam
__host__ __device__ inline double p2_phi(const double* lam, int a) {
  if (a < 3) return lam[a] * (2.0 * lam[a] - 1.0);
  if (a == 3) return 4.0 * lam[0] * lam[1];
  if (a == 4) return 4.0 * lam[1] * lam[2];
  return 4.0 * lam[0] * lam[2];
}

// Block tables: tPhi[a][q] = phi_a(y_q) and tW[q] (FP64, for the self blocks); rB[q][v] (the
// rule's barycentric coordinates), rW[q] and rWP[a][q] = w_q phi_a(y_q) in R.
template <typename R>
__host__ __device__ constexpr size_t p2_table_bytes() {
  return (sizeof(double) * (P2_NH + 8) + sizeof(R) * (24 + 8 + 48) + 15) & ~size_t(15);
}

// Per-warp shared memory: the LIFO (vertices and path codes), the item buffer (vertices
// relative to the first vertex of m, weights C |E'|, kinds), the reduction scratch, the
// reduced sums and the self-block scratch.  R = float keeps the LIFO's vertices in the local
// FP32 frame of the screen, R = double in global FP64 coordinates.
template <typename R>
struct P2Mem {
  R* sv;         // [scap][6]
  uint32_t* sc;  // [scap]: level << LEVEL_SHIFT | 2 bits per level of child indices
  R* iv;         // [IMAX][6]
  R* iw;         // [IMAX]
  int* ik;       // [IMAX]: 1 = FINAL (mollifier evaluated), 0 = INT (mu = 1)
  R* red;        // [NH][RS]
  R* hs;         // [48]
  double* sd;    // [8]
  static __host__ __device__ size_t bytes(int scap) {
    size_t b = sizeof(R) * 6 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * (size_t)P2_IMAX * 7 + sizeof(int) * P2_IMAX;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * ((size_t)P2_NH * P2_RS + 48) + sizeof(double) * 8;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    sv = reinterpret_cast<R*>(base);
    sc = reinterpret_cast<uint32_t*>(sv + 6 * (size_t)scap);
    size_t off = sizeof(R) * 6 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    off = (off + 15) & ~size_t(15);
    iv = reinterpret_cast<R*>(base + off);
    iw = iv + (size_t)P2_IMAX * 6;
    ik = reinterpret_cast<int*>(iw + P2_IMAX);
    off += sizeof(R) * (size_t)P2_IMAX * 7 + sizeof(int) * P2_IMAX;
    off = (off + 15) & ~size_t(15);
    red = reinterpret_cast<R*>(base + off);
    hs = red + (size_t)P2_NH * P2_RS;
    sd = reinterpret_cast<double*>(hs + 48);
  }
};

// Launch bounds: FP32 3 CTAs of 4 warps per SM (168 registers; measured on GB300 at the 2D
// workload's size, 145 ms per assembly against 184 ms with 1 or 2 CTAs and 178 registers);
// FP64 1 (about 240 registers: its state spills at 168).
template <typename R, int KERN>
__global__ void __launch_bounds__(P2_WARPS * 32, std::is_same<R, float>::value ? 3 : 1)
    k_quad_p2(const QParams P) {
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) char smem_raw[];
  double* tPhi = reinterpret_cast<double*>(smem_raw);
  double* tW = tPhi + P2_NH;
  R* rB = reinterpret_cast<R*>(tW + 8);
  R* rW = rB + 24;
  R* rWP = rW + 8;
  for (int t = threadIdx.x; t < P2_NH; t += blockDim.x) {
    const int a = t / P2_NQ, q = t % P2_NQ;
    const double phi = p2_phi(P.B[q], a);
    tPhi[t] = phi;
    rWP[t] = (R)(P.W[q] * phi);
  }
  for (int t = threadIdx.x; t < P2_NQ; t += blockDim.x) {
    tW[t] = P.W[t];
    rW[t] = (R)P.W[t];
  }
  for (int t = threadIdx.x; t < 3 * P2_NQ; t += blockDim.x) rB[t] = (R)P.B[t / 3][t % 3];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  P2Mem<R> wm;
  wm.carve(smem_raw + p2_table_bytes<R>() + (size_t)wid * P2Mem<R>::bytes(P.scap), P.scap);

  unsigned st_items = 0, st_exact = 0, st_eval = 0, st_closed = 0, st_band = 0;
  int err = 0;
  int64_t cur_m = -1;
  // the box of m: FP64 global (exact decisions); R = float also in the local FP32 frame whose
  // origin is m's first vertex v0h + v0l (the element record's float-float pair)
  double v0m[2] = {0.0, 0.0}, mlo[2] = {0.0, 0.0}, mhi[2] = {0.0, 0.0}, vol_md = 0.0;
  float v0h[2] = {0.f, 0.f}, v0l[2] = {0.f, 0.f}, flo[2] = {0.f, 0.f}, fhi[2] = {0.f, 0.f};
  R y[P2_NQ][2];  // inner points of m relative to its first vertex
  f2 yq[3][2];    // R = float: inner points 0-5 packed in pairs
  R vol_m = 0;
  R gsh = 0, gsl = 0;  // lane q < 7: sum of g(y_q) over the pairs of the current m-run

  auto flush_self = [&]() {
    if (lane < P2_NQ) wm.sd[lane] = (double)gsh + (double)gsl;
    gsh = gsl = 0;
    __syncwarp();
    for (int e = lane; e < P2_NBLK; e += 32) {
      const int a = e / P2_NN, b = e % P2_NN;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < P2_NQ; q++) s += tW[q] * tPhi[a * P2_NQ + q] * tPhi[b * P2_NQ + q] * wm.sd[q];
      atomicAdd(&P.selfblk[cur_m * P2_NBLK + e], 2.0 * vol_md * s);
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
      // the last m with pair_off[m] <= g0 (pair_off[0] = 0 <= g0 < pair_off[n_elem]), every
      // lane probing one position per round
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
        double Vm[3][2];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) Vm[a][k] = P.evert[(m * 3 + a) * 2 + k];
#pragma unroll
        for (int k = 0; k < 2; k++) {
          v0m[k] = Vm[0][k];
          mlo[k] = P.blo[m * 2 + k];
          mhi[k] = P.bhi[m * 2 + k];
        }
        vol_md = P.vol[m];
        vol_m = (R)vol_md;
#pragma unroll
        for (int q = 0; q < P2_NQ; q++)
#pragma unroll
          for (int k = 0; k < 2; k++) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 3; a++) s += P.B[q][a] * (Vm[a][k] - v0m[k]);
            y[q][k] = (R)s;
          }
        if constexpr (F32) {
          // the screen's frame and box of m, as the P1 kernel forms them: origin v0h + v0l,
          // vertices 0 and the record's FP32 offsets
          const float* ef = P.ef + m * NL_EF_STRIDE(2);
#pragma unroll
          for (int k = 0; k < 2; k++) {
            v0h[k] = ef[NL_EF_V0HI(2) + k];
            v0l[k] = ef[NL_EF_V0LO(2) + k];
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int a = 1; a < 3; a++) {
              const float v = ef[(a - 1) * 2 + k];
              lo = v < lo ? v : lo;
              hi = v > hi ? v : hi;
            }
            flo[k] = lo;
            fhi[k] = hi;
          }
#pragma unroll
          for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < 2; k++) yq[j][k] = f2pack((float)y[2 * j][k], (float)y[2 * j + 1][k]);
        }
      }
      const int32_t l = P.pair_l[p];
      // E_l: R = float in the local FP32 frame (first vertex from the float-float pairs,
      // the others from the record's FP32 offsets), R = double in global FP64 coordinates
      R Vl[3][2], Vl0[2], JI[2][2], wl;
      if constexpr (F32) {
        const float* ef = P.ef + (int64_t)l * NL_EF_STRIDE(2);
#pragma unroll
        for (int k = 0; k < 2; k++) Vl0[k] = (ef[NL_EF_V0HI(2) + k] - v0h[k]) + (ef[NL_EF_V0LO(2) + k] - v0l[k]);
#pragma unroll
        for (int k = 0; k < 2; k++) {
          Vl[0][k] = Vl0[k];
          Vl[1][k] = Vl0[k] + ef[k];
          Vl[2][k] = Vl0[k] + ef[2 + k];
        }
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
          for (int c = 0; c < 2; c++) JI[r][c] = ef[4 + r * 2 + c];
        wl = P.fC * ef[8];
      } else {
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) Vl[a][k] = P.evert[((int64_t)l * 3 + a) * 2 + k];
#pragma unroll
        for (int k = 0; k < 2; k++) Vl0[k] = Vl[0][k] - v0m[k];
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
          for (int c = 0; c < 2; c++) JI[r][c] = P.jinv[((int64_t)l * 2 + r) * 2 + c];
        wl = P.C * P.vol[l];
      }
      R H[P2_NN][P2_NQ];
#pragma unroll
      for (int d = 0; d < P2_NN; d++)
#pragma unroll
        for (int i = 0; i < P2_NQ; i++) H[d][i] = 0;
      f2 Hq[P2_NN][3];  // R = float: the sums of inner points 0-5 in pairs
#pragma unroll
      for (int d = 0; d < P2_NN; d++)
#pragma unroll
        for (int j = 0; j < 3; j++) Hq[d][j] = 0ull;
      // whether anything was summed for this pair on this lane (a closed form) or by the warp
      // (an integration): pairs with no contribution anywhere write a zero block
      bool contrib = false;
      // the largest distance from the centroid of E_l to its vertices, in the frame of y (the
      // radius of a level-L sub-element is this times 2^(1-L): every midpoint child of a
      // triangle is its parent scaled by 1/2)
      R rad_l = 0;
      if (KERN == NL_KERNEL_CONST) {
        R ct[2];
#pragma unroll
        for (int k = 0; k < 2; k++) ct[k] = (Vl[0][k] + Vl[1][k] + Vl[2][k]) * (R)(1.0 / 3.0);
        R r2 = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
          const R d0 = Vl[a][0] - ct[0], d1 = Vl[a][1] - ct[1];
          const R d2 = d0 * d0 + d1 * d1;
          r2 = r2 > d2 ? r2 : d2;
        }
        rad_l = sqrt(r2);
      }

      // Algorithm 1 decision for the sub-element with vertices V and path code `code`.
      // R = double: eqs. maxdist and mindist in FP64 on global coordinates.  R = float: the
      // P1 kernel's FP32 screen in the local frame (thresholds moved by a proven margin), and
      // the FP64 decision on vertices rebuilt from E_l by the same midpoints where the
      // screened distance falls inside the margin; at L_max only INT (mu = 1, surely) and
      // ZERO (mu = 0, surely) are taken from the screen, everything else is evaluated.
      // count_exact: this lane counts an FP64 re-decision (the root is classified by every
      // lane alike and counted once)
      auto classify = [&](const R (&V)[3][2], uint32_t code, bool count_exact) -> int {
        const int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        const bool last = level == P.L_max;
        const bool l2 = P.mindist_l2 != 0;
        if constexpr (F32) {
          float fam, fan, fe2;
          screen_dists<2>(V, flo, fhi, fam, fan, fe2);
          const bool c_int = fam < P.fint2;
          const bool c_notint = fam > P.fnotint2;
          const bool c_ref = l2 ? fe2 < P.fref2 : fan < P.fdpe - P.margin;
          const bool c_out = l2 ? fe2 > P.fout2 : fan > P.fdpe + P.margin;
          if (last) return c_int ? ACT_INT : (c_out ? ACT_ZERO : ACT_FINAL);
          if (c_int) return ACT_INT;
          if (c_notint && c_ref) return ACT_REFINE;
          if (c_notint && c_out) return ACT_DROP;
          st_exact += count_exact ? 1 : 0;
          return exact_classify<2>(P.evert + (int64_t)l * 6, P.blo + cur_m * 2, P.bhi + cur_m * 2,
                                   code, P.dme, P.dpe, l2);
        } else {
          double amax, amin;
          exact_dists<2>(V, mlo, mhi, amax, amin, l2);
          if (last) return amax < P.dme ? ACT_INT : (amin > P.dpe ? ACT_ZERO : ACT_FINAL);
          if (amax < P.dme) return ACT_INT;
          if (amin < P.dpe) return ACT_REFINE;
          return ACT_DROP;
        }
      };
      // Closed forms (constant kernel).  On a sub-element E' whose point pairs all have mu
      // exactly 1 (INT) or, per inner point y, all 1 or all 0 (FINAL, decided by the ball
      // around E''s centroid), the outer sum at y is C sum_x w_x phi^l_d(x) = C |E'| times the
      // mean of phi^l_d over E' (the degree-5 rule is exact for the quadratic phi^l_d), which
      // the three edge midpoints give exactly (their rule is exact for quadratics).  Added to
      // the inner points in `mask` by the lane that classified E'.
      auto add_closed = [&](const R (&V)[3][2], int level, unsigned mask) {
        R mean[P2_NN];
#pragma unroll
        for (int d = 0; d < P2_NN; d++) mean[d] = 0;
#pragma unroll
        for (int e = 0; e < 3; e++) {
          const int a = e, b = e == 2 ? 0 : e + 1;
          R dx[2];
#pragma unroll
          for (int k = 0; k < 2; k++)
            dx[k] = (V[a][k] + V[b][k]) * (R)0.5 - (F32 ? (R)0 : (R)v0m[k]) - Vl0[k];
          const R l1 = JI[0][0] * dx[0] + JI[0][1] * dx[1];
          const R l2 = JI[1][0] * dx[0] + JI[1][1] * dx[1];
          const R l0 = (R)1 - l1 - l2;
          mean[0] += l0 * ((R)2 * l0 - (R)1);
          mean[1] += l1 * ((R)2 * l1 - (R)1);
          mean[2] += l2 * ((R)2 * l2 - (R)1);
          mean[3] += (R)4 * l0 * l1;
          mean[4] += (R)4 * l1 * l2;
          mean[5] += (R)4 * l0 * l2;
        }
        const R wv = wl * pow2m(R(0), 2 * (level - 1)) * (R)(1.0 / 3.0);
        if constexpr (F32) {
#pragma unroll
          for (int j = 0; j < 3; j++) {
            const float w0 = (mask >> (2 * j)) & 1u ? wv : 0.f, w1 = (mask >> (2 * j + 1)) & 1u ? wv : 0.f;
            const f2 W2 = f2pack(w0, w1);
#pragma unroll
            for (int d = 0; d < P2_NN; d++) Hq[d][j] = f2fma(W2, f2dup(mean[d]), Hq[d][j]);
          }
          const float w6 = (mask >> 6) & 1u ? wv : 0.f;
#pragma unroll
          for (int d = 0; d < P2_NN; d++) H[d][6] = fmaf(w6, mean[d], H[d][6]);
        } else {
#pragma unroll
          for (int i = 0; i < P2_NQ; i++) {
            const R wi = (mask >> i) & 1u ? wv : (R)0;
#pragma unroll
            for (int d = 0; d < P2_NN; d++) H[d][i] += wi * mean[d];
          }
        }
        st_closed++;
        contrib = true;
      };
      // FINAL E' at `level`: for each inner point y, mu is exactly 1 at every point pair if
      // |c - y| < delta - eps - rad - margin, exactly 0 if |c - y| > delta + eps + rad + margin
      // (c the centroid, rad the radius of E').  Adds the closed form and returns true when
      // every inner point is decided.
      auto closed_final = [&](const R (&V)[3][2], int level) -> bool {
        R cen[2];
#pragma unroll
        for (int k = 0; k < 2; k++)
          cen[k] = (V[0][k] + V[1][k] + V[2][k]) * (R)(1.0 / 3.0) - (F32 ? (R)0 : (R)v0m[k]);
        const R rad = rad_l * pow2m(R(0), level - 1);
        const R lo = (R)P.fdme - rad - (R)P.margin, hi = (R)P.fdpe + rad + (R)P.margin;
        const R lo2 = lo > 0 ? lo * lo : (R)-1, hi2 = hi * hi;
        unsigned in_mask = 0;
        bool decided = true;
#pragma unroll
        for (int i = 0; i < P2_NQ; i++) {
          const R d0 = cen[0] - y[i][0], d1 = cen[1] - y[i][1];
          const R d2 = d0 * d0 + d1 * d1;
          const bool in = d2 < lo2, out = d2 > hi2;
          in_mask |= in ? (1u << i) : 0u;
          decided = decided && (in || out);
        }
        if (!decided) return false;
        add_closed(V, level, in_mask);
        return true;
      };
      auto put_item = [&](int slot, const R (&V)[3][2], int level, int fin) {
        R* it = wm.iv + slot * 6;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) it[a * 2 + k] = F32 ? V[a][k] : (R)(V[a][k] - v0m[k]);
        wm.iw[slot] = wl * pow2m(R(0), 2 * (level - 1));
        wm.ik[slot] = fin;
      };
      auto push = [&](int slot, const R (&V)[3][2], uint32_t code) {
        R* r = wm.sv + slot * 6;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int k = 0; k < 2; k++) r[a * 2 + k] = V[a][k];
        wm.sc[slot] = code;
      };
      // the buffered items, one outer point per lane (warp-collective)
      auto integrate = [&](int n_it) {
        const int n_x = n_it * P2_NQ;
        st_eval += (unsigned)(n_x * P2_NQ);
        contrib = true;
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        for (int base = 0; base < n_x; base += 32) {
          const int o = base + lane;
          const bool valid = o < n_x;
          const int it = valid ? o / P2_NQ : 0;
          const int q = valid ? o - it * P2_NQ : 0;
          const R* vi = wm.iv + it * 6;
          const R b0 = rB[q * 3], b1 = rB[q * 3 + 1], b2 = rB[q * 3 + 2];
          const R x0 = b0 * vi[0] + b1 * vi[2] + b2 * vi[4];
          const R x1 = b0 * vi[1] + b1 * vi[3] + b2 * vi[5];
          const R wx = valid ? rW[q] * wm.iw[it] : (R)0;
          const bool fin = wm.ik[it] != 0;
          const R dx0 = x0 - Vl0[0], dx1 = x1 - Vl0[1];
          const R l1 = JI[0][0] * dx0 + JI[0][1] * dx1;
          const R l2 = JI[1][0] * dx0 + JI[1][1] * dx1;
          const R l0 = (R)1 - l1 - l2;
          R bw[P2_NN];  // w_x phi^l_d(x)
          bw[0] = wx * l0 * ((R)2 * l0 - (R)1);
          bw[1] = wx * l1 * ((R)2 * l1 - (R)1);
          bw[2] = wx * l2 * ((R)2 * l2 - (R)1);
          bw[3] = (R)4 * wx * l0 * l1;
          bw[4] = (R)4 * wx * l1 * l2;
          bw[5] = (R)4 * wx * l0 * l2;
          if constexpr (F32) {
            // inner points 0-5 in packed pairs (f32x2), point 6 alone
            const f2 X0 = f2dup(x0), X1 = f2dup(x1), ONE = f2dup(1.f);
            f2 BW[P2_NN];
#pragma unroll
            for (int d = 0; d < P2_NN; d++) BW[d] = f2dup(bw[d]);
#pragma unroll
            for (int j = 0; j < 3; j++) {
              f2 dd = f2sub(X0, yq[j][0]);
              f2 r2 = f2mul(dd, dd);
              dd = f2sub(X1, yq[j][1]);
              r2 = f2fma(dd, dd, r2);
              f2 g = fin ? mollifier2(MK, r2) : ONE;
              if (P.count_band) {
                float a, b;
                f2unpack(r2, a, b);
                st_band += (valid && fin && a >= P.fdme2 && a <= P.fdpe2) ? 1 : 0;
                st_band += (valid && fin && b >= P.fdme2 && b <= P.fdpe2) ? 1 : 0;
              }
              if (KERN == NL_KERNEL_TRUNC_GAUSS) g = f2mul(g, eta_gauss2(P.finv_delta2, r2));
#pragma unroll
              for (int d = 0; d < P2_NN; d++) Hq[d][j] = f2fma(g, BW[d], Hq[d][j]);
            }
            const float d0 = x0 - y[6][0], d1 = x1 - y[6][1];
            const float r2 = fmaf(d1, d1, d0 * d0);
            float g = fin ? mollifier_bf(MK, r2) : 1.f;
            if (P.count_band) st_band += (valid && fin && r2 >= P.fdme2 && r2 <= P.fdpe2) ? 1 : 0;
            if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= __expf(-r2 * P.finv_delta2);
#pragma unroll
            for (int d = 0; d < P2_NN; d++) H[d][6] = fmaf(g, bw[d], H[d][6]);
          } else {
#pragma unroll
            for (int i = 0; i < P2_NQ; i++) {
              const R d0 = x0 - y[i][0], d1 = x1 - y[i][1];
              const R r2 = d0 * d0 + d1 * d1;
              R g = 1;
              if (fin) g = mollifier(P, r2);
              if (P.count_band)
                st_band += (valid && fin && r2 >= P.dme * P.dme && r2 <= P.dpe * P.dpe) ? 1 : 0;
              if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= eta_gauss<R>(P, r2);
#pragma unroll
              for (int d = 0; d < P2_NN; d++) H[d][i] += g * bw[d];
            }
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
          if (lane == 0) add_closed(Vl, 1, 0x7fu);
          act0 = ACT_DROP;
        }
        if (act0 == ACT_INT || act0 == ACT_FINAL) {
          if (lane == 0) put_item(0, Vl, 1, act0 == ACT_FINAL);
          n_it = 1;
        } else if (act0 == ACT_REFINE) {
          if (lane == 0) push(0, Vl, code0);
          sp = 1;
        }
        __syncwarp();
        while (sp > 0) {
          if (n_it > P2_IMAX - 32) {
            integrate(n_it);
            n_it = 0;
          }
          const int np = min(8, sp);
          const int base = sp - np;
          const int par = lane >> 2, c = lane & 3;
          const bool active = par < np;
          R V[3][2];
          uint32_t code = 0;
          if (active) {
            const R* pv = wm.sv + (base + par) * 6;
            const uint32_t pcode = wm.sc[base + par];
            const int plevel = pcode >> LEVEL_SHIFT;
            code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) | (pcode & ((1u << LEVEL_SHIFT) - 1)) |
                   ((uint32_t)c << (2 * (plevel - 1)));
#pragma unroll
            for (int v = 0; v < 3; v++) {
              int ia, ib;
              mid_pair<2>(c, v, ia, ib);
#pragma unroll
              for (int k = 0; k < 2; k++) V[v][k] = midp(pv[ia * 2 + k], pv[ib * 2 + k]);
            }
          }
          __syncwarp();  // parents are read before children overwrite their slots
          int act = active ? classify(V, code, true) : ACT_DROP;
          if (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO) st_items++;
          if (KERN == NL_KERNEL_CONST) {
            if (act == ACT_INT) {
              add_closed(V, code >> LEVEL_SHIFT, 0x7fu);
              act = ACT_DROP;
            } else if (act == ACT_FINAL && closed_final(V, code >> LEVEL_SHIFT)) {
              act = ACT_DROP;
            }
          }
          const unsigned m_it = __ballot_sync(FULL, act == ACT_INT || act == ACT_FINAL);
          const unsigned m_ref = __ballot_sync(FULL, act == ACT_REFINE);
          const unsigned below = (1u << lane) - 1u;
          if (act == ACT_INT || act == ACT_FINAL)
            put_item(n_it + __popc(m_it & below), V, code >> LEVEL_SHIFT, act == ACT_FINAL);
          const int nref = __popc(m_ref);
          const bool overflow = base + nref > P.scap;
          if (overflow) err |= ERR_STACK;
          else if (act == ACT_REFINE) push(base + __popc(m_ref & below), V, code);
          sp = overflow ? base : base + nref;
          n_it += __popc(m_it);
          __syncwarp();  // records and items of this LIFO step are visible to every lane
        }
        if (n_it > 0) integrate(n_it);
      }

      // ---- end of pair: sums over the lanes, cross block, self sums ---------------------------
      R* bp = reinterpret_cast<R*>(P.blk) + (p - P.p_begin) * P2_NBLK;
      if (!__any_sync(FULL, contrib)) {  // every sub-element dropped or beyond delta + eps
        for (int e = lane; e < P2_NBLK; e += 32) bp[e] = (R)0;
        __syncwarp();
        continue;
      }
      if constexpr (F32) {
#pragma unroll
        for (int d = 0; d < P2_NN; d++)
#pragma unroll
          for (int j = 0; j < 3; j++) {
            float a, b;
            f2unpack(Hq[d][j], a, b);
            H[d][2 * j] = a;
            H[d][2 * j + 1] = b;
          }
      }
#pragma unroll
      for (int d = 0; d < P2_NN; d++)
#pragma unroll
        for (int i = 0; i < P2_NQ; i++) wm.red[(d * P2_NQ + i) * P2_RS + lane] = H[d][i];
      __syncwarp();
      for (int j = lane; j < P2_NH; j += 32) {
        R s = 0;
        for (int t = 0; t < 32; t++) s += wm.red[j * P2_RS + t];
        wm.hs[j] = s;
      }
      __syncwarp();
      for (int e = lane; e < P2_NBLK; e += 32) {
        const int a = e / P2_NN, d = e % P2_NN;
        R s = 0;
#pragma unroll
        for (int i = 0; i < P2_NQ; i++) s += rWP[a * P2_NQ + i] * wm.hs[d * P2_NQ + i];
        bp[e] = (R)(-2) * vol_m * s;
      }
      if (lane < P2_NQ) {
        R g = 0;
#pragma unroll
        for (int d = 0; d < P2_NN; d++) g += wm.hs[d * P2_NQ + lane];
        two_sum_add(gsh, gsl, g);
      }
      __syncwarp();  // the scratch is read before the next pair writes it
    }
    flush_stats();
  }
  if (cur_m >= 0) flush_self();
}

template <typename R, int KERN>
nl_status launch_quad_p2(const QParams& P, cudaStream_t s) {
  int dev = 0, nsm = 0;
  NL_CUDA(cudaGetDevice(&dev));
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t per_warp = P2Mem<R>::bytes(P.scap);
  int warps = P2_WARPS;
  while (warps > 1 && p2_table_bytes<R>() + warps * per_warp > (size_t)200 * 1024) warps >>= 1;
  const size_t smem = p2_table_bytes<R>() + warps * per_warp;
  if (smem > (size_t)220 * 1024)
    return fail(NL_EINTERNAL, "P2 assembly kernel needs %zu bytes of shared memory", smem);
  auto kern = k_quad_p2<R, KERN>;
  NL_TRY(allow_smem(kern, smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "P2 assembly kernel does not fit on an SM (smem %zu)", smem);
  kern<<<NL_CNT(nsm * per_sm), warps * 32, smem, s>>>(P);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

// The batches of pairs through k_quad_p2, each followed by the scatter of its cross blocks,
// then the self blocks (and, in FP32, the diagonals from the row sums).
template <typename R, int KERN>
nl_status run_assembly_p2(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s,
                          unsigned long long* scratch, int* err, PhaseTimer& T) {
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
  if (g_block_budget) budget = std::min(budget, g_block_budget);
  int64_t batch = std::max<int64_t>(1 << 20, (int64_t)(budget / (sizeof(R) * P2_NBLK)));
  batch = std::min<int64_t>(batch, p->n_pairs);
  DevBuf<R> blk;
  DevBuf<double> selfblk;
  NL_TRY(blk.alloc((size_t)batch * P2_NBLK, s));
  NL_TRY(selfblk.alloc((size_t)m->n_elem * P2_NBLK, s));
  NL_CUDA(cudaMemsetAsync(selfblk.p, 0, sizeof(double) * m->n_elem * P2_NBLK, s));
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
    NL_TRY((launch_quad_p2<R, KERN>(P, s)));
    NL_TRY(T.mark(0, s));
    NL_TRY(T.mark(1, s));
    NL_TRY((launch_scatter<2, R, P2_NN>(m, p, b0, b1, blk.p, nullptr, 0, values, err, s, h_off.data())));
    NL_TRY(T.mark(1, s));
  }
  NL_TRY(T.mark(1, s));
  NL_TRY((launch_scatter<2, R, P2_NN>(m, p, 0, 0, blk.p, selfblk.p, 1, values, err, s, h_off.data())));
  NL_TRY(T.mark(1, s));
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}

}  // namespace

nl_status assemble_values_p2(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                             const nl_quad_params* qp, nl_precision prec, double* values,
                             nl_assemble_stats* st) {
  if (m->dim != 2 || m->nb != P2_NN) return fail(NL_EINVAL, "nl_assemble: not a mesh of P2 triangles");
  QParams P;
  NL_TRY(fill_qparams("nl_assemble", m, p, kp, qp, prec, &P));
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
    if (f32) rc = gauss ? run_assembly_p2<float, 1>(m, p, P, values, s, scratch.p, err.p, T)
                        : run_assembly_p2<float, 0>(m, p, P, values, s, scratch.p, err.p, T);
    else rc = gauss ? run_assembly_p2<double, 1>(m, p, P, values, s, scratch.p, err.p, T)
                    : run_assembly_p2<double, 0>(m, p, P, values, s, scratch.p, err.p, T);
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
    st->n_point_pairs = (int64_t)hs[1] * P2_NQ * P2_NQ;
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
