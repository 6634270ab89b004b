// nl_quad.cu -- assembly of the mollified nonlocal stiffness matrix on the GPU.
//
// What is computed (Sec. 5, Corollary 1, eqs. J21Nr and J22Nr): for every element pair
// (m, l) of J, with the inner degree-5 rule on E_m (points y, weights w_y, rows = nodes of m)
// and the outer rule on the sub-elements E' of E_l that Algorithm 1 selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_c] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_c(x).
// Algorithm 1 is applied per pair; this is the same computation as the per-l recursion with
// the index set J_l, because the tests and the integration act on every m separately.
//
// How: a persistent grid; each warp takes chunks of consecutive pairs (m-major) from a
// global counter.  For one pair the warp runs Algorithm 1 as a LIFO of refined
// sub-elements ("parent records", vertices + path code) in shared memory: each round pops
// up to 32/2^N parents and every lane builds one child by midpoints, classifies it with the
// box distances of Sec. 5.1 and either drops it, pushes it, or appends it to one of two item
// buffers: INT (max-dist < delta-eps, mu = 1 at every point pair) or FINAL (the sub-element
// reached L_max with the band in reach).  A full buffer is integrated by the whole warp:
// each lane owns one outer point x of the buffered items and a set of 7 inner points y kept
// in registers, and accumulates per y the sums g = sum_x w_x C eta mu and
// h_k = sum_x w_x C eta mu lambda^l_k(x).  At the end of the pair the lanes reduce these and
// the cross block is scattered with FP64 atomics; the self block needs only g and is
// accumulated over the consecutive pairs of the same m before it is scattered.
//
// Precision: R = double evaluates everything in FP64 and classifies in FP64.  R = float
// evaluates gamma_eps in FP32 on coordinates relative to the first vertex of m, and screens
// the classification in FP32: a decision whose FP32 distance lies within a proven margin of
// the threshold is redone in FP64 on vertices rebuilt from E_l by the same midpoint
// sequence, so the decisions are those of a plain FP64 evaluation in both precisions.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>

#include "nl_internal.h"

namespace nlx {

nl_status ensure_device_tables() {
  if (rule(2).n != 7 || rule(3).n != 14)
    return fail(NL_EINTERNAL, "quadrature rule set-up failed");
  return NL_OK;
}

namespace {

constexpr int KIND_INT = 0;
constexpr int KIND_FINAL = 1;
// ACT_ZERO: a sub-element at L_max that Algorithm 1 integrates but whose every point pair is
// farther than delta + eps (mu = 0): counted, not evaluated.
constexpr int ACT_DROP = 0, ACT_INT = 1, ACT_FINAL = 2, ACT_REFINE = 3, ACT_ZERO = 4;
constexpr int ERR_STACK = 1, ERR_CSR = 2;
constexpr int CHUNK = 8;
constexpr int IMAX = 64;
constexpr int LEVEL_SHIFT = 27;

struct QParams {
  int64_t n_pairs, n_elem;
  const int64_t* pair_off;
  const int32_t* pair_l;
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* conn;
  const double* evert;
  const double* blo;
  const double* bhi;
  const double* vol;
  const double* jinv;
  double* values;
  unsigned long long* counter;
  unsigned long long* stats;  // [0] items, [2] exact checks, [3] evaluated pairs, [4] uniform points
  int* err;
  double delta, dme, dpe, C, inv_eps, inv_delta2;
  float fdelta, finv_eps, fdme2, fdpe2, finv_delta2, margin, fdme, fdpe;
  int L_min, L_max, scap, count_band;
  double B[14][4];
  double W[14];
};

template <int D>
struct Geo {
  static constexpr int NV = D + 1;
  static constexpr int NQ = D == 2 ? 7 : 14;
  static constexpr int NCH = 1 << D;
  static constexpr int NPOP = 32 / NCH;
  static constexpr int XPI = D == 2 ? 32 : 16;  // distinct outer points per warp iteration
  static constexpr int NYL = 7;                 // inner points per lane
  static constexpr int NVC = NV * D;            // vertex coordinates of a simplex
  static constexpr int BITS = D;                // path bits per level
};

// child c, vertex v = midpoint of parent vertices (MA, MB); a corner is mid(P, P) = P exactly
__constant__ unsigned char c_mid2[4][3][2] = {{{0, 0}, {0, 1}, {0, 2}},
                                              {{0, 1}, {1, 1}, {1, 2}},
                                              {{0, 2}, {1, 2}, {2, 2}},
                                              {{0, 1}, {1, 2}, {0, 2}}};
__constant__ unsigned char c_mid3[8][4][2] = {
    {{0, 0}, {0, 1}, {0, 2}, {0, 3}}, {{0, 1}, {1, 1}, {1, 2}, {1, 3}},
    {{0, 2}, {1, 2}, {2, 2}, {2, 3}}, {{0, 3}, {1, 3}, {2, 3}, {3, 3}},
    {{0, 1}, {0, 2}, {0, 3}, {1, 3}}, {{0, 1}, {0, 2}, {1, 2}, {1, 3}},
    {{0, 2}, {0, 3}, {1, 3}, {2, 3}}, {{0, 2}, {1, 2}, {1, 3}, {2, 3}}};

template <int D>
__device__ __forceinline__ void mid_pair(int c, int v, int& a, int& b) {
  if (D == 2) {
    a = c_mid2[c][v][0];
    b = c_mid2[c][v][1];
  } else {
    a = c_mid3[c][v][0];
    b = c_mid3[c][v][1];
  }
}

__device__ __forceinline__ double midp(double a, double b) { return __dmul_rn(__dadd_rn(a, b), 0.5); }
__device__ __forceinline__ float midp(float a, float b) { return __fmul_rn(__fadd_rn(a, b), 0.5f); }

// Exact FP64 box distances of Sec. 5.1 (eqs. maxdist, mindist) between a sub-element with
// vertices V and the box (lo2, hi2) of E_m, written as in a plain evaluation.
template <int D>
__device__ void exact_dists(const double (&V)[D + 1][D], const double* lo2, const double* hi2,
                            double& amax, double& amin) {
  double s = 0.0, mn = 0.0;
#pragma unroll
  for (int k = 0; k < D; k++) {
    double lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a <= D; a++) {
      lo = V[a][k] < lo ? V[a][k] : lo;
      hi = V[a][k] > hi ? V[a][k] : hi;
    }
    double d1 = __dsub_rn(lo, hi2[k]);
    double d2 = __dsub_rn(lo2[k], hi);
    double p = __dmul_rn(d1, d1), q = __dmul_rn(d2, d2);
    s = __dadd_rn(s, p > q ? p : q);
    double t = d1 > d2 ? d1 : d2;
    mn = t > mn ? t : mn;
  }
  amax = __dsqrt_rn(s);
  amin = mn;
}

template <int D>
__device__ void screen_dists(const float (&V)[D + 1][D], const float* lo2, const float* hi2,
                             float& amax, float& amin) {
  float s = 0.f, mn = 0.f;
#pragma unroll
  for (int k = 0; k < D; k++) {
    float lo = V[0][k], hi = V[0][k];
#pragma unroll
    for (int a = 1; a <= D; a++) {
      lo = fminf(lo, V[a][k]);
      hi = fmaxf(hi, V[a][k]);
    }
    float d1 = lo - hi2[k], d2 = lo2[k] - hi;
    s += fmaxf(d1 * d1, d2 * d2);
    mn = fmaxf(mn, fmaxf(d1, d2));
  }
  amax = sqrtf(s);
  amin = mn;
}

// Rebuilds the FP64 vertices of the sub-element with path `code` from the vertices of E_l.
template <int D>
__device__ void decode_exact(const double (&Vl)[D + 1][D], uint32_t code, double (&V)[D + 1][D]) {
  int level = code >> LEVEL_SHIFT;
#pragma unroll
  for (int a = 0; a <= D; a++)
#pragma unroll
    for (int k = 0; k < D; k++) V[a][k] = Vl[a][k];
  for (int lv = 2; lv <= level; lv++) {
    int c = (code >> (Geo<D>::BITS * (lv - 2))) & (Geo<D>::NCH - 1);
    double P[D + 1][D];
#pragma unroll
    for (int a = 0; a <= D; a++)
#pragma unroll
      for (int k = 0; k < D; k++) P[a][k] = V[a][k];
#pragma unroll
    for (int v = 0; v <= D; v++) {
      int ia, ib;
      mid_pair<D>(c, v, ia, ib);
#pragma unroll
      for (int k = 0; k < D; k++) {
        double pa = P[0][k], pb = P[0][k];
#pragma unroll
        for (int a = 1; a <= D; a++) {
          pa = (ia == a) ? P[a][k] : pa;
          pb = (ib == a) ? P[a][k] : pb;
        }
        V[v][k] = midp(pa, pb);
      }
    }
  }
}

__device__ __forceinline__ double xi_poly(double s) {
  double t = s * s;
  double p = fma(35.0, t, -180.0);
  p = fma(p, t, 378.0);
  p = fma(p, t, -420.0);
  p = fma(p, t, 315.0);
  return fma(s * p, 1.0 / 256.0, 0.5);
}
__device__ __forceinline__ float xi_poly(float s) {
  float t = s * s;
  float p = fmaf(35.f, t, -180.f);
  p = fmaf(p, t, 378.f);
  p = fmaf(p, t, -420.f);
  p = fmaf(p, t, 315.f);
  return fmaf(s * p, 1.f / 256.f, 0.5f);
}

// mu_{delta,eps}(r) from r^2 (eq. mollifier with argument (delta - r)/eps)
__device__ __forceinline__ double mollifier(const QParams& P, double r2) {
  double dme2 = P.dme * P.dme, dpe2 = P.dpe * P.dpe;
  if (r2 < dme2) return 1.0;
  if (r2 > dpe2) return 0.0;
  double r = sqrt(r2);
  return xi_poly((P.delta - r) * P.inv_eps);
}
__device__ __forceinline__ float mollifier(const QParams& P, float r2) {
  if (r2 < P.fdme2) return 1.f;
  if (r2 > P.fdpe2) return 0.f;
  float r = r2 * rsqrtf(r2);
  return xi_poly((P.fdelta - r) * P.finv_eps);
}

template <typename R>
__device__ __forceinline__ R eta_gauss(const QParams& P, R r2);
template <>
__device__ __forceinline__ double eta_gauss<double>(const QParams& P, double r2) {
  return exp(-r2 * P.inv_delta2);
}
template <>
__device__ __forceinline__ float eta_gauss<float>(const QParams& P, float r2) {
  return __expf(-r2 * P.finv_delta2);
}

__device__ __forceinline__ int64_t csr_find(const int64_t* __restrict__ row_ptr,
                                            const int32_t* __restrict__ col, int32_t i, int32_t j) {
  int64_t lo = row_ptr[i], hi = row_ptr[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    int32_t c = col[mid];
    if (c == j) return mid;
    if (c < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

template <typename R>
__device__ __forceinline__ R shfl_xor(R v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

// Per-warp shared memory: stack records and the two item buffers (SoA), sized at launch.
template <int D, typename R>
struct WarpMem {
  R* rv;          // [NVC][scap]
  uint32_t* rc;   // [scap]
  R* iv;          // [2][NVC][IMAX]
  R* iw;          // [2][IMAX]
  int* ctl;       // [0] sp, [1] n_int, [2] n_final
  static __host__ __device__ size_t bytes(int scap) {
    size_t b = sizeof(R) * (size_t)Geo<D>::NVC * scap + sizeof(uint32_t) * scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * (size_t)2 * Geo<D>::NVC * IMAX + sizeof(R) * 2 * IMAX;
    b += 16;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    rv = reinterpret_cast<R*>(base);
    rc = reinterpret_cast<uint32_t*>(rv + (size_t)Geo<D>::NVC * scap);
    size_t off = sizeof(R) * (size_t)Geo<D>::NVC * scap + sizeof(uint32_t) * scap;
    off = (off + 15) & ~size_t(15);
    iv = reinterpret_cast<R*>(base + off);
    iw = iv + (size_t)2 * Geo<D>::NVC * IMAX;
    ctl = reinterpret_cast<int*>(iw + 2 * IMAX);
  }
};

template <int D, typename R, int KERN>
__global__ void __launch_bounds__(256) k_quad(const QParams P) {
  using G = Geo<D>;
  constexpr int NV = G::NV, NQ = G::NQ, NYL = G::NYL, NVC = G::NVC;
  constexpr bool F32 = std::is_same<R, float>::value;
  extern __shared__ __align__(16) char smem_raw[];
  // CTA-shared tables
  R* sB = reinterpret_cast<R*>(smem_raw);  // [NQ][NV]
  R* sW = sB + 14 * 4;                      // [NQ]
  R* sWB = sW + 16;                         // [NQ][NV]: W[q] * B[q][a]
  const int tid = threadIdx.x;
  for (int t = tid; t < NQ * NV; t += blockDim.x) {
    sB[t] = (R)P.B[t / NV][t % NV];
    sWB[t] = (R)(P.W[t / NV] * P.B[t / NV][t % NV]);
  }
  for (int t = tid; t < NQ; t += blockDim.x) sW[t] = (R)P.W[t];
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5;
  size_t tbl = (sizeof(R) * (14 * 4 * 2 + 16) + 15) & ~size_t(15);
  WarpMem<D, R> wm;
  wm.carve(smem_raw + tbl + (size_t)wid * WarpMem<D, R>::bytes(P.scap), P.scap);

  const int ybase = (D == 3 && lane >= 16) ? 7 : 0;
  const int xl = (D == 3) ? (lane & 15) : lane;

  // accumulators
  R gself[NYL];
#pragma unroll
  for (int i = 0; i < NYL; i++) gself[i] = 0;
  unsigned long long st_items = 0, st_exact = 0, st_eval = 0, st_unif = 0, st_band = 0;
  int err = 0;

  int64_t cur_m = -1;
  double Vm[NV][D];            // global FP64 vertices of m
  double lo_m[D], hi_m[D];     // FP64 box of m
  float flo_m[D], fhi_m[D];    // box of m relative to the origin (FP32 screen)
  double org[D];               // origin of the local coordinates (vertex 0 of m)
  R y[NYL][D];                 // inner points (local coordinates if R = float)
  R vol_m = 0;
  int32_t nodes_m[NV] = {};

  auto flush_self = [&]() {
    // reduce g over the lanes that share the same inner points
#pragma unroll
    for (int i = 0; i < NYL; i++) {
      R v = gself[i];
      if (D == 2) v += shfl_xor(v, 16);
      v += shfl_xor(v, 8);
      v += shfl_xor(v, 4);
      v += shfl_xor(v, 2);
      v += shfl_xor(v, 1);
      gself[i] = v;
    }
    // S[a][b] = 2 vol_m sum_y W B_a B_b g(y)
    int t = (D == 3) ? (lane & 15) : lane;
    R s = 0;
    if (t < NV * NV) {
      int a = t / NV, b = t % NV;
#pragma unroll
      for (int i = 0; i < NYL; i++) {
        int q = ybase + i;
        s += sWB[q * NV + a] * sB[q * NV + b] * gself[i];
      }
    }
    if (D == 3) s += shfl_xor(s, 16);
    if (lane < NV * NV) {
      int a = lane / NV, b = lane % NV;
      double val = 2.0 * (double)vol_m * (double)s;
      int64_t pos = csr_find(P.row_ptr, P.col, nodes_m[a], nodes_m[b]);
      if (pos < 0) err |= ERR_CSR;
      else atomicAdd(&P.values[pos], val);
    }
#pragma unroll
    for (int i = 0; i < NYL; i++) gself[i] = 0;
  };

  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(P.counter, (unsigned long long)CHUNK);
    start = __shfl_sync(0xffffffffu, start, 0);
    if ((int64_t)start >= P.n_pairs) break;
    int64_t end = min((int64_t)start + CHUNK, P.n_pairs);
    // element m of the first pair: pair_off[m] <= start < pair_off[m+1]
    int64_t m;
    if (cur_m >= 0 && P.pair_off[cur_m] <= (int64_t)start && (int64_t)start < P.pair_off[cur_m + 1]) {
      m = cur_m;
    } else {
      // the last m with pair_off[m] <= start (pair_off[0] = 0 <= start < pair_off[n_elem])
      int64_t lo = 0, hi = P.n_elem;
      while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (P.pair_off[mid] <= (int64_t)start) lo = mid;
        else hi = mid;
      }
      m = lo;
    }
    for (int64_t p = (int64_t)start; p < end; p++) {
      while (p >= P.pair_off[m + 1]) m++;
      if (m != cur_m) {
        if (cur_m >= 0) flush_self();
        cur_m = m;
#pragma unroll
        for (int a = 0; a < NV; a++) {
          nodes_m[a] = P.conn[m * NV + a];
#pragma unroll
          for (int k = 0; k < D; k++) Vm[a][k] = P.evert[(m * NV + a) * D + k];
        }
#pragma unroll
        for (int k = 0; k < D; k++) {
          lo_m[k] = P.blo[m * D + k];
          hi_m[k] = P.bhi[m * D + k];
          org[k] = Vm[0][k];
          flo_m[k] = (float)(lo_m[k] - org[k]);
          fhi_m[k] = (float)(hi_m[k] - org[k]);
        }
        vol_m = (R)P.vol[m];
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          int q = ybase + i;
#pragma unroll
          for (int k = 0; k < D; k++) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < NV; a++) s += P.B[q][a] * (F32 ? (Vm[a][k] - org[k]) : Vm[a][k]);
            y[i][k] = (R)s;
          }
        }
      }
      const int32_t l = P.pair_l[p];
      // ---- per-pair set-up --------------------------------------------------------------
      double Vl[NV][D];
#pragma unroll
      for (int a = 0; a < NV; a++)
#pragma unroll
        for (int k = 0; k < D; k++) Vl[a][k] = P.evert[((int64_t)l * NV + a) * D + k];
      R vl0[D], Ji[D][D];
#pragma unroll
      for (int k = 0; k < D; k++) vl0[k] = (R)(F32 ? Vl[0][k] - org[k] : Vl[0][k]);
#pragma unroll
      for (int r = 0; r < D; r++)
#pragma unroll
        for (int c = 0; c < D; c++) Ji[r][c] = (R)P.jinv[((int64_t)l * D + r) * D + c];
      const double vol_l = P.vol[l];
      int32_t nodes_l[NV];
#pragma unroll
      for (int a = 0; a < NV; a++) nodes_l[a] = P.conn[(int64_t)l * NV + a];

      R gp[NYL], hp[D][NYL], ug = 0, uh[D];
#pragma unroll
      for (int i = 0; i < NYL; i++) {
        gp[i] = 0;
#pragma unroll
        for (int k = 0; k < D; k++) hp[k][i] = 0;
      }
#pragma unroll
      for (int k = 0; k < D; k++) uh[k] = 0;

      // classification of a sub-element (Algorithm 1); V in R coordinates
      auto classify = [&](const R (&V)[NV][D], uint32_t code) -> int {
        int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        bool last = level == P.L_max;
        double amax, amin;
        bool certain_int = false, certain_not_int = false, certain_ref = false, certain_out = false;
        if (F32) {
          float fam, fan;
          float Vf[NV][D];
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vf[a][k] = (float)V[a][k];
          screen_dists<D>(Vf, flo_m, fhi_m, fam, fan);
          certain_int = fam < P.fdme - P.margin;
          certain_not_int = fam > P.fdme + P.margin;
          certain_ref = fan < P.fdpe - P.margin;
          certain_out = fan > P.fdpe + P.margin;
          if (last) {
            if (certain_int) return ACT_INT;
            if (certain_out) return ACT_ZERO;
            return ACT_FINAL;
          }
          if (certain_int) return ACT_INT;
          if (certain_not_int && certain_ref) return ACT_REFINE;
          if (certain_not_int && certain_out) return ACT_DROP;
          double Vd[NV][D];
          decode_exact<D>(Vl, code, Vd);
          exact_dists<D>(Vd, lo_m, hi_m, amax, amin);
          st_exact += (code >> LEVEL_SHIFT) == 1 ? (lane == 0) : 1;
        } else {
          double Vd[NV][D];
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vd[a][k] = (double)V[a][k];
          exact_dists<D>(Vd, lo_m, hi_m, amax, amin);
          if (last) {
            if (amax < P.dme) return ACT_INT;
            if (amin > P.dpe) return ACT_ZERO;
            return ACT_FINAL;
          }
        }
        if (amax < P.dme) return ACT_INT;
        if (amin < P.dpe) return ACT_REFINE;
        return ACT_DROP;
      };

      // integrate the buffered items of one kind (warp-collective)
      auto integrate = [&](int kind, int n_it) {
        const R* iv = wm.iv + (size_t)kind * NVC * IMAX;
        const R* iw = wm.iw + kind * IMAX;
        const int n_x = n_it * NQ;
        st_eval += (unsigned long long)n_x * NQ;
        for (int base = 0; base < n_x; base += G::XPI) {
          int o = base + xl;
          bool valid = o < n_x;
          int it = valid ? o / NQ : 0;
          int q = valid ? o - it * NQ : 0;
          R x[D];
#pragma unroll
          for (int k = 0; k < D; k++) {
            R s = 0;
#pragma unroll
            for (int a = 0; a < NV; a++) s += sB[q * NV + a] * iv[(a * D + k) * IMAX + it];
            x[k] = s;
          }
          R wcx = valid ? sW[q] * iw[it] : (R)0;
          R lam[D];
#pragma unroll
          for (int r = 0; r < D; r++) {
            R s = 0;
#pragma unroll
            for (int c = 0; c < D; c++) s += Ji[r][c] * (x[c] - vl0[c]);
            lam[r] = s;
          }
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            R r2 = 0;
#pragma unroll
            for (int k = 0; k < D; k++) {
              R d = x[k] - y[i][k];
              r2 += d * d;
            }
            R g = wcx;
            if (kind == KIND_FINAL) {
              g *= mollifier(P, r2);
              if (P.count_band) st_band += (r2 >= P.fdme2 && r2 <= P.fdpe2 && valid) ? 1 : 0;
            }
            if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= eta_gauss<R>(P, r2);
            gp[i] += g;
#pragma unroll
            for (int k = 0; k < D; k++) hp[k][i] += g * lam[k];
          }
        }
      };

      // A sub-element with max-dist < delta - eps has mu = 1 at every point pair; with the
      // constant kernel its outer sum is sum_q w_q C [1, lambda^l(x_q)] = C |E'| [1,
      // lambda^l(centroid)], because the degree-5 rule integrates linear functions exactly.
      auto closed_int = [&](const R (&V)[NV][D], int level) {
        R cen[D];
#pragma unroll
        for (int k = 0; k < D; k++) {
          R s = 0;
#pragma unroll
          for (int a = 0; a < NV; a++) s += V[a][k];
          cen[k] = s * (R)(1.0 / NV);
        }
        R wv = (R)(P.C * ldexp(vol_l, -D * (level - 1)));
        ug += wv;
#pragma unroll
        for (int r = 0; r < D; r++) {
          R s = 0;
#pragma unroll
          for (int c = 0; c < D; c++) s += Ji[r][c] * (cen[c] - vl0[c]);
          uh[r] += wv * s;
        }
        st_unif++;
      };

      // ---- Algorithm 1 for this pair ----------------------------------------------------------
      if (lane == 0) {
        wm.ctl[0] = 0;
        wm.ctl[1] = 0;
        wm.ctl[2] = 0;
      }
      __syncwarp();
      {
        R V0[NV][D];
#pragma unroll
        for (int a = 0; a < NV; a++)
#pragma unroll
          for (int k = 0; k < D; k++) V0[a][k] = (R)(F32 ? Vl[a][k] - org[k] : Vl[a][k]);
        const uint32_t code0 = 1u << LEVEL_SHIFT;
        int act = classify(V0, code0);
        if (lane == 0) {
          if (act == ACT_REFINE) {
#pragma unroll
            for (int t = 0; t < NVC; t++) wm.rv[t * P.scap] = V0[t / D][t % D];
            wm.rc[0] = code0;
            wm.ctl[0] = 1;
          } else if (KERN == NL_KERNEL_CONST && act == ACT_INT) {
            closed_int(V0, 1);
          } else if (act == ACT_INT || act == ACT_FINAL) {
            int kind = act == ACT_INT ? KIND_INT : KIND_FINAL;
            R* iv = wm.iv + (size_t)kind * NVC * IMAX;
#pragma unroll
            for (int t = 0; t < NVC; t++) iv[t * IMAX] = V0[t / D][t % D];
            wm.iw[kind * IMAX] = (R)(P.C * vol_l);
            wm.ctl[1 + kind] = 1;
          }
        }
        if (lane == 0 && (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO)) st_items++;
        __syncwarp();
      }
      for (;;) {
        int n_int = wm.ctl[1], n_fin = wm.ctl[2];
        if (n_fin > IMAX - 32) {
          integrate(KIND_FINAL, n_fin);
          n_fin = 0;
        }
        if (n_int > IMAX - 32) {
          integrate(KIND_INT, n_int);
          n_int = 0;
        }
        const int sp = wm.ctl[0];
        if (sp == 0) {
          __syncwarp();
          if (lane == 0) {
            wm.ctl[1] = n_int;
            wm.ctl[2] = n_fin;
          }
          __syncwarp();
          break;
        }
        const int np = min(G::NPOP, sp);
        const int base = sp - np;
        const int par = lane / G::NCH, c = lane % G::NCH;
        const bool active = par < np;
        R V[NV][D];
        uint32_t code = 0;
        int act = ACT_DROP;
        if (active) {
          const int slot = base + par;
          uint32_t pcode = wm.rc[slot];
          int plevel = pcode >> LEVEL_SHIFT;
#pragma unroll
          for (int v = 0; v < NV; v++) {
            int ia, ib;
            mid_pair<D>(c, v, ia, ib);
#pragma unroll
            for (int k = 0; k < D; k++)
              V[v][k] = midp(wm.rv[(ia * D + k) * P.scap + slot], wm.rv[(ib * D + k) * P.scap + slot]);
          }
          code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) |
                 (pcode & ((1u << LEVEL_SHIFT) - 1)) | ((uint32_t)c << (G::BITS * (plevel - 1)));
        }
        __syncwarp();
        if (active) act = classify(V, code);
        if (KERN == NL_KERNEL_CONST && act == ACT_INT) {
          closed_int(V, (int)(code >> LEVEL_SHIFT));
          st_items++;
          act = ACT_DROP;
        }
        // append items and push refined sub-elements
        const unsigned m_int = __ballot_sync(0xffffffffu, act == ACT_INT);
        const unsigned m_fin = __ballot_sync(0xffffffffu, act == ACT_FINAL);
        const unsigned m_ref = __ballot_sync(0xffffffffu, act == ACT_REFINE);
        const unsigned below = (1u << lane) - 1u;
        if (act == ACT_INT || act == ACT_FINAL) {
          int kind = act == ACT_INT ? KIND_INT : KIND_FINAL;
          int slot = (kind == KIND_INT ? n_int + __popc(m_int & below) : n_fin + __popc(m_fin & below));
          R* iv = wm.iv + (size_t)kind * NVC * IMAX;
#pragma unroll
          for (int t = 0; t < NVC; t++) iv[t * IMAX + slot] = V[t / D][t % D];
          int level = code >> LEVEL_SHIFT;
          wm.iw[kind * IMAX + slot] = (R)(P.C * ldexp(vol_l, -D * (level - 1)));
          st_items++;
        }
        if (act == ACT_ZERO) st_items++;
        const int nref = __popc(m_ref);
        if (base + nref > P.scap) {
          err |= ERR_STACK;
        } else if (act == ACT_REFINE) {
          int slot = base + __popc(m_ref & below);
#pragma unroll
          for (int t = 0; t < NVC; t++) wm.rv[t * P.scap + slot] = V[t / D][t % D];
          wm.rc[slot] = code;
        }
        __syncwarp();
        if (lane == 0) {
          wm.ctl[0] = (base + nref > P.scap) ? base : base + nref;
          wm.ctl[1] = n_int + __popc(m_int);
          wm.ctl[2] = n_fin + __popc(m_fin);
        }
        __syncwarp();
      }
      {
        int n_int = wm.ctl[1], n_fin = wm.ctl[2];
        if (n_fin > 0) integrate(KIND_FINAL, n_fin);
        if (n_int > 0) integrate(KIND_INT, n_int);
      }
      __syncwarp();
      // ---- end of pair: fold, reduce, scatter the cross block --------------------------------
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ug += shfl_xor(ug, o);
#pragma unroll
        for (int k = 0; k < D; k++) uh[k] += shfl_xor(uh[k], o);
      }
#pragma unroll
      for (int i = 0; i < NYL; i++) {
        gself[i] += gp[i];
        if (xl == 0) gself[i] += ug;  // once per group of lanes that share these inner points
      }
#pragma unroll
      for (int i = 0; i < NYL; i++) {
        R a0 = gp[i];
        R ak[D];
#pragma unroll
        for (int k = 0; k < D; k++) ak[k] = hp[k][i];
#pragma unroll
        for (int o = (D == 2 ? 16 : 8); o > 0; o >>= 1) {
          a0 += shfl_xor(a0, o);
#pragma unroll
          for (int k = 0; k < D; k++) ak[k] += shfl_xor(ak[k], o);
        }
        gp[i] = a0 + ug;
#pragma unroll
        for (int k = 0; k < D; k++) hp[k][i] = ak[k] + uh[k];
      }
      {
        // X[a][c] = vol_m sum_y W B_a(y) H_c(y), H_0 = g - sum_k h_k, H_c = h_{c-1}
        int t = (D == 3) ? (lane & 15) : lane;
        R s = 0;
        if (t < NV * NV) {
          int a = t / NV, c = t % NV;
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            int q = ybase + i;
            R H;
            if (c == 0) {
              H = gp[i];
#pragma unroll
              for (int k = 0; k < D; k++) H -= hp[k][i];
            } else {
              H = hp[0][i];
#pragma unroll
              for (int k = 1; k < D; k++) H = (c - 1 == k) ? hp[k][i] : H;
            }
            s += sWB[q * NV + a] * H;
          }
        }
        if (D == 3) s += shfl_xor(s, 16);
        if (lane < NV * NV) {
          int a = lane / NV, c = lane % NV;
          double val = -2.0 * (double)vol_m * (double)s;
          int64_t pos = csr_find(P.row_ptr, P.col, nodes_m[a], nodes_l[c]);
          if (pos < 0) err |= ERR_CSR;
          else atomicAdd(&P.values[pos], val);
        }
      }
    }
  }
  if (cur_m >= 0) flush_self();
  // statistics and errors
  for (int o = 16; o > 0; o >>= 1) {
    st_items += __shfl_xor_sync(0xffffffffu, st_items, o);
    st_exact += __shfl_xor_sync(0xffffffffu, st_exact, o);
    st_unif += __shfl_xor_sync(0xffffffffu, st_unif, o);
    st_band += __shfl_xor_sync(0xffffffffu, st_band, o);
    err |= __shfl_xor_sync(0xffffffffu, err, o);
  }
  if (lane == 0) {
    atomicAdd(&P.stats[0], st_items);
    atomicAdd(&P.stats[2], st_exact);
    atomicAdd(&P.stats[3], st_eval);
    atomicAdd(&P.stats[4], st_unif);
    atomicAdd(&P.stats[5], st_band);
    if (err) atomicOr(P.err, err);
  }
}

template <int D, typename R, int KERN>
nl_status launch_quad(const QParams& P, cudaStream_t s, int* blocks_out) {
  int dev = 0;
  NL_CUDA(cudaGetDevice(&dev));
  int nsm = 0;
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  size_t tbl = (sizeof(R) * (14 * 4 * 2 + 16) + 15) & ~size_t(15);
  int warps = 8;
  while (warps > 1 && tbl + warps * WarpMem<D, R>::bytes(P.scap) > (size_t)200 * 1024) warps >>= 1;
  const int threads = warps * 32;
  size_t smem = tbl + warps * WarpMem<D, R>::bytes(P.scap);
  if (smem > (size_t)220 * 1024) return fail(NL_EINTERNAL, "assembly kernel needs %zu bytes of shared memory", smem);
  NL_CUDA(cudaFuncSetAttribute(k_quad<D, R, KERN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_quad<D, R, KERN>, threads, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "assembly kernel does not fit on an SM (smem %zu)", smem);
  int blocks = nsm * per_sm;
  k_quad<D, R, KERN><<<NL_CNT(blocks), threads, smem, s>>>(P);
  NL_CUDA(cudaGetLastError());
  if (blocks_out) *blocks_out = blocks;
  return NL_OK;
}

}  // namespace

nl_status assemble_values(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                          const nl_quad_params* qp, nl_precision prec, double* values,
                          nl_assemble_stats* st) {
  const int D = m->dim;
  if (!(kp->eps > 0.0 && kp->eps < kp->delta)) return fail(NL_EINVAL, "nl_assemble: need 0 < eps < delta");
  if (kp->kernel != NL_KERNEL_CONST && kp->kernel != NL_KERNEL_TRUNC_GAUSS)
    return fail(NL_EINVAL, "nl_assemble: unknown kernel %d", kp->kernel);
  const int lmax_cap = D == 2 ? 12 : 9;
  if (qp->L_min < 1 || qp->L_max < qp->L_min || qp->L_max > lmax_cap)
    return fail(NL_EINVAL, "nl_assemble: need 1 <= L_min <= L_max <= %d", lmax_cap);
  if ((qp->rule & ~NL_QUAD_COUNT_BAND) != 0) return fail(NL_EINVAL, "nl_assemble: only rule 0 is available");
  if (prec != NL_PREC_FP64 && prec != NL_PREC_FP32 && prec != NL_PREC_MIXED_TF32 &&
      prec != NL_PREC_MIXED_BF16)
    return fail(NL_EINVAL, "nl_assemble: unknown precision %d", (int)prec);
  cudaStream_t s = m->stream;
  QParams P;
  memset(&P, 0, sizeof P);
  P.n_pairs = p->n_pairs;
  P.n_elem = m->n_elem;
  P.pair_off = p->pair_off;
  P.pair_l = p->pair_l;
  P.row_ptr = p->row_ptr;
  P.col = p->col;
  P.conn = m->conn;
  P.evert = m->evert;
  P.blo = m->blo;
  P.bhi = m->bhi;
  P.vol = m->vol;
  P.jinv = m->jinv;
  P.values = values;
  double C = kp->C_override > 0.0 ? kp->C_override
                                  : kernel_constant(D, kp->kernel, kp->delta, kp->eps);
  if (kp->kappa > 0.0) C *= kp->kappa;
  P.delta = kp->delta;
  P.dme = kp->delta - kp->eps;
  P.dpe = kp->delta + kp->eps;
  P.C = C;
  P.inv_eps = 1.0 / kp->eps;
  P.inv_delta2 = 1.0 / (kp->delta * kp->delta);
  P.fdelta = (float)kp->delta;
  P.finv_eps = (float)(1.0 / kp->eps);
  P.fdme = (float)P.dme;
  P.fdpe = (float)P.dpe;
  P.fdme2 = (float)(P.dme * P.dme);
  P.fdpe2 = (float)(P.dpe * P.dpe);
  P.finv_delta2 = (float)P.inv_delta2;
  // bound on |local coordinates| and on the FP32 error of the screened distances
  double R = kp->delta + kp->eps + 2.0 * m->max_ext;
  P.margin = (float)(2e-5 * R);
  P.L_min = qp->L_min;
  P.count_band = (qp->rule & NL_QUAD_COUNT_BAND) ? 1 : 0;
  P.L_max = qp->L_max;
  int64_t total = 0, pw = 1;
  for (int k = 1; k < qp->L_max; k++) {
    total += pw;
    pw *= (D == 2 ? 4 : 8);
    if (total > 512) break;
  }
  P.scap = (int)std::max<int64_t>(8, std::min<int64_t>(total, 512));
  const Rule& r = rule(D);
  for (int q = 0; q < r.n; q++) {
    for (int a = 0; a <= D; a++) P.B[q][a] = r.bary[q][a];
    P.W[q] = r.w[q];
  }
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
  bool f32 = prec != NL_PREC_FP64;
  bool gauss = kp->kernel == NL_KERNEL_TRUNC_GAUSS;
  if (p->n_pairs > 0) {
    if (D == 2) {
      if (f32) rc = gauss ? launch_quad<2, float, 1>(P, s, nullptr) : launch_quad<2, float, 0>(P, s, nullptr);
      else rc = gauss ? launch_quad<2, double, 1>(P, s, nullptr) : launch_quad<2, double, 0>(P, s, nullptr);
    } else {
      if (f32) rc = gauss ? launch_quad<3, float, 1>(P, s, nullptr) : launch_quad<3, float, 0>(P, s, nullptr);
      else rc = gauss ? launch_quad<3, double, 1>(P, s, nullptr) : launch_quad<3, double, 0>(P, s, nullptr);
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
    const int nq = r.n;
    st->n_pairs = p->n_pairs;
    st->n_items = (int64_t)hs[1];
    st->n_point_pairs = (int64_t)hs[1] * nq * nq;
    st->n_exact_checks = (int64_t)hs[3];
    st->ms_assemble = ms;
    st->n_eval_point_pairs = (int64_t)hs[4];
    st->n_closed_items = (int64_t)hs[5];
    st->n_band_point_pairs = P.count_band ? (int64_t)hs[6] : -1;
  }
  return NL_OK;
}

}  // namespace nlx
