// nl_quad_p2t.cu -- nl_assemble on meshes of quadratic (P2) tetrahedra.
//
// What is computed is the P1 tetrahedron computation of nl_quad_kernel.cuh with the P2 basis
// (Sec. 5, Corollary 1, eqs. J21Nr and J22Nr): for every element pair (m, l) of J, the inner
// 14-point degree-5 rule on E_m (rows = the ten nodes of m) and the outer rule on the
// sub-elements E' of E_l that Algorithm 1 (Bey's midpoint split) selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_d] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_d(x),
// phi the P2 basis: lambda_a (2 lambda_a - 1) at the vertices, 4 lambda_i lambda_j at the
// nodes of the edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  Algorithm 1 looks only at the
// vertices, so it decides exactly as for P1 tetrahedra.
//
// How (k_quad_p2t): the P1 kernels' structure -- a persistent grid, chunks of consecutive
// m-major pairs per warp, Algorithm 1 as a warp LIFO (4 parents x 8 Bey children per round)
// with the P1 kernel's decisions (FP64 in the FP64 path; the FP32 screen and the FP64
// re-decision inside its margin in the FP32 path), buffered sub-elements integrated by the
// warp.  The two half-warps share the outer points (16 per pass) and hold m's inner points
// 0-6 and 7-13: per inner point a lane accumulates H_d(y) = sum_x w_x C eta mu phi^l_d(x) for
// the ten nodes d of l (70 sums).  The end of a pair sums H over the 16 lanes of each half
// through shared memory, writes the 10 x 10 cross block -2 |E_m| sum_y w_y phi^m_a(y) H_d(y)
// and keeps g(y) = sum_d H_d(y) for m's self block.  With the constant kernel an INT
// sub-element adds sum_x w_x C phi^l_d(x), independent of y, to every inner point without
// evaluating point pairs (summed over the warp at the end of the pair).
#include <cuda_runtime.h>

#include "nl_quad_kernel.cuh"

namespace nlx {
namespace {

constexpr int PT_NN = 10;                 // nodes per element
constexpr int PT_NQ = 14;                 // points of the degree-5 tetrahedron rule
constexpr int PT_NYL = 7;                 // inner points per lane
constexpr int PT_XPI = 16;                // outer points per pass
constexpr int PT_NH = PT_NN * PT_NQ;      // H_d(y) per pair
constexpr int PT_NBLK = PT_NN * PT_NN;
constexpr int PT_IMAX = 64;               // buffered sub-elements
constexpr int PT_RS = 17;                 // row stride of the reduction scratch
constexpr int PT_WARPS = 4;

// edge j of the tetrahedron: (ea, eb)
__host__ __device__ constexpr int pt_ea(int j) { return j == 0 ? 0 : j == 1 ? 1 : j == 2 ? 0 : j == 3 ? 0 : j == 4 ? 1 : 2; }
__host__ __device__ constexpr int pt_eb(int j) { return j == 0 ? 1 : j == 1 ? 2 : j == 2 ? 2 : 3; }

// P2 basis of a tetrahedron at barycentric coordinates l[0..3]
template <typename R>
__host__ __device__ __forceinline__ void pt_basis(const R (&l)[4], R (&phi)[PT_NN]) {
#pragma unroll
  for (int a = 0; a < 4; a++) phi[a] = l[a] * ((R)2 * l[a] - (R)1);
#pragma unroll
  for (int j = 0; j < 6; j++) phi[4 + j] = (R)4 * l[pt_ea(j)] * l[pt_eb(j)];
}

// Block tables: tPhi[a][q] = phi_a(y_q), tW[q] (FP64); rB[q][v], rW[q], rWP[a][q] in R.
template <typename R>
__host__ __device__ constexpr size_t pt_table_bytes() {
  return (sizeof(double) * (PT_NH + 16) + sizeof(R) * (PT_NQ * 4 + 16 + PT_NH) + 15) & ~size_t(15);
}

template <typename R>
struct PTMem {
  R* sv;         // [scap][16]: 4 vertices x (x, y, z, pad)
  uint32_t* sc;  // [scap]
  R* iv;         // [IMAX][16]: item vertices (frame of y), padded
  R* iw;         // [IMAX]: C |E'|
  int* ik;       // [IMAX]: 1 = FINAL
  R* red;        // [NH][RS]
  R* hs;         // [NH + 10]
  double* sd;    // [16]
  static __host__ __device__ size_t bytes(int scap) {
    size_t b = sizeof(R) * 16 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * (size_t)PT_IMAX * 17 + sizeof(int) * PT_IMAX;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * ((size_t)PT_NH * PT_RS + PT_NH + 10);
    b = (b + 15) & ~size_t(15);
    b += sizeof(double) * 16;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    sv = reinterpret_cast<R*>(base);
    sc = reinterpret_cast<uint32_t*>(sv + 16 * (size_t)scap);
    size_t off = sizeof(R) * 16 * (size_t)scap + sizeof(uint32_t) * (size_t)scap;
    off = (off + 15) & ~size_t(15);
    iv = reinterpret_cast<R*>(base + off);
    iw = iv + (size_t)PT_IMAX * 16;
    ik = reinterpret_cast<int*>(iw + PT_IMAX);
    off += sizeof(R) * (size_t)PT_IMAX * 17 + sizeof(int) * PT_IMAX;
    off = (off + 15) & ~size_t(15);
    red = reinterpret_cast<R*>(base + off);
    hs = red + (size_t)PT_NH * PT_RS;
    off += sizeof(R) * ((size_t)PT_NH * PT_RS + PT_NH + 10);
    off = (off + 15) & ~size_t(15);
    sd = reinterpret_cast<double*>(base + off);
  }
};

template <typename R, int KERN>
__global__ void __launch_bounds__(PT_WARPS * 32, std::is_same<R, float>::value ? 2 : 1)
    k_quad_p2t(const QParams P) {
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) char smem_raw[];
  double* tPhi = reinterpret_cast<double*>(smem_raw);  // [NN][NQ]
  double* tW = tPhi + PT_NH;                            // [16]
  R* rB = reinterpret_cast<R*>(tW + 16);                // [NQ][4]
  R* rW = rB + PT_NQ * 4;                               // [16]
  R* rWP = rW + 16;                                     // [NN][NQ]
  for (int q = threadIdx.x; q < PT_NQ; q += blockDim.x) {
    double lam[4], phi[PT_NN];
    for (int a = 0; a < 4; a++) lam[a] = P.B[q][a];
    pt_basis<double>(lam, phi);
    for (int a = 0; a < PT_NN; a++) {
      tPhi[a * PT_NQ + q] = phi[a];
      rWP[a * PT_NQ + q] = (R)(P.W[q] * phi[a]);
    }
    tW[q] = P.W[q];
    rW[q] = (R)P.W[q];
    for (int a = 0; a < 4; a++) rB[q * 4 + a] = (R)P.B[q][a];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ybase = lane >= 16 ? PT_NYL : 0;
  const int xl = lane & 15;
  PTMem<R> wm;
  wm.carve(smem_raw + pt_table_bytes<R>() + (size_t)wid * PTMem<R>::bytes(P.scap), P.scap);

  unsigned st_items = 0, st_exact = 0, st_eval = 0, st_closed = 0, st_band = 0;
  int err = 0;
  int64_t cur_m = -1;
  double v0m[3] = {0.0, 0.0, 0.0}, mlo[3] = {0.0, 0.0, 0.0}, mhi[3] = {0.0, 0.0, 0.0}, vol_md = 0.0;
  float v0h[3] = {0.f, 0.f, 0.f}, v0l[3] = {0.f, 0.f, 0.f}, flo[3] = {0.f, 0.f, 0.f};
  float fhi[3] = {0.f, 0.f, 0.f};
  R y[PT_NYL][3];
  R vol_m = 0;
  R gsh = 0, gsl = 0;

  auto flush_self = [&]() {
    if (lane < PT_NQ) wm.sd[lane] = (double)gsh + (double)gsl;
    gsh = gsl = 0;
    __syncwarp();
    for (int e = lane; e < PT_NBLK; e += 32) {
      const int a = e / PT_NN, b = e % PT_NN;
      double s = 0.0;
      for (int q = 0; q < PT_NQ; q++) s += tW[q] * tPhi[a * PT_NQ + q] * tPhi[b * PT_NQ + q] * wm.sd[q];
      atomicAdd(&P.selfblk[cur_m * PT_NBLK + e], 2.0 * vol_md * s);
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
        double Vm[4][3];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 3; k++) Vm[a][k] = P.evert[(m * 4 + a) * 3 + k];
#pragma unroll
        for (int k = 0; k < 3; k++) {
          v0m[k] = Vm[0][k];
          mlo[k] = P.blo[m * 3 + k];
          mhi[k] = P.bhi[m * 3 + k];
        }
        vol_md = P.vol[m];
        vol_m = (R)vol_md;
#pragma unroll
        for (int i = 0; i < PT_NYL; i++) {
          const int q = ybase + i;
#pragma unroll
          for (int k = 0; k < 3; k++) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < 4; a++) s += P.B[q][a] * (Vm[a][k] - v0m[k]);
            y[i][k] = (R)s;
          }
        }
        if constexpr (F32) {
          const float* ef = P.ef + m * NL_EF_STRIDE(3);
#pragma unroll
          for (int k = 0; k < 3; k++) {
            v0h[k] = ef[NL_EF_V0HI(3) + k];
            v0l[k] = ef[NL_EF_V0LO(3) + k];
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int a = 1; a < 4; a++) {
              const float v = ef[(a - 1) * 3 + k];
              lo = v < lo ? v : lo;
              hi = v > hi ? v : hi;
            }
            flo[k] = lo;
            fhi[k] = hi;
          }
        }
      }
      const int32_t l = P.pair_l[p];
      // E_l: R = float in the local FP32 frame, R = double in global FP64 coordinates; Vl0
      // and the inverse Jacobian in the frame of y
      R Vl[4][3], Vl0[3], JI[3][3], wl;
      if constexpr (F32) {
        const float* ef = P.ef + (int64_t)l * NL_EF_STRIDE(3);
#pragma unroll
        for (int k = 0; k < 3; k++) Vl0[k] = (ef[NL_EF_V0HI(3) + k] - v0h[k]) + (ef[NL_EF_V0LO(3) + k] - v0l[k]);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          Vl[0][k] = Vl0[k];
#pragma unroll
          for (int a = 1; a < 4; a++) Vl[a][k] = Vl0[k] + ef[(a - 1) * 3 + k];
        }
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
          for (int c = 0; c < 3; c++) JI[r][c] = ef[9 + r * 3 + c];
        wl = P.fC * ef[18];
      } else {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int k = 0; k < 3; k++) Vl[a][k] = P.evert[((int64_t)l * 4 + a) * 3 + k];
#pragma unroll
        for (int k = 0; k < 3; k++) Vl0[k] = Vl[0][k] - v0m[k];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
          for (int c = 0; c < 3; c++) JI[r][c] = P.jinv[((int64_t)l * 3 + r) * 3 + c];
        wl = P.C * P.vol[l];
      }
      R H[PT_NN][PT_NYL];
#pragma unroll
      for (int d = 0; d < PT_NN; d++)
#pragma unroll
        for (int i = 0; i < PT_NYL; i++) H[d][i] = 0;
      R U[PT_NN];
#pragma unroll
      for (int d = 0; d < PT_NN; d++) U[d] = 0;
      bool contrib = false, has_u = false;

      auto classify = [&](const R (&V)[4][3], uint32_t code, bool count_exact) -> int {
        const int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        const bool last = level == P.L_max;
        const bool l2 = P.mindist_l2 != 0;
        if constexpr (F32) {
          float fam, fan, fe2;
          screen_dists<3>(V, flo, fhi, fam, fan, fe2);
          const bool c_int = fam < P.fint2;
          const bool c_notint = fam > P.fnotint2;
          const bool c_ref = l2 ? fe2 < P.fref2 : fan < P.fdpe - P.margin;
          const bool c_out = l2 ? fe2 > P.fout2 : fan > P.fdpe + P.margin;
          if (last) return c_int ? ACT_INT : (c_out ? ACT_ZERO : ACT_FINAL);
          if (c_int) return ACT_INT;
          if (c_notint && c_ref) return ACT_REFINE;
          if (c_notint && c_out) return ACT_DROP;
          st_exact += count_exact ? 1 : 0;
          return exact_classify<3>(P.evert + (int64_t)l * 12, P.blo + cur_m * 3, P.bhi + cur_m * 3,
                                   code, P.dme, P.dpe, l2);
        } else {
          double amax, amin;
          exact_dists<3>(V, mlo, mhi, amax, amin, l2);
          if (last) return amax < P.dme ? ACT_INT : (amin > P.dpe ? ACT_ZERO : ACT_FINAL);
          if (amax < P.dme) return ACT_INT;
          if (amin < P.dpe) return ACT_REFINE;
          return ACT_DROP;
        }
      };
      // the outer point with rule point q of the sub-element with vertices V (frame of y):
      // position, weight factor and the P2 basis of l there
      auto outer_point = [&](const R* V, int q, R (&x)[3], R (&phi)[PT_NN]) {
#pragma unroll
        for (int k = 0; k < 3; k++)
          x[k] = rB[q * 4] * V[k] + rB[q * 4 + 1] * V[4 + k] + rB[q * 4 + 2] * V[8 + k] + rB[q * 4 + 3] * V[12 + k];
        R lam[4];
        const R d0 = x[0] - Vl0[0], d1 = x[1] - Vl0[1], d2 = x[2] - Vl0[2];
#pragma unroll
        for (int r = 0; r < 3; r++) lam[r + 1] = JI[r][0] * d0 + JI[r][1] * d1 + JI[r][2] * d2;
        lam[0] = (R)1 - lam[1] - lam[2] - lam[3];
        pt_basis<R>(lam, phi);
      };
      // the sub-element's vertices in the frame of y, padded (x, y, z, 0) per vertex
      auto frame = [&](const R (&V)[4][3], R* out) {
#pragma unroll
        for (int a = 0; a < 4; a++) {
#pragma unroll
          for (int k = 0; k < 3; k++) out[a * 4 + k] = F32 ? V[a][k] : (R)(V[a][k] - v0m[k]);
          out[a * 4 + 3] = 0;
        }
      };
      // closed form of an INT sub-element (constant kernel): sum_x w_x C phi^l_d(x), the same
      // at every inner point
      auto closed_int = [&](const R (&V)[4][3], int level) {
        R Vf[16];
        frame(V, Vf);
        const R wv = wl * pow2m(R(0), 3 * (level - 1));
#pragma unroll 1
        for (int q = 0; q < PT_NQ; q++) {  // not unrolled: rare, keeps the code small
          R x[3], phi[PT_NN];
          outer_point(Vf, q, x, phi);
#pragma unroll
          for (int d = 0; d < PT_NN; d++) U[d] += rW[q] * wv * phi[d];
        }
        has_u = true;
        st_closed++;
        contrib = true;
      };
      auto put_item = [&](int slot, const R (&V)[4][3], int level, int fin) {
        frame(V, wm.iv + slot * 16);
        wm.iw[slot] = wl * pow2m(R(0), 3 * (level - 1));
        wm.ik[slot] = fin;
      };
      auto push = [&](int slot, const R (&V)[4][3], uint32_t code) {
        R* r = wm.sv + slot * 16;
#pragma unroll
        for (int a = 0; a < 4; a++) {
#pragma unroll
          for (int k = 0; k < 3; k++) r[a * 4 + k] = V[a][k];
          r[a * 4 + 3] = 0;
        }
        wm.sc[slot] = code;
      };
      auto integrate = [&](int n_it) {
        const int n_x = n_it * PT_NQ;
        st_eval += (unsigned)(n_x * PT_NQ);
        contrib = true;
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        for (int base = 0; base < n_x; base += PT_XPI) {
          const int o = base + xl;
          const bool valid = o < n_x;
          const int it = valid ? o / PT_NQ : 0;
          const int q = valid ? o - it * PT_NQ : 0;
          const bool fin = wm.ik[it] != 0;
          R x[3], phi[PT_NN];
          outer_point(wm.iv + it * 16, q, x, phi);
          const R wx = valid ? rW[q] * wm.iw[it] : (R)0;
          R bw[PT_NN];
#pragma unroll
          for (int d = 0; d < PT_NN; d++) bw[d] = wx * phi[d];
#pragma unroll
          for (int i = 0; i < PT_NYL; i++) {
            const R e0 = x[0] - y[i][0], e1 = x[1] - y[i][1], e2 = x[2] - y[i][2];
            const R r2 = e0 * e0 + e1 * e1 + e2 * e2;
            R g = 1;
            if constexpr (F32) {
              const float mu = mollifier_bf(MK, r2);
              g = fin ? mu : 1.f;
              if (P.count_band) st_band += (valid && fin && r2 >= P.fdme2 && r2 <= P.fdpe2) ? 1 : 0;
            } else {
              if (fin) g = mollifier(P, r2);
              if (P.count_band)
                st_band += (valid && fin && r2 >= P.dme * P.dme && r2 <= P.dpe * P.dpe) ? 1 : 0;
            }
            if (KERN == NL_KERNEL_TRUNC_GAUSS) g *= eta_gauss<R>(P, r2);
#pragma unroll
            for (int d = 0; d < PT_NN; d++) H[d][i] += g * bw[d];
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
          if (lane == 0) closed_int(Vl, 1);
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
          if (n_it > PT_IMAX - 32) {
            integrate(n_it);
            n_it = 0;
          }
          const int np = min(4, sp);
          const int base = sp - np;
          const int par = lane >> 3, c = lane & 7;
          const bool active = par < np;
          R V[4][3];
          uint32_t code = 0;
          if (active) {
            const R* pv = wm.sv + (base + par) * 16;
            const uint32_t pcode = wm.sc[base + par];
            const int plevel = pcode >> LEVEL_SHIFT;
            code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) | (pcode & ((1u << LEVEL_SHIFT) - 1)) |
                   ((uint32_t)c << (3 * (plevel - 1)));
#pragma unroll
            for (int v = 0; v < 4; v++) {
              int ia, ib;
              mid_pair<3>(c, v, ia, ib);
#pragma unroll
              for (int k = 0; k < 3; k++) V[v][k] = midp(pv[ia * 4 + k], pv[ib * 4 + k]);
            }
          }
          __syncwarp();  // parents are read before children overwrite their slots
          int act = active ? classify(V, code, true) : ACT_DROP;
          const int level = code >> LEVEL_SHIFT;
          if (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO) st_items++;
          if (KERN == NL_KERNEL_CONST && act == ACT_INT) {
            closed_int(V, level);
            act = ACT_DROP;
          }
          const unsigned m_it = __ballot_sync(FULL, act == ACT_INT || act == ACT_FINAL);
          const unsigned m_ref = __ballot_sync(FULL, act == ACT_REFINE);
          const unsigned below = (1u << lane) - 1u;
          if (act == ACT_INT || act == ACT_FINAL)
            put_item(n_it + __popc(m_it & below), V, level, act == ACT_FINAL);
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

      // ---- end of pair ---------------------------------------------------------------------
      R* bp = reinterpret_cast<R*>(P.blk) + (p - P.p_begin) * PT_NBLK;
      if (!__any_sync(FULL, contrib)) {
        for (int e = lane; e < PT_NBLK; e += 32) bp[e] = (R)0;
        __syncwarp();
        continue;
      }
      if (__any_sync(FULL, has_u)) {
#pragma unroll
        for (int d = 0; d < PT_NN; d++)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) U[d] += __shfl_xor_sync(FULL, U[d], o);
      }
#pragma unroll
      for (int d = 0; d < PT_NN; d++)
#pragma unroll
        for (int i = 0; i < PT_NYL; i++) wm.red[(d * PT_NQ + ybase + i) * PT_RS + xl] = H[d][i];
      __syncwarp();
      for (int j = lane; j < PT_NH; j += 32) {
        R s = 0;
#pragma unroll
        for (int t = 0; t < PT_XPI; t++) s += wm.red[j * PT_RS + t];
        wm.hs[j] = s + U[j / PT_NQ];
      }
      __syncwarp();
      for (int e = lane; e < PT_NBLK; e += 32) {
        const int a = e / PT_NN, d = e % PT_NN;
        R s = 0;
#pragma unroll
        for (int q = 0; q < PT_NQ; q++) s += rWP[a * PT_NQ + q] * wm.hs[d * PT_NQ + q];
        bp[e] = (R)(-2) * vol_m * s;
      }
      if (lane < PT_NQ) {
        R g = 0;
#pragma unroll
        for (int d = 0; d < PT_NN; d++) g += wm.hs[d * PT_NQ + lane];
        two_sum_add(gsh, gsl, g);
      }
      __syncwarp();  // the scratch is read before the next pair writes it
    }
    flush_stats();
  }
  if (cur_m >= 0) flush_self();
}

template <typename R, int KERN>
nl_status launch_quad_p2t(const QParams& P, cudaStream_t s) {
  int dev = 0, nsm = 0;
  NL_CUDA(cudaGetDevice(&dev));
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t per_warp = PTMem<R>::bytes(P.scap);
  int warps = PT_WARPS;
  while (warps > 1 && pt_table_bytes<R>() + warps * per_warp > (size_t)200 * 1024) warps >>= 1;
  const size_t smem = pt_table_bytes<R>() + warps * per_warp;
  if (smem > (size_t)220 * 1024)
    return fail(NL_EINTERNAL, "P2 tetrahedron assembly kernel needs %zu bytes of shared memory", smem);
  auto kern = k_quad_p2t<R, KERN>;
  NL_TRY(allow_smem(kern, smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "P2 tetrahedron assembly kernel does not fit on an SM (smem %zu)", smem);
  kern<<<NL_CNT(nsm * per_sm), warps * 32, smem, s>>>(P);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

template <typename R, int KERN>
nl_status run_assembly_p2t(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s,
                           unsigned long long* scratch, int* err, PhaseTimer& T) {
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
  if (g_block_budget) budget = std::min(budget, g_block_budget);
  int64_t batch = std::max<int64_t>(1 << 20, (int64_t)(budget / (sizeof(R) * PT_NBLK)));
  batch = std::min<int64_t>(batch, p->n_pairs);
  DevBuf<R> blk;
  DevBuf<double> selfblk;
  NL_TRY(blk.alloc((size_t)batch * PT_NBLK, s));
  NL_TRY(selfblk.alloc((size_t)m->n_elem * PT_NBLK, s));
  NL_CUDA(cudaMemsetAsync(selfblk.p, 0, sizeof(double) * m->n_elem * PT_NBLK, s));
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
    NL_TRY((launch_quad_p2t<R, KERN>(P, s)));
    NL_TRY(T.mark(0, s));
    NL_TRY(T.mark(1, s));
    NL_TRY((launch_scatter<3, R, PT_NN>(m, p, b0, b1, blk.p, nullptr, 0, values, err, s, h_off.data())));
    NL_TRY(T.mark(1, s));
  }
  NL_TRY(T.mark(1, s));
  NL_TRY((launch_scatter<3, R, PT_NN>(m, p, 0, 0, blk.p, selfblk.p, 1, values, err, s, h_off.data())));
  NL_TRY(T.mark(1, s));
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}

}  // namespace

nl_status assemble_values_p2t(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                              const nl_quad_params* qp, nl_precision prec, double* values,
                              nl_assemble_stats* st) {
  if (m->dim != 3 || m->nb != PT_NN) return fail(NL_EINVAL, "nl_assemble: not a mesh of P2 tetrahedra");
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
    if (f32) rc = gauss ? run_assembly_p2t<float, 1>(m, p, P, values, s, scratch.p, err.p, T)
                        : run_assembly_p2t<float, 0>(m, p, P, values, s, scratch.p, err.p, T);
    else rc = gauss ? run_assembly_p2t<double, 1>(m, p, P, values, s, scratch.p, err.p, T)
                    : run_assembly_p2t<double, 0>(m, p, P, values, s, scratch.p, err.p, T);
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
    st->n_point_pairs = (int64_t)hs[1] * PT_NQ * PT_NQ;
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
