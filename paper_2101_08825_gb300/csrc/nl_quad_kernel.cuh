// nl_quad_kernel.cuh -- the assembly kernels, shared by the single-problem and batched paths.
//
// What is computed (Sec. 5, Corollary 1, eqs. J21Nr and J22Nr): for every element pair
// (m, l) of J, with the inner degree-5 rule on E_m (points y, weights w_y, rows = nodes of m)
// and the outer rule on the sub-elements E' of E_l that Algorithm 1 selects for this m,
//   A[m_a, m_b] += 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^m_b(y)
//   A[m_a, l_c] -= 2 sum_{x,y} w_x w_y gamma_eps(x,y) phi^m_a(y) phi^l_c(x).
// Algorithm 1 is applied per pair; this is the same computation as the per-l recursion with
// the index set J_l, because the tests and the integration act on every m separately.
//
// How (k_quad): a persistent grid; each warp takes chunks of consecutive pairs (m-major)
// from a global counter.  For one pair the warp runs Algorithm 1 as a LIFO of refined
// sub-elements ("parent records": vertices + path code) in shared memory: each round pops
// up to 32/2^N parents and every lane builds one child by midpoints, classifies it with the
// box distances of Sec. 5.1 and drops it, pushes it, or appends it to one of two item
// buffers: INT (max-dist < delta-eps: mu = 1 at every point pair) or FINAL (the sub-element
// reached L_max with the band in reach).  With the constant kernel an INT sub-element is
// summed in closed form (the degree-5 rule integrates its linear integrand exactly).  A full
// buffer is integrated by the whole warp: each lane owns one outer point x and 7 inner points
// y kept in registers (3D: two half-warps share x and take y 0-6 and 7-13), and accumulates
// per y the sums g = sum_x w_x C eta mu and h_k = sum_x w_x C eta mu lambda^l_k(x).  At the
// end of the pair every lane contracts its own inner points into the pair's cross block
// -2 vol_m sum_y w_y B_a(y) H_c(y) (H_0 = g - sum_k h_k, H_c = h_{c-1}) and its g per inner
// point, and one warp reduce-scatter (shuffles; 16 values in 2D, 32 in 3D) leaves each entry
// summed on one lane; the cross block goes to a block buffer, and the self block, which only
// needs g, is accumulated over the consecutive pairs of the same m (compensated FP32 or FP64)
// and added to a per-element block.
// k_scatter (one CTA per inner element m, the rows of m's nodes cached in shared memory)
// then adds every block to the CSR values with FP64 atomics.
//
// Precision: R = double evaluates everything in FP64 on global coordinates and classifies
// in FP64.  R = float evaluates gamma_eps in FP32 on coordinates relative to the first
// vertex of m, built from per-element FP32 vertex offsets and one FP64 difference of first
// vertices per pair; the classification is screened in FP32, and a decision whose FP32
// distance lies within a proven margin of its threshold is redone in FP64 on vertices
// rebuilt from E_l by the same midpoint sequence, so the decisions are those of a plain FP64
// evaluation.
//
// Included by exactly the translation units that launch these kernels; everything here has
// internal linkage, so each of them gets its own instantiations.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "nl_internal.h"

namespace nlx {
namespace {

constexpr int KIND_INT = 0;
constexpr int KIND_FINAL = 1;
// ACT_ZERO: a sub-element at L_max that Algorithm 1 integrates but whose every point pair is
// farther than delta + eps (mu = 0): counted, not evaluated.
constexpr int ACT_DROP = 0, ACT_INT = 1, ACT_FINAL = 2, ACT_REFINE = 3, ACT_ZERO = 4;
constexpr int ERR_STACK = 1, ERR_CSR = 2;
constexpr int CHUNK = 32;  // default pairs per grab of the work counter
constexpr int IMAX = 64;
constexpr int LEVEL_SHIFT = 27;

struct QParams {
  int64_t n_elem, p_begin, p_end;
  const int64_t* pair_off;
  const int32_t* pair_l;
  const int32_t* conn;
  const double* evert;
  const double* blo;
  const double* bhi;
  const double* vol;
  const double* jinv;
  const float* ef;
  void* blk;          // [p_end - p_begin][(D+1)^2] cross blocks (R)
  double* selfblk;    // [n_elem][(D+1)^2]
  const int64_t* row_ptr;  // CSR pattern and values: used only by the variant that adds
  const int32_t* col;      // its cross blocks to the values directly
  double* values;
  unsigned long long* counter;
  unsigned long long* stats;  // [0] items, [2] exact checks, [3] evaluated pairs,
                              // [4] closed-form items, [5] band pairs
  int* err;
  double delta, dme, dpe, C, inv_eps, inv_delta2;
  float fdme2, fdpe2, finv_delta2, margin, fdme, fdpe, fC;
  float fmqe, ftqe, fue;     // -1/(4 eps), 3/(4 eps), (1 - delta/eps)/2 (branch-free mollifier)
  float fint2, fnotint2;     // screen thresholds (delta - eps -+ margin)^2 (-1: never)
  float fref2, fout2;        // mindist_l2: (delta + eps -+ 2 margin)^2
  int L_min, L_max, scap, count_band;
  int mindist_l2;            // Algorithm 1's refinement test with the Euclidean minimum distance
  int kernel;  // nl_kernel_kind (read at run time by the batched kernel)
  int chunk;   // consecutive pairs a warp takes from the work counter
  double B[14][4];
  double W[14];
};

// Values per padded vertex in shared memory (see VPad)
__host__ __device__ constexpr int VPadN(int D) { return D == 2 ? 2 : 4; }

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
  static constexpr int NBLK = NV * NV;          // entries of a local block
  static constexpr int EFS = NL_EF_STRIDE(D);
};

// Child c, vertex v = midpoint of parent vertices (a, b); a corner is mid(P, P) = P exactly.
// Triangles: the three corner children, then the middle one.  Tetrahedra (Bey): the four
// corner children, then the four children of the octahedron cut along the x02-x13 diagonal.
// The tables are packed two bits per index into 64-bit constants, so that a lane-dependent
// child index is decoded in registers (a lookup in constant memory with a different address
// per lane would be serialised).
constexpr unsigned char k_mid2[4][3][2] = {{{0, 0}, {0, 1}, {0, 2}},
                                           {{0, 1}, {1, 1}, {1, 2}},
                                           {{0, 2}, {1, 2}, {2, 2}},
                                           {{0, 1}, {1, 2}, {0, 2}}};
constexpr unsigned char k_mid3[8][4][2] = {
    {{0, 0}, {0, 1}, {0, 2}, {0, 3}}, {{0, 1}, {1, 1}, {1, 2}, {1, 3}},
    {{0, 2}, {1, 2}, {2, 2}, {2, 3}}, {{0, 3}, {1, 3}, {2, 3}, {3, 3}},
    {{0, 1}, {0, 2}, {0, 3}, {1, 3}}, {{0, 1}, {0, 2}, {1, 2}, {1, 3}},
    {{0, 2}, {0, 3}, {1, 3}, {2, 3}}, {{0, 2}, {1, 2}, {1, 3}, {2, 3}}};

constexpr uint64_t pack_mid2() {
  uint64_t t = 0;
  for (int c = 0; c < 4; c++)
    for (int v = 0; v < 3; v++)
      for (int j = 0; j < 2; j++) t |= (uint64_t)k_mid2[c][v][j] << (2 * ((c * 3 + v) * 2 + j));
  return t;
}
constexpr uint64_t pack_mid3(int half) {
  uint64_t t = 0;
  for (int c = 0; c < 4; c++)
    for (int v = 0; v < 4; v++)
      for (int j = 0; j < 2; j++)
        t |= (uint64_t)k_mid3[4 * half + c][v][j] << (2 * ((c * 4 + v) * 2 + j));
  return t;
}
constexpr uint64_t MID2 = pack_mid2(), MID3A = pack_mid3(0), MID3B = pack_mid3(1);

template <int D>
__device__ __forceinline__ void mid_pair(int c, int v, int& a, int& b) {
  if (D == 2) {
    const int sh = 2 * ((c * 3 + v) * 2);
    a = (int)(MID2 >> sh) & 3;
    b = (int)(MID2 >> (sh + 2)) & 3;
  } else {
    const uint64_t t = c < 4 ? MID3A : MID3B;
    const int sh = 2 * (((c & 3) * 4 + v) * 2);
    a = (int)(t >> sh) & 3;
    b = (int)(t >> (sh + 2)) & 3;
  }
}

__device__ __forceinline__ double midp(double a, double b) { return __dmul_rn(__dadd_rn(a, b), 0.5); }
__device__ __forceinline__ float midp(float a, float b) { return __fmul_rn(__fadd_rn(a, b), 0.5f); }

// 2^-k as an exact power of two
__device__ __forceinline__ float pow2m(float, int k) { return __int_as_float((127 - k) << 23); }
__device__ __forceinline__ double pow2m(double, int k) {
  return __longlong_as_double((long long)(1023 - k) << 52);
}

// Exact FP64 box distances of Sec. 5.1 (eqs. maxdist, mindist) between a sub-element with
// vertices V and the box (lo2, hi2) of E_m, written as in a plain evaluation.
// With l2, amin is the Euclidean variant that Sec. 5.1 gives after eq. mindistin,
// sqrt(sum_k max(0, d1^k, d2^k)^2), in the same order of operations as a plain evaluation.
template <int D>
__device__ void exact_dists(const double (&V)[D + 1][D], const double* lo2, const double* hi2,
                            double& amax, double& amin, bool l2 = false) {
  double s = 0.0, mn = 0.0, e = 0.0;
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
    const double u = t < 0.0 ? 0.0 : t;
    e = __dadd_rn(e, __dmul_rn(u, u));
  }
  amax = __dsqrt_rn(s);
  amin = l2 ? __dsqrt_rn(e) : mn;
}

// FP32 screen of the same distances: amax is returned squared (no square root on the
// screening path), amin as is, and amin2 the square of the Euclidean variant.
template <int D>
__device__ __forceinline__ void screen_dists(const float (&V)[D + 1][D], const float* lo2,
                                             const float* hi2, float& amax, float& amin,
                                             float& amin2) {
  float s = 0.f, mn = 0.f, e = 0.f;
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
    const float t = fmaxf(d1, d2);
    mn = fmaxf(mn, t);
    const float u = fmaxf(t, 0.f);
    e = fmaf(u, u, e);
  }
  amax = s;  // squared: compared with squared thresholds
  amin = mn;
  amin2 = e;
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

// FP64 decision of Algorithm 1 for a sub-element below L_max (used by the FP32 path when the
// screened distance is within the margin of a threshold): ACT_INT, ACT_REFINE or ACT_DROP.
template <int D>
__device__ __noinline__ int exact_classify(const double* __restrict__ evert_l,
                                           const double* __restrict__ lo_m,
                                           const double* __restrict__ hi_m, uint32_t code,
                                           double dme, double dpe, bool l2) {
  double Vl[D + 1][D], V[D + 1][D], lo2[D], hi2[D];
#pragma unroll
  for (int a = 0; a <= D; a++)
#pragma unroll
    for (int k = 0; k < D; k++) Vl[a][k] = evert_l[a * D + k];
#pragma unroll
  for (int k = 0; k < D; k++) {
    lo2[k] = lo_m[k];
    hi2[k] = hi_m[k];
  }
  decode_exact<D>(Vl, code, V);
  double amax, amin;
  exact_dists<D>(V, lo2, hi2, amax, amin, l2);
  if (amax < dme) return ACT_INT;
  if (amin < dpe) return ACT_REFINE;
  return ACT_DROP;
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
  // coefficients divided by 256 (exact: a power of two)
  float t = s * s;
  float p = fmaf(35.f / 256.f, t, -180.f / 256.f);
  p = fmaf(p, t, 378.f / 256.f);
  p = fmaf(p, t, -420.f / 256.f);
  p = fmaf(p, t, 315.f / 256.f);
  return fmaf(s, p, 0.5f);
}

// mu_{delta,eps}(r) from r^2 (eq. mollifier with argument (delta - r)/eps)
__device__ __forceinline__ double mollifier(const QParams& P, double r2) {
  double dme2 = P.dme * P.dme, dpe2 = P.dpe * P.dpe;
  if (r2 < dme2) return 1.0;
  if (r2 > dpe2) return 0.0;
  double r = sqrt(r2);
  return xi_poly((P.delta - r) * P.inv_eps);
}

// ---- packed FP32 pairs (sm_100 family: add/sub/mul/fma .f32x2, one instruction for two
// lanes of work) for the point-pair loop of the FP32 path ----------------------------------
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2dup(float v) { return f2pack(v, v); }
__device__ __forceinline__ f2 f2add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Asynchronous 16-byte global-to-shared copies (cp.async), used to fetch the next pair's
// element record while the current pair is processed.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// ---- tensor-core pieces of the mixed paths (mma.sync, FP32 accumulation) ------------------
// TF32: a value x is carried as hi + lo, hi = x rounded to TF32 (10 stored mantissa bits) and lo
// = the remainder rounded to TF32: about 22 significant bits together.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
// D += A B, A 16x8 (row), B 8x8 (col), TF32 operands, FP32 accumulators
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// BF16 pairs: (x0, x1) packed with x0 in the low half (the lower matrix index), and the
// two-term split hi + lo of each value (about 16 significant bits together).
__device__ __forceinline__ uint32_t bf16x2(float x0, float x1) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  hi = bf16x2(x0, x1);
  lo = bf16x2(x0 - __uint_as_float(hi << 16), x1 - __uint_as_float(hi & 0xffff0000u));
}
// D += A B, A 16x16 (row), B 16x8 (col), BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// Per-warp staging of one batch of 32 outer points for the tensor-core integration: their
// coordinates (padded vertices) and the weighted P1 basis of E_l at them, split into two
// parts (TF32 or BF16), column-major with a row stride of MMA_BS floats (40: the lanes of one
// fragment load hit distinct banks).
constexpr int MMA_BS = 40;
template <int D>
__host__ __device__ constexpr size_t mma_stage_bytes(int mma) {
  return mma == 0 ? 0 : sizeof(float) * (32 * VPadN(D) + 2 * (D + 1) * MMA_BS);
}

// Hardware reciprocal square root (MUFU, about 2^-22 relative error), no denormal handling.
__device__ __forceinline__ float rsqrt_hw(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// mu_{delta,eps}(r) from r^2 without branches.  r = r2 q with q ~ 1/sqrt(r2) from the
// hardware, refined by one Newton step r' = r (3/2 - r q / 2) folded into the argument
// u = (1 - s)/2 of s = (delta - r')/eps:
//   u = (1 - delta/eps)/2 + r (3/(4 eps) - r q/(4 eps)),
// two FMAs from r and q/(4 eps), the second saturating u to [0, 1] (s to [-1, 1], where xi
// is exactly 1 and 0: xi(+-1) = 1/2 +- 128/256 in FP32), so every point pair takes the same
// path.  r2 = 0 (coinciding points of a self pair) gives q = +inf and r = 0 * inf = NaN, which
// the saturation turns into u = 0: s = 1 and mu = 1, the value at r = 0.
// Constants of the branch-free mollifier, read once per buffer integration (in the batched
// kernel the parameters live in shared memory).
struct MollK {
  float mqe, tqe, ue;  // -1/(4 eps), 3/(4 eps), (1 - delta/eps)/2
};
__device__ __forceinline__ float mollifier_bf(const MollK& K, float r2) {
  const float q = rsqrt_hw(r2);
  const float r = r2 * q;
  const float b = fmaf(r, q * K.mqe, K.tqe);
  float u;
  asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(u) : "f"(r), "f"(b), "f"(K.ue));
  return xi_poly(fmaf(-2.f, u, 1.f));
}
// The two point pairs of a packed r2 in scalar FP32: scalar FMAs take the constants as
// immediate or constant-bank operands, while every packed constant needs a register pair.
__device__ __forceinline__ f2 mollifier2(const MollK& K, f2 r2) {
  float a, b;
  f2unpack(r2, a, b);
  return f2pack(mollifier_bf(K, a), mollifier_bf(K, b));
}
__device__ __forceinline__ f2 eta_gauss2(float inv_delta2, f2 r2) {
  float a, b;
  f2unpack(r2, a, b);
  return f2pack(__expf(-a * inv_delta2), __expf(-b * inv_delta2));
}

// Sum_j A_ij = 0 for every row of the exact discrete operator (sum_j phi_j = 1 at every
// point, so every point pair contributes sum_j (phi_j(y) - phi_j(x)) = 0): the diagonal
// equals minus the sum of the off-diagonal entries.  The FP32 paths rebuild it that way in
// FP64, which removes the row-sum part of their rounding error (warp per row).
__global__ void k_diag_from_rows(int64_t n_rows, const int64_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col, double* __restrict__ values) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_rows) return;
  double s = 0.0;
  int64_t dpos = -1;
  for (int64_t t = row_ptr[i] + lane; t < row_ptr[i + 1]; t += 32) {
    if (col[t] == (int32_t)i) dpos = t;
    else s += values[t];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    int64_t d = __shfl_xor_sync(0xffffffffu, dpos, o);
    dpos = d > dpos ? d : dpos;
  }
  if (lane == 0 && dpos >= 0) values[dpos] = -s;
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

// Compensated accumulation (hi + lo) in the working precision (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  float s = hi + v;
  float bb = s - hi;
  float e = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += e;
}
__device__ __forceinline__ void two_sum_add(double& hi, double& lo, double v) {
  hi += v;
  (void)lo;
}

// A vertex in shared memory: D coordinates padded to 2 (2D) or 4 (3D) values, so that it is
// read and written with one vector access (float2/float4; double2 or two double2).
template <int D>
struct VPad {
  static constexpr int N = D == 2 ? 2 : 4;
};
template <int D, typename R>
__device__ __forceinline__ void vload(const R* __restrict__ p, R (&v)[D]) {
  if constexpr (std::is_same<R, float>::value) {
    if constexpr (D == 2) {
      const float2 t = *reinterpret_cast<const float2*>(p);
      v[0] = t.x;
      v[1] = t.y;
    } else {
      const float4 t = *reinterpret_cast<const float4*>(p);
      v[0] = t.x;
      v[1] = t.y;
      v[2] = t.z;
    }
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x;
    v[1] = t.y;
    if constexpr (D == 3) v[2] = p[2];
  }
}
template <int D, typename R>
__device__ __forceinline__ void vstore(R* __restrict__ p, const R (&v)[D]) {
  if constexpr (std::is_same<R, float>::value) {
    if constexpr (D == 2) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    else *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], 0.f);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    if constexpr (D == 3) p[2] = v[2];
  }
}

// Per-warp shared memory: stack records, two item buffers and a small scratch.  Vertices are
// stored padded (VPad) so that one vector access moves a vertex.
template <int D, typename R>
struct WarpMem {
  R* rv;          // [NV][scap][PAD] stacked sub-element vertices
  uint32_t* rc;   // [scap] path codes
  R* iv;          // [2][NV][IMAX][PAD] buffered items (INT, FINAL)
  R* iw;          // [2][IMAX]
  R* red;         // 16 doubles of scratch (self-block sums)
  float* pf;      // [2][32]: FP32 element records of the current and the next pair
  R* pc;          // [8]: box of the current inner element m (lo, hi)
  static __host__ __device__ size_t bytes(int scap) {
    using G = Geo<D>;
    constexpr int PAD = VPad<D>::N;
    size_t b = sizeof(R) * (size_t)G::NV * PAD * scap + sizeof(uint32_t) * scap;
    b = (b + 15) & ~size_t(15);
    b += sizeof(R) * ((size_t)2 * G::NV * IMAX * PAD + 2 * IMAX) + sizeof(double) * 16 + sizeof(float) * 64 +
         sizeof(R) * 8;
    b += 16;
    return (b + 15) & ~size_t(15);
  }
  __device__ void carve(char* base, int scap) {
    using G = Geo<D>;
    constexpr int PAD = VPad<D>::N;
    rv = reinterpret_cast<R*>(base);
    rc = reinterpret_cast<uint32_t*>(rv + (size_t)G::NV * PAD * scap);
    size_t off = sizeof(R) * (size_t)G::NV * PAD * scap + sizeof(uint32_t) * scap;
    off = (off + 15) & ~size_t(15);
    iv = reinterpret_cast<R*>(base + off);
    iw = iv + (size_t)2 * G::NV * IMAX * PAD;
    red = iw + 2 * IMAX;  // 16-byte aligned: iv and iw hold multiples of 16 bytes
    pf = reinterpret_cast<float*>(reinterpret_cast<char*>(red) + sizeof(double) * 16);
    pc = reinterpret_cast<R*>(pf + 64);
  }
};

template <typename R>
__host__ __device__ constexpr size_t table_bytes() {
  return (sizeof(R) * (14 * 4 * 2 + 16 + 4) + 15) & ~size_t(15);
}

// Position of column j in CSR row i (binary search in global memory), or -1.
__device__ __forceinline__ int64_t csr_find(const int64_t* __restrict__ row_ptr,
                                            const int32_t* __restrict__ col, int32_t i, int32_t j) {
  int64_t lo = row_ptr[i], hi = row_ptr[i + 1] - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int32_t c = col[mid];
    if (c == j) return mid;
    if (c < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// Problems of one batched launch: problem k owns the global pair indices
// [prefix[k], prefix[k+1]) of a concatenated index space.
struct QBatch {
  const QParams* probs;
  const int64_t* prefix;
  int n;
  int64_t total;
};

// DIRECT = true: the cross block of every pair is added to the CSR values at once (global
// binary search, FP64 atomics) instead of going through the block buffer.
// BATCHED = true: the launch covers the problems of Bt (same dimension and precision; the
// kernel profile may differ when KERN = 2); each warp copies the parameters of the problem it
// works on into shared memory and reads them from there.
// Launch shape per dimension (measured on GB300): 2D 8 warps x 2 CTAs (128 registers), 3D 4
// warps x 3 CTAs (up to 168 registers: the 3D state spills at 128).
template <int D>
struct QLaunch {
  static constexpr int THREADS = D == 2 ? 256 : 128;
  static constexpr int MIN_CTAS = D == 2 ? 2 : 3;
};

// MMA = 1 (TF32) or 2 (BF16), R = float only: the per-pair contraction over the outer points
// runs on the tensor cores (see integrate).
template <int D, typename R, int KERN, bool DIRECT = false, bool BATCHED = false, int MMA = 0>
__global__ void __launch_bounds__(QLaunch<D>::THREADS, QLaunch<D>::MIN_CTAS)
    k_quad(const QParams P0, const QBatch Bt) {
  using G = Geo<D>;
  constexpr int NV = G::NV, NQ = G::NQ, NYL = G::NYL, NVC = G::NVC, NBLK = G::NBLK;
  constexpr bool F32 = std::is_same<R, float>::value;
  extern __shared__ __align__(16) char smem_raw[];
  R* sB = reinterpret_cast<R*>(smem_raw);  // [NQ][NV]
  R* sW = sB + 14 * 4;                      // [NQ]
  R* sWB = sW + 16;                         // [NQ][NV]: W[q] * B[q][a]
  for (int t = threadIdx.x; t < NQ * NV; t += blockDim.x) {
    sB[t] = (R)P0.B[t / NV][t % NV];
    sWB[t] = (R)(P0.W[t / NV] * P0.B[t / NV][t % NV]);
  }
  for (int t = threadIdx.x; t < NQ; t += blockDim.x) sW[t] = (R)P0.W[t];
  R* sWBs = sWB + 14 * 4;  // [NV]: sum_q W[q] B[q][a] (the weight of a uniform contribution)
  if (threadIdx.x < NV) {
    double sacc = 0.0;
    for (int q = 0; q < NQ; q++) sacc += P0.W[q] * P0.B[q][threadIdx.x];
    sWBs[threadIdx.x] = (R)sacc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpMem<D, R> wm;
  wm.carve(smem_raw + table_bytes<R>() + (size_t)wid * WarpMem<D, R>::bytes(P0.scap), P0.scap);
  QParams* qcopy = reinterpret_cast<QParams*>(
      smem_raw + table_bytes<R>() + (size_t)(blockDim.x >> 5) * WarpMem<D, R>::bytes(P0.scap) +
      (size_t)wid * ((sizeof(QParams) + 15) & ~size_t(15)));
  const QParams& P = BATCHED ? *qcopy : P0;
  static_assert(MMA == 0 || (std::is_same<R, float>::value && !BATCHED), "tensor-core variants: FP32, single problem");
  float* mstage = reinterpret_cast<float*>(
      smem_raw + table_bytes<R>() + (size_t)(blockDim.x >> 5) * WarpMem<D, R>::bytes(P0.scap) +
      (size_t)wid * mma_stage_bytes<D>(MMA));
  auto is_const = [&]() { return KERN == 2 ? P.kernel == NL_KERNEL_CONST : KERN == NL_KERNEL_CONST; };
  auto is_gauss = [&]() {
    return KERN == 2 ? P.kernel == NL_KERNEL_TRUNC_GAUSS : KERN == NL_KERNEL_TRUNC_GAUSS;
  };

  const int ybase = (D == 3 && lane >= 16) ? 7 : 0;
  const int xl = (D == 3) ? (lane & 15) : lane;

  // per-lane work counters of the current chunk (32-bit: flushed at every chunk's end)
  unsigned st_items = 0, st_exact = 0, st_eval = 0, st_closed = 0, st_band = 0;
  int err = 0;

  // state of the current inner element m
  int64_t cur_m = -1;
  float v0h[D], v0l[D];  // R = float: first vertex of m (origin of the local coordinates), hi + lo

  R y[NYL][D];        // inner points of m (local if R = float)
  f2 yq[3][D];        // R = float: inner points 0-5 of the lane packed in pairs
  // MMA: the inner points of this thread's fragment rows, q = lane/4 (+ 8 in 3D); rows past
  // the rule's points are padding
  constexpr int MROWS = D == 2 ? 1 : 2;
  float ym[MROWS][D];
  R vol_m = 0;
  // The end-of-pair reduce-scatter leaves entry e_rs of NRS values on this lane: the cross
  // block (e < NBLK) and the sums of g at the inner points (NBLK <= e < NBLK + NQ); a lane that
  // holds a g entry keeps its compensated sum over the pairs of the current m-run
  constexpr int NRS = D == 2 ? 16 : 32;
  const int e_rs = NRS == 16 ? (lane >> 1) : lane;
  const bool rs_writer = NRS == 16 ? (lane & 1) == 0 : true;
  R gsh = 0, gsl = 0;

  auto flush_self = [&]() {
    // S[a][b] = 2 vol_m sum_y W B_a B_b g(y), in FP64 from the compensated sums
    double* sd = reinterpret_cast<double*>(wm.red);
    if (rs_writer && e_rs >= NBLK && e_rs < NBLK + NQ) sd[e_rs - NBLK] = (double)gsh + (double)gsl;
    gsh = gsl = 0;
    __syncwarp();
    if (lane < NBLK) {
      int a = lane / NV, b = lane % NV;
      double sacc = 0.0;
#pragma unroll
      for (int q = 0; q < NQ; q++) sacc += (double)sWB[q * NV + a] * (double)sB[q * NV + b] * sd[q];
      atomicAdd(&P.selfblk[cur_m * NBLK + lane], 2.0 * (double)vol_m * sacc);
    }
    __syncwarp();
  };

  // adds the warp's counters to the current problem's statistics and clears them
  auto flush_stats = [&]() {
    for (int o = 16; o > 0; o >>= 1) {
      st_items += __shfl_xor_sync(0xffffffffu, st_items, o);
      st_exact += __shfl_xor_sync(0xffffffffu, st_exact, o);
      st_closed += __shfl_xor_sync(0xffffffffu, st_closed, o);
      st_band += __shfl_xor_sync(0xffffffffu, st_band, o);
      err |= __shfl_xor_sync(0xffffffffu, err, o);
    }
    if (lane == 0) {
      if (st_items) atomicAdd(&P.stats[0], (unsigned long long)st_items);
      if (st_exact) atomicAdd(&P.stats[2], (unsigned long long)st_exact);
      if (st_eval) atomicAdd(&P.stats[3], (unsigned long long)st_eval);  // counted alike by every lane
      if (st_closed) atomicAdd(&P.stats[4], (unsigned long long)st_closed);
      if (st_band) atomicAdd(&P.stats[5], (unsigned long long)st_band);
      if (err) atomicOr(P0.err, err);
    }
    st_items = st_exact = st_eval = st_closed = st_band = 0;
    err = 0;
    __syncwarp();
  };

  int cur_k = BATCHED ? -1 : 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(P0.counter, (unsigned long long)P0.chunk);
    start = __shfl_sync(0xffffffffu, start, 0);
    int64_t g0, g1;
    if (BATCHED) {
      g0 = (int64_t)start;
      if (g0 >= Bt.total) break;
      g1 = min(g0 + (int64_t)P0.chunk, Bt.total);
    } else {
      g0 = P0.p_begin + (int64_t)start;
      if (g0 >= P0.p_end) break;
      g1 = min(g0 + (int64_t)P0.chunk, P0.p_end);
    }
    while (g0 < g1) {
    int64_t goff = 0, gend = g1;
    if (BATCHED) {
      // problem k with prefix[k] <= g0 < prefix[k+1]
      int lo = 0, hi = Bt.n;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (Bt.prefix[mid] <= g0) lo = mid;
        else hi = mid;
      }
      if (lo != cur_k) {
        if (cur_k >= 0) {
          if (cur_m >= 0) flush_self();
          flush_stats();
        }
        const int* src = reinterpret_cast<const int*>(Bt.probs + lo);
        int* dst = reinterpret_cast<int*>(qcopy);
        for (int t = lane; t < (int)(sizeof(QParams) / sizeof(int)); t += 32) dst[t] = src[t];
        __syncwarp();
        cur_k = lo;
        cur_m = -1;
      }
      goff = Bt.prefix[lo];
      gend = min(g1, Bt.prefix[lo + 1]);
    }
    const int64_t p0 = g0 - goff, p1 = gend - goff;
    g0 = gend;
    int64_t m;
    if (cur_m >= 0 && P.pair_off[cur_m] <= p0 && p0 < P.pair_off[cur_m + 1]) {
      m = cur_m;
    } else {
      // the last m with pair_off[m] <= p0 (pair_off[0] = 0 <= p0 < pair_off[n_elem]): a 32-way
      // search, every lane probing one position per round (a few dependent loads instead of
      // log2(n_elem))
      int64_t lo = 0, hi = P.n_elem;  // pair_off[lo] <= p0 < pair_off[hi]
      while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t idx = lo + (int64_t)lane * step;
        const bool le = idx < hi && P.pair_off[idx] <= p0;
        const unsigned bal = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(bal);  // lane 0 probes lo itself, so bal != 0
        const int64_t nlo = lo + (int64_t)last * step;
        hi = min(hi, nlo + step);
        lo = nlo;
      }
      m = lo;
    }
    int64_t m_end = P.pair_off[m + 1];  // end of m's pairs, reloaded only when m advances
    int32_t l_lane = 0;  // pair_l of the pair p0 + 32 * (block) + lane
    for (int64_t p = p0; p < p1; p++) {
      const int jj = (int)(p - p0);
      if ((jj & 31) == 0) {
        const int64_t pq = p + lane;
        l_lane = pq < p1 ? P.pair_l[pq] : 0;
      }
      const int32_t l = __shfl_sync(0xffffffffu, l_lane, jj & 31);
      if constexpr (F32) {
        // the record of this pair was fetched during the previous pair except at the first pair
        // of each block of 32; the next pair's record is fetched now (cp.async groups: wait for
        // all but the group just committed)
        constexpr int NCP = G::EFS / 4;
        if ((jj & 31) == 0) {
          if (lane < NCP) cp_async16(wm.pf + (jj & 1) * 32 + lane * 4, P.ef + (int64_t)l * G::EFS + lane * 4);
          cp_async_commit();
        }
        const int32_t ln = __shfl_sync(0xffffffffu, l_lane, (jj + 1) & 31);
        if (p + 1 < p1 && ((jj + 1) & 31) != 0 && lane < NCP)
          cp_async16(wm.pf + ((jj + 1) & 1) * 32 + lane * 4, P.ef + (int64_t)ln * G::EFS + lane * 4);
        cp_async_commit();
      }
      while (p >= m_end) {
        m++;
        m_end = P.pair_off[m + 1];
      }
      if (m != cur_m) {
        if (cur_m >= 0) flush_self();
        cur_m = m;
        R Vm[NV][D];
        if (F32) {
          const float* ef = P.ef + m * G::EFS;
#pragma unroll
          for (int k = 0; k < D; k++) {
            v0h[k] = ef[NL_EF_V0HI(D) + k];
            v0l[k] = ef[NL_EF_V0LO(D) + k];
          }
#pragma unroll
          for (int k = 0; k < D; k++) Vm[0][k] = 0;
#pragma unroll
          for (int a = 1; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vm[a][k] = (R)ef[(a - 1) * D + k];
          vol_m = (R)ef[2 * D * D];
        } else {
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vm[a][k] = (R)P.evert[m * NVC + a * D + k];
          vol_m = (R)P.vol[m];
        }
#pragma unroll
        for (int k = 0; k < D; k++) {
          R lo = Vm[0][k], hi = Vm[0][k];
#pragma unroll
          for (int a = 1; a < NV; a++) {
            lo = Vm[a][k] < lo ? Vm[a][k] : lo;
            hi = Vm[a][k] > hi ? Vm[a][k] : hi;
          }
          if (lane == 0) {  // box of m (local FP32 coordinates, or global FP64)
            wm.pc[k] = lo;
            wm.pc[D + k] = hi;
          }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          int q = ybase + i;
#pragma unroll
          for (int k = 0; k < D; k++) {
            R s = 0;
#pragma unroll
            for (int a = 0; a < NV; a++) s += sB[q * NV + a] * Vm[a][k];
            y[i][k] = s;
          }
        }
        if constexpr (F32) {
#pragma unroll
          for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < D; k++) yq[j][k] = f2pack((float)y[2 * j][k], (float)y[2 * j + 1][k]);
        }
        if constexpr (MMA != 0) {
#pragma unroll
          for (int r = 0; r < MROWS; r++) {
            const int q = (lane >> 2) + 8 * r;
#pragma unroll
            for (int k = 0; k < D; k++) {
              float s = 0.f;
              if (q < NQ) {
#pragma unroll
                for (int a = 0; a < NV; a++) s += (float)sB[q * NV + a] * (float)Vm[a][k];
              }
              ym[r][k] = s;
            }
          }
        }
      }
      // ---- per-pair set-up ------------------------------------------------------------------
      // Only the first vertex of E_l stays in registers; the whole simplex is rebuilt when the
      // traversal needs it (FP32: from this pair's record in shared memory, which stays until the
      // next pair; FP64: from the element arrays).
      // FP32: the inverse Jacobian of E_l is read from the record in shared memory where it is
      // used (one broadcast load per entry), FP64: registers
      R Vl0[D], Ji[D][D], wl;
      auto JI = [&](int r, int c) -> R {
        if constexpr (F32) return wm.pf[(jj & 1) * 32 + D * D + r * D + c];
        else return Ji[r][c];
      };
      if constexpr (F32) {
        cp_async_wait_prior();
        __syncwarp();
        const float* ef = wm.pf + (jj & 1) * 32;
#pragma unroll
        for (int k = 0; k < D; k++)  // v_0(l) - v_0(m) from the float-float pairs, ~1 ulp
          Vl0[k] = (R)((ef[NL_EF_V0HI(D) + k] - v0h[k]) + (ef[NL_EF_V0LO(D) + k] - v0l[k]));
        wl = (R)P.fC * (R)ef[2 * D * D];
      } else {
#pragma unroll
        for (int k = 0; k < D; k++) Vl0[k] = (R)P.evert[(int64_t)l * NVC + k];
#pragma unroll
        for (int r = 0; r < D; r++)
#pragma unroll
          for (int c = 0; c < D; c++) Ji[r][c] = (R)P.jinv[((int64_t)l * D + r) * D + c];
        wl = (R)(P.C * P.vol[l]);
      }
      auto get_Vl = [&](R (&V)[NV][D]) {
        if constexpr (F32) {
          const float* ef = wm.pf + (jj & 1) * 32;
#pragma unroll
          for (int k = 0; k < D; k++) V[0][k] = Vl0[k];
#pragma unroll
          for (int a = 1; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) V[a][k] = Vl0[k] + (R)ef[(a - 1) * D + k];
        } else {
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) V[a][k] = (R)P.evert[((int64_t)l * NV + a) * D + k];
        }
      };
      // 2D: largest distance from the centroid of E_l to its vertices (see closed_set)
      R rad_l = 0;
      if (D == 2) {
        R Vt[NV][D], ct[D];
        get_Vl(Vt);
#pragma unroll
        for (int k = 0; k < D; k++) ct[k] = (Vt[0][k] + Vt[1][k] + Vt[D][k]) * (R)(1.0 / NV);
        R r2 = 0;
#pragma unroll
        for (int a = 0; a < NV; a++) {
          R d2 = 0;
#pragma unroll
          for (int k = 0; k < D; k++) {
            const R d = Vt[a][k] - ct[k];
            d2 += d * d;
          }
          r2 = r2 > d2 ? r2 : d2;
        }
        rad_l = sqrt(r2);
      }

      R gp[NYL], hp[D][NYL], ug = 0, uh[D];
      f2 gq[3], hq[D][3];  // R = float: accumulators of inner points 0-5 in pairs
#pragma unroll
      for (int i = 0; i < NYL; i++) {
        gp[i] = 0;
#pragma unroll
        for (int k = 0; k < D; k++) hp[k][i] = 0;
      }
#pragma unroll
      for (int j = 0; j < 3; j++) {
        gq[j] = 0ull;
#pragma unroll
        for (int k = 0; k < D; k++) hq[k][j] = 0ull;
      }
#pragma unroll
      for (int k = 0; k < D; k++) uh[k] = 0;
      // MMA: the fragment accumulators of the pair's contraction H_c(y) = sum_x G(x, y) w_x
      // phi^l_c(x) (rows: inner points y, columns: nodes c of l)
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      // whether anything was summed for this pair (a closed form on this lane, or an
      // integration by the warp): pairs with no contribution skip the end-of-pair reduction
      bool contrib = false;

      // Algorithm 1 decision for a sub-element (R coordinates)
      // count_exact: this lane counts an FP64 re-decision (lanes that classify the same
      // sub-element redundantly count it once)
      auto classify = [&](const R (&V)[NV][D], uint32_t code, bool count_exact) -> int {
        const int level = code >> LEVEL_SHIFT;
        if (level < P.L_min) return ACT_REFINE;
        const bool last = level == P.L_max;
        if (F32) {
          float fam, fan;
          float Vf[NV][D];
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vf[a][k] = (float)V[a][k];
          float flo[D], fhi[D];
#pragma unroll
          for (int k = 0; k < D; k++) {
            flo[k] = (float)wm.pc[k];
            fhi[k] = (float)wm.pc[D + k];
          }
          float fe2;
          screen_dists<D>(Vf, flo, fhi, fam, fan, fe2);  // fam = squared aprx-max-dist
          const bool c_int = fam < P.fint2;
          const bool c_notint = fam > P.fnotint2;
          const bool l2 = P.mindist_l2 != 0;
          const bool c_ref = l2 ? fe2 < P.fref2 : fan < P.fdpe - P.margin;
          const bool c_out = l2 ? fe2 > P.fout2 : fan > P.fdpe + P.margin;
          if (last) return c_int ? ACT_INT : (c_out ? ACT_ZERO : ACT_FINAL);
          if (c_int) return ACT_INT;
          if (c_notint && c_ref) return ACT_REFINE;
          if (c_notint && c_out) return ACT_DROP;
          st_exact += count_exact ? 1 : 0;
          return exact_classify<D>(P.evert + (int64_t)l * NVC, P.blo + cur_m * D, P.bhi + cur_m * D,
                                   code, P.dme, P.dpe, P.mindist_l2 != 0);
        } else {
          double Vd[NV][D], lo2[D], hi2[D];
#pragma unroll
          for (int a = 0; a < NV; a++)
#pragma unroll
            for (int k = 0; k < D; k++) Vd[a][k] = (double)V[a][k];
#pragma unroll
          for (int k = 0; k < D; k++) {
            lo2[k] = (double)wm.pc[k];
            hi2[k] = (double)wm.pc[D + k];
          }
          double amax, amin;
          exact_dists<D>(Vd, lo2, hi2, amax, amin, P.mindist_l2 != 0);
          if (last) return amax < P.dme ? ACT_INT : (amin > P.dpe ? ACT_ZERO : ACT_FINAL);
          if (amax < P.dme) return ACT_INT;
          if (amin < P.dpe) return ACT_REFINE;
          return ACT_DROP;
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
        const R wv = wl * pow2m(R(0), D * (level - 1));
        ug += wv;
#pragma unroll
        for (int r = 0; r < D; r++) {
          R s = 0;
#pragma unroll
          for (int c = 0; c < D; c++) s += JI(r, c) * (cen[c] - Vl0[c]);
          uh[r] += wv * s;
        }
        st_closed++;
        contrib = true;
      };

      // A FINAL sub-element E' (L_max reached, the band in reach of the box of m) whose every
      // point lies, for each inner point y of m, either closer than delta - eps - margin or
      // farther than delta + eps + margin (ball around the centroid c of radius
      // R = max |v - c|: |x - y| <= |c - y| + R and >= |c - y| - R) has mu exactly 1 or 0 at
      // each of its point pairs; with the constant kernel its outer sum for an inner point with
      // mu = 1 is C |E'| [1, lambda^l(c)] (degree-5 rule, linear integrand), added to that
      // inner point only.  Returns false (nothing added) unless every inner point is decided.
      // 2D: every lane holds all inner points of m.
      // The lane's inner point i (of the 7 it holds).
      auto lane_y = [&](int i, R (&yi)[D]) {
#pragma unroll
        for (int k = 0; k < D; k++) {
          if constexpr (F32) {
            if (i < 6) {
              float a, b;
              f2unpack(yq[i / 2][k], a, b);
              yi[k] = (i & 1) ? b : a;
            } else {
              yi[k] = y[6][k];
            }
          } else {
            yi[k] = y[i][k];
          }
        }
      };
      // Sub-element with centroid cen and radius rad (every point within rad of cen): for each
      // of the lane's inner points y, mu is exactly 1 at every point pair if |cen - y| is below
      // delta - eps - rad - margin, exactly 0 if above delta + eps + rad + margin.  Returns
      // whether every inner point is decided, and the mask of those with mu = 1.
      auto decide_ball = [&](const R (&cen)[D], R rad, unsigned& in_mask) -> bool {
        const R lo = (R)P.fdme - rad - (R)P.margin, hi = (R)P.fdpe + rad + (R)P.margin;
        const R lo2 = lo > 0 ? lo * lo : (R)-1, hi2 = hi * hi;
        in_mask = 0;
        bool decided = true;
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          R yi[D];
          lane_y(i, yi);
          R d2 = 0;
#pragma unroll
          for (int k = 0; k < D; k++) {
            const R d = cen[k] - yi[k];
            d2 += d * d;
          }
          const bool in = d2 < lo2, out = d2 > hi2;
          in_mask |= in ? (1u << i) : 0u;
          decided = decided && (in || out);
        }
        return decided;
      };
      // Adds the closed-form outer sum C |E'| [1, lambda^l(cen)] (weight wv = C |E'|; the degree-5
      // rule integrates the linear integrand exactly) to the lane's inner points in in_mask.
      auto add_closed = [&](const R (&cen)[D], R wv, unsigned in_mask) {
        R lc[D];  // lambda^l(c)
#pragma unroll
        for (int r = 0; r < D; r++) {
          R t = 0;
#pragma unroll
          for (int c = 0; c < D; c++) t += JI(r, c) * (cen[c] - Vl0[c]);
          lc[r] = t;
        }
        if constexpr (F32) {
#pragma unroll
          for (int j = 0; j < 3; j++) {
            const f2 w2 = f2pack((in_mask >> (2 * j)) & 1u ? wv : 0.f, (in_mask >> (2 * j + 1)) & 1u ? wv : 0.f);
            gq[j] = f2add(gq[j], w2);
#pragma unroll
            for (int k = 0; k < D; k++) hq[k][j] = f2fma(w2, f2dup(lc[k]), hq[k][j]);
          }
          const R w6 = (in_mask >> 6) & 1u ? wv : (R)0;
          gp[6] += w6;
#pragma unroll
          for (int k = 0; k < D; k++) hp[k][6] += w6 * lc[k];
        } else {
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            const R wi = (in_mask >> i) & 1u ? wv : (R)0;
            gp[i] += wi;
#pragma unroll
            for (int k = 0; k < D; k++) hp[k][i] += wi * lc[k];
          }
        }
        contrib = true;
      };

      // A FINAL sub-element E' (L_max reached, the band in reach of the box of m) whose every
      // point pair has mu exactly 1 or 0 (decide_ball) contributes, with the constant kernel,
      // the closed form to the inner points with mu = 1.  2D, at classification time (every
      // lane holds all inner points of m; every midpoint child of a triangle is the parent
      // scaled by 1/2, so the radius of a level-L sub-element is that of E_l times 2^(1-L),
      // with the rounding inside the margin).  Returns false (nothing added) unless every
      // inner point is decided.
      auto closed_set = [&](const R (&V)[NV][D], int level) -> bool {
        if (D != 2) return false;
        R cen[D];
#pragma unroll
        for (int k = 0; k < D; k++) {
          R t = 0;
#pragma unroll
          for (int a = 0; a < NV; a++) t += V[a][k];
          cen[k] = t * (R)(1.0 / NV);
        }
        const R rad = rad_l * pow2m(R(0), level - 1);
        unsigned in_mask;
        if (!decide_ball(cen, rad, in_mask)) return false;
        add_closed(cen, wl * pow2m(R(0), D * (level - 1)), in_mask);
        st_closed++;
        return true;
      };

      // integrate the buffered items of one kind (warp-collective)
      auto integrate = [&](int kind, int n_it) {
        const MollK MK{P.fmqe, P.ftqe, P.fue};
        const bool count_band = P.count_band != 0, gauss = is_gauss();
        const float inv_d2 = P.finv_delta2;
        constexpr int PAD = VPad<D>::N;
        const R* iv = wm.iv + (size_t)kind * NV * IMAX * PAD;
        const R* iw = wm.iw + kind * IMAX;
        const int n_x = n_it * NQ;
        st_eval += (unsigned)(n_x * NQ);
        contrib = contrib || n_x > 0;
        if constexpr (MMA != 0) {
          // Tensor-core contraction.  For each batch of 32 outer points x, lane i stages point
          // i: its coordinates and B[x][c] = w_x phi^l_c(x) (the P1 basis of l, c = 0..D),
          // split into two parts.  Then each thread evaluates G(x, y) = [mu] [eta] at the point
          // pairs of its A-fragment entries (rows: inner points y = lane/4 (+8), columns: outer
          // points), and mma.sync adds A B into the accumulators H_c(y).  The split makes the
          // product accurate to about 2^-22 (TF32) / 2^-16 (BF16): 2D uses fragment rows 8-15
          // for the low parts of A (7 inner points fit in rows 0-6), 3D its 14 inner points use
          // all rows and the low part of A takes a third product.
          float* xs = mstage;              // [32][PAD]
          float* bs = mstage + 32 * PAD;   // [2][NV][MMA_BS]: high and low parts of B
          const int g = lane >> 2, t = lane & 3;
          for (int base = 0; base < n_x; base += 32) {
            {
              const int o = base + lane;
              const bool valid = o < n_x;
              const int it = valid ? o / NQ : 0;
              const int q = valid ? o - it * NQ : 0;
              float x[D];
#pragma unroll
              for (int k = 0; k < D; k++) x[k] = 0.f;
#pragma unroll
              for (int a = 0; a < NV; a++) {
                float va[D];
                vload<D, float>(iv + ((size_t)a * IMAX + it) * PAD, va);
                const float b = sB[q * NV + a];
#pragma unroll
                for (int k = 0; k < D; k++) x[k] += b * va[k];
              }
              const float wcx = valid ? sW[q] * iw[it] : 0.f;
              float ph[NV];
              ph[0] = 1.f;
#pragma unroll
              for (int r = 0; r < D; r++) {
                float s2 = 0.f;
#pragma unroll
                for (int c = 0; c < D; c++) s2 += JI(r, c) * (x[c] - Vl0[c]);
                ph[r + 1] = s2;
                ph[0] -= s2;
              }
              vstore<D, float>(xs + lane * PAD, x);
#pragma unroll
              for (int c = 0; c < NV; c++) {
                const float bv = wcx * ph[c];
                if constexpr (MMA == 1) {
                  uint32_t hi, lo;
                  split_tf32(bv, hi, lo);
                  bs[c * MMA_BS + lane] = __uint_as_float(hi);
                  bs[(NV + c) * MMA_BS + lane] = __uint_as_float(lo);
                } else {
                  // the BF16 rounding of bv (exact as a float), and the remainder
                  const float hi = __uint_as_float(bf16x2(bv, 0.f) << 16);
                  bs[c * MMA_BS + lane] = hi;
                  bs[(NV + c) * MMA_BS + lane] = bv - hi;
                }
              }
            }
            __syncwarp();
            // G at the thread's point pairs: outer points xa, xb (packed), inner point row r
            auto geval = [&](const float (&xa)[D], const float (&xb)[D], int r, bool xva, bool xvb,
                             float& ga, float& gb) {
              f2 d = f2sub(f2pack(xa[0], xb[0]), f2dup(ym[r][0]));
              f2 r2 = f2mul(d, d);
#pragma unroll
              for (int k = 1; k < D; k++) {
                d = f2sub(f2pack(xa[k], xb[k]), f2dup(ym[r][k]));
                r2 = f2fma(d, d, r2);
              }
              f2 gg = f2dup(1.f);
              const bool yv = g + 8 * r < NQ;
              if (kind == KIND_FINAL) {
                gg = mollifier2(MK, r2);
                if (count_band) {
                  float a, b;
                  f2unpack(r2, a, b);
                  st_band += (yv && xva && a >= P.fdme2 && a <= P.fdpe2) ? 1 : 0;
                  st_band += (yv && xvb && b >= P.fdme2 && b <= P.fdpe2) ? 1 : 0;
                }
              }
              if (gauss) gg = (kind == KIND_FINAL) ? f2mul(gg, eta_gauss2(inv_d2, r2)) : eta_gauss2(inv_d2, r2);
              f2unpack(gg, ga, gb);
              ga = yv ? ga : 0.f;
              gb = yv ? gb : 0.f;
            };
            // the products of this batch of 32 outer points accumulate from zero in the tensor
            // cores and are then added to the pair's accumulators in FP32 (at most 32 terms
            // summed inside the MMA chain)
            float part[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (MMA == 1) {
              // m16n8k8: A columns (outer points) t and t+4 of each group of 8
#pragma unroll
              for (int j = 0; j < 4; j++) {
                if (base + 8 * j >= n_x) break;
                const int ia = 8 * j + t, ib = ia + 4;
                float xa[D], xb[D];
                vload<D, float>(xs + ia * PAD, xa);
                vload<D, float>(xs + ib * PAD, xb);
                const bool xva = base + ia < n_x, xvb = base + ib < n_x;
                uint32_t bh0 = 0, bh1 = 0, bl0 = 0, bl1 = 0;
                if (g < NV) {
                  bh0 = __float_as_uint(bs[g * MMA_BS + ia]);
                  bh1 = __float_as_uint(bs[g * MMA_BS + ib]);
                  bl0 = __float_as_uint(bs[(NV + g) * MMA_BS + ia]);
                  bl1 = __float_as_uint(bs[(NV + g) * MMA_BS + ib]);
                }
                if constexpr (D == 2) {
                  float ga, gb;
                  geval(xa, xb, 0, xva, xvb, ga, gb);
                  uint32_t ah0, al0, ah1, al1;
                  split_tf32(ga, ah0, al0);
                  split_tf32(gb, ah1, al1);
                  // rows 0-7: high parts, rows 8-15: low parts of the same inner points
                  mma_tf32(part, ah0, al0, ah1, al1, bh0, bh1);
                  mma_tf32(part, ah0, al0, ah1, al1, bl0, bl1);
                } else {
                  float g0a, g0b, g1a, g1b;
                  geval(xa, xb, 0, xva, xvb, g0a, g0b);
                  geval(xa, xb, 1, xva, xvb, g1a, g1b);
                  uint32_t h0a, l0a, h0b, l0b, h1a, l1a, h1b, l1b;
                  split_tf32(g0a, h0a, l0a);
                  split_tf32(g0b, h0b, l0b);
                  split_tf32(g1a, h1a, l1a);
                  split_tf32(g1b, h1b, l1b);
                  mma_tf32(part, h0a, h1a, h0b, h1b, bh0, bh1);
                  mma_tf32(part, h0a, h1a, h0b, h1b, bl0, bl1);
                  mma_tf32(part, l0a, l1a, l0b, l1b, bh0, bh1);
                }
              }
            } else {
              // m16n8k16: A columns (outer points) 2t, 2t+1, 2t+8, 2t+9 of each group of 16
#pragma unroll
              for (int j = 0; j < 2; j++) {
                if (base + 16 * j >= n_x) break;
                const int i0 = 16 * j + 2 * t;
                float x0[D], x1[D], x8[D], x9[D];
                vload<D, float>(xs + i0 * PAD, x0);
                vload<D, float>(xs + (i0 + 1) * PAD, x1);
                vload<D, float>(xs + (i0 + 8) * PAD, x8);
                vload<D, float>(xs + (i0 + 9) * PAD, x9);
                const bool v0 = base + i0 < n_x, v1 = base + i0 + 1 < n_x;
                const bool v8 = base + i0 + 8 < n_x, v9 = base + i0 + 9 < n_x;
                uint32_t bh0 = 0, bh1 = 0, bl0 = 0, bl1 = 0;
                if (g < NV) {
                  const float2 h01 = *reinterpret_cast<const float2*>(bs + g * MMA_BS + i0);
                  const float2 h89 = *reinterpret_cast<const float2*>(bs + g * MMA_BS + i0 + 8);
                  const float2 l01 = *reinterpret_cast<const float2*>(bs + (NV + g) * MMA_BS + i0);
                  const float2 l89 = *reinterpret_cast<const float2*>(bs + (NV + g) * MMA_BS + i0 + 8);
                  bh0 = bf16x2(h01.x, h01.y);
                  bh1 = bf16x2(h89.x, h89.y);
                  bl0 = bf16x2(l01.x, l01.y);
                  bl1 = bf16x2(l89.x, l89.y);
                }
                if constexpr (D == 2) {
                  float g0, g1, g8, g9;
                  geval(x0, x1, 0, v0, v1, g0, g1);
                  geval(x8, x9, 0, v8, v9, g8, g9);
                  uint32_t h01, l01, h89, l89;
                  split_bf16x2(g0, g1, h01, l01);
                  split_bf16x2(g8, g9, h89, l89);
                  mma_bf16(part, h01, l01, h89, l89, bh0, bh1);
                  mma_bf16(part, h01, l01, h89, l89, bl0, bl1);
                } else {
                  float a0, a1, a8, a9, c0, c1, c8, c9;
                  geval(x0, x1, 0, v0, v1, a0, a1);
                  geval(x8, x9, 0, v8, v9, a8, a9);
                  geval(x0, x1, 1, v0, v1, c0, c1);
                  geval(x8, x9, 1, v8, v9, c8, c9);
                  uint32_t ha01, la01, ha89, la89, hc01, lc01, hc89, lc89;
                  split_bf16x2(a0, a1, ha01, la01);
                  split_bf16x2(a8, a9, ha89, la89);
                  split_bf16x2(c0, c1, hc01, lc01);
                  split_bf16x2(c8, c9, hc89, lc89);
                  mma_bf16(part, ha01, hc01, ha89, hc89, bh0, bh1);
                  mma_bf16(part, ha01, hc01, ha89, hc89, bl0, bl1);
                  mma_bf16(part, la01, lc01, la89, lc89, bh0, bh1);
                }
              }
            }
#pragma unroll
            for (int r = 0; r < 4; r++) acc[r] += part[r];
            __syncwarp();  // the batch is read before the next one is staged
          }
          return;
        }
        for (int base = 0; base < n_x; base += G::XPI) {
          const int o = base + xl;
          const bool valid = o < n_x;
          const int it = valid ? o / NQ : 0;
          const int q = valid ? o - it * NQ : 0;
          R x[D];
#pragma unroll
          for (int k = 0; k < D; k++) x[k] = 0;
#pragma unroll
          for (int a = 0; a < NV; a++) {
            R va[D];
            vload<D, R>(iv + ((size_t)a * IMAX + it) * PAD, va);
            const R b = sB[q * NV + a];
#pragma unroll
            for (int k = 0; k < D; k++) x[k] += b * va[k];
          }
          const R wcx = valid ? sW[q] * iw[it] : (R)0;
          R lam[D];
#pragma unroll
          for (int r = 0; r < D; r++) {
            R s = 0;
#pragma unroll
            for (int c = 0; c < D; c++) s += JI(r, c) * (x[c] - Vl0[c]);
            lam[r] = s;
          }
          if constexpr (F32) {
            // inner points 0-5 in packed pairs, point 6 alone
            // per point pair g = mu (eta): added as w_x g to G and as (w_x lambda_k) g to H_k
            f2 X[D], WL[D];
            float wl[D];
#pragma unroll
            for (int k = 0; k < D; k++) {
              X[k] = f2dup(x[k]);
              wl[k] = wcx * lam[k];
              WL[k] = f2dup(wl[k]);
            }
            const f2 Wx = f2dup(wcx);
#pragma unroll
            for (int j = 0; j < 3; j++) {
              f2 d = f2sub(X[0], yq[j][0]);
              f2 r2 = f2mul(d, d);
#pragma unroll
              for (int k = 1; k < D; k++) {
                d = f2sub(X[k], yq[j][k]);
                r2 = f2fma(d, d, r2);
              }
              f2 g = f2dup(1.f);
              if (kind == KIND_FINAL) {
                g = mollifier2(MK, r2);
                if (count_band) {
                  float a, b;
                  f2unpack(r2, a, b);
                  st_band += (valid && a >= P.fdme2 && a <= P.fdpe2) ? 1 : 0;
                  st_band += (valid && b >= P.fdme2 && b <= P.fdpe2) ? 1 : 0;
                }
              }
              if (gauss) g = (kind == KIND_FINAL) ? f2mul(g, eta_gauss2(inv_d2, r2)) : eta_gauss2(inv_d2, r2);
              gq[j] = f2fma(Wx, g, gq[j]);
#pragma unroll
              for (int k = 0; k < D; k++) hq[k][j] = f2fma(g, WL[k], hq[k][j]);
            }
            float r2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; k++) {
              const float d = x[k] - y[6][k];
              r2 = fmaf(d, d, r2);
            }
            float g = 1.f;
            if (kind == KIND_FINAL) {
              g = mollifier_bf(MK, r2);
              if (count_band) st_band += (valid && r2 >= P.fdme2 && r2 <= P.fdpe2) ? 1 : 0;
            }
            if (gauss) g *= __expf(-r2 * inv_d2);
            gp[6] = fmaf(wcx, g, gp[6]);
#pragma unroll
            for (int k = 0; k < D; k++) hp[k][6] = fmaf(g, wl[k], hp[k][6]);
          } else {
#pragma unroll
            for (int i = 0; i < NYL; i++) {
              R r2 = 0;
#pragma unroll
              for (int k = 0; k < D; k++) {
                const R d = x[k] - y[i][k];
                r2 += d * d;
              }
              R g = wcx;
              if (kind == KIND_FINAL) {
                g *= mollifier(P, r2);
                if (P.count_band)
                  st_band += (valid && r2 >= (R)(P.dme * P.dme) && r2 <= (R)(P.dpe * P.dpe)) ? 1 : 0;
              }
              if (is_gauss()) g *= eta_gauss<R>(P, r2);
              gp[i] += g;
#pragma unroll
              for (int k = 0; k < D; k++) hp[k][i] += g * lam[k];
            }
          }
        }
      };

      // append an item to a buffer slot
      auto put_item = [&](int kind, int slot, const R (&V)[NV][D], int level) {
        constexpr int PAD = VPad<D>::N;
        R* iv = wm.iv + (size_t)kind * NV * IMAX * PAD;
#pragma unroll
        for (int a = 0; a < NV; a++) vstore<D, R>(iv + ((size_t)a * IMAX + slot) * PAD, V[a]);
        wm.iw[kind * IMAX + slot] = wl * pow2m(R(0), D * (level - 1));
      };

      // ---- Algorithm 1 for this pair --------------------------------------------------------
      // The warp-uniform state lives in registers (every lane computes it from the same
      // ballots): sp records on the stack, n_int / n_fin buffered items.  A round expands up to
      // 32/2^n parents, one child per lane; the first round takes its parent, E_l itself, from
      // registers, and in 2D with L_max >= 3 expands two levels at once (16 lanes: the four
      // children and, where a child is refined, its four children).
      {
        int sp = 0, n_int = 0, n_fin = 0;
        const uint32_t code0 = 1u << LEVEL_SHIFT;
        int act0;
        {
          R Vl[NV][D];
          get_Vl(Vl);
          act0 = classify(Vl, code0, lane == 0);
          if (is_const() && act0 == ACT_INT) {
            if (lane == 0) closed_int(Vl, 1);
          } else if (act0 == ACT_INT || act0 == ACT_FINAL) {
            if (lane == 0) put_item(act0 == ACT_INT ? KIND_INT : KIND_FINAL, 0, Vl, 1);
          }
        }
        if (act0 == ACT_INT || act0 == ACT_FINAL || act0 == ACT_ZERO) st_items += (lane == 0);
        bool from_root = act0 == ACT_REFINE;
        if (!(is_const() && act0 == ACT_INT) && (act0 == ACT_INT || act0 == ACT_FINAL)) {
          if (act0 == ACT_INT) n_int = 1;
          else n_fin = 1;
        }
        // child c of the simplex S (registers) by midpoints
        auto child_of = [&](const R (&S)[NV][D], int c, R (&V)[NV][D]) {
#pragma unroll
          for (int v = 0; v < NV; v++) {
            int ia, ib;
            mid_pair<D>(c, v, ia, ib);
#pragma unroll
            for (int k = 0; k < D; k++) {
              R pa = S[0][k], pb = S[0][k];
#pragma unroll
              for (int q = 1; q < NV; q++) {
                pa = (ia == q) ? S[q][k] : pa;
                pb = (ib == q) ? S[q][k] : pb;
              }
              V[v][k] = midp(pa, pb);
            }
          }
        };
        // one classified node per lane: count it, sum it in closed form, buffer it or push it
        auto settle = [&](const R (&V)[NV][D], uint32_t code, int act, int base) {
          const int level = code >> LEVEL_SHIFT;
          if (act == ACT_INT || act == ACT_FINAL || act == ACT_ZERO) st_items++;
          if (is_const() && act == ACT_INT) {
            closed_int(V, level);
            act = ACT_DROP;
          }
          if (is_const() && act == ACT_FINAL && closed_set(V, level)) act = ACT_DROP;
          const unsigned m_int = __ballot_sync(0xffffffffu, act == ACT_INT);
          const unsigned m_fin = __ballot_sync(0xffffffffu, act == ACT_FINAL);
          const unsigned m_ref = __ballot_sync(0xffffffffu, act == ACT_REFINE);
          const unsigned below = (1u << lane) - 1u;
          if (act == ACT_INT || act == ACT_FINAL) {
            const bool fin = act == ACT_FINAL;
            put_item(fin ? KIND_FINAL : KIND_INT,
                     fin ? n_fin + __popc(m_fin & below) : n_int + __popc(m_int & below), V, level);
          }
          const int nref = __popc(m_ref);
          const bool overflow = base + nref > P.scap;
          if (overflow) {
            err |= ERR_STACK;
          } else if (act == ACT_REFINE) {
            const int slot = base + __popc(m_ref & below);
#pragma unroll
            for (int a = 0; a < NV; a++)
              vstore<D, R>(wm.rv + ((size_t)a * P.scap + slot) * VPad<D>::N, V[a]);
            wm.rc[slot] = code;
          }
          sp = overflow ? base : base + nref;
          n_int += __popc(m_int);
          n_fin += __popc(m_fin);
          __syncwarp();  // records and items written in this LIFO step are visible to every lane
        };
        if (D == 2 && from_root && P.L_max >= 3) {
          const int c2 = lane >> 2, c3 = lane & 3;
          R V[NV][D];
          uint32_t code = 0;
          int act = ACT_DROP;
          if (lane < 16) {
            R C[NV][D];
            {
              R Vl[NV][D];
              get_Vl(Vl);
              child_of(Vl, c2, C);
            }
            const uint32_t codeC = (2u << LEVEL_SHIFT) | (uint32_t)c2;
            const int actC = classify(C, codeC, c3 == 0);
            if (actC == ACT_REFINE) {
              child_of(C, c3, V);
              code = (3u << LEVEL_SHIFT) | (uint32_t)c2 | ((uint32_t)c3 << G::BITS);
              act = classify(V, code, true);
            } else if (c3 == 0) {
#pragma unroll
              for (int v = 0; v < NV; v++)
#pragma unroll
                for (int k = 0; k < D; k++) V[v][k] = C[v][k];
              code = codeC;
              act = actC;
            }
          }
          from_root = false;
          settle(V, code, act, 0);
        }
        while (from_root || sp > 0) {
          if (n_fin > IMAX - 32) {
            integrate(KIND_FINAL, n_fin);
            n_fin = 0;
          }
          if (n_int > IMAX - 32) {
            integrate(KIND_INT, n_int);
            n_int = 0;
          }
          const int np = from_root ? 1 : min(G::NPOP, sp);
          const int base = sp - (from_root ? 0 : np);
          const int par = lane / G::NCH, c = lane % G::NCH;
          const bool active = par < np;
          R V[NV][D];
          uint32_t code = 0;
          int act = ACT_DROP;
          if (active) {
            if (from_root) {
              R Vl[NV][D];
              get_Vl(Vl);
              child_of(Vl, c, V);
              code = (2u << LEVEL_SHIFT) | (uint32_t)c;
            } else {
              const int slot = base + par;
              const uint32_t pcode = wm.rc[slot];
              const int plevel = pcode >> LEVEL_SHIFT;
#pragma unroll
              for (int v = 0; v < NV; v++) {
                int ia, ib;
                mid_pair<D>(c, v, ia, ib);
                R pa[D], pb[D];
                vload<D, R>(wm.rv + ((size_t)ia * P.scap + slot) * VPad<D>::N, pa);
                vload<D, R>(wm.rv + ((size_t)ib * P.scap + slot) * VPad<D>::N, pb);
#pragma unroll
                for (int k = 0; k < D; k++) V[v][k] = midp(pa[k], pb[k]);
              }
              code = (((uint32_t)(plevel + 1)) << LEVEL_SHIFT) | (pcode & ((1u << LEVEL_SHIFT) - 1)) |
                     ((uint32_t)c << (G::BITS * (plevel - 1)));
            }
          }
          __syncwarp();  // parent records are read before children overwrite their slots
          from_root = false;
          if (active) act = classify(V, code, true);
          settle(V, code, act, base);
        }
        __syncwarp();
        if (n_fin > 0) integrate(KIND_FINAL, n_fin);
        if (n_int > 0) integrate(KIND_INT, n_int);
      }
      // ---- end of pair: per-lane contraction, warp reduce-scatter, cross block, self sums ------
      // A pair whose every sub-element was dropped (or lies beyond delta + eps) contributes
      // nothing: its cross block is zero and the self sums are unchanged.
      if (!__any_sync(0xffffffffu, contrib)) {
        if (!DIRECT && lane < NBLK) reinterpret_cast<R*>(P.blk)[(p - P.p_begin) * NBLK + lane] = (R)0;
        __syncwarp();
        continue;
      }
      {
        if constexpr (F32) {
#pragma unroll
          for (int j = 0; j < 3; j++) {
            f2unpack(gq[j], gp[2 * j], gp[2 * j + 1]);
#pragma unroll
            for (int k = 0; k < D; k++) f2unpack(hq[k][j], hp[k][2 * j], hp[k][2 * j + 1]);
          }
        }
        // H_0 = g - sum_k h_k, H_c = h_{c-1} (P1 basis of l: phi_0 = 1 - sum_k lambda_k); the
        // closed-form items add the same U_c at every inner point
        R U[NV];
        U[0] = ug;
#pragma unroll
        for (int k = 0; k < D; k++) {
          U[0] -= uh[k];
          U[k + 1] = uh[k];
        }
        // lane partial of sum_y W_y B_a(y) H_c(y) over the lane's inner points, then the lane's g
        // at its inner points (with the uniform part; 3D: both half-warp lanes of an outer
        // point hold part of it), zero elsewhere
        R v[NRS];
#pragma unroll
        for (int a = 0; a < NV; a++)
#pragma unroll
          for (int c = 0; c < NV; c++) v[a * NV + c] = sWBs[a] * U[c];
#pragma unroll
        for (int i = 0; i < NYL; i++) {
          R H[NV];
          H[0] = gp[i];
#pragma unroll
          for (int k = 0; k < D; k++) {
            H[0] -= hp[k][i];
            H[k + 1] = hp[k][i];
          }
#pragma unroll
          for (int a = 0; a < NV; a++) {
            const R wb = sWB[(ybase + i) * NV + a];
#pragma unroll
            for (int c = 0; c < NV; c++) v[a * NV + c] += wb * H[c];
          }
        }
        {
          R ugt = ug;
          if (D == 3) ugt += __shfl_xor_sync(0xffffffffu, ug, 16);
#pragma unroll
          for (int i = 0; i < NYL; i++) {
            if (D == 2) {
              v[NBLK + i] = gp[i] + ugt;
            } else {
              v[NBLK + i] = ybase == 0 ? gp[i] + ugt : (R)0;
              v[NBLK + NYL + i] = ybase == 0 ? (R)0 : gp[i] + ugt;
            }
          }
#pragma unroll
          for (int t = NBLK + NQ; t < NRS; t++) v[t] = 0;
        }
        if constexpr (MMA != 0) {
          // the tensor-core accumulators: H_c(y) for the thread's fragment entries (rows: inner
          // points q = lane/4 (+8); columns c = 2 (lane % 4) and the next one; 2D: rows 8-15 hold
          // the low-part products of the same inner points), contracted like the lane sums above
          // (the reduce-scatter below adds every thread's share)
          const int q0 = lane >> 2, c0 = 2 * (lane & 3);
#pragma unroll
          for (int r = 0; r < MROWS; r++) {
            const int q = q0 + 8 * r;
            const float h0 = D == 2 ? acc[0] + acc[2] : acc[2 * r];
            const float h1 = D == 2 ? acc[1] + acc[3] : acc[2 * r + 1];
            if (q < NQ) {
#pragma unroll
              for (int c = 0; c < NV; c++) {
                const float hc = c == c0 ? h0 : (c == c0 + 1 ? h1 : 0.f);
#pragma unroll
                for (int a = 0; a < NV; a++) v[a * NV + c] += sWB[q * NV + a] * hc;
              }
#pragma unroll
              for (int qq = 0; qq < NQ; qq++) v[NBLK + qq] += qq == q ? h0 + h1 : 0.f;
            }
          }
        }
        // reduce-scatter over the warp: every step sends half of the remaining values to the
        // partner lane and adds the half it keeps; 2D: four steps (offsets 16..2) and a final
        // sum with lane ^ 1 (lane L holds entry L >> 1), 3D: five steps (lane L holds entry L)
#pragma unroll
        for (int half = NRS / 2; half >= 1; half >>= 1) {
          const int off = half * (32 / NRS);
          const bool up = (lane & off) != 0;
#pragma unroll
          for (int j = 0; j < half; j++) {
            const R send = up ? v[j] : v[j + half];
            const R keep = up ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        const R tot_e = NRS == 16 ? v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1) : v[0];
        if (rs_writer && e_rs < NBLK) {
          const R cval = (R)(-2) * vol_m * tot_e;
          if (DIRECT) {
            const int a = e_rs / NV, c = e_rs % NV;
            const int64_t pos = csr_find(P.row_ptr, P.col, P.conn[cur_m * NV + a],
                                         P.conn[(int64_t)l * NV + c]);
            if (pos < 0) err |= ERR_CSR;
            else atomicAdd(&P.values[pos], (double)cval);
          } else {
            reinterpret_cast<R*>(P.blk)[(p - P.p_begin) * NBLK + e_rs] = cval;
          }
        }
        if (e_rs >= NBLK && e_rs < NBLK + NQ) two_sum_add(gsh, gsl, tot_e);
      }
      __syncwarp();
    }
    }  // pairs of one problem within the chunk
    flush_stats();
  }
  if (cur_k >= 0 && cur_m >= 0) flush_self();
}

// ---- scatter of the local blocks into the CSR values ------------------------------------------
// One CTA per inner element m; its contributions (the cross blocks of the pairs p of m in
// [q0, q1), stored at blk[p - p_base], and with_self the self block of m) are summed per CSR
// entry in shared-memory accumulators and each entry is added to the global values once
// (FP64 atomics: the rows of a node are shared by the elements around it).  The accumulators
// have the blocks' precision R: FP64 for the FP64 path; FP32 for the FP32 paths, whose blocks
// are FP32 values already (an entry sums about ten of them; shared-memory FP32 atomics are
// native, FP64 ones are not).
//
// Where the column of an entry is found: every row of m's nodes holds the nodes of every l
// paired with m, so a shared-memory hash table keyed by column node gives, for each of m's
// rows, the entry's position in that row: one lookup per node of l serves all D+1 rows of the
// block.  The table (open addressing, linear probing, at most half full: its size is the
// power of two at least twice the longest of the rows) is built from the rows' column lists.
// If the dynamic shared memory cannot hold it, the columns are cached and each entry is found
// by binary search in its row instead.
__host__ __device__ inline int scatter_table_size(int max_row) {
  int t = 64;
  while (t < 2 * max_row) t <<= 1;
  return t;
}
// nn: nodes per element (rows of the element's blocks)
__host__ __device__ inline size_t scatter_hash_bytes(int nn, int T, int64_t acc_entries,
                                                     size_t acc_size) {
  size_t b = (size_t)T * 4;                               // keys
  b += ((size_t)T * nn * 2 + 7) & ~size_t(7);             // int16 positions per row
  return b + (size_t)acc_entries * acc_size;              // accumulators
}

// NN: nodes per element (D+1 for P1, 6 for P2 triangles); blocks are NN x NN.
template <int D, typename R, int NN = D + 1>
__device__ __forceinline__ void scatter_elem(int64_t m, int64_t q0, int64_t q1, int64_t p_base,
                                             bool with_self, const int32_t* __restrict__ pair_l,
                                             const int32_t* __restrict__ conn,
                                             const int64_t* __restrict__ row_ptr,
                                             const int32_t* __restrict__ col,
                                             const R* __restrict__ blk,
                                             const double* __restrict__ selfblk,
                                             double* __restrict__ values, int* __restrict__ err) {
  constexpr int NV = NN, NB = NV * NV;
  extern __shared__ __align__(16) unsigned char sraw[];
  __shared__ int64_t rbeg[NV];
  __shared__ int rlen[NV], roff[NV + 1];
  __shared__ int32_t nodes[NV];
  __shared__ int overflow, n_keys;
  if (threadIdx.x < NV) {
    int32_t i = conn[m * NV + threadIdx.x];
    nodes[threadIdx.x] = i;
    rbeg[threadIdx.x] = row_ptr[i];
    rlen[threadIdx.x] = (int)(row_ptr[i + 1] - row_ptr[i]);
  }
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    roff[0] = 0;
    for (int a = 0; a < NV; a++) roff[a + 1] = roff[a] + rlen[a];
  }
  __syncthreads();
  const int total = roff[NV];
  int max_len = 0;
#pragma unroll
  for (int a = 0; a < NV; a++) max_len = rlen[a] > max_len ? rlen[a] : max_len;
  unsigned dyn = 0;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const int T = scatter_table_size(max_len);
  const int64_t n = (q1 > q0 ? q1 - q0 : 0);
  if (scatter_hash_bytes(NV, T, total, sizeof(R)) <= (size_t)dyn) {
    int32_t* keys = reinterpret_cast<int32_t*>(sraw);
    int16_t* pos = reinterpret_cast<int16_t*>(keys + T);
    R* acc = reinterpret_cast<R*>(sraw + (((size_t)T * 4 + (size_t)T * NV * 2 + 7) & ~size_t(7)));
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
      keys[t] = -1;
#pragma unroll
      for (int a = 0; a < NV; a++) pos[t * NV + a] = -1;
    }
    for (int t = threadIdx.x; t < total; t += blockDim.x) acc[t] = (R)0;
    __syncthreads();
    const unsigned shift = 32u - (unsigned)(31 - __clz(T));
    auto h0 = [&](int32_t key) -> int { return (int)(((uint32_t)key * 2654435761u) >> shift); };
    for (int a = 0; a < NV; a++)
      for (int t = threadIdx.x; t < rlen[a]; t += blockDim.x) {
        const int32_t key = col[rbeg[a] + t];
        int slot = h0(key), probe = 0;
        for (; probe < T; probe++) {
          const int32_t prev = atomicCAS(&keys[slot], -1, key);
          if (prev == -1 || prev == key) break;
          slot = (slot + 1) & (T - 1);
        }
        if (probe < T) pos[slot * NV + a] = (int16_t)t;
        else overflow = 1;  // cannot happen below half load; checked all the same
      }
    __syncthreads();
    if (!overflow) {
      auto lookup = [&](int32_t key) -> int {
        int slot = h0(key);
        for (int probe = 0; probe < T; probe++) {
          const int32_t k = keys[slot];
          if (k == key) return slot;
          if (k == -1) return -1;
          slot = (slot + 1) & (T - 1);
        }
        return -1;
      };
      // one thread per (pair, node c of l): the D+1 entries of column c of the block
      for (int64_t t = threadIdx.x; t < n * NV; t += blockDim.x) {
        const int64_t p = q0 + t / NV;
        const int c = (int)(t % NV);
        const R* bp = blk + (p - p_base) * NB + c;
        R bv[NV];
        bool any = false;
#pragma unroll
        for (int a = 0; a < NV; a++) {
          bv[a] = bp[a * NV];
          any = any || bv[a] != (R)0;
        }
        if (!any) continue;  // a pair with no contribution (all of it beyond delta + eps)
        const int32_t l = pair_l[p];
        const int slot = lookup(conn[(int64_t)l * NV + c]);
#pragma unroll
        for (int a = 0; a < NV; a++) {
          const int ps = slot < 0 ? -1 : pos[slot * NV + a];
          if (ps < 0) atomicOr(err, ERR_CSR);
          else atomicAdd(&acc[roff[a] + ps], bv[a]);
        }
      }
      if (with_self)
        for (int t = threadIdx.x; t < NB; t += blockDim.x) {
          const int a = t / NV, b = t % NV;
          const int slot = lookup(nodes[b]);
          const int ps = slot < 0 ? -1 : pos[slot * NV + a];
          if (ps < 0) atomicOr(err, ERR_CSR);
          else atomicAdd(&acc[roff[a] + ps], (R)selfblk[m * NB + t]);
        }
      __syncthreads();
      for (int a = 0; a < NV; a++)
        for (int t = threadIdx.x; t < rlen[a]; t += blockDim.x) {
          const double v = (double)acc[roff[a] + t];
          if (v != 0.0) atomicAdd(&values[rbeg[a] + t], v);
        }
      return;
    }
    __syncthreads();  // the table is abandoned; its memory is reused below
  }
  // Elements of ten or more nodes (P2 tetrahedra, Q2 and serendipity hexahedra) whose rows
  // are too long for the table above: a table of the columns the element's blocks touch (the
  // nodes of its pairs' l, and its own nodes for the self block) with R accumulators for a
  // group of G rows at a time.  Each group is added to its rows by one pass over their column
  // lists in order (coalesced), an entry taking its column's sum.  The table fills the
  // shared memory (one CTA per SM), so these elements run 512 threads per CTA.
  if constexpr (NV >= 10) {
    constexpr int TT = 8192;  // table slots; the touched columns may fill at most half
    constexpr size_t KEY_B = (size_t)TT * 4;
    const int G = (size_t)dyn > KEY_B
                      ? (int)min((size_t)NV, ((size_t)dyn - KEY_B) / ((size_t)TT * sizeof(R)))
                      : 0;
    if (G >= 1) {
      int32_t* keys = reinterpret_cast<int32_t*>(sraw);
      R* acc = reinterpret_cast<R*>(sraw + KEY_B);  // [TT][G]
      for (int t = threadIdx.x; t < TT; t += blockDim.x) keys[t] = -1;
      if (threadIdx.x == 0) {
        overflow = 0;
        n_keys = 0;
      }
      __syncthreads();
      auto h0 = [](int32_t key) -> int { return (int)(((uint32_t)key * 2654435761u) >> 19); };
      auto insert = [&](int32_t key) {
        int slot = h0(key);
        for (int probe = 0; probe < TT; probe++) {
          const int32_t prev = atomicCAS(&keys[slot], -1, key);
          if (prev == -1) {
            atomicAdd(&n_keys, 1);
            return;
          }
          if (prev == key) return;
          slot = (slot + 1) & (TT - 1);
        }
        overflow = 1;
      };
      for (int64_t t = threadIdx.x; t < n * NV; t += blockDim.x)
        insert(conn[(int64_t)pair_l[q0 + t / NV] * NV + (int)(t % NV)]);
      if (with_self && threadIdx.x < NV) insert(nodes[threadIdx.x]);
      __syncthreads();
      if (!overflow && 2 * n_keys <= TT) {
        auto lookup = [&](int32_t key) -> int {
          int slot = h0(key);
          for (int probe = 0; probe < TT; probe++) {
            const int32_t k = keys[slot];
            if (k == key) return slot;
            if (k == -1) return -1;
            slot = (slot + 1) & (TT - 1);
          }
          return -1;
        };
        for (int a0 = 0; a0 < NV; a0 += G) {
          const int g = min(G, NV - a0);
          for (int t = threadIdx.x; t < TT * G; t += blockDim.x) acc[t] = (R)0;
          __syncthreads();
          // one thread per (pair, node c of l): the g entries of column c in rows a0, a0+1, ...
          for (int64_t t = threadIdx.x; t < n * NV; t += blockDim.x) {
            const int64_t p = q0 + t / NV;
            const int c = (int)(t % NV);
            const R* bp = blk + (p - p_base) * NB + (size_t)a0 * NV + c;
            const int slot = lookup(conn[(int64_t)pair_l[p] * NV + c]);  // inserted above
            if (slot < 0) {
              atomicOr(err, ERR_CSR);
              continue;
            }
            for (int a = 0; a < g; a++) {
              const R v = bp[a * NV];
              if (v != (R)0) atomicAdd(&acc[slot * G + a], v);
            }
          }
          if (with_self)
            for (int t = threadIdx.x; t < g * NV; t += blockDim.x) {
              const int a = t / NV, b = t % NV;
              const int slot = lookup(nodes[b]);
              if (slot < 0) atomicOr(err, ERR_CSR);
              else atomicAdd(&acc[slot * G + a], (R)selfblk[m * NB + (a0 + a) * NV + b]);
            }
          __syncthreads();
          for (int a = 0; a < g; a++) {
            const int64_t rb = rbeg[a0 + a];
            for (int t = threadIdx.x; t < rlen[a0 + a]; t += blockDim.x) {
              const int slot = lookup(col[rb + t]);
              if (slot < 0) continue;
              const R v = acc[slot * G + a];
              if (v != (R)0) {
                atomicAdd(&values[rb + t], (double)v);
                acc[slot * G + a] = (R)0;  // taken: each column appears once in a row
              }
            }
          }
          __syncthreads();
          // a sum still left had no entry in its row
          for (int t = threadIdx.x; t < TT * G; t += blockDim.x)
            if (t % G < g && acc[t] != (R)0) atomicOr(err, ERR_CSR);
          __syncthreads();
        }
        return;
      }
      __syncthreads();  // the table is abandoned; its memory is reused below
    }
  }
  // the rows' column lists cached in shared memory when they fit, else searched in global
  // memory (elements with very long rows, e.g. 27-node hexahedra)
  const bool cache_rows = (size_t)total * 4 <= (size_t)dyn;
  int32_t* rows = reinterpret_cast<int32_t*>(sraw);
  if (cache_rows)
    for (int a = 0; a < NV; a++)
      for (int t = threadIdx.x; t < rlen[a]; t += blockDim.x) rows[roff[a] + t] = col[rbeg[a] + t];
  __syncthreads();
  auto find = [&](int a, int32_t j) -> int64_t {
    int lo = 0, hi = rlen[a] - 1;
    const int32_t* r = cache_rows ? rows + roff[a] : col + rbeg[a];
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int32_t c = r[mid];
      if (c == j) return rbeg[a] + mid;
      if (c < j) lo = mid + 1;
      else hi = mid - 1;
    }
    return -1;
  };
  // With enough dynamic shared memory the element's contributions are first summed per CSR
  // entry in shared memory; otherwise every contribution goes to the global values directly.
  const int acc_off = (total + 3) & ~3;  // ints before the (8-byte aligned) accumulators
  const bool use_acc = cache_rows && (size_t)acc_off * 4 + (size_t)total * 8 <= (size_t)dyn;
  double* acc = reinterpret_cast<double*>(rows + acc_off);
  if (use_acc) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) acc[t] = 0.0;
    __syncthreads();
  }
  auto add = [&](int a, int64_t pos, double v) {
    if (use_acc) atomicAdd(&acc[roff[a] + (int)(pos - rbeg[a])], v);
    else atomicAdd(&values[pos], v);
  };
  for (int64_t t = threadIdx.x; t < n * NB; t += blockDim.x) {
    const int64_t p = q0 + t / NB;
    const int e = (int)(t % NB);
    const int a = e / NV, c = e % NV;
    const int32_t l = pair_l[p];
    const int64_t pos = find(a, conn[(int64_t)l * NV + c]);
    if (pos < 0) {
      atomicOr(err, ERR_CSR);
      continue;
    }
    add(a, pos, (double)blk[(p - p_base) * NB + e]);
  }
  if (with_self)
    for (int t = threadIdx.x; t < NB; t += blockDim.x) {
      const int a = t / NV, b = t % NV;
      const int64_t pos = find(a, nodes[b]);
      if (pos < 0) atomicOr(err, ERR_CSR);
      else add(a, pos, selfblk[m * NB + t]);
    }
  if (use_acc) {
    __syncthreads();
    for (int a = 0; a < NV; a++)
      for (int t = threadIdx.x; t < rlen[a]; t += blockDim.x) {
        const double v = acc[roff[a] + t];
        if (v != 0.0) atomicAdd(&values[rbeg[a] + t], v);
      }
  }
}

// Dynamic shared memory of the scatter kernels for elements of nn nodes, rows of up to max_row
// columns and blocks of acc_size-byte values: the hash layout when it fits in 200 KB, else
// (ten or more nodes) 200 KB for the table of touched columns, else the cached column lists
// plus FP64 accumulators when that fits, else the column lists only, else 16 bytes (the rows
// are then searched in global memory).
inline size_t scatter_smem_bytes(int nn, int max_row, size_t acc_size) {
  const size_t total = (size_t)nn * (size_t)std::max(1, max_row);
  const size_t hashed =
      scatter_hash_bytes(nn, scatter_table_size(std::max(1, max_row)), (int64_t)total, acc_size);
  if (hashed <= (size_t)200 * 1024) return hashed;
  if (nn >= 10) return (size_t)200 * 1024;  // the table of touched columns (scatter_elem)
  const size_t with_acc = ((total + 3) & ~size_t(3)) * 4 + total * 8;
  if (with_acc <= (size_t)200 * 1024) return with_acc;
  if (total * 4 <= (size_t)200 * 1024) return total * 4;
  return 16;
}

// Single problem: CTA b handles element m_begin + b; with_self = 0 adds the cross blocks of
// the pairs in [p_begin, p_end), with_self = 1 only the self blocks.
// threads per CTA of k_scatter: elements of ten or more nodes (one CTA per SM when their
// tables fill the shared memory) take 512
template <int NN>
struct ScatterThreads {
  static constexpr int N = NN >= 10 ? 512 : 128;
};

template <int D, typename R, int NN = D + 1>
__global__ void __launch_bounds__(ScatterThreads<NN>::N)
    k_scatter(int64_t m_begin, int64_t p_begin, int64_t p_end, const int64_t* __restrict__ pair_off,
              const int32_t* __restrict__ pair_l, const int32_t* __restrict__ conn,
              const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
              const R* __restrict__ blk, const double* __restrict__ selfblk, int with_self,
              double* __restrict__ values, int* __restrict__ err) {
  const int64_t m = m_begin + blockIdx.x;
  int64_t q0 = 0, q1 = 0;
  if (!with_self) {
    q0 = max(pair_off[m], p_begin);
    q1 = min(pair_off[m + 1], p_end);
  }
  scatter_elem<D, R, NN>(m, q0, q1, p_begin, with_self != 0, pair_l, conn, row_ptr, col, blk, selfblk,
                     values, err);
}

// Launch shape of the assembly kernel: warps per CTA (0 = the most that fit in 110 KB of shared
// memory, at most 8; a requested count is lowered until it fits) and CTAs per SM (0 = as many
// as fit).
struct QShape {
  int warps = 0;
  int ctas_per_sm = 0;
};

template <int D, typename R, int KERN, bool DIRECT = false, bool BATCHED = false, int MMA = 0>
nl_status launch_quad(const QParams& P, cudaStream_t s, const QBatch& Bt = QBatch{nullptr, nullptr, 0, 0},
                      QShape shape = QShape{}) {
  int dev = 0;
  NL_CUDA(cudaGetDevice(&dev));
  int nsm = 0;
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t tbl = table_bytes<R>();
  const size_t per_warp = WarpMem<D, R>::bytes(P.scap) +
                          (BATCHED ? ((sizeof(QParams) + 15) & ~size_t(15)) : 0) +
                          mma_stage_bytes<D>(MMA);
  // default: at most 110 KB per CTA (two CTAs per SM); a requested shape may use up to 220 KB
  const size_t limit = (size_t)(shape.warps > 0 ? 220 : 110) * 1024;
  const int max_warps = QLaunch<D>::THREADS / 32;
  int warps = shape.warps > 0 ? std::min(shape.warps, max_warps) : max_warps;
  while (warps > 1 && tbl + warps * per_warp > limit) warps >>= 1;
  const int threads = warps * 32;
  const size_t smem = tbl + warps * per_warp;
  if (smem > (size_t)220 * 1024)
    return fail(NL_EINTERNAL, "assembly kernel needs %zu bytes of shared memory", smem);
  auto kern = k_quad<D, R, KERN, DIRECT, BATCHED, MMA>;
  NL_TRY(allow_smem(kern, smem));
  int per_sm = 0;
  NL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) return fail(NL_EINTERNAL, "assembly kernel does not fit on an SM (smem %zu)", smem);
  if (shape.ctas_per_sm > 0) per_sm = std::min(per_sm, shape.ctas_per_sm);
  kern<<<NL_CNT(nsm * per_sm), threads, smem, s>>>(P, Bt);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

template <int D, typename R, int NN = D + 1>
nl_status launch_scatter(nl_mesh* m, nl_pairs* p, int64_t p_begin, int64_t p_end, const R* blk,
                         const double* selfblk, int with_self, double* values, int* err,
                         cudaStream_t s, const int64_t* h_pair_off) {
  int64_t m_begin = 0, m_end = m->n_elem;
  if (!with_self) {
    // inner elements whose pairs intersect [p_begin, p_end)
    const int64_t* po = h_pair_off;
    m_begin = std::upper_bound(po, po + m->n_elem + 1, p_begin) - po - 1;
    m_end = std::lower_bound(po, po + m->n_elem + 1, p_end) - po;
    m_begin = std::max<int64_t>(0, m_begin);
    m_end = std::min<int64_t>(m->n_elem, std::max(m_end, m_begin));
  }
  if (m_end <= m_begin) return NL_OK;
  const size_t smem = scatter_smem_bytes(NN, p->max_row_nnz, sizeof(R));
  NL_TRY((allow_smem(k_scatter<D, R, NN>, smem)));
  k_scatter<D, R, NN><<<NL_CNT((unsigned)(m_end - m_begin)), ScatterThreads<NN>::N, smem, s>>>(
      m_begin, p_begin, p_end, p->pair_off, p->pair_l, m->conn, p->row_ptr, p->col, blk, selfblk,
      with_self, values, err);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}


// Checks the parameters of one assembly and fills the problem fields of P: mesh and pair
// arrays, the kernel gamma_eps (C_{delta,eps} times kappa, Sec. 2), the Algorithm 1 levels and
// the degree-5 rule.  The caller sets the pair range, the buffers and the work counter.
inline nl_status fill_qparams(const char* who, const nl_mesh* m, const nl_pairs* p,
                              const nl_kernel_params* kp, const nl_quad_params* qp,
                              nl_precision prec, QParams* P) {
  const int D = m->dim;
  if (!kp || !qp) return fail(NL_EINVAL, "%s: kernel or quadrature parameters are NULL", who);
  if (!(kp->eps > 0.0 && kp->eps < kp->delta)) return fail(NL_EINVAL, "%s: need 0 < eps < delta", who);
  if (kp->kernel != NL_KERNEL_CONST && kp->kernel != NL_KERNEL_TRUNC_GAUSS)
    return fail(NL_EINVAL, "%s: unknown kernel %d", who, kp->kernel);
  const int lmax_cap = D == 2 ? 12 : 9;
  if (qp->L_min < 1 || qp->L_max < qp->L_min || qp->L_max > lmax_cap)
    return fail(NL_EINVAL, "%s: need 1 <= L_min <= L_max <= %d", who, lmax_cap);
  if ((qp->rule & ~(NL_QUAD_COUNT_BAND | NL_QUAD_MINDIST_L2)) != 0)
    return fail(NL_EINVAL, "%s: only rule 0 is available", who);
  if (prec != NL_PREC_FP64 && prec != NL_PREC_FP32 && prec != NL_PREC_MIXED_TF32 &&
      prec != NL_PREC_MIXED_BF16)
    return fail(NL_EINVAL, "%s: unknown precision %d", who, (int)prec);
  memset(P, 0, sizeof *P);
  P->n_elem = m->n_elem;
  P->p_begin = 0;
  P->p_end = p->n_pairs;
  P->pair_off = p->pair_off;
  P->pair_l = p->pair_l;
  P->conn = m->conn;
  P->evert = m->evert;
  P->blo = m->blo;
  P->bhi = m->bhi;
  P->vol = m->vol;
  P->jinv = m->jinv;
  P->ef = m->ef;
  P->row_ptr = p->row_ptr;
  P->col = p->col;
  double C = kp->C_override > 0.0 ? kp->C_override
                                   : kernel_constant(D, kp->kernel, kp->delta, kp->eps);
  if (kp->kappa > 0.0) C *= kp->kappa;
  P->delta = kp->delta;
  P->dme = kp->delta - kp->eps;
  P->dpe = kp->delta + kp->eps;
  P->C = C;
  P->fC = (float)C;
  P->inv_eps = 1.0 / kp->eps;
  P->inv_delta2 = 1.0 / (kp->delta * kp->delta);
  P->fdme = (float)P->dme;
  P->fdpe = (float)P->dpe;
  P->fdme2 = (float)(P->dme * P->dme);
  P->fdpe2 = (float)(P->dpe * P->dpe);
  P->finv_delta2 = (float)P->inv_delta2;
  P->fmqe = (float)(-0.25 / kp->eps);
  P->ftqe = (float)(0.75 / kp->eps);
  P->fue = (float)(0.5 * (1.0 - kp->delta / kp->eps));
  // bound on |local coordinates| and on the FP32 error of the screened distances
  P->margin = (float)(2e-5 * (kp->delta + kp->eps + 2.0 * m->max_ext));
  {
    const double lo_t = (double)P->fdme - (double)P->margin, hi_t = (double)P->fdme + (double)P->margin;
    P->fint2 = lo_t > 0.0 ? (float)(lo_t * lo_t) : -1.f;
    P->fnotint2 = (float)(hi_t * hi_t);
  }
  P->L_min = qp->L_min;
  P->L_max = qp->L_max;
  P->count_band = (qp->rule & NL_QUAD_COUNT_BAND) ? 1 : 0;
  P->mindist_l2 = (qp->rule & NL_QUAD_MINDIST_L2) ? 1 : 0;
  {
    // the Euclidean screen: sqrt(dim) <= 2 times the per-axis error bound, squared
    const double lo_r = (double)P->fdpe - 2.0 * (double)P->margin;
    const double hi_r = (double)P->fdpe + 2.0 * (double)P->margin;
    P->fref2 = lo_r > 0.0 ? (float)(lo_r * lo_r) : -1.f;
    P->fout2 = (float)(hi_r * hi_r);
  }
  P->kernel = kp->kernel;
  P->chunk = CHUNK;
  // parent records the LIFO can hold: all sub-elements of levels 1 .. L_max-1 (at most 512)
  int64_t total = 0, pw = 1;
  for (int k = 1; k < qp->L_max; k++) {
    total += pw;
    pw *= (D == 2 ? 4 : 8);
    if (total > 512) break;
  }
  P->scap = (int)std::max<int64_t>(8, std::min<int64_t>(total, 512));
  const Rule& r = rule(D);
  for (int q = 0; q < r.n; q++) {
    for (int a = 0; a <= D; a++) P->B[q][a] = r.bary[q][a];
    P->W[q] = r.w[q];
  }
  return NL_OK;
}

// ---- single-problem assembly (nl_assemble) --------------------------------------------------
// CUDA events around every launch of the assembly kernel and of the scatter, read after the
// assembly's final synchronisation.
struct PhaseTimer {
  std::vector<cudaEvent_t> ev[2];
  ~PhaseTimer() {
    for (auto& v : ev)
      for (cudaEvent_t e : v) cudaEventDestroy(e);
  }
  nl_status mark(int phase, cudaStream_t s) {
    cudaEvent_t e;
    NL_CUDA(cudaEventCreate(&e));
    ev[phase].push_back(e);
    NL_CUDA(cudaEventRecord(e, s));
    return NL_OK;
  }
  // summed elapsed time of the (start, end) pairs of one phase, after synchronisation
  double ms(int phase) const {
    double t = 0.0;
    for (size_t i = 0; i + 1 < ev[phase].size(); i += 2) {
      float x = 0.f;
      if (cudaEventElapsedTime(&x, ev[phase][i], ev[phase][i + 1]) == cudaSuccess) t += x;
    }
    return t;
  }
  int launches(int phase) const { return (int)(ev[phase].size() / 2); }
};

template <int D, typename R, int KERN, int MMA>
nl_status run_assembly(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s,
                       unsigned long long* scratch, int* err, PhaseTimer& T) {
  const int NB = (D + 1) * (D + 1);
  // the block buffer holds the cross blocks of one batch of pairs
  size_t free_b = 0, total_b = 0;
  NL_CUDA(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = std::min<size_t>((size_t)8 << 30, free_b / 4);
  if (g_block_budget) budget = std::min(budget, g_block_budget);
  int64_t batch = std::max<int64_t>(1 << 20, (int64_t)(budget / (sizeof(R) * NB)));
  batch = std::min<int64_t>(batch, p->n_pairs);
  DevBuf<R> blk;
  DevBuf<double> selfblk;
  NL_TRY(blk.alloc((size_t)batch * NB, s));
  NL_TRY(selfblk.alloc((size_t)m->n_elem * NB, s));
  NL_CUDA(cudaMemsetAsync(selfblk.p, 0, sizeof(double) * m->n_elem * NB, s));
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
    NL_TRY((launch_quad<D, R, KERN, false, false, MMA>(P, s)));
    NL_TRY(T.mark(0, s));
    NL_TRY(T.mark(1, s));
    NL_TRY((launch_scatter<D, R>(m, p, b0, b1, blk.p, nullptr, 0, values, err, s, h_off.data())));
    NL_TRY(T.mark(1, s));
  }
  NL_TRY(T.mark(1, s));
  NL_TRY((launch_scatter<D, R>(m, p, 0, 0, blk.p, selfblk.p, 1, values, err, s, h_off.data())));
  NL_TRY(T.mark(1, s));
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}

// One problem (nl_assemble): the batches of pairs through the assembly kernel, each followed
// by the scatter of its cross blocks, then the self blocks (and, in FP32, the diagonals from
// the row sums).  MMA = 0: FP64 or FP32 point-pair arithmetic by prec; 1 / 2: the FP32 path
// with the contraction on the tensor cores in TF32 / BF16.
template <int MMA>
nl_status assemble_single(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                          const nl_quad_params* qp, nl_precision prec, double* values,
                          nl_assemble_stats* st) {
  QParams P;
  NL_TRY(fill_qparams("nl_assemble", m, p, kp, qp, prec, &P));
  const int D = m->dim;
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
    if constexpr (MMA != 0) {
      if (D == 2) rc = gauss ? run_assembly<2, float, 1, MMA>(m, p, P, values, s, scratch.p, err.p, T)
                             : run_assembly<2, float, 0, MMA>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly<3, float, 1, MMA>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly<3, float, 0, MMA>(m, p, P, values, s, scratch.p, err.p, T);
    } else if (D == 2) {
      if (f32) rc = gauss ? run_assembly<2, float, 1, 0>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly<2, float, 0, 0>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly<2, double, 1, 0>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly<2, double, 0, 0>(m, p, P, values, s, scratch.p, err.p, T);
    } else {
      if (f32) rc = gauss ? run_assembly<3, float, 1, 0>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly<3, float, 0, 0>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly<3, double, 1, 0>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly<3, double, 0, 0>(m, p, P, values, s, scratch.p, err.p, T);
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
    const int nq = D == 2 ? 7 : 14;
    st->n_pairs = p->n_pairs;
    st->n_items = (int64_t)hs[1];
    st->n_point_pairs = (int64_t)hs[1] * nq * nq;
    st->n_exact_checks = (int64_t)hs[3];
    st->ms_assemble = ms;
    st->n_eval_point_pairs = (int64_t)hs[4];
    st->n_closed_items = (int64_t)hs[5];
    st->n_band_point_pairs = P.count_band ? (int64_t)hs[6] : -1;
    st->precision_run = MMA == 1 ? NL_PREC_MIXED_TF32
                        : MMA == 2 ? NL_PREC_MIXED_BF16
                        : (f32 ? NL_PREC_FP32 : NL_PREC_FP64);
    st->n_quad_launches = T.launches(0);
    st->ms_quad = T.ms(0);
    st->ms_scatter = T.ms(1);
  }
  return NL_OK;
}

}  // namespace
}  // namespace nlx
