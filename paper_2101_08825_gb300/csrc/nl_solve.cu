// nl_solve.cu -- right-hand side with lifting and the Krylov solvers for A_{free,free} W = F~.
//
// Sec. 2 (eqs. A-F, weak-homo) and Sec. 4: the unknowns are the nodes inside Omega; the
// volume constraint u = g on Gamma is moved to the right-hand side through the lifting
// u = w + g~.  A is nonsymmetric at the quadrature-error level when L_max > 1 (the outer rule
// of Algorithm 1 depends on the pair), so BiCGStab is offered next to CG.  Vectors span all
// nodes; constrained entries of the Krylov vectors stay zero and the SpMV skips them.
//
// All Krylov scalars live on the device: every dot product is reduced inside the kernel
// that produces its operands (per-block partial sums; the last block to finish adds them
// in a fixed order and computes the next scalar), so an iteration is a handful of kernel
// launches with no host round trip; the host reads the residual every CHECK iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "nl_internal.h"

namespace nlx {
namespace {

constexpr int RT = 256;    // block size of the vector kernels
constexpr int RTR = 1024;  // block size of the row (SpMV) kernels: few large blocks, so that
                           // the blocks' partial sums serialise on few atomic tickets
constexpr int CHECK = 8;   // iterations between host convergence checks

// scalar slots (double) shared by the solver kernels
enum : int {
  S_RHO_NEW = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_RR, S_BB, S_RR_OLD, S_BREAK, S_NSLOTS = 16
};
constexpr int NPARTS = 2;  // dot products that one kernel can reduce

// F_i += int_E f phi_i per element of Omega with NB nodes (P1: D+1, P2 triangles 6, P2
// tetrahedra 10); B[q][a] (row stride 16) is the element basis phi_a at rule point q.
template <int NB>
__global__ void k_rhs_elems(int64_t n_elem, const int32_t* __restrict__ conn,
                            const uint8_t* __restrict__ eio, const uint8_t* __restrict__ free_,
                            const double* __restrict__ vol, const double* __restrict__ fn,
                            double f_const, const double* __restrict__ B,
                            const double* __restrict__ W, int nq, double* __restrict__ F) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem || !eio[e]) return;
  int32_t nd[NB];
  double fv[NB];
  for (int a = 0; a < NB; a++) {
    nd[a] = conn[e * NB + a];
    fv[a] = fn ? fn[nd[a]] : 0.0;
  }
  double acc[NB];
  for (int a = 0; a < NB; a++) acc[a] = 0.0;
  for (int q = 0; q < nq; q++) {
    double f = f_const;
    for (int v = 0; v < NB; v++) f += B[q * 16 + v] * fv[v];
    for (int a = 0; a < NB; a++) acc[a] += W[q] * f * B[q * 16 + a];
  }
  for (int a = 0; a < NB; a++)
    if (free_[nd[a]]) atomicAdd(&F[nd[a]], vol[e] * acc[a]);
}

// F_i += int_E f phi_i per quadrilateral of Omega with NB nodes (Q1 4, serendipity 8, Q2 9): Gauss-Legendre
// 3x3 on the unit square mapped by the element's bilinear map; S[q] = (s, t, weight) and
// B[q][a] (row stride 16) the basis at point q.
template <int NB>
__global__ void k_rhs_quads(int64_t n_elem, const int32_t* __restrict__ conn,
                            const uint8_t* __restrict__ eio, const uint8_t* __restrict__ free_,
                            const double* __restrict__ evert, const double* __restrict__ fn,
                            double f_const, const double* __restrict__ B,
                            const double* __restrict__ S, double* __restrict__ F) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem || !eio[e]) return;
  int32_t nd[NB];
  double fv[NB], acc[NB];
  for (int a = 0; a < NB; a++) {
    nd[a] = conn[e * NB + a];
    fv[a] = fn ? fn[nd[a]] : 0.0;
    acc[a] = 0.0;
  }
  double V[4][2];
  for (int a = 0; a < 4; a++)
    for (int k = 0; k < 2; k++) V[a][k] = evert[(e * 4 + a) * 2 + k];
  for (int q = 0; q < 9; q++) {
    const double s = S[q * 3], t = S[q * 3 + 1];
    double xs[2], xt[2];
    for (int k = 0; k < 2; k++) {
      xs[k] = (1.0 - t) * (V[1][k] - V[0][k]) + t * (V[2][k] - V[3][k]);
      xt[k] = (1.0 - s) * (V[3][k] - V[0][k]) + s * (V[2][k] - V[1][k]);
    }
    const double w = S[q * 3 + 2] * fabs(xs[0] * xt[1] - xs[1] * xt[0]);
    double f = f_const;
    for (int v = 0; v < NB; v++) f += B[q * 16 + v] * fv[v];
    for (int a = 0; a < NB; a++) acc[a] += w * f * B[q * 16 + a];
  }
  for (int a = 0; a < NB; a++)
    if (free_[nd[a]]) atomicAdd(&F[nd[a]], acc[a]);
}

// F_i += int_E f phi_i per hexahedron of Omega (Q1, NB = 8, Q2, NB = 27, or serendipity,
// NB = 20; f interpolated in the element space): Gauss-Legendre 3x3x3 on the unit cube mapped by the element's trilinear
// map; G = the 3 points and weights on [0, 1].
template <int NB>
__global__ void k_rhs_hexes(int64_t n_elem, const int32_t* __restrict__ conn,
                            const uint8_t* __restrict__ eio, const uint8_t* __restrict__ free_,
                            const double* __restrict__ evert, const double* __restrict__ fn,
                            double f_const, const double* __restrict__ G, double* __restrict__ F) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem || !eio[e]) return;
  int32_t nd[NB];
  double fv[NB], acc[NB], V[8][3];
  for (int a = 0; a < NB; a++) {
    nd[a] = conn[e * NB + a];
    fv[a] = fn ? fn[nd[a]] : 0.0;
    acc[a] = 0.0;
  }
  for (int a = 0; a < 8; a++)
    for (int k = 0; k < 3; k++) V[a][k] = evert[(e * 8 + a) * 3 + k];
  for (int q = 0; q < 27; q++) {
    const double s = G[q / 9], t = G[(q / 3) % 3], u = G[q % 3];
    const double w = G[3 + q / 9] * G[3 + (q / 3) % 3] * G[3 + q % 3];
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 8; a++) {
      const int c = hex27_code(a);
      const bool bx = c % 3, by = (c / 3) % 3, bz = c / 9;
      const double fs = bx ? s : 1.0 - s, ft = by ? t : 1.0 - t, fu = bz ? u : 1.0 - u;
      const double ds = bx ? 1.0 : -1.0, dt = by ? 1.0 : -1.0, du = bz ? 1.0 : -1.0;
      for (int k = 0; k < 3; k++) {
        J[k][0] += ds * ft * fu * V[a][k];
        J[k][1] += fs * dt * fu * V[a][k];
        J[k][2] += fs * ft * du * V[a][k];
      }
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double phi[NB];
    hex_basis<NB, double>(s, t, u, 1.0, phi);
    double f = f_const;
    for (int a = 0; a < NB; a++) f += phi[a] * fv[a];
    for (int a = 0; a < NB; a++) acc[a] += w * fabs(det) * f * phi[a];
  }
  for (int a = 0; a < NB; a++)
    if (free_[nd[a]]) atomicAdd(&F[nd[a]], acc[a]);
}

__global__ void k_lift(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const uint8_t* __restrict__ free_,
                       const double* __restrict__ g, double* __restrict__ F) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  if (!free_[i]) {
    if (lane == 0) F[i] = 0.0;
    return;
  }
  double s = 0.0;
  for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) {
    int32_t j = col[t];
    if (!free_[j]) s += val[t] * g[j];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) F[i] -= s;
}

// ---- reduction helpers ---------------------------------------------------------------------------
struct Red {
  double* part;       // [NPARTS][max_blocks] partial sums
  unsigned* done;     // blocks finished, reset by the last one
  double* S;          // scalar slots
  int max_blocks;
};

// Block-reduces K values; the last block of the grid sums every block's partials in block
// order and returns true in thread 0 with the totals in tot[].  BS: the largest block size
// the calling kernel is launched with (blockDim.x <= BS).
template <int K, int BS = RT>
__device__ bool reduce_last(const Red& R, double (&v)[K], double (&tot)[K]) {
  __shared__ double ws[K][BS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) ws[k][w] = x;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      double t = lane < (int)(blockDim.x >> 5) ? ws[k][lane] : 0.0;  // warps of this launch
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) R.part[k * R.max_blocks + blockIdx.x] = t;
    }
    if (lane == 0) {
      __threadfence();
      const unsigned ticket = atomicAdd(R.done, 1u);
      last = ticket == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // last block: fixed-order sum of the partials (every thread strides over the blocks, then a
  // fixed tree over the threads)
  if (w != 0) return false;
#pragma unroll
  for (int k = 0; k < K; k++) {
    double t = 0.0;
    for (int j = lane; j < (int)gridDim.x; j += 32) t += ((volatile double*)R.part)[k * R.max_blocks + j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    tot[k] = t;
  }
  if (lane != 0) return false;
  *R.done = 0;
  return true;
}

__device__ __forceinline__ double safe_div(double a, double b, double* brk) {
  if (b == 0.0 || !isfinite(b)) {
    *brk = 1.0;
    return 0.0;
  }
  return a / b;
}

// y = A x on free rows (0 elsewhere; every row when free_ is NULL), warp per row, grid-stride
// over the rows; four
// independent partial sums keep four loads of x in flight per lane.  No reduction here, so the
// grid can fill every SM; the dot products follow in k_spmv_dots.
template <typename X, typename V>
__global__ void __launch_bounds__(RT) k_spmv(int64_t n, const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ col,
                                             const V* __restrict__ val,
                                             const uint8_t* __restrict__ free_,
                                             const X* __restrict__ x, X* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    X s = 0;
    if (!free_ || free_[i]) {
      const int64_t e = rp[i + 1];
      int64_t t = rp[i] + lane;
      X s1 = 0, s2 = 0, s3 = 0;
      for (; t + 96 < e; t += 128) {
        s += (X)val[t] * x[col[t]];
        s1 += (X)val[t + 32] * x[col[t + 32]];
        s2 += (X)val[t + 64] * x[col[t + 64]];
        s3 += (X)val[t + 96] * x[col[t + 96]];
      }
      for (; t < e; t += 32) s += (X)val[t] * x[col[t]];
      s = (s + s1) + (s2 + s3);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[i] = s;
  }
}

// The dot products that follow y = A x, and the scalar they determine:
//   MODE 0 (BiCGStab v = A p): (r^, v) -> alpha = rho_new / (r^, v), rho_old = rho_new
//   MODE 1 (BiCGStab t = A s): (t, s), (t, t) -> omega = (t, s) / (t, t)
//   MODE 2 (CG q = A p):       (p, q) -> alpha = rr / (p, q)
template <typename X, int MODE>
__global__ void __launch_bounds__(RT) k_spmv_dots(int64_t n, const X* __restrict__ x,
                                                  const X* __restrict__ y,
                                                  const X* __restrict__ w1, Red R) {
  double d[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = (double)y[i];
    if (MODE == 0) d[0] += (double)w1[i] * s;
    if (MODE == 1) {
      d[0] += s * (double)x[i];
      d[1] += s * s;
    }
    if (MODE == 2) d[0] += (double)x[i] * s;
  }
  double tot[2];
  if (reduce_last<2>(R, d, tot)) {
    double* S = R.S;
    if (MODE == 0) {
      S[S_ALPHA] = safe_div(S[S_RHO_NEW], tot[0], &S[S_BREAK]);
      S[S_RHO_OLD] = S[S_RHO_NEW];
    } else if (MODE == 1) {
      S[S_OMEGA] = safe_div(tot[0], tot[1], &S[S_BREAK]);
    } else {
      S[S_ALPHA] = safe_div(S[S_RR], tot[0], &S[S_BREAK]);
    }
  }
}

// BiCGStab p = r + beta (p - omega v), beta = (rho_new / rho_old) (alpha / omega)
template <typename X>
__global__ void __launch_bounds__(RT) k_bicg_p(int64_t n, const X* __restrict__ r,
                                               const X* __restrict__ v, X* __restrict__ p,
                                               const double* __restrict__ S) {
  const double om = S[S_OMEGA];
  const double beta = (S[S_RHO_OLD] != 0.0 && om != 0.0)
                          ? (S[S_RHO_NEW] / S[S_RHO_OLD]) * (S[S_ALPHA] / om) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + (X)beta * (p[i] - (X)om * v[i]);
}

// BiCGStab s = r - alpha v
template <typename X>
__global__ void __launch_bounds__(RT) k_bicg_s(int64_t n, const X* __restrict__ r,
                                               const X* __restrict__ v, X* __restrict__ sv,
                                               const double* __restrict__ S) {
  const X a = (X)S[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sv[i] = r[i] - a * v[i];
}

// BiCGStab x += alpha p + omega s; r = s - omega t; (r, r) and (r^, r)
template <typename X>
__global__ void __launch_bounds__(RT) k_bicg_xr(int64_t n, X* __restrict__ x, const X* __restrict__ p,
                                                const X* __restrict__ sv, const X* __restrict__ t,
                                                X* __restrict__ r, const X* __restrict__ rh, Red R) {
  double d[2] = {0.0, 0.0};
  const X a = (X)R.S[S_ALPHA], om = (X)R.S[S_OMEGA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i] + om * sv[i];
    const X ri = sv[i] - om * t[i];
    r[i] = ri;
    d[0] += (double)ri * (double)ri;
    d[1] += (double)rh[i] * (double)ri;
  }
  double tot[2];
  if (reduce_last<2>(R, d, tot)) {
    R.S[S_RR] = tot[0];
    R.S[S_RHO_NEW] = tot[1];
  }
}

// CG x += alpha p; r -= alpha q; (r, r); keeps the previous (r, r) for beta
template <typename X>
__global__ void __launch_bounds__(RT) k_cg_xr(int64_t n, X* __restrict__ x, const X* __restrict__ p,
                                              const X* __restrict__ q, X* __restrict__ r, Red R) {
  double d[2] = {0.0, 0.0};
  const X a = (X)R.S[S_ALPHA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    const X ri = r[i] - a * q[i];
    r[i] = ri;
    d[0] += (double)ri * (double)ri;
  }
  double tot[2];
  if (reduce_last<2>(R, d, tot)) {
    R.S[S_RR_OLD] = R.S[S_RR];
    R.S[S_RR] = tot[0];
  }
}

// CG p = r + beta p, beta = (r, r) / (r, r)_old
template <typename X>
__global__ void __launch_bounds__(RT) k_cg_p(int64_t n, const X* __restrict__ r, X* __restrict__ p,
                                             const double* __restrict__ S) {
  const double beta = S[S_RR_OLD] != 0.0 ? S[S_RR] / S[S_RR_OLD] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + (X)beta * p[i];
}

// r = b - A u (FP64) on free rows, its FP32 copy (optional) and (r, r)
__global__ void __launch_bounds__(RTR) k_residual(int64_t n, const int64_t* __restrict__ rp,
                                                 const int32_t* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const uint8_t* __restrict__ free_,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ b, double* __restrict__ r,
                                                 float* __restrict__ r32, Red R) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[2] = {0.0, 0.0};
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    double s = 0.0;
    if (free_[i])
      for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += val[t] * u[col[t]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const double ri = free_[i] ? b[i] - s : 0.0;
      r[i] = ri;
      if (r32) r32[i] = (float)ri;
      d[0] += ri * ri;
    }
  }
  double tot[2];
  if (reduce_last<2, RTR>(R, d, tot)) R.S[S_RR] = tot[0];
}

// (a, a) of the right-hand side; initialises the scalar slots
template <typename X>
__global__ void __launch_bounds__(RT) k_init_dot(int64_t n, const X* __restrict__ a, Red R) {
  double d[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[0] += (double)a[i] * (double)a[i];
  double tot[2];
  if (reduce_last<2>(R, d, tot)) {
    double* S = R.S;
    S[S_BB] = tot[0];
    S[S_RR] = tot[0];
    S[S_RHO_NEW] = tot[0];
    S[S_RHO_OLD] = 1.0;
    S[S_ALPHA] = 1.0;
    S[S_OMEGA] = 1.0;
    S[S_RR_OLD] = 0.0;
    S[S_BREAK] = 0.0;
  }
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_add_f32_to_f64(int64_t n, const float* __restrict__ d, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] += (double)d[i];
}

struct Ctx {
  cudaStream_t s;
  int64_t n;
  const int64_t* rp;
  const int32_t* col;
  const uint8_t* free_;
  Red R;
  // grids: one block per SM at most for the kernels with a reduction (their partial sums
  // serialise on one atomic ticket); the row kernels use 1024-thread blocks (32 warps per SM)
  int cap = 152;
  unsigned gvec() const { return (unsigned)std::min<int64_t>(cap, (n + 4 * RT - 1) / (4 * RT)); }
  unsigned grow() const { return (unsigned)std::min<int64_t>(cap, (n * 32 + RTR - 1) / RTR); }
  // SpMV without a reduction: up to 8 blocks of 256 threads per SM
  unsigned gspmv() const { return (unsigned)std::min<int64_t>(8 * cap, (n * 32 + RT - 1) / RT); }
};

nl_status read_scalars(Ctx& c, double* h) {
  NL_CUDA(cudaMemcpyAsync(h, c.R.S, sizeof(double) * S_NSLOTS, cudaMemcpyDeviceToHost, c.s));
  NL_CUDA(cudaStreamSynchronize(c.s));
  return NL_OK;
}

// Krylov vectors of one solve (allocated once, so that every Krylov call of an iterative
// refinement uses the same pointers) and the CUDA graph of one batch of CHECK iterations,
// captured at the first full batch and replayed for every later one.  Graphs are used only
// on a stream that can be captured (not the legacy default stream).
template <typename X>
struct KWork {
  DevBuf<X> r, rh, p, v, sv, t;
  cudaGraphExec_t exec = nullptr;
  int exec_solver = -1;
  bool use_graph = false;
  ~KWork() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  nl_status alloc(int64_t n, cudaStream_t s) {
    NL_TRY(r.alloc(n, s));
    NL_TRY(rh.alloc(n, s));
    NL_TRY(p.alloc(n, s));
    NL_TRY(v.alloc(n, s));
    NL_TRY(sv.alloc(n, s));
    NL_TRY(t.alloc(n, s));
    return NL_OK;
  }
};

// One iteration of CG (solver 0) or BiCGStab (solver 1).
template <typename X, typename V>
void krylov_iteration(Ctx& c, const V* val, int solver, X* x, KWork<X>& W) {
  const int64_t n = c.n;
  if (solver == 0) {
    k_spmv<X, V><<<NL_CNT(c.gspmv()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, W.p.p, W.v.p);
    k_spmv_dots<X, 2><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.p.p, W.v.p, nullptr, c.R);
    k_cg_xr<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, x, W.p.p, W.v.p, W.r.p, c.R);
    k_cg_p<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.r.p, W.p.p, c.R.S);
  } else {
    k_bicg_p<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.r.p, W.v.p, W.p.p, c.R.S);
    k_spmv<X, V><<<NL_CNT(c.gspmv()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, W.p.p, W.v.p);
    k_spmv_dots<X, 0><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.p.p, W.v.p, W.rh.p, c.R);
    k_bicg_s<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.r.p, W.v.p, W.sv.p, c.R.S);
    k_spmv<X, V><<<NL_CNT(c.gspmv()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, W.sv.p, W.t.p);
    k_spmv_dots<X, 1><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, W.sv.p, W.t.p, nullptr, c.R);
    k_bicg_xr<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, x, W.p.p, W.sv.p, W.t.p, W.r.p, W.rh.p, c.R);
  }
}

// A batch of `batch` iterations: replayed from the captured graph when it is a full batch and
// graphs are in use, launched kernel by kernel otherwise.
template <typename X, typename V>
nl_status krylov_batch(Ctx& c, const V* val, int solver, X* x, KWork<X>& W, int batch) {
  if (W.use_graph && batch == CHECK) {
    if (!W.exec || W.exec_solver != solver) {
      if (W.exec) {
        cudaGraphExecDestroy(W.exec);
        W.exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int j = 0; j < CHECK; j++) krylov_iteration<X, V>(c, val, solver, x, W);
        e = cudaStreamEndCapture(c.s, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&W.exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {  // run without graphs from here on
        cudaGetLastError();
        W.exec = nullptr;
        W.use_graph = false;
      } else {
        W.exec_solver = solver;
      }
    }
    if (W.exec) {
      NL_CUDA(cudaGraphLaunch(W.exec, c.s));
      for (int j = 0; j < CHECK * (solver == 0 ? 4 : 7); j++) count_launch();
      return NL_OK;
    }
  }
  for (int j = 0; j < batch; j++) krylov_iteration<X, V>(c, val, solver, x, W);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

// Krylov solve of A x = b (x starts at 0) to ||b - A x|| <= tol ||b||.  X = double or float
// (vectors), V = matrix value type.  *it = iterations, *ok when converged.
template <typename X, typename V>
nl_status krylov(Ctx& c, const V* val, int solver, const X* b, X* x, double tol, int max_it, int* it,
                 bool* ok, double* relres, KWork<X>& W) {
  const int64_t n = c.n;
  NL_CUDA(cudaMemsetAsync(x, 0, sizeof(X) * n, c.s));
  NL_CUDA(cudaMemcpyAsync(W.r.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
  k_init_dot<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, b, c.R);
  NL_CUDA(cudaGetLastError());
  double h[S_NSLOTS];
  NL_TRY(read_scalars(c, h));
  const double bb = h[S_BB];
  *it = 0;
  *ok = false;
  *relres = 0.0;
  if (bb == 0.0) {
    *ok = true;
    return NL_OK;
  }
  const double stop2 = tol * tol * bb;
  if (solver == 0) {  // CG: p = r = b
    NL_CUDA(cudaMemcpyAsync(W.p.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
  } else {  // BiCGStab (van der Vorst): r^ = b, p = v = 0, rho_new = (r^, r)
    NL_CUDA(cudaMemcpyAsync(W.rh.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
    NL_CUDA(cudaMemsetAsync(W.p.p, 0, sizeof(X) * n, c.s));
    NL_CUDA(cudaMemsetAsync(W.v.p, 0, sizeof(X) * n, c.s));
  }
  int k = 0;
  while (k < max_it) {
    const int batch = std::min(CHECK, max_it - k);
    NL_TRY((krylov_batch<X, V>(c, val, solver, x, W, batch)));
    k += batch;
    NL_TRY(read_scalars(c, h));
    *it = k;
    *relres = std::sqrt(std::max(h[S_RR], 0.0) / bb);
    if (h[S_RR] <= stop2) {
      *ok = true;
      break;
    }
    if (h[S_BREAK] != 0.0 || !std::isfinite(h[S_RR])) break;
  }
  return NL_OK;
}

}  // namespace

nl_status rhs_values(nl_mesh* m, nl_matrix* A, const double* f_nodes, double f_const,
                     const double* g_nodes, double* F) {
  cudaStream_t s = m->stream;
  const int D = m->dim;
  const Rule& r = rule(D);
  // the element basis at the rule points: P1 the barycentric coordinates; P2 (triangles)
  // lambda_a (2 lambda_a - 1) at the vertices and 4 lambda_a lambda_b at the edge nodes
  // (0,1), (1,2), (0,2)
  std::vector<double> hB(16 * 16, 0.0), hW(16, 0.0);
  static const int ea[6] = {0, 1, 0, 0, 1, 2}, eb[6] = {1, 2, 2, 3, 3, 3};
  for (int q = 0; q < r.n; q++) {
    const double* lam = r.bary[q];
    if (m->order == 2) {
      for (int a = 0; a <= D; a++) hB[q * 16 + a] = lam[a] * (2.0 * lam[a] - 1.0);
      for (int j = 0; j < (D == 2 ? 3 : 6); j++) hB[q * 16 + D + 1 + j] = 4.0 * lam[ea[j]] * lam[eb[j]];
    } else {
      for (int a = 0; a <= D; a++) hB[q * 16 + a] = lam[a];
    }
    hW[q] = r.w[q];
  }
  DevBuf<double> B, W, fn, g;
  NL_TRY(B.alloc(256, s));
  NL_TRY(W.alloc(16, s));
  NL_TRY(g.alloc(m->n_vert, s));
  NL_CUDA(cudaMemcpyAsync(B.p, hB.data(), sizeof(double) * 256, cudaMemcpyHostToDevice, s));
  NL_CUDA(cudaMemcpyAsync(W.p, hW.data(), sizeof(double) * 16, cudaMemcpyHostToDevice, s));
  NL_CUDA(cudaMemcpyAsync(g.p, g_nodes, sizeof(double) * m->n_vert, cudaMemcpyHostToDevice, s));
  if (f_nodes) {
    NL_TRY(fn.alloc(m->n_vert, s));
    NL_CUDA(cudaMemcpyAsync(fn.p, f_nodes, sizeof(double) * m->n_vert, cudaMemcpyHostToDevice, s));
  }
  NL_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * m->n_vert, s));
  unsigned ge = (unsigned)((m->n_elem + RT - 1) / RT);
  DevBuf<double> QB, QS;
  if (m->cell == 1) {
    // Gauss-Legendre 3x3 points (s, t, weight) and the Q1 / Q2 basis there
    std::vector<double> hq(9 * 16, 0.0), hs(27, 0.0);
    const GL3& g = gl3();
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        const int q = 3 * i + j;
        hs[q * 3] = g.g[i];
        hs[q * 3 + 1] = g.g[j];
        hs[q * 3 + 2] = g.w[i] * g.w[j];
        quad_basis<double>(m->order, g.g[i], g.g[j], &hq[q * 16]);
      }
    NL_TRY(QB.alloc(9 * 16, s));
    NL_TRY(QS.alloc(27, s));
    NL_CUDA(cudaMemcpyAsync(QB.p, hq.data(), sizeof(double) * 9 * 16, cudaMemcpyHostToDevice, s));
    NL_CUDA(cudaMemcpyAsync(QS.p, hs.data(), sizeof(double) * 27, cudaMemcpyHostToDevice, s));
  }
  DevBuf<double> HG;
  if (m->cell == 2) {
    const GL3& g = gl3();
    double hg[6] = {g.g[0], g.g[1], g.g[2], g.w[0], g.w[1], g.w[2]};
    NL_TRY(HG.alloc(6, s));
    NL_CUDA(cudaMemcpyAsync(HG.p, hg, sizeof hg, cudaMemcpyHostToDevice, s));
    NL_CUDA(cudaStreamSynchronize(s));  // hg lives on this stack frame
  }
  if (m->cell == 2 && m->nb == 27)
    k_rhs_hexes<27><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                              m->evert, fn.p, f_const, HG.p, F);
  else if (m->cell == 2 && m->nb == 20)
    k_rhs_hexes<20><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                              m->evert, fn.p, f_const, HG.p, F);
  else if (m->cell == 2)
    k_rhs_hexes<8><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->evert, fn.p, f_const, HG.p, F);
  else if (m->cell == 1 && m->nb == 9)
    k_rhs_quads<9><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->evert, fn.p, f_const, QB.p, QS.p, F);
  else if (m->cell == 1 && m->nb == 8)
    k_rhs_quads<8><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->evert, fn.p, f_const, QB.p, QS.p, F);
  else if (m->cell == 1)
    k_rhs_quads<4><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->evert, fn.p, f_const, QB.p, QS.p, F);
  else if (m->nb == 10)
    k_rhs_elems<10><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                              m->vol, fn.p, f_const, B.p, W.p, r.n, F);
  else if (m->nb == 6)
    k_rhs_elems<6><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->vol, fn.p, f_const, B.p, W.p, r.n, F);
  else if (D == 2)
    k_rhs_elems<3><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->vol, fn.p, f_const, B.p, W.p, r.n, F);
  else
    k_rhs_elems<4><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free,
                                             m->vol, fn.p, f_const, B.p, W.p, r.n, F);
  k_lift<<<NL_CNT((unsigned)((m->n_vert * 32 + RT - 1) / RT)), RT, 0, s>>>(
      m->n_vert, A->pairs->row_ptr, A->pairs->col, A->values, m->node_free, g.p, F);
  NL_CUDA(cudaGetLastError());
  NL_CUDA(cudaStreamSynchronize(s));
  return NL_OK;
}

nl_status apply_matrix(const nl_matrix* A, const double* x, double* y) {
  const nl_mesh* m = A->pairs->mesh;
  Ctx c;
  c.s = A->stream;
  c.n = m->n_vert;
  int dev = 0, nsm = 0;
  NL_CUDA(cudaGetDevice(&dev));
  NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  c.cap = std::max(1, nsm);
  if (c.n == 0) return NL_OK;
  k_spmv<double, double><<<NL_CNT(c.gspmv()), RT, 0, c.s>>>(c.n, A->pairs->row_ptr, A->pairs->col,
                                                           A->values, nullptr, x, y);
  NL_CUDA(cudaGetLastError());
  return NL_OK;
}

nl_status solve_system(nl_matrix* A, const nl_vector* rhs, const double* g_nodes, int solver,
                       double rtol, int max_iter, nl_precision prec, double* u_out, int* iters,
                       double* rel_res) {
  nl_mesh* m = A->pairs->mesh;
  cudaStream_t s = m->stream;
  Ctx c;
  c.s = s;
  c.n = m->n_vert;
  c.rp = A->pairs->row_ptr;
  c.col = A->pairs->col;
  c.free_ = m->node_free;
  {
    int dev = 0, nsm = 0;
    NL_CUDA(cudaGetDevice(&dev));
    NL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    c.cap = std::max(1, nsm);
  }
  const int max_blocks = (int)std::max<int64_t>(c.grow(), c.gvec());
  DevBuf<double> part, S, x;
  DevBuf<unsigned> done;
  NL_TRY(part.alloc((size_t)NPARTS * max_blocks, s));
  NL_TRY(S.alloc(S_NSLOTS, s));
  NL_TRY(done.alloc(1, s));
  NL_TRY(x.alloc(c.n, s));
  NL_CUDA(cudaMemsetAsync(done.p, 0, sizeof(unsigned), s));
  NL_CUDA(cudaMemsetAsync(S.p, 0, sizeof(double) * S_NSLOTS, s));
  c.R.part = part.p;
  c.R.done = done.p;
  c.R.S = S.p;
  c.R.max_blocks = max_blocks;
  int it = 0;
  bool ok = false;
  double rr = 0.0;
  const bool graphs = s != nullptr;  // the legacy default stream cannot be captured
  if (prec == NL_PREC_FP64) {
    KWork<double> W;
    NL_TRY(W.alloc(c.n, s));
    W.use_graph = graphs;
    NL_TRY((krylov<double, double>(c, A->values, solver, rhs->v, x.p, rtol, max_iter, &it, &ok, &rr, W)));
  } else {
    // FP32 Krylov inside FP64 iterative refinement: r = F~ - A u in FP64, A d = r in FP32
    DevBuf<float> a32, r32, d32;
    DevBuf<double> r64;
    NL_TRY(a32.alloc(A->pairs->nnz ? A->pairs->nnz : 1, s));
    NL_TRY(r32.alloc(c.n, s));
    NL_TRY(d32.alloc(c.n, s));
    NL_TRY(r64.alloc(c.n, s));
    KWork<float> W;
    NL_TRY(W.alloc(c.n, s));
    W.use_graph = graphs;
    k_f64_to_f32<<<NL_CNT((unsigned)((A->pairs->nnz + RT - 1) / RT + 1)), RT, 0, s>>>(
        A->pairs->nnz, A->values, a32.p);
    NL_CUDA(cudaMemsetAsync(x.p, 0, sizeof(double) * c.n, s));
    k_init_dot<double><<<NL_CNT(c.gvec()), RT, 0, s>>>(c.n, rhs->v, c.R);
    double h[S_NSLOTS];
    NL_TRY(read_scalars(c, h));
    const double bb = h[S_BB];
    int total = 0;
    for (int outer = 0; outer < 60 && total < max_iter; outer++) {
      k_residual<<<NL_CNT(c.grow()), RTR, 0, s>>>(c.n, c.rp, c.col, A->values, c.free_, x.p, rhs->v,
                                                 r64.p, r32.p, c.R);
      NL_TRY(read_scalars(c, h));
      rr = bb > 0.0 ? std::sqrt(h[S_RR] / bb) : 0.0;
      if (rr <= rtol) {
        ok = true;
        break;
      }
      // inner tolerance: 1e-5 (about what one FP32 round reliably gains) while more than that
      // is still needed; once the remaining factor rtol / rr is within reach, half of it (at
      // least 1e-6), so that a round that would end just short of rtol is not followed by a
      // whole extra round
      const double need = rtol / rr;
      const double itol = need < 1e-6 ? 1e-5 : std::min(1e-3, std::max(1e-6, 0.5 * need));
      int inner = 0;
      bool iok = false;
      double irr = 0.0;
      NL_TRY((krylov<float, float>(c, a32.p, solver, r32.p, d32.p, itol, max_iter - total, &inner,
                                   &iok, &irr, W)));
      total += inner;
      k_add_f32_to_f64<<<NL_CNT(c.gvec()), RT, 0, s>>>(c.n, d32.p, x.p);
      if (inner == 0) break;
    }
    it = total;
    if (!ok) {
      k_residual<<<NL_CNT(c.grow()), RTR, 0, s>>>(c.n, c.rp, c.col, A->values, c.free_, x.p, rhs->v,
                                                 r64.p, nullptr, c.R);
      NL_TRY(read_scalars(c, h));
      rr = bb > 0.0 ? std::sqrt(h[S_RR] / bb) : 0.0;
      ok = rr <= rtol;
    }
  }
  std::vector<double> hx(c.n);
  std::vector<uint8_t> fr(c.n);
  NL_CUDA(cudaMemcpyAsync(hx.data(), x.p, sizeof(double) * c.n, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(fr.data(), m->node_free, c.n, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < c.n; i++) u_out[i] = fr[i] ? hx[i] : g_nodes[i];
  if (iters) *iters = it;
  if (rel_res) *rel_res = rr;
  if (!ok) return fail(NL_ENOTCONV, "nl_solve: no convergence to %g in %d iterations (%g)", rtol, it, rr);
  return NL_OK;
}

}  // namespace nlx
