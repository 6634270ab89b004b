// nl_solve.cu -- right-hand side with lifting and the Krylov solvers for A_{free,free} W = F~.
//
// Sec. 2 (eqs. A-F, weak-homo) and Sec. 4: the unknowns are the nodes inside Omega; the
// volume constraint u = g on Gamma is moved to the right-hand side through the lifting
// u = w + g~.  A is nonsymmetric at the quadrature-error level when L_max > 1 (the outer rule
// of Algorithm 1 depends on the pair), so BiCGStab is offered next to CG.  Vectors span all
// nodes; constrained entries of the Krylov vectors stay zero and the SpMV skips them.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "nl_internal.h"

namespace nlx {
namespace {

constexpr int RT = 256;  // reduction / vector kernel block size

template <int D>
__global__ void k_rhs_elems(int64_t n_elem, const int32_t* __restrict__ conn,
                            const uint8_t* __restrict__ eio, const uint8_t* __restrict__ free_,
                            const double* __restrict__ vol, const double* __restrict__ fn,
                            double f_const, const double* __restrict__ B,
                            const double* __restrict__ W, int nq, double* __restrict__ F) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_elem || !eio[e]) return;
  int32_t nd[D + 1];
  double fv[D + 1];
  for (int a = 0; a <= D; a++) {
    nd[a] = conn[e * (D + 1) + a];
    fv[a] = fn ? fn[nd[a]] : 0.0;
  }
  double acc[D + 1];
  for (int a = 0; a <= D; a++) acc[a] = 0.0;
  for (int q = 0; q < nq; q++) {
    double f = f_const;
    for (int v = 0; v <= D; v++) f += B[q * 4 + v] * fv[v];
    for (int a = 0; a <= D; a++) acc[a] += W[q] * f * B[q * 4 + a];
  }
  for (int a = 0; a <= D; a++)
    if (free_[nd[a]]) atomicAdd(&F[nd[a]], vol[e] * acc[a]);
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

// y = A_{free,free} x on free rows, 0 on constrained rows (warp per row)
template <typename V, typename X>
__global__ void k_spmv(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const V* __restrict__ val, const uint8_t* __restrict__ free_,
                       const X* __restrict__ x, X* __restrict__ y) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  X s = 0;
  if (free_[i]) {
    for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += (X)val[t] * x[col[t]];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[i] = s;
}

// residual r = b - A u on free rows (FP64), 0 elsewhere; u holds W on free nodes and 0 elsewhere
__global__ void k_residual(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const uint8_t* __restrict__ free_,
                           const double* __restrict__ u, const double* __restrict__ b,
                           double* __restrict__ r) {
  int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  if (free_[i])
    for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s += val[t] * u[col[t]];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[i] = free_[i] ? b[i] - s : 0.0;
}

// partial dot products per block; the final sum over blocks is done in fixed order
template <typename X>
__global__ void k_dot_partial(int64_t n, const X* __restrict__ a, const X* __restrict__ b,
                              double* __restrict__ part) {
  __shared__ double ws[RT / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RT / 32; w++) t += ws[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_dot_final(int nparts, int nslots, const double* __restrict__ part,
                            double* __restrict__ out) {
  // part holds nslots consecutive groups of nparts partial sums
  int slot = threadIdx.x;
  if (slot >= nslots) return;
  double t = 0.0;
  for (int k = 0; k < nparts; k++) t += part[slot * nparts + k];
  out[slot] = t;
}

template <typename X>
__global__ void k_axpby(int64_t n, X a, const X* __restrict__ x, X b, X* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

// p = r + beta (p - omega v)
template <typename X>
__global__ void k_bicg_p(int64_t n, const X* __restrict__ r, X beta, X omega, const X* __restrict__ v,
                         X* __restrict__ p) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_add_f32_to_f64(int64_t n, const float* __restrict__ d, double* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] += (double)d[i];
}

struct Ctx {
  cudaStream_t s;
  int64_t n;
  const int64_t* rp;
  const int32_t* col;
  const uint8_t* free_;
  int nparts;
  double* part;  // [nparts * 4]
  double* dres;  // [4]
  unsigned gvec() const { return (unsigned)((n + RT - 1) / RT); }
  unsigned grow() const { return (unsigned)((n * 32 + RT - 1) / RT); }
};

// several dot products, one host round trip
template <typename X>
nl_status dots(Ctx& c, int k, const X* const* a, const X* const* b, double* out) {
  for (int j = 0; j < k; j++)
    k_dot_partial<X><<<NL_CNT(c.nparts), RT, 0, c.s>>>(c.n, a[j], b[j], c.part + j * c.nparts);
  k_dot_final<<<NL_CNT(1), 32, 0, c.s>>>(c.nparts, k, c.part, c.dres);
  NL_CUDA(cudaMemcpyAsync(out, c.dres, sizeof(double) * k, cudaMemcpyDeviceToHost, c.s));
  NL_CUDA(cudaStreamSynchronize(c.s));
  return NL_OK;
}

// Krylov solve of A x = b (x starts at 0) to ||b - A x|| <= tol ||b||; X = double or float,
// V = matrix value type.  Returns iterations in *it; *ok when converged.
template <typename X, typename V>
nl_status krylov(Ctx& c, const V* val, int solver, const X* b, X* x, double tol, int max_it, int* it,
                 bool* ok, double* relres) {
  const int64_t n = c.n;
  DevBuf<X> r, rh, p, v, sv, t;
  NL_TRY(r.alloc(n, c.s));
  NL_TRY(p.alloc(n, c.s));
  NL_TRY(v.alloc(n, c.s));
  NL_CUDA(cudaMemsetAsync(x, 0, sizeof(X) * n, c.s));
  NL_CUDA(cudaMemcpyAsync(r.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
  NL_CUDA(cudaMemcpyAsync(p.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
  double bb;
  {
    const X* a1[1] = {b};
    NL_TRY(dots<X>(c, 1, a1, a1, &bb));
  }
  *it = 0;
  *ok = false;
  if (bb == 0.0) {
    *ok = true;
    *relres = 0.0;
    return NL_OK;
  }
  const double stop2 = tol * tol * bb;
  if (solver == 0) {  // CG
    double rr = bb;
    for (int k = 0; k < max_it; k++) {
      k_spmv<V, X><<<NL_CNT(c.grow()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, p.p, v.p);
      double pv;
      {
        const X* a1[1] = {p.p};
        const X* b1[1] = {v.p};
        NL_TRY(dots<X>(c, 1, a1, b1, &pv));
      }
      if (pv == 0.0) break;
      X alpha = (X)(rr / pv);
      k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, alpha, p.p, (X)1, x);
      k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, -alpha, v.p, (X)1, r.p);
      double rr_new;
      {
        const X* a1[1] = {r.p};
        NL_TRY(dots<X>(c, 1, a1, a1, &rr_new));
      }
      *it = k + 1;
      *relres = std::sqrt(rr_new / bb);
      if (rr_new <= stop2) {
        *ok = true;
        break;
      }
      X beta = (X)(rr_new / rr);
      rr = rr_new;
      k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, (X)1, r.p, beta, p.p);  // p = r + beta p
    }
    return NL_OK;
  }
  // BiCGStab (van der Vorst)
  NL_TRY(rh.alloc(n, c.s));
  NL_TRY(sv.alloc(n, c.s));
  NL_TRY(t.alloc(n, c.s));
  NL_CUDA(cudaMemcpyAsync(rh.p, b, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
  NL_CUDA(cudaMemsetAsync(p.p, 0, sizeof(X) * n, c.s));
  NL_CUDA(cudaMemsetAsync(v.p, 0, sizeof(X) * n, c.s));
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  for (int k = 0; k < max_it; k++) {
    double rho_new;
    {
      const X* a1[1] = {rh.p};
      const X* b1[1] = {r.p};
      NL_TRY(dots<X>(c, 1, a1, b1, &rho_new));
    }
    if (rho_new == 0.0 || omega == 0.0) break;
    double beta = (rho_new / rho) * (alpha / omega);
    rho = rho_new;
    k_bicg_p<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, r.p, (X)beta, (X)omega, v.p, p.p);
    k_spmv<V, X><<<NL_CNT(c.grow()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, p.p, v.p);
    double rhv;
    {
      const X* a1[1] = {rh.p};
      const X* b1[1] = {v.p};
      NL_TRY(dots<X>(c, 1, a1, b1, &rhv));
    }
    if (rhv == 0.0) break;
    alpha = rho / rhv;
    // s = r - alpha v
    NL_CUDA(cudaMemcpyAsync(sv.p, r.p, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
    k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, (X)(-alpha), v.p, (X)1, sv.p);
    k_spmv<V, X><<<NL_CNT(c.grow()), RT, 0, c.s>>>(n, c.rp, c.col, val, c.free_, sv.p, t.p);
    double ts_tt[2];
    {
      const X* a2[2] = {t.p, t.p};
      const X* b2[2] = {sv.p, t.p};
      NL_TRY(dots<X>(c, 2, a2, b2, ts_tt));
    }
    omega = ts_tt[1] > 0.0 ? ts_tt[0] / ts_tt[1] : 0.0;
    k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, (X)alpha, p.p, (X)1, x);
    k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, (X)omega, sv.p, (X)1, x);
    // r = s - omega t
    NL_CUDA(cudaMemcpyAsync(r.p, sv.p, sizeof(X) * n, cudaMemcpyDeviceToDevice, c.s));
    k_axpby<X><<<NL_CNT(c.gvec()), RT, 0, c.s>>>(n, (X)(-omega), t.p, (X)1, r.p);
    double rr;
    {
      const X* a1[1] = {r.p};
      NL_TRY(dots<X>(c, 1, a1, a1, &rr));
    }
    *it = k + 1;
    *relres = std::sqrt(rr / bb);
    if (rr <= stop2) {
      *ok = true;
      break;
    }
  }
  return NL_OK;
}

}  // namespace

nl_status rhs_values(nl_mesh* m, nl_matrix* A, const double* f_nodes, double f_const,
                     const double* g_nodes, double* F) {
  cudaStream_t s = m->stream;
  const int D = m->dim;
  const Rule& r = rule(D);
  std::vector<double> hB(16 * 4, 0.0), hW(16, 0.0);
  for (int q = 0; q < r.n; q++) {
    for (int a = 0; a <= D; a++) hB[q * 4 + a] = r.bary[q][a];
    hW[q] = r.w[q];
  }
  DevBuf<double> B, W, fn, g;
  NL_TRY(B.alloc(64, s));
  NL_TRY(W.alloc(16, s));
  NL_TRY(g.alloc(m->n_vert, s));
  NL_CUDA(cudaMemcpyAsync(B.p, hB.data(), sizeof(double) * 64, cudaMemcpyHostToDevice, s));
  NL_CUDA(cudaMemcpyAsync(W.p, hW.data(), sizeof(double) * 16, cudaMemcpyHostToDevice, s));
  NL_CUDA(cudaMemcpyAsync(g.p, g_nodes, sizeof(double) * m->n_vert, cudaMemcpyHostToDevice, s));
  if (f_nodes) {
    NL_TRY(fn.alloc(m->n_vert, s));
    NL_CUDA(cudaMemcpyAsync(fn.p, f_nodes, sizeof(double) * m->n_vert, cudaMemcpyHostToDevice, s));
  }
  NL_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * m->n_vert, s));
  unsigned ge = (unsigned)((m->n_elem + RT - 1) / RT);
  if (D == 2)
    k_rhs_elems<2><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free, m->vol,
                                     fn.p, f_const, B.p, W.p, r.n, F);
  else
    k_rhs_elems<3><<<NL_CNT(ge), RT, 0, s>>>(m->n_elem, m->conn, m->elem_in_omega, m->node_free, m->vol,
                                     fn.p, f_const, B.p, W.p, r.n, F);
  k_lift<<<NL_CNT((unsigned)((m->n_vert * 32 + RT - 1) / RT)), RT, 0, s>>>(
      m->n_vert, A->pairs->row_ptr, A->pairs->col, A->values, m->node_free, g.p, F);
  NL_CUDA(cudaGetLastError());
  NL_CUDA(cudaStreamSynchronize(s));
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
  c.nparts = 120;
  DevBuf<double> part, dres, x;
  NL_TRY(part.alloc(c.nparts * 4, s));
  NL_TRY(dres.alloc(4, s));
  NL_TRY(x.alloc(c.n, s));
  c.part = part.p;
  c.dres = dres.p;
  int it = 0;
  bool ok = false;
  double rr = 0.0;
  if (prec == NL_PREC_FP64) {
    NL_TRY((krylov<double, double>(c, A->values, solver, rhs->v, x.p, rtol, max_iter, &it, &ok, &rr)));
  } else {
    // FP32 Krylov inside FP64 iterative refinement: r = F~ - A u in FP64, A d = r in FP32
    DevBuf<float> a32, r32, d32;
    DevBuf<double> r64;
    NL_TRY(a32.alloc(A->pairs->nnz ? A->pairs->nnz : 1, s));
    NL_TRY(r32.alloc(c.n, s));
    NL_TRY(d32.alloc(c.n, s));
    NL_TRY(r64.alloc(c.n, s));
    k_f64_to_f32<<<NL_CNT((unsigned)((A->pairs->nnz + RT - 1) / RT + 1)), RT, 0, s>>>(A->pairs->nnz, A->values, a32.p);
    NL_CUDA(cudaMemsetAsync(x.p, 0, sizeof(double) * c.n, s));
    double bb;
    {
      const double* a1[1] = {rhs->v};
      NL_TRY(dots<double>(c, 1, a1, a1, &bb));
    }
    int total = 0;
    for (int outer = 0; outer < 60 && total < max_iter; outer++) {
      k_residual<<<NL_CNT(c.grow()), RT, 0, s>>>(c.n, c.rp, c.col, A->values, c.free_, x.p, rhs->v, r64.p);
      double r2;
      {
        const double* a1[1] = {r64.p};
        NL_TRY(dots<double>(c, 1, a1, a1, &r2));
      }
      rr = bb > 0.0 ? std::sqrt(r2 / bb) : 0.0;
      if (rr <= rtol) {
        ok = true;
        break;
      }
      k_f64_to_f32<<<NL_CNT(c.gvec()), RT, 0, s>>>(c.n, r64.p, r32.p);
      int inner = 0;
      bool iok = false;
      double irr = 0.0;
      NL_TRY((krylov<float, float>(c, a32.p, solver, r32.p, d32.p, 1e-5, max_iter - total, &inner,
                                   &iok, &irr)));
      total += inner;
      k_add_f32_to_f64<<<NL_CNT(c.gvec()), RT, 0, s>>>(c.n, d32.p, x.p);
      if (inner == 0) break;
    }
    it = total;
    if (!ok) {
      k_residual<<<NL_CNT(c.grow()), RT, 0, s>>>(c.n, c.rp, c.col, A->values, c.free_, x.p, rhs->v, r64.p);
      double r2;
      const double* a1[1] = {r64.p};
      NL_TRY(dots<double>(c, 1, a1, a1, &r2));
      rr = bb > 0.0 ? std::sqrt(r2 / bb) : 0.0;
      ok = rr <= rtol;
    }
  }
  std::vector<double> h(c.n);
  std::vector<uint8_t> fr(c.n);
  NL_CUDA(cudaMemcpyAsync(h.data(), x.p, sizeof(double) * c.n, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(fr.data(), m->node_free, c.n, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < c.n; i++) u_out[i] = fr[i] ? h[i] : g_nodes[i];
  if (iters) *iters = it;
  if (rel_res) *rel_res = rr;
  if (!ok) return fail(NL_ENOTCONV, "nl_solve: no convergence to %g in %d iterations (%g)", rtol, it, rr);
  return NL_OK;
}

}  // namespace nlx
