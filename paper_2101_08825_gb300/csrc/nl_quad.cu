// nl_quad.cu -- single-problem assembly of the mollified nonlocal stiffness matrix
// (nl_assemble, nl_assemble_noalloc): the pair batches, the block buffer and the scatter around
// the kernels of nl_quad_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "nl_quad_kernel.cuh"

namespace nlx {

thread_local size_t g_block_budget = 0;

nl_status ensure_device_tables() {
  if (rule(2).n != 7 || rule(3).n != 14)
    return fail(NL_EINTERNAL, "quadrature rule set-up failed");
  return NL_OK;
}

namespace {
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

template <int D, typename R, int KERN>
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
    NL_TRY((launch_quad<D, R, KERN>(P, s)));
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

}  // namespace

nl_status assemble_values(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
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
    if (D == 2) {
      if (f32) rc = gauss ? run_assembly<2, float, 1>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly<2, float, 0>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly<2, double, 1>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly<2, double, 0>(m, p, P, values, s, scratch.p, err.p, T);
    } else {
      if (f32) rc = gauss ? run_assembly<3, float, 1>(m, p, P, values, s, scratch.p, err.p, T)
                          : run_assembly<3, float, 0>(m, p, P, values, s, scratch.p, err.p, T);
      else rc = gauss ? run_assembly<3, double, 1>(m, p, P, values, s, scratch.p, err.p, T)
                      : run_assembly<3, double, 0>(m, p, P, values, s, scratch.p, err.p, T);
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
    st->precision_run = f32 ? NL_PREC_FP32 : NL_PREC_FP64;
    st->n_quad_launches = T.launches(0);
    st->ms_quad = T.ms(0);
    st->ms_scatter = T.ms(1);
  }
  return NL_OK;
}

// ---- assembly without device allocation ------------------------------------------------------
// For callers that cannot call cudaMalloc at assembly time: a process that reserves all of
// its device memory when it starts (a serving process with a fixed pool, where a new
// allocation would fail or grow a pool it does not own), or code that must not stall
// other streams on an allocation's implicit synchronisation.  This variant adds every cross
// block to the CSR values directly and keeps its only scratch -- the work counter, the
// counters, the error word and the per-element self blocks -- in the file-scope array below,
// which every GPU that loads this library holds until the process exits.

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB
constexpr size_t NOALLOC_HEADER_BYTES = 256;                 // counters and the error word
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_noalloc_scratch in the current context.  The host-side name of the
// array is not a device address.  The lookup is repeated on every call rather than cached:
// a cached address would dangle after cudaDeviceReset or a re-created primary context, and
// the lookup costs far less than the synchronising call around it.  The first lookup in a
// context can load this library's device code, so the first call belongs before any stream
// capture.
nl_status noalloc_scratch(unsigned char** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
  *out = static_cast<unsigned char*>(ptr);
  return NL_OK;
}

template <int D, typename R, int KERN>
nl_status run_noalloc(nl_mesh* m, nl_pairs* p, QParams P, double* values, cudaStream_t s) {
  NL_TRY((launch_quad<D, R, KERN, true>(P, s)));
  const size_t smem = scatter_smem_bytes(D, p->max_row_nnz);
  if (smem == 0)
    return fail(NL_EINTERNAL, "rows of %d columns exceed the scatter kernel's shared memory", p->max_row_nnz);
  NL_TRY((allow_smem(k_scatter<D, R>, smem)));
  k_scatter<D, R><<<NL_CNT((unsigned)m->n_elem), 128, smem, s>>>(
      0, 0, 0, p->pair_off, p->pair_l, m->conn, p->row_ptr, p->col, (const R*)nullptr, P.selfblk, 1,
      values, P.err);
  NL_CUDA(cudaGetLastError());
  if (std::is_same<R, float>::value) {
    k_diag_from_rows<<<NL_CNT((unsigned)((m->n_vert * 32 + 255) / 256)), 256, 0, s>>>(
        m->n_vert, p->row_ptr, p->col, values);
    NL_CUDA(cudaGetLastError());
  }
  return NL_OK;
}
}  // namespace

nl_status assemble_noalloc(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                           const nl_quad_params* qp, nl_precision prec, double* values,
                           nl_assemble_stats* st) {
  if (!values) return fail(NL_EINVAL, "nl_assemble_noalloc: values is NULL");
  QParams P;
  NL_TRY(fill_qparams("nl_assemble_noalloc", m, p, kp, qp, prec, &P));
  const int D = m->dim;
  const int NB = (D + 1) * (D + 1);
  const int64_t max_elem =
      (int64_t)((NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER_BYTES) / (sizeof(double) * NB));
  if (m->n_elem > max_elem)
    return fail(NL_EINVAL,
                "nl_assemble_noalloc: %lld elements exceed the %zu-byte scratch (at most %lld "
                "elements in %dD); use nl_assemble",
                (long long)m->n_elem, NOALLOC_SCRATCH_BYTES, (long long)max_elem, D);
  unsigned char* scratch = nullptr;
  NL_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = m->stream;
  P.values = values;
  // scratch layout: [0, 64) counter + stats, [64, 68) error word, [256, ...) self blocks.
  // Every call starts by clearing what it accumulates into.
  P.counter = reinterpret_cast<unsigned long long*>(scratch);
  P.stats = P.counter + 1;
  P.err = reinterpret_cast<int*>(scratch + 64);
  P.selfblk = reinterpret_cast<double*>(scratch + NOALLOC_HEADER_BYTES);
  NL_CUDA(cudaMemsetAsync(scratch, 0, NOALLOC_HEADER_BYTES, s));
  NL_CUDA(cudaMemsetAsync(P.selfblk, 0, sizeof(double) * NB * m->n_elem, s));
  NL_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (p->nnz ? p->nnz : 1), s));
  const bool f32 = prec != NL_PREC_FP64;
  const bool gauss = kp->kernel == NL_KERNEL_TRUNC_GAUSS;
  nl_status rc = NL_OK;
  if (p->n_pairs > 0) {
    if (D == 2) {
      if (f32) rc = gauss ? run_noalloc<2, float, 1>(m, p, P, values, s) : run_noalloc<2, float, 0>(m, p, P, values, s);
      else rc = gauss ? run_noalloc<2, double, 1>(m, p, P, values, s) : run_noalloc<2, double, 0>(m, p, P, values, s);
    } else {
      if (f32) rc = gauss ? run_noalloc<3, float, 1>(m, p, P, values, s) : run_noalloc<3, float, 0>(m, p, P, values, s);
      else rc = gauss ? run_noalloc<3, double, 1>(m, p, P, values, s) : run_noalloc<3, double, 0>(m, p, P, values, s);
    }
  }
  if (rc != NL_OK) return rc;
  unsigned long long hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int herr = 0;
  NL_CUDA(cudaMemcpyAsync(hs, scratch, sizeof hs, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaMemcpyAsync(&herr, scratch + 64, sizeof herr, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  if (herr)
    return fail(NL_EINTERNAL, "nl_assemble_noalloc: device check failed (code %d: %s)", herr,
                (herr & ERR_STACK) ? "refinement stack capacity exceeded" : "CSR entry missing");
  if (st) {
    const int nq = D == 2 ? 7 : 14;
    st->n_pairs = p->n_pairs;
    st->n_items = (int64_t)hs[1];
    st->n_point_pairs = (int64_t)hs[1] * nq * nq;
    st->n_exact_checks = (int64_t)hs[3];
    st->ms_assemble = 0.0;
    st->n_eval_point_pairs = (int64_t)hs[4];
    st->n_closed_items = (int64_t)hs[5];
    st->n_band_point_pairs = P.count_band ? (int64_t)hs[6] : -1;
    st->precision_run = f32 ? NL_PREC_FP32 : NL_PREC_FP64;
    st->n_quad_launches = 1;
    st->ms_quad = 0.0;
    st->ms_scatter = 0.0;
  }
  return NL_OK;
}

}  // namespace nlx

extern "C" nl_status nl_assemble_noalloc(nl_mesh* mesh, nl_pairs* pairs, const nl_kernel_params* kp,
                                         const nl_quad_params* qp, nl_precision precision,
                                         double* values, nl_assemble_stats* stats) {
  nlx::clear_error();
  if (!mesh || !pairs || !kp || !qp) return nlx::fail(NL_EINVAL, "nl_assemble_noalloc: NULL argument");
  if (pairs->mesh != mesh) return nlx::fail(NL_EINVAL, "nl_assemble_noalloc: pairs were built on another mesh");
  if (kp->delta != pairs->delta || kp->eps != pairs->eps)
    return nlx::fail(NL_EINVAL, "nl_assemble_noalloc: delta/eps differ from those of the pairs");
  return nlx::assemble_noalloc(mesh, pairs, kp, qp, precision, values, stats);
}
