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

nl_status assemble_values(nl_mesh* m, nl_pairs* p, const nl_kernel_params* kp,
                          const nl_quad_params* qp, nl_precision prec, double* values,
                          nl_assemble_stats* st) {
  // hexahedra (nl_quad_hex.cu), quadrilaterals (nl_quad_quad.cu), P2 triangles (nl_quad_p2.cu; MIXED precisions run
  // their FP32 paths) and the tensor-core variants (nl_quad_mma.cu) are compiled in
  // translation units of their own
  if (m->cell == 2) return assemble_values_hex(m, p, kp, qp, prec, values, st);
  if (m->cell == 1) return assemble_values_quad(m, p, kp, qp, prec, values, st);
  if (m->order == 2) return m->dim == 2 ? assemble_values_p2(m, p, kp, qp, prec, values, st)
                                        : assemble_values_p2t(m, p, kp, qp, prec, values, st);
  if (prec == NL_PREC_MIXED_TF32 || prec == NL_PREC_MIXED_BF16)
    return assemble_values_mma(m, p, kp, qp, prec, values, st);
  return assemble_single<0>(m, p, kp, qp, prec, values, st);
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
  const size_t smem = scatter_smem_bytes(D + 1, p->max_row_nnz, sizeof(R));
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
  if (m->order != 1 || m->cell != 0) return fail(NL_EINVAL, "nl_assemble_noalloc: P1 meshes only; use nl_assemble");
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
