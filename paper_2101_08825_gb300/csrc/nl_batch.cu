// nl_batch.cu -- batched assembly: many problems in one persistent launch (nl_plan_*).
//
// A plan concatenates the m-major pair lists of n problems (one dimension, one precision;
// kernels, delta, eps and Algorithm 1 levels may differ) into one index space.  One launch of
// the assembly kernel covers all of it: every warp takes chunks of that space from a single
// counter, finds the problem of its chunk by a binary search over the pair prefix, and copies
// that problem's parameters into its own shared memory, so pairs of different refinement
// depth and problems of different sizes keep every SM busy until the last chunk.  One scatter
// launch over the concatenated inner elements then adds every cross and self block to that
// problem's CSR values, and (FP32 paths) one launch over the concatenated rows rebuilds the
// diagonals from the row sums.
//
// The launch shape (warps per CTA, CTAs per SM, pairs per grab of the counter) can be picked
// by timing candidates on the plan's own problems, and the whole execution (clears, three
// kernels) can be captured once into a CUDA graph that every execution replays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "nl_quad_kernel.cuh"

namespace nlx {
namespace {

// Per-problem arrays of the batched scatter and diagonal kernels.
struct SDesc {
  const int64_t* pair_off;
  const int32_t* pair_l;
  const int32_t* conn;
  const int64_t* row_ptr;
  const int32_t* col;
  const void* blk;         // cross blocks of the problem's pairs, in pair order
  const double* selfblk;   // [n_elem][(D+1)^2]
  double* values;          // [nnz]
};

__device__ __forceinline__ int find_problem(const int64_t* __restrict__ prefix, int n, int64_t g) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// CTA b: inner element b of the concatenated element lists (eprefix[k] = first element of
// problem k); adds all of its cross blocks and its self block.
template <int D, typename R>
__global__ void __launch_bounds__(128) k_scatter_batched(const SDesc* __restrict__ desc,
                                                         const int64_t* __restrict__ eprefix, int n,
                                                         int* __restrict__ err) {
  __shared__ int k_s;
  if (threadIdx.x == 0) k_s = find_problem(eprefix, n, (int64_t)blockIdx.x);
  __syncthreads();
  const int k = k_s;
  const SDesc d = desc[k];
  const int64_t m = (int64_t)blockIdx.x - eprefix[k];
  const int64_t q0 = d.pair_off[m], q1 = d.pair_off[m + 1];
  scatter_elem<D, R>(m, q0, q1, 0, true, d.pair_l, d.conn, d.row_ptr, d.col,
                     static_cast<const R*>(d.blk), d.selfblk, d.values, err);
}

// Warp per row of the concatenated row lists (vprefix[k] = first row of problem k): the
// diagonal entry becomes minus the sum of the row's other entries (zero row sums).
__global__ void k_diag_batched(const SDesc* __restrict__ desc, const int64_t* __restrict__ vprefix,
                               int n, int64_t total_rows) {
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= total_rows) return;
  const int k = find_problem(vprefix, n, g);
  const int64_t i = g - vprefix[k];
  const int64_t* row_ptr = desc[k].row_ptr;
  const int32_t* col = desc[k].col;
  double* values = desc[k].values;
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

}  // namespace
}  // namespace nlx

struct nl_plan {
  int n = 0, dim = 0;
  nl_precision prec = NL_PREC_FP64;
  int flags = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<nl_pairs*> pairs;
  std::vector<int64_t> pprefix, eprefix, vprefix, voff;  // host copies (n + 1 each)
  std::vector<int> count_band;
  int64_t total_pairs = 0, total_elem = 0, total_rows = 0, total_nnz = 0;
  int max_row_nnz = 0;
  // device
  void* d_probs = nullptr;       // QParams[n]
  nlx::SDesc* d_desc = nullptr;
  int64_t* d_prefix = nullptr;   // pair prefix, then element prefix, then row prefix
  unsigned long long* d_hdr = nullptr;  // [0] counter, problem k: [1 + 8k, 9 + 8k) stats
  int* d_err = nullptr;
  void* d_blk = nullptr;
  double* d_self = nullptr;
  double* d_values = nullptr;
  size_t bytes_blk = 0, bytes_hdr = 0;
  // launch
  nlx::QParams P0;  // parameters of problem 0 with the shared counter, error word and chunk
  nlx::QShape shape;
  int chunk = 32;
  double tuned_ms = 0.0;
  int launches_per_exec = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool executed = false;
};

namespace nlx {
namespace {

template <int D, typename R>
nl_status plan_quad(nl_plan* pl, QShape shape, int chunk) {
  QParams P = pl->P0;
  P.chunk = chunk;
  const QBatch Bt{static_cast<const QParams*>(pl->d_probs), pl->d_prefix, pl->n, pl->total_pairs};
  return launch_quad<D, R, 2, false, true>(P, pl->stream, Bt, shape);
}

nl_status plan_quad_any(nl_plan* pl, QShape shape, int chunk) {
  const bool f32 = pl->prec != NL_PREC_FP64;
  if (pl->dim == 2) return f32 ? plan_quad<2, float>(pl, shape, chunk) : plan_quad<2, double>(pl, shape, chunk);
  return f32 ? plan_quad<3, float>(pl, shape, chunk) : plan_quad<3, double>(pl, shape, chunk);
}

// One execution: clear the counters, the self blocks and the values; assemble; scatter; diagonal.
nl_status plan_enqueue(nl_plan* pl) {
  cudaStream_t s = pl->stream;
  const int D = pl->dim;
  const int NB = (D + 1) * (D + 1);
  NL_CUDA(cudaMemsetAsync(pl->d_hdr, 0, pl->bytes_hdr, s));
  NL_CUDA(cudaMemsetAsync(pl->d_err, 0, sizeof(int), s));
  NL_CUDA(cudaMemsetAsync(pl->d_self, 0, sizeof(double) * NB * std::max<int64_t>(1, pl->total_elem), s));
  NL_CUDA(cudaMemsetAsync(pl->d_values, 0, sizeof(double) * std::max<int64_t>(1, pl->total_nnz), s));
  int launches = 0;
  if (pl->total_pairs > 0) {
    NL_TRY(plan_quad_any(pl, pl->shape, pl->chunk));
    launches++;
  }
  if (pl->total_elem > 0) {
    const size_t smem = scatter_smem_bytes(D + 1, pl->max_row_nnz, pl->prec != NL_PREC_FP64 ? 4 : 8);
    const bool f32 = pl->prec != NL_PREC_FP64;
    const int64_t* ep = pl->d_prefix + (pl->n + 1);
    if (D == 2) {
      if (f32) k_scatter_batched<2, float><<<NL_CNT((unsigned)pl->total_elem), 128, smem, s>>>(pl->d_desc, ep, pl->n, pl->d_err);
      else k_scatter_batched<2, double><<<NL_CNT((unsigned)pl->total_elem), 128, smem, s>>>(pl->d_desc, ep, pl->n, pl->d_err);
    } else {
      if (f32) k_scatter_batched<3, float><<<NL_CNT((unsigned)pl->total_elem), 128, smem, s>>>(pl->d_desc, ep, pl->n, pl->d_err);
      else k_scatter_batched<3, double><<<NL_CNT((unsigned)pl->total_elem), 128, smem, s>>>(pl->d_desc, ep, pl->n, pl->d_err);
    }
    NL_CUDA(cudaGetLastError());
    launches++;
  }
  if (pl->prec != NL_PREC_FP64 && pl->total_rows > 0) {
    const int64_t* vp = pl->d_prefix + 2 * (pl->n + 1);
    k_diag_batched<<<NL_CNT((unsigned)((pl->total_rows * 32 + 255) / 256)), 256, 0, s>>>(
        pl->d_desc, vp, pl->n, pl->total_rows);
    NL_CUDA(cudaGetLastError());
    launches++;
  }
  pl->launches_per_exec = launches;
  return NL_OK;
}

template <typename F>
nl_status kernel_smem_setup(F* kern, size_t smem) {
  return allow_smem(kern, smem);
}

// Raises the scatter kernel's shared-memory ceiling before any capture.
nl_status plan_prepare_scatter(nl_plan* pl) {
  const size_t smem = scatter_smem_bytes(pl->dim + 1, pl->max_row_nnz, pl->prec != NL_PREC_FP64 ? 4 : 8);
  const bool f32 = pl->prec != NL_PREC_FP64;
  if (pl->dim == 2) return f32 ? kernel_smem_setup(k_scatter_batched<2, float>, smem) : kernel_smem_setup(k_scatter_batched<2, double>, smem);
  return f32 ? kernel_smem_setup(k_scatter_batched<3, float>, smem) : kernel_smem_setup(k_scatter_batched<3, double>, smem);
}

// Times every candidate shape of the assembly kernel on the plan's problems (one untimed
// run first) and keeps the fastest.  The kernel's outputs are cleared by every execution.
nl_status plan_autotune(nl_plan* pl) {
  cudaStream_t s = pl->stream;
  std::vector<std::pair<QShape, int>> cands;
  const int wmax = pl->dim == 2 ? 8 : 4;
  for (int w : {wmax, wmax / 2})
    for (int c : {0, 1})
      for (int ch : {8, 32, 128}) {
        QShape sh;
        sh.warps = w;
        sh.ctas_per_sm = c;
        cands.push_back({sh, ch});
      }
  NL_CUDA(cudaMemsetAsync(pl->d_hdr, 0, pl->bytes_hdr, s));
  NL_TRY(plan_quad_any(pl, QShape{}, 32));
  float best = 1e30f;
  for (auto& c : cands) {
    NL_CUDA(cudaMemsetAsync(pl->d_hdr, 0, pl->bytes_hdr, s));
    NL_CUDA(cudaEventRecord(pl->ev0, s));
    NL_TRY(plan_quad_any(pl, c.first, c.second));
    NL_CUDA(cudaEventRecord(pl->ev1, s));
    NL_CUDA(cudaEventSynchronize(pl->ev1));
    float ms = 0.f;
    NL_CUDA(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
    if (ms < best) {
      best = ms;
      pl->shape = c.first;
      pl->chunk = c.second;
    }
  }
  pl->tuned_ms = best;
  int herr = 0;
  NL_CUDA(cudaMemcpyAsync(&herr, pl->d_err, sizeof herr, cudaMemcpyDeviceToHost, s));
  NL_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(NL_EINTERNAL, "nl_plan_create: device check failed while tuning (code %d)", herr);
  return NL_OK;
}

void plan_free(nl_plan* pl) {
  if (!pl) return;
  cudaStream_t s = pl->stream;
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->ev0) cudaEventDestroy(pl->ev0);
  if (pl->ev1) cudaEventDestroy(pl->ev1);
  dev_free(pl->d_probs, 0, s);
  dev_free(pl->d_desc, 0, s);
  dev_free(pl->d_prefix, 0, s);
  dev_free(pl->d_hdr, 0, s);
  dev_free(pl->d_err, 0, s);
  dev_free(pl->d_blk, 0, s);
  dev_free(pl->d_self, 0, s);
  dev_free(pl->d_values, 0, s);
  cudaStreamSynchronize(s);
  if (pl->own_stream) cudaStreamDestroy(s);
  for (nl_pairs* p : pl->pairs) pairs_release(p);
  delete pl;
}

}  // namespace
}  // namespace nlx

extern "C" {

nl_status nl_plan_create(int n, nl_mesh* const* meshes, nl_pairs* const* pairs,
                         const nl_kernel_params* kps, const nl_quad_params* qps,
                         nl_precision precision, int flags, void* cuda_stream, nl_plan** out) {
  using namespace nlx;
  clear_error();
  if (!out || !meshes || !pairs || !kps || !qps) return fail(NL_EINVAL, "nl_plan_create: NULL argument");
  if (n < 1 || n > (1 << 20)) return fail(NL_EINVAL, "nl_plan_create: need 1 <= n <= 2^20 problems");
  if (flags & ~(NL_PLAN_AUTOTUNE | NL_PLAN_GRAPH)) return fail(NL_EINVAL, "nl_plan_create: unknown flags %d", flags);
  const int D = meshes[0] ? meshes[0]->dim : 0;
  std::vector<QParams> probs(n);
  int scap = 0;
  for (int k = 0; k < n; k++) {
    if (!meshes[k] || !pairs[k]) return fail(NL_EINVAL, "nl_plan_create: problem %d has a NULL mesh or pairs", k);
    if (meshes[k]->dim != D) return fail(NL_EINVAL, "nl_plan_create: problem %d is %dD, problem 0 is %dD", k, meshes[k]->dim, D);
    if (pairs[k]->mesh != meshes[k]) return fail(NL_EINVAL, "nl_plan_create: problem %d: pairs of another mesh", k);
    if (meshes[k]->order != 1 || meshes[k]->cell != 0)
      return fail(NL_EINVAL, "nl_plan_create: problem %d: plans take P1 meshes only (use nl_assemble)", k);
    if (kps[k].delta != pairs[k]->delta || kps[k].eps != pairs[k]->eps)
      return fail(NL_EINVAL, "nl_plan_create: problem %d: delta/eps differ from those of its pairs", k);
    NL_TRY(fill_qparams("nl_plan_create", meshes[k], pairs[k], &kps[k], &qps[k], precision, &probs[k]));
    scap = std::max(scap, probs[k].scap);
  }
  nl_plan* pl = new nl_plan();
  pl->n = n;
  pl->dim = D;
  pl->prec = precision;
  pl->flags = flags;
  pl->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!pl->stream) {
    if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete pl;
      return fail(NL_ECUDA, "nl_plan_create: cannot create the plan's stream");
    }
    pl->own_stream = true;
  }
  pl->pprefix.assign(n + 1, 0);
  pl->eprefix.assign(n + 1, 0);
  pl->vprefix.assign(n + 1, 0);
  pl->voff.assign(n + 1, 0);
  for (int k = 0; k < n; k++) {
    // the pair lists and patterns were complete when nl_pairs_build returned; the mesh
    // stream is drained so that the plan's stream sees them
    cudaStreamSynchronize(meshes[k]->stream);
    pairs[k]->refs.fetch_add(1);
    pl->pairs.push_back(pairs[k]);
    pl->pprefix[k + 1] = pl->pprefix[k] + pairs[k]->n_pairs;
    pl->eprefix[k + 1] = pl->eprefix[k] + meshes[k]->n_elem;
    pl->vprefix[k + 1] = pl->vprefix[k] + meshes[k]->n_vert;
    pl->voff[k + 1] = pl->voff[k] + pairs[k]->nnz;
    pl->max_row_nnz = std::max(pl->max_row_nnz, pairs[k]->max_row_nnz);
    pl->count_band.push_back(probs[k].count_band);
  }
  pl->total_pairs = pl->pprefix[n];
  pl->total_elem = pl->eprefix[n];
  pl->total_rows = pl->vprefix[n];
  pl->total_nnz = pl->voff[n];
  if (pl->total_elem > INT32_MAX || pl->total_rows * 32 / 256 > INT32_MAX) {
    plan_free(pl);
    return fail(NL_EINVAL, "nl_plan_create: the problems hold more than 2^31-1 elements in all");
  }
  cudaStream_t s = pl->stream;
  const int NB = (D + 1) * (D + 1);
  const size_t rsz = precision == NL_PREC_FP64 ? sizeof(double) : sizeof(float);
  pl->bytes_blk = (size_t)pl->total_pairs * NB * rsz;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    plan_free(pl);
    return fail(NL_ECUDA, "nl_plan_create: cudaMemGetInfo failed");
  }
  if (pl->bytes_blk > free_b / 2) {
    plan_free(pl);
    return fail(NL_ENOMEM,
                "nl_plan_create: the block buffer of %lld pairs (%zu bytes) exceeds half of the "
                "free device memory; use fewer problems per plan or nl_assemble",
                (long long)pl->total_pairs, pl->bytes_blk);
  }
  pl->bytes_hdr = sizeof(unsigned long long) * (1 + 8 * (size_t)n);
  auto A = [&](size_t bytes) { return dev_alloc(std::max<size_t>(bytes, 16), s); };
  pl->d_probs = A(sizeof(QParams) * n);
  pl->d_desc = static_cast<SDesc*>(A(sizeof(SDesc) * n));
  pl->d_prefix = static_cast<int64_t*>(A(sizeof(int64_t) * 3 * (n + 1)));
  pl->d_hdr = static_cast<unsigned long long*>(A(pl->bytes_hdr));
  pl->d_err = static_cast<int*>(A(sizeof(int)));
  pl->d_blk = A(pl->bytes_blk);
  pl->d_self = static_cast<double*>(A(sizeof(double) * NB * (size_t)pl->total_elem));
  pl->d_values = static_cast<double*>(A(sizeof(double) * (size_t)pl->total_nnz));
  if (!pl->d_probs || !pl->d_desc || !pl->d_prefix || !pl->d_hdr || !pl->d_err || !pl->d_blk ||
      !pl->d_self || !pl->d_values) {
    plan_free(pl);
    return fail(NL_ENOMEM, "nl_plan_create: device allocation failed");
  }
  std::vector<SDesc> desc(n);
  for (int k = 0; k < n; k++) {
    QParams& P = probs[k];
    P.scap = scap;
    P.p_begin = 0;
    P.p_end = pairs[k]->n_pairs;
    P.blk = static_cast<char*>(pl->d_blk) + (size_t)pl->pprefix[k] * NB * rsz;
    P.selfblk = pl->d_self + (size_t)pl->eprefix[k] * NB;
    P.values = pl->d_values + pl->voff[k];
    P.counter = pl->d_hdr;
    P.stats = pl->d_hdr + 1 + 8 * (size_t)k;
    P.err = pl->d_err;
    P.chunk = 32;
    desc[k] = SDesc{pairs[k]->pair_off, pairs[k]->pair_l, meshes[k]->conn, pairs[k]->row_ptr,
                    pairs[k]->col, P.blk, P.selfblk, P.values};
  }
  pl->P0 = probs[0];
  std::vector<int64_t> pre(3 * (n + 1));
  std::copy(pl->pprefix.begin(), pl->pprefix.end(), pre.begin());
  std::copy(pl->eprefix.begin(), pl->eprefix.end(), pre.begin() + (n + 1));
  std::copy(pl->vprefix.begin(), pl->vprefix.end(), pre.begin() + 2 * (n + 1));
  nl_status st = NL_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (st == NL_OK && e != cudaSuccess) st = cuda_fail(e, what);
  };
  check(cudaMemcpyAsync(pl->d_probs, probs.data(), sizeof(QParams) * n, cudaMemcpyHostToDevice, s), "plan upload");
  check(cudaMemcpyAsync(pl->d_desc, desc.data(), sizeof(SDesc) * n, cudaMemcpyHostToDevice, s), "plan upload");
  check(cudaMemcpyAsync(pl->d_prefix, pre.data(), sizeof(int64_t) * pre.size(), cudaMemcpyHostToDevice, s), "plan upload");
  check(cudaMemsetAsync(pl->d_err, 0, sizeof(int), s), "plan clear");
  check(cudaStreamSynchronize(s), "plan upload");
  check(cudaEventCreate(&pl->ev0), "cudaEventCreate");
  check(cudaEventCreate(&pl->ev1), "cudaEventCreate");
  if (st == NL_OK) st = plan_prepare_scatter(pl);
  if (st == NL_OK && (flags & NL_PLAN_AUTOTUNE) && pl->total_pairs > 0) st = plan_autotune(pl);
  if (st == NL_OK && (flags & NL_PLAN_GRAPH)) {
    // one plain execution first sets every kernel attribute outside the capture
    st = plan_enqueue(pl);
    if (st == NL_OK) check(cudaStreamSynchronize(s), "nl_plan_create");
    if (st == NL_OK) check(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    if (st == NL_OK) {
      nl_status est = plan_enqueue(pl);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (est != NL_OK) st = est;
      else check(e, "cudaStreamEndCapture");
      if (st == NL_OK) {
        pl->graph = g;
        check(cudaGraphInstantiate(&pl->gexec, g, 0), "cudaGraphInstantiate");
      } else if (g) {
        cudaGraphDestroy(g);
      }
    }
  }
  if (st != NL_OK) {
    plan_free(pl);
    return st;
  }
  *out = pl;
  return NL_OK;
}

nl_status nl_plan_execute(nl_plan* pl) {
  using namespace nlx;
  clear_error();
  if (!pl) return fail(NL_EINVAL, "nl_plan_execute: NULL plan");
  NL_CUDA(cudaEventRecord(pl->ev0, pl->stream));
  if (pl->gexec) {
    NL_CUDA(cudaGraphLaunch(pl->gexec, pl->stream));
    for (int i = 0; i < pl->launches_per_exec; i++) count_launch();
  } else {
    NL_TRY(plan_enqueue(pl));
  }
  NL_CUDA(cudaEventRecord(pl->ev1, pl->stream));
  pl->executed = true;
  return NL_OK;
}

nl_status nl_plan_sync(nl_plan* pl, nl_assemble_stats* stats) {
  using namespace nlx;
  clear_error();
  if (!pl) return fail(NL_EINVAL, "nl_plan_sync: NULL plan");
  if (!pl->executed) return fail(NL_EINVAL, "nl_plan_sync: the plan has not been executed");
  std::vector<unsigned long long> hs(1 + 8 * (size_t)pl->n);
  int herr = 0;
  NL_CUDA(cudaMemcpyAsync(hs.data(), pl->d_hdr, pl->bytes_hdr, cudaMemcpyDeviceToHost, pl->stream));
  NL_CUDA(cudaMemcpyAsync(&herr, pl->d_err, sizeof herr, cudaMemcpyDeviceToHost, pl->stream));
  NL_CUDA(cudaStreamSynchronize(pl->stream));
  float ms = 0.f;
  NL_CUDA(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
  if (herr)
    return fail(NL_EINTERNAL, "nl_plan_sync: device check failed (code %d: %s)", herr,
                (herr & ERR_STACK) ? "refinement stack capacity exceeded" : "CSR entry missing");
  if (stats) {
    const int nq = pl->dim == 2 ? 7 : 14;
    for (int k = 0; k < pl->n; k++) {
      const unsigned long long* h = hs.data() + 1 + 8 * (size_t)k;
      nl_assemble_stats& s = stats[k];
      s.n_pairs = pl->pprefix[k + 1] - pl->pprefix[k];
      s.n_items = (int64_t)h[0];
      s.n_point_pairs = (int64_t)h[0] * nq * nq;
      s.n_exact_checks = (int64_t)h[2];
      s.ms_assemble = ms;
      s.n_eval_point_pairs = (int64_t)h[3];
      s.n_closed_items = (int64_t)h[4];
      s.n_band_point_pairs = pl->count_band[k] ? (int64_t)h[5] : -1;
      s.precision_run = pl->prec != NL_PREC_FP64 ? NL_PREC_FP32 : NL_PREC_FP64;
      s.n_quad_launches = 1;
      s.ms_quad = 0.0;
      s.ms_scatter = 0.0;
    }
  }
  return NL_OK;
}

nl_status nl_plan_values(const nl_plan* pl, int k, double** values, int64_t* nnz) {
  using namespace nlx;
  clear_error();
  if (!pl || k < 0 || k >= pl->n) return fail(NL_EINVAL, "nl_plan_values: bad plan or index");
  if (values) *values = pl->d_values + pl->voff[k];
  if (nnz) *nnz = pl->voff[k + 1] - pl->voff[k];
  return NL_OK;
}

nl_status nl_plan_export(const nl_plan* pl, int k, double* values) {
  using namespace nlx;
  clear_error();
  if (!pl || !values || k < 0 || k >= pl->n) return fail(NL_EINVAL, "nl_plan_export: bad argument");
  const int64_t nnz = pl->voff[k + 1] - pl->voff[k];
  if (nnz)
    NL_CUDA(cudaMemcpyAsync(values, pl->d_values + pl->voff[k], sizeof(double) * nnz,
                            cudaMemcpyDeviceToHost, pl->stream));
  NL_CUDA(cudaStreamSynchronize(pl->stream));
  return NL_OK;
}

nl_status nl_plan_matrix(const nl_plan* pl, int k, nl_matrix** A) {
  using namespace nlx;
  clear_error();
  if (!pl || !A || k < 0 || k >= pl->n) return fail(NL_EINVAL, "nl_plan_matrix: bad argument");
  nl_pairs* pairs = pl->pairs[k];
  nl_matrix* M = *A;
  bool fresh = false;
  if (M && M->pairs != pairs) return fail(NL_EINVAL, "nl_plan_matrix: *A has another pattern");
  if (!M) {
    M = new nl_matrix();
    M->pairs = pairs;
    M->stream = pairs->mesh->stream;
    pairs->refs.fetch_add(1);
    M->values = static_cast<double*>(dev_alloc(sizeof(double) * (pairs->nnz ? pairs->nnz : 1), M->stream));
    if (!M->values) {
      pairs_release(pairs);
      delete M;
      return fail(NL_ENOMEM, "nl_plan_matrix: cannot allocate %lld values", (long long)pairs->nnz);
    }
    fresh = true;
  }
  cudaError_t e = cudaSuccess;
  if (pairs->nnz) e = cudaMemcpyAsync(M->values, pl->d_values + pl->voff[k], sizeof(double) * pairs->nnz,
                                      cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) {
    if (fresh) nl_matrix_destroy(M);
    return cuda_fail(e, "nl_plan_matrix");
  }
  *A = M;
  return NL_OK;
}

nl_status nl_plan_shape(const nl_plan* pl, int* warps, int* ctas_per_sm, int* chunk, double* tuned_ms,
                        int* graph) {
  using namespace nlx;
  clear_error();
  if (!pl) return fail(NL_EINVAL, "nl_plan_shape: NULL plan");
  if (warps) *warps = pl->shape.warps;
  if (ctas_per_sm) *ctas_per_sm = pl->shape.ctas_per_sm;
  if (chunk) *chunk = pl->chunk;
  if (tuned_ms) *tuned_ms = pl->tuned_ms;
  if (graph) *graph = pl->gexec ? 1 : 0;
  return NL_OK;
}

void nl_plan_destroy(nl_plan* pl) { nlx::plan_free(pl); }

}  // extern "C"
