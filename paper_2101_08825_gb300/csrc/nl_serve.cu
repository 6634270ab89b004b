// nl_serve.cu -- a serving loop for assemble + solve requests with continuous batching.
//
// Every request describes a structured box mesh, a kernel, Algorithm 1 levels, a precision,
// a manufactured solution and a solver.  The server owns max_slots worker threads, each with
// its own non-blocking CUDA stream.  A request waits in a FIFO queue until a slot is idle and
// its estimated device footprint fits into the memory budget left over by the requests in
// flight (a request larger than the whole budget runs alone); requests arriving while others
// run are admitted as slots and memory free up, so their kernels overlap on the device.
// Each admitted request runs the whole path on its slot's stream -- mesh, pair search and
// pattern, assembly, right-hand side with lifting, Krylov solve -- keeps its mesh, pattern,
// matrix and Krylov vectors on the device while it runs, and releases them when it is done.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nl_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  nl_request req;
  nl_result res;
  size_t est = 0;
  bool done = false;
};

double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// Rough upper estimate of the device bytes one request holds at its peak.
size_t estimate_bytes(const nl_request& r, size_t block_budget) {
  const int D = r.dim;
  double cells = 1.0, verts = 1.0;
  for (int k = 0; k < D; k++) {
    cells *= r.cells[k] + 2.0 * r.layer;
    verts *= r.cells[k] + 2.0 * r.layer + 1.0;
  }
  const double epc = D == 2 ? 2.0 : 6.0;
  const double n_elem = cells * epc;
  const double reach = std::ceil((r.kernel.delta + r.kernel.eps) / r.h);
  const double span = 2.0 * reach + 3.0;
  const double ppe = epc * std::pow(span, D);
  const double pairs = n_elem * ppe;
  const double nnz = verts * std::pow(span, D);
  const double mesh = n_elem * (96.0 + 48.0 + 80.0 + 8.0 + 16.0) + verts * 40.0;
  const double nb = (D + 1.0) * (D + 1.0);
  const double blk = std::min((double)block_budget, pairs * nb * 4.0) + n_elem * nb * 8.0;
  const double solve = verts * 8.0 * 14.0 + nnz * 4.0;
  return (size_t)(mesh + pairs * 4.0 + nnz * 12.0 + blk + solve) + ((size_t)16 << 20);
}

double ms_u(int ms, int D, const double* x) {
  double s = (ms == 0) ? 1.0 : 0.0;
  for (int k = 0; k < D; k++) {
    const double t = x[k];
    s += ms == 0 ? t : ms == 1 ? t * t : t * t * t;
  }
  return s;
}

}  // namespace

struct nl_server {
  size_t budget = 0;
  int slots = 0;
  int device = 0;
  size_t block_budget = (size_t)256 << 20;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Job> jobs;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies;
  double first_submit = -1.0, last_done = 0.0;
  Clock::time_point t0;
};

namespace {

// Runs one request on `stream`; fills res (status, counts, error, timings except submit).
void run_request(nl_server* S, cudaStream_t stream, Job& job) {
  const nl_request& r = job.req;
  nl_result& res = job.res;
  nl_mesh* mesh = nullptr;
  nl_pairs* pairs = nullptr;
  nl_matrix* A = nullptr;
  nl_vector* rhs = nullptr;
  nlx::g_block_budget = S->block_budget;
  auto finish = [&](nl_status st) {
    res.status = st;
    if (st != NL_OK && res.message[0] == 0) snprintf(res.message, sizeof res.message, "%s", nl_last_error());
    nl_vector_destroy(rhs);
    nl_matrix_destroy(A);
    nl_pairs_destroy(pairs);
    nl_mesh_destroy(mesh);
  };
  nl_status st = nl_mesh_create_box(r.dim, r.cells, r.h, r.lo, r.layer, r.jitter, r.seed, stream, &mesh);
  if (st != NL_OK) return finish(st);
  int dim = 0;
  int64_t nv = 0, ne = 0;
  nl_mesh_info(mesh, &dim, &nv, &ne);
  std::vector<double> coords((size_t)dim * nv);
  std::vector<int32_t> conn((size_t)(dim + 1) * ne);
  std::vector<uint8_t> eio(ne), nf(nv);
  if ((st = nl_mesh_export(mesh, coords.data(), conn.data(), eio.data(), nf.data())) != NL_OK)
    return finish(st);
  if ((st = nl_pairs_build(mesh, r.kernel.delta, r.kernel.eps, &pairs)) != NL_OK) return finish(st);
  nl_assemble_stats ast;
  memset(&ast, 0, sizeof ast);
  if ((st = nl_assemble(mesh, pairs, &r.kernel, &r.quad, r.precision, &A, &ast)) != NL_OK)
    return finish(st);
  // u = g on the layer; f = -L_eps u = -Laplace(u) for the manufactured solutions used here
  std::vector<double> g(nv), f(nv);
  for (int64_t i = 0; i < nv; i++) {
    double x[3] = {0, 0, 0};
    for (int k = 0; k < dim; k++) x[k] = coords[(size_t)k * nv + i];
    g[i] = ms_u(r.ms, dim, x);
    double lap = 0.0;
    for (int k = 0; k < dim; k++) lap += r.ms == 1 ? 2.0 : r.ms == 2 ? 6.0 * x[k] : 0.0;
    f[i] = -lap;
  }
  if ((st = nl_rhs(mesh, A, f.data(), 0.0, g.data(), &rhs)) != NL_OK) return finish(st);
  std::vector<double> u(nv);
  int iters = 0;
  double rr = 0.0;
  st = nl_solve(A, rhs, g.data(), r.solver, r.rtol, r.max_iter,
                r.precision == NL_PREC_FP64 ? NL_PREC_FP64 : NL_PREC_FP32, u.data(), &iters, &rr);
  if (st != NL_OK) snprintf(res.message, sizeof res.message, "%s", nl_last_error());
  res.iters = iters;
  res.rel_res = rr;
  // ||u - u_h|| over Omega with the degree-5 rule on every element of Omega
  const nlx::Rule& rule = nlx::rule(dim);
  double err2 = 0.0;
  for (int64_t e = 0; e < ne; e++) {
    if (!eio[e]) continue;
    double V[4][3] = {{0}}, uh[4];
    for (int a = 0; a <= dim; a++) {
      const int32_t v = conn[(size_t)e * (dim + 1) + a];
      uh[a] = u[v];
      for (int k = 0; k < dim; k++) V[a][k] = coords[(size_t)k * nv + v];
    }
    double vol;
    if (dim == 2) {
      vol = 0.5 * std::fabs((V[1][0] - V[0][0]) * (V[2][1] - V[0][1]) - (V[2][0] - V[0][0]) * (V[1][1] - V[0][1]));
    } else {
      double a[3], b[3], c[3];
      for (int k = 0; k < 3; k++) {
        a[k] = V[1][k] - V[0][k];
        b[k] = V[2][k] - V[0][k];
        c[k] = V[3][k] - V[0][k];
      }
      vol = std::fabs(a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                      a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
    }
    for (int q = 0; q < rule.n; q++) {
      double x[3] = {0, 0, 0}, uq = 0.0;
      for (int a = 0; a <= dim; a++) {
        uq += rule.bary[q][a] * uh[a];
        for (int k = 0; k < dim; k++) x[k] += rule.bary[q][a] * V[a][k];
      }
      const double d = ms_u(r.ms, dim, x) - uq;
      err2 += rule.w[q] * vol * d * d;
    }
  }
  res.l2_err_omega = std::sqrt(err2);
  res.n_pairs = ast.n_pairs;
  res.n_point_pairs = ast.n_point_pairs;
  nl_pairs_info(pairs, nullptr, &res.nnz);
  res.n_vert = nv;
  if (r.u_out) memcpy(r.u_out, u.data(), sizeof(double) * nv);
  finish(st);
}

void worker_main(nl_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  for (;;) {
    uint64_t ticket = 0;
    Job* job = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        if (S->pending.empty()) return false;
        const Job& head = S->jobs[S->pending.front()];
        return S->in_use + head.est <= S->budget || S->running == 0;
      });
      if (S->stop) break;
      ticket = S->pending.front();
      S->pending.pop_front();
      job = &S->jobs[ticket];
      S->in_use += job->est;
      S->running++;
      job->res.t_start_ms = ms_since(S->t0);
    }
    run_request(S, stream, *job);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      job->res.t_done_ms = ms_since(S->t0);
      job->done = true;
      S->in_use -= job->est;
      S->running--;
      S->latencies.push_back(job->res.t_done_ms - job->res.t_submit_ms);
      S->last_done = job->res.t_done_ms;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

nl_status nl_serve_create(size_t device_mem_budget, int max_slots, nl_server** out) {
  nlx::clear_error();
  if (!out) return nlx::fail(NL_EINVAL, "nl_serve_create: out is NULL");
  if (max_slots < 1 || max_slots > 64) return nlx::fail(NL_EINVAL, "nl_serve_create: max_slots must be in [1, 64]");
  if (device_mem_budget < ((size_t)64 << 20)) return nlx::fail(NL_EINVAL, "nl_serve_create: budget below 64 MiB");
  NL_TRY(nlx::ensure_device_tables());
  nl_server* S = new nl_server();
  S->budget = device_mem_budget;
  S->slots = max_slots;
  S->block_budget = std::min<size_t>((size_t)256 << 20, device_mem_budget / (4 * (size_t)max_slots) + 1);
  S->t0 = Clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return nlx::fail(NL_ECUDA, "nl_serve_create: no current device");
  }
  for (int i = 0; i < max_slots; i++) S->workers.emplace_back(worker_main, S);
  *out = S;
  return NL_OK;
}

nl_status nl_serve_submit(nl_server* S, const nl_request* req, uint64_t* ticket) {
  nlx::clear_error();
  if (!S || !req || !ticket) return nlx::fail(NL_EINVAL, "nl_serve_submit: NULL argument");
  if (req->dim != 2 && req->dim != 3) return nlx::fail(NL_EINVAL, "nl_serve_submit: dim must be 2 or 3");
  if (!(req->kernel.eps > 0.0 && req->kernel.eps < req->kernel.delta))
    return nlx::fail(NL_EINVAL, "nl_serve_submit: need 0 < eps < delta");
  if (req->ms < 0 || req->ms > 2) return nlx::fail(NL_EINVAL, "nl_serve_submit: ms must be 0, 1 or 2");
  if (req->solver != 0 && req->solver != 1) return nlx::fail(NL_EINVAL, "nl_serve_submit: solver must be 0 or 1");
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t t = S->next_ticket++;
  Job& job = S->jobs[t];
  job.req = *req;
  memset(&job.res, 0, sizeof job.res);
  job.res.status = NL_EBUSY;
  job.res.t_submit_ms = ms_since(S->t0);
  if (S->first_submit < 0) S->first_submit = job.res.t_submit_ms;
  job.est = estimate_bytes(*req, S->block_budget);
  S->pending.push_back(t);
  *ticket = t;
  S->cv_work.notify_all();
  return NL_OK;
}

static nl_status take_result(nl_server* S, uint64_t ticket, nl_result* out) {
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return nlx::fail(NL_EINVAL, "nl_serve: unknown ticket %llu", (unsigned long long)ticket);
  if (!it->second.done) return NL_EBUSY;
  if (out) *out = it->second.res;
  S->jobs.erase(it);
  return NL_OK;
}

nl_status nl_serve_poll(nl_server* S, uint64_t ticket, nl_result* out) {
  nlx::clear_error();
  if (!S) return nlx::fail(NL_EINVAL, "nl_serve_poll: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  return take_result(S, ticket, out);
}

nl_status nl_serve_wait(nl_server* S, uint64_t ticket, double timeout_ms, nl_result* out) {
  nlx::clear_error();
  if (!S) return nlx::fail(NL_EINVAL, "nl_serve_wait: NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
  for (;;) {
    nl_status st = take_result(S, ticket, out);
    if (st != NL_EBUSY) return st;
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      st = take_result(S, ticket, out);
      if (st != NL_EBUSY) return st;
      return nlx::fail(NL_ETIMEOUT, "nl_serve_wait: ticket %llu not done after %.1f ms",
                       (unsigned long long)ticket, timeout_ms);
    }
  }
}

nl_status nl_serve_stats(nl_server* S, double* p50_ms, double* p99_ms, double* solves_per_s) {
  nlx::clear_error();
  if (!S) return nlx::fail(NL_EINVAL, "nl_serve_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    const double pos = p * (l.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (solves_per_s) {
    const double span = S->last_done - S->first_submit;
    *solves_per_s = (span > 0 && !l.empty()) ? 1e3 * l.size() / span : 0.0;
  }
  return NL_OK;
}

void nl_serve_destroy(nl_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
