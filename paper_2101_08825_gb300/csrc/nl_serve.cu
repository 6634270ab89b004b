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
#include <memory>
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
  bool small = false;  // few enough pairs to be assembled in a batched plan with others
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

// Rough upper estimate of a request's element pairs.
double estimate_pairs(const nl_request& r) {
  const int D = r.dim;
  double cells = 1.0;
  for (int k = 0; k < D; k++) cells *= r.cells[k] + 2.0 * r.layer;
  const double epc = D == 2 ? 2.0 : 6.0;
  const double span = 2.0 * std::ceil((r.kernel.delta + r.kernel.eps) / r.h) + 3.0;
  return cells * epc * epc * std::pow(span, D);
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
  double small_pairs = 4.0e6;  // requests below this many (estimated) pairs are batched
  int max_group = 16;          // requests per batched plan
  int64_t groups = 0;
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

// A request's mesh and pattern on the device, and the host copy of its mesh (for the
// manufactured solution and the error).
struct Prepared {
  nl_mesh* mesh = nullptr;
  nl_pairs* pairs = nullptr;
  int dim = 0;
  int64_t nv = 0, ne = 0;
  std::vector<double> coords;
  std::vector<int32_t> conn;
  std::vector<uint8_t> eio, nf;
  ~Prepared() {
    nl_pairs_destroy(pairs);
    nl_mesh_destroy(mesh);
  }
};

nl_status prepare(const nl_request& r, cudaStream_t stream, Prepared& pr) {
  NL_TRY(nl_mesh_create_box(r.dim, r.cells, r.h, r.lo, r.layer, r.jitter, r.seed, stream, &pr.mesh));
  nl_mesh_info(pr.mesh, &pr.dim, &pr.nv, &pr.ne);
  pr.coords.resize((size_t)pr.dim * pr.nv);
  pr.conn.resize((size_t)(pr.dim + 1) * pr.ne);
  pr.eio.resize(pr.ne);
  pr.nf.resize(pr.nv);
  NL_TRY(nl_mesh_export(pr.mesh, pr.coords.data(), pr.conn.data(), pr.eio.data(), pr.nf.data()));
  return nl_pairs_build(pr.mesh, r.kernel.delta, r.kernel.eps, &pr.pairs);
}

// Right-hand side with lifting, solve and error of one request whose matrix is assembled.
nl_status solve_and_report(const nl_request& r, Prepared& pr, nl_matrix* A,
                           const nl_assemble_stats& ast, nl_result& res) {
  const int dim = pr.dim;
  const int64_t nv = pr.nv, ne = pr.ne;
  // u = g on the layer; f = -L_eps u = -Laplace(u) for the manufactured solutions used here
  std::vector<double> g(nv), f(nv);
  for (int64_t i = 0; i < nv; i++) {
    double x[3] = {0, 0, 0};
    for (int k = 0; k < dim; k++) x[k] = pr.coords[(size_t)k * nv + i];
    g[i] = ms_u(r.ms, dim, x);
    double lap = 0.0;
    for (int k = 0; k < dim; k++) lap += r.ms == 1 ? 2.0 : r.ms == 2 ? 6.0 * x[k] : 0.0;
    f[i] = -lap;
  }
  nl_vector* rhs = nullptr;
  nl_status st = nl_rhs(pr.mesh, A, f.data(), 0.0, g.data(), &rhs);
  if (st != NL_OK) return st;
  std::vector<double> u(nv);
  int iters = 0;
  double rr = 0.0;
  st = nl_solve(A, rhs, g.data(), r.solver, r.rtol, r.max_iter,
                r.precision == NL_PREC_FP64 ? NL_PREC_FP64 : NL_PREC_FP32, u.data(), &iters, &rr);
  nl_vector_destroy(rhs);
  if (st != NL_OK) snprintf(res.message, sizeof res.message, "%s", nl_last_error());
  res.iters = iters;
  res.rel_res = rr;
  // ||u - u_h|| over Omega with the degree-5 rule on every element of Omega
  const nlx::Rule& rule = nlx::rule(dim);
  double err2 = 0.0;
  for (int64_t e = 0; e < ne; e++) {
    if (!pr.eio[e]) continue;
    double V[4][3] = {{0}}, uh[4];
    for (int a = 0; a <= dim; a++) {
      const int32_t v = pr.conn[(size_t)e * (dim + 1) + a];
      uh[a] = u[v];
      for (int k = 0; k < dim; k++) V[a][k] = pr.coords[(size_t)k * nv + v];
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
  nl_pairs_info(pr.pairs, nullptr, &res.nnz);
  res.n_vert = nv;
  if (r.u_out) memcpy(r.u_out, u.data(), sizeof(double) * nv);
  return st;
}

void set_status(nl_result& res, nl_status st) {
  res.status = st;
  if (st != NL_OK && res.message[0] == 0) snprintf(res.message, sizeof res.message, "%s", nl_last_error());
}

// Runs one request on `stream`: mesh, pairs, its own assembly, solve.
void run_request(nl_server* S, cudaStream_t stream, Job& job) {
  const nl_request& r = job.req;
  nlx::g_block_budget = S->block_budget;
  Prepared pr;
  nl_status st = prepare(r, stream, pr);
  if (st != NL_OK) return set_status(job.res, st);
  nl_assemble_stats ast;
  memset(&ast, 0, sizeof ast);
  nl_matrix* A = nullptr;
  st = nl_assemble(pr.mesh, pr.pairs, &r.kernel, &r.quad, r.precision, &A, &ast);
  if (st == NL_OK) st = solve_and_report(r, pr, A, ast, job.res);
  nl_matrix_destroy(A);
  set_status(job.res, st);
}

// Runs a group of small requests of one dimension and precision class: each request's mesh
// and pattern on `stream`, then one batched plan assembles all of them in a single launch of
// the assembly kernel (and one scatter), then every request is solved; complete() is called
// for each request as soon as its own result is ready.  If the plan cannot be created (device
// memory), the requests are assembled one by one.
template <typename F>
void run_group(nl_server* S, cudaStream_t stream, const std::vector<Job*>& js, F complete) {
  nlx::g_block_budget = S->block_budget;
  const int n = (int)js.size();
  std::vector<std::unique_ptr<Prepared>> prs(n);
  std::vector<int> idx;
  for (int k = 0; k < n; k++) {
    prs[k].reset(new Prepared());
    const nl_status st = prepare(js[k]->req, stream, *prs[k]);
    if (st != NL_OK) {
      set_status(js[k]->res, st);
      prs[k].reset();
      complete(*js[k]);
    } else {
      idx.push_back(k);
    }
  }
  if (idx.empty()) return;
  std::vector<nl_mesh*> ms;
  std::vector<nl_pairs*> ps;
  std::vector<nl_kernel_params> kps;
  std::vector<nl_quad_params> qps;
  for (int k : idx) {
    ms.push_back(prs[k]->mesh);
    ps.push_back(prs[k]->pairs);
    kps.push_back(js[k]->req.kernel);
    qps.push_back(js[k]->req.quad);
  }
  const nl_precision prec = js[idx[0]]->req.precision == NL_PREC_FP64 ? NL_PREC_FP64 : NL_PREC_FP32;
  nl_plan* plan = nullptr;
  nl_status pst = nl_plan_create((int)idx.size(), ms.data(), ps.data(), kps.data(), qps.data(),
                                 prec, 0, stream, &plan);
  std::vector<nl_assemble_stats> stats(idx.size());
  if (pst == NL_OK) pst = nl_plan_execute(plan);
  if (pst == NL_OK) pst = nl_plan_sync(plan, stats.data());
  for (size_t j = 0; j < idx.size(); j++) {
    const int k = idx[j];
    Job& job = *js[k];
    nl_matrix* A = nullptr;
    nl_status st;
    if (pst == NL_OK) {
      st = nl_plan_matrix(plan, (int)j, &A);
      if (st == NL_OK) st = solve_and_report(job.req, *prs[k], A, stats[j], job.res);
    } else {
      nl_assemble_stats ast;
      memset(&ast, 0, sizeof ast);
      st = nl_assemble(prs[k]->mesh, prs[k]->pairs, &job.req.kernel, &job.req.quad,
                       job.req.precision, &A, &ast);
      if (st == NL_OK) st = solve_and_report(job.req, *prs[k], A, ast, job.res);
    }
    nl_matrix_destroy(A);
    set_status(job.res, st);
    complete(job);
  }
  nl_plan_destroy(plan);
}

void worker_main(nl_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  auto complete = [&](Job& job) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      job.res.t_done_ms = ms_since(S->t0);
      job.done = true;
      S->in_use -= job.est;
      S->running--;
      S->latencies.push_back(job.res.t_done_ms - job.res.t_submit_ms);
      S->last_done = job.res.t_done_ms;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  };
  for (;;) {
    std::vector<Job*> group;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        if (S->pending.empty()) return false;
        const Job& head = S->jobs[S->pending.front()];
        return S->in_use + head.est <= S->budget || S->running == 0;
      });
      if (S->stop) break;
      const double now = ms_since(S->t0);
      Job* head = &S->jobs[S->pending.front()];
      S->pending.pop_front();
      S->in_use += head->est;
      S->running++;
      head->res.t_start_ms = now;
      group.push_back(head);
      if (head->small) {
        // continuous batching of small requests: later small requests of the same dimension
        // and precision class that fit the memory left join this one's launch
        for (auto it = S->pending.begin(); it != S->pending.end() && (int)group.size() < S->max_group;) {
          Job& o = S->jobs[*it];
          if (o.small && o.req.dim == head->req.dim &&
              (o.req.precision == NL_PREC_FP64) == (head->req.precision == NL_PREC_FP64) &&
              S->in_use + o.est <= S->budget) {
            S->in_use += o.est;
            S->running++;
            o.res.t_start_ms = now;
            o.res.group = (int32_t)S->groups;
            group.push_back(&o);
            it = S->pending.erase(it);
          } else {
            ++it;
          }
        }
        if (group.size() > 1) head->res.group = (int32_t)S->groups++;
      }
    }
    if (group.size() == 1) {
      run_request(S, stream, *group[0]);
      complete(*group[0]);
    } else {
      run_group(S, stream, group, complete);
    }
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
  job.small = estimate_pairs(*req) <= S->small_pairs;
  job.res.group = -1;
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
