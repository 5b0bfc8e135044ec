// Batch executor and request server: many independent fracture problems on
// one GPU at once.  Neither has a counterpart in the paper, which solves one
// problem per run; they exist because small instances cannot fill a GB300 by
// themselves (their kernels are launch- and latency-bound), while several of
// them running on separate streams overlap on the device.
//
// Concurrency model: host worker threads, each owning one non-blocking CUDA
// stream.  A worker drives one problem at a time through the ordinary solver
// (the same Newton / active-set / FGMRES code as pff_solve_loading_steps), so
// a problem's result does not depend on what else runs.  The library's shared
// state (allocator bookkeeping, autotune cache, profiler) is mutex-guarded and
// graph capture is thread-local, so workers need no further coordination.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pff_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes of a problem with nn nodes in dim dimensions and an FGMRES
// restart of m: the Krylov basis (V: m+1, Z: m vectors, and V's FP32 copy),
// plus per node the state, the stencils and their FP32 copies, both AMG
// hierarchies and the set-up temporaries (measured peaks of the stream-ordered
// pool: about 12 KB per node for a 2d 256^2 request including the fixed cost
// below, 20.3 KB per node for the 3d 128^3 one), plus a fixed allowance for
// module load and pool granularity.  The per-cell quadrature records of the residual and the
// phase-field assembly come on top (fewer cells than nodes, so nn bounds them).
int64_t estimate_bytes(int dim, int64_t nn, int m) {
  const int64_t ndof = (int64_t)(dim + 1) * nn;
  const int64_t krylov = (int64_t)(2 * m + 3) * ndof * 8 + (int64_t)(m + 1) * ndof * 4;
  const int64_t per_node = dim == 2 ? 6000 : 19500;
  return krylov + per_node * nn + 8 * pff::qp_doubles(dim, nn) + (512LL << 20);
}

int64_t nodes_of(int dim, const int32_t* n_cells) {
  int64_t nn = 1;
  for (int a = 0; a < dim; ++a) nn *= (int64_t)n_cells[a] + 1;
  return nn;
}

struct StreamGuard {
  cudaStream_t s = nullptr;
  StreamGuard() {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      throw pff::Failure{PFF_ERR_CUDA, "cannot create a worker stream"};
  }
  ~StreamGuard() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  }
};

int worker_count(int requested, int jobs) {
  int w = requested > 0 ? requested : std::min(jobs, 16);
  return std::max(1, std::min(w, std::max(1, jobs)));
}

}  // namespace

// ------------------------------------------------------------- server ------
struct Job {
  int64_t id = 0;
  int dim = 2;
  int32_t n_cells[3] = {1, 1, 1};
  std::vector<double> axis[3];
  double E = 1, nu = 0.2, Gc = 1, kappa = 1e-10, eps = 0.1, l0 = 0.25;
  std::vector<double> schedule, cod_x, cod;
  bool keep = false;
  std::vector<double> u, phi;
  std::vector<uint8_t> active;
  pff_request_result res{};
};

struct pff_server {
  int64_t budget = 0;
  pff_options opts{};
  Clock::time_point t0 = Clock::now();
  std::mutex mu;
  std::condition_variable cv_work;   // queue or capacity changed
  std::condition_variable cv_done;   // a request finished
  std::deque<Job*> queue;
  std::unordered_map<int64_t, Job*> jobs;
  int64_t reserved = 0, peak = 0;
  int running = 0, finished = 0, max_running = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Solve one admitted request on stream s; fills job->res (status, results).
void run_job(pff_server* srv, Job* J, cudaStream_t s) {
  pff_problem* P = nullptr;
  int rc = PFF_OK;
  try {
    const double* ax[3] = {J->axis[0].data(), J->axis[1].data(), J->axis[2].data()};
    P = pff::create_problem(J->dim, J->n_cells, ax, s);
    rc = pff_set_material(P, J->E, J->nu, J->Gc, J->kappa, J->eps);
    if (rc == PFF_OK) rc = pff_set_crack(P, J->l0);
    std::vector<pff_step_report> reps(J->schedule.size());
    if (rc == PFF_OK)
      rc = pff_solve_loading_steps(P, (int)J->schedule.size(), J->schedule.data(), &srv->opts,
                                   reps.data());
    for (const auto& r : reps) {
      J->res.newton_its += r.newton_its;
      J->res.krylov_its += r.krylov_its;
      J->res.converged_steps += r.converged;
    }
    if (rc == PFF_OK) {
      // one COD line per abscissa: along y in 2d, along z through y = 0 in 3d
      std::vector<double> pts;
      pts.reserve(J->cod_x.size() * (J->dim - 1));
      for (double x : J->cod_x) {
        pts.push_back(x);
        if (J->dim == 3) pts.push_back(0.0);
      }
      J->cod.assign(J->cod_x.size(), 0.0);
      rc = pff_eval_tcv_cod(P, (int)J->cod_x.size(), pts.data(), &J->res.tcv, J->cod.data());
    }
    if (rc == PFF_OK && J->keep) {
      const size_t n = (size_t)P->n_nodes;
      J->u.resize(n * J->dim);
      J->phi.resize(n);
      J->active.resize(n);
      rc = pff_get_solution(P, J->u.data(), J->phi.data(), J->active.data());
    }
  } catch (const pff::Failure& f) {
    pff::set_error(f.code, f.msg);
    rc = f.code;
  } catch (...) {
    rc = PFF_ERR_INVALID_ARG;
  }
  if (P) pff_destroy(P);
  J->res.status = rc;
}

void worker_loop_on(pff_server* srv, StreamGuard& sg) {
  std::unique_lock<std::mutex> lk(srv->mu);
  while (true) {
    // admit the head of the queue when it fits (or when nothing else runs)
    srv->cv_work.wait(lk, [&] {
      if (srv->stop) return true;
      if (srv->queue.empty()) return false;
      const Job* h = srv->queue.front();
      return srv->running == 0 || srv->reserved + h->res.bytes <= srv->budget;
    });
    if (srv->stop) return;
    Job* J = srv->queue.front();
    srv->queue.pop_front();
    srv->reserved += J->res.bytes;
    srv->peak = std::max(srv->peak, srv->reserved);
    srv->running += 1;
    srv->max_running = std::max(srv->max_running, srv->running);
    J->res.t_admit = srv->now();
    // the next worker may admit the new head right away if it fits too
    srv->cv_work.notify_all();
    lk.unlock();
    run_job(srv, J, sg.s);
    lk.lock();
    J->res.t_finish = srv->now();
    J->res.done = 1;
    srv->reserved -= J->res.bytes;
    srv->running -= 1;
    srv->finished += 1;
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

void worker_loop(pff_server* srv) {
  try {
    StreamGuard sg;
    worker_loop_on(srv, sg);
  } catch (...) {
    // no stream for this worker: the others serve the queue
  }
}

}  // namespace

extern "C" {

int64_t pff_request_bytes(int dim, const int32_t* n_cells) {
  if ((dim != 2 && dim != 3) || !n_cells) return -1;
  return estimate_bytes(dim, nodes_of(dim, n_cells), 40);
}

int pff_batch_solve(int n, pff_problem* const* problems, const int* n_steps,
                    const double* const* schedules, const pff_options* opts,
                    pff_step_report* const* reports, int n_workers, int* status) {
  try {
    if (n < 0 || (n > 0 && (!problems || !n_steps || !schedules || !reports))) {
      pff::set_error(PFF_ERR_INVALID_ARG, "pff_batch_solve: NULL or negative argument");
      return PFF_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i) {
      if (!problems[i] || n_steps[i] < 0 || (n_steps[i] > 0 && (!schedules[i] || !reports[i]))) {
        pff::set_error(PFF_ERR_INVALID_ARG, "pff_batch_solve: bad problem, schedule or report");
        return PFF_ERR_INVALID_ARG;
      }
      for (int j = 0; j < i; ++j)
        if (problems[j] == problems[i]) {
          pff::set_error(PFF_ERR_INVALID_ARG, "pff_batch_solve: a problem appears twice");
          return PFF_ERR_INVALID_ARG;
        }
    }
    // largest first: the long solves start early and the short ones fill in
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return problems[a]->n_dofs > problems[b]->n_dofs;
    });
    std::vector<int> st(n, PFF_OK);
    std::mutex mu;
    size_t next = 0;
    auto work = [&]() {
      StreamGuard sg;
      while (true) {
        int i;
        {
          std::lock_guard<std::mutex> g(mu);
          if (next >= order.size()) return;
          i = order[next++];
        }
        pff_problem* P = problems[i];
        void* own = P->stream;
        int rc = pff_set_stream(P, sg.s);
        if (rc == PFF_OK)
          rc = pff_solve_loading_steps(P, n_steps[i], schedules[i], opts, reports[i]);
        const int rc2 = pff_set_stream(P, own);
        st[i] = rc != PFF_OK ? rc : rc2;
      }
    };
    const int w = worker_count(n_workers, n);
    std::vector<std::thread> th;
    for (int k = 1; k < w; ++k) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
    int rc = PFF_OK;
    for (int i = 0; i < n; ++i) {
      if (status) status[i] = st[i];
      if (rc == PFF_OK && st[i] != PFF_OK) rc = st[i];
    }
    if (rc != PFF_OK) pff::set_error(rc, "pff_batch_solve: at least one problem failed");
    return rc;
  } catch (const pff::Failure& f) {
    pff::set_error(f.code, f.msg);
    return f.code;
  } catch (const std::exception& e) {
    pff::set_error(PFF_ERR_INVALID_ARG, e.what());
    return PFF_ERR_INVALID_ARG;
  }
}

int pff_server_create(int64_t budget_bytes, int n_workers, const pff_options* opts,
                      pff_server** out) {
  if (!out || budget_bytes <= 0 || n_workers < 1 || n_workers > 64) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_create: bad budget, worker count or out");
    return PFF_ERR_INVALID_ARG;
  }
  if (pff_check_options(opts) != PFF_OK) return PFF_ERR_INVALID_ARG;   // message already set
  auto* S = new pff_server();
  S->budget = budget_bytes;
  pff_default_options(&S->opts);
  if (opts) S->opts = *opts;
  try {
    for (int k = 0; k < n_workers; ++k) S->workers.emplace_back(worker_loop, S);
  } catch (...) {
    pff_server_destroy(S);
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_create: cannot start workers");
    return PFF_ERR_INVALID_ARG;
  }
  *out = S;
  return PFF_OK;
}

int pff_server_submit(pff_server* S, const pff_request* r, int64_t* id) {
  if (!S || !r || !id || (r->dim != 2 && r->dim != 3) || r->n_steps < 0 || r->n_cod < 0 ||
      (r->n_steps > 0 && !r->schedule) || (r->n_cod > 0 && !r->cod_x)) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_submit: bad request");
    return PFF_ERR_INVALID_ARG;
  }
  auto* J = new Job();
  J->dim = r->dim;
  for (int a = 0; a < r->dim; ++a) {
    if (r->n_cells[a] < 1 || !r->axis_coords[a]) {
      delete J;
      pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_submit: bad mesh");
      return PFF_ERR_INVALID_ARG;
    }
    J->n_cells[a] = r->n_cells[a];
    J->axis[a].assign(r->axis_coords[a], r->axis_coords[a] + r->n_cells[a] + 1);
  }
  J->E = r->E;
  J->nu = r->nu;
  J->Gc = r->Gc;
  J->kappa = r->kappa;
  J->eps = r->eps;
  J->l0 = r->l0;
  J->schedule.assign(r->schedule, r->schedule + r->n_steps);
  J->cod_x.assign(r->cod_x, r->cod_x + r->n_cod);
  J->keep = r->keep_solution != 0;
  const int64_t nn = nodes_of(J->dim, J->n_cells);
  J->res.n_dofs = (int64_t)(J->dim + 1) * nn;
  J->res.bytes = estimate_bytes(J->dim, nn, std::min(60, std::max(2, S->opts.krylov_restart)));
  std::lock_guard<std::mutex> g(S->mu);
  if (S->stop) {
    delete J;
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_submit: server is stopping");
    return PFF_ERR_INVALID_ARG;
  }
  J->id = S->next_id++;
  J->res.t_submit = S->now();
  S->jobs[J->id] = J;
  S->queue.push_back(J);
  *id = J->id;
  S->cv_work.notify_all();
  return PFF_OK;
}

static Job* find_job(pff_server* S, int64_t id) {
  auto it = S->jobs.find(id);
  return it == S->jobs.end() ? nullptr : it->second;
}

int pff_server_result(pff_server* S, int64_t id, pff_request_result* res) {
  if (!S || !res) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  Job* J = find_job(S, id);
  if (!J) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_result: unknown request");
    return PFF_ERR_INVALID_ARG;
  }
  *res = J->res;
  return PFF_OK;
}

int pff_server_wait(pff_server* S, int64_t id, double timeout_s, pff_request_result* res) {
  if (!S) return PFF_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  Job* J = find_job(S, id);
  if (!J) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_wait: unknown request");
    return PFF_ERR_INVALID_ARG;
  }
  auto done = [&] { return J->res.done != 0; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, done);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
    if (res) *res = J->res;
    pff::set_error(PFF_ERR_TIMEOUT, "pff_server_wait: request not finished in time");
    return PFF_ERR_TIMEOUT;
  }
  if (res) *res = J->res;
  return PFF_OK;
}

int pff_server_cod(pff_server* S, int64_t id, double* cod) {
  if (!S || !cod) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  Job* J = find_job(S, id);
  if (!J || !J->res.done) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_cod: unknown or unfinished request");
    return PFF_ERR_INVALID_ARG;
  }
  std::copy(J->cod.begin(), J->cod.end(), cod);
  return PFF_OK;
}

int pff_server_solution(pff_server* S, int64_t id, double* u, double* phi, uint8_t* active) {
  if (!S) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  Job* J = find_job(S, id);
  if (!J || !J->res.done || !J->keep || J->res.status != PFF_OK) {
    pff::set_error(PFF_ERR_INVALID_ARG,
                   "pff_server_solution: request unknown, unfinished, failed or not kept");
    return PFF_ERR_INVALID_ARG;
  }
  if (u) std::copy(J->u.begin(), J->u.end(), u);
  if (phi) std::copy(J->phi.begin(), J->phi.end(), phi);
  if (active) std::copy(J->active.begin(), J->active.end(), active);
  return PFF_OK;
}

int pff_server_release(pff_server* S, int64_t id) {
  if (!S) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  Job* J = find_job(S, id);
  if (!J || !J->res.done) {
    pff::set_error(PFF_ERR_INVALID_ARG, "pff_server_release: unknown or unfinished request");
    return PFF_ERR_INVALID_ARG;
  }
  S->jobs.erase(id);
  delete J;
  return PFF_OK;
}

int pff_server_stats_get(pff_server* S, pff_server_stats* st) {
  if (!S || !st) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  st->budget_bytes = S->budget;
  st->reserved_bytes = S->reserved;
  st->peak_reserved_bytes = S->peak;
  st->queued = (int)S->queue.size();
  st->running = S->running;
  st->finished = S->finished;
  st->max_running = S->max_running;
  return PFF_OK;
}

void pff_server_destroy(pff_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    S->queue.clear();
    S->cv_work.notify_all();
  }
  for (auto& t : S->workers)
    if (t.joinable()) t.join();
  for (auto& kv : S->jobs) delete kv.second;
  delete S;
}

}  // extern "C"
