// Continuous-batching request server: DM and inertia solves of systems of
// different sizes, admitted by device-memory footprint, running concurrently
// on per-slot CUDA streams.
//
// Admission: when a slot is idle, the first queued request (in arrival order)
// whose footprint (workspace for `batch` poles of its plan, from the
// stream-ordered allocator) fits the budget that running requests leave free;
// a request passed over kMaxBypass times blocks the ones behind it until it
// fits, so large requests are not starved. Requests that
// arrive while others run are admitted as slots and memory free up, and their
// kernels overlap on the device with those of the running requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.hpp"

using pexsi::CudaError;
using pexsi::ck;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t ticket = 0;
  pexsi_request req{};
  std::vector<double> H, S, shifts;
  int batch = 1;
  int64_t footprint = 0;
  enum State { QUEUED, RUNNING, DONE } state = QUEUED;
  std::atomic<bool> cancel{false};
  int bypassed = 0;  // times a later request was admitted before this one
  pexsi_result res{};
  Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct pexsi_server {
  pexsi_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_ticket = 1;
  int64_t budget = 0, in_use = 0, peak_bytes = 0;
  int running = 0, peak_running = 0;
  int64_t submitted = 0, completed = 0, cancelled = 0, failed = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
};

namespace {

void finish(pexsi_server* s, const std::shared_ptr<Request>& r, int status) {
  r->t_end = Clock::now();
  r->res.status = status;
  r->res.latency_ms = ms_between(r->t_submit, r->t_end);
  r->res.queue_ms = r->state == Request::RUNNING ? ms_between(r->t_submit, r->t_start) : r->res.latency_ms;
  r->res.run_ms = r->state == Request::RUNNING ? ms_between(r->t_start, r->t_end) : 0.0;
  r->state = Request::DONE;
  if (status == PEXSI_OK) ++s->completed;
  else if (status == PEXSI_ERR_CANCELLED) ++s->cancelled;
  else ++s->failed;
}

// Runs one admitted request on `st` with a workspace from the stream-ordered
// allocator.
int execute(Request& r, cudaStream_t st, std::string* err) {
  const pexsi_plan* p = r.req.plan;
  const size_t nnz = size_t(p->sym.nnz);
  pexsi::Workspace ws;
  ws.stream = st;
  ws.use_graphs = false;  // a request's workspace lives for one request
  int rc = PEXSI_OK;
  try {
    pexsi::workspace_alloc(p, ws, r.batch, st, true);
    ck(cudaMemcpyAsync(ws.H, r.H.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st), "H2D(H)");
    const double* dS = nullptr;
    if (!r.S.empty()) {
      ck(cudaMemcpyAsync(ws.S, r.S.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st), "H2D(S)");
      dS = ws.S;
    }
    if (r.req.n_shifts > 0)
      rc = pexsi::inertia_range(p, ws, nullptr, ws.H, dS, r.shifts.data(), r.req.n_shifts, r.req.counts, err);
    if (rc == PEXSI_OK && r.req.n_poles > 0) {
      double *o_dm = ws.out, *o_edm = ws.out + nnz, *o_fdm = ws.out + 2 * nnz;
      double* d_dm = r.req.dm ? o_dm : nullptr;
      double* d_edm = r.req.edm ? o_edm : nullptr;
      double* d_fdm = r.req.fdm ? o_fdm : nullptr;
      pexsi_dm_info info;
      // one device batch at a time so a cancellation takes effect between
      // them; the first batch (accumulate = 0) clears the status words and
      // the last one (info) reports a breakdown or timed-out wait of any batch
      for (int b0 = 0; b0 < r.req.n_poles && rc == PEXSI_OK; b0 += r.batch) {
        if (r.cancel.load()) { rc = PEXSI_ERR_CANCELLED; break; }
        int b1 = std::min(r.req.n_poles, b0 + r.batch);
        bool last = b1 == r.req.n_poles;
        rc = pexsi::dm_range(p, ws, nullptr, ws.H, dS, r.req.mu, r.req.beta, r.req.n_poles, r.req.delta_e, b0, b1,
                             b0 > 0, d_dm, d_edm, d_fdm, last ? &info : nullptr, err);
        if (last && rc == PEXSI_OK) {
          r.res.trace_dm_s = info.trace_dm_s;
          r.res.trace_edm_s = info.trace_edm_s;
          r.res.trace_fdm_s = info.trace_fdm_s;
          r.res.breakdown_front = info.breakdown_front;
        }
        if (rc == PEXSI_ERR_BREAKDOWN) r.res.breakdown_front = info.breakdown_front;
      }
      if (rc == PEXSI_OK) {
        if (r.req.dm) ck(cudaMemcpyAsync(r.req.dm, o_dm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st), "D2H");
        if (r.req.edm) ck(cudaMemcpyAsync(r.req.edm, o_edm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st), "D2H");
        if (r.req.fdm) ck(cudaMemcpyAsync(r.req.fdm, o_fdm, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st), "D2H");
      }
    }
    pexsi::workspace_free(ws);
    ck(cudaStreamSynchronize(st), "sync");
  } catch (const CudaError& ce) {
    pexsi::workspace_free(ws);
    cudaStreamSynchronize(st);
    *err = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
    return PEXSI_ERR_CUDA;
  }
  return rc;
}

// The queued request to admit next: the first (in arrival order) whose
// footprint fits what running requests leave of the budget. A request may be
// passed over by later, smaller ones at most kMaxBypass times; after that
// nothing behind it is admitted until it fits, so a large request cannot
// starve. Returns queue.end() when none may run now.
constexpr int kMaxBypass = 8;

std::deque<std::shared_ptr<Request>>::iterator next_admissible(pexsi_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (s->in_use + (*it)->footprint <= s->budget) return it;
    if ((*it)->bypassed >= kMaxBypass) break;  // it waits for room; no one passes it
  }
  return s->queue.end();
}

void worker(pexsi_server* s, int slot) {
  cudaSetDevice(s->opts.device);
  cudaStream_t st = s->streams[slot];
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || next_admissible(s) != s->queue.end(); });
      if (s->stop && s->queue.empty()) return;
      auto it = next_admissible(s);
      if (it == s->queue.end()) {
        if (s->stop) return;
        continue;
      }
      for (auto q = s->queue.begin(); q != it; ++q) ++(*q)->bypassed;
      r = *it;
      s->queue.erase(it);
      r->state = Request::RUNNING;
      r->t_start = Clock::now();
      s->in_use += r->footprint;
      s->peak_bytes = std::max(s->peak_bytes, s->in_use);
      ++s->running;
      s->peak_running = std::max(s->peak_running, s->running);
      r->res.max_concurrent = s->running;
    }
    std::string err;
    int rc = execute(*r, st, &err);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->footprint;
      --s->running;
      finish(s, r, rc);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

int pexsi_server_opts_default(pexsi_server_opts* o) {
  if (!o) return PEXSI_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->device = 0;
  o->slots = 4;
  o->batch = 8;
  return PEXSI_OK;
}

int pexsi_server_create(const pexsi_server_opts* opts, pexsi_server** out) {
  if (!out) return PEXSI_ERR_INVALID_ARG;
  *out = nullptr;
  pexsi_server_opts o;
  pexsi_server_opts_default(&o);
  if (opts) {
    o = *opts;
    if (o.slots <= 0) o.slots = 4;
    if (o.batch <= 0) o.batch = 8;
  }
  if (o.slots > 64 || o.batch > pexsi::kMaxBatch || o.device < 0) return PEXSI_ERR_INVALID_ARG;
  auto* s = new (std::nothrow) pexsi_server();
  if (!s) return PEXSI_ERR_NOMEM;
  s->opts = o;
  try {
    ck(cudaSetDevice(o.device), "cudaSetDevice");
    size_t free_b = 0, total_b = 0;
    ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    s->budget = o.hbm_budget > 0 ? o.hbm_budget : int64_t(0.6 * double(free_b));
    s->streams.resize(o.slots, nullptr);
    for (int i = 0; i < o.slots; ++i) ck(cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking), "stream");
  } catch (const CudaError&) {
    for (auto st : s->streams)
      if (st) cudaStreamDestroy(st);
    delete s;
    return PEXSI_ERR_CUDA;
  }
  for (int i = 0; i < o.slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return PEXSI_OK;
}

int pexsi_server_submit(pexsi_server* s, const pexsi_request* req, int64_t* ticket) {
  if (!s || !req || !ticket || !req->plan || !req->H) return PEXSI_ERR_INVALID_ARG;
  const pexsi_plan* p = req->plan;
  if (p->opts.device != s->opts.device) return PEXSI_ERR_INVALID_ARG;
  if (req->n_poles < 0 || (req->n_poles & 1) || req->n_shifts < 0 || (req->n_shifts > 0 && (!req->shifts || !req->counts)))
    return PEXSI_ERR_INVALID_ARG;
  if (req->n_poles == 0 && req->n_shifts == 0) return PEXSI_ERR_INVALID_ARG;
  if (req->n_poles > 0 && !(req->beta > 0 && req->delta_e > 0)) return PEXSI_ERR_INVALID_ARG;
  auto r = std::make_shared<Request>();
  r->req = *req;
  const size_t nnz = size_t(p->sym.nnz);
  try {
    r->H.assign(req->H, req->H + nnz);
    if (req->S) r->S.assign(req->S, req->S + nnz);
    if (req->n_shifts > 0) r->shifts.assign(req->shifts, req->shifts + req->n_shifts);
  } catch (const std::bad_alloc&) {
    return PEXSI_ERR_NOMEM;
  }
  // batch: the server's, shrunk until one request fits the whole budget
  int batch = std::max(1, std::min(s->opts.batch, std::max(req->n_poles, (req->n_shifts + 1) / 2)));
  while (batch > 1 && pexsi::bytes_fixed(p) + batch * pexsi::bytes_per_pole(p) > s->budget) --batch;
  r->batch = batch;
  r->footprint = pexsi::bytes_fixed(p) + batch * pexsi::bytes_per_pole(p);
  if (r->footprint > s->budget) return PEXSI_ERR_NOMEM;
  r->res.batch = batch;
  r->res.footprint_bytes = r->footprint;
  r->res.breakdown_front = -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return PEXSI_ERR_INVALID_ARG;
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    ++s->submitted;
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return PEXSI_OK;
}

int pexsi_server_poll(pexsi_server* s, int64_t ticket, pexsi_result* result) {
  if (!s) return PEXSI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return PEXSI_ERR_INVALID_ARG;
  if (it->second->state != Request::DONE) return PEXSI_PENDING;
  if (result) *result = it->second->res;
  return PEXSI_OK;
}

int pexsi_server_wait(pexsi_server* s, int64_t ticket, pexsi_result* result) {
  if (!s) return PEXSI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return PEXSI_ERR_INVALID_ARG;
  std::shared_ptr<Request> r = it->second;
  s->cv_done.wait(lk, [&] { return r->state == Request::DONE; });
  if (result) *result = r->res;
  return PEXSI_OK;
}

int pexsi_server_cancel(pexsi_server* s, int64_t ticket) {
  if (!s) return PEXSI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return PEXSI_ERR_INVALID_ARG;
    std::shared_ptr<Request> r = it->second;
    if (r->state == Request::QUEUED) {
      s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
      finish(s, r, PEXSI_ERR_CANCELLED);
    } else if (r->state == Request::RUNNING) {
      r->cancel.store(true);
    }
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return PEXSI_OK;
}

int pexsi_server_release(pexsi_server* s, int64_t ticket) {
  if (!s) return PEXSI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end() || it->second->state != Request::DONE) return PEXSI_ERR_INVALID_ARG;
  s->all.erase(it);
  return PEXSI_OK;
}

int pexsi_server_get_stats(pexsi_server* s, pexsi_server_stats* st) {
  if (!s || !st) return PEXSI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->cancelled = s->cancelled;
  st->failed = s->failed;
  st->queued = int64_t(s->queue.size());
  st->running = s->running;
  st->bytes_in_use = s->in_use;
  st->peak_bytes = s->peak_bytes;
  st->budget = s->budget;
  st->peak_concurrent = s->peak_running;
  return PEXSI_OK;
}

int pexsi_server_destroy(pexsi_server* s) {
  if (!s) return PEXSI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->queue) finish(s, r, PEXSI_ERR_CANCELLED);
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto& t : s->workers) t.join();
  cudaSetDevice(s->opts.device);
  for (auto st : s->streams)
    if (st) cudaStreamDestroy(st);
  delete s;
  return PEXSI_OK;
}

}  // extern "C"
