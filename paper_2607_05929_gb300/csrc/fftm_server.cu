// Serving runtime: a request queue over one GPU (no counterpart in the paper, whose
// solver runs one problem per MPI job).
//
// A request is a problem description plus a sequence of load steps.  The server keeps
// up to `max_slots` solves resident at once, each on its own CUDA stream, so the
// fixed-point iterations of different solves interleave on the device (continuous
// batching: a queued request is admitted as soon as a slot and enough of the memory
// budget are free; each resident solve keeps its fields and acceleration history on
// the device until its last load step).  Admission is first-fit over the queue in
// arrival order against the budget, using fftm_problem_workspace_bytes.
//
// Every solve runs the same kernels with the same launch shapes as it would alone;
// none of them uses atomics, so a result does not depend on what else is resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fftm.h"
#include "../../include/fftm_server.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long long id = 0;
  fftm_problem_desc desc;
  std::vector<uint16_t> phase;
  std::vector<fftm_material> mats;
  std::vector<fftm_load> loads;
  void* u_out = nullptr;  // host buffer for the final u^f (optional)
  size_t u_out_bytes = 0;
  size_t need = 0;        // workspace bytes
  double t_submit = 0.0;
  std::vector<std::pair<int, int>> options;  // fftm_set_option calls for the request's problem
};

}  // namespace

struct fftm_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int max_slots = 1;
  long long next_id = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::deque<fftm_result> done;
  int active = 0;
  int live = 0;      // workers that created their stream and context and are serving
  int started = 0;   // workers that finished starting up (successfully or not)
  std::condition_variable cv_start;
  std::vector<std::thread> workers;
  std::string error;
  std::vector<std::pair<int, int>> options;  // applied to the problems of requests submitted later
};

namespace {

// Host-side fault injection for the tests: the next g_fail_starts workers fail to start as if
// their stream or context could not be created.
std::atomic<int> g_fail_starts{0};

int fail(fftm_server* s, const std::string& msg, int code) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->error = msg;
  return code;
}

// Run one request to completion on the worker's context; fills `r`.
void run_request(fftm_ctx* ctx, Request& q, fftm_result& r) {
  std::memset(&r, 0, sizeof(r));
  r.id = q.id;
  r.t_submit = q.t_submit;
  r.t_start = now_s();
  fftm_problem* p = nullptr;
  q.desc.phase = q.phase.data();
  q.desc.materials = q.mats.data();
  int st = fftm_problem_create(ctx, &q.desc, &p);
  for (size_t k = 0; st == FFTM_OK && k < q.options.size(); ++k) st = fftm_set_option(p, q.options[k].first, q.options[k].second);
  if (st == FFTM_OK) {
    for (size_t k = 0; k < q.loads.size() && st >= 0; ++k) {
      st = fftm_set_load(p, &q.loads[k]);
      if (st < 0) break;
      fftm_step_report rep;
      st = fftm_solve_step(p, &rep, nullptr, nullptr, 0);
      if (st < 0) break;
      r.iterations += rep.iterations;
      r.steps += 1;
      r.converged_steps += rep.converged;
      r.err = rep.err;
      std::memcpy(r.mean_P, rep.mean_P, sizeof(r.mean_P));
    }
    if (st >= 0 && q.u_out) st = fftm_get_field(p, FFTM_FIELD_U, q.u_out, 0, q.u_out_bytes);
  }
  r.status = st < 0 ? st : (r.converged_steps == r.steps ? FFTM_OK : FFTM_NOT_CONVERGED);
  if (st < 0) std::strncpy(r.message, fftm_last_error(), sizeof(r.message) - 1);
  if (p) fftm_problem_destroy(p);
  r.t_end = now_s();
}

// Fail every queued request (no worker is left to run them).
void fail_queue_locked(fftm_server* s) {
  while (!s->queue.empty()) {
    fftm_result r;
    std::memset(&r, 0, sizeof(r));
    r.id = s->queue.front()->id;
    r.t_submit = s->queue.front()->t_submit;
    r.t_start = r.t_end = now_s();
    r.status = FFTM_E_CUDA;
    std::strncpy(r.message, "no server worker is running", sizeof(r.message) - 1);
    s->queue.pop_front();
    s->done.push_back(r);
  }
}

void worker_main(fftm_server* s) {
  cudaStream_t stream = nullptr;
  fftm_ctx* ctx = nullptr;
  bool ok = false;
  int expected = g_fail_starts.load();
  while (expected > 0 && !g_fail_starts.compare_exchange_weak(expected, expected - 1)) {
  }
  if (expected <= 0)
    ok = cudaSetDevice(s->device) == cudaSuccess &&
         cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
         fftm_ctx_create(&ctx, s->device, stream) == FFTM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->started += 1;
    if (ok) s->live += 1;
    else s->error = "worker could not create its stream or context";
  }
  s->cv_start.notify_all();
  if (!ok) {
    if (stream) cudaStreamDestroy(stream);
    return;
  }
  for (;;) {
    std::unique_ptr<Request> q;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stopping && s->queue.empty()) break;
        // first fit in arrival order against the memory budget
        auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const std::unique_ptr<Request>& r) {
          return s->in_use + r->need <= s->budget;
        });
        if (it != s->queue.end()) {
          q = std::move(*it);
          s->queue.erase(it);
          s->in_use += q->need;
          s->active += 1;
          break;
        }
        s->cv_work.wait(lk);
      }
    }
    if (!q) break;
    fftm_result r;
    run_request(ctx, *q, r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= q->need;
      s->active -= 1;
      s->done.push_back(r);
    }
    s->cv_work.notify_all();  // memory freed: another queued request may fit now
    s->cv_done.notify_all();
  }
  fftm_ctx_destroy(ctx);
  cudaStreamDestroy(stream);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->live -= 1;
    if (s->live == 0) fail_queue_locked(s);
  }
  s->cv_done.notify_all();
}

}  // namespace

extern "C" {

int fftm_server_create(int device, size_t memory_budget, int max_slots, fftm_server** out) {
  if (!out || max_slots < 1 || max_slots > 64) return FFTM_E_INVALID;
  // every worker set to fail at start needs no device (host-side tests of that path)
  const bool all_fail = g_fail_starts.load() >= max_slots;
  if (!all_fail) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return FFTM_E_INVALID;
    if (memory_budget == 0) {
      size_t free_b = 0, total_b = 0;
      cudaSetDevice(device);
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return FFTM_E_CUDA;
      memory_budget = free_b / 10 * 9;  // leave a tenth for the runtime and other users
    }
  }
  fftm_server* s = new (std::nothrow) fftm_server;
  if (!s) return FFTM_E_NOMEM;
  s->device = device;
  s->budget = memory_budget;
  s->max_slots = max_slots;
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s);
  int live = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_start.wait(lk, [&] { return s->started == max_slots; });
    live = s->live;
  }
  if (live == 0) {  // nothing could start: report it instead of queueing requests nobody runs
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
    return FFTM_E_CUDA;
  }
  *out = s;
  return FFTM_OK;
}

int fftm_server_submit(fftm_server* s, const fftm_request* req, long long* id) {
  if (!s || !req || !req->desc || !req->desc->phase || !req->desc->materials || req->n_loads < 1 || !req->loads)
    return FFTM_E_INVALID;
  size_t need = 0;
  int st = fftm_problem_workspace_bytes(req->desc, &need);
  if (st != FFTM_OK) return st;
  need += 64u << 20;  // scratch, tables and allocator slack per resident solve
  if (need > s->budget) return fail(s, "request larger than the server's memory budget", FFTM_E_NOMEM);
  auto q = std::make_unique<Request>();
  q->desc = *req->desc;
  const size_t nvox = (size_t)q->desc.n[0] * q->desc.n[1] * q->desc.n[2];
  q->phase.assign(req->desc->phase, req->desc->phase + nvox);
  q->mats.assign(req->desc->materials, req->desc->materials + req->desc->n_phases);
  q->loads.assign(req->loads, req->loads + req->n_loads);
  q->u_out = req->u_out;
  q->u_out_bytes = req->u_out_bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->options = s->options;
  }
  q->need = need;
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return FFTM_E_INVALID;
    if (s->live == 0) return FFTM_E_CUDA;
    q->id = s->next_id++;
    if (id) *id = q->id;
    s->queue.push_back(std::move(q));
  }
  s->cv_work.notify_all();
  return FFTM_OK;
}

int fftm_server_poll(fftm_server* s, fftm_result* out, int max_results, int wait_for_one, int* n_out) {
  if (!s || !n_out || (max_results > 0 && !out)) return FFTM_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait_for_one)
    s->cv_done.wait(lk, [&] { return !s->done.empty() || (s->queue.empty() && s->active == 0) || s->live == 0; });
  int n = 0;
  while (n < max_results && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = n;
  return FFTM_OK;
}

int fftm_server_pending(fftm_server* s, int* queued, int* active, size_t* bytes_in_use) {
  if (!s) return FFTM_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->queue.size();
  if (active) *active = s->active;
  if (bytes_in_use) *bytes_in_use = s->in_use;
  return FFTM_OK;
}

int fftm_server_destroy(fftm_server* s) {
  if (!s) return FFTM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return FFTM_OK;
}

int fftm_server_inject_start_failures(int count) {
  if (count < 0) return FFTM_E_INVALID;
  g_fail_starts.store(count);
  return FFTM_OK;
}

}  // extern "C"

extern "C" int fftm_server_set_option(fftm_server* s, int option, int value) {
  if (!s) return FFTM_E_INVALID;
  if (option != FFTM_OPT_RESIDUAL_PASSES && option != FFTM_OPT_RESIDUAL_TILE && option != FFTM_OPT_DEVICE_LOOP &&
      option != FFTM_OPT_CUDA_GRAPH)
    return FFTM_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& o : s->options)
    if (o.first == option) {
      o.second = value;
      return FFTM_OK;
    }
  s->options.emplace_back(option, value);
  return FFTM_OK;
}
