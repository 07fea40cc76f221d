// Serving: jobs (observable, one layer of gates applied n_layers times,
// product state) submitted from any host thread run concurrently on the GPU.
//
// Continuous batching: the server keeps `slots` worker threads, each with its
// own CUDA stream.  A free worker takes the oldest queued job whose memory
// reservation fits in what the running jobs leave of the budget, so a job that
// arrives while others run starts as soon as a slot and memory are free, and
// the kernels of different jobs overlap on the device.  A job runs in its own
// context (tables resident on the device for its whole life) whose memory
// budget is its reservation; if the job outgrows it (PP_ERR_CAPACITY) it is put
// back at the head of the queue with four times the reservation, up to the
// server budget.  Every job's result depends only on the job: contexts share
// nothing, and per-job work is the same as a single pp_create /
// pp_apply_layer / pp_expect sequence.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pp.h"
#include "pp_internal.h"

namespace {

struct Job {
  uint64_t id = 0;
  pp_config cfg{};
  std::vector<uint64_t> x, z;
  std::vector<double> coef;
  std::vector<pp_pauli> gates;
  std::vector<double> theta;
  std::vector<double> bloch;
  int n_layers = 0;
  int boundary = 1;
  size_t reserve = 0;
  std::chrono::steady_clock::time_point t_submit, t_start;
};

struct Done {
  pp_job_result r{};
};

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct pp_server {
  size_t budget = 0;
  size_t default_reserve = 0;
  size_t reserved = 0;  // sum of the reservations of running jobs
  int device = 0;
  bool stopping = false;
  uint64_t next_id = 1;
  std::deque<std::unique_ptr<Job>> queue;
  std::map<uint64_t, Done> results;
  int64_t running = 0, completed = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a job or memory became available
  std::condition_variable cv_done;  // waiters: a job finished
  std::vector<std::thread> workers;
};

namespace {

// Oldest queued job whose reservation fits; nullptr if none.
std::unique_ptr<Job> take_fitting(pp_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (s->reserved + (*it)->reserve <= s->budget) {
      std::unique_ptr<Job> j = std::move(*it);
      s->queue.erase(it);
      return j;
    }
  }
  return nullptr;
}

// Run one job on `stream`: returns its status; fills r.
pp_status run_job(const Job& j, cudaStream_t stream, pp_job_result& r) {
  pp_config cfg = j.cfg;
  cfg.cuda_stream = stream;
  cfg.mem_budget_bytes = j.reserve;
  cfg.layer_kernel = 0;  // one kernel per gate: jobs on other streams can interleave
  pp_ctx* ctx = nullptr;
  pp_status st = pp_create(&cfg, (int64_t)j.coef.size() / cfg.batch, j.x.data(), j.z.data(),
                           j.coef.data(), &ctx);
  for (int l = 0; st == PP_OK && l < j.n_layers; ++l)
    st = pp_apply_layer(ctx, (int)j.gates.size(), j.gates.data(), j.theta.data(), j.boundary);
  if (st == PP_OK) st = pp_expect(ctx, j.bloch.data(), &r.value);
  if (st != PP_OK) snprintf(r.message, sizeof(r.message), "%s", pp_last_error());
  if (ctx) {
    pp_stats_t stats;
    if (pp_stats(ctx, &stats) == PP_OK) {
      r.live_terms = stats.live_terms;
      r.gate_updates = stats.gate_updates;
      r.device_bytes = stats.device_bytes;
    }
    pp_destroy(ctx);
  }
  return st;
}

void worker_main(pp_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t stream = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    std::unique_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stopping || (j = take_fitting(s)) != nullptr; });
      if (!j) break;  // stopping and nothing left that fits
      s->reserved += j->reserve;
      s->running++;
    }
    j->t_start = Clock::now();
    pp_job_result r;
    memset(&r, 0, sizeof(r));
    pp_status st = PP_ERR_CUDA;
    if (have_stream) {
      st = run_job(*j, stream, r);
    } else {
      snprintf(r.message, sizeof(r.message), "%s", "the worker could not create its CUDA stream");
    }
    const auto t_end = Clock::now();
    std::unique_lock<std::mutex> lock(s->mu);
    s->reserved -= j->reserve;
    s->running--;
    if (st == PP_ERR_CAPACITY && j->reserve < s->budget) {
      // grow the reservation and retry first
      j->reserve = std::min(s->budget, j->reserve * 4);
      s->queue.push_front(std::move(j));
    } else {
      r.done = 1;
      r.status = st;
      r.queue_ms = ms_between(j->t_submit, j->t_start);
      r.run_ms = ms_between(j->t_start, t_end);
      r.latency_ms = ms_between(j->t_submit, t_end);
      r.reserved_bytes = j->reserve;
      s->results[j->id].r = r;
      s->completed++;
      s->cv_done.notify_all();
    }
    s->cv_work.notify_all();
  }
  if (have_stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

pp_status pp_server_create(int slots, size_t mem_budget_bytes, size_t default_job_bytes,
                           pp_server** out) {
  if (!out || slots < 1 || slots > 256 || mem_budget_bytes == 0) {
    ppk::set_last_error("pp_server_create: need 1..256 slots and a nonzero memory budget");
    return PP_ERR_ARG;
  }
  pp_server* s = new pp_server();
  s->budget = mem_budget_bytes;
  s->default_reserve = default_job_bytes ? default_job_bytes : ((size_t)64 << 20);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    ppk::set_last_error("pp_server_create: no CUDA device");
    return PP_ERR_CUDA;
  }
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return PP_OK;
}

pp_status pp_submit(pp_server* s, const pp_job* job, uint64_t* job_id) {
  if (!s || !job || !job_id) {
    ppk::set_last_error("pp_submit: null argument");
    return PP_ERR_ARG;
  }
  const pp_config& cfg = job->cfg;
  const int W = (cfg.n_qubits + 63) / 64;
  if (cfg.n_qubits < 1 || cfg.n_qubits > 256 || cfg.batch < 1 || job->n_terms < 0 ||
      job->n_layer_gates < 0 || job->n_layers < 0 || !job->bloch ||
      (job->n_terms > 0 && (!job->x || !job->z || !job->coef)) ||
      (job->n_layer_gates > 0 && (!job->gates || !job->theta))) {
    ppk::set_last_error("pp_submit: bad job description");
    return PP_ERR_ARG;
  }
  auto j = std::make_unique<Job>();
  j->cfg = cfg;
  j->x.assign(job->x, job->x + job->n_terms * W);
  j->z.assign(job->z, job->z + job->n_terms * W);
  j->coef.assign(job->coef, job->coef + job->n_terms * cfg.batch);
  j->gates.assign(job->gates, job->gates + job->n_layer_gates);
  j->theta.assign(job->theta, job->theta + (size_t)job->n_layer_gates * cfg.batch);
  j->bloch.assign(job->bloch, job->bloch + 3 * cfg.n_qubits);
  j->n_layers = job->n_layers;
  j->boundary = job->symmetric_boundary;
  j->reserve = job->mem_bytes ? job->mem_bytes : s->default_reserve;
  std::lock_guard<std::mutex> lock(s->mu);
  if (j->reserve > s->budget) {
    ppk::set_last_error("pp_submit: job reservation exceeds the server memory budget");
    return PP_ERR_REJECTED;
  }
  if (s->stopping) {
    ppk::set_last_error("pp_submit: server is shutting down");
    return PP_ERR_STATE;
  }
  j->id = s->next_id++;
  j->t_submit = Clock::now();
  *job_id = j->id;
  s->results[j->id] = Done();
  s->queue.push_back(std::move(j));
  s->cv_work.notify_one();
  return PP_OK;
}

pp_status pp_server_poll(pp_server* s, uint64_t job_id, pp_job_result* out) {
  if (!s || !out) return PP_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->results.find(job_id);
  if (it == s->results.end()) {
    ppk::set_last_error("pp_server_poll: unknown job id");
    return PP_ERR_ARG;
  }
  *out = it->second.r;
  return PP_OK;
}

pp_status pp_server_wait(pp_server* s, uint64_t job_id, pp_job_result* out) {
  if (!s || !out) return PP_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->results.find(job_id);
  if (it == s->results.end()) {
    ppk::set_last_error("pp_server_wait: unknown job id");
    return PP_ERR_ARG;
  }
  s->cv_done.wait(lock, [&] { return s->results[job_id].r.done != 0; });
  *out = s->results[job_id].r;
  return PP_OK;
}

pp_status pp_server_stats(pp_server* s, int64_t* queued, int64_t* running, int64_t* completed,
                          size_t* reserved_bytes) {
  if (!s) return PP_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (queued) *queued = (int64_t)s->queue.size();
  if (running) *running = s->running;
  if (completed) *completed = s->completed;
  if (reserved_bytes) *reserved_bytes = s->reserved;
  return PP_OK;
}

pp_status pp_server_destroy(pp_server* s) {
  if (!s) return PP_OK;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    // let queued jobs finish first
    s->cv_done.wait(lock, [&] { return s->queue.empty() && s->running == 0; });
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return PP_OK;
}

}  // extern "C"
