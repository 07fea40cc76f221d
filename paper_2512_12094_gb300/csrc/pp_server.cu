// Serving: jobs (observable, one layer of gates applied n_layers times,
// product state) submitted from any host thread run concurrently on the GPU.
//
// Continuous batching: the server keeps `slots` worker threads, each with its
// own CUDA stream.  A free worker takes the queued job with the shortest
// predicted run time (learned from the jobs finished so far, less a credit
// for the time waited) whose memory reservation fits in what the running jobs
// leave of the budget, so a job that arrives while others run starts as soon
// as a slot and memory are free, and the kernels of different jobs overlap on
// the device.  A job runs in its own
// context (tables resident on the device for its whole life) whose memory
// budget is its reservation; each of its layers runs as one persistent launch
// on the share of the GPU's co-resident blocks it holds for that layer
// (an equal share among the running jobs, at least 1/slots).
//
// Reservations follow the jobs' live-term counts.  A job's first reservation
// is the memory of a table for its observable (unless the job names one).
// Between layers the worker compares the context's device memory, scaled by
// the growth of the live-term count over the last layer, with the
// reservation and asks the server for more before the next layer; a layer
// that still runs out of room (PP_ERR_CAPACITY, the context restored to its
// state before the layer) gets twice the reservation and is applied again.
// The job never starts over.  A running job waiting for more memory has
// priority over queued jobs; a queued job that younger jobs have passed
// kMaxBypass times is passed no more.  If every running job waits for memory
// the one that notices gives its memory back and is queued again at the head
// with the reservation it asked for (the only case where work is repeated).
// Every job's result depends only on the job: contexts share nothing, and
// per-job work is the same as a single pp_create / pp_apply_layer / pp_expect
// sequence.
#include <algorithm>
#include <chrono>
#include <cmath>
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

#include <nvtx3/nvToolsExt.h>

#include "../../include/pp.h"
#include "pp_admission.h"
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
  int grows = 0;     // reservation increases
  int restarts = 0;  // times the job gave its memory back and started over
  int bypassed = 0;  // younger jobs admitted while this one waited at the queue's head
  size_t want_next = 0;  // reservation asked for when the job gave its memory back
  double feat[ppadm::kFeat] = {};  // features of the cost model (job_features)
  bool started = false;
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
  int64_t growing = 0;  // running jobs waiting for a larger reservation
  int slots = 1;
  int device = 0;
  bool stopping = false;
  uint64_t next_id = 1;
  std::deque<std::unique_ptr<Job>> queue;
  std::map<uint64_t, Done> results;
  int64_t running = 0, completed = 0;
  int units_free = 0;  // share units of the GPU's co-resident blocks not held by a layer
  ppadm::CostModel cost;  // predicted run times of queued jobs (admission order)
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a job or memory became available
  std::condition_variable cv_done;  // waiters: a job finished
  std::vector<std::thread> workers;
};

namespace {

constexpr size_t kMiB = (size_t)1 << 20;
size_t round_mib(double b) { return ((size_t)std::ceil(b / (double)kMiB) + 1) * kMiB; }

// Device memory of a context holding `terms` strings: two tables with room
// for four times the terms (entries, coefficients and a hash index of at
// least 1.5x the capacity), the dense copy kept while a layer runs, and a
// megabyte of fixed buffers.
size_t estimate_job_bytes(const pp_config& cfg, int64_t terms) {
  const double W = (double)((cfg.n_qubits + 63) / 64);
  const bool batched = cfg.batch > 1 || cfg.coef_type == PP_COEF_F32;
  const double row = batched ? (double)cfg.batch * (cfg.coef_type == PP_COEF_F32 ? 4.0 : 8.0) + 1.0
                             : 8.0;
  const double cap = std::max<double>(4.0 * (double)terms, 1024.0);
  const double table = cap * (16.0 * W + row) + 2.0 * cap * 8.0;
  return round_mib(2.0 * table + (double)terms * (16.0 * W + row) + (double)kMiB);
}

// Admission order (ppadm::admission_key): the lowest predicted cost first,
// less one (natural-log) unit for every kAgeSeconds a job has waited, so that
// cheap jobs do not queue behind expensive ones and an expensive job still
// comes to the front.  A job that gave its memory back keeps its place (it
// has waited longest).
//
// The queued job first in admission order whose reservation fits; nullptr if
// none.  Jobs waiting to grow come first, and a job passed kMaxBypass times by
// jobs after it in that order blocks them (ppadm::pick_admission).
std::unique_ptr<Job> take_fitting(pp_server* s) {
  if (s->growing > 0) return nullptr;
  const Clock::time_point now = Clock::now();
  const size_t q = s->queue.size();
  std::vector<double> key(q);
  std::vector<char> fits(q);
  std::vector<int> bypassed(q);
  for (size_t k = 0; k < q; ++k) {
    const Job& j = *s->queue[k];
    const double waited = std::chrono::duration<double>(now - j.t_submit).count();
    key[k] = ppadm::admission_key(s->cost.predict(j.feat), waited, j.restarts > 0);
    fits[k] = s->reserved + j.reserve <= s->budget;
    bypassed[k] = j.bypassed;
  }
  const long pick = ppadm::pick_admission(key, fits, bypassed);
  for (size_t k = 0; k < q; ++k) s->queue[k]->bypassed = bypassed[k];
  if (pick < 0) return nullptr;
  auto it = s->queue.begin() + (std::ptrdiff_t)pick;
  std::unique_ptr<Job> out = std::move(*it);
  s->queue.erase(it);
  return out;
}

// Share units for one layer of a job whose launch would use the fraction
// `wanted` of the GPU.  Every layer gets 1/slots of the GPU, as a fixed split
// would give it (a table may grow far beyond its size at the layer's start
// and relaunch on more blocks after a stall).  A job that can use more gets
// up to an equal share among the running jobs.  A queued job that fits in
// memory is admitted as soon as a slot is free, so fewer running jobs than
// slots means the others wait for memory: then a few large jobs, or one at
// the end of a stream, get the GPU instead of leaving it idle.  Waits until
// 1/slots is free; units come back at the end of every layer, so the wait
// ends.
int acquire_units(pp_server* s, double wanted) {
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    const int take = ppadm::share_units(s->slots, s->running, wanted, s->units_free);
    if (take > 0) {
      s->units_free -= take;
      return take;
    }
    s->cv_work.wait(lock);
  }
}

void release_units(pp_server* s, int units) {
  std::lock_guard<std::mutex> lock(s->mu);
  s->units_free += units;
  s->cv_work.notify_all();
}

enum class Grow { kGranted, kNever, kGiveBack };

// Raise a running job's reservation to `want` (capped at the budget),
// waiting for running jobs to free memory.  kNever: the job is at the budget
// already; kGiveBack: every running job waits for memory, so this one must
// release its own.
Grow grow_reservation(pp_server* s, Job& j, size_t want) {
  std::unique_lock<std::mutex> lock(s->mu);
  want = std::min(want, s->budget);
  if (want <= j.reserve) return Grow::kNever;
  s->growing++;
  for (;;) {
    if (s->reserved - j.reserve + want <= s->budget) {
      s->reserved += want - j.reserve;
      j.reserve = want;
      j.grows++;
      s->growing--;
      return Grow::kGranted;
    }
    if (s->growing >= s->running) {  // nobody can finish and free memory
      s->growing--;
      j.want_next = want;  // ask for this much when admitted again
      return Grow::kGiveBack;
    }
    s->cv_work.wait(lock);
  }
}

// Run one job on `stream`: returns its status; fills r.  *give_back is set
// when the job released its memory to let others finish (it is queued
// again).
pp_status run_job(pp_server* s, Job& j, cudaStream_t stream, pp_job_result& r, bool* give_back) {
  // one named range per job on the host timeline for profilers (NVTX)
  char range_name[48];
  snprintf(range_name, sizeof(range_name), "job %llu", (unsigned long long)j.id);
  nvtxRangePushA(range_name);
  struct PopRange {
    ~PopRange() { nvtxRangePop(); }
  } pop_range_;
  *give_back = false;
  pp_config cfg = j.cfg;
  cfg.cuda_stream = stream;
  cfg.mem_budget_bytes = j.reserve;
  pp_ctx* ctx = nullptr;
  // a reactive increase: twice the reservation; false when the job must stop
  auto grow_or_stop = [&](pp_status& st) {
    const Grow g = grow_reservation(s, j, 2 * j.reserve);
    if (g == Grow::kGranted) {
      if (ctx) pp_set_budget(ctx, j.reserve);
      return true;
    }
    if (g == Grow::kGiveBack) *give_back = true;
    (void)st;
    return false;
  };
  pp_status st;
  for (;;) {
    cfg.mem_budget_bytes = j.reserve;
    st = pp_create(&cfg, (int64_t)j.coef.size() / cfg.batch, j.x.data(), j.z.data(),
                   j.coef.data(), &ctx);
    if (st != PP_ERR_CAPACITY || !grow_or_stop(st)) break;
  }
  int64_t live_prev = -1;
  for (int l = 0; st == PP_OK && l < j.n_layers; ++l) {
    // proactive: the memory the context holds, scaled by the live-term
    // growth of the last layer, should fit the reservation
    pp_stats_t stats;
    if (pp_stats(ctx, &stats) == PP_OK) {
      const double growth =
          live_prev > 0 ? std::max(1.0, (double)stats.live_terms / (double)live_prev) : 1.0;
      const size_t predicted = round_mib((double)stats.device_bytes * std::min(growth, 16.0));
      live_prev = stats.live_terms;
      if (predicted > j.reserve) {
        const Grow g = grow_reservation(s, j, predicted);
        if (g == Grow::kGranted) pp_set_budget(ctx, j.reserve);
        if (g == Grow::kGiveBack) {
          *give_back = true;
          st = PP_ERR_CAPACITY;
          break;
        }
      }
    }
    for (;;) {
      // A layer runs in one persistent launch on the share units it holds
      // (a job running alone gets the whole GPU); the units go back before
      // any wait for memory, so no job waits for memory while holding units
      // another job needs in order to finish.
      const double wanted = ppk::layer_fraction_wanted(ctx);
      const int units = wanted > 0.0 ? acquire_units(s, wanted) : 0;
      if (units > 0) ppk::set_grid_fraction(ctx, (double)units / ppadm::kShareUnits);
      st = pp_apply_layer(ctx, (int)j.gates.size(), j.gates.data(), j.theta.data(), j.boundary);
      if (units > 0) release_units(s, units);
      if (st != PP_ERR_CAPACITY || !grow_or_stop(st)) break;
    }
  }
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
    if (!j->started) {
      j->t_start = Clock::now();
      j->started = true;
    }
    pp_job_result r;
    memset(&r, 0, sizeof(r));
    pp_status st = PP_ERR_CUDA;
    bool give_back = false;
    if (have_stream) {
      st = run_job(s, *j, stream, r, &give_back);
    } else {
      snprintf(r.message, sizeof(r.message), "%s", "the worker could not create its CUDA stream");
    }
    const auto t_end = Clock::now();
    std::unique_lock<std::mutex> lock(s->mu);
    s->reserved -= j->reserve;  // every granted increase was added to `reserved`
    s->running--;
    if (give_back) {
      j->reserve = j->want_next;
      j->restarts++;
      j->bypassed = 0;
      s->queue.push_front(std::move(j));
    } else {
      r.done = 1;
      r.status = st;
      r.queue_ms = ms_between(j->t_submit, j->t_start);
      r.run_ms = ms_between(j->t_start, t_end);
      r.latency_ms = ms_between(j->t_submit, t_end);
      r.reserved_bytes = j->reserve;
      r.grows = j->grows;
      r.restarts = j->restarts;
      if (st == PP_OK && r.run_ms > 0.0) s->cost.add(j->feat, std::log(r.run_ms));
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
  s->slots = slots;
  s->default_reserve = default_job_bytes;  // 0: each job's reservation is estimated
  s->units_free = ppadm::kShareUnits;
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
  ppadm::job_features(cfg, job->n_layers, job->n_layer_gates, j->feat);
  j->reserve = job->mem_bytes ? job->mem_bytes
                              : (s->default_reserve ? s->default_reserve
                                                    : estimate_job_bytes(cfg, job->n_terms));
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
