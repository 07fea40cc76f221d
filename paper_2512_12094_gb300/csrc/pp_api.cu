// Host side of the C ABI declared in include/pp.h.
//
// A context owns two term tables of equal capacity (the live one and a
// spare used as the destination of merges and compactions), a device
// control block, and small constant tables.  By default all gates of a layer
// run in one cooperative launch with a grid barrier between gates; otherwise
// (and for batched rows) each gate is one kernel and repeated layers are
// replayed from captured CUDA graphs.  The host reads the control block once
// per layer: a gate that finds less than twice its input size free does
// nothing and raises `stall`; the host then grows the tables and relaunches
// the layer from that gate (earlier gates skip themselves).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pp.h"
#include "pp_internal.h"
#include "pp_symmetry_host.h"

using namespace ppk;

namespace {

// A named range on the host timeline for profilers (NVTX); costs nothing
// when no tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

thread_local std::string g_last_error;

pp_status fail(pp_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

}  // namespace

void ppk::set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

pp_status cuda_fail(cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(PP_ERR_OOM, msg);
  return fail(PP_ERR_CUDA, msg);
}

#define PP_CUDA(call)                                    \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);  \
  } while (0)

#define PP_TRY(call)                   \
  do {                                 \
    pp_status _s = (call);             \
    if (_s != PP_OK) return _s;        \
  } while (0)

uint64_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

int popcount64(uint64_t v) { return __builtin_popcountll(v); }

struct Buf {
  uint64_t* keys = nullptr;
  double* coef = nullptr;           // single FP64 column
  void* rows = nullptr;             // batched rows [cap][B]
  unsigned char* alive = nullptr;   // batched liveness
  uint64_t* index = nullptr;
  uint64_t cap = 0;
  uint64_t icap = 0;
};

struct ArgsEntry {
  std::vector<unsigned char> sig;  // the cached bytes (gate arguments or cos/sin columns)
  GateArgs* d_args = nullptr;      // device copy
  size_t n = 0;                    // its size in bytes
  uint64_t last_use = 0;
};

struct GraphEntry {
  std::vector<unsigned char> sig;  // bytes of the gate arguments
  int grid = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

// row_bytes: coefficient bytes per string (8, or B x element size + 1 for the
// liveness byte of batched rows)
size_t table_bytes(uint64_t cap, uint64_t icap, int W, size_t row_bytes) {
  return (size_t)cap * (16 * W + row_bytes) + (size_t)icap * 8;
}

}  // namespace

struct pp_ctx {
  pp_config cfg{};
  int n = 0, W = 1;
  int B = 1;             // angle sets (columns)
  bool batched = false;  // rows + liveness bytes instead of one FP64 column
  int f32 = 0;           // batched rows hold float
  size_t esize = 8;      // bytes per row element
  size_t row_bytes() const { return batched ? (size_t)B * esize + 1 : 8; }
  std::vector<ArgsEntry> cs_cache;  // per-gate cos/sin columns (batched)
  std::vector<std::vector<unsigned char>> sym_ok;  // layers (gates + angles) already validated
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 1;
  int gate_bps = 4;   // resident gate-kernel blocks per SM
  int layer_bps = 0;  // co-resident layer-kernel blocks per SM (0: no cooperative path)
  int layer_threads = kBlock;   // block size of the persistent layer kernel
  int bps_by_threads[2] = {0, 0};  // co-resident blocks per SM with 256 / 1024 threads
  std::vector<ArgsEntry> arg_cache;
  cudaEvent_t ev_layer[2] = {nullptr, nullptr};
  Buf buf[2];
  int active = 0;
  DevTable* d_desc = nullptr;  // [3]: table 0, table 1, active copy
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;     // pinned mirror
  double* d_damp = nullptr;    // (1-p)^k
  double* d_ldamp = nullptr;   // exp(-gamma k)
  double* d_partials = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;     // pinned
  double* d_bloch = nullptr;
  double* d_sn = nullptr;      // S_n overlap table
  double* d_sn_work = nullptr;
  std::vector<double> sn_bloch;  // bloch vectors the S_n table was built for
  uint64_t n_terms = 0;          // host mirror of DevCtl::n_terms
  int64_t n_live = 0;
  bool live_known = true;  // n_live equals the device's count (false after a kernel changed it unread)
  bool merged = true;
  bool obs_invariant = false;
  size_t bytes = 0;
  int64_t merges = 0, compactions = 0, regrows = 0, stalls = 0;
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  int overlap_grid = 0;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_start, ev_end;  // per gate position (profile_kernels)
  double last_growth = 2.0;  // stored entries after / before the gates of the last layer
  double grid_scale = 1.0;   // blocks per launch relative to the default sizing (pp_tune)
  double index_factor = 1.5; // hash index slots per table entry of capacity (pp_tune)
  double grid_frac = 1.0;    // a persistent layer launch takes at most this fraction of the GPU
  double gate_ms = 0.0;
  int64_t gates_timed = 0;
  void* sort_scratch = nullptr;  // scratch of the sort-based merge (merge_method 1)
  size_t sort_scratch_bytes = 0;
};

namespace {

// The library's stream-ordered memory pool on the current device, created
// once.  It keeps freed memory mapped (no release threshold), so tables
// that are freed and allocated again -- a table moved when it grows, the
// next context of a server -- reuse memory instead of mapping it anew at
// every synchronise, as the default pool would.  The memory stays with the
// process until it exits.
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

// Pinned host blocks of the per-context mirrors, kept for reuse: freeing
// pinned memory waits for the whole device.
std::mutex g_pinned_mu;
std::vector<std::pair<size_t, void*>> g_pinned_free;

cudaError_t pinned_get(void** p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    for (size_t k = 0; k < g_pinned_free.size(); ++k) {
      if (g_pinned_free[k].first == bytes) {
        *p = g_pinned_free[k].second;
        g_pinned_free.erase(g_pinned_free.begin() + (long)k);
        return cudaSuccess;
      }
    }
  }
  return cudaMallocHost(p, bytes);
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  if (g_pinned_free.size() < 256) {
    g_pinned_free.emplace_back(bytes, p);
    return;
  }
  cudaFreeHost(p);
}

// Host-side fault injection (pp_debug_fail_alloc_after): allocations left
// before one fails as if the device were out of memory; negative = off.
std::atomic<long long> g_fail_alloc_after{-1};

pp_status dmalloc(pp_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  for (long long left = g_fail_alloc_after.load(); left >= 0;) {
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {
        *p = nullptr;
        return fail(PP_ERR_OOM, "device allocation failed (injected by pp_debug_fail_alloc_after)");
      }
      break;
    }
  }
  cudaMemPool_t pool = lib_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, c->stream)
                       : cudaMallocAsync(p, bytes, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  c->bytes += bytes;
  return PP_OK;
}

void dfree(pp_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  cudaFreeAsync(p, c->stream);
  c->bytes -= (bytes == 0 ? 16 : bytes);
}

// Index slots per dense entry of capacity: the index is a power of two of at
// least index_factor (1.5 unless pp_tune chose another) times the capacity, so
// its load stays below 2/3 even when the table is full (a gate stalls before
// that can happen) and is about 1/4 at a layer start.  (An index sized for
// the stored entries instead, at up to half load, was measured slower: the
// longer probe chains of births' slot claims, one atomic round trip each,
// cost more than the smaller footprint saved in lookups.)
uint64_t index_cap_for(const pp_ctx* c, uint64_t cap) {
  return next_pow2((uint64_t)std::ceil(c->index_factor * (double)cap));
}

void free_buf(pp_ctx* c, Buf& b) {
  dfree(c, b.keys, (size_t)b.cap * 16 * c->W);
  dfree(c, b.coef, (size_t)b.cap * 8);
  dfree(c, b.rows, (size_t)b.cap * c->B * c->esize);
  dfree(c, b.alive, (size_t)b.cap);
  dfree(c, b.index, (size_t)b.icap * 8);
  b = Buf();
}

// All arrays of a table of `cap` entries, or none: a failed allocation
// releases what was taken and leaves b empty.
pp_status alloc_buf(pp_ctx* c, Buf& b, uint64_t cap) {
  b = Buf();
  b.cap = cap;
  b.icap = index_cap_for(c, cap);
  pp_status st = dmalloc(c, (void**)&b.keys, (size_t)cap * 16 * c->W);
  if (st == PP_OK && c->batched) {
    st = dmalloc(c, (void**)&b.rows, (size_t)cap * c->B * c->esize);
    if (st == PP_OK) st = dmalloc(c, (void**)&b.alive, (size_t)cap);
  } else if (st == PP_OK) {
    st = dmalloc(c, (void**)&b.coef, (size_t)cap * 8);
  }
  if (st == PP_OK) st = dmalloc(c, (void**)&b.index, (size_t)b.icap * 8);
  if (st == PP_OK) {
    const cudaError_t e = cudaMemsetAsync(b.index, 0, (size_t)b.icap * 8, c->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
  }
  if (st != PP_OK) free_buf(c, b);
  return st;
}

DevTable desc_of(const pp_ctx* c, const Buf& b) {
  DevTable t = {};
  t.keys = b.keys;
  t.coef = b.coef;
  t.index = b.index;
  t.cap = b.cap;
  t.imask = b.icap ? b.icap - 1 : 0;
  t.rows = b.rows;
  t.alive = b.alive;
  t.B = c->B;
  t.f32 = c->f32;
  return t;
}

// Host to device copy ordered on the context's stream, complete on return.
// A plain cudaMemcpy from pageable memory goes through the legacy default
// stream and may return before its DMA lands; kernels on a non-blocking
// stream do not wait for it and could read what was there before (in a
// server, memory another job just freed).
cudaError_t upload(pp_ctx* c, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

// Write the descriptors of both tables and the active copy (only called when
// a table is (re)allocated).
pp_status publish_desc(pp_ctx* c) {
  DevTable h[3] = {desc_of(c, c->buf[0]), desc_of(c, c->buf[1]), desc_of(c, c->buf[c->active])};
  PP_CUDA(upload(c, c->d_desc, h, sizeof(h)));
  return PP_OK;
}

// Make the active copy point at c->active (stream ordered, device to device).
pp_status activate(pp_ctx* c, int which) {
  c->active = which;
  PP_CUDA(cudaMemcpyAsync(c->d_desc + 2, c->d_desc + which, sizeof(DevTable),
                          cudaMemcpyDeviceToDevice, c->stream));
  return PP_OK;
}

pp_status read_ctl(pp_ctx* c) {
  PP_CUDA(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
  PP_CUDA(cudaStreamSynchronize(c->stream));
  return PP_OK;
}

pp_status check_device_error(pp_ctx* c) {
  unsigned e = c->h_ctl->error;
  if (!e) return PP_OK;
  if (e & kErrTimeout) {
    const DevCtl& h = *c->h_ctl;
    const char* what = h.to_kind == 1   ? "the grid barrier of the layer kernel"
                       : h.to_kind == 2 ? "the grid barrier of the batched layer kernel"
                       : h.to_kind == 3 ? "a claimed index slot"
                                        : "a device wait";
    return fail(PP_ERR_TIMEOUT,
                std::string("a bounded device wait ran out: ") + what + " (gate " +
                    std::to_string(h.to_gate) + ", counter " + std::to_string(h.to_seen) +
                    " of " + std::to_string(h.to_target) + ")");
  }
  const DevCtl& h = *c->h_ctl;
  if (e & kErrAppend) {
    std::string where;
    if (h.to_kind == 4)
      where = " (gate " + std::to_string(h.to_gate) + ", position " + std::to_string(h.to_seen) +
              " of capacity " + std::to_string(h.to_target) + ")";
    return fail(PP_ERR_INTERNAL, "append past table capacity" + where);
  }
  std::string where;
  if (h.to_kind == 5)
    where = " (gate " + std::to_string(h.to_gate) + ", T0 " + std::to_string(h.to_seen) +
            ", index mask " + std::to_string(h.to_target) + ")";
  return fail(PP_ERR_INTERNAL, "hash index probe bound exhausted" + where);
}

int grid_for(pp_ctx* c, uint64_t items, int per_thread) {
  uint64_t want = (items + (uint64_t)kBlock * per_thread - 1) / ((uint64_t)kBlock * per_thread);
  uint64_t maxg = (uint64_t)c->sms * 8;
  if (want < 1) want = 1;
  if (want > maxg) want = maxg;
  return (int)want;
}

// Set n_next (append cursor) and n_live before a merge or compaction into
// the spare table (a one-thread kernel on the stream: no host round trip).
// reset_occ: the table being filled becomes the active one, so its keys
// rebuild the occupancy masks.
pp_status ctl_prepare_insert(pp_ctx* c, unsigned long long first_free, bool reset_occ = true) {
  PP_CUDA(launch_ctl_insert(c->stream, c->d_ctl, first_free, 0, reset_occ ? 1 : 0));
  c->launches += 1;
  return PP_OK;
}

// n_terms <- n_next (device to device) and read the control block back.
pp_status ctl_commit(pp_ctx* c) {
  PP_CUDA(cudaMemcpyAsync(&c->d_ctl->n_terms, &c->d_ctl->n_next, 8, cudaMemcpyDeviceToDevice,
                          c->stream));
  PP_TRY(read_ctl(c));
  PP_TRY(check_device_error(c));
  c->n_terms = c->h_ctl->n_terms;
  c->n_live = c->h_ctl->n_live;
  c->live_known = true;
  return PP_OK;
}

// Copy the kept entries of the active table into `dst` (fresh index) and make
// it active.  extra_eps / extra_wmax implement pp_truncate.
pp_status compact_into(pp_ctx* c, int dst, double extra_eps, int extra_wmax) {
  Range range_("compact");
  Buf& d = c->buf[dst];
  PP_CUDA(cudaMemsetAsync(d.index, 0, (size_t)d.icap * 8, c->stream));
  PP_TRY(ctl_prepare_insert(c, 0));
  if (c->batched) {
    PP_CUDA(launch_compact_batched(c->W, grid_for(c, c->n_terms, 4), c->stream,
                                   desc_of(c, c->buf[c->active]), c->n_terms, desc_of(c, d), 1,
                                   extra_eps, extra_wmax, c->d_ctl));
  } else {
    PP_CUDA(launch_compact(c->W, grid_for(c, c->n_terms, 4), c->stream,
                           desc_of(c, c->buf[c->active]), c->n_terms, desc_of(c, d), 1,
                           c->cfg.coeff_eps, extra_eps, extra_wmax, c->d_ctl));
  }
  c->launches += 1;
  if (extra_eps == 0.0 && extra_wmax < 0 && c->live_known) {
    // A compaction without extra truncation keeps exactly the live entries,
    // whose count the host already holds, so the control block is updated on
    // the stream without a round trip (errors surface at the next read).
    PP_CUDA(cudaMemcpyAsync(&c->d_ctl->n_terms, &c->d_ctl->n_next, 8, cudaMemcpyDeviceToDevice,
                            c->stream));
    c->n_terms = (uint64_t)std::max<int64_t>(c->n_live, 0);
  } else {
    PP_TRY(ctl_commit(c));
  }
  PP_TRY(activate(c, dst));
  c->compactions++;
  return PP_OK;
}

pp_status ensure_capacity(pp_ctx* c, uint64_t need) {
  if (need <= c->buf[c->active].cap) return PP_OK;
  uint64_t cap = std::max<uint64_t>(need, 1024);
  cap = (cap + 1023) & ~1023ull;
  size_t add = 2 * table_bytes(cap, index_cap_for(c, cap), c->W, c->row_bytes());
  size_t keep = c->bytes - 2 * table_bytes(c->buf[0].cap, c->buf[0].icap, c->W, c->row_bytes());
  if (c->cfg.mem_budget_bytes && keep + add > c->cfg.mem_budget_bytes)
    return fail(PP_ERR_CAPACITY, "term table of capacity " + std::to_string(cap) +
                                     " exceeds the memory budget");
  // A failed allocation leaves the context as it was: the spare table is put
  // back at the capacity it had (the pool has just received those bytes), or
  // the active table keeps its entries at the larger capacity.
  const uint64_t old_cap = c->buf[c->active].cap;
  int spare = 1 - c->active;
  free_buf(c, c->buf[spare]);
  pp_status st = alloc_buf(c, c->buf[spare], cap);
  if (st != PP_OK) {
    const std::string msg = g_last_error;
    if (alloc_buf(c, c->buf[spare], old_cap) == PP_OK) PP_TRY(publish_desc(c));
    return fail(st, msg);
  }
  PP_TRY(publish_desc(c));
  PP_TRY(compact_into(c, spare, 0.0, -1));
  int old = 1 - c->active;
  free_buf(c, c->buf[old]);
  st = alloc_buf(c, c->buf[old], cap);
  if (st != PP_OK) {
    // the entries now live in the larger table; restore a spare of the old size
    // would break the equal-capacity rule, so move them back
    const std::string msg = g_last_error;
    if (alloc_buf(c, c->buf[old], old_cap) == PP_OK && publish_desc(c) == PP_OK &&
        compact_into(c, old, 0.0, -1) == PP_OK) {
      free_buf(c, c->buf[1 - c->active]);
      if (alloc_buf(c, c->buf[1 - c->active], old_cap) == PP_OK) PP_TRY(publish_desc(c));
    }
    return fail(st, msg);
  }
  PP_TRY(publish_desc(c));
  c->regrows++;
  return PP_OK;
}

// Make room before (or in the middle of) a layer: drop truncated entries when
// they are a quarter of the table or more, then make sure the capacity holds
// factor x the entries.  The caller derives factor from how much the previous
// layer grew the table, so that a layer rarely stalls (every stall costs a
// host round trip, a compaction and a relaunch); untouched capacity costs
// memory, not bandwidth.  Under a memory budget the growth falls back to the
// least that lets the next gate run.
pp_status make_room(pp_ctx* c, uint64_t factor = 2) {
  if (c->cfg.coeff_eps > 0.0 && c->n_terms > 0 && 4 * (c->n_terms - c->n_live) >= c->n_terms)
    PP_TRY(compact_into(c, 1 - c->active, 0.0, -1));
  const uint64_t cap = c->buf[c->active].cap;
  if (factor * c->n_terms <= cap) return PP_OK;
  const uint64_t least = c->n_terms * 4;
  const uint64_t generous = std::max<uint64_t>(least, factor * c->n_terms * 3 / 2);
  const pp_status st = ensure_capacity(c, generous);
  if (st != PP_ERR_CAPACITY || generous == least) return st;
  if (2 * c->n_terms <= cap) return PP_OK;  // the next gate fits; grow at a stall
  return ensure_capacity(c, least);
}

// Scratch for a sort-based merge of up to `count` entries, kept by the
// context between merges.  False (use the hash merge) when merges are to use
// the hash table, the strings are too wide for the sort, or the scratch would
// not fit in the memory budget.
bool sort_merge_ready(pp_ctx* c, uint64_t count) {
  if (c->cfg.merge_method != PP_MERGE_SORT || !sort_merge_supported(c->n)) return false;
  const size_t need = sort_merge_scratch_bytes(std::max<uint64_t>(count, 1), c->n);
  if (need <= c->sort_scratch_bytes) return true;
  const size_t grow = need - c->sort_scratch_bytes;
  if (c->cfg.mem_budget_bytes && c->bytes + grow > c->cfg.mem_budget_bytes) return false;
  dfree(c, c->sort_scratch, c->sort_scratch_bytes);
  c->sort_scratch = nullptr;
  c->sort_scratch_bytes = 0;
  if (dmalloc(c, &c->sort_scratch, need) != PP_OK) {
    c->sort_scratch = nullptr;
    return false;
  }
  c->sort_scratch_bytes = need;
  return true;
}

// Accumulate the active table (after optional canonicalisation) into the
// spare table and make it active: the merge of Algorithms 2 and 3.
pp_status merge_active(pp_ctx* c, int group) {
  Range range_("merge");
  int dst = 1 - c->active;
  Buf& d = c->buf[dst];
  Buf& s = c->buf[c->active];
  PP_CUDA(cudaMemsetAsync(d.index, 0, (size_t)d.icap * 8, c->stream));
  PP_TRY(ctl_prepare_insert(c, 0));
  if (sort_merge_ready(c, c->n_terms)) {
    // radix sort + segmented reduce; batched rows are finalized by the reduce
    PP_CUDA(launch_merge_sorted(group, c->n, -1, c->stream, s.keys, c->batched ? nullptr : s.coef,
                                s.rows, c->f32, s.alive, c->n_terms, nullptr,
                                c->cfg.coeff_eps > 0.0 ? 1 : 0, desc_of(c, d), 1,
                                c->cfg.coeff_eps, c->d_ctl, c->sort_scratch, 0));
    if (!c->batched)
      PP_CUDA(launch_finalize(grid_for(c, c->n_terms, 4), c->stream, desc_of(c, d), c->d_ctl,
                              c->cfg.coeff_eps));
    c->launches += 30;
  } else if (c->batched) {
    // FP64 accumulation rows, rounded to the storage type by the finalize pass
    double* acc = nullptr;
    const size_t acc_bytes = (size_t)std::max<uint64_t>(c->n_terms, 1) * c->B * sizeof(double);
    PP_TRY(dmalloc(c, (void**)&acc, acc_bytes));
    PP_CUDA(cudaMemsetAsync(acc, 0, acc_bytes, c->stream));
    PP_CUDA(launch_merge_batched(c->W, group, c->n, -1, c->f32, grid_for(c, c->n_terms, 32),
                                 c->stream, s.keys, s.rows, s.alive, c->n_terms, desc_of(c, d), acc,
                                 c->d_ctl));
    PP_CUDA(launch_finalize_batched(grid_for(c, c->n_terms, 32), c->stream, desc_of(c, d), acc,
                                    c->d_ctl, c->cfg.coeff_eps));
    dfree(c, acc, acc_bytes);
  } else {
    PP_CUDA(launch_merge_insert(c->W, group, c->n, -1, grid_for(c, c->n_terms, 4), c->stream,
                                s.keys, s.coef, c->n_terms, nullptr,
                                c->cfg.coeff_eps > 0.0 ? 1 : 0, desc_of(c, d), c->d_ctl));
    PP_CUDA(launch_finalize(grid_for(c, c->n_terms, 4), c->stream, desc_of(c, d), c->d_ctl,
                            c->cfg.coeff_eps));
  }
  c->launches += 2;
  PP_TRY(ctl_commit(c));
  PP_TRY(activate(c, dst));
  c->merged = true;
  c->merges++;
  return PP_OK;
}

// The symmetry merge of a layer queued right behind its gates, before the
// host knows whether they all ran: every step checks the layer's stall flag
// on the device and does nothing if a gate stopped for capacity.  The host
// reads the control block once afterwards (finish_queued_merge) instead of
// once after the gates and once after the merge.
pp_status queue_merge(pp_ctx* c, int group) {
  Range range_("queue merge");
  const int dst = 1 - c->active;
  Buf& d = c->buf[dst];
  Buf& s = c->buf[c->active];
  PP_CUDA(cudaMemsetAsync(d.index, 0, (size_t)d.icap * 8, c->stream));
  PP_CUDA(launch_ctl_insert(c->stream, c->d_ctl, 0, 1));
  const int grid = c->sms * 8;  // grid-stride; the count is on the device
  if (sort_merge_ready(c, s.cap)) {
    // the entry count is on the device; the table's capacity bounds it
    PP_CUDA(launch_merge_sorted(group, c->n, -1, c->stream, s.keys, s.coef, nullptr, 0, nullptr,
                                s.cap, &c->d_ctl->n_terms, c->cfg.coeff_eps > 0.0 ? 1 : 0,
                                desc_of(c, d), 1, c->cfg.coeff_eps, c->d_ctl, c->sort_scratch, 1));
    c->launches += 29;
  } else {
    PP_CUDA(launch_merge_insert(c->W, group, c->n, -1, grid, c->stream, s.keys, s.coef, 0,
                                &c->d_ctl->n_terms, c->cfg.coeff_eps > 0.0 ? 1 : 0,
                                desc_of(c, d), c->d_ctl, 1));
  }
  PP_CUDA(launch_finalize(grid, c->stream, desc_of(c, d), c->d_ctl, c->cfg.coeff_eps, 1));
  PP_CUDA(launch_ctl_commit(c->stream, c->d_ctl, 1));
  c->launches += 4;
  return PP_OK;
}

// After the control block was read and showed no stall: the queued merge ran.
pp_status finish_queued_merge(pp_ctx* c) {
  c->n_terms = c->h_ctl->n_terms;
  c->n_live = c->h_ctl->n_live;
  c->live_known = true;
  PP_TRY(activate(c, 1 - c->active));
  c->merged = true;
  c->merges++;
  return PP_OK;
}

bool key_has_bits_beyond(const uint64_t* x, const uint64_t* z, int n, int W) {
  for (int j = 0; j < W; ++j) {
    int lo = 64 * j;
    uint64_t valid = (n >= lo + 64) ? ~0ull : ((n > lo) ? ((1ull << (n - lo)) - 1ull) : 0ull);
    if ((x[j] | z[j]) & ~valid) return true;
  }
  return false;
}

// Symmetry groups on host-side strings (pp_symmetry_host.h).
using ppsym::bloch_invariant;
using ppsym::generators;
using ppsym::group_kind;
using ppsym::group_lx;
using ppsym::HKey;
using ppsym::multiset_invariant;
using ppsym::valid_group;

pp_status validate_config(const pp_config* cfg) {
  if (!cfg) return fail(PP_ERR_ARG, "config is null");
  if (cfg->n_qubits < 1 || cfg->n_qubits > 64 * kMaxW)
    return fail(PP_ERR_ARG, "n_qubits must be in 1..256");
  if (!valid_group(cfg->symmetry, cfg->n_qubits))
    return fail(PP_ERR_ARG, "unknown symmetry, or a torus width that does not divide n_qubits");
  if (cfg->batch < 1 || cfg->batch > 512) return fail(PP_ERR_ARG, "batch must be in 1..512");
  if (cfg->coef_type != PP_COEF_F64 && cfg->coef_type != PP_COEF_F32)
    return fail(PP_ERR_ARG, "unknown coef_type");
  if ((cfg->batch > 1 || cfg->coef_type == PP_COEF_F32) && cfg->noise_mode == PP_NOISE_PER_LAYER)
    return fail(PP_ERR_ARG, "per-layer noise needs batch 1 and FP64 storage");
  if (!(cfg->coeff_eps >= 0.0)) return fail(PP_ERR_ARG, "coeff_eps must be >= 0");
  if (cfg->noise_mode < PP_NOISE_NONE || cfg->noise_mode > PP_NOISE_PER_LAYER)
    return fail(PP_ERR_ARG, "unknown noise mode");
  if (cfg->noise_mode != PP_NOISE_NONE && !(cfg->noise_p >= 0.0))
    return fail(PP_ERR_ARG, "noise_p must be >= 0");
  if (cfg->merge_method != PP_MERGE_HASH && cfg->merge_method != PP_MERGE_SORT)
    return fail(PP_ERR_ARG, "unknown merge_method");
  if (cfg->wait_limit < 0) return fail(PP_ERR_ARG, "wait_limit must be >= 0");
  if (!(cfg->room_factor >= 0.0) || !std::isfinite(cfg->room_factor))
    return fail(PP_ERR_ARG, "room_factor must be finite and >= 0");
  if (cfg->block_threads != 0 && cfg->block_threads != 256 && cfg->block_threads != 1024)
    return fail(PP_ERR_ARG, "block_threads must be 0, 256 or 1024");
  return PP_OK;
}

// Replace the operator held by the active table with sum_i coef[i] s_i
// (arrays on the host or, with on_device, on the device): check the strings,
// record whether the observable is invariant under the group, and accumulate
// the strings (as representatives when a group is set) with truncation.
pp_status ingest_terms(pp_ctx* c, int64_t n_terms, const uint64_t* x, const uint64_t* z,
                       const double* coef, bool on_device, bool assume_invariant = false) {
  const int W = c->W;
  pp_status st;
  // Observable invariance (host copy needed for the check).
  std::vector<uint64_t> hx, hz;
  std::vector<double> hc;
  if (n_terms > 0) {
    hx.resize((size_t)n_terms * W);
    hz.resize((size_t)n_terms * W);
    hc.resize((size_t)n_terms * c->B);
    if (on_device) {
      if (cudaMemcpyAsync(hx.data(), x, hx.size() * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(hz.data(), z, hz.size() * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(hc.data(), coef, hc.size() * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fail(PP_ERR_CUDA, "reading device term arrays failed");
    } else {
      memcpy(hx.data(), x, hx.size() * 8);
      memcpy(hz.data(), z, hz.size() * 8);
      memcpy(hc.data(), coef, hc.size() * 8);
    }
    for (int64_t i = 0; i < n_terms; ++i)
      if (key_has_bits_beyond(&hx[i * W], &hz[i * W], c->n, W))
        return fail(PP_ERR_ARG, "a string has bits at or above n_qubits");
  }
  if (c->cfg.symmetry != PP_SYM_NONE && assume_invariant) {
    c->obs_invariant = true;  // terms in representative form stand for an invariant operator
  } else if (c->cfg.symmetry != PP_SYM_NONE) {
    // the observable is invariant when every column is
    c->obs_invariant = true;
    for (int b = 0; b < c->B && c->obs_invariant; ++b) {
      std::map<HKey, double> acc;
      for (int64_t i = 0; i < n_terms; ++i) {
        HKey k(2 * W);
        for (int j = 0; j < W; ++j) {
          k[j] = hx[i * W + j];
          k[W + j] = hz[i * W + j];
        }
        acc[k] += hc[(size_t)i * c->B + b];
      }
      std::vector<HKey> ks;
      std::vector<double> vs;
      for (auto& kv : acc) {
        ks.push_back(kv.first);
        vs.push_back(kv.second);
      }
      c->obs_invariant = multiset_invariant(c->cfg.symmetry, c->n, W, ks, vs, 1e-12);
    }
  }

  // Ingest: pack, then accumulate (with representatives when a group is set)
  // into the active table, which starts empty.
  PP_CUDA(cudaMemsetAsync(c->buf[c->active].index, 0, (size_t)c->buf[c->active].icap * 8,
                          c->stream));
  if (n_terms == 0) {
    PP_TRY(ctl_prepare_insert(c, 0));
    PP_TRY(ctl_commit(c));
  }
  if (n_terms > 0) {
    uint64_t* d_keys = nullptr;
    double* d_coef = nullptr;
    double* acc = nullptr;
    const size_t key_bytes = (size_t)n_terms * 16 * W, coef_bytes = hc.size() * 8;
    const size_t acc_bytes = c->batched ? (size_t)n_terms * c->B * sizeof(double) : 0;
    // the staging buffers go back to the pool on every exit
    auto release = [&](pp_status r) {
      dfree(c, d_keys, key_bytes);
      dfree(c, d_coef, coef_bytes);
      dfree(c, acc, acc_bytes);
      return r;
    };
    if ((st = dmalloc(c, (void**)&d_keys, key_bytes)) != PP_OK ||
        (st = dmalloc(c, (void**)&d_coef, coef_bytes)) != PP_OK ||
        (c->batched && (st = dmalloc(c, (void**)&acc, acc_bytes)) != PP_OK))
      return release(st);
    std::vector<uint64_t> packed((size_t)n_terms * 2 * W);
    for (int64_t i = 0; i < n_terms; ++i)
      for (int j = 0; j < W; ++j) {
        packed[i * 2 * W + j] = hx[i * W + j];
        packed[i * 2 * W + W + j] = hz[i * W + j];
      }
    if (cudaMemcpyAsync(d_keys, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_coef, hc.data(), coef_bytes, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
      return release(fail(PP_ERR_CUDA, "term upload failed"));
    if ((st = ctl_prepare_insert(c, 0)) != PP_OK) return release(st);
    cudaError_t e;
    if (c->batched) {
      e = cudaMemsetAsync(acc, 0, acc_bytes, c->stream);
      if (e == cudaSuccess)
        e = launch_merge_batched(W, c->cfg.symmetry, c->n, c->cfg.max_weight, 0,
                                 grid_for(c, n_terms, 32), c->stream, d_keys, d_coef, nullptr,
                                 (uint64_t)n_terms, desc_of(c, c->buf[c->active]), acc, c->d_ctl);
      if (e == cudaSuccess)
        e = launch_finalize_batched(grid_for(c, n_terms, 32), c->stream,
                                    desc_of(c, c->buf[c->active]), acc, c->d_ctl,
                                    c->cfg.coeff_eps);
      if (e != cudaSuccess) return release(cuda_fail(e, "batched ingest"));
    } else {
      e = launch_merge_insert(W, c->cfg.symmetry, c->n, c->cfg.max_weight, grid_for(c, n_terms, 4),
                              c->stream, d_keys, d_coef, (uint64_t)n_terms, nullptr, 0,
                              desc_of(c, c->buf[c->active]), c->d_ctl);
      if (e == cudaSuccess)
        e = launch_finalize(grid_for(c, n_terms, 4), c->stream, desc_of(c, c->buf[c->active]),
                            c->d_ctl, c->cfg.coeff_eps);
      if (e != cudaSuccess) return release(cuda_fail(e, "ingest merge"));
    }
    // the packed host copy is read by the upload above: keep it until the
    // stream has passed it (ctl_commit synchronises)
    if ((st = ctl_commit(c)) != PP_OK) return release(st);
    release(PP_OK);
  }
  c->merged = true;
  return PP_OK;
}

pp_status create_common(const pp_config* cfg, int64_t n_terms, const uint64_t* x,
                        const uint64_t* z, const double* coef, bool on_device, pp_ctx** out) {
  if (!out) return fail(PP_ERR_ARG, "out is null");
  *out = nullptr;
  PP_TRY(validate_config(cfg));
  if (n_terms < 0) return fail(PP_ERR_ARG, "n_terms < 0");
  if (n_terms > 0 && (!x || !z || !coef)) return fail(PP_ERR_ARG, "null term arrays");
  if ((uint64_t)n_terms >= (1ull << 31)) return fail(PP_ERR_ARG, "too many input terms");
  pp_ctx* c = new pp_ctx();
  c->cfg = *cfg;
  c->n = cfg->n_qubits;
  c->W = (c->n + 63) / 64;
  c->B = cfg->batch;
  c->batched = cfg->batch > 1 || cfg->coef_type == PP_COEF_F32;
  c->f32 = cfg->coef_type == PP_COEF_F32 ? 1 : 0;
  c->esize = c->f32 ? 4 : 8;
  c->sms = std::max(1, device_sm_count());
  c->gate_bps = gate_blocks_per_sm(c->W);

  auto cleanup = [&](pp_status st) {
    pp_destroy(c);
    return st;
  };
  {
    int dev = 0, coop = 0;
    const cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cleanup(cuda_fail(de, "no usable CUDA device (cudaGetDevice)"));
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && c->batched) {
      c->layer_bps = layer_batched_blocks_per_sm(c->W, c->f32);
    } else if (coop) {
      c->bps_by_threads[0] = layer_blocks_per_sm(c->W, kBlock);
      c->bps_by_threads[1] = c->W <= 2 ? layer_blocks_per_sm(c->W, 1024) : 0;
      // 256 threads by default: 1024-thread blocks (one per SM, a quarter of
      // the barrier arrivals and birth reservations) measured slower on the
      // ring job; pp_tune may still choose them
      const int want = cfg->block_threads ? cfg->block_threads : kBlock;
      c->layer_threads = (want == 1024 && c->bps_by_threads[1] > 0) ? 1024 : kBlock;
      c->layer_bps = c->bps_by_threads[c->layer_threads == 1024 ? 1 : 0];
    }
    if (cudaEventCreate(&c->ev_layer[0]) != cudaSuccess ||
        cudaEventCreate(&c->ev_layer[1]) != cudaSuccess)
      return cleanup(fail(PP_ERR_CUDA, "event creation failed"));
  }
  if (cfg->cuda_stream) {
    c->stream = (cudaStream_t)cfg->cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    c->own_stream = true;
  }
  const int W = c->W;
  pp_status st;
  if ((st = dmalloc(c, (void**)&c->d_desc, 3 * sizeof(DevTable))) != PP_OK) return cleanup(st);
  if ((st = dmalloc(c, (void**)&c->d_ctl, sizeof(DevCtl))) != PP_OK) return cleanup(st);
  if (pinned_get((void**)&c->h_ctl, sizeof(DevCtl)) != cudaSuccess ||
      pinned_get((void**)&c->h_out, sizeof(double) * cfg->batch) != cudaSuccess)
    return cleanup(fail(PP_ERR_OOM, "pinned host allocation failed"));
  memset(c->h_ctl, 0, sizeof(DevCtl));
  c->overlap_grid = c->sms * 4;
  if ((st = dmalloc(c, (void**)&c->d_partials, sizeof(double) * c->overlap_grid * c->B)) != PP_OK ||
      (st = dmalloc(c, (void**)&c->d_out, sizeof(double) * c->B)) != PP_OK ||
      (st = dmalloc(c, (void**)&c->d_bloch, sizeof(double) * 3 * c->n)) != PP_OK ||
      (st = dmalloc(c, (void**)&c->d_damp, sizeof(double) * (c->n + 1))) != PP_OK ||
      (st = dmalloc(c, (void**)&c->d_ldamp, sizeof(double) * (c->n + 1))) != PP_OK)
    return cleanup(st);
  {
    std::vector<double> damp(c->n + 1, 1.0), ldamp(c->n + 1, 1.0);
    for (int k = 1; k <= c->n; ++k) damp[k] = damp[k - 1] * (1.0 - cfg->noise_p);
    for (int k = 0; k <= c->n; ++k) ldamp[k] = std::exp(-cfg->noise_p * (double)k);
    if (upload(c, c->d_damp, damp.data(), damp.size() * 8) != cudaSuccess ||
        upload(c, c->d_ldamp, ldamp.data(), ldamp.size() * 8) != cudaSuccess)
      return cleanup(fail(PP_ERR_CUDA, "constant table upload failed"));
    DevCtl zero;
    memset(&zero, 0, sizeof(zero));
    zero.wait_limit = (unsigned)cfg->wait_limit;  // 0: the kernels' default bound
    if (upload(c, c->d_ctl, &zero, sizeof(zero)) != cudaSuccess)
      return cleanup(fail(PP_ERR_CUDA, "control block init failed"));
  }
  uint64_t cap = std::max<uint64_t>(4 * (uint64_t)n_terms, 1024);
  cap = (cap + 1023) & ~1023ull;
  size_t need = 2 * table_bytes(cap, index_cap_for(c, cap), W, c->row_bytes()) + c->bytes;
  if (cfg->mem_budget_bytes && need > cfg->mem_budget_bytes)
    return cleanup(fail(PP_ERR_CAPACITY, "initial table exceeds the memory budget"));
  if ((st = alloc_buf(c, c->buf[0], cap)) != PP_OK || (st = alloc_buf(c, c->buf[1], cap)) != PP_OK)
    return cleanup(st);
  c->active = 0;
  if ((st = publish_desc(c)) != PP_OK) return cleanup(st);

  if ((st = ingest_terms(c, n_terms, x, z, coef, on_device)) != PP_OK) return cleanup(st);
  *out = c;
  return PP_OK;
}

// Build the gate arguments of one layer in application (reversed) order.
// theta is [n_gates][B]; src receives the time index of every argument.
pp_status build_gates(pp_ctx* c, int n_gates, const pp_pauli* gates, const double* theta,
                      std::vector<GateArgs>& out, std::vector<int>& src) {
  const int W = c->W;
  out.clear();
  src.clear();
  for (int t = n_gates - 1; t >= 0; --t) {
    const pp_pauli& P = gates[t];
    for (int j = W; j < kMaxW; ++j)
      if (P.x[j] || P.z[j]) return fail(PP_ERR_ARG, "gate has bits in unused words");
    if (key_has_bits_beyond(P.x, P.z, c->n, W))
      return fail(PP_ERR_ARG, "gate has bits at or above n_qubits");
    for (int b = 0; b < c->B; ++b)
      if (!std::isfinite(theta[(size_t)t * c->B + b])) return fail(PP_ERR_ARG, "non-finite angle");
    GateArgs g;
    memset(&g, 0, sizeof(g));
    int pyy = 0, pivot = -1;
    uint64_t pmask = 0;
    for (int j = 0; j < W; ++j) {
      g.px[j] = P.x[j];
      g.pz[j] = P.z[j];
      g.supp[j] = P.x[j] | P.z[j];
      pyy += popcount64(P.x[j] & P.z[j]);
    }
    for (int j = 0; j < 2 * W && pivot < 0; ++j) {
      uint64_t w = j < W ? P.x[j] : P.z[j - W];
      if (w) {
        pivot = j;
        pmask = w & (~w + 1);
      }
    }
    if (pivot < 0) continue;  // identity generator: a global phase, nothing to do
    g.cth = std::cos(theta[(size_t)t * c->B]);
    g.sth = std::sin(theta[(size_t)t * c->B]);
    g.damp = (c->cfg.noise_mode == PP_NOISE_PER_GATE) ? c->d_damp : nullptr;
    g.eps = c->cfg.coeff_eps;
    g.use_eps = c->cfg.coeff_eps > 0.0 ? 1 : 0;
    memcpy(&g.eps_bits, &g.eps, 8);
    g.wmax = c->cfg.max_weight;
    g.pyy = pyy & 3;
    if (pivot < W)
      g.pvx[pivot] = pmask;
    else
      g.pvz[pivot - W] = pmask;
    g.gate_id = (unsigned)out.size();
    out.push_back(g);
    src.push_back(t);
  }
  return PP_OK;
}

// Device copy of a byte block, cached by content (gate arguments, per-gate
// cos/sin columns).
pp_status cached_upload(pp_ctx* c, std::vector<ArgsEntry>& cache,
                        std::vector<unsigned char>&& bytes, const void** out) {
  c->graph_clock++;
  for (auto& e : cache) {
    if (e.sig == bytes) {
      e.last_use = c->graph_clock;
      *out = e.d_args;
      return PP_OK;
    }
  }
  if (cache.size() >= 16) {
    auto it = std::min_element(cache.begin(), cache.end(), [](const ArgsEntry& a, const ArgsEntry& b) {
      return a.last_use < b.last_use;
    });
    dfree(c, it->d_args, it->n);
    cache.erase(it);
  }
  ArgsEntry ent;
  ent.n = bytes.size();
  PP_TRY(dmalloc(c, (void**)&ent.d_args, ent.n));
  PP_CUDA(upload(c, ent.d_args, bytes.data(), ent.n));
  ent.sig = std::move(bytes);
  ent.last_use = c->graph_clock;
  *out = ent.d_args;
  cache.push_back(std::move(ent));
  return PP_OK;
}

// Batched: cos and sin of every column of every gate, in the row element
// type, and the pointer of each gate's block in its arguments.
pp_status batched_columns(pp_ctx* c, std::vector<GateArgs>& args, const std::vector<int>& src,
                          const double* theta) {
  const int B = c->B;
  std::vector<unsigned char> bytes(args.size() * 2 * B * c->esize);
  for (size_t k = 0; k < args.size(); ++k) {
    const double* th = theta + (size_t)src[k] * B;
    for (int b = 0; b < B; ++b) {
      const double cv = std::cos(th[b]), sv = std::sin(th[b]);
      if (c->f32) {
        float* f = reinterpret_cast<float*>(bytes.data()) + k * 2 * B;
        f[b] = (float)cv;
        f[B + b] = (float)sv;
      } else {
        double* d = reinterpret_cast<double*>(bytes.data()) + k * 2 * B;
        d[b] = cv;
        d[B + b] = sv;
      }
    }
  }
  const void* dev = nullptr;
  PP_TRY(cached_upload(c, c->cs_cache, std::move(bytes), &dev));
  for (size_t k = 0; k < args.size(); ++k)
    args[k].csb = static_cast<const unsigned char*>(dev) + k * 2 * B * c->esize;
  return PP_OK;
}

pp_status ensure_events(pp_ctx* c, size_t k) {
  while (c->ev_start.size() < k) {
    cudaEvent_t a, b;
    PP_CUDA(cudaEventCreate(&a));
    PP_CUDA(cudaEventCreate(&b));
    c->ev_start.push_back(a);
    c->ev_end.push_back(b);
  }
  return PP_OK;
}

// Queue the gate kernels; with profile_kernels each is bracketed by event
// records (inside a capture they must be external records to become event
// nodes of the graph).
cudaError_t enqueue_gates(pp_ctx* c, const std::vector<GateArgs>& args, int grid, bool capturing) {
  const DevTable* tab = c->d_desc + 2;
  const bool prof = c->cfg.profile_kernels != 0;
  const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  for (size_t k = 0; k < args.size(); ++k) {
    cudaError_t e;
    if (prof && (e = cudaEventRecordWithFlags(c->ev_start[k], c->stream, flags)) != cudaSuccess)
      return e;
    e = c->batched ? launch_gate_batched(c->W, c->f32, grid, c->stream, tab, c->d_ctl, args[k], k > 0)
                   : launch_gate(c->W, grid, c->stream, tab, c->d_ctl, args[k], k > 0);
    if (e != cudaSuccess) return e;
    if (prof && (e = cudaEventRecordWithFlags(c->ev_end[k], c->stream, flags)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

pp_status launch_layer_gates(pp_ctx* c, const std::vector<GateArgs>& args, int grid) {
  if (c->cfg.profile_kernels) PP_TRY(ensure_events(c, args.size()));
  c->launches += (int64_t)args.size();
  if (!c->cfg.use_graphs || args.size() < 2) {
    PP_CUDA(enqueue_gates(c, args, grid, false));
    return PP_OK;
  }
  std::vector<unsigned char> sig(args.size() * sizeof(GateArgs));
  memcpy(sig.data(), args.data(), sig.size());
  c->graph_clock++;
  for (auto& e : c->graphs) {
    if (e.grid == grid && e.sig == sig) {
      e.last_use = c->graph_clock;
      PP_CUDA(cudaGraphLaunch(e.exec, c->stream));
      return PP_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  PP_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = enqueue_gates(c, args, grid, true);
  if (ce != cudaSuccess) {
    cudaStreamEndCapture(c->stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ce, "gate launch during capture");
  }
  PP_CUDA(cudaStreamEndCapture(c->stream, &graph));
  GraphEntry ent;
  ent.sig = std::move(sig);
  ent.grid = grid;
  ent.last_use = c->graph_clock;
  cudaError_t e = cudaGraphInstantiate(&ent.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  if (c->graphs.size() >= 16) {
    auto it = std::min_element(c->graphs.begin(), c->graphs.end(),
                               [](const GraphEntry& a, const GraphEntry& b) {
                                 return a.last_use < b.last_use;
                               });
    cudaGraphExecDestroy(it->exec);
    c->graphs.erase(it);
  }
  c->graphs.push_back(std::move(ent));
  PP_CUDA(cudaGraphLaunch(c->graphs.back().exec, c->stream));
  return PP_OK;
}

// Add the durations of gate kernels [from, to) of the last launch (the
// stream has been synchronised).
pp_status collect_gate_times(pp_ctx* c, unsigned from, unsigned to) {
  if (!c->cfg.profile_kernels) return PP_OK;
  for (unsigned k = from; k < to && k < c->ev_start.size(); ++k) {
    float ms = 0.f;
    PP_CUDA(cudaEventElapsedTime(&ms, c->ev_start[k], c->ev_end[k]));
    c->gate_ms += ms;
    c->gates_timed++;
  }
  return PP_OK;
}

// Device copy of a layer's gate arguments (cached by content).
pp_status device_args(pp_ctx* c, const std::vector<GateArgs>& args, const GateArgs** out) {
  std::vector<unsigned char> sig(args.size() * sizeof(GateArgs));
  memcpy(sig.data(), args.data(), sig.size());
  c->graph_clock++;
  for (auto& e : c->arg_cache) {
    if (e.sig == sig) {
      e.last_use = c->graph_clock;
      *out = e.d_args;
      return PP_OK;
    }
  }
  if (c->arg_cache.size() >= 16) {
    auto it = std::min_element(c->arg_cache.begin(), c->arg_cache.end(),
                               [](const ArgsEntry& a, const ArgsEntry& b) {
                                 return a.last_use < b.last_use;
                               });
    dfree(c, it->d_args, it->n);
    c->arg_cache.erase(it);
  }
  ArgsEntry ent;
  ent.n = args.size() * sizeof(GateArgs);
  PP_TRY(dmalloc(c, (void**)&ent.d_args, ent.n));
  PP_CUDA(upload(c, ent.d_args, args.data(), ent.n));
  ent.sig = std::move(sig);
  ent.last_use = c->graph_clock;
  *out = ent.d_args;
  c->arg_cache.push_back(std::move(ent));
  return PP_OK;
}

pp_status ensure_merged(pp_ctx* c) {
  if (c->merged) return PP_OK;
  return merge_active(c, PP_SYM_NONE);
}

// Dense copy of the stored entries [0, n) of the active table (keys and
// coefficients or rows; no index).
pp_status take_snapshot(pp_ctx* c, Buf& s, uint64_t n) {
  s = Buf();
  if (n == 0) return PP_OK;
  const size_t need = (size_t)n * (16 * c->W + c->row_bytes());
  if (c->cfg.mem_budget_bytes && c->bytes + need > c->cfg.mem_budget_bytes)
    return fail(PP_ERR_CAPACITY, "no room in the memory budget for the copy that lets a layer be undone");
  const Buf& a = c->buf[c->active];
  PP_TRY(dmalloc(c, (void**)&s.keys, (size_t)n * 16 * c->W));
  PP_CUDA(cudaMemcpyAsync(s.keys, a.keys, (size_t)n * 16 * c->W, cudaMemcpyDeviceToDevice, c->stream));
  if (c->batched) {
    PP_TRY(dmalloc(c, &s.rows, (size_t)n * c->B * c->esize));
    PP_TRY(dmalloc(c, (void**)&s.alive, (size_t)n));
    PP_CUDA(cudaMemcpyAsync(s.rows, a.rows, (size_t)n * c->B * c->esize, cudaMemcpyDeviceToDevice,
                            c->stream));
    PP_CUDA(cudaMemcpyAsync(s.alive, a.alive, (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    PP_TRY(dmalloc(c, (void**)&s.coef, (size_t)n * 8));
    PP_CUDA(cudaMemcpyAsync(s.coef, a.coef, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  s.cap = n;
  return PP_OK;
}

void free_snapshot(pp_ctx* c, Buf& s, uint64_t n) {
  dfree(c, s.keys, (size_t)n * 16 * c->W);
  dfree(c, s.coef, (size_t)n * 8);
  dfree(c, s.rows, (size_t)n * c->B * c->esize);
  dfree(c, s.alive, (size_t)n);
  s = Buf();
}

// Rebuild the active table (entries and index) from a snapshot of n entries.
// The active table's capacity never drops below what it held at the
// snapshot, so the entries fit.
pp_status restore_snapshot(pp_ctx* c, const Buf& s, uint64_t n) {
  Buf& d = c->buf[c->active];
  if (d.cap < n) return fail(PP_ERR_INTERNAL, "table shrank below its size before the layer");
  PP_CUDA(cudaMemsetAsync(d.index, 0, (size_t)d.icap * 8, c->stream));
  PP_TRY(ctl_prepare_insert(c, 0));
  if (n > 0) {
    DevTable src = desc_of(c, s);
    src.index = nullptr;
    src.imask = 0;
    if (c->batched) {
      PP_CUDA(launch_compact_batched(c->W, grid_for(c, n, 4), c->stream, src, n, desc_of(c, d), 1,
                                     0.0, -1, c->d_ctl));
    } else {
      PP_CUDA(launch_compact(c->W, grid_for(c, n, 4), c->stream, src, n, desc_of(c, d), 1,
                             c->cfg.coeff_eps, 0.0, -1, c->d_ctl));
    }
    c->launches += 1;
  }
  PP_TRY(ctl_commit(c));
  PP_TRY(activate(c, c->active));
  c->merged = true;
  return PP_OK;
}

// Blocks a persistent layer launch over a table of n_now stored strings asks
// for: one string per thread per pass (batched rows B/32 times as many, and
// sized for the table the layer is expected to reach), times the tuner's grid
// scale; never more than the GPU holds at once.
uint64_t layer_grid_want(const pp_ctx* c, uint64_t n_now) {
  const int nt = c->batched ? kBlock : c->layer_threads;
  const uint64_t rowf = c->batched ? std::max<uint64_t>(1, (uint64_t)c->B / 32) : 1;
  const double grow = c->batched ? std::max(1.25, c->last_growth) : 1.25;
  const double e = std::max(1.0, (double)n_now * grow);
  const uint64_t want = (uint64_t)std::ceil(e * (double)rowf * c->grid_scale / nt);
  const uint64_t full = std::max<uint64_t>(1, (uint64_t)c->sms * c->layer_bps);
  return std::min<uint64_t>(std::max<uint64_t>(want, 1), full);
}

// Everything pp_apply_layer does after the entry merge: damping, room, the
// gate launches (with the capacity-stall loop) and the boundary merge.
pp_status apply_layer_core(pp_ctx* c, std::vector<GateArgs>& args, const std::vector<int>& src_t,
                           const double* theta, int symmetric_boundary) {
  if (c->cfg.noise_mode == PP_NOISE_PER_LAYER && c->n_terms > 0) {
    PP_CUDA(launch_damp_layer(c->W, grid_for(c, c->n_terms, 4), c->stream,
                              desc_of(c, c->buf[c->active]), c->d_ctl, c->d_ldamp, c->cfg.coeff_eps));
    c->live_known = false;  // damping may truncate entries
    c->launches += 1;
  }
  // room for 2 x room_factor (1.25 unless configured) times the growth the
  // previous layer showed, and at least twice the stored terms
  const double rf = c->cfg.room_factor > 0.0 ? c->cfg.room_factor : 1.25;
  const uint64_t factor =
      std::max<uint64_t>(2, (uint64_t)std::ceil(2.0 * rf * std::max(1.0, c->last_growth)));
  PP_TRY(make_room(c, factor));
  const uint64_t n_start = std::max<uint64_t>(c->n_terms, 1);
  const uint64_t est = std::max<uint64_t>(c->n_terms + c->n_terms / 4, 1);
  const bool layered = c->cfg.layer_kernel && c->layer_bps > 0;
  if (c->batched && !args.empty()) PP_TRY(batched_columns(c, args, src_t, theta));
  int grid_b = 1;
  // batched rows take a warp B/32 steps per pair, so they get B/32 times the blocks
  const uint64_t rowf = c->batched ? std::max<uint64_t>(1, (uint64_t)c->B / 32) : 1;
  // persistent: one string per thread per pass, never more blocks than can
  // be co-resident (the grid barrier needs all of them).  Batched rows size
  // the grid for the table the layer is expected to reach (the previous
  // layer's growth), since their row work dwarfs the scan and a table that
  // grows tenfold within the layer would otherwise run on a tenth of the
  // blocks; a relaunch after a stall sizes it again.
  auto layered_grid = [&](uint64_t n_now) {
    const uint64_t want = layer_grid_want(c, n_now);
    const uint64_t room = std::max<uint64_t>(
        1, (uint64_t)std::floor((double)c->sms * c->layer_bps * c->grid_frac));
    return (int)std::min<uint64_t>(want, room);
  };
  if (layered) {
    grid_b = layered_grid(c->n_terms);
  } else {
    // a power of two so that captured graphs are reused
    while ((double)grid_b * kBlock < (double)(est * rowf) * c->grid_scale) grid_b <<= 1;
    grid_b = std::min(grid_b, c->sms * (c->batched ? 8 : c->gate_bps));
  }
  const GateArgs* d_args = nullptr;
  if (layered && !args.empty()) PP_TRY(device_args(c, args, &d_args));
  // with a group (single column) the boundary merge is queued right behind the
  // gates, guarded by the stall flag, so one read of the control block serves both
  const bool queue_it = symmetric_boundary && c->cfg.symmetry != PP_SYM_NONE && !c->batched;
  bool merged_now = false;
  if (!args.empty()) {
    unsigned first = 0;
    for (;;) {
      PP_CUDA(launch_chain_init(c->stream, c->d_ctl, first));
      if (layered) {
        if (c->cfg.profile_kernels) PP_CUDA(cudaEventRecord(c->ev_layer[0], c->stream));
        if (c->batched)
          PP_CUDA(launch_layer_batched(c->W, c->f32, grid_b, c->stream, c->d_desc + 2, c->d_ctl,
                                       d_args, (unsigned)args.size()));
        else
          PP_CUDA(launch_layer(c->W, c->layer_threads, grid_b, c->stream, c->d_desc + 2, c->d_ctl,
                               d_args, (unsigned)args.size()));
        if (c->cfg.profile_kernels) PP_CUDA(cudaEventRecord(c->ev_layer[1], c->stream));
        c->launches += 1;
      } else {
        PP_TRY(launch_layer_gates(c, args, grid_b));
      }
      PP_CUDA(launch_chain_finish(c->stream, c->d_ctl, (unsigned)args.size()));
      c->launches += 2;
      if (queue_it) PP_TRY(queue_merge(c, c->cfg.symmetry));
      PP_TRY(read_ctl(c));
      PP_TRY(check_device_error(c));
      const unsigned end = c->h_ctl->stall ? c->h_ctl->stall - 1u : (unsigned)args.size();
      if (layered) {
        if (c->cfg.profile_kernels && end > first) {
          float ms = 0.f;
          PP_CUDA(cudaEventElapsedTime(&ms, c->ev_layer[0], c->ev_layer[1]));
          c->gate_ms += ms;
          c->gates_timed++;
        }
      } else {
        PP_TRY(collect_gate_times(c, first, end));
      }
      if (!c->h_ctl->stall) {
        // stored entries after the last gate (a queued merge leaves after_terms)
        const uint64_t after = c->h_ctl->after_terms;
        c->last_growth = (double)after / (double)n_start;
        if (queue_it) {
          PP_TRY(finish_queued_merge(c));
          merged_now = true;
        } else {
          c->n_terms = c->h_ctl->n_terms;
          c->n_live = c->h_ctl->n_live;
          c->live_known = true;
        }
        break;
      }
      // gate `end` found too little room (the queued merge did nothing):
      // compact and grow, then resume there
      c->stalls++;
      c->n_terms = c->h_ctl->n_terms;
      c->n_live = c->h_ctl->n_live;
      c->live_known = true;
      PP_TRY(make_room(c, std::max<uint64_t>(factor, 4)));
      if (layered) grid_b = layered_grid(c->n_terms);
      first = end;
    }
  }
  if (symmetric_boundary && c->cfg.symmetry != PP_SYM_NONE && !merged_now) {
    PP_TRY(merge_active(c, c->cfg.symmetry));
  }
  return PP_OK;
}

}  // namespace

extern "C" {

pp_status pp_config_default(pp_config* cfg) {
  if (!cfg) return fail(PP_ERR_ARG, "config is null");
  memset(cfg, 0, sizeof(*cfg));
  cfg->symmetry = PP_SYM_NONE;
  cfg->batch = 1;
  cfg->coef_type = PP_COEF_F64;
  cfg->coeff_eps = 0.0;
  cfg->max_weight = -1;
  cfg->noise_mode = PP_NOISE_NONE;
  cfg->noise_p = 0.0;
  cfg->mem_budget_bytes = 0;
  cfg->cuda_stream = nullptr;
  cfg->check_symmetry = 1;
  cfg->use_graphs = 1;
  cfg->profile_kernels = 0;
  cfg->layer_kernel = 1;
  cfg->merge_method = PP_MERGE_HASH;
  cfg->wait_limit = 0;
  cfg->room_factor = 0.0;
  cfg->block_threads = 0;
  return PP_OK;
}

pp_status pp_debug_fail_alloc_after(int64_t n) {
  g_fail_alloc_after.store(n < 0 ? -1 : (long long)n);
  return PP_OK;
}

pp_status pp_create(const pp_config* cfg, int64_t n_terms, const uint64_t* x, const uint64_t* z,
                    const double* coef, pp_ctx** out) {
  Range range_("pp_create");
  return create_common(cfg, n_terms, x, z, coef, false, out);
}

pp_status pp_create_device(const pp_config* cfg, int64_t n_terms, const uint64_t* x,
                           const uint64_t* z, const double* coef, pp_ctx** out) {
  Range range_("pp_create_device");
  return create_common(cfg, n_terms, x, z, coef, true, out);
}

pp_status pp_import(pp_ctx* c, int64_t n_terms, const uint64_t* x, const uint64_t* z,
                    const double* coef) {
  Range range_("pp_import");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (n_terms < 0) return fail(PP_ERR_ARG, "n_terms < 0");
  if (n_terms > 0 && (!x || !z || !coef)) return fail(PP_ERR_ARG, "null term arrays");
  if ((uint64_t)n_terms >= (1ull << 31)) return fail(PP_ERR_ARG, "too many input terms");
  PP_TRY(ensure_capacity(c, std::max<uint64_t>(4 * (uint64_t)n_terms, 1024)));
  return ingest_terms(c, n_terms, x, z, coef, false, true);
}

pp_status pp_destroy(pp_ctx* c) {
  if (!c) return PP_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& e : c->graphs) cudaGraphExecDestroy(e.exec);
  c->graphs.clear();
  for (auto e : c->ev_start) cudaEventDestroy(e);
  for (auto e : c->ev_end) cudaEventDestroy(e);
  for (auto& a : c->arg_cache) dfree(c, a.d_args, a.n);
  c->arg_cache.clear();
  for (auto e : c->ev_layer)
    if (e) cudaEventDestroy(e);
  free_buf(c, c->buf[0]);
  free_buf(c, c->buf[1]);
  dfree(c, c->sort_scratch, c->sort_scratch_bytes);
  dfree(c, c->d_desc, 3 * sizeof(DevTable));
  dfree(c, c->d_ctl, sizeof(DevCtl));
  dfree(c, c->d_damp, sizeof(double) * (c->n + 1));
  dfree(c, c->d_ldamp, sizeof(double) * (c->n + 1));
  dfree(c, c->d_partials, sizeof(double) * c->overlap_grid * c->B);
  dfree(c, c->d_out, sizeof(double) * c->B);
  for (auto& a : c->cs_cache) dfree(c, a.d_args, a.n);
  c->cs_cache.clear();
  dfree(c, c->d_bloch, sizeof(double) * 3 * c->n);
  size_t sn = (size_t)(c->n + 1) * (c->n + 1) * (c->n + 1) * sizeof(double);
  dfree(c, c->d_sn, sn);
  dfree(c, c->d_sn_work, sn);
  if (c->stream) cudaStreamSynchronize(c->stream);
  pinned_put(c->h_ctl, sizeof(DevCtl));
  pinned_put(c->h_out, sizeof(double) * c->B);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return PP_OK;
}

pp_status pp_apply_layer(pp_ctx* c, int n_gates, const pp_pauli* gates, const double* theta,
                         int symmetric_boundary) {
  Range range_("pp_apply_layer");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (n_gates < 0 || (n_gates > 0 && (!gates || !theta)))
    return fail(PP_ERR_ARG, "bad gate arrays");
  std::vector<GateArgs> args;
  std::vector<int> src_t;
  PP_TRY(build_gates(c, n_gates, gates, theta, args, src_t));
  // a layer already validated for this context (same gates and angles: a
  // Trotter step repeated) is not checked again
  std::vector<unsigned char> sig;
  bool validated = false;
  if (c->cfg.symmetry != PP_SYM_NONE && c->cfg.check_symmetry && n_gates > 0) {
    sig.resize((size_t)n_gates * (sizeof(pp_pauli) + sizeof(double) * c->B));
    memcpy(sig.data(), gates, (size_t)n_gates * sizeof(pp_pauli));
    memcpy(sig.data() + (size_t)n_gates * sizeof(pp_pauli), theta,
           (size_t)n_gates * sizeof(double) * c->B);
    for (const auto& v : c->sym_ok) validated |= (v == sig);
  }
  if (c->cfg.symmetry != PP_SYM_NONE && c->cfg.check_symmetry && n_gates > 0 && !validated) {
    std::vector<HKey> ks;
    for (int t = 0; t < n_gates; ++t) {
      HKey k(2 * c->W);
      for (int j = 0; j < c->W; ++j) {
        k[j] = gates[t].x[j];
        k[c->W + j] = gates[t].z[j];
      }
      ks.push_back(k);
    }
    for (int b = 0; b < c->B; ++b) {
      std::vector<double> vs(n_gates);
      for (int t = 0; t < n_gates; ++t) vs[t] = theta[(size_t)t * c->B + b];
      if (!multiset_invariant(c->cfg.symmetry, c->n, c->W, ks, vs, 0.0))
        return fail(PP_ERR_SYMMETRY, "layer gate multiset is not invariant under the group");
    }
    if (c->sym_ok.size() >= 8) c->sym_ok.erase(c->sym_ok.begin());
    c->sym_ok.push_back(std::move(sig));
  }
  PP_TRY(ensure_merged(c));
  // With a memory budget a layer may stop with PP_ERR_CAPACITY part way
  // through; the table is then put back as it was before the call, from a
  // dense copy taken here (counted against the budget).
  const bool keep_state = c->cfg.mem_budget_bytes > 0;
  Buf snap;
  const uint64_t snap_n = c->n_terms;
  if (keep_state) {
    const pp_status ts = take_snapshot(c, snap, snap_n);
    if (ts != PP_OK) {
      free_snapshot(c, snap, snap_n);
      return ts;
    }
  }
  pp_status st = apply_layer_core(c, args, src_t, theta, symmetric_boundary);
  if (st == PP_ERR_CAPACITY && keep_state) {
    const std::string msg = g_last_error;
    const pp_status rs = restore_snapshot(c, snap, snap_n);
    free_snapshot(c, snap, snap_n);
    if (rs != PP_OK) return rs;
    g_last_error = msg + " (context restored to its state before the call)";
    return PP_ERR_CAPACITY;
  }
  if (keep_state) free_snapshot(c, snap, snap_n);
  return st;
}

// Give both tables an index of f slots per entry of capacity (empty: the
// caller rebuilds the active one, e.g. with restore_snapshot).  False when the
// new index would not fit the memory budget or cannot be allocated.
bool set_index_factor(pp_ctx* c, double f) {
  if (f == c->index_factor) return true;
  const double old = c->index_factor;
  c->index_factor = f;
  size_t grow = 0;
  for (int b = 0; b < 2; ++b) {
    const uint64_t icap = index_cap_for(c, c->buf[b].cap);
    if (icap > c->buf[b].icap) grow += (size_t)(icap - c->buf[b].icap) * 8;
  }
  if (c->cfg.mem_budget_bytes && c->bytes + grow > c->cfg.mem_budget_bytes) {
    c->index_factor = old;
    return false;
  }
  for (int b = 0; b < 2; ++b) {
    Buf& d = c->buf[b];
    dfree(c, d.index, (size_t)d.icap * 8);
    d.index = nullptr;
    d.icap = index_cap_for(c, d.cap);
    if (dmalloc(c, (void**)&d.index, (size_t)d.icap * 8) != PP_OK ||
        cudaMemsetAsync(d.index, 0, (size_t)d.icap * 8, c->stream) != cudaSuccess) {
      // fall back to the old factor (the pool just received those bytes)
      c->index_factor = old;
      for (int k = 0; k <= b; ++k) {
        Buf& r = c->buf[k];
        dfree(c, r.index, (size_t)r.icap * 8);
        r.icap = index_cap_for(c, r.cap);
        if (dmalloc(c, (void**)&r.index, (size_t)r.icap * 8) != PP_OK) r.index = nullptr;
        else cudaMemsetAsync(r.index, 0, (size_t)r.icap * 8, c->stream);
      }
      publish_desc(c);
      return false;
    }
  }
  return publish_desc(c) == PP_OK;
}

pp_status pp_tune(pp_ctx* c, int n_gates, const pp_pauli* gates, const double* theta,
                  double* chosen_scale) {
  Range range_("pp_tune");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (n_gates < 0 || (n_gates > 0 && (!gates || !theta)))
    return fail(PP_ERR_ARG, "bad gate arrays");
  std::vector<GateArgs> args;
  std::vector<int> src_t;
  PP_TRY(build_gates(c, n_gates, gates, theta, args, src_t));
  PP_TRY(ensure_merged(c));
  if (c->n_terms == 0 || args.empty()) {  // nothing to time
    if (chosen_scale) *chosen_scale = c->grid_scale;
    return PP_OK;
  }
  // the table, the device statistics and the host counters, put back after every trial
  Buf snap;
  const uint64_t n0 = c->n_terms;
  {
    const pp_status ts = take_snapshot(c, snap, n0);
    if (ts != PP_OK) {
      free_snapshot(c, snap, n0);
      return ts;
    }
  }
  PP_TRY(read_ctl(c));
  struct Counters {
    double updates;
    unsigned long long gates_done, ac_total;
    double skipped_updates;
    unsigned long long gates_skipped;
  } saved = {c->h_ctl->updates, c->h_ctl->gates_done, c->h_ctl->ac_total,
             c->h_ctl->skipped_updates, c->h_ctl->gates_skipped};
  static_assert(offsetof(DevCtl, gates_skipped) - offsetof(DevCtl, updates) == 32,
                "statistics counters are contiguous");
  const int64_t launches = c->launches, merges = c->merges, compactions = c->compactions,
                regrows = c->regrows, stalls = c->stalls, timed = c->gates_timed;
  const double gate_ms = c->gate_ms, growth = c->last_growth;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto finish = [&](pp_status st) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    free_snapshot(c, snap, n0);
    return st;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return finish(fail(PP_ERR_CUDA, "event creation failed"));
  // Coordinate search: first the launch shape (the persistent layer kernel,
  // where the device has one, or one kernel per gate) with the hash index's
  // load factor, at the current grid scale; then the grid scale for the
  // winner.  Every trial applies the layer to the same table and is undone.
  struct Trial {
    double scale, factor;
    int persistent;
    int threads;  // block size of the persistent kernel
  };
  std::vector<Trial> trials;
  const int lk0 = c->cfg.layer_kernel ? 1 : 0;
  for (double f : {1.5, 3.0}) {
    if (c->batched) {
      if (c->layer_bps > 0) trials.push_back({c->grid_scale, f, 1, kBlock});
    } else {
      for (int k = 0; k < 2; ++k)
        if (c->bps_by_threads[k] > 0) trials.push_back({c->grid_scale, f, 1, k ? 1024 : kBlock});
    }
    trials.push_back({c->grid_scale, f, 0, c->layer_threads});
  }
  Trial best = {c->grid_scale, c->index_factor, lk0, c->layer_threads};
  double best_ms = 1e300;
  auto run_trial = [&](const Trial& tr, pp_status* err) -> double {
    *err = PP_OK;
    if (!set_index_factor(c, tr.factor)) return 1e300;  // beyond the budget: not a candidate
    pp_status st = restore_snapshot(c, snap, n0);  // the table and a fresh index
    if (st != PP_OK) {
      *err = st;
      return 1e300;
    }
    c->cfg.layer_kernel = tr.persistent;
    c->grid_scale = tr.scale;
    if (!c->batched) {
      c->layer_threads = tr.threads;
      c->layer_bps = c->bps_by_threads[tr.threads == 1024 ? 1 : 0];
    }
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) {
      *err = fail(PP_ERR_CUDA, "event record failed");
      return 1e300;
    }
    st = apply_layer_core(c, args, src_t, theta, 0);
    float ms = 0.f;
    if (st == PP_OK &&
        (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = fail(PP_ERR_CUDA, "timing a trial failed");
    *err = st;
    return st == PP_OK ? (double)ms : 1e300;
  };
  auto put_back = [&](const Trial& tr) {
    set_index_factor(c, tr.factor);
    c->cfg.layer_kernel = tr.persistent;
    c->grid_scale = tr.scale;
    if (!c->batched) {
      c->layer_threads = tr.threads;
      c->layer_bps = c->bps_by_threads[tr.threads == 1024 ? 1 : 0];
    }
    return restore_snapshot(c, snap, n0);
  };
  for (const Trial& tr : trials) {
    pp_status st;
    const double ms = run_trial(tr, &st);
    if (st != PP_OK) {
      put_back(best);
      return finish(st);
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = tr;
    }
  }
  for (double scale : {0.5, 2.0, 4.0}) {
    Trial tr = best;
    tr.scale = scale;
    pp_status st;
    const double ms = run_trial(tr, &st);
    if (st != PP_OK) {
      put_back(best);
      return finish(st);
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = tr;
    }
  }
  {
    const pp_status rs = put_back(best);
    if (rs != PP_OK) return finish(rs);
  }
  const double best_scale = best.scale;
  if (upload(c, &c->d_ctl->updates, &saved, sizeof(saved)) != cudaSuccess)
    return finish(fail(PP_ERR_CUDA, "restoring statistics failed"));
  c->launches = launches;
  c->merges = merges;
  c->compactions = compactions;
  c->regrows = regrows;
  c->stalls = stalls;
  c->gates_timed = timed;
  c->gate_ms = gate_ms;
  c->last_growth = growth;
  if (chosen_scale) *chosen_scale = best_scale;
  return finish(PP_OK);
}

pp_status pp_canonicalize(pp_ctx* c) {
  Range range_("pp_canonicalize");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (c->cfg.symmetry == PP_SYM_NONE) return fail(PP_ERR_STATE, "context has no symmetry");
  if (c->n_terms == 0) return PP_OK;
  Buf& b = c->buf[c->active];
  PP_CUDA(launch_canon_inplace(c->W, c->cfg.symmetry, c->n, grid_for(c, c->n_terms, 4), c->stream,
                               b.keys, b.keys, c->n_terms, c->d_ctl));
  c->launches += 1;
  c->merged = false;
  PP_CUDA(cudaStreamSynchronize(c->stream));
  return PP_OK;
}

pp_status pp_merge(pp_ctx* c) {
  Range range_("pp_merge");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  return merge_active(c, PP_SYM_NONE);
}

pp_status pp_truncate(pp_ctx* c, double eps, int max_weight) {
  Range range_("pp_truncate");
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (!(eps >= 0.0)) return fail(PP_ERR_ARG, "eps must be >= 0");
  PP_TRY(ensure_merged(c));
  return compact_into(c, 1 - c->active, eps, max_weight);
}

pp_status pp_expect(pp_ctx* c, const double* bloch, double* out) {
  Range range_("pp_expect");
  if (!c || !bloch || !out) return fail(PP_ERR_ARG, "null argument");
  const int n = c->n, W = c->W;
  for (int i = 0; i < 3 * n; ++i)
    if (!std::isfinite(bloch[i])) return fail(PP_ERR_ARG, "non-finite Bloch component");
  OverlapArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.group = group_kind(c->cfg.symmetry);
  a.lx = group_lx(c->cfg.symmetry);
  if (a.group != PP_SYM_NONE) {
    if (bloch_invariant(c->cfg.symmetry, n, bloch)) {
      a.group = PP_SYM_NONE;  // Eq. 2: orbit members have equal overlaps
    } else if (!c->obs_invariant) {
      return fail(PP_ERR_SYMMETRY, "neither the state nor the observable is invariant");
    }
  }
  bool basis = true;
  for (int q = 0; q < n && basis; ++q)
    basis = bloch[3 * q] == 0.0 && bloch[3 * q + 1] == 0.0 &&
            (bloch[3 * q + 2] == 1.0 || bloch[3 * q + 2] == -1.0);
  if (basis) {
    a.basis = 1;
    for (int q = 0; q < n; ++q)
      if (bloch[3 * q + 2] == -1.0) a.bits[q >> 6] |= 1ull << (q & 63);
  }
  PP_CUDA(cudaMemcpyAsync(c->d_bloch, bloch, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                          c->stream));
  a.bloch = c->d_bloch;
  if (a.group == PP_SYM_SN) {
    size_t sn = (size_t)(n + 1) * (n + 1) * (n + 1);
    if (!c->d_sn) {
      PP_TRY(dmalloc(c, (void**)&c->d_sn, sn * sizeof(double)));
      PP_TRY(dmalloc(c, (void**)&c->d_sn_work, sn * sizeof(double)));
    }
    std::vector<double> bv(bloch, bloch + 3 * n);
    if (bv != c->sn_bloch) {
      PP_CUDA(launch_sn_table(n, c->stream, c->d_bloch, c->d_sn_work, c->d_sn));
      c->launches += 1;
      c->sn_bloch = bv;
    }
    a.sn_table = c->d_sn;
  }
  if (c->batched) {
    PP_CUDA(launch_overlap_batched(W, c->overlap_grid, c->stream, desc_of(c, c->buf[c->active]),
                                   c->n_terms, a, c->d_partials, c->d_out));
  } else {
    PP_CUDA(launch_overlap(W, c->overlap_grid, c->stream, c->buf[c->active].keys,
                           c->buf[c->active].coef, c->n_terms, nullptr, a, c->d_partials,
                           c->d_out));
  }
  c->launches += 2;
  PP_CUDA(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * c->B, cudaMemcpyDeviceToHost,
                          c->stream));
  PP_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(out, c->h_out, sizeof(double) * c->B);
  return PP_OK;
}

pp_status pp_expect_basis(pp_ctx* c, const uint8_t* bits, double* out) {
  if (!c || !bits || !out) return fail(PP_ERR_ARG, "null argument");
  std::vector<double> bloch((size_t)3 * c->n, 0.0);
  for (int q = 0; q < c->n; ++q) bloch[3 * q + 2] = bits[q] ? -1.0 : 1.0;
  return pp_expect(c, bloch.data(), out);
}

pp_status pp_num_terms(pp_ctx* c, int64_t* live, int64_t* stored) {
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  PP_TRY(read_ctl(c));
  c->n_terms = c->h_ctl->n_terms;
  c->n_live = c->h_ctl->n_live;
  c->live_known = true;
  if (live) *live = c->n_live;
  if (stored) *stored = (int64_t)c->n_terms;
  return PP_OK;
}

pp_status pp_export(pp_ctx* c, int64_t capacity, uint64_t* x, uint64_t* z, double* coef,
                    int64_t* n_out) {
  Range range_("pp_export");
  if (!c || !n_out) return fail(PP_ERR_ARG, "null argument");
  PP_TRY(ensure_merged(c));
  PP_TRY(read_ctl(c));
  const int W = c->W;
  int spare = 1 - c->active;
  Buf& d = c->buf[spare];
  // compact into the spare table without an index, then copy it out (the
  // active table stays active, and so do its occupancy masks)
  PP_TRY(ctl_prepare_insert(c, 0, false));
  if (c->batched) {
    PP_CUDA(launch_compact_batched(W, grid_for(c, c->n_terms, 4), c->stream,
                                   desc_of(c, c->buf[c->active]), c->n_terms, desc_of(c, d), 0,
                                   0.0, -1, c->d_ctl));
  } else {
    PP_CUDA(launch_compact(W, grid_for(c, c->n_terms, 4), c->stream, desc_of(c, c->buf[c->active]),
                           c->n_terms, desc_of(c, d), 0, c->cfg.coeff_eps, 0.0, -1, c->d_ctl));
  }
  c->launches += 1;
  PP_TRY(read_ctl(c));
  PP_TRY(check_device_error(c));
  const int64_t m = (int64_t)c->h_ctl->n_next;
  // restore the control block of the live table
  PP_TRY(ctl_prepare_insert(c, c->n_terms, false));
  {
    long long live = c->n_live;
    PP_CUDA(cudaMemcpyAsync(&c->d_ctl->n_live, &live, 8, cudaMemcpyHostToDevice, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
  }
  *n_out = m;
  if (capacity < m) return fail(PP_ERR_ARG, "export capacity too small");
  if (m == 0) return PP_OK;
  if (!x || !z || !coef) return fail(PP_ERR_ARG, "null output arrays");
  std::vector<uint64_t> packed((size_t)m * 2 * W);
  PP_CUDA(cudaMemcpyAsync(packed.data(), d.keys, packed.size() * 8, cudaMemcpyDeviceToHost,
                          c->stream));
  if (c->batched) {
    double* tmp = nullptr;
    const size_t bytes = (size_t)m * c->B * sizeof(double);
    PP_TRY(dmalloc(c, (void**)&tmp, bytes));
    PP_CUDA(launch_rows_to_double(grid_for(c, (uint64_t)m * c->B, 4), c->stream, desc_of(c, d),
                                  (uint64_t)m, tmp));
    PP_CUDA(cudaMemcpyAsync(coef, tmp, bytes, cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    dfree(c, tmp, bytes);
  } else {
    PP_CUDA(cudaMemcpyAsync(coef, d.coef, (size_t)m * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  PP_CUDA(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < m; ++i)
    for (int j = 0; j < W; ++j) {
      x[i * W + j] = packed[i * 2 * W + j];
      z[i * W + j] = packed[i * 2 * W + W + j];
    }
  return PP_OK;
}

pp_status pp_stats(pp_ctx* c, pp_stats_t* out) {
  if (!c || !out) return fail(PP_ERR_ARG, "null argument");
  PP_TRY(read_ctl(c));
  out->live_terms = c->h_ctl->n_live;
  out->stored_terms = (int64_t)c->h_ctl->n_terms;
  out->capacity = (int64_t)c->buf[c->active].cap;
  out->gate_updates = c->h_ctl->updates;
  out->gates_applied = (int64_t)c->h_ctl->gates_done;
  out->merges = c->merges;
  out->compactions = c->compactions;
  out->regrows = c->regrows;
  out->device_bytes = c->bytes;
  out->anticommuting_terms = (double)c->h_ctl->ac_total;
  out->kernel_launches = c->launches;
  out->gate_kernel_ms = c->gate_ms;
  out->gate_kernels_timed = c->gates_timed;
  out->grid_scale = c->grid_scale;
  out->skipped_updates = c->h_ctl->skipped_updates;
  out->gates_skipped = (int64_t)c->h_ctl->gates_skipped;
  out->index_factor = c->index_factor;
  out->persistent = (c->cfg.layer_kernel && c->layer_bps > 0) ? 1 : 0;
  out->block_threads = out->persistent ? (c->batched ? kBlock : c->layer_threads) : kBlock;
  out->stalls = c->stalls;
  {
    const Buf& a = c->buf[c->active];
    out->index_slots = (int64_t)a.icap;
  }
  return PP_OK;
}

pp_status pp_set_grid_fraction(pp_ctx* c, double fraction) {
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  if (!(fraction > 0.0 && fraction <= 1.0)) return fail(PP_ERR_ARG, "fraction must be in (0, 1]");
  ppk::set_grid_fraction(c, fraction);
  return PP_OK;
}

pp_status pp_set_budget(pp_ctx* c, size_t mem_budget_bytes) {
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  c->cfg.mem_budget_bytes = mem_budget_bytes;
  return PP_OK;
}

pp_status pp_synchronize(pp_ctx* c) {
  if (!c) return fail(PP_ERR_ARG, "ctx is null");
  PP_CUDA(cudaStreamSynchronize(c->stream));
  return PP_OK;
}

const char* pp_last_error(void) { return g_last_error.c_str(); }

// ----------------------------------------------------------- stateless calls

pp_status pp_canonical_keys(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                            uint64_t* keys_out, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxW) return fail(PP_ERR_ARG, "bad n_qubits");
  if (!valid_group(symmetry, n_qubits)) return fail(PP_ERR_ARG, "bad symmetry");
  if (m < 0 || (m > 0 && (!keys_in || !keys_out))) return fail(PP_ERR_ARG, "bad arrays");
  if (m == 0) return PP_OK;
  const int W = (n_qubits + 63) / 64;
  int sms = std::max(1, device_sm_count());
  int grid = (int)std::min<int64_t>((m + kBlock * 4 - 1) / (kBlock * 4), (int64_t)sms * 8);
  PP_CUDA(launch_canon_inplace(W, symmetry, n_qubits, std::max(grid, 1), (cudaStream_t)stream,
                               keys_out, keys_in, (uint64_t)m));
  return PP_OK;
}

pp_status pp_merge_terms(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                         const double* coef_in, uint64_t* keys_out, double* coef_out,
                         int64_t* m_out, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxW) return fail(PP_ERR_ARG, "bad n_qubits");
  if (!valid_group(symmetry, n_qubits)) return fail(PP_ERR_ARG, "bad symmetry");
  if (!m_out || m < 0 || (m > 0 && (!keys_in || !coef_in || !keys_out || !coef_out)))
    return fail(PP_ERR_ARG, "bad arrays");
  if ((uint64_t)m >= (1ull << 31)) return fail(PP_ERR_ARG, "too many terms");
  *m_out = 0;
  if (m == 0) return PP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int W = (n_qubits + 63) / 64;
  const uint64_t icap = next_pow2(2 * (uint64_t)m);
  uint64_t* index = nullptr;
  DevCtl* ctl = nullptr;
  PP_CUDA(cudaMallocAsync((void**)&index, icap * 8, s));
  cudaError_t e = cudaMallocAsync((void**)&ctl, sizeof(DevCtl), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(index, s);
    return cuda_fail(e, "cudaMallocAsync");
  }
  DevTable dst = {};
  dst.keys = keys_out;
  dst.coef = coef_out;
  dst.index = index;
  dst.cap = (uint64_t)m;
  dst.imask = icap - 1;
  int sms = std::max(1, device_sm_count());
  int grid = (int)std::min<int64_t>((m + kBlock * 4 - 1) / (kBlock * 4), (int64_t)sms * 8);
  DevCtl h;
  memset(&h, 0, sizeof(h));
  if ((e = cudaMemsetAsync(index, 0, icap * 8, s)) == cudaSuccess &&
      (e = cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s)) == cudaSuccess &&
      (e = launch_merge_insert(W, symmetry, n_qubits, -1, std::max(grid, 1), s, keys_in, coef_in,
                               (uint64_t)m, nullptr, 0, dst, ctl)) == cudaSuccess &&
      (e = cudaMemcpyAsync(&h, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s)) == cudaSuccess) {
    e = cudaStreamSynchronize(s);
  }
  cudaFreeAsync(index, s);
  cudaFreeAsync(ctl, s);
  if (e != cudaSuccess) return cuda_fail(e, "pp_merge_terms");
  if (h.error) return fail(PP_ERR_INTERNAL, "device error in merge");
  *m_out = (int64_t)h.n_next;
  return PP_OK;
}

pp_status pp_merge_terms_sorted(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                                const double* coef_in, uint64_t* keys_out, double* coef_out,
                                int64_t* m_out, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxW) return fail(PP_ERR_ARG, "bad n_qubits");
  if (!sort_merge_supported(n_qubits))
    return fail(PP_ERR_ARG, "the sort-based merge takes n_qubits <= 64");
  if (!valid_group(symmetry, n_qubits)) return fail(PP_ERR_ARG, "bad symmetry");
  if (!m_out || m < 0 || (m > 0 && (!keys_in || !coef_in || !keys_out || !coef_out)))
    return fail(PP_ERR_ARG, "bad arrays");
  if ((uint64_t)m >= (1ull << 31)) return fail(PP_ERR_ARG, "too many terms");
  *m_out = 0;
  if (m == 0) return PP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sbytes = sort_merge_scratch_bytes((uint64_t)m, n_qubits);
  void* scratch = nullptr;
  DevCtl* ctl = nullptr;
  PP_CUDA(cudaMallocAsync(&scratch, sbytes, s));
  cudaError_t e = cudaMallocAsync((void**)&ctl, sizeof(DevCtl), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(scratch, s);
    return cuda_fail(e, "cudaMallocAsync");
  }
  DevTable dst = {};
  memset(&dst, 0, sizeof(dst));
  dst.keys = keys_out;
  dst.coef = coef_out;
  dst.cap = (uint64_t)m;
  DevCtl h;
  memset(&h, 0, sizeof(h));
  if ((e = cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s)) == cudaSuccess &&
      (e = launch_merge_sorted(symmetry, n_qubits, -1, s, keys_in, coef_in, nullptr, 0, nullptr,
                               (uint64_t)m, nullptr, 0, dst, 0, 0.0, ctl, scratch, 0)) ==
          cudaSuccess &&
      (e = cudaMemcpyAsync(&h, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s)) == cudaSuccess) {
    e = cudaStreamSynchronize(s);
  }
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(ctl, s);
  if (e != cudaSuccess) return cuda_fail(e, "pp_merge_terms_sorted");
  if (h.error) return fail(PP_ERR_INTERNAL, "device error in merge");
  *m_out = (int64_t)h.n_next;
  return PP_OK;
}

pp_status pp_overlap_sum(int n_qubits, int symmetry, int64_t m, const uint64_t* keys,
                         const double* coef, const double* bloch, double* out, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxW) return fail(PP_ERR_ARG, "bad n_qubits");
  if (!valid_group(symmetry, n_qubits)) return fail(PP_ERR_ARG, "bad symmetry");
  if (m < 0 || !out || !bloch || (m > 0 && (!keys || !coef))) return fail(PP_ERR_ARG, "bad arrays");
  cudaStream_t s = (cudaStream_t)stream;
  const int W = (n_qubits + 63) / 64;
  int sms = std::max(1, device_sm_count());
  int grid = sms * 4;
  double* partials = nullptr;
  double *sn = nullptr, *work = nullptr;
  size_t snb = (size_t)(n_qubits + 1) * (n_qubits + 1) * (n_qubits + 1) * sizeof(double);
  PP_CUDA(cudaMallocAsync((void**)&partials, sizeof(double) * grid, s));
  cudaError_t e = cudaSuccess;
  if (symmetry == PP_SYM_SN) {
    if ((e = cudaMallocAsync((void**)&sn, snb, s)) == cudaSuccess)
      e = cudaMallocAsync((void**)&work, snb, s);
  }
  OverlapArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n_qubits;
  a.group = group_kind(symmetry);
  a.lx = group_lx(symmetry);
  a.basis = 0;
  a.bloch = bloch;
  a.sn_table = sn;
  if (e == cudaSuccess && symmetry == PP_SYM_SN) e = launch_sn_table(n_qubits, s, bloch, work, sn);
  if (e == cudaSuccess)
    e = launch_overlap(W, grid, s, keys, coef, (uint64_t)m, nullptr, a, partials, out);
  if (partials) cudaFreeAsync(partials, s);
  if (sn) cudaFreeAsync(sn, s);
  if (work) cudaFreeAsync(work, s);
  if (e != cudaSuccess) return cuda_fail(e, "pp_overlap_sum");
  return PP_OK;
}

}  // extern "C"

bool ppk::valid_group_code(int code, int n) { return valid_group(code, n); }

void ppk::set_grid_fraction(pp_ctx* c, double frac) {
  if (c) c->grid_frac = std::min(1.0, std::max(frac, 1e-9));
}

double ppk::layer_fraction_wanted(const pp_ctx* c) {
  if (!c || !c->cfg.layer_kernel || c->layer_bps <= 0) return 0.0;
  const double full = (double)c->sms * c->layer_bps;
  return std::min(1.0, (double)layer_grid_want(c, c->n_terms) / full);
}
