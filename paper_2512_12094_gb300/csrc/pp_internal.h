// Internal declarations shared by the kernels (pp_kernels.cu) and the host
// side of the C ABI (pp_api.cu).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace ppk {

constexpr int kMaxW = 4;                    // up to 256 qubits
constexpr uint32_t kPendingIdx = 0xFFFFFFFFu;  // index slot claimed, dense position not yet published
constexpr int kBlock = 256;

// Device-side error bits (DevCtl::error / err_pending).
enum : unsigned {
  kErrProbe = 1u,    // a hash probe walked the whole index without finding a slot
  kErrTimeout = 2u,  // a bounded wait for a published slot ran out
  kErrAppend = 4u,   // an append went past the dense capacity
};

// Term table: dense arrays of keys and coefficients plus an open-addressing
// index from key to dense position.
//   keys  [cap][2W]  x words then z words of each string
//   coef  [cap]      FP64 coefficient; a truncated entry holds +0.0
//   index [icap]     slot = (tag << 32) | dense position, 0 = empty
// Batched tables (B angle sets, or FP32 storage) keep a row of B
// coefficients per string in `rows` ([cap][B] of float or double) and a
// liveness byte per string in `alive` instead of using `coef`: a row is dead
// when every column was truncated, and readers treat a dead row as zeros.
struct DevTable {
  uint64_t* keys;
  double* coef;
  uint64_t* index;
  uint64_t cap;
  uint64_t imask;  // icap - 1, icap a power of two >= 1.5 cap
  void* rows;
  unsigned char* alive;
  int B;
  int f32;  // rows hold float (1) or double (0)
};

// Per-context counters in device memory.
//
// Between operations the table size is (n_terms, n_live).  Inside a layer the
// gate kernels pass it along without any end-of-kernel bookkeeping: gate g
// (layer-local id) reads its input size from slot (g+2)%3, records it in slot
// g%3, appends births by atomics on cnt[g%3], accumulates its live-count
// change in dlt[g%3], and clears slot (g+1)%3 for gate g+1.  Every block of a
// gate therefore reads the same, final values written by gate g-1.  Lines hit
// by many blocks are kept apart so that different L2 slices serve them.
struct alignas(128) DevCtl {
  unsigned long long n_terms;  // stored entries [0, n_terms) between operations
  long long n_live;            // entries holding a kept coefficient
  unsigned int stall;          // 1 + id of a gate that found too little capacity; 0 = none
  unsigned int first_gate;     // gates with a smaller layer-local id skip themselves
  unsigned int error;          // error bits (any kernel)
  unsigned int wait_limit;     // microseconds a bounded device wait may last; 0 = the default
  alignas(128) unsigned long long base[3];  // stored entries entering the gate of a slot
  long long live_base[3];                   // live entries entering the gate of a slot
  alignas(128) unsigned long long cnt[3];   // births appended by the gate of a slot
  alignas(128) long long dlt[3];            // live-count change by the gate of a slot
  // error bits raised by the gate of a slot (also ORed into error).  A
  // cooperative layer reads the slot of the gate it has just finished after
  // the grid barrier: only that gate's blocks can have written it, so every
  // block takes the same decision, whereas error may already hold a bit set
  // by a fast block in the next gate.
  unsigned int gerr[3];
  alignas(128) double updates;              // sum of live terms entering each gate
  unsigned long long gates_done;
  unsigned long long ac_total;              // sum of live anticommuting terms per gate
  double skipped_updates;                   // live terms entering gates the occupancy test skipped
  unsigned long long gates_skipped;
  // OR of the x words and of the z words of every stored string (a superset
  // is allowed): a gate P with (x_P & occ_z) | (z_P & occ_x) == 0 commutes
  // with every string, so the layer kernel skips it without a scan.
  alignas(128) unsigned long long occ[2 * kMaxW];
  // State a cooperative layer kernel leaves on exit (block 0 writes it): the
  // stored and live entries after the last gate it applied.  It has lines of
  // its own because other blocks may still be reading the gate slots when
  // block 0 leaves.  chain_finish takes it when exit_set is 1, else the slot
  // of the last gate; it copies the stored count to after_terms, which a
  // merge queued behind the layer leaves alone.
  alignas(128) unsigned long long exit_terms;
  long long exit_live;
  unsigned int exit_set;
  unsigned int entry_stop;  // chain_init: an error was already set (every block returns)
  unsigned long long after_terms;
  alignas(128) unsigned long long n_next;   // append cursor of merge / compaction kernels
  alignas(128) unsigned int bar_root;       // grid-barrier counter of the cooperative layer
                                            // kernel (grows by gridDim per barrier)
  // The first device error and where it happened: kind 1 grid barrier of
  // the layer kernel, 2 of the batched layer kernel, 3 claimed index slot
  // (bounded waits that ran out: the counter seen against the one waited
  // for); 4 a birth past the capacity (its position and the capacity); 5 an
  // index probe that walked the whole index (T0 and the index mask); with
  // the layer-local gate id.
  alignas(128) unsigned int to_kind;
  unsigned int to_gate;
  unsigned int to_seen;
  unsigned int to_target;
};

struct GateArgs {
  uint64_t px[kMaxW], pz[kMaxW], supp[kMaxW];
  double cth, sth;         // cos(theta), sin(theta), computed on the host
  const double* damp;      // (1-p)^k, k = 0..n, or nullptr when no per-gate noise
  double eps;              // coefficient truncation; 0 = off
  uint64_t eps_bits;       // bit pattern of eps: |c| < eps  <=>  (bits(c) & ~sign) < eps_bits
  int use_eps;             // eps > 0
  int wmax;                // weight truncation; < 0 = off
  int pyy;                 // popcount(px & pz) mod 4 (the Y count of P)
  uint64_t pvx[kMaxW], pvz[kMaxW];  // one bit of P (x or z plane): the pair member
                                    // with this bit clear owns the pair
  unsigned int gate_id;    // layer-local position in application order
  const void* csb;         // batched: cos[B] then sin[B] of this gate (row element type)
};

struct OverlapArgs {
  int n;
  int group;        // 0 plain, 1 Z_n orbit average, 2 S_n table lookup,
                    // 3 D_n / 4 torus average over the group elements
  int lx;           // torus lattice width (group 4)
  int basis;        // 1: rho is a computational basis state given by bits
  uint64_t bits[kMaxW];
  const double* bloch;     // [n][3] device array (product mode)
  const double* sn_table;  // [(n+1)^3] orbit-averaged overlaps (group 2)
};

// ---------------------------------------------------------------- launchers
// All return the launch status; W is the number of words per mask.

// Before the first gate of a (resumed) layer: slot (first+2)%3 <- (n_terms,
// n_live), counters of slot first%3 cleared, stall cleared.
cudaError_t launch_chain_init(cudaStream_t s, DevCtl* ctl, unsigned first_gate);
// Before a merge or compaction into a fresh table: append cursor n_next <-
// first_free, live count <- 0, and with reset_occ the occupancy masks <- 0
// (the kernels that fill the table OR its keys back in).  Stream ordered, no
// host round trip.
cudaError_t launch_ctl_insert(cudaStream_t s, DevCtl* ctl, unsigned long long first_free,
                              int guarded = 0, int reset_occ = 1);
// n_terms <- n_next (after a merge or compaction); guarded as above.
cudaError_t launch_ctl_commit(cudaStream_t s, DevCtl* ctl, int guarded);
// After the gates of a layer (n_gates of them): (n_terms, n_live) <- the state
// after the last gate that ran.
cudaError_t launch_chain_finish(cudaStream_t s, DevCtl* ctl, unsigned n_gates);

// All gates of a layer in one cooperative launch (grid <= co-resident blocks);
// gates points to n_gates GateArgs in device memory.  threads: block size,
// 256 or 1024 (1024 for W <= 2 only).
cudaError_t launch_layer(int W, int threads, int grid, cudaStream_t s, const DevTable* tab,
                         DevCtl* ctl, const GateArgs* gates, unsigned n_gates);
// co-resident layer-kernel blocks per SM for that block size (0: none)
int layer_blocks_per_sm(int W, int threads);

// One gate kernel.  With pdl set it is launched with programmatic stream
// serialisation: it may start while the previous kernel on the stream
// finishes and waits (griddepcontrol) before touching any data.
cudaError_t launch_gate(int W, int grid, cudaStream_t s, const DevTable* tab, DevCtl* ctl,
                        const GateArgs& g, bool pdl);

// src entries [0, count) (count read from *count_dev when count_dev != null)
// -> drop those heavier than wmax (>= 0) -> representatives under `group`
// -> accumulate into dst (dst index clear, ctl->n_next = first free dense
// position).  Entries whose coefficient is +0.0 are skipped when skip_zero.
cudaError_t launch_merge_insert(int W, int group, int n, int wmax, int grid, cudaStream_t s,
                                const uint64_t* src_keys, const double* src_coef,
                                uint64_t count, const unsigned long long* count_dev,
                                int skip_zero, DevTable dst, DevCtl* ctl, int guarded = 0);

// Coefficient truncation (eps > 0) of dst entries [0, ctl->n_next); adds the
// live count to ctl->n_live.  guarded: do nothing if ctl->stall or
// ctl->error is set (a merge queued behind a layer that may have stopped for
// capacity or failed).
cudaError_t launch_finalize(int grid, cudaStream_t s, DevTable dst, DevCtl* ctl, double eps,
                            int guarded = 0);

// Copy entries of src[0, count) that are kept (not truncated under eps, and
// |c| >= extra_eps when extra_eps > 0, weight <= extra_wmax when >= 0) into
// dst, ctl->n_next as append cursor; inserts into dst's (clear) index when
// with_index.  Adds the copied count to ctl->n_live.
cudaError_t launch_compact(int W, int grid, cudaStream_t s, DevTable src, uint64_t count,
                           DevTable dst, int with_index, double eps, double extra_eps,
                           int extra_wmax, DevCtl* ctl);

// keys[i] = representative of keys_in[i] (keys may equal keys_in); with ctl,
// the representatives are ORed into its occupancy masks.
cudaError_t launch_canon_inplace(int W, int group, int n, int grid, cudaStream_t s,
                                 uint64_t* keys, const uint64_t* keys_in, uint64_t count,
                                 DevCtl* ctl = nullptr);

// c <- c * table[weight(Q)] then coefficient truncation, over [0, n_terms);
// adds the change of the live count to ctl->n_live.
cudaError_t launch_damp_layer(int W, int grid, cudaStream_t s, DevTable t, DevCtl* ctl,
                              const double* table, double eps);

// sum_i coef[i] ov(keys[i]) -> partials[grid] -> out[0] (two passes, fixed order).
cudaError_t launch_overlap(int W, int grid, cudaStream_t s, const uint64_t* keys,
                           const double* coef, uint64_t count,
                           const unsigned long long* count_dev, const OverlapArgs& a,
                           double* partials, double* out);

// S_n orbit-averaged overlap table [(n+1)^3] for a product state (one block);
// work is a scratch buffer of the same size.
cudaError_t launch_sn_table(int n, cudaStream_t s, const double* bloch, double* work,
                            double* table);

// x [m][W], z [m][W] (device) -> keys [m][2W]; *bad |= 1 if a string has
// bits at or above n.
cudaError_t launch_pack_keys(int W, int n, int grid, cudaStream_t s, const uint64_t* x,
                             const uint64_t* z, uint64_t m, uint64_t* keys, unsigned* bad);

// Message returned by pp_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Is code a known group (pp_symmetry, with the torus width above the low
// byte for PP_SYM_TORUS) for n qubits?
bool valid_group_code(int code, int n);

}  // namespace ppk
struct pp_ctx;
namespace ppk {
// Limit a context's persistent layer launches to the fraction `frac` (0, 1]
// of the GPU's co-resident blocks, so that contexts whose fractions add up to
// at most 1 (the server's jobs) can run their layers at the same time.
void set_grid_fraction(pp_ctx* c, double frac);
// The fraction of the GPU's co-resident blocks the context's next persistent
// layer launch would use with no limit (0 when it has no persistent path).
double layer_fraction_wanted(const pp_ctx* c);

// ------------------------------------------------------- batched launchers
// Same contracts as the single-column kernels above, on B-column rows.
cudaError_t launch_gate_batched(int W, int f32, int grid, cudaStream_t s, const DevTable* tab,
                                DevCtl* ctl, const GateArgs& g, bool pdl);
// All gates of a batched layer in one cooperative launch (grid <= co-resident
// blocks), as launch_layer for the single column.
cudaError_t launch_layer_batched(int W, int f32, int grid, cudaStream_t s, const DevTable* tab,
                                 DevCtl* ctl, const GateArgs* gates, unsigned n_gates);
int layer_batched_blocks_per_sm(int W, int f32);  // 0: no cooperative path
// src rows: element type f32 (1) / double (0), or double input rows when
// src_alive == nullptr (ingest); acc: [cap][B] doubles, zeroed by the caller.
cudaError_t launch_merge_batched(int W, int group, int n, int wmax, int src_f32, int grid,
                                 cudaStream_t s, const uint64_t* src_keys, const void* src_rows,
                                 const unsigned char* src_alive, uint64_t count, DevTable dst,
                                 double* acc, DevCtl* ctl);
// acc rows -> dst rows (element type of dst), liveness by the any-column rule.
cudaError_t launch_finalize_batched(int grid, cudaStream_t s, DevTable dst, const double* acc,
                                    DevCtl* ctl, double eps);
cudaError_t launch_compact_batched(int W, int grid, cudaStream_t s, DevTable src, uint64_t count,
                                   DevTable dst, int with_index, double extra_eps,
                                   int extra_wmax, DevCtl* ctl);
// out[B] = sum over live strings of row * overlap; partials: [grid][B].
cudaError_t launch_overlap_batched(int W, int grid, cudaStream_t s, DevTable t, uint64_t count,
                                   const OverlapArgs& a, double* partials, double* out);
// rows (any element type) -> doubles [count][B] (export)
cudaError_t launch_rows_to_double(int grid, cudaStream_t s, DevTable t, uint64_t count,
                                  double* out);

// ------------------------------------------------------ sort-based merge
// The merge of launch_merge_insert / launch_merge_batched done as an LSD radix
// sort of the representatives (exact keys; n <= 64, one word per mask) and a
// segmented FP64 reduce in input order (deterministic sums).  Single column:
// src_coef != nullptr (entries equal to +0.0 skipped when skip_zero); batched:
// src_coef == nullptr, src_rows / src_f32 / src_alive describe the source rows
// and the reduce also writes liveness by the any-column rule under eps and adds
// the live count (no finalize pass needed).  The distinct keys go to dst from
// ctl->n_next on, which is advanced; with_index: they are also inserted into
// dst's (clear) index.  scratch: sort_merge_scratch_bytes(count, n) bytes;
// count is an upper bound when count_dev is given.  guarded as above.
bool sort_merge_supported(int n);
size_t sort_merge_scratch_bytes(uint64_t count, int n);
cudaError_t launch_merge_sorted(int group, int n, int wmax, cudaStream_t s,
                                const uint64_t* src_keys, const double* src_coef,
                                const void* src_rows, int src_f32,
                                const unsigned char* src_alive, uint64_t count,
                                const unsigned long long* count_dev, int skip_zero, DevTable dst,
                                int with_index, double eps, DevCtl* ctl, void* scratch,
                                int guarded);

int device_sm_count();
int gate_blocks_per_sm(int W);  // resident gate-kernel blocks per SM

}  // namespace ppk
