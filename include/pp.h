/*
 * pp.h -- C ABI of the GB300 symmetry-merging Pauli propagation library.
 *
 * The library evolves an observable O = sum_s c_s s, s a Pauli string over n
 * qubits, backwards through a circuit of Pauli rotations (the Heisenberg
 * picture of Appendix A), merges strings related by a symmetry group into
 * orbit representatives (Algorithm 1, Eq. O-merging; Algorithms 2 and 3) and
 * returns Tr[rho O_0] for a product state rho.  All per-term work runs in the
 * library's CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 * --------------------------------
 * Pauli strings: W = ceil(n/64) words per mask, qubit q in word q/64, bit
 *   q%64.  x bit set for X and Y, z bit set for Z and Y (the symplectic form
 *   of Appendix E).  Arrays of strings are row-major [m][W].
 * Gates: a gate is exp(-i theta P / 2).  For P anticommuting with Q the
 *   conjugation is U^dag Q U = cos(theta) Q + sin(theta) (i P Q) (App. A,
 *   Prop. 1 proof; the paper writes the angle without the factor 1/2).
 * Orbit representatives: the lowest integer representation of Appendix E
 *   with digits I=0, X=1, Y=2, Z=3 and qubit q carrying weight 4^q.
 * Truncation (Sec. "Numerical examples", coefficient truncation): after every
 *   gate and every merge a term is kept iff |c| >= coeff_eps (when
 *   coeff_eps > 0) and its Pauli weight is <= max_weight (when >= 0).  After
 *   a symmetry merge c is the merged coefficient, the sum over the members of
 *   the orbit (Eq. O-merging), so a representative can survive although each
 *   member alone would not, and the reverse when the members cancel.
 * Errors: every call returns a pp_status; no C++ exception crosses the ABI.
 *   pp_last_error() gives a message for the calling thread's last failure.
 * Threads: a pp_ctx is used by one host thread at a time.
 * Memory: host pointers passed in are read before the call returns and are
 *   never retained.  Device memory of a context is owned by the context and
 *   comes from the library's stream-ordered memory pool (one per device);
 *   pp_destroy returns it to that pool, which keeps it mapped for later
 *   contexts until the process exits.
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PP_OK = 0,
  PP_ERR_ARG = 1,       /* invalid argument (sizes, null pointers, enum values) */
  PP_ERR_OOM = 2,       /* a device allocation failed */
  PP_ERR_CAPACITY = 3,  /* the term table would exceed mem_budget_bytes */
  PP_ERR_SYMMETRY = 4,  /* layer, observable or state does not have the declared symmetry */
  PP_ERR_CUDA = 5,      /* a CUDA runtime call failed */
  PP_ERR_TIMEOUT = 6,   /* a bounded device wait ran out */
  PP_ERR_BUSY = 7,      /* server queue full */
  PP_ERR_REJECTED = 8,  /* job can never fit the server's memory budget */
  PP_ERR_STATE = 9,     /* call not valid in the context's current state */
  PP_ERR_INTERNAL = 10  /* device-side consistency check failed (hash probe bound) */
} pp_status;

/* Symmetry groups (Sec. "Symmetry" and Appendix B of the paper).
 *  PP_SYM_ZN     translations of a ring of n qubits (Algorithm 2);
 *  PP_SYM_SN     all permutations of the n qubits (Algorithm 3);
 *  PP_SYM_DN     translations and reflections of a ring (dihedral group);
 *  PP_SYM_TORUS  translations of an Lx x Ly torus, qubit q = x + Lx y, used as
 *                PP_SYM_TORUS_LX(Lx) = 4 | (Lx << 8); Lx must divide n.
 * Every representative is the lowest-integer member of its orbit
 * (I=0, X=1, Y=2, Z=3, qubit q the digit of weight 4^q).  A `symmetry`
 * argument anywhere in this API takes one of these codes. */
typedef enum {
  PP_SYM_NONE = 0,
  PP_SYM_ZN = 1,
  PP_SYM_SN = 2,
  PP_SYM_DN = 3,
  PP_SYM_TORUS = 4
} pp_symmetry;
#define PP_SYM_TORUS_LX(lx) ((int)PP_SYM_TORUS | ((int)(lx) << 8))
typedef enum { PP_COEF_F64 = 0, PP_COEF_F32 = 1 } pp_coef_type;
typedef enum { PP_NOISE_NONE = 0, PP_NOISE_PER_GATE = 1, PP_NOISE_PER_LAYER = 2 } pp_noise_mode;

/* How identical strings (or representatives) are accumulated by a merge --
 * the "if s~ is in D~ accumulate, else insert" loop of Algorithms 2 and 3:
 *  PP_MERGE_HASH  open-addressing device hash table, atomicCAS on key slots and
 *                 FP64 atomicAdd on coefficients (rounding order not fixed);
 *  PP_MERGE_SORT  LSD radix sort of the representatives and a segmented FP64
 *                 reduce of each run of equal keys in input order: the sums are
 *                 reproducible bit for bit.  Needs n_qubits <= 64; wider
 *                 strings, or a scratch that would not fit the memory budget,
 *                 use the hash table.  Its scratch (about 41 bytes per table
 *                 entry for n <= 32, 57 for n <= 64) stays with the context. */
typedef enum { PP_MERGE_HASH = 0, PP_MERGE_SORT = 1 } pp_merge_method;

/* A Pauli rotation generator P: words [0, W) of x and z are used, the rest
 * must be zero. */
typedef struct {
  uint64_t x[4];
  uint64_t z[4];
} pp_pauli;

typedef struct {
  int n_qubits;            /* 1..256 */
  int symmetry;            /* pp_symmetry: group used by merges and overlaps */
  int batch;               /* B = number of angle sets sharing the circuit, 1..512; every
                              string then carries B coefficients and is kept iff some
                              column satisfies the truncation rule */
  int coef_type;           /* pp_coef_type: storage (and gate arithmetic) precision of the
                              coefficients; merges accumulate and overlaps sum in FP64
                              in both cases */
  double coeff_eps;        /* coefficient truncation threshold; 0 = off */
  int max_weight;          /* Pauli-weight truncation; < 0 = off */
  int noise_mode;          /* pp_noise_mode */
  double noise_p;          /* per-gate: p of (1-p)^k damping; per-layer: gamma of exp(-gamma |Q|) */
  size_t mem_budget_bytes; /* ceiling on the context's device memory; 0 = no ceiling */
  void* cuda_stream;       /* cudaStream_t to run on; NULL = the context creates its own */
  int check_symmetry;      /* nonzero: validate layers against the group (PP_ERR_SYMMETRY) */
  int use_graphs;          /* nonzero: replay repeated layers from captured CUDA graphs */
  int profile_kernels;     /* nonzero: bracket every kernel that applies gates with CUDA
                              events on the context's stream and accumulate their
                              durations into pp_stats_t.gate_kernel_ms */
  int layer_kernel;        /* nonzero (default): all gates of a layer run in one persistent
                              cooperative kernel with a grid barrier between gates; zero:
                              one kernel per gate, replayed from CUDA graphs */
  int merge_method;        /* pp_merge_method of the symmetry and identical-string merges
                              after ingest (ingest itself uses the hash table) */
  int block_threads;       /* threads per block of the persistent layer kernel: 256 (several
                              blocks per SM) or 1024 (one per SM; one-word and two-word
                              strings, single column); 0 = 256 */
  int wait_limit;          /* microseconds a bounded device wait (the grid barrier between
                              gates, a merge waiting for a claimed index slot) may last before
                              it gives up: the kernel records the failure and returns, and the
                              call reports PP_ERR_TIMEOUT; 0 = the default, 30 s (a gate over
                              gigabytes of batched rows takes seconds).  >= 0. */
  double room_factor;      /* headroom a layer asks for before its first gate: room for
                              2 x room_factor x (the previous layer's growth) times the
                              stored terms, and at least twice them; a layer that outgrows
                              it stops part way, grows the table and goes on (pp_stats_t
                              stalls).  0 = the default, 1.25; smaller values trade
                              stalls for memory.  >= 0. */
} pp_config;

typedef struct pp_ctx pp_ctx;

typedef struct {
  int64_t live_terms;      /* terms with a kept coefficient */
  int64_t stored_terms;    /* table entries including truncated slots awaiting compaction */
  int64_t capacity;        /* table capacity in terms */
  double gate_updates;     /* sum over applied gates of the live terms entering the gate */
  int64_t gates_applied;
  int64_t merges;          /* symmetry or identical-string merges performed */
  int64_t compactions;
  int64_t regrows;
  size_t device_bytes;     /* device memory currently held by the context */
  double anticommuting_terms; /* sum over applied gates of live terms anticommuting with P */
  int64_t kernel_launches; /* kernels launched by the context (graph nodes included) */
  double gate_kernel_ms;   /* with profile_kernels: summed duration of the kernels that applied
                              gates (one per layer, or one per gate without layer_kernel) */
  int64_t gate_kernels_timed; /* number of launches summed in gate_kernel_ms */
  double grid_scale;       /* blocks per gate pass relative to the default sizing (pp_tune) */
  double skipped_updates;  /* the part of gate_updates from gates that no stored string could
                              anticommute with (nor, with per-gate noise, overlap): the layer
                              kernel tests them against the OR of all keys and skips the scan */
  int64_t gates_skipped;   /* number of such gates */
  double index_factor;     /* hash index slots per table entry of capacity (pp_tune) */
  int64_t persistent;      /* 1: layers run in one persistent kernel, 0: one kernel per gate */
  int64_t block_threads;   /* threads per block of the kernels that apply gates */
  int64_t stalls;          /* times a layer stopped part way for room, grew the table and went on */
  int64_t index_slots;     /* hash index slots of the active table (a power of two) */
} pp_stats_t;

/* Fill *cfg with defaults: n_qubits = 0 (must be set), no symmetry, batch 1,
 * FP64, truncation off, no noise, no budget, own stream, checks and graphs on. */
pp_status pp_config_default(pp_config* cfg);

/* Create a context holding O = sum_i coef[i] s_i (Algorithm 1, step 1).
 * x, z: host arrays [n_terms][W]; coef: host array [n_terms][batch].  Duplicate
 * strings accumulate.  With cfg->symmetry != PP_SYM_NONE the strings are
 * mapped to their orbit representatives and merged, giving O~_L of Alg. 1.
 * The truncation rules are then applied.  n_terms may be 0.
 * Errors: PP_ERR_ARG (bad config, null pointers with n_terms > 0, string bits
 * beyond n_qubits), PP_ERR_OOM, PP_ERR_CAPACITY, PP_ERR_CUDA. */
pp_status pp_create(const pp_config* cfg, int64_t n_terms, const uint64_t* x,
                    const uint64_t* z, const double* coef, pp_ctx** out);

/* As pp_create, but x, z and coef are device pointers (same layout) that
 * stay owned by the caller and are only read, on the context's stream,
 * before the call returns. */
pp_status pp_create_device(const pp_config* cfg, int64_t n_terms, const uint64_t* x,
                           const uint64_t* z, const double* coef, pp_ctx** out);

/* Replace the operator held by ctx with sum_i coef[i] s_i, for example a
 * table saved with pp_export, to resume a propagation (checkpoint and
 * restart).  Host arrays in pp_create's layout: x, z [n_terms][W],
 * coef [n_terms][batch], only read during the call.  Identical strings
 * accumulate and the truncation rules apply, as at creation.  With a group,
 * strings are folded into their representatives and the operator is taken
 * to be invariant -- the form pp_export returns for such a context.
 * Errors: PP_ERR_ARG (null arrays, n_terms < 0, bits at or above n_qubits),
 * PP_ERR_CAPACITY, PP_ERR_OOM, PP_ERR_CUDA. */
pp_status pp_import(pp_ctx* ctx, int64_t n_terms, const uint64_t* x, const uint64_t* z,
                    const double* coef);

/* Release every device and host resource of ctx.  NULL is accepted. */
pp_status pp_destroy(pp_ctx* ctx);

/* Autotuning (an implementation facility; the paper has no counterpart).
 * Times one application of the layer (gates in time order, theta [n_gates][batch],
 * as for pp_apply_layer, without the boundary merge) on the context's current
 * table and undoes it, for each candidate setting, then keeps the fastest for the
 * context's later layers.  The search is coordinate-wise: first the launch shape
 * (all gates of a layer in one persistent kernel where the device allows it, with
 * blocks of 256 or 1024 threads, or one kernel per gate from CUDA graphs) together
 * with the hash index's load factor
 * (1.5 or 3 index slots per table entry of capacity), then the grid size (0.5, 1, 2
 * or 4 times the default number of blocks).  A candidate whose index would not fit
 * the memory budget is left out.  The choice is visible in pp_stats_t (grid_scale,
 * index_factor, persistent, block_threads; *chosen_scale when not NULL).  The terms and
 * coefficients that later calls produce do not depend on the choice; the order of
 * table entries may (merge sums use FP64 atomics, whose rounding order is never
 * fixed).  An empty table leaves the setting as it is.
 * Errors: as pp_apply_layer (the table is restored). */
pp_status pp_tune(pp_ctx* ctx, int n_gates, const pp_pauli* gates, const double* theta,
                  double* chosen_scale);

/* One Heisenberg layer O_{l-1} = U_l^dag O~_l U_l (Algorithm 1, step 2a, and
 * Appendix A).  gates[0..n_gates) and theta[n_gates][batch] describe U_l in TIME
 * order; they are applied from the last to the first.  Per gate: per-gate
 * damping (noise_mode PER_GATE: c <- c (1-p)^k, k = non-identity sites of Q on
 * the gate's support), conjugation, merge of identical strings, truncation.
 * noise_mode PER_LAYER damps every term by exp(-p |Q|) once before the gates
 * (the noise layer follows U_l in time; batch 1 with FP64 storage only).  With symmetric_boundary != 0 the
 * layer ends with the symmetry merge of Eq. (O-merging) (Algorithm 2 for
 * Z_n, Algorithm 3 for S_n) and another truncation.  Callers apply layers
 * from the last (l = L) to the first (l = 1).
 * The merge is exact (Theorem 1) when the layer's unitary commutes with the
 * group, e.g. a product of commuting sublayers each mapped onto itself; the
 * check below tests the multiset only, so for an ordered product of
 * non-commuting gates the merge holds up to the ordering (Trotter) error.
 * Errors: PP_ERR_ARG; PP_ERR_SYMMETRY when check_symmetry is set and the gate
 * multiset (with angles) is not mapped onto itself by the group generators;
 * PP_ERR_CAPACITY when the table would exceed mem_budget_bytes -- the context
 * is then back at its state before the call (a dense copy of the table,
 * counted against the budget, is taken at the start of every call on a
 * context with a budget), so the caller may raise the budget with
 * pp_set_budget and call again; PP_ERR_OOM, PP_ERR_CUDA, PP_ERR_INTERNAL
 * (after these the context holds a partly applied layer). */
pp_status pp_apply_layer(pp_ctx* ctx, int n_gates, const pp_pauli* gates, const double* theta,
                         int symmetric_boundary);

/* Replace every string by its orbit representative under the context's
 * group (for Z_n the translation with the lowest digit integer, Algorithm 2;
 * for S_n the layout Z^{nZ} Y^{nY} X^{nX} on the lowest qubits, Algorithm 3)
 * without accumulating: the table may then hold duplicates
 * until pp_merge.  Any later call that needs unique strings merges first.
 * Errors: PP_ERR_STATE when the context has no symmetry. */
pp_status pp_canonicalize(pp_ctx* ctx);

/* Accumulate identical strings (the merge step of Algorithms 2 and 3 and of
 * standard PP), then apply the truncation rules.  Coefficient sums use FP64
 * atomics, so their rounding order is not fixed. */
pp_status pp_merge(pp_ctx* ctx);

/* Drop every term with |c| < eps (eps > 0) or weight > max_weight (>= 0).
 * Does not change the rules applied by later calls. */
pp_status pp_truncate(pp_ctx* ctx, double eps, int max_weight);

/* Tr[rho O] (Algorithm 1, step 3) for rho = prod_q (I + bx X + by Y + bz Z)/2,
 * bloch = host array [n][3] of (bx, by, bz).  With a symmetry each
 * representative r contributes c_r times the orbit average of Tr[rho g.r],
 * which equals Tr[rho r] when rho is symmetric (Eq. 2) and keeps the result
 * exact for a symmetric O when rho is not.  The sum is accumulated in FP64
 * in a fixed order.  out receives `batch` doubles (one per angle set).
 * Errors: PP_ERR_SYMMETRY when neither rho nor the ingested O is invariant. */
pp_status pp_expect(pp_ctx* ctx, const double* bloch, double* out);

/* pp_expect for the computational basis state |b_0 ... b_{n-1}> (Alg. 1 step
 * 3 with rho a basis state): bits[q] in {0, 1}; the same as pp_expect with
 * Bloch vectors (0, 0, 1 - 2 b_q).  out: batch doubles.  Same errors as
 * pp_expect. */
pp_status pp_expect_basis(pp_ctx* ctx, const uint8_t* bits, double* out);

/* Number of live terms and of stored table entries. */
pp_status pp_num_terms(pp_ctx* ctx, int64_t* live, int64_t* stored);

/* Copy the live terms to host arrays x, z [capacity][W] and coef
 * [capacity][batch] (FP64); *n_out receives the count.  PP_ERR_ARG if capacity is too
 * small (nothing written; *n_out still receives the count). */
pp_status pp_export(pp_ctx* ctx, int64_t capacity, uint64_t* x, uint64_t* z, double* coef,
                    int64_t* n_out);

/* Counters of the context (host copy, synchronises the stream). */
pp_status pp_stats(pp_ctx* ctx, pp_stats_t* out);

/* Raise or lower the memory budget of a context (0 = no ceiling). */
pp_status pp_set_budget(pp_ctx* ctx, size_t mem_budget_bytes);

/* Limit the context's persistent layer launches (one cooperative launch per
 * layer whose blocks wait for one another at a barrier between gates) to the
 * fraction `fraction` in (0, 1] of the blocks the GPU holds at once (default
 * 1).  Contexts driven from different host threads may apply layers at the
 * same time only if the fractions of those running together add up to at
 * most 1: then every launch fits beside the others.  A launch over a small
 * table uses fewer blocks than its fraction allows.  Takes effect at the
 * context's next layer.  PP_ERR_ARG for a fraction outside (0, 1]. */
pp_status pp_set_grid_fraction(pp_ctx* ctx, double fraction);

/* Wait for all work queued by ctx. */
pp_status pp_synchronize(pp_ctx* ctx);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* pp_last_error(void);

/* Host-side fault injection for tests of failure handling (the paper has no
 * counterpart).  After n further device allocations by any context of this
 * process, the next one fails as if the device were out of memory: the call
 * that needed it returns PP_ERR_OOM.  Table growth that fails this way leaves
 * the context as it was before the call, so it may be used again.  The
 * injection fires once; n < 0 turns it off.  Never touches the GPU. */
pp_status pp_debug_fail_alloc_after(int64_t n);

/* ------------------------------------------------------------------------
 * Stateless entry points on caller-owned device arrays.  Keys are device
 * arrays [m][2W] with the x words of a string followed by its z words.  All
 * work is queued on `stream` (cudaStream_t, NULL = default stream); the call
 * returns once it is queued unless stated otherwise.
 * ------------------------------------------------------------------------ */

/* keys_out[i] = orbit representative of keys_in[i] (Algorithms 2 and 3).
 * keys_out may equal keys_in. */
pp_status pp_canonical_keys(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                            uint64_t* keys_out, void* stream);

/* Accumulate identical strings of (keys_in, coef_in)[0..m) after mapping each
 * to its representative under `symmetry` (PP_SYM_NONE: identity), i.e. the
 * merge loop of Algorithms 2 and 3.  Writes the distinct strings and their
 * FP64 sums to keys_out [m][2W], coef_out [m] in unspecified order and the
 * count to *m_out (host pointer; the call synchronises the stream).  Uses a
 * temporary device hash table obtained with cudaMallocAsync on `stream`. */
pp_status pp_merge_terms(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                         const double* coef_in, uint64_t* keys_out, double* coef_out,
                         int64_t* m_out, void* stream);

/* pp_merge_terms by radix sort and segmented reduce (PP_MERGE_SORT): the
 * distinct strings come out in ascending order of the packed key (x | z << 32
 * for n <= 32, otherwise z then x as a 128-bit integer), and each sum is taken
 * in input order, so the output is the same bit for bit on every call.
 * n_qubits must be at most 64 (PP_ERR_ARG otherwise).  Uses temporary device
 * memory from cudaMallocAsync on `stream` (about 41 or 57 bytes per input
 * term); synchronises the stream. */
pp_status pp_merge_terms_sorted(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                                const double* coef_in, uint64_t* keys_out, double* coef_out,
                                int64_t* m_out, void* stream);

/* *out (device pointer, one double) = sum_i coef[i] ov(keys[i]), ov the
 * product-state overlap of pp_expect (orbit-averaged under `symmetry`),
 * bloch a device array [n][3].  Deterministic two-pass FP64 reduction. */
pp_status pp_overlap_sum(int n_qubits, int symmetry, int64_t m, const uint64_t* keys,
                         const double* coef, const double* bloch, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Serving (continuous batching of independent propagation jobs).  The paper
 * has no counterpart; a job is the Algorithm 1 computation of one request.
 * ------------------------------------------------------------------------ */

typedef struct pp_server pp_server;

/* One request: O (x, z [n_terms][W], coef [n_terms][cfg.batch]), one layer of
 * gates in time order (gates [n_layer_gates], theta [n_layer_gates][batch])
 * applied n_layers times (Trotter steps; pp_apply_layer semantics, with the
 * symmetry merge after each layer when symmetric_boundary != 0), and the
 * product state bloch [n][3].  cfg.cuda_stream and cfg.mem_budget_bytes are
 * set by the server.  mem_bytes: device memory reserved for the job when it
 * is admitted (0 = the server's default, or an estimate from n_terms when the
 * server has none).  The reservation then follows the job: before each layer
 * it is raised to the context's device memory times the growth of its
 * live-term count over the previous layer, and a layer that still runs out of
 * room is applied again (from the state before it) with twice the
 * reservation, up to the server budget.  All arrays are copied by pp_submit. */
typedef struct {
  pp_config cfg;
  int64_t n_terms;
  const uint64_t* x;
  const uint64_t* z;
  const double* coef;
  int n_layer_gates;
  const pp_pauli* gates;
  const double* theta;
  int n_layers;
  int symmetric_boundary;
  const double* bloch;
  size_t mem_bytes;
} pp_job;

typedef struct {
  int done;             /* 0 while queued or running */
  int status;           /* pp_status of the job */
  double value;         /* Tr[rho O_0] (first angle set) */
  int64_t live_terms;
  double gate_updates;
  size_t device_bytes;  /* peak-time device memory of the job's context */
  size_t reserved_bytes;
  double queue_ms;      /* submit -> start */
  double run_ms;        /* start -> finish */
  double latency_ms;    /* submit -> finish */
  char message[160];    /* the failing call's error text when status != PP_OK */
  int grows;            /* times the reservation was raised while the job ran */
  int restarts;         /* times the job gave its memory back and started again (only
                           when every running job was waiting for memory) */
} pp_job_result;

/* A server with `slots` worker threads, each owning a CUDA stream on the
 * calling thread's current device.  Jobs are admitted among those whose
 * reservation fits in mem_budget_bytes minus the reservations of running
 * jobs, in order of predicted run time (a regression of the log run times of
 * finished jobs on the job's layers, gates per layer, threshold, noise, n and
 * group) less one natural-log unit per 10 s waited, so short jobs do not
 * wait behind long ones and every job reaches the front; their kernels
 * overlap on the device.  A running job waiting for a larger reservation is
 * served before any queued job is admitted, and a queued job that jobs after
 * it in that order have passed 8 times is not passed again.
 * default_job_bytes: reservation of jobs that name none; 0 = estimate each
 * from its observable (two tables with room for 4 n_terms strings plus fixed
 * buffers).  Errors: PP_ERR_ARG, PP_ERR_CUDA. */
pp_status pp_server_create(int slots, size_t mem_budget_bytes, size_t default_job_bytes,
                           pp_server** out);

/* Queue a job (thread-safe); *job_id identifies it.  PP_ERR_REJECTED when its
 * reservation can never fit the budget, PP_ERR_ARG for a malformed job. */
pp_status pp_submit(pp_server* server, const pp_job* job, uint64_t* job_id);

/* Result so far (done = 0 while pending); PP_ERR_ARG for an unknown id. */
pp_status pp_server_poll(pp_server* server, uint64_t job_id, pp_job_result* out);

/* Block until the job is done. */
pp_status pp_server_wait(pp_server* server, uint64_t job_id, pp_job_result* out);

/* Queue length, running jobs, completed jobs, reserved bytes (any may be NULL). */
pp_status pp_server_stats(pp_server* server, int64_t* queued, int64_t* running,
                          int64_t* completed, size_t* reserved_bytes);

/* Finish every queued job, then stop the workers and free the server. */
pp_status pp_server_destroy(pp_server* server);

/* pp_merge_terms without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run -- a serving loop whose device memory is sized
 * once at start-up (an allocation later could fail under load, or stall the
 * device while it synchronises), or an application that hands out every
 * device allocation from its own pool.  The result is the same as pp_merge_terms
 * (distinct strings in keys_out, FP64 sums in coef_out, unspecified order),
 * but:
 *  - the count is written to *m_out_dev, a DEVICE pointer owned by the
 *    caller (-1 if a device-side check failed), and the call returns as soon
 *    as the work is queued on `stream` (nothing is synchronised);
 *  - the hash index and control block live in one static device array of
 *    about 8 MiB that the library keeps on every device where it is used
 *    until the process exits, so m is limited to 524288 terms (PP_ERR_ARG
 *    with a message beyond that);
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address belongs to the device's context
 *    as it was then: no call may follow a cudaDeviceReset of that device in
 *    the same process;
 *  - all calls on a device share the array: calls whose work overlaps on
 *    the device race and must be serialised by the caller.  Each call clears
 *    what it uses before using it.
 * No cudaMalloc, cudaMallocAsync, cudaFree or allocating library routine is
 * called. */
pp_status pp_merge_terms_noalloc(int n_qubits, int symmetry, int64_t m, const uint64_t* keys_in,
                                 const double* coef_in, uint64_t* keys_out, double* coef_out,
                                 int64_t* m_out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
