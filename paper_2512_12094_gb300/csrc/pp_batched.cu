// Batched propagation: one circuit, B angle sets.  Every string carries a row
// of B coefficients (float or double); the pair structure of a gate depends
// on the keys only, so the key work (anticommutation test, partner lookup,
// ownership) is done once per string and a warp then streams the B columns of
// the pair with coalesced row loads and stores.  A string is kept iff some
// column has |c| >= eps (a dead row reads as zeros).  Merge accumulation and
// overlap sums are FP64 whatever the storage type.
#include "pp_device.cuh"

namespace ppk {
namespace {

constexpr unsigned kAll = 0xFFFFFFFFu;
constexpr int kMaxBOverlap = 512;

// Arithmetic without FMA contraction, per storage type.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float flip(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ (neg ? (int)0x80000000u : 0));
}
__device__ __forceinline__ double flip(double v, bool neg) { return with_sign(v, neg); }

// |v| >= eps on bit patterns (eps_bits = bits of eps in the storage type).
__device__ __forceinline__ bool big(float v, uint64_t eb) {
  return (__float_as_uint(v) & 0x7FFFFFFFu) >= (uint32_t)eb;
}
__device__ __forceinline__ bool big(double v, uint64_t eb) { return (dbits(v) & kAbsMask) >= eb; }

template <typename T>
__device__ __forceinline__ uint64_t eps_bits_of(double eps) {
  if (sizeof(T) == 4) return (uint64_t)__float_as_uint((float)eps);
  return dbits(eps);
}

template <typename T>
__device__ __forceinline__ T ld_row(const T* p) {
  return __ldcg(p);
}

template <int W>
__device__ __forceinline__ Key<W> shfl_key(const Key<W>& k, int src) {
  Key<W> r;
#pragma unroll
  for (int j = 0; j < 2 * W; ++j) r.w[j] = __shfl_sync(kAll, k.w[j], src);
  return r;
}

// ------------------------------------------------------------ gate pass

// One pair action of a batched gate: what a string's thread decided from the
// keys, handed to whichever warp of the block streams the rows.
template <int W>
struct RowAction {
  Key<W> R;        // the partner key (births)
  uint32_t ii;     // the string's row
  int32_t jj;      // the partner's row, -1 when absent
  uint8_t act;     // 1 damp only, 2 owned pair, 3 birth of the partner, 4 rotate only
  uint8_t kq, kr;  // non-identity letters on the gate's support (damping)
  uint8_t flags;   // 1 string alive, 2 partner alive, 4 i P Q = -R
};

// Shared memory of one batched gate pass.
template <int W, typename T>
struct BatchedShared {
  long long delta[kBlock / 32];
  unsigned long long ac[kBlock / 32];
  unsigned wcnt[kBlock / 32];
  unsigned err;
  T cs[2 * 512];  // this gate's cos[0, B), sin[B, 2B) (B <= 512)
  RowAction<W> queue[kBlock];
};

// Columns a lane streams at once: each lane holds kColU columns of each row in
// registers, so the loads of a whole 256-column FP64 row pair are in flight
// together instead of one column at a time.
constexpr int kColU = 8;

// One gate over the rows [0, T0) by one block.  The block takes its equal
// share of [0, T0), kBlock strings at a time; every thread decides its string's action
// from the keys, the actions are compacted into a shared queue, and the
// block's warps take them in turn, each streaming the rows of one action with
// coalesced loads and stores.  So a chunk with many actions keeps every warp
// busy.  Births go to T0 + atomicAdd(cnt_slot); the block's live-count change
// goes to *dlt_slot and its anticommuting count to ctl->ac_total.  Every
// thread of the block must call this; it ends with the block synchronised.
template <int W, typename T>
__device__ __forceinline__ void gate_pass_batched(const DevTable& t, DevCtl* ctl, const GateArgs& g,
                                                  uint64_t T0, unsigned long long* cnt_slot,
                                                  long long* dlt_slot, BatchedShared<W, T>& sh) {
  constexpr int kWarps = kBlock / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = t.B;
  T* rows = static_cast<T*>(t.rows);
  const T* cs = sh.cs;
  const bool noise = g.damp != nullptr;
  const bool use_eps = g.use_eps != 0;
  const uint64_t eb = use_eps ? eps_bits_of<T>(g.eps) : 0ull;
  long long delta = 0;
  unsigned long long n_ac = 0;
  unsigned err = 0;
  // block b takes [T0 b / G, T0 (b+1) / G) in chunks of kBlock strings, so
  // every block of the grid has strings (and row actions) even when the table
  // is smaller than the grid times kBlock; the chunk count is block-uniform
  const uint64_t G = gridDim.x;
  const uint64_t r0 = T0 * blockIdx.x / G, r1 = T0 * (blockIdx.x + 1) / G;
  for (uint64_t cbase = r0; cbase < r1; cbase += kBlock) {
    const uint64_t i = cbase + threadIdx.x;
    int act = 0, kq = 0, kr = 0;
    int64_t jr = -1;
    bool aliveQ = false, aliveR = false, neg = false;
    Key<W> R;
    if (i < r1) {
      const Key<W> Q = ld_key_cg<W>(t.keys, i);
      aliveQ = __ldcg(t.alive + i) != 0;
      int acnt = 0;
#pragma unroll
      for (int j = 0; j < W; ++j) {
        acnt += __popcll(g.px[j] & Q.z(j)) + __popcll(g.pz[j] & Q.x(j));
        if (noise) kq += __popcll((Q.x(j) | Q.z(j)) & g.supp[j]);
      }
      if ((acnt & 1) == 0) {
        if (noise && kq && aliveQ) act = 1;
      } else {
        uint64_t pw = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          R.x(j) = Q.x(j) ^ g.px[j];
          R.z(j) = Q.z(j) ^ g.pz[j];
          pw |= (Q.x(j) & g.pvx[j]) | (Q.z(j) & g.pvz[j]);
        }
        // ownership by the pivot bit, as in the single-column kernel
        if (aliveQ || pw == 0) {
          const uint64_t h = key_hash(R);
          jr = index_find_old<W>(t, R, h, tag_of(h), T0, err);
          if (jr == -2) note_first(ctl, 5u, g.gate_id, (unsigned)T0, (unsigned)t.imask);
        }
        neg = sigma_of<W>(g, Q) < 0;
        // live anticommuting rows from values before the gate: the owner
        // counts a stored pair, anyone else only itself (as in the FP64 kernel)
        if (jr < 0) n_ac += aliveQ;
        if (jr >= 0) {
          if (pw == 0) {
            aliveR = __ldcg(t.alive + jr) != 0;
            n_ac += (unsigned long long)aliveQ + (unsigned long long)aliveR;
            if (aliveQ || aliveR) {
              act = 2;
              if (noise) {
#pragma unroll
                for (int j = 0; j < W; ++j) kr += __popcll((R.x(j) | R.z(j)) & g.supp[j]);
              }
            }
          }
        } else if (jr == -1 && aliveQ) {
          act = (g.wmax < 0 || weight(R) <= g.wmax) ? 3 : 4;
        }
      }
    }
    // compact the block's actions into the queue, in string order
    const unsigned bal = __ballot_sync(kAll, act != 0);
    if (lane == 0) sh.wcnt[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, n_queue = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      before += (w < warp) ? sh.wcnt[w] : 0u;
      n_queue += sh.wcnt[w];
    }
    if (act) {
      RowAction<W>& a = sh.queue[before + __popc(bal & ((1u << lane) - 1u))];
      a.R = R;
      a.ii = (uint32_t)i;
      a.jj = (int32_t)jr;
      a.act = (uint8_t)act;
      a.kq = (uint8_t)kq;
      a.kr = (uint8_t)kr;
      a.flags = (uint8_t)((aliveQ ? 1 : 0) | (aliveR ? 2 : 0) | (neg ? 4 : 0));
    }
    __syncthreads();
    for (unsigned q = warp; q < n_queue; q += kWarps) {
      const RowAction<W>& A = sh.queue[q];
      const int a = A.act;
      const uint64_t ii = A.ii;
      const long long jj = A.jj;
      const bool aQ = (A.flags & 1) != 0, aR = (A.flags & 2) != 0, ng = (A.flags & 4) != 0;
      const int kqq = A.kq, krr = A.kr;
      const T fq = kqq ? (T)g.damp[kqq] : (T)1, fr = krr ? (T)g.damp[krr] : (T)1;
      T* rq = rows + ii * B;
      bool anyQ = false, anyR = false;
      if (a == 1) {
        for (int c0 = 0; c0 < B; c0 += 32 * kColU) {
          T v[kColU];
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            v[u] = col < B ? ld_row(rq + col) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            if (col < B) {
              const T d = mul_rn(v[u], fq);
              rq[col] = d;
              anyQ |= big(d, eb);
            }
          }
        }
      } else if (a == 2) {
        T* rr = rows + (uint64_t)jj * B;
        for (int c0 = 0; c0 < B; c0 += 32 * kColU) {
          T vq[kColU], vr[kColU];
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            vq[u] = (col < B && aQ) ? ld_row(rq + col) : (T)0;
            vr[u] = (col < B && aR) ? ld_row(rr + col) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            if (col < B) {
              T dq = vq[u], dr = vr[u];
              if (kqq) dq = mul_rn(dq, fq);
              if (krr) dr = mul_rn(dr, fr);
              const T c = cs[col], sn = cs[B + col];
              const T sQ = mul_rn(sn, dq), sR = mul_rn(sn, dr);
              const T nq = add_rn(mul_rn(c, dq), flip(sR, !ng));
              const T nr = add_rn(mul_rn(c, dr), flip(sQ, ng));
              rq[col] = nq;
              rr[col] = nr;
              anyQ |= big(nq, eb);
              anyR |= big(nr, eb);
            }
          }
        }
      } else {
        // first pass: which of Q's new row and the child row survive
        for (int c0 = 0; c0 < B; c0 += 32 * kColU) {
          T v[kColU];
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            v[u] = col < B ? ld_row(rq + col) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            if (col < B) {
              T dq = v[u];
              if (kqq) dq = mul_rn(dq, fq);
              anyQ |= big(mul_rn(cs[col], dq), eb);
              if (a == 3) anyR |= big(mul_rn(cs[B + col], dq), eb);
            }
          }
        }
      }
      anyQ = __any_sync(kAll, anyQ) || !use_eps;
      anyR = __any_sync(kAll, anyR) || !use_eps;
      if (a >= 3) {
        const bool birth = (a == 3) && anyR;
        unsigned long long idx = 0;
        if (birth) {
          if (lane == 0) idx = T0 + atomicAdd(cnt_slot, 1ull);
          idx = __shfl_sync(kAll, idx, 0);
          if (idx >= t.cap) {
            err |= kErrAppend;
            if (lane == 0) note_first(ctl, 4u, g.gate_id, (unsigned)idx, (unsigned)t.cap);
          }
        }
        const bool write_child = birth && idx < t.cap;
        T* rn = rows + idx * B;
        for (int c0 = 0; c0 < B; c0 += 32 * kColU) {
          T v[kColU];
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            v[u] = col < B ? ld_row(rq + col) : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kColU; ++u) {
            const int col = c0 + 32 * u + lane;
            if (col < B) {
              T dq = v[u];
              if (kqq) dq = mul_rn(dq, fq);
              rq[col] = mul_rn(cs[col], dq);
              if (write_child) rn[col] = flip(mul_rn(cs[B + col], dq), ng);
            }
          }
        }
        if (lane == 0) {
          t.alive[ii] = anyQ ? 1 : 0;
          delta += (long long)anyQ - 1;
          if (write_child) {
            const Key<W> Rs = A.R;
            st_key<W>(t.keys, idx, Rs);
            t.alive[idx] = 1;
            const uint64_t h = key_hash(Rs);
            const unsigned e0 = err;
            index_claim(t, h & t.imask, ((uint64_t)tag_of(h) << 32) | idx, err);
            if (err != e0) note_first(ctl, 5u, g.gate_id, (unsigned)T0, (unsigned)t.imask);
            delta += 1;
          }
        }
      } else if (lane == 0) {
        if (a == 1) {
          t.alive[ii] = anyQ ? 1 : 0;
          delta += (long long)anyQ - 1;
        } else {
          t.alive[ii] = anyQ ? 1 : 0;
          t.alive[jj] = anyR ? 1 : 0;
          delta += (long long)anyQ - (long long)aQ + (long long)anyR - (long long)aR;
        }
      }
    }
    __syncthreads();  // the queue is rewritten by the next chunk
  }
  delta = warp_sum(delta);
  n_ac = warp_sum(n_ac);
  if (lane == 0) {
    sh.delta[warp] = delta;
    sh.ac[warp] = n_ac;
  }
  if (err) atomicOr(&sh.err, err);
  __syncthreads();
  if (threadIdx.x == 0) {
    long long d = 0;
    unsigned long long ac = 0;
    for (int w = 0; w < kWarps; ++w) {
      d += sh.delta[w];
      ac += sh.ac[w];
    }
    if (d) atomicAdd(reinterpret_cast<unsigned long long*>(dlt_slot), (unsigned long long)d);
    if (ac) atomicAdd(&ctl->ac_total, ac);
    if (sh.err) {
      atomicOr(&ctl->error, sh.err);
      atomicOr(&ctl->gerr[cnt_slot - ctl->cnt], sh.err);
    }
    sh.err = 0;
  }
  __syncthreads();
}

template <int W, typename T>
__device__ __forceinline__ void stage_columns(BatchedShared<W, T>& sh, const GateArgs& g, int B) {
  for (int k = threadIdx.x; k < 2 * B; k += kBlock) sh.cs[k] = static_cast<const T*>(g.csb)[k];
}

// One kernel per gate (the graph / PDL path), with the slot protocol of the
// single-column gate_kernel.
template <int W, typename T>
__global__ void __launch_bounds__(kBlock) gate_batched_kernel(const DevTable* __restrict__ tabp,
                                                              DevCtl* __restrict__ ctl,
                                                              GateArgs g) {
  __shared__ BatchedShared<W, T> sh;
  const unsigned gid = g.gate_id;
  const int slot = (int)(gid % 3u), prev = (int)((gid + 2u) % 3u), next = (int)((gid + 1u) % 3u);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const DevTable t = *tabp;
  const unsigned long long T0 = __ldcg(&ctl->base[prev]) + __ldcg(&ctl->cnt[prev]);
  const long long L0 = __ldcg(&ctl->live_base[prev]) + __ldcg(&ctl->dlt[prev]);
  bool run = (gid >= __ldcg(&ctl->first_gate)) && (__ldcg(&ctl->stall) == 0u) &&
             (__ldcg(&ctl->error) == 0u);
  const bool room = gate_fits(t, T0);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0 && run && !room) ctl->stall = gid + 1;
    if (blockIdx.x == 0 && run && room) {
      ctl->base[slot] = T0;
      ctl->live_base[slot] = L0;
      ctl->cnt[next] = 0;
      ctl->dlt[next] = 0;
      ctl->gerr[next] = 0;
      atomicAdd(&ctl->updates, (double)L0);
      atomicAdd(&ctl->gates_done, 1ull);
#pragma unroll
      for (int j = 0; j < W; ++j) {
        if (g.px[j]) atomicOr(&ctl->occ[j], (unsigned long long)g.px[j]);
        if (g.pz[j]) atomicOr(&ctl->occ[kMaxW + j], (unsigned long long)g.pz[j]);
      }
    }
    sh.err = 0;
  }
  if (!(run && room)) {
    asm volatile("griddepcontrol.launch_dependents;");
    return;
  }
  stage_columns<W, T>(sh, g, t.B);
  __syncthreads();
  gate_pass_batched<W, T>(t, ctl, g, T0, &ctl->cnt[slot], &ctl->dlt[slot], sh);
  asm volatile("griddepcontrol.launch_dependents;");
}

__device__ __forceinline__ unsigned ld_acquire_u32b(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of the cooperative batched layer kernel (the same protocol as
// the single-column layer kernel: a counter that only grows, release /
// acquire, bounded wait).
__device__ __forceinline__ bool grid_sync_b(DevCtl* ctl, unsigned& target, int& s_ok,
                                            unsigned limit, unsigned gate) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&ctl->bar_root), "r"(1u)
                 : "memory");
    const unsigned long long deadline = wait_deadline(limit);
    unsigned seen;
    while ((int)((seen = ld_acquire_u32b(&ctl->bar_root)) - target) < 0) {
      if (global_ns() > deadline) {
        ok = 0;
        note_timeout(ctl, 2u, gate, seen, target);
        break;
      }
      __nanosleep(16);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// All gates of a batched layer in one cooperative launch, organised like the
// single-column layer_kernel: the table size travels in registers, gates are
// separated by a grid barrier, gates that no stored string can touch are
// skipped by the occupancy test, and executed gates take the counter slots
// by their ordinal.  On leaving, block 0 records the state in the exit
// record, which chain_finish reads.
template <int W, typename T>
__global__ void __launch_bounds__(kBlock, W == 1 ? 3 : 2)
    layer_batched_kernel(const DevTable* __restrict__ tabp, DevCtl* __restrict__ ctl,
                         const GateArgs* __restrict__ gates, unsigned n_gates) {
  __shared__ BatchedShared<W, T> sh;
  __shared__ GateArgs s_gate;
  __shared__ int s_ok;
  const DevTable t = *tabp;
  const unsigned first = __ldcg(&ctl->first_gate);
  const int q0 = (int)((first + 2u) % 3u);
  unsigned long long T0 = __ldcg(&ctl->base[q0]) + __ldcg(&ctl->cnt[q0]);
  long long L0 = __ldcg(&ctl->live_base[q0]) + __ldcg(&ctl->dlt[q0]);
  uint64_t ox[W], oz[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    ox[j] = __ldcg(&ctl->occ[j]);
    oz[j] = __ldcg(&ctl->occ[kMaxW + j]);
  }
  unsigned target = 0;
  const unsigned wlimit = wait_limit_of(ctl);
  if (threadIdx.x == 0) sh.err = 0;
  if (__ldcg(&ctl->entry_stop) != 0u) return;  // written before the launch: uniform
  unsigned e = 0;
  unsigned end = n_gates;
  for (unsigned gid = first; gid < n_gates; ++gid) {
    __syncthreads();  // the previous gate's readers of s_gate and sh.cs are done
    {
      const unsigned* src = reinterpret_cast<const unsigned*>(gates + gid);
      unsigned* dst = reinterpret_cast<unsigned*>(&s_gate);
      for (unsigned k = threadIdx.x; k < sizeof(GateArgs) / 4; k += kBlock) dst[k] = __ldg(src + k);
    }
    __syncthreads();
    const GateArgs& g = s_gate;
    uint64_t touch = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      touch |= (g.px[j] & oz[j]) | (g.pz[j] & ox[j]);
      if (g.damp) touch |= g.supp[j] & (ox[j] | oz[j]);
    }
    if (touch == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&ctl->updates, (double)L0);
        atomicAdd(&ctl->gates_done, 1ull);
        atomicAdd(&ctl->skipped_updates, (double)L0);
        atomicAdd(&ctl->gates_skipped, 1ull);
      }
      continue;
    }
    if (!gate_fits(t, T0)) {  // the same decision in every block
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->stall = gid + 1;
      end = gid;
      break;
    }
    const int slot = (int)(e % 3u), next = (int)((e + 1u) % 3u);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->cnt[next] = 0;
      ctl->dlt[next] = 0;
      ctl->gerr[next] = 0;
      atomicAdd(&ctl->updates, (double)L0);
      atomicAdd(&ctl->gates_done, 1ull);
    }
    stage_columns<W, T>(sh, g, t.B);
    __syncthreads();
    gate_pass_batched<W, T>(t, ctl, g, T0, &ctl->cnt[slot], &ctl->dlt[slot], sh);
#pragma unroll
    for (int j = 0; j < W; ++j) {
      ox[j] |= g.px[j];
      oz[j] |= g.pz[j];
    }
    if (gridDim.x == 1) {
      __threadfence();
      __syncthreads();
    } else if (!grid_sync_b(ctl, target, s_ok, wlimit, gid)) {
      return;
    }
    T0 += __ldcg(&ctl->cnt[slot]);
    L0 += __ldcg(&ctl->dlt[slot]);
    ++e;
    if (__ldcg(&ctl->gerr[slot]) != 0u) return;  // written by this gate only: uniform
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->exit_terms = T0;
    ctl->exit_live = L0;
    ctl->exit_set = 1u;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      ctl->occ[j] = ox[j];
      ctl->occ[kMaxW + j] = oz[j];
    }
  }
}

// --------------------------------------------------------- merge / insert

// One warp per source string: lane 0 maps the key to its representative and
// finds or claims its slot (same protocol as the single-column merge); the
// warp then adds the row into the FP64 accumulator row of that slot.
template <int W, int G, typename S>
__global__ void __launch_bounds__(kBlock)
    merge_batched_kernel(const uint64_t* __restrict__ src_keys, const S* __restrict__ src_rows,
                         const unsigned char* __restrict__ src_alive, uint64_t count, int wmax,
                         int n, int lx, DevTable dst, double* acc, DevCtl* ctl) {
  constexpr int kWarps = kBlock / 32;
  const int lane = threadIdx.x & 31;
  const int B = dst.B;
  const unsigned wlimit = wait_limit_of(ctl);
  unsigned err = 0;
  OccAcc<W> occ;
  unsigned long long* index = reinterpret_cast<unsigned long long*>(dst.index);
  const uint64_t wstride = (uint64_t)gridDim.x * kWarps;
  for (uint64_t e = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); e < count; e += wstride) {
    long long idx = -1;
    if (lane == 0 && (!src_alive || src_alive[e])) {
      Key<W> K = ld_key<W>(src_keys, e);
      if (wmax < 0 || weight(K) <= wmax) {
        canon<W, G>(K, n, lx);
        occ.add(K);
        const uint64_t h = key_hash(K);
        const uint32_t tag = tag_of(h);
        uint64_t pos = h & dst.imask;
        for (uint64_t probe = 0; probe <= dst.imask && idx < 0; ++probe) {
          unsigned long long sv = __ldcg(index + pos);
          if (sv == 0ull) {
            const unsigned long long mine = ((unsigned long long)tag << 32) | kPendingIdx;
            const unsigned long long old = atomicCAS(index + pos, 0ull, mine);
            if (old == 0ull) {
              const unsigned long long k = atomicAdd(&ctl->n_next, 1ull);
              if (k >= dst.cap) {
                err |= kErrAppend;
                break;
              }
              st_key<W>(dst.keys, k, K);
              __threadfence();
              atomicExch(index + pos, ((unsigned long long)tag << 32) | k);
              idx = (long long)k;
              break;
            }
            sv = old;
          }
          if ((uint32_t)(sv >> 32) == tag) {
            // read the slot again with acquire semantics before using its position
            sv = ld_acquire_u64(index + pos);
            if ((uint32_t)sv == kPendingIdx) {
              const unsigned long long deadline = wait_deadline(wlimit);
              while ((uint32_t)sv == kPendingIdx && global_ns() <= deadline) {
                __nanosleep(64);
                sv = ld_acquire_u64(index + pos);
              }
            }
            if ((uint32_t)sv == kPendingIdx) {
              note_timeout(ctl, 3u, 0u, (unsigned)pos, 0u);
              break;
            }
            if (keys_equal(ld_key_cg<W>(dst.keys, (uint32_t)sv), K)) {
              idx = (long long)(uint32_t)sv;
              break;
            }
          }
          pos = (pos + 1) & dst.imask;
        }
      }
    }
    idx = __shfl_sync(kAll, idx, 0);
    if (idx >= 0) {
      const S* sr = src_rows + e * B;
      double* ar = acc + (uint64_t)idx * B;
      for (int col = lane; col < B; col += 32) atomicAdd(ar + col, (double)sr[col]);
    }
  }
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
    finalize_batched_kernel(DevTable dst, const double* __restrict__ acc, DevCtl* ctl, double eps) {
  constexpr int kWarps = kBlock / 32;
  const int lane = threadIdx.x & 31;
  const int B = dst.B;
  T* rows = static_cast<T*>(dst.rows);
  const uint64_t n = *reinterpret_cast<volatile unsigned long long*>(&ctl->n_next);
  const bool use_eps = eps > 0.0;
  const uint64_t eb = use_eps ? eps_bits_of<T>(eps) : 0ull;
  long long live = 0;
  const uint64_t wstride = (uint64_t)gridDim.x * kWarps;
  for (uint64_t e = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); e < n; e += wstride) {
    bool any = false;
    for (int col = lane; col < B; col += 32) {
      const T v = (T)acc[e * B + col];
      rows[e * B + col] = v;
      any |= big(v, eb);
    }
    any = __any_sync(kAll, any) || !use_eps;
    if (lane == 0) {
      dst.alive[e] = any ? 1 : 0;
      live += any;
    }
  }
  if (lane == 0 && live) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live),
                                   (unsigned long long)live);
}

// Kept strings of src (alive, and with extra_eps > 0 some column >= extra_eps,
// weight <= extra_wmax when >= 0) -> dst, one warp-level atomic per 32.
template <int W, typename T>
__global__ void __launch_bounds__(kBlock)
    compact_batched_kernel(DevTable src, uint64_t count, DevTable dst, int with_index,
                           double extra_eps, int extra_wmax, DevCtl* ctl) {
  constexpr int kWarps = kBlock / 32;
  const int lane = threadIdx.x & 31;
  const int B = src.B;
  const T* srows = static_cast<const T*>(src.rows);
  T* drows = static_cast<T*>(dst.rows);
  const uint64_t xb = extra_eps > 0.0 ? eps_bits_of<T>(extra_eps) : 0ull;
  unsigned err = 0;
  long long live = 0;
  OccAcc<W> occ;
  const uint64_t wstride = (uint64_t)gridDim.x * kWarps * 32;
  for (uint64_t base = ((uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)) * 32; base < count;
       base += wstride) {
    const uint64_t i = base + lane;
    bool keep = false;
    if (i < count && src.alive[i]) {
      keep = extra_wmax < 0 || weight(ld_key<W>(src.keys, i)) <= extra_wmax;
    }
    if (extra_eps > 0.0) {  // any-column rule at the extra threshold, row by row
      unsigned cand = __ballot_sync(kAll, keep);
      while (cand) {
        const int sl = __ffs(cand) - 1;
        cand &= cand - 1;
        const uint64_t e = base + sl;
        bool any = false;
        for (int col = lane; col < B; col += 32) any |= big(srows[e * B + col], xb);
        any = __any_sync(kAll, any);
        if (lane == sl) keep = any;
      }
    }
    const unsigned ballot = __ballot_sync(kAll, keep);
    if (!ballot) continue;
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(&ctl->n_next, (unsigned long long)__popc(ballot));
    b0 = __shfl_sync(kAll, b0, 0);
    unsigned rest = ballot;
    while (rest) {
      const int sl = __ffs(rest) - 1;
      const uint64_t e = base + sl;
      const uint64_t k = b0 + __popc(ballot & ((1u << sl) - 1u));
      rest &= rest - 1;
      if (k >= dst.cap) {
        err |= kErrAppend;
        continue;
      }
      for (int col = lane; col < B; col += 32) drows[k * B + col] = srows[e * B + col];
      if (lane == 0) {
        const Key<W> K = ld_key<W>(src.keys, e);
        st_key<W>(dst.keys, k, K);
        occ.add(K);
        dst.alive[k] = 1;
        ++live;
        if (with_index) {
          const uint64_t h = key_hash(K);
          index_claim(dst, h & dst.imask, ((uint64_t)tag_of(h) << 32) | k, err);
        }
      }
    }
  }
  if (lane == 0 && live) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live),
                                   (unsigned long long)live);
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

// Per-column overlap sums: warp w of a block accumulates column c of the live
// rows it visits in s_acc[w][c]; blocks write [grid][B] partials.
template <int W, typename T>
__global__ void __launch_bounds__(kBlock)
    overlap_batched_kernel(DevTable t, uint64_t count, OverlapArgs a, double* partials) {
  constexpr int kWarps = kBlock / 32;
  __shared__ double s_acc[kWarps][kMaxBOverlap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = t.B;
  const T* rows = static_cast<const T*>(t.rows);
  for (int col = lane; col < B; col += 32) s_acc[warp][col] = 0.0;
  const uint64_t wstride = (uint64_t)gridDim.x * kWarps;
  for (uint64_t e = (uint64_t)blockIdx.x * kWarps + warp; e < count; e += wstride) {
    if (!t.alive[e]) continue;  // warp-uniform
    double ov = 0.0;
    if (lane == 0) {
      const Key<W> k = ld_key<W>(t.keys, e);
      ov = a.group == 1   ? overlap_zn<W>(k, a)
           : a.group == 2 ? overlap_sn<W>(k, a)
           : (a.group == 3 || a.group == 4) ? overlap_group<W>(k, a)
                                             : overlap_plain<W>(k, a);
    }
    ov = __shfl_sync(kAll, ov, 0);
    if (ov != 0.0)
      for (int col = lane; col < B; col += 32) s_acc[warp][col] += (double)rows[e * B + col] * ov;
  }
  __syncthreads();
  for (int col = threadIdx.x; col < B; col += kBlock) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += s_acc[w][col];
    partials[(uint64_t)blockIdx.x * B + col] = s;
  }
}

__global__ void reduce_columns_kernel(const double* partials, int grid, int B, double* out) {
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < B; col += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < grid; ++b) s += partials[(uint64_t)b * B + col];
    out[col] = s;
  }
}

template <typename T>
__global__ void rows_to_double_kernel(const T* rows, uint64_t n, double* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (double)rows[i];
}

}  // namespace

// ---------------------------------------------------------------- launchers

#define PPB_W(W, ...)                                        \
  switch (W) {                                               \
    case 1: { constexpr int WW = 1; __VA_ARGS__; break; }    \
    case 2: { constexpr int WW = 2; __VA_ARGS__; break; }    \
    case 3: { constexpr int WW = 3; __VA_ARGS__; break; }    \
    case 4: { constexpr int WW = 4; __VA_ARGS__; break; }    \
    default: return cudaErrorInvalidValue;                   \
  }

template <int W, typename T>
static cudaError_t launch_gate_batched_w(int grid, cudaStream_t s, const DevTable* tab,
                                         DevCtl* ctl, const GateArgs& g, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, gate_batched_kernel<W, T>, tab, ctl, g);
}

template <int W, typename T>
static cudaError_t launch_layer_batched_w(int grid, cudaStream_t s, const DevTable* tab,
                                          DevCtl* ctl, const GateArgs* gates, unsigned n_gates) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, layer_batched_kernel<W, T>, tab, ctl, gates, n_gates);
}

cudaError_t launch_layer_batched(int W, int f32, int grid, cudaStream_t s, const DevTable* tab,
                                 DevCtl* ctl, const GateArgs* gates, unsigned n_gates) {
  if (f32) {
    PPB_W(W, return (launch_layer_batched_w<WW, float>(grid, s, tab, ctl, gates, n_gates)));
  } else {
    PPB_W(W, return (launch_layer_batched_w<WW, double>(grid, s, tab, ctl, gates, n_gates)));
  }
  return cudaErrorInvalidValue;
}

int layer_batched_blocks_per_sm(int W, int f32) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
#define PPB_OCC(WW)                                                                         \
  e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, layer_batched_kernel<WW, float>, \
                                                          kBlock, 0)                          \
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, layer_batched_kernel<WW, double>, \
                                                          kBlock, 0)
  switch (W) {
    case 1: PPB_OCC(1); break;
    case 2: PPB_OCC(2); break;
    case 3: PPB_OCC(3); break;
    case 4: PPB_OCC(4); break;
  }
#undef PPB_OCC
  return (e == cudaSuccess && nb > 0) ? nb : 0;
}

cudaError_t launch_gate_batched(int W, int f32, int grid, cudaStream_t s, const DevTable* tab,
                                DevCtl* ctl, const GateArgs& g, bool pdl) {
  if (f32) {
    PPB_W(W, return (launch_gate_batched_w<WW, float>(grid, s, tab, ctl, g, pdl)));
  } else {
    PPB_W(W, return (launch_gate_batched_w<WW, double>(grid, s, tab, ctl, g, pdl)));
  }
  return cudaErrorInvalidValue;
}

template <int W, int G>
static cudaError_t merge_b_g(int n, int lx, int wmax, int src_f32, int grid, cudaStream_t s,
                             const uint64_t* src_keys, const void* src_rows,
                             const unsigned char* src_alive, uint64_t count, DevTable dst,
                             double* acc, DevCtl* ctl) {
  if (src_f32)
    merge_batched_kernel<W, G, float><<<grid, kBlock, 0, s>>>(
        src_keys, static_cast<const float*>(src_rows), src_alive, count, wmax, n, lx, dst, acc, ctl);
  else
    merge_batched_kernel<W, G, double><<<grid, kBlock, 0, s>>>(
        src_keys, static_cast<const double*>(src_rows), src_alive, count, wmax, n, lx, dst, acc, ctl);
  return cudaGetLastError();
}

cudaError_t launch_merge_batched(int W, int group, int n, int wmax, int src_f32, int grid,
                                 cudaStream_t s, const uint64_t* src_keys, const void* src_rows,
                                 const unsigned char* src_alive, uint64_t count, DevTable dst,
                                 double* acc, DevCtl* ctl) {
  const int lx = group >> 8;  // group code: kind | (torus width << 8)
#define PPB_G(GG)                                                                          \
  PPB_W(W, return (merge_b_g<WW, GG>(n, lx, wmax, src_f32, grid, s, src_keys, src_rows,   \
                                     src_alive, count, dst, acc, ctl)))
  switch (group & 0xFF) {
    case 0: PPB_G(0);
    case 1: PPB_G(1);
    case 2: PPB_G(2);
    case 3: PPB_G(3);
    case 4: PPB_G(4);
    default:
      return cudaErrorInvalidValue;
  }
#undef PPB_G
}

cudaError_t launch_finalize_batched(int grid, cudaStream_t s, DevTable dst, const double* acc,
                                    DevCtl* ctl, double eps) {
  if (dst.f32)
    finalize_batched_kernel<float><<<grid, kBlock, 0, s>>>(dst, acc, ctl, eps);
  else
    finalize_batched_kernel<double><<<grid, kBlock, 0, s>>>(dst, acc, ctl, eps);
  return cudaGetLastError();
}

cudaError_t launch_compact_batched(int W, int grid, cudaStream_t s, DevTable src, uint64_t count,
                                   DevTable dst, int with_index, double extra_eps,
                                   int extra_wmax, DevCtl* ctl) {
  if (src.f32) {
    PPB_W(W, (compact_batched_kernel<WW, float><<<grid, kBlock, 0, s>>>(
                 src, count, dst, with_index, extra_eps, extra_wmax, ctl)));
  } else {
    PPB_W(W, (compact_batched_kernel<WW, double><<<grid, kBlock, 0, s>>>(
                 src, count, dst, with_index, extra_eps, extra_wmax, ctl)));
  }
  return cudaGetLastError();
}

cudaError_t launch_overlap_batched(int W, int grid, cudaStream_t s, DevTable t, uint64_t count,
                                   const OverlapArgs& a, double* partials, double* out) {
  if (t.B > kMaxBOverlap) return cudaErrorInvalidValue;
  if (t.f32) {
    PPB_W(W, (overlap_batched_kernel<WW, float><<<grid, kBlock, 0, s>>>(t, count, a, partials)));
  } else {
    PPB_W(W, (overlap_batched_kernel<WW, double><<<grid, kBlock, 0, s>>>(t, count, a, partials)));
  }
  reduce_columns_kernel<<<(t.B + 255) / 256, 256, 0, s>>>(partials, grid, t.B, out);
  return cudaGetLastError();
}

cudaError_t launch_rows_to_double(int grid, cudaStream_t s, DevTable t, uint64_t count,
                                  double* out) {
  const uint64_t n = count * (uint64_t)t.B;
  if (t.f32)
    rows_to_double_kernel<float><<<grid, kBlock, 0, s>>>(static_cast<const float*>(t.rows), n, out);
  else
    rows_to_double_kernel<double><<<grid, kBlock, 0, s>>>(static_cast<const double*>(t.rows), n,
                                                          out);
  return cudaGetLastError();
}

}  // namespace ppk
