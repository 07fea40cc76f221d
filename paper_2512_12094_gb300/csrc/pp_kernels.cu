// CUDA kernels of the Pauli propagation hot path (sm_103a).
//
// Data layout (one term table):
//   keys  [cap][2W] uint64   x words then z words; loaded as W 16-byte vectors
//   coef  [cap]     double   +0.0 marks a truncated entry when eps > 0
//   index [icap]    uint64   (tag << 32) | dense position; 0 = empty slot
//
// Per gate (Appendix A, Prop. 1 proof, with U = exp(-i theta P / 2)):
//   Q commutes with P      -> Q unchanged (only per-gate damping)
//   Q anticommutes with P  -> cos(theta) Q + sin(theta) (i P Q),  i P Q = sigma R,
//                             R = Q xor P.
// Q and R = Q xor P form a pair that the gate mixes by a 2x2 rotation.  One
// thread owns each pair (the member whose "pivot" bit of P is clear), reads
// both coefficients and writes both results, so the update needs no atomics
// and is computed exactly as cos*c_Q + (+-sin*c_R) in FP64 without FMA
// contraction.  A partner that is not in the table is staged in shared
// memory, appended at the end of the gate (one atomic per block) and
// inserted into the index; it is unique to its parent, so the insert never
// races with another insert of the same key.
#include <cooperative_groups.h>

#include "pp_device.cuh"

namespace cg = cooperative_groups;

namespace ppk {
namespace {

// Births (partners not yet in the table) are staged in shared memory and
// appended with one atomic per block at the end of a gate; a block whose
// staging area fills up appends the rest directly, one atomic per warp.
template <int W, int NT = kBlock>
struct GateStage {
  static constexpr int kCap = ((W == 1) ? 512 : ((W <= 3) ? 256 : 128)) * NT / kBlock;
  uint64_t key[kCap][2 * W];
  double coef[kCap];
  uint64_t slot[kCap];  // index slot claimed for the birth (pending until published)
};

// Per-warp worklist.  A warp scans kU strings per lane (all loads in flight
// at once), keeps the anticommuting ones (key and offset in the warp's chunk)
// here, then works through the list with every lane busy: the dependent
// lookup chain (index slot -> partner key -> coefficients) then runs once per
// 32 anticommuting strings instead of once per 32 scanned strings.
template <int W, int NT = kBlock>
struct GateList {
  static constexpr int kU = (W <= 2) ? 4 : 2;
  static constexpr int kItems = 32 * kU;
  uint64_t key[NT / 32][kItems][2 * W];
  unsigned short off[NT / 32][kItems];
};

template <int NT = kBlock>
struct GateShared {
  long long delta[NT / 32];
  unsigned long long ac[NT / 32];
  unsigned nstage;
  unsigned err;
  unsigned long long base;
};

// One gate over the stored entries [0, T0) by one block of a grid (see the
// file comment).  Births go to dense positions T0 + atomicAdd(cnt_slot).
// The block's live-count change is added to *dlt_slot and its anticommuting
// count to ctl->ac_total.  Ends with the block's threads synchronised.
template <int W, int NT>
__device__ __forceinline__ void gate_pass(const DevTable& t, DevCtl* ctl, const GateArgs& g,
                                          uint64_t T0, unsigned long long* cnt_slot,
                                          long long* dlt_slot, GateStage<W, NT>& stage,
                                          GateList<W, NT>& list, GateShared<NT>& sh) {
  constexpr int kWarps = NT / 32;
  constexpr int kU = GateList<W, NT>::kU;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
  const bool noise = g.damp != nullptr;
  const bool use_eps = g.use_eps != 0;
  const uint64_t eps_bits = g.eps_bits;
  // liveness and truncation on bit patterns (see kAbsMask)
  auto is_dead = [&](double c) { return use_eps && is_zero_bits(c); };
  auto trunc = [&](double c) { return (use_eps && (dbits(c) & kAbsMask) < eps_bits) ? 0.0 : c; };
  long long delta = 0;
  unsigned long long n_ac = 0;  // live anticommuting terms (for the byte model)
  unsigned err = 0;
  // Block b takes the contiguous range [T0 b / G, T0 (b+1) / G) and splits it
  // into nt equal tiles of at most NT * kU strings, each split equally
  // over the warps: every block does the same number of equally sized tiles,
  // so blocks reach the grid barrier together, and a small table spreads one
  // string per lane over all warps.  nt is block-uniform, so every lane of a
  // warp reaches the ballots below.
  const uint64_t G = gridDim.x;
  const uint64_t b0 = T0 * blockIdx.x / G;
  const uint64_t Rn = T0 * (blockIdx.x + 1) / G - b0;
  constexpr uint64_t kTileMax = (uint64_t)NT * kU;
  const uint64_t nt = (Rn + kTileMax - 1) / kTileMax;
  auto warp_range = [&](uint64_t tt, uint64_t& ws, uint64_t& we) {
    const uint64_t ts = b0 + Rn * tt / nt, te = b0 + Rn * (tt + 1) / nt;
    ws = ts + (te - ts) * warp / kWarps;  // at most 32 kU strings per warp
    we = ts + (te - ts) * (warp + 1) / kWarps;
  };
  Key<W> Q[kU];
  auto load_tile = [&](uint64_t ws, uint64_t we) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint64_t i = ws + (uint64_t)(u * 32 + lane);
      if (i < we) Q[u] = ld_key_cg<W>(t.keys, i);
    }
  };
  uint64_t ws = 0, we = 0;
  if (nt > 0) {
    warp_range(0, ws, we);
    load_tile(ws, we);
  }
  for (uint64_t tt = 0; tt < nt; ++tt) {
    // ---- phase A: test the loaded strings, compact the anticommuting ones
    unsigned n_items = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint64_t i = ws + (uint64_t)(u * 32 + lane);
      bool ac = false;
      if (i < we) {
        int acnt = 0, kq = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          acnt += __popcll(g.px[j] & Q[u].z(j)) + __popcll(g.pz[j] & Q[u].x(j));
          if (noise) kq += __popcll((Q[u].x(j) | Q[u].z(j)) & g.supp[j]);
        }
        ac = (acnt & 1) != 0;
        if (!ac && noise && kq) {  // commuting term: damping only
          const double c = ld_coef(t.coef, i);
          if (!is_dead(c)) {
            const double d = trunc(__dmul_rn(c, g.damp[kq]));
            delta -= is_dead(d);
            t.coef[i] = d;
          }
        }
      }
      const unsigned bal = __ballot_sync(kFull, ac);
      if (ac) {
        const unsigned p = n_items + __popc(bal & lanes_below);
#pragma unroll
        for (int j = 0; j < 2 * W; ++j) list.key[warp][p][j] = Q[u].w[j];
        list.off[warp][p] = (unsigned short)(u * 32 + lane);
      }
      n_items += __popc(bal);
    }
    __syncwarp();
    const uint64_t wb = ws;  // offsets in the list are relative to this
    // the next tile's keys load while this tile's list is worked through
    if (tt + 1 < nt) {
      warp_range(tt + 1, ws, we);
      load_tile(ws, we);
    }
    // ---- phase B: the anticommuting strings, one per lane
    for (unsigned k0 = 0; k0 < n_items; k0 += 32) {
      const unsigned k = k0 + lane;
      bool want = false;
      double child = 0.0;
      uint64_t i = 0;
      Key<W> R;
      if (k < n_items) {
        Key<W> Qk;
#pragma unroll
        for (int j = 0; j < 2 * W; ++j) Qk.w[j] = list.key[warp][k][j];
        i = wb + list.off[warp][k];
        int kq = 0;
        uint64_t pw = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          R.x(j) = Qk.x(j) ^ g.px[j];
          R.z(j) = Qk.z(j) ^ g.pz[j];
          if (noise) kq += __popcll((Qk.x(j) | Qk.z(j)) & g.supp[j]);
          pw |= (Qk.x(j) & g.pvx[j]) | (Qk.z(j) & g.pvz[j]);
        }
        const double cQ = ld_coef(t.coef, i);
        const bool liveQ = !is_dead(cQ);
        // The member of {Q, R} with the pivot bit of P clear owns the pair,
        // decided from keys only.  Every member starts its lookup without
        // waiting for its own coefficient; the owner loads the partner's
        // coefficient together with its key.
        const bool owner = pw == 0;
        double cRo = 0.0;
        const uint64_t h = key_hash(R);
        // a truncated non-owner has nothing to do (its partner owns the pair
        // or is absent, and it has no birth): its lookup stops at the first slot
        const int64_t jr = index_find_old<W>(t, R, h, tag_of(h), T0, err, owner, &cRo, owner || liveQ);
        const bool neg = sigma_of<W>(g, Qk) < 0;  // i P Q = -R
        const double cR = (jr >= 0 && owner) ? cRo : 0.0;
        // live anticommuting strings, counted from values before the gate: the
        // owner counts a stored pair (its partner may be rewriting the other
        // member meanwhile), anyone else counts only itself
        if (jr >= 0)
          n_ac += owner ? (unsigned long long)liveQ + (unsigned long long)!is_dead(cR) : 0ull;
        else
          n_ac += liveQ;
        // owner with its partner stored, or a live string whose partner is new
        const bool own = jr >= 0 && owner && (liveQ || !is_dead(cR));
        const bool birth = jr == -1 && liveQ;
        if (own || birth) {
          // one instruction sequence for both cases (a birth has c_R = 0 and
          // uses only the products of c_Q); the FP64 pipe is narrow here
          double dQ = cQ, dR = cR;
          if (noise) {
            int kr = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) kr += __popcll((R.x(j) | R.z(j)) & g.supp[j]);
            if (kq) dQ = __dmul_rn(dQ, g.damp[kq]);
            if (own && kr) dR = __dmul_rn(dR, g.damp[kr]);
          }
          const double aQ = __dmul_rn(g.cth, dQ);
          const double sQ = __dmul_rn(g.sth, dQ);  // child of Q lands on R: +-sQ
          const double aR = __dmul_rn(g.cth, dR);
          const double sR = __dmul_rn(g.sth, dR);  // child of R lands on Q: -+sR
          const double mQ = __dadd_rn(aQ, with_sign(sR, !neg));
          const double mR = __dadd_rn(aR, with_sign(sQ, neg));
          const double nQ = trunc(own ? mQ : aQ);
          t.coef[i] = nQ;
          if (own) {
            const double nR = trunc(mR);
            delta += (long long)!is_dead(nQ) - (long long)liveQ + (long long)!is_dead(nR) -
                     (long long)!is_dead(cR);
            t.coef[jr] = nR;
          } else {
            delta -= is_dead(nQ);
            child = with_sign(sQ, neg);
            want = (g.wmax < 0 || weight(R) <= g.wmax) &&
                   !(use_eps && (dbits(child) & kAbsMask) < eps_bits);
          }
        }
      }
      // stage the births of this warp in shared memory (one shared atomic per warp)
      const unsigned ballot = __ballot_sync(kFull, want);
      if (ballot) {
        const int leader = __ffs(ballot) - 1;
        unsigned b0 = 0;
        if (lane == leader) b0 = atomicAdd(&sh.nstage, (unsigned)__popc(ballot));
        b0 = __shfl_sync(kFull, b0, leader);
        const unsigned pos = b0 + __popc(ballot & lanes_below);
        const bool staged = want && pos < (unsigned)GateStage<W, NT>::kCap;
        const bool direct = want && !staged;
        if (staged) {
#pragma unroll
          for (int j = 0; j < 2 * W; ++j) stage.key[pos][j] = R.w[j];
          stage.coef[pos] = child;
        }
        const unsigned over = __ballot_sync(kFull, direct);
        if (over) {  // staging area full: append straight away
          const int ol = __ffs(over) - 1;
          unsigned long long ob = 0;
          if (lane == ol) ob = T0 + atomicAdd(cnt_slot, (unsigned long long)__popc(over));
          ob = __shfl_sync(kFull, ob, ol);
          if (direct) {
            const uint64_t idx = ob + __popc(over & lanes_below);
            if (idx < t.cap) {
              st_key<W>(t.keys, idx, R);
              t.coef[idx] = child;
              const uint64_t h = key_hash(R);
              index_claim(t, h & t.imask, ((uint64_t)tag_of(h) << 32) | idx, err);
            } else {
              err |= kErrAppend;
            }
          }
        }
        delta += want;
      }
    }
    __syncwarp();  // the list is rewritten by the next tile
  }
  // the next kernel on the stream may now be scheduled (it waits for this grid)
  asm volatile("griddepcontrol.launch_dependents;");

  __syncthreads();
  const unsigned nst = min(sh.nstage, (unsigned)GateStage<W, NT>::kCap);
  if (nst) {
    // The block's positions are reserved while its births claim their index
    // slots, so the two round trips overlap.  A claimed slot holds the
    // pending position until it is published below: lookups of this gate only
    // accept positions below T0, and births are never looked up by the gate
    // that creates them, so neither ordering matters.
    if (threadIdx.x == 0) sh.base = T0 + atomicAdd(cnt_slot, (unsigned long long)nst);
    for (unsigned k = threadIdx.x; k < nst; k += NT) {
      Key<W> R;
#pragma unroll
      for (int j = 0; j < 2 * W; ++j) R.w[j] = stage.key[k][j];
      const uint64_t h = key_hash(R);
      stage.slot[k] = index_claim_pending(t, h & t.imask, tag_of(h), err);
    }
    __syncthreads();
    for (unsigned k = threadIdx.x; k < nst; k += NT) {
      const uint64_t idx = sh.base + k;
      const uint64_t sl = stage.slot[k];
      if (idx < t.cap) {
        Key<W> R;
#pragma unroll
        for (int j = 0; j < 2 * W; ++j) R.w[j] = stage.key[k][j];
        st_key<W>(t.keys, idx, R);
        t.coef[idx] = stage.coef[k];
        if (sl <= t.imask) {  // this thread owns the claimed slot
          const uint64_t h = key_hash(R);
          reinterpret_cast<unsigned long long*>(t.index)[sl] =
              ((unsigned long long)tag_of(h) << 32) | idx;
        }
      } else {
        err |= kErrAppend;
      }
    }
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
    unsigned long long a = 0;
    for (int w = 0; w < kWarps; ++w) {
      d += sh.delta[w];
      a += sh.ac[w];
    }
    // fire-and-forget reductions: no block waits for another
    if (d) atomicAdd(reinterpret_cast<unsigned long long*>(dlt_slot), (unsigned long long)d);
    if (a) atomicAdd(&ctl->ac_total, a);
    if (sh.err) {
      atomicOr(&ctl->error, sh.err);
      atomicOr(&ctl->gerr[cnt_slot - ctl->cnt], sh.err);
    }
    sh.nstage = 0;
    sh.err = 0;
  }
  __syncthreads();
}

// One kernel per gate (the graph / PDL path).  Gate g reads its input size
// from slot (g+2)%3 of the control block, which gate g-1 finished writing.
template <int W>
__global__ void __launch_bounds__(kBlock) gate_kernel(const DevTable* __restrict__ tabp,
                                                      DevCtl* __restrict__ ctl, GateArgs g) {
  __shared__ GateStage<W, kBlock> stage;
  __shared__ GateList<W, kBlock> list;
  __shared__ GateShared<kBlock> sh;
  const unsigned gid = g.gate_id;
  const int slot = (int)(gid % 3u), prev = (int)((gid + 2u) % 3u), next = (int)((gid + 1u) % 3u);
  // With programmatic dependent launch this kernel may already be resident
  // while the previous gate finishes; wait for its results first.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const DevTable t = *tabp;
  // every thread reads the (final) state left by the previous gate
  const unsigned long long T0 = __ldcg(&ctl->base[prev]) + __ldcg(&ctl->cnt[prev]);
  const long long L0 = __ldcg(&ctl->live_base[prev]) + __ldcg(&ctl->dlt[prev]);
  bool run = (gid >= __ldcg(&ctl->first_gate)) && (__ldcg(&ctl->stall) == 0u) &&
             (__ldcg(&ctl->error) == 0u);
  const bool room = gate_fits(t, T0);
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0 && run && !room) ctl->stall = gid + 1;  // every block skips
    if (blockIdx.x == 0 && run && room) {
      ctl->base[slot] = T0;
      ctl->live_base[slot] = L0;
      ctl->cnt[next] = 0;
      ctl->dlt[next] = 0;
      ctl->gerr[next] = 0;
      atomicAdd(&ctl->updates, (double)L0);
      atomicAdd(&ctl->gates_done, 1ull);
      // births R = Q xor P add at most P's letters to the occupancy masks
#pragma unroll
      for (int j = 0; j < W; ++j) {
        if (g.px[j]) atomicOr(&ctl->occ[j], (unsigned long long)g.px[j]);
        if (g.pz[j]) atomicOr(&ctl->occ[kMaxW + j], (unsigned long long)g.pz[j]);
      }
    }
    sh.nstage = 0;
    sh.err = 0;
  }
  run = run && room;
  if (!run) {
    asm volatile("griddepcontrol.launch_dependents;");
    return;
  }
  __syncthreads();
  gate_pass<W, kBlock>(t, ctl, g, T0, &ctl->cnt[slot], &ctl->dlt[slot], stage, list, sh);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident): every
// block adds 1 to a counter that only grows during the launch (release) and
// waits until it reaches (barrier number) x (blocks) (acquire).  The wait is
// bounded: on timeout the error bit is set and false is returned.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(DevCtl* ctl, unsigned& target, int& s_ok,
                                          unsigned limit, unsigned gate) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(&ctl->bar_root, 1u);
    const unsigned long long deadline = wait_deadline(limit);
    unsigned seen;
    while ((int)((seen = ld_acquire_u32(&ctl->bar_root)) - target) < 0) {
      if (global_ns() > deadline) {
        ok = 0;
        note_timeout(ctl, 1u, gate, seen, target);
        break;
      }
      __nanosleep(16);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// All gates of a layer in one cooperative launch: the table size travels in
// registers and consecutive gates are separated by a grid barrier instead of
// a kernel boundary.  Gate ids and the capacity stall are the same as for
// gate_kernel, so chain_init / chain_finish serve both: on leaving, block 0
// records the table size in the control block's exit record, which
// chain_finish reads.
//
// Occupancy test: every block keeps the OR of the x and of the z words of all
// stored strings (read from the control block, then widened by the letters
// of each gate it applies, since a birth Q xor P only adds P's letters).  A
// gate whose generator meets no letter that anticommutes with it -- and, with
// per-gate noise, no letter on its support at all -- leaves every string as
// it is; all blocks reach the same decision, so they skip it without a scan
// or a barrier.  Its updates are counted as for any other gate (and, apart,
// as skipped).  Executed gates take the counter slots by their ordinal e in
// this launch.
template <int W, int NT>
struct LayerSmem {
  GateStage<W, NT> stage;
  GateList<W, NT> list;
  GateShared<NT> sh;
  GateArgs gate[2];  // current gate and the prefetched next one
  int ok;
};

// Blocks of NT threads: 256 (four or two per SM) or 1024 (one per SM: a
// quarter of the blocks take part in each barrier and each birth
// reservation).  Shared memory is dynamic (LayerSmem).
template <int W, int NT>
__global__ void __launch_bounds__(NT, NT == 1024 ? 1 : ((W == 1) ? 4 : 2))
    layer_kernel(const DevTable* __restrict__ tabp, DevCtl* __restrict__ ctl,
                 const GateArgs* __restrict__ gates, unsigned n_gates) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LayerSmem<W, NT>& S = *reinterpret_cast<LayerSmem<W, NT>*>(smem_raw);
  GateStage<W, NT>& stage = S.stage;
  GateList<W, NT>& list = S.list;
  GateShared<NT>& sh = S.sh;
  GateArgs* s_gate = S.gate;
  int& s_ok = S.ok;
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
  unsigned target = 0;  // barrier counter value to wait for (cleared by chain_init)
  const unsigned wlimit = wait_limit_of(ctl);
  if (threadIdx.x == 0) {
    sh.nstage = 0;
    sh.err = 0;
  }
  auto fetch_args = [&](unsigned gid, int buf) {
    const unsigned* src = reinterpret_cast<const unsigned*>(gates + gid);
    unsigned* dst = reinterpret_cast<unsigned*>(&s_gate[buf]);
    for (unsigned k = threadIdx.x; k < sizeof(GateArgs) / 4; k += NT) dst[k] = __ldg(src + k);
  };
  if (__ldcg(&ctl->entry_stop) != 0u) return;  // written before the launch: uniform
  if (first < n_gates) fetch_args(first, 0);
  unsigned e = 0;  // gates executed by this launch
  int buf = 0;
  unsigned end = n_gates;  // first gate not applied
  for (unsigned gid = first; gid < n_gates; ++gid, buf ^= 1) {
    __syncthreads();  // s_gate[buf] complete; the other buffer is free
    const GateArgs& g = s_gate[buf];
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
      if (gid + 1 < n_gates) fetch_args(gid + 1, buf ^ 1);
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
    gate_pass<W, NT>(t, ctl, g, T0, &ctl->cnt[slot], &ctl->dlt[slot], stage, list, sh);
#pragma unroll
    for (int j = 0; j < W; ++j) {
      ox[j] |= g.px[j];
      oz[j] |= g.pz[j];
    }
    if (gid + 1 < n_gates) fetch_args(gid + 1, buf ^ 1);  // overlaps the barrier wait
    if (gridDim.x == 1) {
      // a small table in one block: its own writes and atomics, ordered by a
      // fence and the block barrier, are all the next gate depends on
      __threadfence();
      __syncthreads();
    } else if (!grid_sync(ctl, target, s_ok, wlimit, gid)) {
      return;
    }
    T0 += __ldcg(&ctl->cnt[slot]);
    L0 += __ldcg(&ctl->dlt[slot]);
    ++e;
    if (__ldcg(&ctl->gerr[slot]) != 0u) return;  // written by this gate only: uniform
  }
  // the state after the last gate applied, in the exit record (not a gate
  // slot: slower blocks may still be reading the slot of the last gate when
  // block 0 gets here), and the widened occupancy masks
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

__global__ void ctl_insert_kernel(DevCtl* ctl, unsigned long long first_free, int guarded,
                                  int reset_occ) {
  if (guarded && queued_layer_stopped(ctl)) return;
  ctl->n_next = first_free;
  ctl->n_live = 0;
  if (reset_occ)
    for (int j = 0; j < 2 * kMaxW; ++j) ctl->occ[j] = 0ull;
}

__global__ void ctl_commit_kernel(DevCtl* ctl, int guarded) {
  if (guarded && queued_layer_stopped(ctl)) return;
  ctl->n_terms = ctl->n_next;
}

__global__ void chain_init_kernel(DevCtl* ctl, unsigned first_gate) {
  const int q = (int)((first_gate + 2u) % 3u);
  ctl->bar_root = 0;
  ctl->base[q] = ctl->n_terms;
  ctl->live_base[q] = ctl->n_live;
  for (int k = 0; k < 3; ++k) {
    ctl->cnt[k] = 0;
    ctl->dlt[k] = 0;
    ctl->gerr[k] = 0;
  }
  ctl->stall = 0;
  ctl->first_gate = first_gate;
  ctl->exit_set = 0;
  ctl->entry_stop = ctl->error != 0u ? 1u : 0u;
}

__global__ void chain_finish_kernel(DevCtl* ctl, unsigned n_gates) {
  if (ctl->exit_set) {
    ctl->n_terms = ctl->exit_terms;
    ctl->n_live = ctl->exit_live;
  } else {
    const unsigned end = ctl->stall ? ctl->stall - 1u : n_gates;  // first gate not applied
    const int q = (int)((end + 2u) % 3u);                         // slot of gate end-1
    ctl->n_terms = ctl->base[q] + ctl->cnt[q];
    ctl->n_live = ctl->live_base[q] + ctl->dlt[q];
  }
  ctl->after_terms = ctl->n_terms;
}

// ------------------------------------------------------ merge / insert

template <int W, int G>
__global__ void __launch_bounds__(kBlock)
    merge_insert_kernel(const uint64_t* __restrict__ src_keys, const double* __restrict__ src_coef,
                        uint64_t count, const unsigned long long* count_dev, int skip_zero,
                        int wmax, int n, int lx, DevTable dst, DevCtl* ctl, int guarded) {
  // guarded: queued behind a layer before its outcome is known; nothing to
  // do if that layer stopped for capacity
  if (guarded && queued_layer_stopped(ctl)) return;
  const uint64_t T = count_dev ? *count_dev : count;
  const unsigned wlimit = wait_limit_of(ctl);
  unsigned err = 0;
  OccAcc<W> occ;
  unsigned long long* index = reinterpret_cast<unsigned long long*>(dst.index);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    const double c = src_coef[i];
    if (skip_zero && c == 0.0) continue;
    Key<W> K = ld_key<W>(src_keys, i);
    if (wmax >= 0 && weight(K) > wmax) continue;
    canon<W, G>(K, n, lx);
    occ.add(K);
    const uint64_t h = key_hash(K);
    const uint32_t tag = tag_of(h);
    uint64_t pos = h & dst.imask;
    bool done = false;
    for (uint64_t probe = 0; probe <= dst.imask; ++probe) {
      unsigned long long s = __ldcg(index + pos);
      if (s == 0ull) {
        const unsigned long long mine = ((unsigned long long)tag << 32) | kPendingIdx;
        const unsigned long long old = atomicCAS(index + pos, 0ull, mine);
        if (old == 0ull) {
          cg::coalesced_group grp = cg::coalesced_threads();
          unsigned long long b0 = 0;
          if (grp.thread_rank() == 0) b0 = atomicAdd(&ctl->n_next, (unsigned long long)grp.size());
          b0 = grp.shfl(b0, 0);
          const unsigned long long idx = b0 + grp.thread_rank();
          if (idx >= dst.cap) {
            err |= kErrAppend;
          } else {
            st_key<W>(dst.keys, idx, K);
            dst.coef[idx] = c;
            __threadfence();
            atomicExch(index + pos, ((unsigned long long)tag << 32) | idx);
          }
          done = true;
          break;
        }
        s = old;
      }
      if ((uint32_t)(s >> 32) == tag) {
        // read the slot again with acquire semantics before using its position
        s = ld_acquire_u64(index + pos);
        if ((uint32_t)s == kPendingIdx) {
          const unsigned long long deadline = wait_deadline(wlimit);
          while ((uint32_t)s == kPendingIdx && global_ns() <= deadline) {
            __nanosleep(64);
            s = ld_acquire_u64(index + pos);
          }
        }
        if ((uint32_t)s == kPendingIdx) {
          note_timeout(ctl, 3u, 0u, (unsigned)pos, 0u);
          done = true;
          break;
        }
        const uint32_t idx = (uint32_t)s;
        if (keys_equal(ld_key_cg<W>(dst.keys, idx), K)) {
          atomicAdd(dst.coef + idx, c);
          done = true;
          break;
        }
      }
      pos = (pos + 1) & dst.imask;
    }
    if (!done) err |= kErrProbe;
  }
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

// Coefficient truncation of the merged entries and live count.
__global__ void __launch_bounds__(kBlock) finalize_kernel(DevTable t, DevCtl* ctl, double eps,
                                                         int guarded) {
  __shared__ long long s_live[kBlock / 32];
  if (guarded && queued_layer_stopped(ctl)) return;
  const uint64_t T = *reinterpret_cast<volatile unsigned long long*>(&ctl->n_next);
  long long live = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    if (eps > 0.0) {
      const double c = t.coef[i];
      if (c != 0.0 && !(fabs(c) >= eps)) {
        t.coef[i] = 0.0;
      } else {
        live += (c != 0.0);
      }
    } else {
      live += 1;
    }
  }
  live = warp_sum(live);
  if ((threadIdx.x & 31) == 0) s_live[threadIdx.x >> 5] = live;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < kBlock / 32; ++w) s += s_live[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live), (unsigned long long)s);
  }
}

// Copy kept entries into a fresh table (unique keys).  extra_eps / extra_wmax
// implement pp_truncate on top of the context's own rule.
template <int W>
__global__ void __launch_bounds__(kBlock)
    compact_kernel(DevTable src, uint64_t count, DevTable dst, int with_index, double eps,
                   double extra_eps, int extra_wmax, DevCtl* ctl) {
  const int lane = threadIdx.x & 31;
  unsigned err = 0;
  long long live = 0;
  OccAcc<W> occ;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < count;
       base += stride) {
    const uint64_t i = base + lane;
    bool keep = false;
    Key<W> K;
    double c = 0.0;
    if (i < count) {
      c = src.coef[i];
      keep = !dead(c, eps);
      if (keep && extra_eps > 0.0 && !(fabs(c) >= extra_eps)) keep = false;
      if (keep) {
        K = ld_key<W>(src.keys, i);
        if (extra_wmax >= 0 && weight(K) > extra_wmax) keep = false;
      }
    }
    const unsigned ballot = __ballot_sync(kFull, keep);
    if (ballot) {
      const int leader = __ffs(ballot) - 1;
      unsigned long long b0 = 0;
      if (lane == leader) b0 = atomicAdd(&ctl->n_next, (unsigned long long)__popc(ballot));
      b0 = __shfl_sync(kFull, b0, leader);
      if (keep) {
        const uint64_t idx = b0 + __popc(ballot & ((1u << lane) - 1u));
        if (idx >= dst.cap) {
          err |= kErrAppend;
        } else {
          st_key<W>(dst.keys, idx, K);
          dst.coef[idx] = c;
          occ.add(K);
          ++live;
          if (with_index) {
            const uint64_t h = key_hash(K);
            index_claim(dst, h & dst.imask, ((uint64_t)tag_of(h) << 32) | idx, err);
          }
        }
      }
    }
  }
  live = warp_sum(live);
  if (lane == 0 && live) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live), (unsigned long long)live);
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

template <int W, int G>
__global__ void __launch_bounds__(kBlock)
    canon_inplace_kernel(uint64_t* keys, const uint64_t* keys_in, uint64_t count, int n, int lx,
                         DevCtl* ctl) {
  OccAcc<W> occ;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    Key<W> k = ld_key_cg<W>(keys_in, i);
    canon<W, G>(k, n, lx);
    st_key<W>(keys, i, k);
    occ.add(k);
  }
  if (ctl) occ.flush(ctl);
}

template <int W>
__global__ void __launch_bounds__(kBlock)
    damp_layer_kernel(DevTable t, DevCtl* ctl, const double* table, double eps) {
  __shared__ long long s_d[kBlock / 32];
  const uint64_t T = *reinterpret_cast<volatile unsigned long long*>(&ctl->n_terms);
  long long delta = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    const double c = t.coef[i];
    if (dead(c, eps)) continue;
    const int w = weight(ld_key<W>(t.keys, i));
    if (w == 0) continue;
    const double d = trunc_c(__dmul_rn(c, table[w]), eps);
    if (dead(d, eps)) --delta;
    t.coef[i] = d;
  }
  delta = warp_sum(delta);
  if ((threadIdx.x & 31) == 0) s_d[threadIdx.x >> 5] = delta;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < kBlock / 32; ++w) s += s_d[w];
    if (s) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live), (unsigned long long)s);
  }
}

template <int W>
__global__ void __launch_bounds__(kBlock)
    overlap_kernel(const uint64_t* __restrict__ keys, const double* __restrict__ coef,
                   uint64_t count, const unsigned long long* count_dev, OverlapArgs a,
                   double* partials) {
  __shared__ double s_acc[kBlock / 32];
  const uint64_t T = count_dev ? *count_dev : count;
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    const double c = coef[i];
    if (c == 0.0) continue;
    const Key<W> k = ld_key<W>(keys, i);
    double ov;
    if (a.group == 1)
      ov = overlap_zn<W>(k, a);
    else if (a.group == 3 || a.group == 4)
      ov = overlap_group<W>(k, a);
    else if (a.group == 2)
      ov = overlap_sn<W>(k, a);
    else
      ov = overlap_plain<W>(k, a);
    acc += c * ov;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += s_acc[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kBlock) reduce_partials_kernel(const double* partials, int m,
                                                                double* out) {
  __shared__ double s_acc[kBlock / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc += partials[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) s += s_acc[w];
    out[0] = s;
  }
}

// Orbit average of Tr[rho g.s] over S_n as a function of (n_X, n_Y, n_Z):
// sites are filled in order, site k drawing each remaining letter with
// probability (remaining count) / (remaining sites).  E_k over states
// (x, y, z) of remaining counts; every step is a convex combination.
__global__ void __launch_bounds__(1024) sn_table_kernel(int n, const double* bloch, double* table,
                                                       double* work) {
  const int S = n + 1;
  const size_t total = (size_t)S * S * S;
  // after n steps the result must sit in `table`: start in whichever buffer
  // makes the last write land there
  double* nxt = (n & 1) ? work : table;
  double* cur = (n & 1) ? table : work;
  for (size_t i = threadIdx.x; i < total; i += blockDim.x) nxt[i] = (i == 0) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    const int left = n - k;
    const double bX = bloch[3 * k], bY = bloch[3 * k + 1], bZ = bloch[3 * k + 2];
    for (size_t f = threadIdx.x; f < total; f += blockDim.x) {
      const int z = (int)(f % S), y = (int)((f / S) % S), x = (int)(f / ((size_t)S * S));
      double v = 0.0;
      if (x + y + z <= left) {
        const int iI = left - x - y - z;
        if (iI > 0) v += (double)iI * nxt[f];
        if (x > 0) v += (double)x * bX * nxt[f - (size_t)S * S];
        if (y > 0) v += (double)y * bY * nxt[f - S];
        if (z > 0) v += (double)z * bZ * nxt[f - 1];
        v /= (double)left;
      }
      cur[f] = v;
    }
    __syncthreads();
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

// x [m][W], z [m][W] -> keys [m][2W]; flags strings with bits at or above n.
template <int W>
__global__ void __launch_bounds__(kBlock)
    pack_keys_kernel(const uint64_t* __restrict__ x, const uint64_t* __restrict__ z, uint64_t m,
                     int n, uint64_t* keys, unsigned* bad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    Key<W> k;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      k.x(j) = x[i * W + j];
      k.z(j) = z[i * W + j];
      const int lo = 64 * j;
      const uint64_t valid = (n >= lo + 64) ? ~0ull : ((n > lo) ? ((1ull << (n - lo)) - 1ull) : 0ull);
      ok &= ((k.x(j) | k.z(j)) & ~valid) == 0ull;
    }
    st_key<W>(keys, i, k);
    if (!ok) atomicOr(bad, 1u);
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers

#define PP_DISPATCH_W(W, ...)                     \
  switch (W) {                                    \
    case 1: { constexpr int WW = 1; __VA_ARGS__; break; } \
    case 2: { constexpr int WW = 2; __VA_ARGS__; break; } \
    case 3: { constexpr int WW = 3; __VA_ARGS__; break; } \
    case 4: { constexpr int WW = 4; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;        \
  }

cudaError_t launch_ctl_insert(cudaStream_t s, DevCtl* ctl, unsigned long long first_free,
                              int guarded, int reset_occ) {
  ctl_insert_kernel<<<1, 1, 0, s>>>(ctl, first_free, guarded, reset_occ);
  return cudaGetLastError();
}

cudaError_t launch_ctl_commit(cudaStream_t s, DevCtl* ctl, int guarded) {
  ctl_commit_kernel<<<1, 1, 0, s>>>(ctl, guarded);
  return cudaGetLastError();
}

cudaError_t launch_chain_init(cudaStream_t s, DevCtl* ctl, unsigned first_gate) {
  chain_init_kernel<<<1, 1, 0, s>>>(ctl, first_gate);
  return cudaGetLastError();
}

cudaError_t launch_chain_finish(cudaStream_t s, DevCtl* ctl, unsigned n_gates) {
  chain_finish_kernel<<<1, 1, 0, s>>>(ctl, n_gates);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_gate_w(int grid, cudaStream_t s, const DevTable* tab, DevCtl* ctl,
                          const GateArgs& g, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, gate_kernel<W>, tab, ctl, g);
}

// The layer kernel's dynamic shared memory must be allowed above 48 KB once
// per instantiation (and before an occupancy query).
template <int W, int NT>
cudaError_t layer_smem_setup() {
  static cudaError_t done = cudaFuncSetAttribute(
      layer_kernel<W, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)sizeof(LayerSmem<W, NT>));
  return done;
}

template <int W, int NT>
cudaError_t launch_layer_w(int grid, cudaStream_t s, const DevTable* tab, DevCtl* ctl,
                           const GateArgs* gates, unsigned n_gates) {
  cudaError_t e = layer_smem_setup<W, NT>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(LayerSmem<W, NT>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, layer_kernel<W, NT>, tab, ctl, gates, n_gates);
}

template <int W, int NT>
int layer_bps_w() {
  int nb = 0;
  if (layer_smem_setup<W, NT>() != cudaSuccess) return 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, layer_kernel<W, NT>, NT, sizeof(LayerSmem<W, NT>));
  return (e == cudaSuccess && nb > 0) ? nb : 0;
}

cudaError_t launch_layer(int W, int threads, int grid, cudaStream_t s, const DevTable* tab,
                         DevCtl* ctl, const GateArgs* gates, unsigned n_gates) {
  if (threads == 1024) {
    switch (W) {
      case 1: return launch_layer_w<1, 1024>(grid, s, tab, ctl, gates, n_gates);
      case 2: return launch_layer_w<2, 1024>(grid, s, tab, ctl, gates, n_gates);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (W) {
    case 1: return launch_layer_w<1, kBlock>(grid, s, tab, ctl, gates, n_gates);
    case 2: return launch_layer_w<2, kBlock>(grid, s, tab, ctl, gates, n_gates);
    case 3: return launch_layer_w<3, kBlock>(grid, s, tab, ctl, gates, n_gates);
    case 4: return launch_layer_w<4, kBlock>(grid, s, tab, ctl, gates, n_gates);
    default: return cudaErrorInvalidValue;
  }
}

int layer_blocks_per_sm(int W, int threads) {
  if (threads == 1024) {
    switch (W) {
      case 1: return layer_bps_w<1, 1024>();
      case 2: return layer_bps_w<2, 1024>();
      default: return 0;
    }
  }
  switch (W) {
    case 1: return layer_bps_w<1, kBlock>();
    case 2: return layer_bps_w<2, kBlock>();
    case 3: return layer_bps_w<3, kBlock>();
    case 4: return layer_bps_w<4, kBlock>();
    default: return 0;
  }
}

cudaError_t launch_gate(int W, int grid, cudaStream_t s, const DevTable* tab, DevCtl* ctl,
                        const GateArgs& g, bool pdl) {
  switch (W) {
    case 1: return launch_gate_w<1>(grid, s, tab, ctl, g, pdl);
    case 2: return launch_gate_w<2>(grid, s, tab, ctl, g, pdl);
    case 3: return launch_gate_w<3>(grid, s, tab, ctl, g, pdl);
    case 4: return launch_gate_w<4>(grid, s, tab, ctl, g, pdl);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_merge_insert(int W, int group, int n, int wmax, int grid, cudaStream_t s,
                                  const uint64_t* src_keys, const double* src_coef,
                                  uint64_t count, const unsigned long long* count_dev,
                                  int skip_zero, DevTable dst, DevCtl* ctl, int guarded) {
  const int lx = group >> 8;  // group code: kind | (torus width << 8)
#define PP_MERGE_G(GG)                                                                     \
  PP_DISPATCH_W(W, (merge_insert_kernel<WW, GG><<<grid, kBlock, 0, s>>>(                   \
                       src_keys, src_coef, count, count_dev, skip_zero, wmax, n, lx, dst, ctl, guarded)))
  switch (group & 0xFF) {
    case 0: PP_MERGE_G(0); break;
    case 1: PP_MERGE_G(1); break;
    case 2: PP_MERGE_G(2); break;
    case 3: PP_MERGE_G(3); break;
    case 4: PP_MERGE_G(4); break;
    default:
      return cudaErrorInvalidValue;
  }
#undef PP_MERGE_G
  return cudaGetLastError();
}

cudaError_t launch_finalize(int grid, cudaStream_t s, DevTable dst, DevCtl* ctl, double eps,
                            int guarded) {
  finalize_kernel<<<grid, kBlock, 0, s>>>(dst, ctl, eps, guarded);
  return cudaGetLastError();
}

cudaError_t launch_compact(int W, int grid, cudaStream_t s, DevTable src, uint64_t count,
                           DevTable dst, int with_index, double eps, double extra_eps,
                           int extra_wmax, DevCtl* ctl_dst) {
  PP_DISPATCH_W(W, (compact_kernel<WW><<<grid, kBlock, 0, s>>>(src, count, dst, with_index, eps,
                                                               extra_eps, extra_wmax, ctl_dst)));
  return cudaGetLastError();
}

cudaError_t launch_canon_inplace(int W, int group, int n, int grid, cudaStream_t s,
                                 uint64_t* keys, const uint64_t* keys_in, uint64_t count,
                                 DevCtl* ctl) {
  const int lx = group >> 8;
#define PP_CANON_G(GG) \
  PP_DISPATCH_W(W, (canon_inplace_kernel<WW, GG><<<grid, kBlock, 0, s>>>(keys, keys_in, count, n, \
                                                                        lx, ctl)))
  switch (group & 0xFF) {
    case 1: PP_CANON_G(1); break;
    case 2: PP_CANON_G(2); break;
    case 3: PP_CANON_G(3); break;
    case 4: PP_CANON_G(4); break;
    default: PP_CANON_G(0); break;
  }
#undef PP_CANON_G
  return cudaGetLastError();
}

cudaError_t launch_damp_layer(int W, int grid, cudaStream_t s, DevTable t, DevCtl* ctl,
                              const double* table, double eps) {
  PP_DISPATCH_W(W, (damp_layer_kernel<WW><<<grid, kBlock, 0, s>>>(t, ctl, table, eps)));
  return cudaGetLastError();
}

cudaError_t launch_overlap(int W, int grid, cudaStream_t s, const uint64_t* keys,
                           const double* coef, uint64_t count,
                           const unsigned long long* count_dev, const OverlapArgs& a,
                           double* partials, double* out) {
  PP_DISPATCH_W(W, (overlap_kernel<WW><<<grid, kBlock, 0, s>>>(keys, coef, count, count_dev, a,
                                                               partials)));
  reduce_partials_kernel<<<1, kBlock, 0, s>>>(partials, grid, out);
  return cudaGetLastError();
}

cudaError_t launch_sn_table(int n, cudaStream_t s, const double* bloch, double* work,
                            double* table) {
  sn_table_kernel<<<1, 1024, 0, s>>>(n, bloch, table, work);
  return cudaGetLastError();
}

cudaError_t launch_pack_keys(int W, int n, int grid, cudaStream_t s, const uint64_t* x,
                             const uint64_t* z, uint64_t m, uint64_t* keys, unsigned* bad) {
  PP_DISPATCH_W(W, (pack_keys_kernel<WW><<<grid, kBlock, 0, s>>>(x, z, m, n, keys, bad)));
  return cudaGetLastError();
}

int gate_blocks_per_sm(int W) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (W) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gate_kernel<1>, kBlock, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gate_kernel<2>, kBlock, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gate_kernel<3>, kBlock, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gate_kernel<4>, kBlock, 0); break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 4;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

}  // namespace ppk
