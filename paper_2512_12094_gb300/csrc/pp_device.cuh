// Device helpers shared by the CUDA translation units of the library: key
// loads and stores, hashing, the key -> position index, the sign rule of a
// Pauli product, orbit representatives and product-state overlaps.
#pragma once

#include "pp_internal.h"

namespace ppk {
namespace {


constexpr unsigned kFull = 0xFFFFFFFFu;
// Default bound of a device wait (a grid barrier or a pending index slot),
// in microseconds of the GPU's global timer: 30 s, far above the longest
// gate (a gate over gigabytes of batched rows takes seconds) and far below a
// hang.  A context may set another bound (DevCtl::wait_limit); a wait that
// runs out sets kErrTimeout and returns, so the host reports PP_ERR_TIMEOUT.
constexpr unsigned kDefaultWaitLimit = 30u * 1000u * 1000u;

// Record the first device error with where it happened (only the first
// record is kept); the caller sets the error bit.
__device__ __forceinline__ void note_first(DevCtl* ctl, unsigned kind, unsigned gate,
                                           unsigned a, unsigned b) {
  if (atomicCAS(&ctl->to_kind, 0u, kind) == 0u) {
    ctl->to_gate = gate;
    ctl->to_seen = a;
    ctl->to_target = b;
  }
}

// Record where a bounded wait gave up and set the timeout error bit.
__device__ __forceinline__ void note_timeout(DevCtl* ctl, unsigned kind, unsigned gate,
                                             unsigned seen, unsigned target) {
  note_first(ctl, kind, gate, seen, target);
  atomicOr(&ctl->error, kErrTimeout);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Deadline of a wait that starts now, limit_us microseconds away.
__device__ __forceinline__ unsigned long long wait_deadline(unsigned limit_us) {
  return global_ns() + 1000ull * (unsigned long long)limit_us;
}
// A merge queued behind a layer before the layer's outcome is known does
// nothing when a gate of that layer stopped for capacity or failed.
__device__ __forceinline__ bool queued_layer_stopped(const DevCtl* ctl) {
  return *reinterpret_cast<const volatile unsigned*>(&ctl->stall) != 0u ||
         *reinterpret_cast<const volatile unsigned*>(&ctl->error) != 0u;
}

// Room for one more gate on a table of T0 stored entries: a gate appends at
// most one birth per string, so the capacity must hold 2 T0 (the index has
// at least 1.5 slots per entry of capacity).  Every block of a gate takes the
// same decision from the same T0.
__device__ __forceinline__ bool gate_fits(const DevTable& t, uint64_t T0) {
  return 2ull * T0 <= t.cap;
}

__device__ __forceinline__ unsigned wait_limit_of(const DevCtl* ctl) {
  const unsigned v = *reinterpret_cast<const volatile unsigned*>(&ctl->wait_limit);
  return v ? v : kDefaultWaitLimit;
}

template <int W>
struct Key {
  uint64_t w[2 * W];  // x[0..W), z[0..W)
  __device__ __forceinline__ uint64_t& x(int i) { return w[i]; }
  __device__ __forceinline__ uint64_t& z(int i) { return w[W + i]; }
  __device__ __forceinline__ uint64_t x(int i) const { return w[i]; }
  __device__ __forceinline__ uint64_t z(int i) const { return w[W + i]; }
};

template <int W>
__device__ __forceinline__ Key<W> ld_key(const uint64_t* __restrict__ keys, uint64_t i) {
  Key<W> k;
  const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + i * (2 * W));
#pragma unroll
  for (int j = 0; j < W; ++j) {
    ulonglong2 v = __ldg(p + j);
    k.w[2 * j] = v.x;
    k.w[2 * j + 1] = v.y;
  }
  return k;
}

// Load through L2 only (entries that other threads may have written in the
// same kernel).
template <int W>
__device__ __forceinline__ Key<W> ld_key_cg(const uint64_t* keys, uint64_t i) {
  Key<W> k;
  const ulonglong2* p = reinterpret_cast<const ulonglong2*>(keys + i * (2 * W));
#pragma unroll
  for (int j = 0; j < W; ++j) {
    ulonglong2 v = __ldcg(p + j);
    k.w[2 * j] = v.x;
    k.w[2 * j + 1] = v.y;
  }
  return k;
}

template <int W>
__device__ __forceinline__ void st_key(uint64_t* keys, uint64_t i, const Key<W>& k) {
  ulonglong2* p = reinterpret_cast<ulonglong2*>(keys + i * (2 * W));
#pragma unroll
  for (int j = 0; j < W; ++j) p[j] = make_ulonglong2(k.w[2 * j], k.w[2 * j + 1]);
}

template <int W>
__device__ __forceinline__ bool keys_equal(const Key<W>& a, const Key<W>& b) {
  bool eq = true;
#pragma unroll
  for (int j = 0; j < 2 * W; ++j) eq &= (a.w[j] == b.w[j]);
  return eq;
}

// 64-bit hash of a key built from 32-bit multiplies only (murmur3-style
// mixing of the 32-bit halves, two lanes with different constants).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

template <int W>
__device__ __forceinline__ uint64_t key_hash(const Key<W>& k) {
  uint32_t a = 0x9E3779B9u, b = 0x7F4A7C15u;
#pragma unroll
  for (int j = 0; j < 2 * W; ++j) {
    const uint32_t lo = (uint32_t)k.w[j], hi = (uint32_t)(k.w[j] >> 32);
    a = (a ^ lo) * 0xcc9e2d51u;
    a = __funnelshift_l(a, a, 15) ^ hi;
    a *= 0x1b873593u;
    b = (b ^ hi) * 0x27d4eb2fu;
    b = __funnelshift_l(b, b, 13) ^ lo;
    b *= 0x165667b1u;
  }
  return ((uint64_t)fmix32(a ^ b) << 32) | fmix32(b + 0x9E3779B9u * a);
}

__device__ __forceinline__ uint32_t tag_of(uint64_t h) { return (uint32_t)(h >> 32) | 0x80000000u; }

template <int W>
__device__ __forceinline__ int weight(const Key<W>& k) {
  int w = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) w += __popcll(k.x(j) | k.z(j));
  return w;
}

// Find key k in the index.  Returns its dense position, -1 when it is not
// present, or -2 (error bit set) when the probe bound is exhausted.
template <int W>
__device__ __forceinline__ int64_t index_find(const DevTable& t, const Key<W>& k, uint64_t h,
                                              uint32_t tag, unsigned& err) {
  uint64_t pos = h & t.imask;
  for (uint64_t probe = 0; probe <= t.imask; ++probe) {
    uint64_t s = __ldcg(reinterpret_cast<const unsigned long long*>(t.index) + pos);
    if (s == 0) return -1;
    if ((uint32_t)(s >> 32) == tag) {
      uint32_t idx = (uint32_t)s;
      if (idx != kPendingIdx && keys_equal(ld_key_cg<W>(t.keys, idx), k)) return (int64_t)idx;
    }
    pos = (pos + 1) & t.imask;
  }
  err |= kErrProbe;
  return -2;
}

// Claim an empty slot for a key whose dense position is already written.
__device__ __forceinline__ void index_claim(const DevTable& t, uint64_t pos, uint64_t val,
                                            unsigned& err) {
  unsigned long long* idx = reinterpret_cast<unsigned long long*>(t.index);
  for (uint64_t probe = 0; probe <= t.imask; ++probe) {
    if (atomicCAS(idx + pos, 0ull, (unsigned long long)val) == 0ull) return;
    pos = (pos + 1) & t.imask;
  }
  err |= kErrProbe;
}

// Accumulates the OR of keys in registers and adds it to a control block's
// occupancy masks with one atomic per word and warp.
template <int W>
struct OccAcc {
  uint64_t m[2 * W];
  __device__ __forceinline__ OccAcc() {
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) m[j] = 0;
  }
  __device__ __forceinline__ void add(const Key<W>& k) {
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) m[j] |= k.w[j];
  }
  // every lane of the warp must call this
  __device__ __forceinline__ void flush(DevCtl* ctl) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) {
      uint64_t v = m[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
      // word j of the key is word (j % W) of x (j < W) or of z
      const int slot = (j < W) ? j : (kMaxW + j - W);
      if (lane == 0 && v) atomicOr(&ctl->occ[slot], (unsigned long long)v);
    }
  }
};

// Acquire load of an index slot: pairs with the fence and exchange that
// publish a slot's dense position, so the key and coefficient written before
// the publication are visible to the reader.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Claim an empty slot with a pending position (published later by its
// owner); returns the slot, or ~0 (error bit set) if the probe bound runs out.
__device__ __forceinline__ uint64_t index_claim_pending(const DevTable& t, uint64_t pos,
                                                        uint32_t tag, unsigned& err) {
  unsigned long long* idx = reinterpret_cast<unsigned long long*>(t.index);
  const unsigned long long val = ((unsigned long long)tag << 32) | kPendingIdx;
  for (uint64_t probe = 0; probe <= t.imask; ++probe) {
    if (atomicCAS(idx + pos, 0ull, val) == 0ull) return pos;
    pos = (pos + 1) & t.imask;
  }
  err |= kErrProbe;
  return ~0ull;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ----------------------------------------------------------- gate kernel

template <int W>
__device__ __forceinline__ int sigma_of(const GateArgs& g, const Key<W>& q) {
  // P Q = i^E R with E = sum_sites px pz + qx qz + 2 pz qx - (px^qx)(pz^qz)
  // (P = i^{px pz} X^px Z^pz per site); i P Q = i^{E+1} R and E+1 is even.
  int e = g.pyy;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    e += __popcll(q.x(j) & q.z(j)) + 2 * __popcll(g.pz[j] & q.x(j)) -
         __popcll((g.px[j] ^ q.x(j)) & (g.pz[j] ^ q.z(j)));
  }
  return ((e + 1) & 3) == 0 ? 1 : -1;
}

__device__ __forceinline__ bool dead(double c, double eps) { return eps > 0.0 && c == 0.0; }
__device__ __forceinline__ double trunc_c(double c, double eps) {
  return (eps > 0.0 && !(fabs(c) >= eps)) ? 0.0 : c;
}

// The FP64 pipe of this GPU issues 2 instructions per cycle per SM, so the
// gate kernel keeps it for the rotation arithmetic only: zero tests and
// threshold compares run on the integer bit patterns (for finite doubles,
// |a| < |b| exactly when (bits(a) & ~sign) < (bits(b) & ~sign) as unsigned).
constexpr uint64_t kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t kSignBit = 0x8000000000000000ull;
__device__ __forceinline__ uint64_t dbits(double c) { return (uint64_t)__double_as_longlong(c); }
__device__ __forceinline__ bool is_zero_bits(double c) { return (dbits(c) << 1) == 0ull; }
__device__ __forceinline__ double with_sign(double c, bool negate) {
  return __longlong_as_double((long long)(dbits(c) ^ (negate ? kSignBit : 0ull)));
}

// -------------------------------------------------- canonicalisation

// Digit word of Def. "Lowest integer representation": bit 2q = x_q ^ z_q,
// bit 2q+1 = z_q, so the 2-bit digit of qubit q is I=0, X=1, Y=2, Z=3.
__device__ __forceinline__ uint64_t spread32(uint32_t a) {
  uint64_t x = a;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__device__ __forceinline__ uint64_t digits32(uint32_t x, uint32_t z) {
  return spread32(x ^ z) | (spread32(z) << 1);
}

template <int W>
__device__ __forceinline__ int digit_at(const Key<W>& k, int q) {
  const int xb = (int)((k.x(q >> 6) >> (q & 63)) & 1ull);
  const int zb = (int)((k.z(q >> 6) >> (q & 63)) & 1ull);
  return (zb << 1) | (xb ^ zb);
}

// n-bit masks over W words (bits at or above n are zero).
template <int W>
struct Mask {
  uint64_t w[W];
};

template <int W>
__device__ __forceinline__ Mask<W> nbits_mask(int n) {
  Mask<W> m;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const int b = n - 64 * i;
    m.w[i] = b >= 64 ? ~0ull : (b > 0 ? ((1ull << b) - 1ull) : 0ull);
  }
  return m;
}

// Logical shifts of a W-word value by s bits (0 <= s < 64 W); words are
// picked with compile-time indices only, so nothing spills to local memory.
template <int W>
__device__ __forceinline__ Mask<W> mask_shr(const Mask<W>& v, int s) {
  Mask<W> o;
  const int ws = s >> 6, bs = s & 63;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int t = 0; t < W; ++t) {
      lo = (t == i + ws) ? v.w[t] : lo;
      hi = (t == i + ws + 1) ? v.w[t] : hi;
    }
    o.w[i] = bs ? ((lo >> bs) | (hi << (64 - bs))) : lo;
  }
  return o;
}

template <int W>
__device__ __forceinline__ Mask<W> mask_shl(const Mask<W>& v, int s) {
  Mask<W> o;
  const int ws = s >> 6, bs = s & 63;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int t = 0; t < W; ++t) {
      hi = (t == i - ws) ? v.w[t] : hi;
      lo = (t == i - ws - 1) ? v.w[t] : lo;
    }
    o.w[i] = bs ? ((hi << bs) | (lo >> (64 - bs))) : hi;
  }
  return o;
}

// Cyclic shift of an n-bit mask toward bit 0: bit q of the result is bit
// (q + j) mod n of v (0 <= j < n).  This is the translation T^j of the
// paper's example (T moves the letter of qubit q + 1 to qubit q).
template <int W>
__device__ __forceinline__ Mask<W> mask_rot(const Mask<W>& v, int j, int n, const Mask<W>& nm) {
  if (j == 0) return v;
  if constexpr (W == 1) {
    Mask<1> o;
    o.w[0] = ((v.w[0] >> j) | (v.w[0] << (n - j))) & nm.w[0];
    return o;
  } else {
    const Mask<W> a = mask_shr<W>(v, j), b = mask_shl<W>(v, n - j);
    Mask<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = (a.w[i] | b.w[i]) & nm.w[i];
    return o;
  }
}

// More than one bit set.
template <int W>
__device__ __forceinline__ bool mask_many(const Mask<W>& v) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) c += __popcll(v.w[i]);
  return c > 1;
}

template <int W>
__device__ __forceinline__ bool mask_any(const Mask<W>& v) {
  uint64_t a = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) a |= v.w[i];
  return a != 0;
}

template <int W>
__device__ __forceinline__ Key<W> rotate_key(const Key<W>& k, int j, int n, const Mask<W>& nm) {
  Mask<W> x, z;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    x.w[i] = k.x(i);
    z.w[i] = k.z(i);
  }
  x = mask_rot<W>(x, j, n, nm);
  z = mask_rot<W>(z, j, n, nm);
  Key<W> r;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    r.x(i) = x.w[i];
    r.z(i) = z.w[i];
  }
  return r;
}

template <int W>
__device__ __forceinline__ bool key_less(const Key<W>& a, const Key<W>& b);

// Set bit s of a W-word mask (compile-time word indices only).
template <int W>
__device__ __forceinline__ void mask_set(Mask<W>& m, int s) {
#pragma unroll
  for (int t = 0; t < W; ++t) m.w[t] |= (t == (s >> 6)) ? (1ull << (s & 63)) : 0ull;
}

// Strings with at most this many sites that differ from the smallest digit
// find their longest runs by walking the gaps between those sites.
constexpr int kZnGapWalk = 12;

// A run of `gap` d's ends just before site s: keep s if the run is the
// longest so far (L), alone if it is longer than all before.
template <int W>
__device__ __forceinline__ void zn_take_gap(Mask<W>& cand, int& L, int gap, int s) {
  if (gap > L) {
    L = gap;
#pragma unroll
    for (int i = 0; i < W; ++i) cand.w[i] = 0;
  }
  if (gap == L) mask_set<W>(cand, s);
}

// Z_n (Algorithm 2): the translation with the lowest digit integer.  Instead
// of comparing all n translations, the search keeps only those that can be
// lowest: the top digit of the lowest one is the smallest digit d present,
// and the longer the run of d at the top, the lower the integer (a shorter
// run is followed by a larger digit).  So the candidates put a longest
// cyclic run of d on the top qubits n-L..n-1, that is, translate by j where
// j is the site just after the run.  The runs are found in one of two ways,
// both giving every longest run:
//  * few sites differ from d (a low-weight string, d = I): walk the gaps
//    between consecutive such sites, cyclically; a gap before site s is a
//    run ending just before s, so j = s;
//  * otherwise (runs are short): shrink the mask of d's, cur &= T cur, until
//    one more step would empty it; after L-1 steps bit p marks a window
//    p..p+L-1 of d's, and j = p + L mod n.
// The (usually one) candidates are then narrowed digit by digit on masks.
// Equal to the exhaustive search by construction; tested bit for bit against
// the oracle's enumeration.
template <int W>
__device__ __forceinline__ void canon_zn(Key<W>& k, int n) {
  const Mask<W> nm = nbits_mask<W>(n);
  Mask<W> sup, dm;
  bool any_i = false, any_x = false, any_y = false;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    sup.w[i] = k.x(i) | k.z(i);
    any_i |= (~sup.w[i] & nm.w[i]) != 0;
    any_x |= (k.x(i) & ~k.z(i)) != 0;
    any_y |= (k.x(i) & k.z(i)) != 0;
  }
  // mask of the smallest digit present: I, else X, else Y, else Z
#pragma unroll
  for (int i = 0; i < W; ++i) {
    dm.w[i] = any_i ? (~sup.w[i] & nm.w[i])
                    : (any_x ? (k.x(i) & ~k.z(i)) : (any_y ? (k.x(i) & k.z(i)) : (k.z(i) & ~k.x(i))));
  }
  Mask<W> E;  // sites that differ from d
  int n_other = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    E.w[i] = ~dm.w[i] & nm.w[i];
    n_other += __popcll(E.w[i]);
  }
  if (n_other == 0) return;  // one letter everywhere: every translation is the same string
  Mask<W> cand;
#pragma unroll
  for (int i = 0; i < W; ++i) cand.w[i] = 0;
  int L = -1;  // length of the longest runs
  if (n_other <= kZnGapWalk) {
    int first = -1, prev = -1;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      uint64_t m = E.w[i];
      while (m) {
        const int s = 64 * i + __ffsll((long long)m) - 1;
        m &= m - 1;
        if (first < 0) first = s;
        else zn_take_gap<W>(cand, L, s - prev - 1, s);
        prev = s;
      }
    }
    zn_take_gap<W>(cand, L, first + n - prev - 1, first);  // the run wrapping past qubit n-1
  } else {
    Mask<W> cur = dm;
    L = 1;
    for (;;) {
      const Mask<W> r = mask_rot<W>(cur, 1, n, nm);
      Mask<W> nx;
#pragma unroll
      for (int i = 0; i < W; ++i) nx.w[i] = cur.w[i] & r.w[i];
      if (!mask_any<W>(nx)) break;
      cur = nx;
      ++L;
    }
    cand = mask_rot<W>(cur, n - L, n, nm);  // bit p of cur -> bit (p + L) mod n
  }
  // The candidates share the run on the top L qubits.  Below it, digit by
  // digit from the top, keep the candidates with the smallest digit (high
  // bit, then low bit of the digit), all candidates at once on masks; after
  // kZnNarrow digits (or all n - L, when several left give the same string)
  // any candidates still tied are compared as whole rotated strings.
  constexpr int kZnNarrow = 2;
  Mask<W> zp, lp;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    zp.w[i] = k.z(i);
    lp.w[i] = k.x(i) ^ k.z(i);
  }
  for (int kk = 1; kk <= kZnNarrow && kk <= n - L && mask_many<W>(cand); ++kk) {
    const int sft = n - L - kk;  // bit j of the rotation = the digit at j - L - kk
    const Mask<W> hi = mask_rot<W>(zp, sft, n, nm);
    Mask<W> c0;
    bool any0 = false;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      c0.w[i] = cand.w[i] & ~hi.w[i];
      any0 |= c0.w[i] != 0;
    }
    if (any0) cand = c0;
    const Mask<W> lo = mask_rot<W>(lp, sft, n, nm);
    Mask<W> c1;
    bool any1 = false;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      c1.w[i] = cand.w[i] & ~lo.w[i];
      any1 |= c1.w[i] != 0;
    }
    if (any1) cand = c1;
  }
  Key<W> best = k;
  bool first_c = true;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint64_t m = cand.w[i];
    while (m) {
      const int j = 64 * i + __ffsll((long long)m) - 1;
      m &= m - 1;
      const Key<W> r = rotate_key<W>(k, j, n, nm);
      if (first_c || key_less<W>(r, best)) best = r;
      first_c = false;
    }
  }
  k = best;
}

__device__ __forceinline__ uint64_t range_word(int w, int lo, int hi) {
  int a = lo - 64 * w, b = hi - 64 * w;
  a = a < 0 ? 0 : a;
  b = b > 64 ? 64 : b;
  if (b <= a) return 0ull;
  const uint64_t upto_b = (b == 64) ? ~0ull : ((1ull << b) - 1ull);
  const uint64_t below_a = (1ull << a) - 1ull;  // a < 64 here
  return upto_b & ~below_a;
}

// S_n (Algorithm 3): count n_X, n_Y, n_Z and write Z^{nZ} Y^{nY} X^{nX} I...
template <int W>
__device__ __forceinline__ void canon_sn(Key<W>& k) {
  int nx = 0, ny = 0, nz = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    nx += __popcll(k.x(j) & ~k.z(j));
    ny += __popcll(k.x(j) & k.z(j));
    nz += __popcll(k.z(j) & ~k.x(j));
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    k.z(j) = range_word(j, 0, nz + ny);
    k.x(j) = range_word(j, nz, nz + ny + nx);
  }
}

// Digit-integer order of Definition "Lowest integer representation": the
// first differing digit from the most significant qubit decides.
template <int W>
__device__ __forceinline__ bool key_less(const Key<W>& a, const Key<W>& b) {
#pragma unroll
  for (int j = W - 1; j >= 0; --j) {
    const uint64_t la = a.x(j) ^ a.z(j), lb = b.x(j) ^ b.z(j);  // low digit bits
    const uint64_t diff = (a.z(j) ^ b.z(j)) | (la ^ lb);
    if (diff) {
      const int q = 63 - __clzll((long long)diff);
      const int va = (int)(((a.z(j) >> q) & 1ull) << 1 | ((la >> q) & 1ull));
      const int vb = (int)(((b.z(j) >> q) & 1ull) << 1 | ((lb >> q) & 1ull));
      return va < vb;
    }
  }
  return false;
}

// Reflection of the ring: the letter of qubit q moves to qubit n-1-q.
template <int W>
__device__ __forceinline__ Key<W> reflect_key(const Key<W>& k, int n) {
  Key<W> r;
  if constexpr (W == 1) {
    r.x(0) = __brevll(k.x(0)) >> (64 - n);
    r.z(0) = __brevll(k.z(0)) >> (64 - n);
  } else {
    // reversing the word order and the bits of every word sends bit q to
    // bit 64 W - 1 - q; a shift right by 64 W - n brings it to n - 1 - q
    Mask<W> xm, zm;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      xm.w[j] = __brevll(k.x(W - 1 - j));
      zm.w[j] = __brevll(k.z(W - 1 - j));
    }
    xm = mask_shr<W>(xm, 64 * W - n);
    zm = mask_shr<W>(zm, 64 * W - n);
#pragma unroll
    for (int j = 0; j < W; ++j) {
      r.x(j) = xm.w[j];
      r.z(j) = zm.w[j];
    }
  }
  return r;
}

// D_n (rotations and reflections of a ring): the lower of the Z_n
// representatives of the string and of its reflection, since every
// reflection is a rotation of the one reflection above.
template <int W>
__device__ __forceinline__ void canon_dn(Key<W>& k, int n) {
  Key<W> r = reflect_key<W>(k, n);
  canon_zn<W>(k, n);
  canon_zn<W>(r, n);
  if (key_less<W>(r, k)) k = r;
}

// Translations of an lx x (n / lx) torus, qubit q = x + lx y: lowest digit
// integer over all (dx, dy).  One word: a translation is a cyclic shift of
// every row by dx (masks) and of the whole string by lx * dy.
__device__ __forceinline__ uint64_t rot_bits(uint64_t m, int s, int n, uint64_t nmask) {
  return s == 0 ? m : (((m << s) | (m >> (n - s))) & nmask);
}

__device__ __forceinline__ void canon_torus_w1(Key<1>& k, int n, int lx) {
  typedef unsigned __int128 u128;
  const int ly = n / lx;
  const uint64_t nmask = (n == 64) ? ~0ull : ((1ull << n) - 1ull);
  const uint64_t x = k.x(0), z = k.z(0);
  auto dig = [](uint64_t xx, uint64_t zz) {
    return (u128)digits32((uint32_t)xx, (uint32_t)zz) |
           ((u128)digits32((uint32_t)(xx >> 32), (uint32_t)(zz >> 32)) << 64);
  };
  u128 best = dig(x, z);
  uint64_t bx = x, bz = z;
  for (int dx = 0; dx < lx; ++dx) {
    // columns [0, lx - dx) move up by dx, the rest wrap down by lx - dx
    uint64_t low = 0;
    const uint64_t row = (lx - dx >= 64) ? ~0ull : ((1ull << (lx - dx)) - 1ull);
    for (int y = 0; y < ly; ++y) low |= row << (lx * y);  // lx * y < n <= 64
    const uint64_t high = nmask & ~low;
    const uint64_t sx = dx == 0 ? x : (((x & low) << dx) | ((x & high) >> (lx - dx)));
    const uint64_t sz = dx == 0 ? z : (((z & low) << dx) | ((z & high) >> (lx - dx)));
    for (int dy = 0; dy < ly; ++dy) {
      const uint64_t tx = rot_bits(sx, lx * dy, n, nmask), tz = rot_bits(sz, lx * dy, n, nmask);
      const u128 v = dig(tx, tz);
      if (v < best) {
        best = v;
        bx = tx;
        bz = tz;
      }
    }
  }
  k.x(0) = bx;
  k.z(0) = bz;
}

template <int W>
__device__ __forceinline__ int torus_src(int q, int dx, int dy, int lx, int ly) {
  int x = q % lx - dx, y = q / lx - dy;
  x += (x < 0) ? lx : 0;
  y += (y < 0) ? ly : 0;
  return x + lx * y;
}

// Several words: compare translations digit by digit from the most
// significant qubit (the letter at q comes from torus_src(q)).
template <int W>
__device__ __forceinline__ void canon_torus_generic(Key<W>& k, int n, int lx) {
  const int ly = n / lx;
  int bdx = 0, bdy = 0;
  for (int dy = 0; dy < ly; ++dy)
    for (int dx = 0; dx < lx; ++dx) {
      if (dx == 0 && dy == 0) continue;
      int cmp = 0;
      for (int q = n - 1; q >= 0 && cmp == 0; --q) {
        const int a = digit_at<W>(k, torus_src<W>(q, dx, dy, lx, ly));
        const int b = digit_at<W>(k, torus_src<W>(q, bdx, bdy, lx, ly));
        cmp = (a < b) ? -1 : ((a > b) ? 1 : 0);
      }
      if (cmp < 0) {
        bdx = dx;
        bdy = dy;
      }
    }
  if (bdx == 0 && bdy == 0) return;
  Key<W> r;
#pragma unroll
  for (int j = 0; j < 2 * W; ++j) r.w[j] = 0;
  for (int q = 0; q < n; ++q) {
    const int src = torus_src<W>(q, bdx, bdy, lx, ly);
    r.x(q >> 6) |= ((k.x(src >> 6) >> (src & 63)) & 1ull) << (q & 63);
    r.z(q >> 6) |= ((k.z(src >> 6) >> (src & 63)) & 1ull) << (q & 63);
  }
  k = r;
}

// Group codes: 0 none, 1 Z_n, 2 S_n, 3 D_n, 4 torus translations (lattice
// width lx passed separately).
template <int W, int G>
__device__ __forceinline__ void canon(Key<W>& k, int n, int lx) {
  if constexpr (G == 1) {
    canon_zn<W>(k, n);
  } else if constexpr (G == 2) {
    canon_sn<W>(k);
  } else if constexpr (G == 3) {
    canon_dn<W>(k, n);
  } else if constexpr (G == 4) {
    if constexpr (W == 1) {
      canon_torus_w1(k, n, lx);
    } else {
      canon_torus_generic<W>(k, n, lx);
    }
  }
}

// ------------------------------------------------------------- overlap

template <int W>
__device__ __forceinline__ double overlap_plain(const Key<W>& k, const OverlapArgs& a) {
  if (a.basis) {
    uint64_t xo = 0;
    int par = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      xo |= k.x(j);
      par += __popcll(k.z(j) & a.bits[j]);
    }
    if (xo) return 0.0;
    return (par & 1) ? -1.0 : 1.0;
  }
  double v = 1.0;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    uint64_t m = k.x(j) | k.z(j);
    while (m) {
      const int b = __ffsll((long long)m) - 1;
      m &= m - 1;
      const int q = 64 * j + b;
      const int xb = (int)((k.x(j) >> b) & 1ull), zb = (int)((k.z(j) >> b) & 1ull);
      const int l = xb ? (zb ? 1 : 0) : 2;  // X -> 0, Y -> 1, Z -> 2
      v *= a.bloch[3 * q + l];
    }
  }
  return v;
}

// Average of Tr[rho T^j r] over the n translations.
template <int W>
__device__ __forceinline__ double overlap_zn(const Key<W>& k, const OverlapArgs& a) {
  const int n = a.n;
  double acc = 0.0;
  if (a.basis) {
    uint64_t xo = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) xo |= k.x(j);
    if (xo) return 0.0;
    for (int s = 0; s < n; ++s) {
      int par = 0;
#pragma unroll
      for (int j = 0; j < W; ++j) {
        uint64_t m = k.z(j);
        while (m) {
          const int b = __ffsll((long long)m) - 1;
          m &= m - 1;
          int q = 64 * j + b - s;
          q += (q < 0) ? n : 0;
          par += (int)((a.bits[q >> 6] >> (q & 63)) & 1ull);
        }
      }
      acc += (par & 1) ? -1.0 : 1.0;
    }
    return acc / (double)n;
  }
  for (int s = 0; s < n; ++s) {
    double v = 1.0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      uint64_t m = k.x(j) | k.z(j);
      while (m) {
        const int b = __ffsll((long long)m) - 1;
        m &= m - 1;
        int q = 64 * j + b - s;
        q += (q < 0) ? n : 0;
        const int xb = (int)((k.x(j) >> b) & 1ull), zb = (int)((k.z(j) >> b) & 1ull);
        const int l = xb ? (zb ? 1 : 0) : 2;
        v *= a.bloch[3 * q + l];
      }
    }
    acc += v;
  }
  return acc / (double)n;
}

// Average of Tr[rho g r] over the elements g of D_n (2n: q -> j +- q) or of
// the torus translations (lx * ly: (x, y) -> (x + dx, y + dy)).
template <int W>
__device__ __forceinline__ double overlap_group(const Key<W>& k, const OverlapArgs& a) {
  const int n = a.n;
  const bool dn = a.group == 3;
  const int lx = dn ? 1 : a.lx, ly = dn ? 1 : n / a.lx;
  const int n_el = dn ? 2 * n : n;
  double acc = 0.0;
  for (int e = 0; e < n_el; ++e) {
    const int j = dn ? (e >> 1) : 0, refl = dn ? (e & 1) : 0;
    const int dx = dn ? 0 : e % lx, dy = dn ? 0 : e / lx;
    double v = 1.0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t m = k.x(w) | k.z(w);
      while (m) {
        const int b = __ffsll((long long)m) - 1;
        m &= m - 1;
        const int q = 64 * w + b;
        int t;
        if (dn) {
          t = refl ? (j - q) : (j + q);
          t %= n;
          t += (t < 0) ? n : 0;
        } else {
          const int x = (q % lx + dx) % lx, y = (q / lx + dy) % ly;
          t = x + lx * y;
        }
        const int xb = (int)((k.x(w) >> b) & 1ull), zb = (int)((k.z(w) >> b) & 1ull);
        const int l = xb ? (zb ? 1 : 0) : 2;  // X -> 0, Y -> 1, Z -> 2
        v *= a.bloch[3 * t + l];
      }
    }
    acc += v;
  }
  return acc / (double)n_el;
}

template <int W>
__device__ __forceinline__ double overlap_sn(const Key<W>& k, const OverlapArgs& a) {
  int nx = 0, ny = 0, nz = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    nx += __popcll(k.x(j) & ~k.z(j));
    ny += __popcll(k.x(j) & k.z(j));
    nz += __popcll(k.z(j) & ~k.x(j));
  }
  const int S = a.n + 1;
  return a.sn_table[((size_t)nx * S + ny) * S + nz];
}

__device__ __forceinline__ double ld_coef(const double* c, uint64_t i) { return __ldcg(c + i); }

// Find key k among the entries that existed when the gate started (dense
// position < T0); slots of this gate's births are skipped without reading
// their keys, so births need no fence before they are published.  With
// load_coef, a candidate's coefficient is loaded together with its key and
// stored to *c on a match: one dependent round trip fewer for a caller that
// needs the coefficient of the entry it finds.
template <int W>
__device__ __forceinline__ int64_t index_find_old(const DevTable& t, const Key<W>& k, uint64_t h,
                                                  uint32_t tag, uint64_t T0, unsigned& err,
                                                  bool load_coef = false, double* c = nullptr,
                                                  bool need = true) {
  uint64_t pos = h & t.imask;
  for (uint64_t probe = 0; probe <= t.imask; ++probe) {
    const uint64_t s = __ldcg(reinterpret_cast<const unsigned long long*>(t.index) + pos);
    if (s == 0) return -1;
    // a caller with nothing to do whether or not the key is stored gives up
    // here; `need` is evaluated only now, so its own loads overlap the first
    // slot's
    if (!need) return -3;
    if ((uint32_t)(s >> 32) == tag) {
      const uint32_t idx = (uint32_t)s;
      if ((uint64_t)idx < T0) {
        const double cc = load_coef ? ld_coef(t.coef, idx) : 0.0;
        if (keys_equal(ld_key_cg<W>(t.keys, idx), k)) {
          if (load_coef) *c = cc;
          return (int64_t)idx;
        }
      }
    }
    pos = (pos + 1) & t.imask;
  }
  err |= kErrProbe;
  return -2;
}

}  // namespace
}  // namespace ppk
