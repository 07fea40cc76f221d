// Sort-based merge: the merge loop of Algorithms 2 and 3 ("if the
// representative is already present accumulate, else insert") done as an LSD
// radix sort of the representatives followed by a segmented FP64 reduce of
// every run of equal keys, set against the open-addressing hash merge of
// pp_kernels.cu.
//
// Elements are (sort key, payload).  The sort key is the representative
// itself, packed exactly: for n <= 32 one word x | z << 32, for n <= 64 the two
// words (x, z).  The payload is the coefficient (single column) or the source
// index (batched rows, whose B columns are gathered by the reduce).  Each pass
// sorts by one byte of the key, stably, so equal keys keep their input order
// and every run is summed in input order: the merge is deterministic, unlike
// the atomic hash merge.  A pass whose byte is the same for every element is
// skipped (the device records which buffer holds the data); canonical keys of
// short strings leave many such bytes.
//
// Per pass: a histogram kernel (per-block byte counts), a scan kernel (one
// block per byte value: exclusive scan along the blocks) and a scatter kernel
// that ranks the elements of its tile stably per byte value (warp match,
// then a running count per byte value in shared memory) and writes them to
// their final positions.  Pass 0 also drops the elements the filter rejects.
#include <algorithm>

#include "pp_device.cuh"

namespace ppk {
namespace {

constexpr int kST = 256;                 // threads per sort block
constexpr int kSItems = 8;               // elements per thread per tile
constexpr int kSTile = kST * kSItems;    // elements per tile
constexpr int kSWarps = kST / 32;
constexpr int kMaxPasses = 16;
constexpr int kLongRun = 64;             // runs longer than this are summed by a warp

// Device bookkeeping of one sorted merge (in the scratch block).
struct SortCtl {
  unsigned long long T;       // input elements (before the filter)
  unsigned long long m;       // elements after the filter
  unsigned long long base;    // first output position in the destination table
  unsigned long long total;   // distinct keys (runs)
  unsigned long long n_long;  // runs longer than kLongRun
  int sel[kMaxPasses + 1];    // buffer (0 / 1) holding the data entering pass p
  unsigned err;
};

struct SortBufs {
  uint64_t* k0[2];  // sort key word 0 (x | z << 32, or x)
  uint64_t* k1[2];  // sort key word 1 (z) when KW = 2
  uint64_t* pay[2]; // coefficient bits or source index
  unsigned char* keep;
  unsigned* hist;   // [256][NB] counts, scanned in place
  unsigned* tot;    // [256] per-byte totals of the current pass
  unsigned* btot;   // [NB] runs per reduce block, scanned in place
  unsigned* headpos;  // [m] sorted position of the first element of each run
  unsigned* longrun;  // [m] runs handed to the warp reduce
  SortCtl* sc;
};

__device__ __forceinline__ bool stalled(const DevCtl* ctl, int guarded) {
  return guarded && queued_layer_stopped(ctl);
}

// Byte `pos` (0..15) of the sort key (word 0 holds bytes 0..7).
template <int KW>
__device__ __forceinline__ unsigned byte_of(uint64_t a, uint64_t b, int pos) {
  const uint64_t w = (KW == 2 && pos >= 8) ? b : a;
  return (unsigned)(w >> (8 * (pos & 7))) & 0xFFu;
}

// Representative of every input string, packed as a sort key, with the
// payload and the filter flag, at its input position.
template <int W, int G, int KW>
__global__ void __launch_bounds__(kST)
    sort_prep_kernel(const uint64_t* __restrict__ src_keys, const double* __restrict__ src_coef,
                     const unsigned char* __restrict__ src_alive, uint64_t count,
                     const unsigned long long* count_dev, int skip_zero, int wmax, int n, int lx,
                     SortBufs sb, const DevCtl* ctl, int guarded) {
  if (stalled(ctl, guarded)) return;
  const uint64_t T = count_dev ? *count_dev : count;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sb.sc->T = T;
    sb.sc->sel[0] = 0;
    sb.sc->err = 0;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T; i += stride) {
    bool keep;
    uint64_t pay;
    if (src_coef) {
      const double c = src_coef[i];
      keep = !(skip_zero && c == 0.0);
      pay = (uint64_t)__double_as_longlong(c);
    } else {
      keep = src_alive == nullptr || src_alive[i] != 0;
      pay = i;
    }
    Key<W> K = ld_key<W>(src_keys, i);
    if (wmax >= 0 && weight(K) > wmax) keep = false;
    canon<W, G>(K, n, lx);
    if (KW == 1) {
      sb.k0[0][i] = K.x(0) | (K.z(0) << 32);
    } else {
      sb.k0[0][i] = K.x(0);
      sb.k1[0][i] = K.z(0);
    }
    sb.pay[0][i] = pay;
    sb.keep[i] = keep ? 1 : 0;
  }
}

// Pass q sorts by byte `pos` of the key.
template <int KW, bool P0>
__global__ void __launch_bounds__(kST)
    sort_hist_kernel(SortBufs sb, int q, int pos, const DevCtl* ctl, int guarded) {
  __shared__ unsigned s_h[256];
  if (stalled(ctl, guarded)) return;
  const uint64_t N = P0 ? sb.sc->T : sb.sc->m;
  const int cur = sb.sc->sel[q];
  const uint64_t* k0 = sb.k0[cur];
  const uint64_t* k1 = sb.k1[cur];
  s_h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t0 = (uint64_t)blockIdx.x * kSTile;
#pragma unroll
  for (int r = 0; r < kSItems; ++r) {
    const uint64_t e = t0 + (uint64_t)r * kST + threadIdx.x;
    if (e < N && (!P0 || sb.keep[e])) {
      const unsigned d = byte_of<KW>(k0[e], KW == 2 ? k1[e] : 0ull, pos);
      atomicAdd(&s_h[d], 1u);
    }
  }
  __syncthreads();
  sb.hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s_h[threadIdx.x];
}

// One block per byte value: exclusive scan of its counts along the blocks.
__global__ void __launch_bounds__(kST) sort_scan_kernel(SortBufs sb, int nb, const DevCtl* ctl,
                                                        int guarded) {
  __shared__ unsigned s_w[kSWarps];
  __shared__ unsigned s_carry;
  if (stalled(ctl, guarded)) return;
  unsigned* row = sb.hist + (size_t)blockIdx.x * nb;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nb; c0 += kST) {
    const int i = c0 + threadIdx.x;
    const unsigned v = i < nb ? row[i] : 0u;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned wbase = 0, all = 0;
    for (int w = 0; w < kSWarps; ++w) {
      wbase += (w < warp) ? s_w[w] : 0u;
      all += s_w[w];
    }
    const unsigned carry = s_carry;
    if (i < nb) row[i] = carry + wbase + x - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) sb.tot[blockIdx.x] = s_carry;
}

// Stable scatter of one pass.  Pass 0 reads the prepared elements with their
// filter flags and writes only the kept ones.  A later pass whose byte is the
// same for all elements moves nothing (the next pass reads the same buffer).
template <int KW, bool P0>
__global__ void __launch_bounds__(kST)
    sort_scatter_kernel(SortBufs sb, int q, int pos, const DevCtl* ctl, int guarded) {
  __shared__ unsigned s_base[256];            // global start of each byte value
  __shared__ unsigned s_cnt[kSWarps][256];    // per-warp counts, then prefixes
  __shared__ unsigned s_run[256];             // elements of each value so far in the tile
  __shared__ int s_skip;
  if (stalled(ctl, guarded)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t N = P0 ? sb.sc->T : sb.sc->m;
  const int cur = sb.sc->sel[q];
  {
    // exclusive scan of the 256 per-byte totals (one value per thread)
    const unsigned v = sb.tot[tid];
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_cnt[0][warp] = x;
    if (tid == 0) s_skip = 0;
    __syncthreads();
    unsigned wb = 0, all = 0;
    for (int w = 0; w < kSWarps; ++w) {
      wb += (w < warp) ? s_cnt[0][w] : 0u;
      all += s_cnt[0][w];
    }
    s_base[tid] = wb + x - v;
    if (!P0 && (uint64_t)v == N && N > 0) s_skip = 1;  // every element has this byte
    __syncthreads();
    if (blockIdx.x == 0 && tid == 0) {
      const int skip = s_skip;
      sb.sc->sel[q + 1] = skip ? cur : 1 - cur;
      if (P0) sb.sc->m = all;
    }
    for (int w = 0; w < kSWarps; ++w) s_cnt[w][tid] = 0;
    s_run[tid] = 0;
    __syncthreads();
  }
  if (s_skip) return;
  const uint64_t* ik0 = sb.k0[cur];
  const uint64_t* ik1 = sb.k1[cur];
  const uint64_t* ipay = sb.pay[cur];
  uint64_t* ok0 = sb.k0[1 - cur];
  uint64_t* ok1 = sb.k1[1 - cur];
  uint64_t* opay = sb.pay[1 - cur];
  const unsigned nb = gridDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * kSTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSItems; ++r) {
    const uint64_t e = t0 + (uint64_t)r * kST + tid;
    const bool valid = e < N && (!P0 || sb.keep[e]);
    uint64_t a = 0, b = 0, p = 0;
    unsigned d = 256;  // a value no element has: invalid lanes group together
    if (valid) {
      a = ik0[e];
      if (KW == 2) b = ik1[e];
      p = ipay[e];
      d = byte_of<KW>(a, b, pos);
    }
    const unsigned peers = __match_any_sync(kFull, d);
    const unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      // running prefix over the warps, in warp order, for byte value tid
      unsigned x = s_run[tid];
      for (int w = 0; w < kSWarps; ++w) {
        const unsigned c = s_cnt[w][tid];
        s_cnt[w][tid] = x;
        x += c;
      }
      s_run[tid] = x;
    }
    __syncthreads();
    if (valid) {
      const uint64_t pos = (uint64_t)s_base[d] + sb.hist[(size_t)d * nb + blockIdx.x] +
                           s_cnt[warp][d] + rank;
      ok0[pos] = a;
      if (KW == 2) ok1[pos] = b;
      opay[pos] = p;
    }
    __syncthreads();
    for (int w = 0; w < kSWarps; ++w) s_cnt[w][tid] = 0;
    __syncthreads();
  }
}

template <int KW>
__device__ __forceinline__ bool same_key(const SortBufs& sb, int buf, uint64_t i, uint64_t j) {
  return sb.k0[buf][i] == sb.k0[buf][j] && (KW == 1 || sb.k1[buf][i] == sb.k1[buf][j]);
}

// Runs per block of the sorted elements (a run starts where the key changes).
template <int KW>
__global__ void __launch_bounds__(kST)
    run_count_kernel(SortBufs sb, int passes, const DevCtl* ctl, int guarded) {
  __shared__ unsigned s_w[kSWarps];
  if (stalled(ctl, guarded)) return;
  const uint64_t m = sb.sc->m;
  const int buf = sb.sc->sel[passes];
  const uint64_t t0 = (uint64_t)blockIdx.x * kSTile;
  unsigned c = 0;
  for (int r = 0; r < kSItems; ++r) {
    const uint64_t j = t0 + (uint64_t)r * kST + threadIdx.x;
    if (j < m && (j == 0 || !same_key<KW>(sb, buf, j, j - 1))) ++c;
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned s = 0;
    for (int w = 0; w < kSWarps; ++w) s += s_w[w];
    sb.btot[blockIdx.x] = s;
  }
}

// Exclusive scan of the runs per block (one block); places the output at the
// destination table's append cursor and advances it.
__global__ void __launch_bounds__(1024) run_scan_kernel(SortBufs sb, int nb, DevCtl* ctl,
                                                        int guarded) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  if (stalled(ctl, guarded)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const unsigned long long v = i < nb ? sb.btot[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned long long wb = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      wb += (w < warp) ? s_w[w] : 0ull;
      all += s_w[w];
    }
    const unsigned long long carry = s_carry;
    if (i < nb) sb.btot[i] = (unsigned)(carry + wb + x - v);
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + all;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long base = ctl->n_next;
    sb.sc->base = base;
    sb.sc->total = s_carry;
    sb.sc->n_long = 0;
    ctl->n_next = base + s_carry;
  }
}

// Sorted position of the first element of every run.
template <int KW>
__global__ void __launch_bounds__(kST)
    run_heads_kernel(SortBufs sb, int passes, const DevCtl* ctl, int guarded) {
  __shared__ unsigned s_w[kSWarps];
  __shared__ unsigned s_carry;
  if (stalled(ctl, guarded)) return;
  const uint64_t m = sb.sc->m;
  const int buf = sb.sc->sel[passes];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t t0 = (uint64_t)blockIdx.x * kSTile;
  if (threadIdx.x == 0) s_carry = sb.btot[blockIdx.x];
  __syncthreads();
  for (int r = 0; r < kSItems; ++r) {
    const uint64_t j = t0 + (uint64_t)r * kST + threadIdx.x;
    const bool head = j < m && (j == 0 || !same_key<KW>(sb, buf, j, j - 1));
    const unsigned bal = __ballot_sync(kFull, head);
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    unsigned wb = 0, all = 0;
    for (int w = 0; w < kSWarps; ++w) {
      wb += (w < warp) ? s_w[w] : 0u;
      all += s_w[w];
    }
    const unsigned carry = s_carry;
    if (head) sb.headpos[carry + wb + __popc(bal & ((1u << lane) - 1u))] = (unsigned)j;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + all;
    __syncthreads();
  }
}

template <int W, int KW>
__device__ __forceinline__ Key<W> unpack_key(uint64_t a, uint64_t b) {
  Key<W> K;
#pragma unroll
  for (int j = 0; j < 2 * W; ++j) K.w[j] = 0;
  if (KW == 1) {
    K.x(0) = a & 0xFFFFFFFFull;
    K.z(0) = a >> 32;
  } else {
    K.x(0) = a;
    K.z(0) = b;
  }
  return K;
}

// One thread per run: the run's key and its coefficient sum (input order)
// into the destination table, and the key into its index.  Runs longer than
// kLongRun are left to run_long_kernel.
template <int W, int KW>
__global__ void __launch_bounds__(kST)
    run_sum_kernel(SortBufs sb, int passes, DevTable dst, int with_index, DevCtl* ctl,
                   int guarded) {
  if (stalled(ctl, guarded)) return;
  const uint64_t m = sb.sc->m, total = sb.sc->total, base = sb.sc->base;
  const int buf = sb.sc->sel[passes];
  const uint64_t* k0 = sb.k0[buf];
  const uint64_t* k1 = sb.k1[buf];
  const uint64_t* pay = sb.pay[buf];
  unsigned err = 0;
  OccAcc<W> occ;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
    const uint64_t j0 = sb.headpos[r];
    const uint64_t j1 = (r + 1 < total) ? (uint64_t)sb.headpos[r + 1] : m;
    const uint64_t idx = base + r;
    if (idx >= dst.cap) {
      err |= kErrAppend;
      continue;
    }
    const Key<W> K = unpack_key<W, KW>(k0[j0], KW == 2 ? k1[j0] : 0ull);
    st_key<W>(dst.keys, idx, K);
    occ.add(K);
    if (j1 - j0 <= (uint64_t)kLongRun) {
      double s = 0.0;
      for (uint64_t j = j0; j < j1; ++j) s = __dadd_rn(s, __longlong_as_double((long long)pay[j]));
      dst.coef[idx] = s;
    } else {
      const unsigned long long q = atomicAdd(&sb.sc->n_long, 1ull);
      sb.longrun[q] = (unsigned)r;
    }
    if (with_index) {
      const uint64_t h = key_hash(K);
      index_claim(dst, h & dst.imask, ((uint64_t)tag_of(h) << 32) | idx, err);
    }
  }
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

// One warp per long run: lane l sums elements l, l + 32, ... of the run in
// order, then the warp adds the 32 partial sums in a fixed tree.
__global__ void __launch_bounds__(kST)
    run_long_kernel(SortBufs sb, int passes, DevTable dst, const DevCtl* ctl, int guarded) {
  if (stalled(ctl, guarded)) return;
  const uint64_t m = sb.sc->m, total = sb.sc->total, base = sb.sc->base, nl = sb.sc->n_long;
  const uint64_t* pay = sb.pay[sb.sc->sel[passes]];
  const int lane = threadIdx.x & 31;
  const uint64_t wstride = (uint64_t)gridDim.x * kSWarps;
  for (uint64_t q = (uint64_t)blockIdx.x * kSWarps + (threadIdx.x >> 5); q < nl; q += wstride) {
    const uint64_t r = sb.longrun[q];
    const uint64_t j0 = sb.headpos[r];
    const uint64_t j1 = (r + 1 < total) ? (uint64_t)sb.headpos[r + 1] : m;
    double s = 0.0;
    for (uint64_t j = j0 + lane; j < j1; j += 32)
      s = __dadd_rn(s, __longlong_as_double((long long)pay[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kFull, s, o));
    if (lane == 0 && base + r < dst.cap) dst.coef[base + r] = s;
  }
}

// Batched rows: one warp per run sums the source rows of its elements in
// input order (lane l owns columns l, l + 32, ...), stores the row in the
// destination's element type, sets liveness by the any-column rule and adds
// the live count; lane 0 writes the key and claims its index slot.
template <int W, int KW, typename S, typename T>
__global__ void __launch_bounds__(kST)
    run_rows_kernel(SortBufs sb, int passes, const S* __restrict__ src_rows, DevTable dst,
                    int with_index, double eps, DevCtl* ctl, int guarded) {
  if (stalled(ctl, guarded)) return;
  constexpr int kCols = 512 / 32;  // B <= 512
  const uint64_t m = sb.sc->m, total = sb.sc->total, base = sb.sc->base;
  const int buf = sb.sc->sel[passes];
  const int lane = threadIdx.x & 31;
  const int B = dst.B;
  T* rows = static_cast<T*>(dst.rows);
  const bool use_eps = eps > 0.0;
  const T teps = (T)eps;  // liveness is decided in the storage type, as by the hash merge
  unsigned err = 0;
  long long live = 0;
  OccAcc<W> occ;
  const uint64_t wstride = (uint64_t)gridDim.x * kSWarps;
  for (uint64_t r = (uint64_t)blockIdx.x * kSWarps + (threadIdx.x >> 5); r < total; r += wstride) {
    const uint64_t j0 = sb.headpos[r];
    const uint64_t j1 = (r + 1 < total) ? (uint64_t)sb.headpos[r + 1] : m;
    const uint64_t idx = base + r;
    if (idx >= dst.cap) {
      err |= kErrAppend;
      continue;
    }
    double acc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) acc[c] = 0.0;
    for (uint64_t j = j0; j < j1; ++j) {
      const S* sr = src_rows + sb.pay[buf][j] * (uint64_t)B;
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        const int col = lane + 32 * c;
        if (col < B) acc[c] = __dadd_rn(acc[c], (double)sr[col]);
      }
    }
    bool any = false;
    T* dr = rows + idx * (uint64_t)B;
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const int col = lane + 32 * c;
      if (col < B) {
        const T v = (T)acc[c];
        dr[col] = v;
        any |= (v < (T)0 ? -v : v) >= teps;
      }
    }
    any = __any_sync(kFull, any) || !use_eps;
    if (lane == 0) {
      const Key<W> K = unpack_key<W, KW>(sb.k0[buf][j0], KW == 2 ? sb.k1[buf][j0] : 0ull);
      st_key<W>(dst.keys, idx, K);
      occ.add(K);
      dst.alive[idx] = any ? 1 : 0;
      live += any;
      if (with_index) {
        const uint64_t h = key_hash(K);
        index_claim(dst, h & dst.imask, ((uint64_t)tag_of(h) << 32) | idx, err);
      }
    }
  }
  if (lane == 0 && live)
    atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_live), (unsigned long long)live);
  occ.flush(ctl);
  if (err) atomicOr(&ctl->error, err);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Layout of the scratch block for up to `cap` input elements.
SortBufs carve(void* scratch, uint64_t cap, int KW) {
  unsigned char* p = static_cast<unsigned char*>(scratch);
  const uint64_t nb = (cap + kSTile - 1) / kSTile;
  SortBufs sb;
  sb.sc = reinterpret_cast<SortCtl*>(p);
  p += align256(sizeof(SortCtl));
  for (int b = 0; b < 2; ++b) {
    sb.k0[b] = reinterpret_cast<uint64_t*>(p);
    p += align256(cap * 8);
    sb.k1[b] = nullptr;
    if (KW == 2) {
      sb.k1[b] = reinterpret_cast<uint64_t*>(p);
      p += align256(cap * 8);
    }
    sb.pay[b] = reinterpret_cast<uint64_t*>(p);
    p += align256(cap * 8);
  }
  sb.keep = p;
  p += align256(cap);
  sb.hist = reinterpret_cast<unsigned*>(p);
  p += align256((size_t)256 * nb * 4);
  sb.tot = reinterpret_cast<unsigned*>(p);
  p += align256(256 * 4);
  sb.btot = reinterpret_cast<unsigned*>(p);
  p += align256(nb * 4);
  sb.headpos = reinterpret_cast<unsigned*>(p);
  p += align256(cap * 4);
  sb.longrun = reinterpret_cast<unsigned*>(p);
  return sb;
}

// Bytes of the sort key that can differ between keys of n qubits.
int key_passes(int KW, int n, int* list) {
  int np = 0;
  const int bytes = (n + 7) / 8;  // of each half (KW = 1) or word (KW = 2)
  for (int h = 0; h < 2; ++h)
    for (int k = 0; k < bytes; ++k) list[np++] = (KW == 1 ? 4 * h : 8 * h) + k;
  return np;
}

template <int W, int G, int KW>
cudaError_t merge_sorted_wgk(int n, int lx, int wmax, cudaStream_t s, const uint64_t* src_keys,
                             const double* src_coef, const void* src_rows, int src_f32,
                             const unsigned char* src_alive, uint64_t count,
                             const unsigned long long* count_dev, int skip_zero, DevTable dst,
                             int with_index, double eps, DevCtl* ctl, void* scratch, int guarded) {
  const uint64_t cap = std::max<uint64_t>(count, 1);  // an upper bound when count_dev is given
  const SortBufs sb = carve(scratch, cap, KW);
  const int nb = (int)((cap + kSTile - 1) / kSTile);
  const int sms = std::max(1, device_sm_count());
  const int gs = (int)std::min<uint64_t>((cap + kST - 1) / kST, (uint64_t)sms * 8);
  sort_prep_kernel<W, G, KW><<<gs, kST, 0, s>>>(src_keys, src_coef, src_alive, count, count_dev,
                                                skip_zero, wmax, n, lx, sb, ctl, guarded);
  int list[kMaxPasses];
  const int np = key_passes(KW, n, list);
  for (int q = 0; q < np; ++q) {
    if (q == 0) {
      sort_hist_kernel<KW, true><<<nb, kST, 0, s>>>(sb, q, list[q], ctl, guarded);
    } else {
      sort_hist_kernel<KW, false><<<nb, kST, 0, s>>>(sb, q, list[q], ctl, guarded);
    }
    sort_scan_kernel<<<256, kST, 0, s>>>(sb, nb, ctl, guarded);
    if (q == 0) {
      sort_scatter_kernel<KW, true><<<nb, kST, 0, s>>>(sb, q, list[q], ctl, guarded);
    } else {
      sort_scatter_kernel<KW, false><<<nb, kST, 0, s>>>(sb, q, list[q], ctl, guarded);
    }
  }
  run_count_kernel<KW><<<nb, kST, 0, s>>>(sb, np, ctl, guarded);
  run_scan_kernel<<<1, 1024, 0, s>>>(sb, nb, ctl, guarded);
  run_heads_kernel<KW><<<nb, kST, 0, s>>>(sb, np, ctl, guarded);
  if (src_coef) {
    run_sum_kernel<W, KW><<<gs, kST, 0, s>>>(sb, np, dst, with_index, ctl, guarded);
    run_long_kernel<<<gs, kST, 0, s>>>(sb, np, dst, ctl, guarded);
  } else {
    const int gw = (int)std::min<uint64_t>((cap + kSWarps - 1) / kSWarps, (uint64_t)sms * 16);
    if (src_f32 && dst.f32)
      run_rows_kernel<W, KW, float, float><<<gw, kST, 0, s>>>(
          sb, np, static_cast<const float*>(src_rows), dst, with_index, eps, ctl, guarded);
    else if (src_f32)
      run_rows_kernel<W, KW, float, double><<<gw, kST, 0, s>>>(
          sb, np, static_cast<const float*>(src_rows), dst, with_index, eps, ctl, guarded);
    else if (dst.f32)
      run_rows_kernel<W, KW, double, float><<<gw, kST, 0, s>>>(
          sb, np, static_cast<const double*>(src_rows), dst, with_index, eps, ctl, guarded);
    else
      run_rows_kernel<W, KW, double, double><<<gw, kST, 0, s>>>(
          sb, np, static_cast<const double*>(src_rows), dst, with_index, eps, ctl, guarded);
  }
  return cudaGetLastError();
}

}  // namespace

size_t sort_merge_scratch_bytes(uint64_t count, int n) {
  const int KW = n <= 32 ? 1 : 2;
  const uint64_t cap = std::max<uint64_t>(count, 1);
  const uint64_t nb = (cap + kSTile - 1) / kSTile;
  return align256(sizeof(SortCtl)) + 2 * (KW + 1) * align256(cap * 8) + align256(cap) +
         align256((size_t)256 * nb * 4) + align256(256 * 4) + align256(nb * 4) +
         align256(cap * 4) + align256(cap * 4);
}

bool sort_merge_supported(int n) { return n >= 1 && n <= 64; }

cudaError_t launch_merge_sorted(int group, int n, int wmax, cudaStream_t s,
                                const uint64_t* src_keys, const double* src_coef,
                                const void* src_rows, int src_f32,
                                const unsigned char* src_alive, uint64_t count,
                                const unsigned long long* count_dev, int skip_zero, DevTable dst,
                                int with_index, double eps, DevCtl* ctl, void* scratch,
                                int guarded) {
  if (!sort_merge_supported(n)) return cudaErrorInvalidValue;
  const int lx = group >> 8;
#define PPS_G(GG)                                                                             \
  return n <= 32 ? merge_sorted_wgk<1, GG, 1>(n, lx, wmax, s, src_keys, src_coef, src_rows,    \
                                              src_f32, src_alive, count, count_dev, skip_zero, \
                                              dst, with_index, eps, ctl, scratch, guarded)     \
                 : merge_sorted_wgk<1, GG, 2>(n, lx, wmax, s, src_keys, src_coef, src_rows,    \
                                              src_f32, src_alive, count, count_dev, skip_zero, \
                                              dst, with_index, eps, ctl, scratch, guarded)
  switch (group & 0xFF) {
    case 0: PPS_G(0);
    case 1: PPS_G(1);
    case 2: PPS_G(2);
    case 3: PPS_G(3);
    case 4: PPS_G(4);
    default:
      return cudaErrorInvalidValue;
  }
#undef PPS_G
}

}  // namespace ppk
