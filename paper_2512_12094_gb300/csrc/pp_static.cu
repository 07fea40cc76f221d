// pp_merge_terms_noalloc: the identical-string / orbit merge of
// pp_merge_terms for callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc / cudaMallocAsync are not
// allowed once it is running -- for example a serving loop whose device
// memory is sized when it starts and may not grow afterwards (an allocation
// later could fail under load, or stall the device while it synchronises), or
// an embedding application that hands out every device allocation from its
// own pool.  Such a caller still owns its inputs and outputs
// and passes them in; the only memory this call needs beyond them (a hash
// index and a small control block) lives in the static device array below.
//
// The array is loaded with the library: every GPU on which the library is
// used holds it (kScratchBytes, about 8 MiB) until the process exits.  All
// calls on a device share it, so calls whose work overlaps on that device
// (different streams, or different host threads) race and must be
// serialised by the caller.  Each call clears the part of the array it uses
// before using it; the contents left behind are those of the last call.
#include <mutex>
#include <string>

#include "../../include/pp.h"
#include "pp_internal.h"

namespace ppk {
namespace {

// Index slots of the scratch hash table: a power of two holding at least twice
// the number of input terms.
constexpr uint64_t kStaticIndexSlots = 1ull << 20;
constexpr int64_t kStaticMaxTerms = (int64_t)(kStaticIndexSlots / 2);  // 524288
constexpr size_t kIndexBytes = kStaticIndexSlots * sizeof(unsigned long long);
constexpr size_t kCtlOffset = (kIndexBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtlOffset + (sizeof(DevCtl) + 255) / 256 * 256;

// Scratch of pp_merge_terms_noalloc: [index slots | control block].
static __device__ __align__(256) unsigned char g_merge_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_merge_scratch on the current device, looked up once per
// device (the name of the array in host code is only a host-side handle).
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_merge_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Zero the index slots this call uses and the control block.
__global__ void clear_scratch_kernel(unsigned long long* index, uint64_t slots, DevCtl* ctl) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride)
    index[i] = 0ull;
  if (blockIdx.x == 0) {
    unsigned* w = reinterpret_cast<unsigned*>(ctl);
    for (unsigned k = threadIdx.x; k < sizeof(DevCtl) / 4; k += blockDim.x) w[k] = 0u;
  }
}

// Number of distinct strings, or -1 when the merge kernel reported an error.
__global__ void write_count_kernel(const DevCtl* ctl, int64_t* m_out) {
  *m_out = ctl->error ? -1 : (int64_t)ctl->n_next;
}

uint64_t pow2_at_least(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace
}  // namespace ppk

using namespace ppk;

extern "C" pp_status pp_merge_terms_noalloc(int n_qubits, int symmetry, int64_t m,
                                            const uint64_t* keys_in, const double* coef_in,
                                            uint64_t* keys_out, double* coef_out,
                                            int64_t* m_out_dev, void* stream) {
  if (n_qubits < 1 || n_qubits > 64 * kMaxW) {
    set_last_error("pp_merge_terms_noalloc: n_qubits must be in 1..256");
    return PP_ERR_ARG;
  }
  if (!valid_group_code(symmetry, n_qubits)) {
    set_last_error("pp_merge_terms_noalloc: unknown symmetry");
    return PP_ERR_ARG;
  }
  if (m < 0 || !m_out_dev || (m > 0 && (!keys_in || !coef_in || !keys_out || !coef_out))) {
    set_last_error("pp_merge_terms_noalloc: bad sizes or null arrays");
    return PP_ERR_ARG;
  }
  if (m > kStaticMaxTerms) {
    set_last_error("pp_merge_terms_noalloc: at most " + std::to_string(kStaticMaxTerms) +
                   " input terms (the static scratch index holds " +
                   std::to_string(kStaticIndexSlots) + " slots); got " + std::to_string(m));
    return PP_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    set_last_error(std::string("pp_merge_terms_noalloc: cudaGetSymbolAddress: ") +
                   cudaGetErrorString(e));
    return PP_ERR_CUDA;
  }
  unsigned long long* index = reinterpret_cast<unsigned long long*>(base);
  DevCtl* ctl = reinterpret_cast<DevCtl*>(base + kCtlOffset);
  const uint64_t slots = pow2_at_least(2 * (uint64_t)(m > 0 ? m : 1));
  const int W = (n_qubits + 63) / 64;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const uint64_t want = ((uint64_t)m + kBlock * 4 - 1) / (kBlock * 4);
  const int grid = (int)(want < 1 ? 1 : (want > (uint64_t)sms * 8 ? (uint64_t)sms * 8 : want));
  clear_scratch_kernel<<<sms, kBlock, 0, s>>>(index, slots, ctl);
  e = cudaGetLastError();
  if (e == cudaSuccess && m > 0) {
    DevTable dst = {};
    dst.keys = keys_out;
    dst.coef = coef_out;
    dst.index = reinterpret_cast<uint64_t*>(index);
    dst.cap = (uint64_t)m;
    dst.imask = slots - 1;
    e = launch_merge_insert(W, symmetry, n_qubits, -1, grid, s, keys_in, coef_in, (uint64_t)m,
                            nullptr, 0, dst, ctl);
  }
  if (e == cudaSuccess) {
    write_count_kernel<<<1, 1, 0, s>>>(ctl, m_out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_last_error(std::string("pp_merge_terms_noalloc: ") + cudaGetErrorString(e));
    return PP_ERR_CUDA;
  }
  return PP_OK;
}
