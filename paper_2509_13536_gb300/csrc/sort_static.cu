// mgs_sort_pairs_noalloc: the radix sort of mgs_sort_pairs for callers that cannot
// allocate device memory.  Its scratch is one file-scope __device__ array, so every
// GPU that loads the library holds it (about 13 MB) until the process exits.
#include <mutex>

#include "internal.h"

namespace mgs {
namespace {

constexpr int64_t kMax = MGS_SORT_NOALLOC_MAX;
// key and value ping-pong buffers, the identity-permutation buffer, then the
// histogram / scan scratch of radix_sort_pairs (sort_scratch_words(kMax) fits in 1<<17)
constexpr size_t kScratchWords = size_t(1) << 17;
constexpr size_t kWords = 3 * size_t(kMax) + kScratchWords;

__device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

std::mutex g_mu;
void* g_addr[256];  // device address of g_noalloc_scratch, per device ordinal

// Host code may not use g_noalloc_scratch as a pointer: its host-side name is a
// stand-in.  Look up the device address once per device, with that device current.
cudaError_t scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<uint32_t*>(g_addr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, uint32_t* vals_out, int64_t n,
                                             int32_t begin_bit, int32_t end_bit, void* stream) {
  set_error("");
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit) {
    set_error("need n >= 0 and 0 <= begin_bit < end_bit <= 32");
    return MGS_ERR_INVALID;
  }
  if (n > kMax) {
    set_error("n = " + std::to_string(n) + " exceeds MGS_SORT_NOALLOC_MAX = " + std::to_string(kMax) +
              "; use mgs_sort_pairs with a workspace");
    return MGS_ERR_UNSUPPORTED;
  }
  if (n > 0 && (!keys || (!vals && !vals_out))) {
    set_error("NULL keys or values");
    return MGS_ERR_INVALID;
  }
  if ((size_t)sort_scratch_words(kMax) > kScratchWords) {
    set_error("internal: static sort scratch too small");
    return MGS_ERR_UNSUPPORTED;
  }
  uint32_t* base = nullptr;
  MGS_TRY_CUDA(scratch_for_current_device(&base));
  if (n == 0) return MGS_OK;
  uint32_t* kalt = base;
  uint32_t* valt = base + kMax;
  uint32_t* vtmp = base + 2 * kMax;
  uint32_t* scratch = base + 3 * kMax;
  const bool iota = vals == nullptr;
  uint32_t* vdst = iota ? vals_out : vals;
  uint32_t* K[2] = {keys, kalt};
  uint32_t* V[2] = {iota ? vtmp : vals, valt};
  cudaError_t e;
  int cur = radix_sort_pairs(K, V, n, begin_bit, end_bit, iota, scratch, s, &e);
  if (e != cudaSuccess) return cuda_status(e, "radix sort");
  if (cur == 1) MGS_TRY_CUDA(cudaMemcpyAsync(keys, kalt, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  if (V[cur] != vdst) MGS_TRY_CUDA(cudaMemcpyAsync(vdst, V[cur], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  return MGS_OK;
}
