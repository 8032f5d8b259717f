// Device-wide exclusive scan and stable LSD radix sort (8-bit digits) for sm_103a.
//
// Reduce-then-scan structure, no inter-block waiting: every pass is a histogram
// kernel, a scan of the digit-major histogram table, and a stable scatter.  Blocks
// own 4096 consecutive items; inside a block, items are ranked round by round (256
// at a time) with warp peer masks (match instruction, or one ballot per digit bit) and
// per-warp digit counters in shared memory, which keeps equal keys in input order.
#include "internal.h"

namespace mgs {
namespace {

constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// --- scan ---
// n_dev (optional): the item count in device memory, at most n (the grid's size); the
// kernels below take it in place of n, so a launch sized for a capacity needs no host
// round trip to learn the count.
__device__ __forceinline__ int64_t count_of(int64_t n, const uint32_t* n_dev) {
  return n_dev ? min(n, (int64_t)*n_dev) : n;
}

__global__ void __launch_bounds__(kSortThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              const uint32_t* __restrict__ gather,
                                                              int64_t n, uint32_t* __restrict__ sums,
                                                              const uint32_t* __restrict__ n_dev) {
  n = count_of(n, n_dev);
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) {  // a block past the device count (grid sized for a capacity)
    if (threadIdx.x == 0) sums[blockIdx.x] = 0u;
    return;
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kSortPerThread; ++i) {
    int64_t k = base + i * kSortThreads + threadIdx.x;
    if (k < n) acc += in[gather ? gather[k] : k];
  }
  __shared__ uint32_t s[kWarps];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kWarps; ++w) t += s[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of sums[0..nb) in place by one block; sums[nb] = total.
__global__ void __launch_bounds__(1024) k_scan_spine(uint32_t* sums, int64_t nb, uint32_t* total) {
  __shared__ uint32_t s[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t k = base + threadIdx.x;
    uint32_t x = k < nb ? sums[k] : 0u;
    uint32_t inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((threadIdx.x & 31) >= o) inc += y;
    }
    if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint32_t w = s[threadIdx.x], wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (threadIdx.x >= o) wi += y;
      }
      s[threadIdx.x] = wi - w;
    }
    __syncthreads();
    uint32_t excl = carry + s[threadIdx.x >> 5] + inc - x;
    if (k < nb) sums[k] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[nb] = carry;
    if (total) *total = carry;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_scan_down(const uint32_t* in,
                                                            const uint32_t* __restrict__ gather,
                                                            int64_t n, const uint32_t* __restrict__ sums,
                                                            uint32_t* out, const uint32_t* __restrict__ n_dev) {
  n = count_of(n, n_dev);
  __shared__ uint32_t tile[kSortTile];
  __shared__ uint32_t s[kWarps];
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;  // nothing of this block's range exists
#pragma unroll
  for (int i = 0; i < kSortPerThread; ++i) {
    int idx = i * kSortThreads + threadIdx.x;
    int64_t k = base + idx;
    tile[idx] = k < n ? in[gather ? gather[k] : k] : 0u;
  }
  __syncthreads();
  uint32_t loc[kSortPerThread];
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kSortPerThread; ++i) {
    loc[i] = acc;
    acc += tile[threadIdx.x * kSortPerThread + i];
  }
  uint32_t inc = acc;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if ((threadIdx.x & 31) >= o) inc += y;
  }
  if ((threadIdx.x & 31) == 31) s[threadIdx.x >> 5] = inc;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wpre += s[w];
  uint32_t off = sums[blockIdx.x] + wpre + inc - acc;
#pragma unroll
  for (int i = 0; i < kSortPerThread; ++i) tile[threadIdx.x * kSortPerThread + i] = off + loc[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortPerThread; ++i) {
    int idx = i * kSortThreads + threadIdx.x;
    int64_t k = base + idx;
    if (k < n) out[k] = tile[idx];
  }
}

// --- radix sort ---
// Per-block digit histogram of one pass.  Each thread reads 16 consecutive keys with
// vector loads and counts runs of equal digits in registers; a run costs one atomic
// on the warp's private shared histogram (keys emitted per Gaussian, and high digits,
// come in long runs).
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             int64_t n, int shift, uint32_t mask, int nb,
                                                             uint32_t* __restrict__ hist, bool drop,
                                                             const uint32_t* __restrict__ n_dev) {
  n = count_of(n, n_dev);
  const int t = threadIdx.x, w = t >> 5;
  if ((int64_t)blockIdx.x * kSortTile >= n) {  // past the device count: an empty column
    hist[(int64_t)t * nb + blockIdx.x] = 0;
    return;
  }
  __shared__ uint32_t h[kWarps][256];
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) h[ww][t] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * kSortTile + (int64_t)t * kSortPerThread;
  uint32_t k[kSortPerThread];
  // i0 is a multiple of 16 keys, so keys + i0 is 16-byte aligned exactly when keys is;
  // a caller's 4-byte aligned array (an offset view) takes the scalar path
  if (i0 + kSortPerThread <= n && (reinterpret_cast<uintptr_t>(keys) & 15) == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(keys + i0);
#pragma unroll
    for (int q = 0; q < kSortPerThread / 4; ++q) {
      const uint4 v = p[q];
      k[4 * q] = v.x; k[4 * q + 1] = v.y; k[4 * q + 2] = v.z; k[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kSortPerThread; ++q) k[q] = i0 + q < n ? keys[i0 + q] : 0u;
  }
  const int m = (int)(n - i0 < kSortPerThread ? (n - i0 > 0 ? n - i0 : 0) : kSortPerThread);
  if (m > 0) {
    // dropped keys (drop: key == kSortDrop) count under the out-of-range digit 256
    uint32_t cur = (drop && k[0] == kSortDrop) ? 256u : (k[0] >> shift) & mask, cnt = 1;
#pragma unroll
    for (int q = 1; q < kSortPerThread; ++q) {
      if (q < m) {
        const uint32_t d = (drop && k[q] == kSortDrop) ? 256u : (k[q] >> shift) & mask;
        if (d == cur) {
          ++cnt;
        } else {
          if (cur < 256u) atomicAdd(&h[w][cur], cnt);
          cur = d;
          cnt = 1;
        }
      }
    }
    if (cur < 256u) atomicAdd(&h[w][cur], cnt);
  }
  __syncthreads();
  uint32_t tot = 0;
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) tot += h[ww][t];
  hist[(int64_t)t * nb + blockIdx.x] = tot;
}

// Stable scatter of one pass.  Warp w owns the contiguous items [512 w, 512 w + 512) of
// the block's 4096 and ranks them round by round (32 at a time) with peer masks and
// warp-local digit counters, so stability needs no block barrier per round.  One
// block-wide prefix over the warps' counts then gives every item its position in the
// block's digit-sorted order; items are staged in shared memory in that order and
// written out as coalesced runs per digit.
template <bool kBallot>
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t n, int shift,
    uint32_t mask, int nb, const uint32_t* __restrict__ hist, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, bool drop, const uint32_t* __restrict__ n_dev, uint32_t* __restrict__ rng,
    uint32_t n_valid) {
  n = count_of(n, n_dev);
  if ((int64_t)blockIdx.x * kSortTile >= n) return;  // past the device count: nothing to move
  constexpr int kPerWarp = kSortTile / kWarps;  // 512
  constexpr int kRounds = kPerWarp / 32;        // 16
  __shared__ uint32_t s_wcnt[kWarps][256];      // per-warp digit counts, then exclusive offsets
  __shared__ uint32_t s_goff[256];              // global start of (digit, this block)
  __shared__ uint32_t s_boff[256];              // start of the digit in the block's sorted order
  __shared__ uint32_t s_key[kSortTile];
  __shared__ uint32_t s_val[kSortTile];
  __shared__ uint32_t s_nkeep;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const int n_here = (int)(n - base < kSortTile ? n - base : (int64_t)kSortTile);
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) s_wcnt[ww][t] = 0;
  s_goff[t] = hist[(int64_t)t * nb + blockIdx.x];
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  const int nbits = __popc(mask);
  uint32_t key[kRounds], val[kRounds], rank[kRounds];
  // all 32 loads of the warp's segment in flight before the ranking starts
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int i = w * kPerWarp + r * 32 + lane;
    const bool valid = i < n_here;
    key[r] = valid ? __ldcs(kin + base + i) : 0u;
    val[r] = valid ? (vin ? __ldcs(vin + base + i) : (uint32_t)(base + i)) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int i = w * kPerWarp + r * 32 + lane;
    const bool valid = i < n_here && !(drop && key[r] == kSortDrop);
    const uint32_t d = valid ? (key[r] >> shift) & mask : 256u;
    // lanes holding the same digit: the match instruction costs more the more distinct
    // digits a round holds, the ballot form (one ballot per digit bit) costs the same
    // for any round
    uint32_t peers;
    if (kBallot) {
      peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (b < nbits) {
          const bool bit = (d >> b) & 1u;
          const uint32_t bal = __ballot_sync(0xffffffffu, bit);
          peers &= bit ? bal : ~bal;
        }
      }
    } else {
      peers = __match_any_sync(0xffffffffu, d);
    }
    const uint32_t before = valid ? s_wcnt[w][d] : 0u;
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) s_wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // thread t = digit t: offsets of the warps within the digit, and the digit's block start
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t c = s_wcnt[ww][t];
      s_wcnt[ww][t] = run;
      run += c;
    }
    // exclusive scan of the per-digit block totals (run) over the 256 digits
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    __shared__ uint32_t s_wsum[kWarps];
    if (lane == 31) s_wsum[w] = inc;
    __syncthreads();
    uint32_t pre = 0;
    for (int ww = 0; ww < w; ++ww) pre += s_wsum[ww];
    s_boff[t] = pre + inc - run;
    if (t == kSortThreads - 1) s_nkeep = pre + inc;  // items of this block that are kept
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int i = w * kPerWarp + r * 32 + lane;
    if (i < n_here && !(drop && key[r] == kSortDrop)) {
      const uint32_t d = (key[r] >> shift) & mask;
      const uint32_t pos = s_boff[d] + s_wcnt[w][d] + rank[r];
      s_key[pos] = key[r];
      s_val[pos] = val[r];
    }
  }
  __syncthreads();
  for (int i = t; i < (int)s_nkeep; i += kSortThreads) {
    const uint32_t k = s_key[i];
    const uint32_t d = (k >> shift) & mask;
    const uint32_t pos = s_goff[d] + (uint32_t)i - s_boff[d];
    if (!rng) kout[pos] = k;  // a ranged sort keeps the ranges and values, not the keys
    vout[pos] = s_val[i];
    if (rng && k < n_valid) {
      // Ranges of equal keys, on the last pass: the block's run of digit d is sorted by
      // key (earlier passes sorted the lower digits), so a change of key inside the run
      // is a range boundary; a run's first and last keys may continue in the runs of the
      // neighbouring blocks, so those take atomic min / max (rng: (first, end) pairs).
      const uint32_t ii = (uint32_t)i, re = d < 255 ? s_boff[d + 1] : s_nkeep;
      if (ii == s_boff[d]) atomicMin(rng + 2 * k, pos);
      else if (s_key[i - 1] != k) rng[2 * k] = pos;
      if (ii + 1 == re) atomicMax(rng + 2 * k + 1, pos + 1);
      else if (s_key[i + 1] != k) rng[2 * k + 1] = pos + 1;
    }
  }
}

__global__ void k_ranges_init(uint2* __restrict__ ranges, uint32_t n) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) ranges[t] = make_uint2(0xffffffffu, 0u);
}

__global__ void k_ranges_fix(uint2* __restrict__ ranges, uint32_t n) {  // keys absent: empty range
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && ranges[t].x == 0xffffffffu) ranges[t] = make_uint2(0u, 0u);
}


}  // namespace

int64_t sort_scratch_words(int64_t n) {
  int64_t nb = div_up(std::max<int64_t>(n, 1), kSortTile);
  int64_t hist = 256 * nb;
  int64_t spine = div_up(std::max<int64_t>(hist, n), kSortTile) + 1;
  return align_up((size_t)hist, 64) + align_up((size_t)spine, 64);
}

cudaError_t scan_exclusive_u32(const uint32_t* in, const uint32_t* gather, uint32_t* out,
                               int64_t n, uint32_t* scratch, uint32_t* total_dev, cudaStream_t s,
                               const uint32_t* n_dev) {
  if (n <= 0) {
    if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
    return cudaSuccess;
  }
  int64_t nb = div_up(n, kSortTile);
  uint32_t* sums = scratch;
  k_scan_reduce<<<(unsigned)nb, kSortThreads, 0, s>>>(in, gather, n, sums, n_dev);
  k_scan_spine<<<1, 1024, 0, s>>>(sums, nb, total_dev);
  k_scan_down<<<(unsigned)nb, kSortThreads, 0, s>>>(in, gather, n, sums, out, n_dev);
  count_launch(3);
  return cudaGetLastError();
}

int radix_sort_pairs(uint32_t* k[2], uint32_t* v[2], int64_t n, int begin_bit, int end_bit,
                     bool vals_iota, uint32_t* scratch, cudaStream_t s, cudaError_t* err, int64_t n_keep,
                     const uint32_t* n_dev, const uint32_t* n_keep_dev, uint2* ranges, uint32_t n_valid) {
  *err = cudaSuccess;
  int cur = 0;
  if (ranges) {  // every key value below n_valid starts empty; the last pass fills the ranges
    k_ranges_init<<<(unsigned)div_up(std::max<uint32_t>(n_valid, 1), 256), 256, 0, s>>>(ranges, n_valid);
    count_launch();
  }
  if (n <= 0) {
    if (ranges) {
      k_ranges_fix<<<(unsigned)div_up(std::max<uint32_t>(n_valid, 1), 256), 256, 0, s>>>(ranges, n_valid);
      count_launch();
      *err = cudaGetLastError();
    }
    return 0;
  }
  bool drop = n_keep >= 0;  // first pass drops kSortDrop keys; n_keep of them remain
  uint32_t* hist = scratch;
  uint32_t* spine = scratch + align_up((size_t)256 * div_up(n, kSortTile), 64);
  bool first = true;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    if (n <= 0) break;
    const int nb = (int)div_up(n, kSortTile);
    const uint32_t mask = (1u << std::min(8, end_bit - shift)) - 1u;
    k_radix_hist<<<nb, kSortThreads, 0, s>>>(k[cur], n, shift, mask, nb, hist, drop, n_dev);
    count_launch(2);
    *err = scan_exclusive_u32(hist, nullptr, hist, (int64_t)256 * nb, spine, nullptr, s);
    if (*err != cudaSuccess) return cur;
    const uint32_t* vin = (first && vals_iota) ? nullptr : v[cur];
    // Full 8-bit digits below the top byte take the ballot form: there (low bytes of tile
    // ids, middle bytes of depths) a warp's 32 keys hold nearly 32 distinct digits.  The
    // top byte and the first, dropping pass of the depth sort hold few distinct digits
    // per round and keep the match instruction.
    uint32_t* rng = (ranges && shift + 8 >= end_bit) ? reinterpret_cast<uint32_t*>(ranges) : nullptr;
    if (mask == 0xffu && !drop && shift < 24)
      k_radix_scatter<true><<<nb, kSortThreads, 0, s>>>(k[cur], vin, n, shift, mask, nb, hist, k[cur ^ 1],
                                                        v[cur ^ 1], drop, n_dev, rng, n_valid);
    else
      k_radix_scatter<false><<<nb, kSortThreads, 0, s>>>(k[cur], vin, n, shift, mask, nb, hist, k[cur ^ 1],
                                                         v[cur ^ 1], drop, n_dev, rng, n_valid);
    cur ^= 1;
    first = false;
    if (drop) {
      // the kept keys: a host count shrinks the grid, a device count keeps the grid and
      // bounds the kernels
      if (n_keep_dev) n_dev = n_keep_dev;
      else n = n_keep;
      drop = false;
    }
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return cur;
  }
  if (first && vals_iota) {
    // no pass ran: materialise the identity permutation
    *err = cudaErrorInvalidValue;
  }
  if (ranges && *err == cudaSuccess) {
    k_ranges_fix<<<(unsigned)div_up(std::max<uint32_t>(n_valid, 1), 256), 256, 0, s>>>(ranges, n_valid);
    count_launch();
    *err = cudaGetLastError();
  }
  return cur;
}


}  // namespace mgs
