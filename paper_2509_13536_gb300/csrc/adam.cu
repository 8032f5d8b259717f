// Optimiser step and loss helper, sm_103a.  Both are streaming (HBM-bound) kernels:
// one launch covers every parameter array, each element is read and written once.
#include <cmath>

#include "internal.h"

namespace mgs {
namespace {

struct AdamHyper {
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
  int zero_grads;
};

__device__ __forceinline__ float adam_update(float p, float& g, float& m, float& v, const AdamHyper& h) {
  float gi = g;
  m = h.b1 * m + (1.f - h.b1) * gi;
  v = h.b2 * v + (1.f - h.b2) * gi * gi;
  if (h.zero_grads) g = 0.f;
  return p - h.lr * (m / h.c1) / (sqrtf(v / h.c2) + h.eps);
}

// The parameter arrays of one step: block b works on the segment whose block range
// holds b; each thread owns 4 consecutive elements (16-byte vector accesses on the f32
// gradient and moment arrays).
struct AdamSeg {
  void* p;
  float* g;
  float* m;
  float* v;
  int64_t n;
  int dt;          // storage type of p
  int block_end;   // one past the last block of this segment
};
struct AdamTable {
  AdamSeg seg[5];
  int n_seg;
};
constexpr int kAdamThreads = 256;
constexpr int kAdamUnroll = 2;  // 16-byte groups per thread, strided by the block's width
constexpr int kAdamPerBlock = 4 * kAdamThreads * kAdamUnroll;

template <typename T>
__device__ __forceinline__ void adam_seg(T* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                         float* __restrict__ v, int64_t n, int64_t i, const AdamHyper& h) {
  if (i >= n) return;
  if (i + 4 <= n) {
    float4 gg = *reinterpret_cast<float4*>(g + i), mm = *reinterpret_cast<float4*>(m + i),
           vv = *reinterpret_cast<float4*>(v + i);
    float pp[4];
    if constexpr (sizeof(T) == 4) {
      float4 q = *reinterpret_cast<float4*>(p + i);
      pp[0] = q.x; pp[1] = q.y; pp[2] = q.z; pp[3] = q.w;
    } else {
      for (int k = 0; k < 4; ++k) pp[k] = ld(p + i + k);
    }
    pp[0] = adam_update(pp[0], gg.x, mm.x, vv.x, h);
    pp[1] = adam_update(pp[1], gg.y, mm.y, vv.y, h);
    pp[2] = adam_update(pp[2], gg.z, mm.z, vv.z, h);
    pp[3] = adam_update(pp[3], gg.w, mm.w, vv.w, h);
    *reinterpret_cast<float4*>(m + i) = mm;
    *reinterpret_cast<float4*>(v + i) = vv;
    if (h.zero_grads) *reinterpret_cast<float4*>(g + i) = gg;
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p + i) = make_float4(pp[0], pp[1], pp[2], pp[3]);
    } else {
      for (int k = 0; k < 4; ++k) st(p + i + k, pp[k]);
    }
  } else {
    for (int64_t k = i; k < n; ++k) {
      float gk = g[k], mk = m[k], vk = v[k];
      float x = adam_update(ld(p + k), gk, mk, vk, h);
      m[k] = mk;
      v[k] = vk;
      if (h.zero_grads) g[k] = gk;
      st(p + k, x);
    }
  }
}

__global__ void __launch_bounds__(kAdamThreads) k_adam(const __grid_constant__ AdamTable tab, const AdamHyper h) {
  int s = 0;
  while (s + 1 < tab.n_seg && (int)blockIdx.x >= tab.seg[s].block_end) ++s;
  const AdamSeg& q = tab.seg[s];
  const int b0 = s ? tab.seg[s - 1].block_end : 0;
  const int64_t i0 = (int64_t)((int)blockIdx.x - b0) * kAdamPerBlock + 4 * threadIdx.x;
#pragma unroll
  for (int u = 0; u < kAdamUnroll; ++u) {
    const int64_t i = i0 + (int64_t)u * 4 * kAdamThreads;
    switch (q.dt) {  // uniform per block
      case MGS_F16: adam_seg((__half*)q.p, q.g, q.m, q.v, q.n, i, h); break;
      case MGS_BF16: adam_seg((__nv_bfloat16*)q.p, q.g, q.m, q.v, q.n, i, h); break;
      default: adam_seg((float*)q.p, q.g, q.m, q.v, q.n, i, h); break;
    }
  }
}

__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ pred, const float* __restrict__ target,
                                            int64_t n, float scale, float* __restrict__ grad,
                                            float* __restrict__ loss) {
  float acc = 0.f;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float d = pred[k] - target[k];
    grad[k] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
    acc += fabsf(d);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, acc * scale);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

}  // namespace

cudaError_t launch_adam(const mgs_gaussians_mut& p, const mgs_grads& g, const mgs_grads& m,
                        const mgs_grads& v, float lr, float b1, float b2, float eps, int step,
                        int zero_grads, cudaStream_t s) {
  // Bias corrections 1 - beta^t in double: in float32, 1 - powf(0.999, 2) keeps only ~4
  // significant digits (the rounding of beta^2 is ~1e-5 of the difference), which moved
  // second-step updates by ~1e-5 relative.  Rounded once to float, they now cancel with
  // the (1 - beta) factors of the moment updates as in exact arithmetic.
  AdamHyper h{lr, b1, b2, eps, (float)(1.0 - std::pow((double)b1, (double)step)),
              (float)(1.0 - std::pow((double)b2, (double)step)), zero_grads};
  const int64_t n = p.n;
  const int64_t K3 = (int64_t)(p.sh_degree + 1) * (p.sh_degree + 1) * 3;
  struct Seg { void* p; int dt; float* g; float* m; float* v; int64_t n; } list[5] = {
      {p.means, MGS_F32, g.means, m.means, v.means, 3 * n},
      {p.log_scales, p.geom_dtype, g.log_scales, m.log_scales, v.log_scales, 3 * n},
      {p.quats, p.quat_dtype, g.quats, m.quats, v.quats, 4 * n},
      {p.opacity_logit, p.attr_dtype, g.opacity_logit, m.opacity_logit, v.opacity_logit, n},
      {p.sh, p.attr_dtype, g.sh, m.sh, v.sh, K3 * n}};
  AdamTable tab{};
  int64_t blocks = 0;
  for (const Seg& q : list) {
    if (q.n <= 0) continue;
    blocks += div_up(q.n, kAdamPerBlock);
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    tab.seg[tab.n_seg++] = AdamSeg{q.p, q.g, q.m, q.v, q.n, q.dt, (int)blocks};
  }
  if (blocks == 0) return cudaSuccess;
  k_adam<<<(unsigned)blocks, kAdamThreads, 0, s>>>(tab, h);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_l1(const float* pred, const float* target, int64_t n, float scale, float* grad,
                      float* loss, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = std::min<int64_t>(div_up(n, 256), (int64_t)sm_count() * 8);
  k_l1<<<(unsigned)blocks, 256, 0, s>>>(pred, target, n, scale, grad, loss);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgs
