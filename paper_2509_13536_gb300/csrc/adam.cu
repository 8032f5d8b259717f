// Optimiser step and loss helper, sm_103a.  Both are streaming (HBM-bound) kernels:
// one launch covers every parameter array, each element is read and written once.
#include "internal.h"

namespace mgs {
namespace {

struct AdamSeg {
  void* p;          // parameter (f32/f16/bf16)
  int dtype;
  float* g;
  float* m;
  float* v;
  int64_t n;
  int64_t start;    // first global element of this segment
};
struct AdamArgs {
  AdamSeg seg[5];
  int nseg;
  int64_t total;
  float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
  int zero_grads;
};

template <typename T>
__device__ __forceinline__ void adam_one(T* p, float* g, float* m, float* v, int64_t i,
                                         const AdamArgs& a) {
  float gi = g[i];
  if (a.zero_grads) g[i] = 0.f;
  float mi = a.b1 * m[i] + (1.f - a.b1) * gi;
  float vi = a.b2 * v[i] + (1.f - a.b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float mh = mi / a.c1, vh = vi / a.c2;
  float x = ld(p + i) - a.lr * mh / (sqrtf(vh) + a.eps);
  st(p + i, x);
}

__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamArgs a) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int s = 0;
    while (s + 1 < a.nseg && a.seg[s + 1].start <= k) ++s;
    const AdamSeg& S = a.seg[s];
    int64_t i = k - S.start;
    switch (S.dtype) {
      case MGS_F16: adam_one((__half*)S.p, S.g, S.m, S.v, i, a); break;
      case MGS_BF16: adam_one((__nv_bfloat16*)S.p, S.g, S.m, S.v, i, a); break;
      default: adam_one((float*)S.p, S.g, S.m, S.v, i, a); break;
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
  AdamArgs a{};
  a.zero_grads = zero_grads;
  const int64_t n = p.n;
  const int64_t K3 = (int64_t)(p.sh_degree + 1) * (p.sh_degree + 1) * 3;
  struct { void* p; int dt; float* g; float* m; float* v; int64_t n; } list[5] = {
      {p.means, MGS_F32, g.means, m.means, v.means, 3 * n},
      {p.log_scales, p.attr_dtype, g.log_scales, m.log_scales, v.log_scales, 3 * n},
      {p.quats, p.attr_dtype, g.quats, m.quats, v.quats, 4 * n},
      {p.opacity_logit, p.attr_dtype, g.opacity_logit, m.opacity_logit, v.opacity_logit, n},
      {p.sh, p.attr_dtype, g.sh, m.sh, v.sh, K3 * n}};
  int64_t start = 0;
  for (int k = 0; k < 5; ++k) {
    a.seg[k] = AdamSeg{list[k].p, list[k].dt, list[k].g, list[k].m, list[k].v, list[k].n, start};
    start += list[k].n;
  }
  a.nseg = 5;
  a.total = start;
  a.lr = lr; a.b1 = b1; a.b2 = b2; a.eps = eps;
  a.c1 = 1.f - powf(b1, (float)step);
  a.c2 = 1.f - powf(b2, (float)step);
  if (a.total == 0) return cudaSuccess;
  int64_t blocks = std::min<int64_t>(div_up(a.total, 256), (int64_t)sm_count() * 8);
  k_adam<<<(unsigned)blocks, 256, 0, s>>>(a);
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
