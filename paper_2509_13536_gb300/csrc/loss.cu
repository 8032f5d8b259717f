// Mapping loss of Sec. II-E (Eq. 12) and its gradient with respect to the rendered
// images, plus the isotropic term on the scales, sm_103a.
//
// Per view:  L = (1-lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)) + w_depth mean [dt>0]|d - dt|
// SSIM per channel and pixel with the 11x11 Gaussian window (sigma 1.5, normalised),
// C1 = 0.01^2, C2 = 0.03^2, windows cut by the image border (zero padding).  SSIM at a
// pixel depends on x only through the window moments m1 = E[x], m2 = E[x^2], m3 = E[xy],
// so the forward pass leaves per pixel dS/dm1, dS/dm2, dS/dm3, and the reverse pass is
// the same window applied to those three maps:
//   dL/dx(p) = -lambda/n sum_q w(q-p) (dS/dm1(q) + 2 x(p) dS/dm2(q) + y(p) dS/dm3(q))
//              + (1-lambda)/n sign(x(p) - y(p)),   n = 3HW.
// Both passes stage a 32x32 output tile with a 5-pixel halo in shared memory and run
// the window as two separable 11-tap passes; a thread computes 4 neighbouring outputs
// of a pass from one 14-value strip, so each shared value is loaded once per 4 outputs.  Sums go through per-block partials that
// one block per view adds in a fixed order, so the loss is deterministic.
#include "internal.h"

namespace mgs {
namespace {

constexpr int kTX = 32, kTY = 32, kH = 5, kIX = kTX + 2 * kH, kIY = kTY + 2 * kH, kTaps = 11;
constexpr int kRB = 4;  // outputs per thread along the pass direction (register blocking)
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Window {
  float w[kTaps];
};

// Per-view planes of one call, passed by value (at most MGS_MAX_VIEWS views).
struct Planes {
  const float* x[MGS_MAX_VIEWS];   // rendered rgb [3][H][W]
  const float* y[MGS_MAX_VIEWS];   // target rgb
  const float* d[MGS_MAX_VIEWS];   // rendered depth [H][W]
  const float* dt[MGS_MAX_VIEWS];  // target depth or NULL
  float* grgb[MGS_MAX_VIEWS];      // dL/d(rendered rgb), written
  float* gd[MGS_MAX_VIEWS];        // dL/d(rendered depth), written (or NULL)
};

// Zero-padded load of an input tile of one plane into shared memory.
__device__ __forceinline__ void load_tile(float (*dst)[kIX], const float* __restrict__ src, int W, int H,
                                          int x0, int y0) {
  for (int i = threadIdx.x; i < kIX * kIY; i += blockDim.x) {
    const int ty = i / kIX, tx = i - ty * kIX;
    const int gx = x0 - kH + tx, gy = y0 - kH + ty;
    dst[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? src[(size_t)gy * W + gx] : 0.f;
  }
}

// grid (tiles_x, tiles_y, views * 3); 256 threads
__global__ void __launch_bounds__(256) k_ssim_fwd(int W, int H, const Window win,
                                                  const __grid_constant__ Planes P,
                                                  float* __restrict__ dmaps, float* __restrict__ part) {
  __shared__ float sx[kIY][kIX], sy[kIY][kIX];
  __shared__ float h[5][kIY][kTX];
  __shared__ float red[2][8];
  const int v = blockIdx.z / 3, c = blockIdx.z % 3;
  const size_t HW = (size_t)W * H;
  const float* X = P.x[v] + c * HW;
  const float* Y = P.y[v] + c * HW;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  load_tile(sx, X, W, H, x0, y0);
  load_tile(sy, Y, W, H, x0, y0);
  __syncthreads();
  // horizontal pass: input row r, output columns c0 .. c0+3
  for (int i = threadIdx.x; i < kIY * (kTX / kRB); i += blockDim.x) {
    const int r = i / (kTX / kRB), c0 = (i - r * (kTX / kRB)) * kRB;
    float xv[kTaps + kRB - 1], yv[kTaps + kRB - 1];
#pragma unroll
    for (int k = 0; k < kTaps + kRB - 1; ++k) { xv[k] = sx[r][c0 + k]; yv[k] = sy[r][c0 + k]; }
#pragma unroll
    for (int o = 0; o < kRB; ++o) {
      float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) {
        const float x = xv[o + k], y = yv[o + k], wk = win.w[k];
        a = fmaf(wk, x, a);
        b = fmaf(wk, y, b);
        aa = fmaf(wk, x * x, aa);
        bb = fmaf(wk, y * y, bb);
        ab = fmaf(wk, x * y, ab);
      }
      h[0][r][c0 + o] = a; h[1][r][c0 + o] = b; h[2][r][c0 + o] = aa; h[3][r][c0 + o] = bb; h[4][r][c0 + o] = ab;
    }
  }
  __syncthreads();
  float ssum = 0.f, l1 = 0.f;
  float* D1 = dmaps + ((size_t)blockIdx.z * 3 + 0) * HW;
  float* D2 = dmaps + ((size_t)blockIdx.z * 3 + 1) * HW;
  float* D3 = dmaps + ((size_t)blockIdx.z * 3 + 2) * HW;
  // vertical pass: output column col, output rows r0 .. r0+3
  for (int i = threadIdx.x; i < kTX * (kTY / kRB); i += blockDim.x) {
    const int col = i % kTX, r0 = (i / kTX) * kRB;
    float m[5][kRB];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      float hv[kTaps + kRB - 1];
#pragma unroll
      for (int k = 0; k < kTaps + kRB - 1; ++k) hv[k] = h[q][r0 + k][col];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) acc = fmaf(win.w[k], hv[o + k], acc);
        m[q][o] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < kRB; ++o) {
      const int r = r0 + o, gx = x0 + col, gy = y0 + r;
      if (gx >= W || gy >= H) continue;
      const float mx = m[0][o], my = m[1][o], mxx = m[2][o], myy = m[3][o], mxy = m[4][o];
      const float vx = mxx - mx * mx, vy = myy - my * my, cxy = mxy - mx * my;
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
      const float iB = 1.f / (B1 * B2);
      const float S = A1 * A2 * iB;
      ssum += S;
      const float dmu = 2.f * my * A2 * iB - S * 2.f * mx / B1;  // dS/dmu_x at fixed variances
      const float dvx = -S / B2;                                  // dS/dsigma_x^2
      const float dcxy = 2.f * A1 * iB;                           // dS/dsigma_xy
      const size_t q = (size_t)gy * W + gx;
      D1[q] = dmu - 2.f * mx * dvx - my * dcxy;
      D2[q] = dvx;
      D3[q] = dcxy;
      l1 += fabsf(sx[r + kH][col + kH] - sy[r + kH][col + kH]);
    }
  }
  // block partials (SSIM sum, L1 sum) in a fixed order
  for (int o = 16; o; o >>= 1) {
    ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ssum; red[1][threadIdx.x >> 5] = l1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    for (int k = 0; k < 8; ++k) { a += red[0][k]; b += red[1][k]; }
    const size_t bi = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[2 * bi] = a;
    part[2 * bi + 1] = b;
  }
}

// grid (tiles_x, tiles_y, views * 3); 256 threads
__global__ void __launch_bounds__(256) k_ssim_bwd(int W, int H, const Window win, float lambda,
                                                  const __grid_constant__ Planes P,
                                                  const float* __restrict__ dmaps) {
  __shared__ float t[3][kIY][kIX];
  __shared__ float h[3][kIY][kTX];
  const int v = blockIdx.z / 3, c = blockIdx.z % 3;
  const size_t HW = (size_t)W * H;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  for (int m = 0; m < 3; ++m) load_tile(t[m], dmaps + ((size_t)blockIdx.z * 3 + m) * HW, W, H, x0, y0);
  __syncthreads();
  for (int i = threadIdx.x; i < kIY * (kTX / kRB); i += blockDim.x) {
    const int r = i / (kTX / kRB), c0 = (i - r * (kTX / kRB)) * kRB;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float tv[kTaps + kRB - 1];
#pragma unroll
      for (int k = 0; k < kTaps + kRB - 1; ++k) tv[k] = t[q][r][c0 + k];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) acc = fmaf(win.w[k], tv[o + k], acc);
        h[q][r][c0 + o] = acc;
      }
    }
  }
  __syncthreads();
  const float* X = P.x[v] + c * HW;
  const float* Y = P.y[v] + c * HW;
  float* G = P.grgb[v] + c * HW;
  const float inv_n = 1.f / (3.f * (float)HW);
  for (int i = threadIdx.x; i < kTX * (kTY / kRB); i += blockDim.x) {
    const int col = i % kTX, r0 = (i / kTX) * kRB;
    float a3[3][kRB];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float hv[kTaps + kRB - 1];
#pragma unroll
      for (int k = 0; k < kTaps + kRB - 1; ++k) hv[k] = h[q][r0 + k][col];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) acc = fmaf(win.w[k], hv[o + k], acc);
        a3[q][o] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < kRB; ++o) {
      const int gx = x0 + col, gy = y0 + r0 + o;
      if (gx >= W || gy >= H) continue;
      const size_t p = (size_t)gy * W + gx;
      const float xv = X[p], yv = Y[p];
      const float dssim = a3[0][o] + 2.f * xv * a3[1][o] + yv * a3[2][o];
      const float diff = xv - yv;
      const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
      G[p] = ((1.f - lambda) * sgn - lambda * dssim) * inv_n;
    }
  }
}

// Depth residual: one thread per pixel of every view; block partials of |d - dt|.
__global__ void __launch_bounds__(256) k_depth_l1(int W, int H, float w_depth,
                                                  const __grid_constant__ Planes P, float* __restrict__ part) {
  __shared__ float red[8];
  const size_t HW = (size_t)W * H;
  const int v = blockIdx.y;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  if (p < HW) {
    const float* Dt = P.dt[v];
    float g = 0.f;
    if (Dt) {
      const float dt = Dt[p], diff = P.d[v][p] - dt;
      if (dt > 0.f) {
        acc = fabsf(diff);
        g = w_depth * (diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f)) / (float)HW;
      }
    }
    if (P.gd[v]) P.gd[v][p] = g;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int k = 0; k < 8; ++k) a += red[k];
    part[(size_t)v * gridDim.x + blockIdx.x] = a;
  }
}

// The loss with lambda = 0 (no SSIM): the rgb L1 and the depth residual of 4
// consecutive pixels per thread in one pass (16-byte accesses when every plane allows),
// block partials (0, l1) into part_rgb and the depth sums into part_depth, both at
// view v's stride.
constexpr int kFlatPx = 4 * 256;  // pixels per block of k_l1_depth

__device__ __forceinline__ float sgn(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(256) k_l1_depth(int W, int H, float w_depth, const __grid_constant__ Planes P,
                                                  bool vec, float* __restrict__ part_rgb, size_t stride_rgb,
                                                  float* __restrict__ part_depth, size_t stride_depth) {
  __shared__ float red[2][8];
  const size_t HW = (size_t)W * H;
  const int v = blockIdx.y;
  const size_t p0 = (size_t)blockIdx.x * kFlatPx + 4 * threadIdx.x;
  const float inv_rgb = 1.f / (3.f * (float)HW);
  const float* Dt = P.dt[v];
  float l1 = 0.f, dd = 0.f;
  if (vec && p0 + 4 <= HW) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 x = *reinterpret_cast<const float4*>(P.x[v] + c * HW + p0);
      const float4 y = *reinterpret_cast<const float4*>(P.y[v] + c * HW + p0);
      const float4 d = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
      l1 += fabsf(d.x) + fabsf(d.y) + fabsf(d.z) + fabsf(d.w);
      *reinterpret_cast<float4*>(P.grgb[v] + c * HW + p0) =
          make_float4(sgn(d.x) * inv_rgb, sgn(d.y) * inv_rgb, sgn(d.z) * inv_rgb, sgn(d.w) * inv_rgb);
    }
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (Dt) {
      const float4 t = *reinterpret_cast<const float4*>(Dt + p0);
      const float4 r = *reinterpret_cast<const float4*>(P.d[v] + p0);
      const float e[4] = {r.x - t.x, r.y - t.y, r.z - t.z, r.w - t.w};
      const float tt[4] = {t.x, t.y, t.z, t.w};
      float gg[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool on = tt[k] > 0.f;
        dd += on ? fabsf(e[k]) : 0.f;
        gg[k] = on ? w_depth * sgn(e[k]) / (float)HW : 0.f;
      }
      g = make_float4(gg[0], gg[1], gg[2], gg[3]);
    }
    if (P.gd[v]) *reinterpret_cast<float4*>(P.gd[v] + p0) = g;
  } else {
    for (size_t p = p0; p < p0 + 4 && p < HW; ++p) {
      for (int c = 0; c < 3; ++c) {
        const float d = P.x[v][c * HW + p] - P.y[v][c * HW + p];
        l1 += fabsf(d);
        P.grgb[v][c * HW + p] = sgn(d) * inv_rgb;
      }
      float g = 0.f;
      if (Dt) {
        const float t = Dt[p], e = P.d[v][p] - t;
        if (t > 0.f) {
          dd += fabsf(e);
          g = w_depth * sgn(e) / (float)HW;
        }
      }
      if (P.gd[v]) P.gd[v][p] = g;
    }
  }
  for (int o = 16; o; o >>= 1) {
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = l1;
    red[1][threadIdx.x >> 5] = dd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    for (int k = 0; k < 8; ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    part_rgb[2 * (v * stride_rgb + blockIdx.x)] = 0.f;
    part_rgb[2 * (v * stride_rgb + blockIdx.x) + 1] = a;
    part_depth[v * stride_depth + blockIdx.x] = b;
  }
}

// Per view: add the block partials in a fixed order (double accumulator) and weight them.
// View v's rgb partials are (ssim, l1) pairs n_rgb_parts long at v * stride_rgb, its
// depth partials n_depth_parts long at v * stride_depth.
__global__ void k_loss_reduce(int n_views, int n_rgb_parts, size_t stride_rgb, int n_depth_parts,
                              size_t stride_depth, const float* __restrict__ part_ssim,
                              const float* __restrict__ part_depth, float lambda, float w_depth,
                              double n_rgb, double n_px, float* __restrict__ loss) {
  const int v = blockIdx.x;
  __shared__ double red[3][256];
  double s = 0, l1 = 0, dd = 0;
  for (int i = threadIdx.x; i < n_rgb_parts; i += blockDim.x) {
    const size_t bi = (size_t)v * stride_rgb + i;
    s += part_ssim[2 * bi];
    l1 += part_ssim[2 * bi + 1];
  }
  for (int i = threadIdx.x; i < n_depth_parts; i += blockDim.x) dd += part_depth[(size_t)v * stride_depth + i];
  red[0][threadIdx.x] = s; red[1][threadIdx.x] = l1; red[2][threadIdx.x] = dd;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[3 * v] = (float)((1.0 - lambda) * red[1][0] / n_rgb);
    loss[3 * v + 1] = (float)(lambda * (1.0 - red[0][0] / n_rgb));
    loss[3 * v + 2] = (float)(w_depth * red[2][0] / n_px);
  }
}

// Isotropic term: w_iso/(3n) sum_i sum_k |s_ik - mean_k s_ik|, s = exp(log s); the
// gradient is added to grad_ls.  Block partials, then one block adds them in order.
template <typename T>
__global__ void __launch_bounds__(256) k_iso(int64_t n, const T* __restrict__ ls, float scale,
                                             float* __restrict__ gls, float* __restrict__ part) {
  __shared__ float red[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  if (i < n) {
    float s[3], sg[3];
    for (int k = 0; k < 3; ++k) s[k] = expf(ld(ls + 3 * i + k));
    const float mean = (s[0] + s[1] + s[2]) * (1.f / 3.f);
    float sgsum = 0.f;
    for (int k = 0; k < 3; ++k) {
      const float dl = s[k] - mean;
      acc += fabsf(dl);
      sg[k] = dl > 0.f ? 1.f : (dl < 0.f ? -1.f : 0.f);
      sgsum += sg[k];
    }
    if (gls)
      for (int k = 0; k < 3; ++k) gls[3 * i + k] += scale * (sg[k] - sgsum * (1.f / 3.f)) * s[k];
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int k = 0; k < 8; ++k) a += red[k];
    part[blockIdx.x] = a;
  }
}

__global__ void k_sum_partials(int64_t nb, const float* __restrict__ part, float scale, float* __restrict__ out) {
  __shared__ double red[256];
  double s = 0;
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)(scale * red[0]);
}

Window make_window() {
  double w[kTaps], sum = 0;
  for (int i = 0; i < kTaps; ++i) {
    const double t = i - kH;
    w[i] = std::exp(-t * t / (2 * 1.5 * 1.5));
    sum += w[i];
  }
  Window win;
  for (int i = 0; i < kTaps; ++i) win.w[i] = (float)(w[i] / sum);
  return win;
}

}  // namespace

LossLayout loss_layout(int n_views, int width, int height) {
  LossLayout L{};
  const int64_t HW = (int64_t)width * height;
  L.tiles_x = (int)div_up(width, kTX);
  L.tiles_y = (int)div_up(height, kTY);
  L.nb_ssim = L.tiles_x * L.tiles_y;
  L.nb_depth = (int)div_up(HW, 256);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  L.dmaps = take(sizeof(float) * 9 * (size_t)n_views * HW);
  L.part_ssim = take(sizeof(float) * 2 * 3 * (size_t)n_views * L.nb_ssim);
  L.part_depth = take(sizeof(float) * (size_t)n_views * L.nb_depth);
  L.bytes = off;
  return L;
}

cudaError_t launch_mapping_loss(int n_views, int width, int height, const LossLayout& L, char* ws,
                                const mgs_image* rendered, const mgs_image* target, const mgs_image* grad,
                                float lambda, float w_depth, float* loss, cudaStream_t s) {
  Planes P{};
  for (int v = 0; v < n_views; ++v) {
    P.x[v] = rendered[v].rgb;
    P.y[v] = target[v].rgb;
    P.d[v] = rendered[v].depth;
    P.dt[v] = target[v].depth;
    P.grgb[v] = grad[v].rgb;
    P.gd[v] = grad[v].depth;
  }
  float* dmaps = reinterpret_cast<float*>(ws + L.dmaps);
  float* part_ssim = reinterpret_cast<float*>(ws + L.part_ssim);
  float* part_depth = reinterpret_cast<float*>(ws + L.part_depth);
  const Window win = make_window();
  const dim3 grid(L.tiles_x, L.tiles_y, 3 * n_views);
  const double HW = (double)width * height;
  if (lambda == 0.f) {
    // one pass for the rgb L1 and the depth residual; its partials fit the SSIM layout
    // (HW / 1024 blocks per view <= 3 x 32x32 tiles, HW / 1024 <= HW / 256)
    const size_t hw = (size_t)width * height;
    bool vec = hw % 4 == 0;
    for (int v = 0; v < n_views && vec; ++v)
      for (const void* q : {(const void*)P.x[v], (const void*)P.y[v], (const void*)P.d[v], (const void*)P.dt[v],
                            (const void*)P.grgb[v], (const void*)P.gd[v]})
        vec = vec && (reinterpret_cast<uintptr_t>(q) & 15) == 0;
    const int nbf = (int)div_up(hw, (size_t)kFlatPx);
    k_l1_depth<<<dim3(nbf, n_views), 256, 0, s>>>(width, height, w_depth, P, vec, part_ssim,
                                                  (size_t)3 * L.nb_ssim, part_depth, (size_t)L.nb_depth);
    k_loss_reduce<<<n_views, 256, 0, s>>>(n_views, nbf, (size_t)3 * L.nb_ssim, nbf, (size_t)L.nb_depth,
                                          part_ssim, part_depth, lambda, w_depth, 3.0 * HW, HW, loss);
    count_launch(2);
    return cudaGetLastError();
  }
  k_ssim_fwd<<<grid, 256, 0, s>>>(width, height, win, P, dmaps, part_ssim);
  k_ssim_bwd<<<grid, 256, 0, s>>>(width, height, win, lambda, P, dmaps);
  k_depth_l1<<<dim3(L.nb_depth, n_views), 256, 0, s>>>(width, height, w_depth, P, part_depth);
  k_loss_reduce<<<n_views, 256, 0, s>>>(n_views, 3 * L.nb_ssim, (size_t)3 * L.nb_ssim, L.nb_depth,
                                        (size_t)L.nb_depth, part_ssim, part_depth, lambda, w_depth,
                                        3.0 * HW, HW, loss);
  count_launch(4);
  return cudaGetLastError();
}

size_t iso_workspace_bytes(int64_t n) { return align_up(sizeof(float) * (size_t)std::max<int64_t>(1, div_up(n, 256))); }

cudaError_t launch_iso_loss(const mgs_gaussians& g, float w_iso, float* grad_ls, float* loss, char* ws,
                            cudaStream_t s) {
  const int64_t nb = std::max<int64_t>(1, div_up(g.n, 256));
  float* part = reinterpret_cast<float*>(ws);
  const float scale = g.n > 0 ? w_iso / (3.f * (float)g.n) : 0.f;
  if (g.n > 0) {
    switch (g.geom_dtype) {
      case MGS_F16: k_iso<__half><<<(unsigned)nb, 256, 0, s>>>(g.n, (const __half*)g.log_scales, scale, grad_ls, part); break;
      case MGS_BF16: k_iso<__nv_bfloat16><<<(unsigned)nb, 256, 0, s>>>(g.n, (const __nv_bfloat16*)g.log_scales, scale, grad_ls, part); break;
      default: k_iso<float><<<(unsigned)nb, 256, 0, s>>>(g.n, (const float*)g.log_scales, scale, grad_ls, part); break;
    }
  } else {
    cudaError_t e = cudaMemsetAsync(part, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
  }
  k_sum_partials<<<1, 256, 0, s>>>(nb, part, scale, loss);
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace mgs
