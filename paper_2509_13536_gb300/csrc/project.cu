// Per-Gaussian projection (Sec. II-C, Eq. 1-2) and its reverse pass, sm_103a.
//
// Forward: one thread loads one Gaussian's parameters once for every view of the call
// and tests each view cheaply; the warp then shares out the (Gaussian, view) items that
// pass among its lanes (the Gaussian's mean and R S from shared memory, its SH row from
// L1), so the parameters cross HBM about once per call however many keyframes are drawn.
// Reverse: one thread per Gaussian, in order of its number of gradient views, sums the
// chain rule over those views.
// The camera-space mean and the projected centre are carried in double-float
// (two f32 words) so that the depth key and the pixel-space centre are correctly
// rounded; everything else is plain f32.
#include "internal.h"

namespace mgs {
namespace {

struct GaussPre {
  float mu[3];
  float qn[4], qnorm;
  float Rq[9];
  float s[3];
  float S3[6];  // xx xy xz yy yz zz
  float RS[9];  // Rq diag(s): Sigma = RS RS^T
  float o;
};

template <typename T>
__device__ __forceinline__ void load_gauss(int64_t g, const float* means, const Geom& geo, const T* ol,
                                           GaussPre& G) {
  for (int k = 0; k < 3; ++k) G.mu[k] = __ldg(means + 3 * g + k);
  float q[4];
  for (int k = 0; k < 4; ++k) q[k] = ld_dt(geo.qs, geo.qdt, 4 * g + k);
  G.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  float inv = 1.f / G.qnorm;
  for (int k = 0; k < 4; ++k) G.qn[k] = q[k] * inv;
  quat_rot(G.qn, G.Rq);
  for (int k = 0; k < 3; ++k) G.s[k] = expf(ld_dt(geo.ls, geo.dt, 3 * g + k));
  float s2[3] = {G.s[0] * G.s[0], G.s[1] * G.s[1], G.s[2] * G.s[2]};
  const float* R = G.Rq;
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) G.RS[3 * a + k] = R[3 * a + k] * G.s[k];
  G.S3[0] = R[0] * R[0] * s2[0] + R[1] * R[1] * s2[1] + R[2] * R[2] * s2[2];
  G.S3[1] = R[0] * R[3] * s2[0] + R[1] * R[4] * s2[1] + R[2] * R[5] * s2[2];
  G.S3[2] = R[0] * R[6] * s2[0] + R[1] * R[7] * s2[1] + R[2] * R[8] * s2[2];
  G.S3[3] = R[3] * R[3] * s2[0] + R[4] * R[4] * s2[1] + R[5] * R[5] * s2[2];
  G.S3[4] = R[3] * R[6] * s2[0] + R[4] * R[7] * s2[1] + R[5] * R[8] * s2[2];
  G.S3[5] = R[6] * R[6] * s2[0] + R[7] * R[7] * s2[1] + R[8] * R[8] * s2[2];
  G.o = 1.f / (1.f + expf(-ld(ol + g)));
}

template <int DEG, typename T>
__device__ __forceinline__ void load_sh(int64_t g, const T* sh, float* c) {
  constexpr int K3 = (DEG + 1) * (DEG + 1) * 3;
  const T* p = sh + g * K3;
#pragma unroll
  for (int k = 0; k < K3; ++k) c[k] = ld(p + k);
}

struct ViewGeom {
  bool ok;                // in front of the near plane with a positive-definite 2D covariance
  float tx, ty, tz;
  float u_hi, u_lo, v_hi, v_lo;
  float xr, yr;
  bool clampx, clampy;
  float T[6];             // J W
  float a, b, c;          // dilated 2D covariance
  float A, B, C;          // its inverse
  float dir[3], vnorm;
};

// Unit view direction mu - C (the camera centre as a double-float pair) and its length.
__device__ __forceinline__ void view_direction(const float mu[3], const View& V, float dir[3], float& vnorm) {
  float d[3] = {__fsub_rn(__fsub_rn(mu[0], V.C[0]), V.C_lo[0]), __fsub_rn(__fsub_rn(mu[1], V.C[1]), V.C_lo[1]),
                __fsub_rn(__fsub_rn(mu[2], V.C[2]), V.C_lo[2])};
  vnorm = sqrtf(__fmaf_rn(d[2], d[2], __fmaf_rn(d[1], d[1], __fmul_rn(d[0], d[0]))));
  const float iv = __frcp_rn(vnorm);
  dir[0] = __fmul_rn(d[0], iv); dir[1] = __fmul_rn(d[1], iv); dir[2] = __fmul_rn(d[2], iv);
}

__device__ __forceinline__ void view_geom(const GaussPre& G, const View& V, ViewGeom& P) {
  DF p[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    DF acc = two_prod(V.R[3 * r + 0], G.mu[0]);
    acc = df_add(acc, two_prod(V.R[3 * r + 1], G.mu[1]));
    acc = df_add(acc, two_prod(V.R[3 * r + 2], G.mu[2]));
    p[r] = df_add(acc, DF{V.t[r], 0.f});
  }
  P.tx = p[0].hi; P.ty = p[1].hi; P.tz = p[2].hi;
  P.ok = P.tz > V.near_z;
  if (!P.ok) return;
  DF uq = df_axpc(V.fx, df_div(p[0], p[2]), V.cx);
  DF vq = df_axpc(V.fy, df_div(p[1], p[2]), V.cy);
  P.u_hi = uq.hi; P.u_lo = uq.lo; P.v_hi = vq.hi; P.v_lo = vq.lo;
  float tz = P.tz, itz = 1.f / tz;
  P.xr = P.tx * itz;
  P.yr = P.ty * itz;
  P.clampx = P.xr < -V.limx || P.xr > V.limx;
  P.clampy = P.yr < -V.limy || P.yr > V.limy;
  float xc = fminf(V.limx, fmaxf(-V.limx, P.xr));
  float yc = fminf(V.limy, fmaxf(-V.limy, P.yr));
  float J00 = V.fx * itz, J02 = -V.fx * xc * itz, J11 = V.fy * itz, J12 = -V.fy * yc * itz;
  const float* W = V.R;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P.T[c] = J00 * W[c] + J02 * W[6 + c];
    P.T[3 + c] = J11 * W[3 + c] + J12 * W[6 + c];
  }
  // Sigma_I = T Sigma T^T + 0.3 I with Sigma = RS RS^T, formed as M M^T, M = T RS:
  // the diagonal entries are sums of squares and det(M M^T) a sum of squared 2x2 minors
  // (Cauchy-Binet), so neither cancels when the Gaussian is long along the view ray.
  const float* RS = G.RS;
  float M0[3], M1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    M0[k] = P.T[0] * RS[k] + P.T[1] * RS[3 + k] + P.T[2] * RS[6 + k];
    M1[k] = P.T[3] * RS[k] + P.T[4] * RS[3 + k] + P.T[5] * RS[6 + k];
  }
  float aa = M0[0] * M0[0] + M0[1] * M0[1] + M0[2] * M0[2];
  float cc = M1[0] * M1[0] + M1[1] * M1[1] + M1[2] * M1[2];
  P.b = M0[0] * M1[0] + M0[1] * M1[1] + M0[2] * M1[2];
  P.a = aa + kDilation;
  P.c = cc + kDilation;
  float m01 = M0[0] * M1[1] - M0[1] * M1[0];
  float m02 = M0[0] * M1[2] - M0[2] * M1[0];
  float m12 = M0[1] * M1[2] - M0[2] * M1[1];
  float det = (m01 * m01 + m02 * m02 + m12 * m12) + kDilation * (aa + cc) + kDilation * kDilation;
  P.ok = det > 0.f;
  if (!P.ok) return;
  float idet = 1.f / det;
  P.A = P.c * idet;
  P.B = -P.b * idet;
  P.C = P.a * idet;
  view_direction(G.mu, V, P.dir, P.vnorm);
}

// Tile rect of the square of half-width r around the centre (inclusive bounds).
__device__ __forceinline__ bool tile_rect(const ViewGeom& P, const View& V, int& r, int rc[4]) {
  float mid = 0.5f * (P.a + P.c), hd = 0.5f * (P.a - P.c);
  float lam = mid + sqrtf(fmaxf(0.1f, hd * hd + P.b * P.b));  // mid^2 - det, without cancellation
  r = (int)ceilf(3.f * sqrtf(lam));
  float rf = (float)r;
  float fx0 = floorf(__fsub_rn(P.u_hi, rf) * 0.0625f), fx1 = floorf(__fadd_rn(P.u_hi, rf) * 0.0625f);
  float fy0 = floorf(__fsub_rn(P.v_hi, rf) * 0.0625f), fy1 = floorf(__fadd_rn(P.v_hi, rf) * 0.0625f);
  rc[0] = (int)fmaxf(0.f, fminf(fx0, (float)V.tiles_x));
  rc[1] = (int)fmaxf(0.f, fminf(fy0, (float)V.tiles_y));
  rc[2] = (int)fminf((float)(V.tiles_x - 1), fmaxf(fx1, -1.f));
  rc[3] = (int)fminf((float)(V.tiles_y - 1), fmaxf(fy1, -1.f));
  return rc[0] <= rc[2] && rc[1] <= rc[3];
}

template <int DEG>
__device__ __forceinline__ void colour(const float* c, const float dir[3], float raw[3]) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  float Y[K];
  sh_basis<DEG>(dir, Y, nullptr);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) acc = __fmaf_rn(c[3 * k + ch], Y[k], acc);
    raw[ch] = acc;
  }
}

// Whether Gaussian (mu, largest scale smax) can be drawn in view V: false only where the
// full test (in front of the near plane, a tile rect that meets the image) must fail.
// The rect is the square of half-width ceil(3 sqrt(lambda_max)) around the projected
// centre; lambda_max <= trace = |J W R S|_F^2 + 0.6 <= smax^2 |J|_F^2 + 0.6 (R S has
// spectral norm smax, W is a rotation), and the rect's own lambda estimate exceeds
// lambda_max by at most sqrt(0.1).  The bound is widened by 1 % and 2 px; NaNs,
// overflow, or a depth within 1e-5 of the near plane leave the decision to the full
// test.
__device__ __forceinline__ bool maybe_drawn(const float mu[3], float smax, const View& V) {
  const float tz = fmaf(V.R[6], mu[0], fmaf(V.R[7], mu[1], fmaf(V.R[8], mu[2], V.t[2])));
  if (tz <= V.near_z - 1e-5f) return false;
  if (!(tz > V.near_z + 1e-5f)) return true;
  const float tx = fmaf(V.R[0], mu[0], fmaf(V.R[1], mu[1], fmaf(V.R[2], mu[2], V.t[0])));
  const float ty = fmaf(V.R[3], mu[0], fmaf(V.R[4], mu[1], fmaf(V.R[5], mu[2], V.t[1])));
  const float itz = 1.f / tz, xr = tx * itz, yr = ty * itz;
  const float xc = fminf(V.limx, fmaxf(-V.limx, xr)), yc = fminf(V.limy, fmaxf(-V.limy, yr));
  const float tr = smax * smax * (V.fx * V.fx * (1.f + xc * xc) + V.fy * V.fy * (1.f + yc * yc)) * itz * itz + 1.f;
  const float r = 3.03f * sqrtf(tr) + 2.f;
  const float u = fmaf(V.fx, xr, V.cx), v = fmaf(V.fy, yr, V.cy);
  if (!(r < 1e30f) || !(fabsf(u) < 1e30f) || !(fabsf(v) < 1e30f)) return true;
  return u - r < 16.f * (float)V.tiles_x + 1.f && u + r > -1.f && v - r < 16.f * (float)V.tiles_y + 1.f &&
         v + r > -1.f;
}

// Buckets of the reverse projection's work plan: Gaussians by the number of views they
// take a gradient from (0..MGS_MAX_VIEWS).
constexpr int kPlanBuckets = MGS_MAX_VIEWS + 1;
static_assert(kPlanBuckets <= kPlanDirtyWord, "the bucket counts end before the dirty word");
constexpr int kPreThreads = 256;
constexpr int kPreWarps = kPreThreads / 32;
constexpr int kOwnWords = 13;  // per Gaussian, for the items of its warp: mean, R S, log2 o

template <int DEG, typename T>
__global__ void __launch_bounds__(kPreThreads, 4) k_preprocess(int64_t N, const float* __restrict__ means,
                                                    const Geom geo,
                                                    const T* __restrict__ ol, const T* __restrict__ sh,
                                                    const __grid_constant__ ViewTable vt,
                                                    float4* __restrict__ rec, uint2* __restrict__ rects,
                                                    uint32_t* __restrict__ touched,
                                                    uint32_t* __restrict__ dkeys,
                                                    unsigned long long* __restrict__ counters,
                                                    float4* __restrict__ moments, uint2* __restrict__ gmask,
                                                    uint32_t* __restrict__ bcounts) {
  // Each thread takes one Gaussian through a cheap test per view (maybe_drawn) and writes
  // the empty outputs of the views it cannot be drawn in.  The (Gaussian, view) items
  // that remain -- a quarter of them on the room map, where most of the map is behind
  // the camera or outside the image -- are then dealt out to the lanes of the warp, 32 at
  // a time, so that the full projection, the SH colour and the tile count run with every
  // lane busy instead of once per view for every Gaussian of the warp.  A lane reads the
  // Gaussian it works on (mean, R S, log2 o) from shared memory and its SH row from L1.
  // For a render that a reverse pass may follow (moments, gmask and bcounts given), an
  // item also clears its moment accumulators, and each Gaussian leaves its drawing views,
  // its gradient views (drawn and reaching a tile) and its bucket count for the reverse
  // projection's work plan.
  __shared__ View s_view[MGS_MAX_VIEWS];
  __shared__ float s_own[kPreWarps][kOwnWords][32];
  __shared__ uint32_t s_dr[kPreWarps][32], s_td[kPreWarps][32];
  __shared__ uint32_t s_bucket[kPlanBuckets];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&vt.v[0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_view[0]);
    const int words = vt.n_views * (int)(sizeof(View) / 4);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
  }
  if (bcounts)
    for (int b = threadIdx.x; b < kPlanBuckets; b += blockDim.x) s_bucket[b] = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  s_dr[w][lane] = 0;
  s_td[w][lane] = 0;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g0 = g - lane;  // the warp's first Gaussian
  uint32_t cand = 0;            // views in which this thread's Gaussian may be drawn
  if (g < N) {
    GaussPre G;
    load_gauss(g, means, geo, ol, G);
    const float smax = fmaxf(G.s[0], fmaxf(G.s[1], G.s[2]));
    for (int v = 0; v < vt.n_views; ++v) {
      if (maybe_drawn(G.mu, smax, vt.v[v])) {
        cand |= 1u << v;
      } else {
        const int64_t item = (int64_t)v * N + g;
        rects[item] = make_uint2(1u, 0u);  // empty rect: x0 = 1 > x1 = 0
        touched[item] = 0;
        dkeys[item] = kSortDrop;  // undrawn: left out by the depth sort
      }
    }
    for (int k = 0; k < 3; ++k) s_own[w][k][lane] = G.mu[k];
    for (int k = 0; k < 9; ++k) s_own[w][3 + k][lane] = G.RS[k];
    s_own[w][12][lane] = log2f(G.o);
  }
  // exclusive prefix of the lanes' candidate counts
  const uint32_t nc = __popc(cand);
  uint32_t inc = nc;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t off = inc - nc, total = __shfl_sync(0xffffffffu, inc, 31);
  __syncwarp();  // the warp's s_own rows are written
  unsigned long long my_keys = 0;
  unsigned int my_vis = 0;
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int K3 = K * 3;
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t i = base + lane;
    int owner = 0;  // the last lane whose candidates start at or before item i
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const uint32_t o = __shfl_sync(0xffffffffu, off, owner + step);
      if (o <= i) owner += step;
    }
    const uint32_t ocand = __shfl_sync(0xffffffffu, cand, owner);
    const uint32_t ooff = __shfl_sync(0xffffffffu, off, owner);
    if (i < total) {
      const int v = (int)__fns(ocand, 0u, (int)(i - ooff) + 1);
      const View& V = s_view[v];
      const int64_t go = g0 + owner, item = (int64_t)v * N + go;
      GaussPre G;  // the geometry reads only the mean and R S
      for (int k = 0; k < 3; ++k) G.mu[k] = s_own[w][k][owner];
      for (int k = 0; k < 9; ++k) G.RS[k] = s_own[w][3 + k][owner];
      const float lo = s_own[w][12][owner];
      ViewGeom P;
      view_geom(G, V, P);
      int r = 0, rc[4];
      if (P.ok && tile_rect(P, V, r, rc)) {
        const float4 r0 = make_float4(P.u_hi, P.v_hi, P.u_lo, P.v_lo);
        const float4 r1 = make_float4(-0.5f * kLog2e * P.A, -kLog2e * P.B, -0.5f * kLog2e * P.C, lo);
        rec[3 * item + 0] = r0;
        rec[3 * item + 1] = r1;
        rects[item] = make_uint2((uint32_t)rc[0] | ((uint32_t)rc[1] << 16), (uint32_t)rc[2] | ((uint32_t)rc[3] << 16));
        const uint32_t count = cull_count(make_cull(r0, r1), rc);
        float raw[3];
        {  // colour: the coefficients stream from L1
          float Y[K];
          sh_basis<DEG>(P.dir, Y, nullptr);
          const T* p = sh + go * K3;
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc = __fmaf_rn(ld(p + 3 * k + ch), Y[k], acc);
            raw[ch] = acc;
          }
        }
        rec[3 * item + 2] = make_float4(fmaxf(0.f, raw[0]), fmaxf(0.f, raw[1]), fmaxf(0.f, raw[2]), P.tz);
        touched[item] = count;
        dkeys[item] = count ? __float_as_uint(P.tz) : kSortDrop;
        if (moments) {
          const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          moments[3 * item] = z;
          moments[3 * item + 1] = z;
          moments[3 * item + 2] = z;
        }
        atomicOr(&s_dr[w][owner], 1u << v);
        if (count) atomicOr(&s_td[w][owner], 1u << v);
        my_keys += count;
        my_vis += count ? 1u : 0u;
      } else {
        rects[item] = make_uint2(1u, 0u);
        touched[item] = 0;
        dkeys[item] = kSortDrop;
      }
    }
  }
  __syncwarp();  // the warp's view masks are complete
  if (g < N) {
    const uint32_t todo = s_td[w][lane];
    if (gmask) gmask[g] = make_uint2(s_dr[w][lane], todo);
    if (bcounts) atomicAdd(&s_bucket[__popc(todo)], 1u);
  }
  for (int o = 16; o; o >>= 1) {
    my_keys += __shfl_xor_sync(0xffffffffu, my_keys, o);
    my_vis += __shfl_xor_sync(0xffffffffu, my_vis, o);
  }
  // one pair of atomics per block: per warp, tens of thousands of atomics on two
  // addresses serialise
  __shared__ unsigned long long s_keys[kPreWarps];
  __shared__ unsigned int s_vis[kPreWarps];
  if (lane == 0) {
    s_keys[w] = my_keys;
    s_vis[w] = my_vis;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long k = 0, vv = 0;
    for (int ww = 0; ww < kPreWarps; ++ww) {
      k += s_keys[ww];
      vv += s_vis[ww];
    }
    if (k || vv) {
      atomicAdd(&counters[0], k);
      atomicAdd(&counters[1], vv);
    }
  }
  if (bcounts)
    for (int b = threadIdx.x; b < kPlanBuckets; b += blockDim.x)
      if (s_bucket[b]) atomicAdd(&bcounts[b], s_bucket[b]);
}

template <int DEG, typename T>
__global__ void __launch_bounds__(256) k_project_one(int64_t N, const float* __restrict__ means,
                                                     const Geom geo,
                                                     const T* __restrict__ ol, const T* __restrict__ sh,
                                                     const __grid_constant__ View V, float* mean2d,
                                                     float* conic, float* rgb, float* depth,
                                                     int32_t* radius, int32_t* rect) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  GaussPre G;
  load_gauss(g, means, geo, ol, G);
  ViewGeom P;
  view_geom(G, V, P);
  int r = 0, rc[4] = {0, 0, -1, -1};
  bool drawn = P.ok && tile_rect(P, V, r, rc);
  if (!P.ok) { r = 0; rc[0] = rc[1] = 0; rc[2] = rc[3] = -1; }
  if (depth) depth[g] = P.tz;
  if (mean2d) {
    mean2d[2 * g] = P.ok ? P.u_hi + P.u_lo : 0.f;
    mean2d[2 * g + 1] = P.ok ? P.v_hi + P.v_lo : 0.f;
  }
  if (conic) {
    conic[3 * g] = P.ok ? P.A : 0.f;
    conic[3 * g + 1] = P.ok ? P.B : 0.f;
    conic[3 * g + 2] = P.ok ? P.C : 0.f;
  }
  if (radius) radius[g] = P.ok ? r : 0;
  if (rect)
    for (int k = 0; k < 4; ++k) rect[4 * g + k] = rc[k];
  if (rgb) {
    constexpr int K3 = (DEG + 1) * (DEG + 1) * 3;
    float c[K3];
    load_sh<DEG>(g, sh, c);
    float raw[3] = {0.f, 0.f, 0.f};
    if (P.ok) colour<DEG>(c, P.dir, raw);
    for (int ch = 0; ch < 3; ++ch) rgb[3 * g + ch] = P.ok ? fmaxf(0.f, raw[ch]) : 0.f;
  }
  (void)drawn;
}

// ---------------- reverse pass ----------------
// Work plan: the Gaussians in order of the number of views they take a gradient from,
// most first, so that the lanes of a warp walk the same number of views (in index
// order a warp runs as many view iterations as its busiest lane, 2.7x the mean on a
// map whose neighbouring indices lie in different views).  Bucket b holds the
// Gaussians with b such views; the forward projection counted the buckets and left
// each Gaussian's view masks.  The scatter's blocks reserve their slots with one atomic
// per bucket; the order inside a bucket changes no result (each Gaussian is still one
// thread's sum over its views in view order).
// Moment accumulators before a reverse pass: the forward projection cleared those of the
// drawn items and marked them clean; a reverse pass marks them dirty.  A second reverse
// pass of the same render finds them dirty and clears the whole buffer.
__global__ void __launch_bounds__(256) k_moments_clear(float4* __restrict__ moments, int64_t n,
                                                       const uint32_t* __restrict__ dirty) {
  if (*dirty == 0u) return;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    moments[i] = z;
}

__global__ void __launch_bounds__(256) k_bwd_scatter(int64_t N, const uint2* __restrict__ gmask,
                                                     const uint32_t* __restrict__ counts,
                                                     uint32_t* __restrict__ cursor, uint32_t* __restrict__ list,
                                                     uint32_t* __restrict__ ldrawn, uint32_t* __restrict__ ltodo) {
  __shared__ uint32_t s_cnt[kPlanBuckets], s_base[kPlanBuckets];
  for (int b = threadIdx.x; b < kPlanBuckets; b += blockDim.x) s_cnt[b] = 0;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t drawn = 0, todo = 0, rank = 0;
  int b = 0;
  if (g < N) {
    const uint2 mk = gmask[g];
    drawn = mk.x;
    todo = mk.y;
    b = __popc(todo);
    rank = atomicAdd(&s_cnt[b], 1u);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kPlanBuckets; c += blockDim.x) {
    uint32_t base = 0;
    for (int h = c + 1; h < kPlanBuckets; ++h) base += counts[h];  // heavier buckets first
    s_base[c] = s_cnt[c] ? base + atomicAdd(&cursor[c], s_cnt[c]) : 0u;
  }
  __syncthreads();
  if (g < N) {
    const int64_t pos = (int64_t)s_base[b] + rank;  // < N: the buckets partition the N Gaussians
    if (pos < N) {
      list[pos] = (uint32_t)g;
      ldrawn[pos] = drawn;
      ltodo[pos] = todo;
    }
  }
}

// moments of a (view, Gaussian) item, accumulated by the backward blend over pixels p:
//   m0 = sum gp, m1 = sum gp dx, m2 = sum gp dy, m3 = sum gp dx^2, m4 = sum gp dx dy,
//   m5 = sum gp dy^2, m6..8 = sum w dL/drgb, m9 = sum w dL/ddepth,
// with gp = dL/dpower, w the blend weight and (dx, dy) = centre - pixel.
constexpr int kPreBwdThreads = 128;
template <int DEG, typename T>
__global__ void __launch_bounds__(kPreBwdThreads, 3) k_preprocess_bwd(int64_t N, const float* __restrict__ means,
                                                        const Geom geo,
                                                        const T* __restrict__ ol, const T* __restrict__ sh,
                                                        const __grid_constant__ ViewTable vt,
                                                        const float4* __restrict__ moments,
                                                        const uint32_t* __restrict__ list,
                                                        const uint32_t* __restrict__ ldrawn,
                                                        const uint32_t* __restrict__ ltodo,
                                                        uint32_t* __restrict__ dirty, mgs_grads grads) {
  // Thread t takes the t-th Gaussian of the work plan (its views with a gradient,
  // `todo`, and its drawing views) and walks its own views in view order; the lanes of
  // a warp run the per-view body together on different views, with the view constants
  // read from a shared-memory copy (the index differs per lane).
  __shared__ View s_view[MGS_MAX_VIEWS];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&vt.v[0]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_view[0]);
    const int words = vt.n_views * (int)(sizeof(View) / 4);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *dirty = 1u;  // the moments now hold this pass's sums
  if (t >= N) return;
  constexpr int K = (DEG + 1) * (DEG + 1);
  const int64_t g = list[t];
  if (g >= N) return;  // a plan left by a render of another map: skip, never read out of bounds
  const uint32_t drawn = ldrawn[t];
  // drawn views in which it reached a tile (else a zero gradient); views past the call's
  // are masked off, again against a plan left by another render
  uint32_t todo = ltodo[t] & (vt.n_views >= 32 ? ~0u : (1u << vt.n_views) - 1u);
  const float vis = (float)__popc(drawn);
  const bool ow = grads.overwrite != 0;
  if (drawn == 0) {  // no view draws it: a zero gradient (stored only when overwriting)
    if (ow) {
      for (int k = 0; k < 3; ++k) grads.means[3 * g + k] = 0.f;
      for (int k = 0; k < 3; ++k) grads.log_scales[3 * g + k] = 0.f;
      for (int k = 0; k < 4; ++k) grads.quats[4 * g + k] = 0.f;
      grads.opacity_logit[g] = 0.f;
      float* gsh = grads.sh + g * 3 * K;
      for (int k = 0; k < 3 * K; ++k) gsh[k] = 0.f;
    }
    return;
  }
  GaussPre G;
  load_gauss(g, means, geo, ol, G);
  float c[3 * K];
  load_sh<DEG>(g, sh, c);
  float dmu[3] = {0.f, 0.f, 0.f}, dS3[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, dop = 0.f;
  float dsh[3 * K];
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) dsh[k] = 0.f;
  float stat = 0.f;
  while (todo) {
    const int v = __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t item = (int64_t)v * N + g;
    const View& V = s_view[v];
    float4 q0 = moments[3 * item], q1 = moments[3 * item + 1], q2 = moments[3 * item + 2];
    ViewGeom P;
    view_geom(G, V, P);
    float m0 = q0.x, m1 = q0.y, m2 = q0.z, m3 = q0.w, m4 = q1.x, m5 = q1.y;
    float du = -(P.A * m1 + P.B * m2), dv = -(P.B * m1 + P.C * m2);
    float dA = -0.5f * m3, dB = -m4, dC = -0.5f * m5;
    dop += m0 / G.o;
    float dcol[3] = {q1.z, q1.w, q2.x};
    float dd = q2.y;
    float dm[3] = {0.f, 0.f, 0.f};
    // colour
    {
      float Y[K], dY[K][3];
      sh_basis<DEG>(P.dir, Y, dY);
      float ddir[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        float raw = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) raw = __fmaf_rn(c[3 * k + ch], Y[k], raw);
        if (raw < 0.f) continue;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          dsh[3 * k + ch] += dcol[ch] * Y[k];
          if (DEG > 0) {
            float w = dcol[ch] * c[3 * k + ch];
            ddir[0] += w * dY[k][0];
            ddir[1] += w * dY[k][1];
            ddir[2] += w * dY[k][2];
          }
        }
      }
      if (DEG > 0) {
        float dt = ddir[0] * P.dir[0] + ddir[1] * P.dir[1] + ddir[2] * P.dir[2];
        float iv = 1.f / P.vnorm;
        for (int k = 0; k < 3; ++k) dm[k] += (ddir[k] - P.dir[k] * dt) * iv;
      }
    }
    // centre and depth
    float tx = P.tx, ty = P.ty, tz = P.tz, itz = 1.f / tz, itz2 = itz * itz;
    float dp[3] = {du * V.fx * itz, dv * V.fy * itz, dd - (du * V.fx * tx + dv * V.fy * ty) * itz2};
    // conic -> 2D covariance: Gs = -M Gm M, M = [[A,B],[B,C]], Gm = [[dA, dB/2],[dB/2, dC]]
    float hB = 0.5f * dB;
    float t00 = P.A * dA + P.B * hB, t01 = P.A * hB + P.B * dC;
    float t10 = P.B * dA + P.C * hB, t11 = P.B * hB + P.C * dC;
    float G00 = -(t00 * P.A + t01 * P.B), G01 = -(t00 * P.B + t01 * P.C);
    float G11 = -(t10 * P.B + t11 * P.C);
    // cov = T S3 T^T + 0.3 I  ->  dS3 += T^T Gs T ; dT = 2 Gs T S3
    float GT0[3], GT1[3];
    for (int k = 0; k < 3; ++k) {
      GT0[k] = G00 * P.T[k] + G01 * P.T[3 + k];
      GT1[k] = G01 * P.T[k] + G11 * P.T[3 + k];
    }
    dS3[0] += P.T[0] * GT0[0] + P.T[3] * GT1[0];
    dS3[1] += P.T[0] * GT0[1] + P.T[3] * GT1[1];
    dS3[2] += P.T[0] * GT0[2] + P.T[3] * GT1[2];
    dS3[3] += P.T[1] * GT0[1] + P.T[4] * GT1[1];
    dS3[4] += P.T[1] * GT0[2] + P.T[4] * GT1[2];
    dS3[5] += P.T[2] * GT0[2] + P.T[5] * GT1[2];
    const float* S = G.S3;
    float dT0[3], dT1[3];
    dT0[0] = 2.f * (GT0[0] * S[0] + GT0[1] * S[1] + GT0[2] * S[2]);
    dT0[1] = 2.f * (GT0[0] * S[1] + GT0[1] * S[3] + GT0[2] * S[4]);
    dT0[2] = 2.f * (GT0[0] * S[2] + GT0[1] * S[4] + GT0[2] * S[5]);
    dT1[0] = 2.f * (GT1[0] * S[0] + GT1[1] * S[1] + GT1[2] * S[2]);
    dT1[1] = 2.f * (GT1[0] * S[1] + GT1[1] * S[3] + GT1[2] * S[4]);
    dT1[2] = 2.f * (GT1[0] * S[2] + GT1[1] * S[4] + GT1[2] * S[5]);
    const float* W = V.R;
    float dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
    float dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
    float dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
    float dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
    dp[2] -= (V.fx * dJ00 + V.fy * dJ11) * itz2;
    if (!P.clampx) {
      dp[0] -= V.fx * itz2 * dJ02;
      dp[2] += 2.f * V.fx * tx * itz2 * itz * dJ02;
    } else {
      float xc = fminf(V.limx, fmaxf(-V.limx, P.xr));
      dp[2] += V.fx * xc * itz2 * dJ02;
    }
    if (!P.clampy) {
      dp[1] -= V.fy * itz2 * dJ12;
      dp[2] += 2.f * V.fy * ty * itz2 * itz * dJ12;
    } else {
      float yc = fminf(V.limy, fmaxf(-V.limy, P.yr));
      dp[2] += V.fy * yc * itz2 * dJ12;
    }
    for (int k = 0; k < 3; ++k) dm[k] += W[k] * dp[0] + W[3 + k] * dp[1] + W[6 + k] * dp[2];
    for (int k = 0; k < 3; ++k) dmu[k] += dm[k];
    stat += sqrtf(dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]);
  }
  // S3 = Rq diag(s^2) Rq^T  ->  log-scales and quaternion
  const float* R = G.Rq;
  float H[9] = {dS3[0], dS3[1], dS3[2], dS3[1], dS3[3], dS3[4], dS3[2], dS3[4], dS3[5]};
  float HR[9];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) HR[3 * a + k] = H[3 * a] * R[k] + H[3 * a + 1] * R[3 + k] + H[3 * a + 2] * R[6 + k];
  float dls[3], dR[9];
  for (int k = 0; k < 3; ++k) {
    float rhr = R[k] * HR[k] + R[3 + k] * HR[3 + k] + R[6 + k] * HR[6 + k];
    float s2 = G.s[k] * G.s[k];
    dls[k] = 2.f * s2 * rhr;
    for (int a = 0; a < 3; ++a) dR[3 * a + k] = 2.f * HR[3 * a + k] * s2;
  }
  float dqn[4];
  quat_rot_vjp(G.qn, dR, dqn);
  float dot = dqn[0] * G.qn[0] + dqn[1] * G.qn[1] + dqn[2] * G.qn[2] + dqn[3] * G.qn[3];
  float iq = 1.f / G.qnorm;
  auto put = [ow](float* p, float v) { *p = ow ? v : *p + v; };
  for (int k = 0; k < 3; ++k) put(grads.means + 3 * g + k, dmu[k]);
  for (int k = 0; k < 3; ++k) put(grads.log_scales + 3 * g + k, dls[k]);
  for (int k = 0; k < 4; ++k) put(grads.quats + 4 * g + k, (dqn[k] - G.qn[k] * dot) * iq);
  put(grads.opacity_logit + g, dop * G.o * (1.f - G.o));
  float* gsh = grads.sh + g * 3 * K;
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) put(gsh + k, dsh[k]);
  if (grads.grad_stat) grads.grad_stat[g] += stat;
  if (grads.vis_count) grads.vis_count[g] += vis;
}

template <typename T>
cudaError_t launch_pre_t(int deg, int64_t N, const mgs_gaussians& g, const ViewTable& vt,
                         float4* rec, uint2* rects, uint32_t* touched, uint32_t* dkeys,
                         unsigned long long* counters, const FwdPlanOut& fb, cudaStream_t s) {
  unsigned grid = (unsigned)div_up(N, kPreThreads);
  const Geom geo{g.log_scales, g.quats, g.geom_dtype, g.quat_dtype};
  const T* ol = (const T*)g.opacity_logit;
  const T* sh = (const T*)g.sh;
  switch (deg) {
    case 0: k_preprocess<0, T><<<grid, kPreThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, rec, rects, touched, dkeys, counters, fb.moments, fb.gmask, fb.bcounts); break;
    case 1: k_preprocess<1, T><<<grid, kPreThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, rec, rects, touched, dkeys, counters, fb.moments, fb.gmask, fb.bcounts); break;
    case 2: k_preprocess<2, T><<<grid, kPreThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, rec, rects, touched, dkeys, counters, fb.moments, fb.gmask, fb.bcounts); break;
    default: k_preprocess<3, T><<<grid, kPreThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, rec, rects, touched, dkeys, counters, fb.moments, fb.gmask, fb.bcounts); break;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bwd_t(int deg, int64_t N, const mgs_gaussians& g, const ViewTable& vt, float4* moments,
                         const BwdPlan& pl, const mgs_grads& gr, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(pl.counts + kPlanCountWords, 0, kPlanCountWords * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const unsigned pgrid = (unsigned)div_up(N, 256);
  k_bwd_scatter<<<pgrid, 256, 0, s>>>(N, pl.gmask, pl.counts, pl.counts + kPlanCountWords, pl.list, pl.ldrawn,
                                       pl.ltodo);
  count_launch();
  unsigned grid = (unsigned)div_up(N, kPreBwdThreads);
  const Geom geo{g.log_scales, g.quats, g.geom_dtype, g.quat_dtype};
  const T* ol = (const T*)g.opacity_logit;
  const T* sh = (const T*)g.sh;
  switch (deg) {
    case 0: k_preprocess_bwd<0, T><<<grid, kPreBwdThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, moments, pl.list, pl.ldrawn, pl.ltodo, pl.counts + kPlanDirtyWord, gr); break;
    case 1: k_preprocess_bwd<1, T><<<grid, kPreBwdThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, moments, pl.list, pl.ldrawn, pl.ltodo, pl.counts + kPlanDirtyWord, gr); break;
    case 2: k_preprocess_bwd<2, T><<<grid, kPreBwdThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, moments, pl.list, pl.ldrawn, pl.ltodo, pl.counts + kPlanDirtyWord, gr); break;
    default: k_preprocess_bwd<3, T><<<grid, kPreBwdThreads, 0, s>>>(N, g.means, geo, ol, sh, vt, moments, pl.list, pl.ldrawn, pl.ltodo, pl.counts + kPlanDirtyWord, gr); break;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_proj_t(int deg, int64_t N, const mgs_gaussians& g, const View& V, float* mean2d,
                          float* conic, float* rgb, float* depth, int32_t* radius, int32_t* rect,
                          cudaStream_t s) {
  unsigned grid = (unsigned)div_up(N, 256);
  const Geom geo{g.log_scales, g.quats, g.geom_dtype, g.quat_dtype};
  const T* ol = (const T*)g.opacity_logit;
  const T* sh = (const T*)g.sh;
  switch (deg) {
    case 0: k_project_one<0, T><<<grid, 256, 0, s>>>(N, g.means, geo, ol, sh, V, mean2d, conic, rgb, depth, radius, rect); break;
    case 1: k_project_one<1, T><<<grid, 256, 0, s>>>(N, g.means, geo, ol, sh, V, mean2d, conic, rgb, depth, radius, rect); break;
    case 2: k_project_one<2, T><<<grid, 256, 0, s>>>(N, g.means, geo, ol, sh, V, mean2d, conic, rgb, depth, radius, rect); break;
    default: k_project_one<3, T><<<grid, 256, 0, s>>>(N, g.means, geo, ol, sh, V, mean2d, conic, rgb, depth, radius, rect); break;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_preprocess(const mgs_gaussians& g, const ViewTable& vt, float4* rec,
                              uint2* rects, uint32_t* touched, uint32_t* dkeys,
                              unsigned long long* counters, const FwdPlanOut& fb, cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  switch (g.attr_dtype) {
    case MGS_F16: return launch_pre_t<__half>(g.sh_degree, g.n, g, vt, rec, rects, touched, dkeys, counters, fb, s);
    case MGS_BF16: return launch_pre_t<__nv_bfloat16>(g.sh_degree, g.n, g, vt, rec, rects, touched, dkeys, counters, fb, s);
    default: return launch_pre_t<float>(g.sh_degree, g.n, g, vt, rec, rects, touched, dkeys, counters, fb, s);
  }
}

cudaError_t launch_moments_clear(float4* moments, int64_t n, const uint32_t* dirty, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(div_up(n, 256), 152 * 8);
  k_moments_clear<<<(unsigned)blocks, 256, 0, s>>>(moments, n, dirty);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const mgs_gaussians& g, const ViewTable& vt, float4* moments,
                                  const BwdPlan& pl, const mgs_grads& gr, cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  switch (g.attr_dtype) {
    case MGS_F16: return launch_bwd_t<__half>(g.sh_degree, g.n, g, vt, moments, pl, gr, s);
    case MGS_BF16: return launch_bwd_t<__nv_bfloat16>(g.sh_degree, g.n, g, vt, moments, pl, gr, s);
    default: return launch_bwd_t<float>(g.sh_degree, g.n, g, vt, moments, pl, gr, s);
  }
}

cudaError_t launch_project_one(const mgs_gaussians& g, const View& V, float* mean2d, float* conic,
                               float* rgb, float* depth, int32_t* radius, int32_t* rect,
                               cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  switch (g.attr_dtype) {
    case MGS_F16: return launch_proj_t<__half>(g.sh_degree, g.n, g, V, mean2d, conic, rgb, depth, radius, rect, s);
    case MGS_BF16: return launch_proj_t<__nv_bfloat16>(g.sh_degree, g.n, g, V, mean2d, conic, rgb, depth, radius, rect, s);
    default: return launch_proj_t<float>(g.sh_degree, g.n, g, V, mean2d, conic, rgb, depth, radius, rect, s);
  }
}

}  // namespace mgs
