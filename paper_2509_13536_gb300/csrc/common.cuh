// Device-side helpers shared by the sm_103a kernels of libmemgs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "memgs.h"

namespace mgs {

constexpr int kTile = MGS_TILE;             // tile edge, px
constexpr int kTilePix = kTile * kTile;     // 256 pixels = 256 threads per tile CTA
constexpr float kAlphaMin = 1.0f / 255.0f;  // skip below
constexpr float kLog2AlphaMin = -7.994353436858858f;  // log2(1/255): the same test on the base-2 exponent of alpha
constexpr float kLog2_255 = 7.994353436858858f;

// Whether the 0.99 clamp can bind for a projected record (A', B', C', log2 o): alpha =
// 2^e, e = p2 + log2 o, p2 = A' dx^2 + B' dx dy + C' dy^2 <= 0.  The blends evaluate e with
// five roundings, which move it by at most 3 eps tr' |d|^2 + eps |log2 o| (tr' = -(A' + C');
// |B'| |dx dy| <= tr' |d|^2 / 2), while -p2 >= (det' / tr') |d|^2.  When tr'^2 <= 1e5 det'
// the first bound is far below -p2, so the evaluated e stays at or below log2 o (1 - 2 eps),
// and with o <= 0.98 the evaluated alpha (ex2.approx, relative error ~2^-22) stays below
// 0.99: the clamp and its zero derivative never apply.  Blend loops skip both for groups
// of such entries.
__device__ __forceinline__ bool clamp_possible(float4 r1) {
  const float tr = -(r1.x + r1.z);
  const float det = __fsub_rn(__fmul_rn(r1.x, r1.z), __fmul_rn(0.25f, __fmul_rn(r1.y, r1.y)));
  return !(r1.w <= -0.029146346f) || !(__fmul_rn(tr, tr) <= __fmul_rn(1e5f, det));  // log2(0.98)
}
constexpr float kAlphaMax = 0.99f;          // clamp
constexpr float kTStop = 1e-4f;             // stop once T falls below
constexpr float kDilation = 0.3f;           // px^2 added to the 2D covariance diagonal
constexpr float kFovClamp = 1.3f;           // ray clamp factor in the Jacobian
constexpr float kLog2e = 1.4426950408889634f;

// Real orthonormal spherical harmonics, Cartesian forms on the unit sphere; each
// constant is the normalisation written next to it.
constexpr float kSh0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSh1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kSh2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kSh2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kSh2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kSh3a = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
constexpr float kSh3b = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kSh3c = 0.45704579946446577f;  // sqrt(21/(2 pi))/4
constexpr float kSh3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kSh3e = 1.4453057213202769f;   // sqrt(105/pi)/4

// Per-view constants, passed by value to every kernel of a render call.
struct View {
  float R[9], t[3];
  float fx, fy, cx, cy, near_z;
  float C[3];          // camera centre in world coordinates (rounded)
  float C_lo[3];       // C - (double) C[] rounded: the centre as a double-float pair
  float limx, limy;    // 1.3 * half field of view (tangent)
  int width, height, tiles_x, tiles_y;
  int tile_base;       // first global tile id of this view
  int64_t item_base;   // first (view, Gaussian) item of this view: items of view v are
                       // item_base + i for Gaussian i of the view's map (n_items of them)
  int64_t n_items;
  float* rgb;          // forward outputs
  float* depth;
  float* alpha;
  const float* g_rgb;  // backward cotangents (may be null)
  const float* g_depth;
  const float* g_alpha;
  float* T_final;      // per-pixel saved state (workspace)
  uint32_t* n_contrib;
};

struct ViewTable {
  int n_views;
  int n_tiles;         // sum over views
  View v[MGS_MAX_VIEWS];
};

__device__ __forceinline__ int view_of_item(const ViewTable& vt, int64_t item) {
  int v = 0;
  while (v + 1 < vt.n_views && vt.v[v + 1].item_base <= item) ++v;
  return v;
}

__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int tile) {
  int v = 0;
  while (v + 1 < vt.n_views && vt.v[v + 1].tile_base <= tile) ++v;
  return v;
}

// --- storage types: attributes may be f32, f16 or bf16; arithmetic is f32 ---
__device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void st(float* p, float x) { *p = x; }
__device__ __forceinline__ void st(__half* p, float x) { *p = __float2half_rn(x); }
__device__ __forceinline__ void st(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }

// Geometry group of a map (log-scales, quaternions) with their runtime storage types.
struct Geom {
  const void* ls;
  const void* qs;
  int dt;   // log-scales
  int qdt;  // quaternions
};

// runtime-typed access for the small geometry groups (log-scales, quaternions)
__device__ __forceinline__ float ld_dt(const void* p, int dt, int64_t i) {
  switch (dt) {
    case MGS_F16: return __half2float(static_cast<const __half*>(p)[i]);
    case MGS_BF16: return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
    default: return __ldg(static_cast<const float*>(p) + i);
  }
}
__device__ __forceinline__ void st_dt(void* p, int dt, int64_t i, float x) {
  switch (dt) {
    case MGS_F16: static_cast<__half*>(p)[i] = __float2half_rn(x); break;
    case MGS_BF16: static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16_rn(x); break;
    default: static_cast<float*>(p)[i] = x; break;
  }
}
__device__ __forceinline__ void cp_dt(void* dst, const void* src, int dt, int64_t i, int64_t j) {
  if (dt == MGS_F32) static_cast<float*>(dst)[i] = static_cast<const float*>(src)[j];
  else static_cast<uint16_t*>(dst)[i] = static_cast<const uint16_t*>(src)[j];
}

// --- error-free transformations (double-float arithmetic in f32) ---
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, lo);
}
// x / y for double-float x, y (one Newton correction).
__device__ __forceinline__ DF df_div(DF x, DF y) {
  float q1 = __fdiv_rn(x.hi, y.hi);
  DF p = two_prod(q1, y.hi);
  float r = __fsub_rn(__fsub_rn(x.hi, p.hi), p.lo);
  r = __fadd_rn(r, __fsub_rn(x.lo, __fmul_rn(q1, y.lo)));
  float q2 = __fdiv_rn(r, y.hi);
  return fast_two_sum(q1, q2);
}
// a * x + c with f32 a, c and double-float x.
__device__ __forceinline__ DF df_axpc(float a, DF x, float c) {
  DF p = two_prod(a, x.hi);
  p.lo = __fmaf_rn(a, x.lo, p.lo);
  DF s = two_sum(p.hi, c);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, p.lo));
}

// 1/x by the MUFU reciprocal (x in [0.01, 1] where the blends use it).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Rotation matrix of the unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(const float q[4], float R[9]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// Gradient of sum_ij G_ij R_ij with respect to the unit quaternion.
__device__ __forceinline__ void quat_rot_vjp(const float q[4], const float G[9], float dq[4]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  dq[0] = 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  dq[1] = 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.f * x * G[8]);
  dq[2] = 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.f * y * G[8]);
  dq[3] = 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

// Spherical-harmonic basis at unit direction d (K = (DEG+1)^2 values) and, when
// dY != nullptr, the gradient of each Cartesian polynomial with respect to d.
template <int DEG>
__device__ __forceinline__ void sh_basis(const float d[3], float* Y, float (*dY)[3]) {
  float x = d[0], y = d[1], z = d[2];
  Y[0] = kSh0;
  if (dY) { dY[0][0] = dY[0][1] = dY[0][2] = 0.f; }
  if (DEG < 1) return;
  Y[1] = kSh1 * y; Y[2] = kSh1 * z; Y[3] = kSh1 * x;
  if (dY) {
    dY[1][0] = 0.f; dY[1][1] = kSh1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = kSh1;
    dY[3][0] = kSh1; dY[3][1] = 0.f; dY[3][2] = 0.f;
  }
  if (DEG < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSh2a * x * y;
  Y[5] = kSh2a * y * z;
  Y[6] = kSh2b * (3.f * zz - 1.f);
  Y[7] = kSh2a * x * z;
  Y[8] = kSh2c * (xx - yy);
  if (dY) {
    dY[4][0] = kSh2a * y; dY[4][1] = kSh2a * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = kSh2a * z; dY[5][2] = kSh2a * y;
    dY[6][0] = 0.f; dY[6][1] = 0.f; dY[6][2] = kSh2b * 6.f * z;
    dY[7][0] = kSh2a * z; dY[7][1] = 0.f; dY[7][2] = kSh2a * x;
    dY[8][0] = kSh2c * 2.f * x; dY[8][1] = -kSh2c * 2.f * y; dY[8][2] = 0.f;
  }
  if (DEG < 3) return;
  Y[9] = kSh3a * y * (3.f * xx - yy);
  Y[10] = kSh3b * x * y * z;
  Y[11] = kSh3c * y * (5.f * zz - 1.f);
  Y[12] = kSh3d * z * (5.f * zz - 3.f);
  Y[13] = kSh3c * x * (5.f * zz - 1.f);
  Y[14] = kSh3e * z * (xx - yy);
  Y[15] = kSh3a * x * (xx - 3.f * yy);
  if (dY) {
    dY[9][0] = kSh3a * 6.f * x * y; dY[9][1] = kSh3a * 3.f * (xx - yy); dY[9][2] = 0.f;
    dY[10][0] = kSh3b * y * z; dY[10][1] = kSh3b * x * z; dY[10][2] = kSh3b * x * y;
    dY[11][0] = 0.f; dY[11][1] = kSh3c * (5.f * zz - 1.f); dY[11][2] = kSh3c * 10.f * y * z;
    dY[12][0] = 0.f; dY[12][1] = 0.f; dY[12][2] = kSh3d * (15.f * zz - 3.f);
    dY[13][0] = kSh3c * (5.f * zz - 1.f); dY[13][1] = 0.f; dY[13][2] = kSh3c * 10.f * x * z;
    dY[14][0] = kSh3e * 2.f * x * z; dY[14][1] = -kSh3e * 2.f * y * z; dY[14][2] = kSh3e * (xx - yy);
    dY[15][0] = kSh3a * 3.f * (xx - yy); dY[15][1] = -kSh3a * 6.f * x * y; dY[15][2] = 0.f;
  }
}

// Fragment evaluation in the blend kernels' rounding (the counting pass uses it; the
// blends evaluate the same operations on packed pairs).  xy: Gaussian centre relative
// to the tile origin; co: conic pre-scaled by -log2(e)/2 (A, C) and -log2(e) (B), plus
// log2(opacity).  Returns the base-2 exponent of alpha before the clamp:
// alpha = min(0.99, 2^e), and the Gaussian passes the 1/255 cutoff iff e >= log2(1/255).
// The exponent of a positive-definite conic is never positive, so there is no separate
// "exponent > 0" test: a float32 evaluation that comes out positive is rounding near the
// centre, where the exact alpha is the opacity.
__device__ __forceinline__ float frag_exp2(float2 xy, float4 co, float pxf, float pyf, float& dx,
                                           float& dy) {
  dx = __fsub_rn(xy.x, pxf);
  dy = __fsub_rn(xy.y, pyf);
  float t = __fmaf_rn(co.x, dx, __fmul_rn(co.y, dy));
  return __fmaf_rn(t, dx, __fmaf_rn(__fmul_rn(co.z, dy), dy, co.w));
}

// ---- exact tile culling ----------------------------------------------------------
// A Gaussian can only pass the alpha >= 1/255 test where o 2^p2 >= 1/255, i.e. inside
// the ellipse  a dx^2 + 2 b dx dy + c dy^2 <= kappa  with (a, 2b, c) = -(A', B', C')
// from the projected record and kappa = log2(255 o) = log2(o) + log2(255).  Tiles of the 3-sigma rect that
// this ellipse does not reach hold no pixel where the Gaussian contributes, so
// dropping them changes no output.  The ellipse is enlarged (kappa by 1e-4 relative +
// 1e-3, extents by 1e-2 px), far beyond the error of the approximate MUFU
// reciprocal / square root / log used here and of the blend's own f32 evaluation.
// Both the counting pass and the key emission evaluate these functions on the same
// stored record values with explicit intrinsics, so they agree exactly.
struct Cull {
  float a, b, c, det, kappa, ex, ey, ux, uy, ia, bia, dyL;
  bool none;   // no pixel can reach the cutoff
  bool full;   // degenerate form: keep the whole rect
};

__device__ __forceinline__ float sqrt_approx(float x) {  // x >= 0
  return x > 0.f ? __fmul_rn(x, rsqrtf(x)) : 0.f;
}

__device__ __forceinline__ Cull make_cull(float4 r0, float4 r1) {
  Cull q;
  q.ux = r0.x;
  q.uy = r0.y;
  q.a = -r1.x;
  q.b = __fmul_rn(-0.5f, r1.y);
  q.c = -r1.z;
  q.kappa = __fmaf_rn(__fadd_rn(r1.w, kLog2_255), 1.0001f, 1e-3f);  // r1.w = log2(o)
  q.none = !(q.kappa > 0.f);
  q.det = __fsub_rn(__fmul_rn(q.a, q.c), __fmul_rn(q.b, q.b));
  q.full = !(q.det > 0.f) || !(q.a > 0.f) || !(q.c > 0.f);
  q.ex = q.ey = q.ia = q.bia = q.dyL = 0.f;
  if (q.none || q.full) return q;
  const float kd = __fdividef(q.kappa, q.det);
  q.ex = __fadd_rn(sqrt_approx(__fmul_rn(kd, q.c)), 1e-2f);
  q.ey = __fadd_rn(sqrt_approx(__fmul_rn(kd, q.a)), 1e-2f);
  q.ia = __fdividef(1.f, q.a);
  q.bia = __fmul_rn(q.b, q.ia);
  q.dyL = __fdividef(__fmul_rn(q.b, q.ex), q.c);  // height of the leftmost point
  return q;
}

__device__ __forceinline__ int tiles_lo(float X) {  // first tile whose last pixel centre >= X
  return (int)fmaxf(-1.f, fminf(65536.f, ceilf(__fmul_rn(__fsub_rn(X, 15.f), 0.0625f))));
}
__device__ __forceinline__ int tiles_hi(float X) {  // last tile whose first pixel centre <= X
  return (int)fmaxf(-1.f, fminf(65536.f, floorf(__fmul_rn(X, 0.0625f))));
}

// Rows of the rect [y0, y1] the ellipse can reach.
__device__ __forceinline__ void cull_rows(const Cull& q, int& y0, int& y1) {
  if (q.full) return;
  if (q.none) { y1 = y0 - 1; return; }
  y0 = max(y0, tiles_lo(__fsub_rn(q.uy, q.ey)));
  y1 = min(y1, tiles_hi(__fadd_rn(q.uy, q.ey)));
}

// Columns of tile row ty (inside rect columns [x0, x1]) the ellipse can reach: the
// x-extent of the ellipse within the row's band of pixel centres, taken at the band
// ends or at the ellipse's leftmost / rightmost point when that lies in the band.
__device__ __forceinline__ void cull_cols(const Cull& q, int ty, int& x0, int& x1) {
  if (q.full) return;
  if (q.none) { x1 = x0 - 1; return; }
  float lo = fmaxf(__fsub_rn((float)(ty * kTile), q.uy), -q.ey);
  float hi = fminf(__fsub_rn((float)(ty * kTile + kTile - 1), q.uy), q.ey);
  if (lo > hi) { x1 = x0 - 1; return; }
  const float ak = __fmul_rn(q.a, q.kappa);
  const float hl = __fmul_rn(sqrt_approx(__fsub_rn(ak, __fmul_rn(q.det, __fmul_rn(lo, lo)))), q.ia);
  const float hh = __fmul_rn(sqrt_approx(__fsub_rn(ak, __fmul_rn(q.det, __fmul_rn(hi, hi)))), q.ia);
  const float ml = __fmul_rn(-q.bia, lo), mh = __fmul_rn(-q.bia, hi);
  float xmin, xmax;
  if (q.dyL >= lo && q.dyL <= hi) xmin = -q.ex;
  else xmin = fminf(__fsub_rn(ml, hl), __fsub_rn(mh, hh));
  if (-q.dyL >= lo && -q.dyL <= hi) xmax = q.ex;
  else xmax = fmaxf(__fadd_rn(ml, hl), __fadd_rn(mh, hh));
  x0 = max(x0, tiles_lo(__fsub_rn(__fadd_rn(q.ux, xmin), 1e-2f)));
  x1 = min(x1, tiles_hi(__fadd_rn(__fadd_rn(q.ux, xmax), 1e-2f)));
}

// Number of tiles of the inclusive rect rc the Gaussian can contribute to.
__device__ __forceinline__ uint32_t cull_count(const Cull& q, const int rc[4]) {
  int y0 = rc[1], y1 = rc[3];
  cull_rows(q, y0, y1);
  uint32_t n = 0;
  for (int y = y0; y <= y1; ++y) {
    int x0 = rc[0], x1 = rc[2];
    cull_cols(q, y, x0, x1);
    if (x1 >= x0) n += (uint32_t)(x1 - x0 + 1);
  }
  return n;
}

}  // namespace mgs
