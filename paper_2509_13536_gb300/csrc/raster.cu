// Tile blend kernels (Sec. II-E, Eq. 11), forward and reverse, sm_103a.
//
// One CTA owns one 16x16 tile of one view.  Forward (128 threads, two pixels of one
// column each): batches of 256 sorted entries are gathered into shared memory and
// every thread walks them front to back for its two pixels, with transmittance and
// the colour/depth sums in registers as packed f32 pairs; the CTA leaves as soon as
// all its pixels stopped.
//
// Reverse (256 threads, one pixel each): the tile's entries are walked back to front
// in batches of 16.  In the pixel phase each thread runs the back-to-front recursion
// for its pixel (T recovered by division; of the colour and depth behind each
// Gaussian only their dot product with the pixel's cotangent is needed, one scalar),
// two entries at a time so that what does not depend on the running T goes through
// packed f32 pairs, and writes two numbers per (pixel, entry) into shared memory:
// gp = dL/dpower and the blend weight w.  In the
// Gaussian phase each half-warp owns its 16 pixels (two rows of the warp's 8x4 block) and
// each of its lanes one entry; it sums gp, k gp, k^2 gp (k the column) and w times the
// cotangent along each row and forms the ten moments the per-Gaussian chain rule needs;
// the eight warps' partial sums meet
// in shared memory, are added by all threads (half-warp = entry, lane = moment) and go
// out as three 16-byte vector atomics per entry.
// There is no per-fragment shuffle or atomic.
//
// Both per-fragment loops are branch-free: a Gaussian that fails the alpha test (or
// comes after the pixel stopped) enters with alpha = 0, which leaves every running
// quantity unchanged.  A warp then issues one path instead of the union of the
// contributing and skipping paths of its 32 pixels.
#include <type_traits>

#include "internal.h"

namespace mgs {
namespace {

// Forward: each thread blends two pixels of one column (rows 2 r and 2 r + 1), so the
// per-entry arithmetic runs on packed f32 pairs (each element rounds exactly as the
// scalar operation would).  Shared memory holds every entry with its values
// duplicated, (v, v), so one 16-byte load yields two operand pairs.
constexpr int kFwdThreads = kTilePix / 2;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

__global__ void __launch_bounds__(kFwdThreads) k_blend_fwd(const __grid_constant__ ViewTable vt,
                                                          const float4* __restrict__ rec,
                                                          const uint32_t* __restrict__ vals,
                                                          const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ order) {
  __shared__ float4 s_xy[kTilePix];   // (x, x, y, y) tile-relative centre
  __shared__ float4 s_ab[kTilePix];   // (A, A, B, B) scaled conic
  __shared__ float4 s_co[kTilePix];   // (C, C, log2 o, log2 o)
  __shared__ float4 s_rg[kTilePix];   // (r, r, g, g)
  __shared__ float4 s_bd[kTilePix];   // (b, b, depth, depth)
  __shared__ uint32_t s_clamp[kFwdThreads / 32];  // per warp: its bits of the batch's 32 group flags
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  if ((unsigned)tile >= (unsigned)vt.n_tiles) return;  // an order left by another render
  const View& V = vt.v[view_of_tile(vt, tile)];
  const int local = tile - V.tile_base;
  const int x0 = (local % V.tiles_x) * kTile, y0 = (local / V.tiles_x) * kTile;
  const int t = threadIdx.x;
  // each warp an 8x8 block of the tile (its pixels stop at similar list positions), each
  // thread two vertically adjacent pixels
  const int wq = t >> 5, ln = t & 31;
  const int lx = 8 * (wq & 1) + (ln & 7), ly = 8 * (wq >> 1) + 2 * (ln >> 3);
  const int px = x0 + lx, py = y0 + ly;
  const bool in0 = px < V.width && py < V.height, in1 = px < V.width && py + 1 < V.height;
  const float x0f = (float)x0, y0f = (float)y0;
  const float2 npx = f2(-(float)lx, -(float)lx), npy = f2(-(float)ly, -(float)(ly + 1));
  const uint2 range = ranges[tile];
  const int n = (int)(range.y - range.x);
  float2 T = f2(in0 ? 1.f : 0.f, in1 ? 1.f : 0.f);
  float2 C0 = f2(0.f, 0.f), C1 = C0, C2 = C0, D = C0;
  const float2 m1 = f2(-1.f, -1.f);
  uint32_t last0 = 0, last1 = 0;
  for (int b = 0; b < n; b += kTilePix) {
    if (__syncthreads_count(T.x >= kTStop || T.y >= kTStop) == 0) break;
    uint32_t clamp_bits = 0;  // bit g: the clamp may bind for an entry of group g (entries 8g..8g+7)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = t + h * kFwdThreads, e = b + k;
      bool cl = false;
      if (e < n) {
        const uint32_t idx = vals[range.x + e];
        const float4 r0 = rec[3 * (size_t)idx], r1 = rec[3 * (size_t)idx + 1], r2 = rec[3 * (size_t)idx + 2];
        const float x = __fadd_rn(__fsub_rn(r0.x, x0f), r0.z), y = __fadd_rn(__fsub_rn(r0.y, y0f), r0.w);
        s_xy[k] = make_float4(x, x, y, y);
        s_ab[k] = make_float4(r1.x, r1.x, r1.y, r1.y);
        s_co[k] = make_float4(r1.z, r1.z, r1.w, r1.w);
        s_rg[k] = make_float4(r2.x, r2.x, r2.y, r2.y);
        s_bd[k] = make_float4(r2.z, r2.z, r2.w, r2.w);
        cl = clamp_possible(r1);
      }
      // lanes 8q..8q+7 of warp w hold group 4 w + 16 h + q
      const uint32_t bal = __ballot_sync(0xffffffffu, cl);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if ((bal >> (8 * q)) & 0xffu) clamp_bits |= 1u << (4 * (t >> 5) + 16 * h + q);
    }
    if ((t & 31) == 0) s_clamp[t >> 5] = clamp_bits;
    __syncthreads();
    uint32_t clamp_mask = 0;
#pragma unroll
    for (int w = 0; w < kFwdThreads / 32; ++w) clamp_mask |= s_clamp[w];
    const int cnt = min(kTilePix, n - b);
    for (int j0 = 0; j0 < cnt; j0 += 8) {
      if (__all_sync(0xffffffffu, T.x < kTStop && T.y < kTStop)) break;
      const int jn = min(8, cnt - j0);
      auto entry = [&](int jj, auto clampc) {
          const int j = j0 + jj;
          const float4 xy = s_xy[j], ab = s_ab[j], co = s_co[j];
          const float2 dx = __fadd2_rn(f2(xy.x, xy.y), npx);
          const float2 dy = __fadd2_rn(f2(xy.z, xy.w), npy);
          const float2 tt = __ffma2_rn(f2(ab.x, ab.y), dx, __fmul2_rn(f2(ab.z, ab.w), dy));
          // base-2 exponent of alpha, log2 o folded in: alpha = min(0.99, 2^ee)
          const float2 ee = __ffma2_rn(tt, dx, __ffma2_rn(__fmul2_rn(f2(co.x, co.y), dy), dy, f2(co.z, co.w)));
          float2 al = f2(ex2_approx(ee.x), ex2_approx(ee.y));
          if constexpr (decltype(clampc)::value) al = f2(fminf(kAlphaMax, al.x), fminf(kAlphaMax, al.y));
          const bool on0 = T.x >= kTStop && ee.x >= kLog2AlphaMin;
          const bool on1 = T.y >= kTStop && ee.y >= kLog2AlphaMin;
          const float2 wt = __fmul2_rn(al, T);
          const float2 w = f2(on0 ? wt.x : 0.f, on1 ? wt.y : 0.f);
          const float4 rg = s_rg[j], bd = s_bd[j];
          C0 = __ffma2_rn(f2(rg.x, rg.y), w, C0);
          C1 = __ffma2_rn(f2(rg.z, rg.w), w, C1);
          C2 = __ffma2_rn(f2(bd.x, bd.y), w, C2);
          D = __ffma2_rn(f2(bd.z, bd.w), w, D);
          T = __ffma2_rn(w, m1, T);  // T - w, rounded once
          last0 = on0 ? (uint32_t)(b + j + 1) : last0;
          last1 = on1 ? (uint32_t)(b + j + 1) : last1;
      };
      using Clamp = std::true_type;
      using NoClamp = std::false_type;
      if (jn == 8 && !((clamp_mask >> (j0 >> 3)) & 1u)) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) entry(jj, NoClamp{});
      } else if (jn == 8) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) entry(jj, Clamp{});
      } else {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < jn) entry(jj, Clamp{});
      }
    }
  }
  const size_t HW = (size_t)V.width * V.height;
  if (in0) {
    const size_t o = (size_t)py * V.width + px;
    V.rgb[o] = C0.x; V.rgb[HW + o] = C1.x; V.rgb[2 * HW + o] = C2.x;
    V.depth[o] = D.x; V.alpha[o] = 1.f - T.x; V.T_final[o] = T.x; V.n_contrib[o] = last0;
  }
  if (in1) {
    const size_t o = (size_t)(py + 1) * V.width + px;
    V.rgb[o] = C0.y; V.rgb[HW + o] = C1.y; V.rgb[2 * HW + o] = C2.y;
    V.depth[o] = D.y; V.alpha[o] = 1.f - T.y; V.T_final[o] = T.y; V.n_contrib[o] = last1;
  }
}

// Backward blend (reverse of Eq. 11).  A batch of kBwdBatch entries is walked back to
// front by every pixel (pixel phase), which leaves per (pixel, entry) the two scalars
// the Gaussian needs: gp = dL/dalpha * alpha (zero where the clamp or a cutoff holds)
// and w = alpha T (the weight of its colour and depth).  They go through shared memory
// transposed, and in the Gaussian phase each half-warp sums one tile row of them per
// entry into the ten moments the chain rule of Eq. 1-2 needs.
constexpr int kBwdBatch = 16;
constexpr int kBwdStride = kBwdBatch + 2;  // padded row: 16-byte aligned, conflict-free both ways
// CTAs per tile: each takes 16 / kBwdSplit rows, so its barriers wait only for the pixels
// of its own part and it walks only down to its own longest list
constexpr int kBwdSplit = 1;
constexpr int kBwdThreads = kTilePix / kBwdSplit;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kMom = 10;
constexpr int kRedStride = kMom + 1;     // per-entry row of partial moments (odd: no conflicts)

struct BwdSmem {
  float2 gw[kBwdThreads][kBwdStride];       // (gp, w) per pixel and entry; after the Gaussian
                                            // phase each warp's rows hold its partial moments
  float4 g[kBwdThreads];                    // per pixel dL/d(r, g, b, depth)
  float4 raw[2][kBwdBatch][3];              // records of the next batch, landed by cp.async
  // entries 2p and 2p+1 side by side, so one 16-byte load gives two operand pairs
  float4 q_xy[2][kBwdBatch / 2];            // (x, x', y, y') tile-relative centre
  float4 q_ab[2][kBwdBatch / 2];            // (A, A', B, B') scaled conic
  float4 q_co[2][kBwdBatch / 2];            // (C, C', log2 o, log2 o')
  float4 q_rg[2][kBwdBatch / 2];            // (r, r', g, g')
  float4 q_bd[2][kBwdBatch / 2];            // (b, b', depth, depth')
  uint32_t idx[2][kBwdBatch];
  int clamp[2];                             // the 0.99 clamp may bind for an entry of the batch
  int lmax;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(kBwdThreads, 5 * kBwdSplit) k_blend_bwd(const __grid_constant__ ViewTable vt,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ vals,
                                                           const uint2* __restrict__ ranges,
                                                           const uint32_t* __restrict__ order,
                                                           float4* __restrict__ moments) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
  const int tile = order ? (int)order[blockIdx.x / kBwdSplit] : (int)(blockIdx.x / kBwdSplit);
  if ((unsigned)tile >= (unsigned)vt.n_tiles) return;  // an order left by another render
  const int part = blockIdx.x % kBwdSplit;
  const int row0 = part * (kTile / kBwdSplit);  // first tile row of this CTA's part
  const View& V = vt.v[view_of_tile(vt, tile)];
  const int local = tile - V.tile_base;
  const int x0 = (local % V.tiles_x) * kTile, y0 = (local / V.tiles_x) * kTile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // each warp an 8x4 block of the tile (bx = warp & 1, by = warp >> 1); half-warp h holds
  // its rows 2h and 2h + 1, eight pixels each
  const int lx = 8 * (warp & 1) + (lane & 7), ly = row0 + 4 * (warp >> 1) + (lane >> 3);
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < V.width && py < V.height;
  const float pxf = (float)lx, pyf = (float)ly, x0f = (float)x0, y0f = (float)y0;
  const uint2 range = ranges[tile];
  if (t == 0) S.lmax = 0;
  size_t o = (size_t)py * V.width + px, HW = (size_t)V.width * V.height;
  uint32_t nc = 0;
  float T = 1.f, Tf = 1.f, gR = 0.f, gG = 0.f, gB = 0.f, gD = 0.f, gA = 0.f;
  if (inside) {
    nc = V.n_contrib[o];
    Tf = V.T_final[o];
    T = Tf;
    if (V.g_rgb) { gR = V.g_rgb[o]; gG = V.g_rgb[HW + o]; gB = V.g_rgb[2 * HW + o]; }
    if (V.g_depth) gD = V.g_depth[o];
    if (V.g_alpha) gA = V.g_alpha[o];
  }
  S.g[t] = make_float4(gR, gG, gB, gD);
  __syncthreads();
  if (nc) atomicMax(&S.lmax, (int)nc);
  __syncthreads();
  const int L = S.lmax;
  const float gAT = gA * Tf;
  float sig = 0.f;
  // Gaussian-phase lane roles: entry e of the batch, the half-warp's two pixel rows
  const int e = lane & (kBwdBatch - 1), half = lane >> 4;
  const int prow = warp * 32 + half * kTile;
  float* const red_own = reinterpret_cast<float*>(&S.gw[warp * 32][0]);
  // Batches run back to front.  Threads t < kBwdBatch keep the list indices of the next
  // two batches in registers and land the next batch's records by cp.async, so the
  // gather overlaps the current batch.
  int base = L > 0 ? ((L - 1) / kBwdBatch) * kBwdBatch : -1;
  uint32_t idx_cur = 0, idx_next = 0;
  if (t < kBwdBatch && base >= 0) {
    if (base + t < L) {
      idx_cur = vals[range.x + base + t];
      const float4* src = rec + 3 * (size_t)idx_cur;
      cp_async16(&S.raw[0][t][0], src);
      cp_async16(&S.raw[0][t][1], src + 1);
      cp_async16(&S.raw[0][t][2], src + 2);
    }
    cp_async_commit();
    if (base >= kBwdBatch) idx_next = vals[range.x + base - kBwdBatch + t];
  }
  for (int buf = 0; base >= 0; base -= kBwdBatch, buf ^= 1) {
    const int cnt = min(kBwdBatch, L - base);
    if (t < kBwdBatch) {
      cp_async_wait_all();
      // entries past the end of a partial batch are zeroed: their pair partner then
      // reads finite values (they enter with alpha = 0)
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
      float x = 0.f, y = 0.f;
      bool cl = false;
      if (t < cnt) {
        r0 = S.raw[buf][t][0];
        r1 = S.raw[buf][t][1];
        r2 = S.raw[buf][t][2];
        x = __fadd_rn(__fsub_rn(r0.x, x0f), r0.z);
        y = __fadd_rn(__fsub_rn(r0.y, y0f), r0.w);
        S.idx[buf][t] = idx_cur;
        cl = clamp_possible(r1);
      }
      const uint32_t bal = __ballot_sync((1u << kBwdBatch) - 1u, cl);
      if (t == 0) S.clamp[buf] = bal != 0u;
      const int pp = t >> 1, sl = t & 1;
      float* const qxy = reinterpret_cast<float*>(&S.q_xy[buf][pp]);
      float* const qab = reinterpret_cast<float*>(&S.q_ab[buf][pp]);
      float* const qco = reinterpret_cast<float*>(&S.q_co[buf][pp]);
      float* const qrg = reinterpret_cast<float*>(&S.q_rg[buf][pp]);
      float* const qbd = reinterpret_cast<float*>(&S.q_bd[buf][pp]);
      qxy[sl] = x; qxy[2 + sl] = y;
      qab[sl] = r1.x; qab[2 + sl] = r1.y;
      qco[sl] = r1.z; qco[2 + sl] = r1.w;
      qrg[sl] = r2.x; qrg[2 + sl] = r2.y;
      qbd[sl] = r2.z; qbd[2 + sl] = r2.w;
      if (base >= kBwdBatch) {  // the next batch is full: every t < kBwdBatch has an entry
        const float4* src = rec + 3 * (size_t)idx_next;
        cp_async16(&S.raw[buf ^ 1][t][0], src);
        cp_async16(&S.raw[buf ^ 1][t][1], src + 1);
        cp_async16(&S.raw[buf ^ 1][t][2], src + 2);
        cp_async_commit();
        idx_cur = idx_next;
        if (base >= 2 * kBwdBatch) idx_next = vals[range.x + base - 2 * kBwdBatch + t];
      }
    }
    __syncthreads();
    // pixel phase: branch-free back-to-front recursion; sigma = S . g (colour and depth
    // behind, dotted with the pixel's cotangent) is all the recursion needs
    const bool wrun = __any_sync(0xffffffffu, (uint32_t)base < nc);
    if (wrun) {
      const int lim = (int)nc - base;
      // chk: whether some pixel of the warp ends inside the batch (then j < lim matters).
      // Entries go in pairs (2p+1 first, then 2p): what does not depend on the running
      // T and sigma is computed for both at once on packed f32 pairs.
      const float2 npx = make_float2(-pxf, -pxf), npy = make_float2(-pyf, -pyf);
      const float2 gR2 = make_float2(gR, gR), gG2 = make_float2(gG, gG), gB2 = make_float2(gB, gB),
                   gD2 = make_float2(gD, gD), gAT2 = make_float2(gAT, gAT);
      const float2 m1 = make_float2(-1.f, -1.f), one2 = make_float2(1.f, 1.f);
      auto pair = [&](int p, auto chk, auto clampc) {
          constexpr bool kClamp = decltype(clampc)::value;
          const float4 xy = S.q_xy[buf][p], ab = S.q_ab[buf][p], co = S.q_co[buf][p];
          const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), npx);
          const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), npy);
          const float2 tt = __ffma2_rn(make_float2(ab.x, ab.y), dx, __fmul2_rn(make_float2(ab.z, ab.w), dy));
          const float2 ee = __ffma2_rn(tt, dx, __ffma2_rn(__fmul2_rn(make_float2(co.x, co.y), dy), dy,
                                                          make_float2(co.z, co.w)));
          const float2 a = make_float2(ex2_approx(ee.x), ex2_approx(ee.y));  // alpha before the clamp
          bool on0 = ee.x >= kLog2AlphaMin, on1 = ee.y >= kLog2AlphaMin;
          if constexpr (decltype(chk)::value) {
            on0 = on0 && 2 * p < lim;
            on1 = on1 && 2 * p + 1 < lim;
          }
          const float2 alc = kClamp ? make_float2(on0 ? fminf(kAlphaMax, a.x) : 0.f, on1 ? fminf(kAlphaMax, a.y) : 0.f)
                                    : make_float2(on0 ? a.x : 0.f, on1 ? a.y : 0.f);
          const float2 om = __ffma2_rn(alc, m1, one2);  // 1 - alpha
          const float2 rom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
          const float4 rg = S.q_rg[buf][p], bd = S.q_bd[buf][p];
          const float2 cg = __ffma2_rn(make_float2(rg.x, rg.y), gR2,
                                       __ffma2_rn(make_float2(rg.z, rg.w), gG2,
                                                  __ffma2_rn(make_float2(bd.x, bd.y), gB2,
                                                             __fmul2_rn(make_float2(bd.z, bd.w), gD2))));
          const float2 gar = __fmul2_rn(gAT2, rom);
          // the recursion itself (T before each entry, sigma behind it) stays scalar; the
          // rest of dL/dalpha goes through one packed FMA
          const float Tb1 = T * rom.y;
          const float d1 = cg.y - sig;
          sig = fmaf(alc.y, d1, sig);
          const float Tb0 = Tb1 * rom.x;
          const float d0 = cg.x - sig;
          sig = fmaf(alc.x, d0, sig);
          T = Tb0;
          const float2 Tb = make_float2(Tb0, Tb1);
          const float2 dLda = __ffma2_rn(Tb, make_float2(d0, d1), gar);
          // dL/dalpha * alpha where alpha is unclamped (alc = alpha there; 0 when skipped)
          const float2 gp = __fmul2_rn(dLda, alc);
          const float2 w = __fmul2_rn(alc, Tb);
          *reinterpret_cast<float4*>(&S.gw[t][2 * p]) =
              kClamp ? make_float4(a.x <= kAlphaMax ? gp.x : 0.f, w.x, a.y <= kAlphaMax ? gp.y : 0.f, w.y)
                     : make_float4(gp.x, w.x, gp.y, w.y);
      };
      using Yes = std::true_type;
      using No = std::false_type;
      const bool bclamp = S.clamp[buf] != 0;
      if (cnt == kBwdBatch && __all_sync(0xffffffffu, lim >= kBwdBatch)) {  // every pixel walks it all
        if (bclamp) {
#pragma unroll
          for (int p = kBwdBatch / 2 - 1; p >= 0; --p) pair(p, No{}, Yes{});
        } else {
#pragma unroll
          for (int p = kBwdBatch / 2 - 1; p >= 0; --p) pair(p, No{}, No{});
        }
      } else if (cnt == kBwdBatch) {  // full batch: no per-entry guard
        if (bclamp) {
#pragma unroll
          for (int p = kBwdBatch / 2 - 1; p >= 0; --p) pair(p, Yes{}, Yes{});
        } else {
#pragma unroll
          for (int p = kBwdBatch / 2 - 1; p >= 0; --p) pair(p, Yes{}, No{});
        }
      } else {
#pragma unroll
        for (int p = kBwdBatch / 2 - 1; p >= 0; --p)
          if (2 * p < cnt) pair(p, Yes{}, Yes{});
      }
    }
    // Gaussian phase for the 32 pixels this warp just walked (skipped when all of them
    // ended before the batch; tracking per-pixel contributions costs more than it
    // saves): per row sums of gp, k gp, k^2 gp with k the column offset from the centre
    // of the block's eight columns, then the moments about the centre of the Gaussian
    // (dx = xy.x - x_centre - k, dy constant along each row).
    __syncwarp();  // this warp's gw rows are written by its own lanes
    float m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.f;
    if (wrun && e < cnt) {
      float s0[2] = {0.f, 0.f}, k1[2] = {0.f, 0.f}, k2[2] = {0.f, 0.f};
      float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
#pragma unroll
      for (int k = 0; k < kTile; ++k) {
        const float2 gw = S.gw[prow + k][e];
        const float4 gg = S.g[prow + k];
        constexpr float c0 = -3.5f;
        const float kc = c0 + (float)(k & 7);
        const int r = k >> 3;
        s0[r] += gw.x;
        k1[r] = fmaf(kc, gw.x, k1[r]);
        k2[r] = fmaf(kc * kc, gw.x, k2[r]);
        w0 = fmaf(gw.y, gg.x, w0);
        w1 = fmaf(gw.y, gg.y, w1);
        w2 = fmaf(gw.y, gg.z, w2);
        w3 = fmaf(gw.y, gg.w, w3);
      }
      const float* const qxy = reinterpret_cast<const float*>(&S.q_xy[buf][e >> 1]);
      const float xc = qxy[e & 1] - (float)(8 * (warp & 1)) - 3.5f;
      const float dy0 = qxy[2 + (e & 1)] - (float)(row0 + 4 * (warp >> 1) + 2 * half);
      const float dy1 = dy0 - 1.f;
      const float ma = fmaf(xc, s0[0], -k1[0]), mb = fmaf(xc, s0[1], -k1[1]);  // sum gp (xc - kc)
      m[0] = s0[0] + s0[1];
      m[1] = ma + mb;
      m[2] = fmaf(dy0, s0[0], dy1 * s0[1]);
      m[3] = fmaf(xc, fmaf(xc, s0[0], -2.f * k1[0]), k2[0]) +   // sum gp (xc - kc)^2
             fmaf(xc, fmaf(xc, s0[1], -2.f * k1[1]), k2[1]);
      m[4] = fmaf(dy0, ma, dy1 * mb);
      m[5] = fmaf(dy0 * dy0, s0[0], dy1 * dy1 * s0[1]);
      m[6] = w0;
      m[7] = w1;
      m[8] = w2;
      m[9] = w3;
    }
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] += __shfl_down_sync(0xffffffffu, m[k], kTile);
    __syncwarp();  // every lane is done reading this warp's gw rows
    if (half == 0) {
#pragma unroll
      for (int k = 0; k < kMom; ++k) red_own[e * kRedStride + k] = m[k];
    }
    __syncthreads();
    // Cross-warp sum, spread over all threads: half-warp q owns entries q, q + 2 warps, ...,
    // its lane k moment k; lanes 0, 4, 8 then add four consecutive moments with one
    // vector atomic.
    for (int q = 2 * warp + half; q < kBwdBatch; q += 2 * kBwdWarps) {
      const int k = e;
      float r = 0.f;
      if (q < cnt && k < kMom) {
#pragma unroll
        for (int ww = 0; ww < kBwdWarps; ++ww)
          r += reinterpret_cast<const float*>(&S.gw[ww * 32][0])[q * kRedStride + k];
      }
      const float r1 = __shfl_down_sync(0xffffffffu, r, 1);
      const float r2 = __shfl_down_sync(0xffffffffu, r, 2);
      const float r3 = __shfl_down_sync(0xffffffffu, r, 3);
      const uint32_t nz = __ballot_sync(0xffffffffu, r != 0.f) >> (16 * half);
      if (q < cnt && (k & 3) == 0 && k < kMom && (nz & 0xffffu)) {
        float4* dst = moments + 3 * (size_t)S.idx[buf][q] + (k >> 2);
        atomicAdd(dst, make_float4(r, r1, (k < 8) ? r2 : 0.f, (k < 8) ? r3 : 0.f));
      }
    }
    // No barrier here: the next batch's records go to the other buffer, and gw is next
    // written after the next batch's barrier.
  }
}

// Counting pass over the saved forward state: per pixel, entries evaluated by the
// forward pass (up to its stop, else the whole range), how many of them contributed,
// and how many the backward pass walks (up to the last contributor).
__global__ void __launch_bounds__(kTilePix) k_frag_stats(const __grid_constant__ ViewTable vt,
                                                         const float4* __restrict__ rec,
                                                         const uint32_t* __restrict__ vals,
                                                         const uint2* __restrict__ ranges,
                                                         unsigned long long* __restrict__ out) {
  const int tile = blockIdx.x;
  const View& V = vt.v[view_of_tile(vt, tile)];
  const int local = tile - V.tile_base;
  const int x0 = (local % V.tiles_x) * kTile, y0 = (local / V.tiles_x) * kTile;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = x0 + lx, py = y0 + ly;
  unsigned long long ev = 0, co = 0, bw = 0;
  if (px < V.width && py < V.height) {
    size_t o = (size_t)py * V.width + px;
    uint32_t nc = V.n_contrib[o];
    float Tf = V.T_final[o];
    uint2 range = ranges[tile];
    uint32_t ne = Tf < kTStop ? nc : range.y - range.x;
    const float x0f = (float)x0, y0f = (float)y0;
    for (uint32_t e = 0; e < ne; ++e) {
      uint32_t idx = vals[range.x + e];
      float4 r0 = rec[3 * (size_t)idx], r1 = rec[3 * (size_t)idx + 1];
      float2 xy = make_float2(__fadd_rn(__fsub_rn(r0.x, x0f), r0.z), __fadd_rn(__fsub_rn(r0.y, y0f), r0.w));
      float dx, dy;
      if (frag_exp2(xy, r1, (float)lx, (float)ly, dx, dy) >= kLog2AlphaMin) ++co;
    }
    ev = ne;
    bw = nc;
  }
  // padded work: a warp (tile) issues its longest pixel's list for all its lanes (pixels).
  // Forward warps hold 8x8 pixel blocks (four per tile), backward warps 8x4 blocks (eight).
  __shared__ unsigned long long s_max[2], s_fw[4], s_bw[8];
  if (threadIdx.x < 4) s_fw[threadIdx.x] = 0;
  if (threadIdx.x < 8) s_bw[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_max[0] = s_max[1] = 0;
  __syncthreads();
  atomicMax(&s_fw[2 * (ly >> 3) + (lx >> 3)], ev);
  atomicMax(&s_bw[2 * (ly >> 2) + (lx >> 3)], bw);
  atomicMax(&s_max[0], ev);
  atomicMax(&s_max[1], bw);
  for (int s = 16; s; s >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, s);
    co += __shfl_xor_sync(0xffffffffu, co, s);
    bw += __shfl_xor_sync(0xffffffffu, bw, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], ev);
    atomicAdd(&out[1], co);
    atomicAdd(&out[2], bw);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&out[3], (unsigned long long)kTilePix * s_max[0]);
    atomicAdd(&out[4], (unsigned long long)kTilePix * s_max[1]);
    atomicAdd(&out[5], 64ull * (s_fw[0] + s_fw[1] + s_fw[2] + s_fw[3]));
    atomicAdd(&out[6], 32ull * (s_bw[0] + s_bw[1] + s_bw[2] + s_bw[3] + s_bw[4] + s_bw[5] + s_bw[6] + s_bw[7]));
  }
}

// Longest-first tile order: the blend grids are dispatched in block order, so tiles are
// given to blocks by list length (classes of 128 entries, longest class first; inside a
// class, runs of tiles in index order).  Long tiles then start early instead of running
// alone at the end of the grid.
constexpr int kOrderBuckets = 64;

__device__ __forceinline__ int order_class(uint2 r) {  // 0 = the longest lists
  const uint32_t len = r.y - r.x;
  return kOrderBuckets - 1 - (int)min(len >> 7, (uint32_t)(kOrderBuckets - 1));
}

__global__ void __launch_bounds__(256) k_order_count(const uint2* __restrict__ ranges, int n_tiles,
                                                     uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) atomicAdd(&s_cnt[order_class(ranges[t])], 1u);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets && s_cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_order_scatter(const uint2* __restrict__ ranges, int n_tiles,
                                                       const uint32_t* __restrict__ counts,
                                                       uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_wcnt[8][kOrderBuckets];  // per warp and class, then exclusive offsets
  __shared__ uint32_t s_base[kOrderBuckets];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < 8 * kOrderBuckets; k += blockDim.x) (&s_wcnt[0][0])[k] = 0;
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = t < n_tiles ? order_class(ranges[t]) : kOrderBuckets;
  // rank among the earlier lanes of the same class, so each block's run of a class
  // keeps tile order
  const uint32_t peers = __match_any_sync(0xffffffffu, c);
  const uint32_t rank_w = __popc(peers & ((1u << lane) - 1u));
  if (c < kOrderBuckets && rank_w == 0) s_wcnt[w][c] = __popc(peers);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets) {
    const int k = threadIdx.x;
    uint32_t run = 0;
    for (int ww = 0; ww < 8; ++ww) {
      const uint32_t x = s_wcnt[ww][k];
      s_wcnt[ww][k] = run;
      run += x;
    }
    uint32_t base = 0;
    for (int h = 0; h < k; ++h) base += counts[h];
    s_base[k] = run ? base + atomicAdd(&cursor[k], run) : 0u;
  }
  __syncthreads();
  if (c < kOrderBuckets) {
    const uint32_t pos = s_base[c] + s_wcnt[w][c] + rank_w;  // < n_tiles: the classes partition the tiles
    if (pos < (uint32_t)n_tiles) order[pos] = (uint32_t)t;
  }
}

}  // namespace

cudaError_t launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* counts, uint32_t* order,
                              cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * kOrderBuckets * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)div_up(n_tiles, 256);
  k_order_count<<<grid, 256, 0, s>>>(ranges, n_tiles, counts);
  count_launch();
  k_order_scatter<<<grid, 256, 0, s>>>(ranges, n_tiles, counts, counts + kOrderBuckets, order);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_frag_stats(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                              const uint2* ranges, unsigned long long* out, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  k_frag_stats<<<vt.n_tiles, kTilePix, 0, s>>>(vt, rec, vals, ranges, out);
  count_launch();
  return cudaGetLastError();
}


size_t blend_bwd_smem() { return sizeof(BwdSmem); }

cudaError_t launch_blend_fwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, const uint32_t* order, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  k_blend_fwd<<<vt.n_tiles, kFwdThreads, 0, s>>>(vt, rec, vals, ranges, order);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, const uint32_t* order, float4* moments, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_blend_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(BwdSmem));
  if (e != cudaSuccess) return e;
  k_blend_bwd<<<vt.n_tiles * kBwdSplit, kBwdThreads, sizeof(BwdSmem), s>>>(vt, rec, vals, ranges, order, moments);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgs
