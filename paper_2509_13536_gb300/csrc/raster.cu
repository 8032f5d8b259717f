// Tile blend kernels (Sec. II-E, Eq. 11), forward and reverse, sm_103a.
//
// One CTA of 256 threads owns one 16x16 tile of one view.  Forward: batches of
// 256 sorted entries are gathered into shared memory (one entry per thread) and
// every thread walks them front to back for its pixel, with transmittance and the
// colour/depth sums in registers; the CTA leaves as soon as all its pixels stopped.
//
// Reverse: the tile's entries are walked back to front in batches of 16.  In the
// pixel phase each thread runs the back-to-front recursion for its pixel (T recovered
// by division; of the colour and depth behind each Gaussian only their dot product
// with the pixel's cotangent is needed, one scalar) and writes two numbers per
// (pixel, entry) into shared memory: gp = dL/dpower and the blend weight w.  In the
// Gaussian phase each half-warp owns one tile row and each of its lanes one entry; it
// sums gp, k gp, k^2 gp (k the column) and w times the cotangent along the row and forms
// the ten moments the per-Gaussian chain rule needs; the eight warps' partial sums meet
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

__global__ void __launch_bounds__(kTilePix) k_blend_fwd(const __grid_constant__ ViewTable vt,
                                                        const float4* __restrict__ rec,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint2* __restrict__ ranges) {
  __shared__ float2 s_xy[kTilePix];
  __shared__ float4 s_co[kTilePix];
  __shared__ float4 s_col[kTilePix];
  const int tile = blockIdx.x;
  const View& V = vt.v[view_of_tile(vt, tile)];
  const int local = tile - V.tile_base;
  const int x0 = (local % V.tiles_x) * kTile, y0 = (local / V.tiles_x) * kTile;
  const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
  const int px = x0 + lx, py = y0 + ly;
  const bool inside = px < V.width && py < V.height;
  const float pxf = (float)lx, pyf = (float)ly, x0f = (float)x0, y0f = (float)y0;
  const uint2 range = ranges[tile];
  const int n = (int)(range.y - range.x);
  // A pixel blends an entry while T (before it) is still >= kTStop: the Gaussian that
  // takes T below the threshold is the last one blended.  Pixels outside the image
  // start at T = 0 and take nothing.
  float T = inside ? 1.f : 0.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  uint32_t last = 0;
  for (int b = 0; b < n; b += kTilePix) {
    if (__syncthreads_count(T >= kTStop) == 0) break;
    int e = b + threadIdx.x;
    if (e < n) {
      uint32_t idx = vals[range.x + e];
      float4 r0 = rec[3 * (size_t)idx], r1 = rec[3 * (size_t)idx + 1], r2 = rec[3 * (size_t)idx + 2];
      s_xy[threadIdx.x] = make_float2(__fadd_rn(__fsub_rn(r0.x, x0f), r0.z), __fadd_rn(__fsub_rn(r0.y, y0f), r0.w));
      s_co[threadIdx.x] = r1;
      s_col[threadIdx.x] = r2;
    }
    __syncthreads();
    const int cnt = min(kTilePix, n - b);
    for (int j0 = 0; j0 < cnt; j0 += 8) {
      if (__all_sync(0xffffffffu, T < kTStop)) break;
      const int jn = min(8, cnt - j0);
      auto entry = [&](int jj) {
          const int j = j0 + jj;
          float dx, dy;
          const float4 co = s_co[j];
          const float p2 = frag_exp2(s_xy[j], co, pxf, pyf, dx, dy);
          const float a = __fmul_rn(co.w, ex2_approx(p2));
          const float al = fminf(kAlphaMax, a);
          const bool on = T >= kTStop && p2 <= 0.f && al >= kAlphaMin;
          const float4 c = s_col[j];
          const float w = on ? __fmul_rn(al, T) : 0.f;
          C0 = __fmaf_rn(c.x, w, C0);
          C1 = __fmaf_rn(c.y, w, C1);
          C2 = __fmaf_rn(c.z, w, C2);
          D = __fmaf_rn(c.w, w, D);
          T = __fsub_rn(T, w);
          last = on ? (uint32_t)(b + j + 1) : last;
      };
      if (jn == 8) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) entry(jj);
      } else {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
          if (jj < jn) entry(jj);
      }
    }
  }
  if (inside) {
    size_t o = (size_t)py * V.width + px, HW = (size_t)V.width * V.height;
    V.rgb[o] = C0;
    V.rgb[HW + o] = C1;
    V.rgb[2 * HW + o] = C2;
    V.depth[o] = D;
    V.alpha[o] = 1.f - T;
    V.T_final[o] = T;
    V.n_contrib[o] = last;
  }
}

// Backward blend (reverse of Eq. 11).  A batch of kBwdBatch entries is walked back to
// front by every pixel (pixel phase), which leaves per (pixel, entry) the two scalars
// the Gaussian needs: gp = dL/dalpha * alpha (zero where the clamp or a cutoff holds)
// and w = alpha T (the weight of its colour and depth).  They go through shared memory
// transposed, and in the Gaussian phase each half-warp sums one tile row of them per
// entry into the ten moments the chain rule of Eq. 1-2 needs.
constexpr int kBwdBatch = 16;
constexpr int kBwdStride = kBwdBatch + 1;  // padded row: conflict-free both ways
constexpr int kBwdWarps = kTilePix / 32;
constexpr int kMom = 10;
constexpr int kRedStride = kMom + 1;     // per-entry row of partial moments (odd: no conflicts)

struct BwdSmem {
  float2 gw[kTilePix][kBwdStride];          // (gp, w) per pixel and entry; after the Gaussian
                                            // phase each warp's rows hold its partial moments
  float4 g[kTilePix];                       // per pixel dL/d(r, g, b, depth)
  float4 raw[2][kBwdBatch][3];              // records of the next batch, landed by cp.async
  float2 xy[2][kBwdBatch];                  // tile-relative centre
  float4 co[2][kBwdBatch];                  // scaled conic, opacity
  float4 col[2][kBwdBatch];                 // colour, depth
  uint32_t idx[2][kBwdBatch];
  int lmax;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(kTilePix, 5) k_blend_bwd(const __grid_constant__ ViewTable vt,
                                                           const float4* __restrict__ rec,
                                                           const uint32_t* __restrict__ vals,
                                                           const uint2* __restrict__ ranges,
                                                           float4* __restrict__ moments) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
  const int tile = blockIdx.x;
  const View& V = vt.v[view_of_tile(vt, tile)];
  const int local = tile - V.tile_base;
  const int x0 = (local % V.tiles_x) * kTile, y0 = (local / V.tiles_x) * kTile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int lx = t & (kTile - 1), ly = t / kTile;
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
  // Gaussian-phase lane roles: entry e of the batch, tile row 2 warp + half
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
      if (t < cnt) {
        const float4 r0 = S.raw[buf][t][0];
        S.xy[buf][t] = make_float2(__fadd_rn(__fsub_rn(r0.x, x0f), r0.z), __fadd_rn(__fsub_rn(r0.y, y0f), r0.w));
        S.co[buf][t] = S.raw[buf][t][1];
        S.col[buf][t] = S.raw[buf][t][2];
        S.idx[buf][t] = idx_cur;
      }
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
      // chk: whether some pixel of the warp ends inside the batch (then j < lim matters)
      auto entry = [&](int j, auto chk) {
          float dx, dy;
          const float4 co = S.co[buf][j];
          const float p2 = frag_exp2(S.xy[buf][j], co, pxf, pyf, dx, dy);
          const float a = __fmul_rn(co.w, ex2_approx(p2));
          const float al = fminf(kAlphaMax, a);
          bool on = p2 <= 0.f && al >= kAlphaMin;
          if constexpr (decltype(chk)::value) on = on && j < lim;
          const float alc = on ? al : 0.f;
          const float4 c = S.col[buf][j];
          const float rom = __fdividef(1.f, 1.f - alc);
          const float Tb = T * rom;
          const float cg = fmaf(c.x, gR, fmaf(c.y, gG, fmaf(c.z, gB, c.w * gD)));
          const float d = cg - sig;
          const float dLda = fmaf(Tb, d, gAT * rom);
          sig = fmaf(alc, d, sig);
          S.gw[t][j] = make_float2((on && a <= kAlphaMax) ? dLda * a : 0.f, alc * Tb);
          T = Tb;
      };
      using Yes = std::true_type;
      using No = std::false_type;
      if (cnt == kBwdBatch && __all_sync(0xffffffffu, lim >= kBwdBatch)) {  // every pixel walks it all
#pragma unroll
        for (int j = kBwdBatch - 1; j >= 0; --j) entry(j, No{});
      } else if (cnt == kBwdBatch) {  // full batch: no per-entry guard
#pragma unroll
        for (int j = kBwdBatch - 1; j >= 0; --j) entry(j, Yes{});
      } else {
#pragma unroll
        for (int j = kBwdBatch - 1; j >= 0; --j)
          if (j < cnt) entry(j, Yes{});
      }
    }
    // Gaussian phase for the 32 pixels this warp just walked (skipped when all of them
    // ended before the batch; tracking per-pixel contributions costs more than it
    // saves): per row sums of gp, k gp, k^2 gp with
    // k the column offset from the tile centre, then the moments about the centre of
    // the Gaussian (dx = xy.x - 7.5 - k, dy constant along the row).
    __syncwarp();  // this warp's gw rows are written by its own lanes
    float m[kMom];
#pragma unroll
    for (int k = 0; k < kMom; ++k) m[k] = 0.f;
    if (wrun && e < cnt) {
      float s0 = 0.f, k1 = 0.f, k2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
#pragma unroll
      for (int k = 0; k < kTile; ++k) {
        const float2 gw = S.gw[prow + k][e];
        const float4 gg = S.g[prow + k];
        constexpr float c0 = -7.5f;
        const float kc = c0 + (float)k;
        s0 += gw.x;
        k1 = fmaf(kc, gw.x, k1);
        k2 = fmaf(kc * kc, gw.x, k2);
        w0 = fmaf(gw.y, gg.x, w0);
        w1 = fmaf(gw.y, gg.y, w1);
        w2 = fmaf(gw.y, gg.z, w2);
        w3 = fmaf(gw.y, gg.w, w3);
      }
      const float2 xy = S.xy[buf][e];
      const float xc = xy.x - 7.5f, dy = xy.y - (float)(prow / kTile);
      const float m1 = fmaf(xc, s0, -k1);                    // sum gp (xc - kc)
      m[0] = s0;
      m[1] = m1;
      m[2] = dy * s0;
      m[3] = fmaf(xc, fmaf(xc, s0, -2.f * k1), k2);          // sum gp (xc - kc)^2
      m[4] = dy * m1;
      m[5] = dy * dy * s0;
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
    // Cross-warp sum, spread over all threads: half-warp q owns entry q, its lane k
    // moment k; lanes 0, 4, 8 then add four consecutive moments with one vector atomic.
    {
      const int q = 2 * warp + half, k = e;
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
      float p2 = frag_exp2(xy, r1, (float)lx, (float)ly, dx, dy);
      if (p2 > 0.f) continue;
      float a = __fmul_rn(r1.w, ex2_approx(p2));
      if (fminf(kAlphaMax, a) >= kAlphaMin) ++co;
    }
    ev = ne;
    bw = nc;
  }
  // padded work: a warp (tile) issues its longest pixel's list for all its lanes (pixels)
  unsigned long long ev_w = ev, bw_w = bw;
  for (int s = 16; s; s >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, s);
    co += __shfl_xor_sync(0xffffffffu, co, s);
    bw += __shfl_xor_sync(0xffffffffu, bw, s);
    ev_w = max(ev_w, __shfl_xor_sync(0xffffffffu, ev_w, s));
    bw_w = max(bw_w, __shfl_xor_sync(0xffffffffu, bw_w, s));
  }
  __shared__ unsigned long long s_max[2];
  if (threadIdx.x == 0) s_max[0] = s_max[1] = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], ev);
    atomicAdd(&out[1], co);
    atomicAdd(&out[2], bw);
    atomicAdd(&out[5], 32ull * ev_w);
    atomicAdd(&out[6], 32ull * bw_w);
    atomicMax(&s_max[0], ev_w);
    atomicMax(&s_max[1], bw_w);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&out[3], (unsigned long long)kTilePix * s_max[0]);
    atomicAdd(&out[4], (unsigned long long)kTilePix * s_max[1]);
  }
}

}  // namespace

cudaError_t launch_frag_stats(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                              const uint2* ranges, unsigned long long* out, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  k_frag_stats<<<vt.n_tiles, kTilePix, 0, s>>>(vt, rec, vals, ranges, out);
  count_launch();
  return cudaGetLastError();
}


size_t blend_bwd_smem() { return sizeof(BwdSmem); }

cudaError_t launch_blend_fwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  k_blend_fwd<<<vt.n_tiles, kTilePix, 0, s>>>(vt, rec, vals, ranges);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, float4* moments, cudaStream_t s) {
  if (vt.n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_blend_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(BwdSmem));
  if (e != cudaSuccess) return e;
  k_blend_bwd<<<vt.n_tiles, kTilePix, sizeof(BwdSmem), s>>>(vt, rec, vals, ranges, moments);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgs
