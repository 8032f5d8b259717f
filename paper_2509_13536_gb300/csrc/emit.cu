// Key emission (Sec. II-E, tile-based rendering), sm_103a: every drawn (view, Gaussian)
// item, in front-to-back order, writes one (global tile id, item) pair per tile its
// alpha >= 1/255 ellipse reaches.  The stable tile sort that follows then leaves each
// tile's list in depth order.
#include "internal.h"

namespace mgs {
namespace {

// Key emission writes, for item k of the front-to-back order, its keys at offsets[k] ..
// offsets[k] + count - 1: tiles row by row, columns ascending within a row.  It never
// writes more than the count the projection pass gave the item (the same culling
// functions on the same record); any shortfall is padded with the sentinel tile id
// n_tiles, which sorts last and is ignored by the range build.
//
// Warp-cooperative emission of one item's keys (all 32 lanes call it with the same
// item): lane l culls row y0 + l of a 32-row chunk, a warp scan places the rows, and the
// chunk's keys are written 32 positions at a time by consecutive lanes (coalesced), each
// lane finding its position's row by a binary search over the rows' prefixes.
__device__ __forceinline__ void emit_item_coop(uint32_t item, uint32_t off, uint32_t cnt, int lane,
                                               const uint2* __restrict__ rects, const float4* __restrict__ rec,
                                               int64_t N, const ViewTable& vt, uint32_t* __restrict__ tkeys,
                                               uint32_t* __restrict__ tvals) {
  const int v = view_of_item(vt, item);
  const View& V = vt.v[v];
  const uint2 rc = rects[item];
  const Cull q = make_cull(rec[3 * (size_t)item], rec[3 * (size_t)item + 1]);
  int y0 = rc.x >> 16, y1 = rc.y >> 16;
  cull_rows(q, y0, y1);
  const int rx0 = rc.x & 0xffff, rx1 = rc.y & 0xffff;
  uint32_t w = 0;
  for (int yb = y0; yb <= y1 && w < cnt; yb += 32) {
    const int y = yb + lane;
    int x0 = rx0, x1 = rx1;
    if (y <= y1) cull_cols(q, y, x0, x1);
    else x1 = x0 - 1;
    const uint32_t nx = x1 >= x0 ? (uint32_t)(x1 - x0 + 1) : 0u;
    uint32_t inc = nx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const uint32_t excl = inc - nx;
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    // the chunk's keys, 32 positions at a time: position c belongs to the last row whose
    // exclusive prefix is <= c (empty rows share the next row's prefix; rows past y1
    // carry the total)
    const uint32_t lim = min(total, cnt - w);
    for (uint32_t c0 = 0; c0 < lim; c0 += 32) {
      const uint32_t c = c0 + (uint32_t)lane;
      int r = 0;
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const uint32_t e = __shfl_sync(0xffffffffu, excl, (r + step) & 31);
        if (r + step < 32 && e <= c) r += step;
      }
      const int bx0 = __shfl_sync(0xffffffffu, x0, r);
      const uint32_t bex = __shfl_sync(0xffffffffu, excl, r);
      if (c < lim) {
        tkeys[off + w + c] = (uint32_t)(V.tile_base + (yb + r) * V.tiles_x + bx0) + (c - bex);
        tvals[off + w + c] = item;
      }
    }
    w += total;
  }
  for (uint32_t pos = w + lane; pos < cnt; pos += 32) {
    tkeys[off + pos] = (uint32_t)vt.n_tiles;
    tvals[off + pos] = item;
  }
}

// Items of at most kRowsMax tile rows are emitted through per-lane row tables: each lane
// culls its item's rows into shared memory (first column and the exclusive prefix of
// the row lengths), then the warp writes the keys of its 32 consecutive items -- one
// contiguous range of the output, since the offsets are a scan in the same order -- 32
// positions at a time: lane l takes position base + l, finds the item that owns it by
// a binary search over the lanes' offsets and the row by a search of that item's
// table.  Every store of the warp is coalesced.  Taller items go through the
// cooperative path above, one at a time.
constexpr int kRowsMax = 16;  // a power of two (binary search below)
constexpr int kRowStride = kRowsMax + 1;  // odd: lanes reading different items' tables spread over banks
constexpr int kEmitThreads = 256;

__global__ void __launch_bounds__(kEmitThreads) k_emit(int64_t n_vis, int64_t N, const uint32_t* __restrict__ dvals,
                                                       const uint32_t* __restrict__ offsets,
                                                       const uint32_t* __restrict__ touched,
                                                       const uint2* __restrict__ rects,
                                                       const float4* __restrict__ rec,
                                                       const __grid_constant__ ViewTable vt,
                                                       uint32_t* __restrict__ tkeys, uint32_t* __restrict__ tvals,
                                                       const uint32_t* __restrict__ n_vis_dev) {
  __shared__ uint32_t s_pre[kEmitThreads][kRowStride];  // exclusive prefix of the row lengths
  __shared__ int32_t s_x0[kEmitThreads][kRowStride];    // first tile column of each row
  if (n_vis_dev) n_vis = min(n_vis, (int64_t)*n_vis_dev);
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((k & ~int64_t(31)) >= n_vis) return;  // whole warp beyond the end
  const bool valid = k < n_vis;
  uint32_t item = 0, off = 0xffffffffu, cnt = 0;
  if (valid) {
    item = dvals[k];
    off = offsets[k];
    cnt = touched[item];
  }
  // this lane's item: rows after culling, their first columns and prefix lengths
  int rows = 0;
  uint32_t w = 0, tile_row0 = 0, tiles_x = 0;
  bool tall = false;
  if (cnt > 0) {
    const View& V = vt.v[view_of_item(vt, item)];
    const uint2 rc = rects[item];
    const Cull q = make_cull(rec[3 * (size_t)item], rec[3 * (size_t)item + 1]);
    int y0 = rc.x >> 16, y1 = rc.y >> 16;
    cull_rows(q, y0, y1);
    rows = max(0, y1 - y0 + 1);
    tiles_x = (uint32_t)V.tiles_x;
    tile_row0 = (uint32_t)(V.tile_base + y0 * V.tiles_x);
    if (rows > kRowsMax) {
      tall = true;
    } else {
      for (int r = 0; r < rows; ++r) {
        int x0 = rc.x & 0xffff, x1 = rc.y & 0xffff;
        cull_cols(q, y0 + r, x0, x1);
        s_pre[threadIdx.x][r] = w;
        s_x0[threadIdx.x][r] = x0;
        if (x1 >= x0) w += (uint32_t)(x1 - x0 + 1);
      }
    }
  }
  __syncwarp();
  const uint32_t first = __shfl_sync(0xffffffffu, off, 0);
  const uint32_t end = __reduce_max_sync(0xffffffffu, valid ? off + cnt : 0u);
  for (uint32_t base = first; base < end; base += 32) {
    const uint32_t p = base + (uint32_t)lane;
    // owner: the last lane whose range starts at or before p (lanes without keys share
    // the next lane's offset, lanes past the end carry an offset of 2^32 - 1)
    int o = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const int c = o + step;
      const uint32_t oc = __shfl_sync(0xffffffffu, off, c & 31);
      if (c < 32 && oc <= p) o = c;
    }
    const uint32_t o_off = __shfl_sync(0xffffffffu, off, o);
    const uint32_t o_item = __shfl_sync(0xffffffffu, item, o);
    const uint32_t o_w = __shfl_sync(0xffffffffu, w, o);
    const int o_rows = __shfl_sync(0xffffffffu, rows, o);
    const uint32_t o_row0 = __shfl_sync(0xffffffffu, tile_row0, o);
    const uint32_t o_tx = __shfl_sync(0xffffffffu, tiles_x, o);
    const bool o_tall = __shfl_sync(0xffffffffu, (int)tall, o) != 0;
    if (p >= end || o_tall) continue;
    const uint32_t qp = p - o_off;
    uint32_t key = (uint32_t)vt.n_tiles;  // shortfall: sentinel
    if (qp < o_w) {
      const uint32_t* pre = s_pre[wbase + o];
      int r = 0;
#pragma unroll
      for (int step = kRowsMax / 2; step; step >>= 1) {
        const int c = r + step;
        if (c < o_rows && pre[c] <= qp) r = c;
      }
      key = o_row0 + (uint32_t)r * o_tx + (uint32_t)s_x0[wbase + o][r] + (qp - pre[r]);
    }
    tkeys[p] = key;
    tvals[p] = o_item;
  }
  uint32_t big = __ballot_sync(0xffffffffu, tall);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const uint32_t it = __shfl_sync(0xffffffffu, item, src);
    const uint32_t of = __shfl_sync(0xffffffffu, off, src);
    const uint32_t cn = __shfl_sync(0xffffffffu, cnt, src);
    emit_item_coop(it, of, cn, lane, rects, rec, N, vt, tkeys, tvals);
  }
}

}  // namespace

cudaError_t launch_emit(int64_t n_vis, int64_t N, const uint32_t* dvals, const uint32_t* offsets,
                        const uint32_t* touched, const uint2* rects, const float4* rec, const ViewTable& vt,
                        uint32_t* tkeys, uint32_t* tvals, cudaStream_t s, const uint32_t* n_vis_dev) {
  if (n_vis <= 0) return cudaSuccess;
  k_emit<<<(unsigned)div_up(n_vis, kEmitThreads), kEmitThreads, 0, s>>>(n_vis, N, dvals, offsets, touched, rects, rec, vt, tkeys,
                                                       tvals, n_vis_dev);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgs
