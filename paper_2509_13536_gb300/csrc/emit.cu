// Key emission (Sec. II-E, tile-based rendering), sm_103a: every drawn (view, Gaussian)
// item, in front-to-back order, writes one (global tile id, item) pair per tile its
// alpha >= 1/255 ellipse reaches.  The stable tile sort that follows then leaves each
// tile's list in depth order.
#include "internal.h"

namespace mgs {
namespace {

// Key emission over the items in front-to-back order, one thread per item: the
// thread writes one (global tile id, item) pair per tile its alpha >= 1/255 ellipse
// reaches (row by row).  Items with more than 32 keys are written cooperatively by
// the whole warp afterwards.  An item never writes more than the count the projection
// pass gave it; any shortfall is padded with the sentinel tile id n_tiles, which sorts
// last and is ignored by the range build.
__device__ __forceinline__ void emit_item(uint32_t item, uint32_t off, uint32_t cnt, int lane, int stride,
                                          const uint2* __restrict__ rects, const float4* __restrict__ rec,
                                          int64_t N, const ViewTable& vt, uint32_t* __restrict__ tkeys,
                                          uint32_t* __restrict__ tvals) {
  const int v = view_of_item(vt, item);
  const View& V = vt.v[v];
  const uint2 rc = rects[item];
  const Cull q = make_cull(rec[3 * (size_t)item], rec[3 * (size_t)item + 1]);
  int y0 = rc.x >> 16, y1 = rc.y >> 16;
  cull_rows(q, y0, y1);
  uint32_t w = 0;
  for (int y = y0; y <= y1 && w < cnt; ++y) {
    int x0 = rc.x & 0xffff, x1 = rc.y & 0xffff;
    cull_cols(q, y, x0, x1);
    const int nx = x1 - x0 + 1;
    for (int dx = lane; dx < nx; dx += stride) {
      const uint32_t pos = w + (uint32_t)dx;
      if (pos < cnt) {
        tkeys[off + pos] = (uint32_t)(V.tile_base + y * V.tiles_x + x0 + dx);
        tvals[off + pos] = item;
      }
    }
    if (nx > 0) w += (uint32_t)nx;
  }
  for (uint32_t pos = w + lane; pos < cnt; pos += stride) {
    tkeys[off + pos] = (uint32_t)vt.n_tiles;
    tvals[off + pos] = item;
  }
}

// Warp-cooperative emission of one item's keys (all 32 lanes call it with the same
// item): lane l culls row y0 + l of a 32-row chunk, a warp scan places the rows, and the
// rows' keys are written by consecutive lanes (coalesced).  Same keys, same order and the
// same count bound as emit_item.
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
    const int nrows = min(32, y1 - yb + 1);
    for (int r = 0; r < nrows; ++r) {
      const uint32_t bnx = __shfl_sync(0xffffffffu, nx, r);
      const int bx0 = __shfl_sync(0xffffffffu, x0, r);
      const uint32_t bbase = w + __shfl_sync(0xffffffffu, excl, r);
      const uint32_t tile0 = (uint32_t)(V.tile_base + (yb + r) * V.tiles_x + bx0);
      for (uint32_t dx = lane; dx < bnx; dx += 32) {
        const uint32_t pos = bbase + dx;
        if (pos < cnt) {
          tkeys[off + pos] = tile0 + dx;
          tvals[off + pos] = item;
        }
      }
    }
    w += total;
  }
  for (uint32_t pos = w + lane; pos < cnt; pos += 32) {
    tkeys[off + pos] = (uint32_t)vt.n_tiles;
    tvals[off + pos] = item;
  }
}

constexpr uint32_t kEmitCoop = 32;

__global__ void __launch_bounds__(256) k_emit(int64_t n_vis, int64_t N, const uint32_t* __restrict__ dvals,
                                              const uint32_t* __restrict__ offsets,
                                              const uint32_t* __restrict__ touched,
                                              const uint2* __restrict__ rects, const float4* __restrict__ rec,
                                              const __grid_constant__ ViewTable vt,
                                              uint32_t* __restrict__ tkeys, uint32_t* __restrict__ tvals,
                                              const uint32_t* __restrict__ n_vis_dev) {
  if (n_vis_dev) n_vis = min(n_vis, (int64_t)*n_vis_dev);
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((k & ~int64_t(31)) >= n_vis) return;  // whole warp beyond the end
  uint32_t item = 0, off = 0, cnt = 0;
  if (k < n_vis) {
    item = dvals[k];
    off = offsets[k];
    cnt = touched[item];
  }
  if (cnt > 0 && cnt <= kEmitCoop) emit_item(item, off, cnt, 0, 1, rects, rec, N, vt, tkeys, tvals);
  uint32_t big = __ballot_sync(0xffffffffu, cnt > kEmitCoop);
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
  k_emit<<<(unsigned)div_up(n_vis, 256), 256, 0, s>>>(n_vis, N, dvals, offsets, touched, rects, rec, vt, tkeys,
                                                       tvals, n_vis_dev);
  count_launch();
  return cudaGetLastError();
}

}  // namespace mgs
