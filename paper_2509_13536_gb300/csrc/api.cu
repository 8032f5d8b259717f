// C ABI of libmemgs: argument validation, workspace carving and launch sequencing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace mgs {

// kernels of the other translation units
cudaError_t launch_preprocess(const mgs_gaussians& g, const ViewTable& vt, float4* rec, uint2* rects,
                              uint32_t* touched, uint32_t* dkeys, unsigned long long* counters,
                              const FwdPlanOut& fb, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const mgs_gaussians& g, const ViewTable& vt, float4* moments,
                                  const BwdPlan& pl, const mgs_grads& gr, cudaStream_t s);
cudaError_t launch_project_one(const mgs_gaussians& g, const View& V, float* mean2d, float* conic,
                               float* rgb, float* depth, int32_t* radius, int32_t* rect, cudaStream_t s);
cudaError_t launch_emit(int64_t n_vis, int64_t N, const uint32_t* dvals, const uint32_t* offsets,
                        const uint32_t* touched, const uint2* rects, const float4* rec, const ViewTable& vt,
                        uint32_t* tkeys, uint32_t* tvals, cudaStream_t s, const uint32_t* n_vis_dev = nullptr);
cudaError_t launch_blend_fwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, const uint32_t* order, cudaStream_t s);
cudaError_t launch_blend_bwd(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                             const uint2* ranges, const uint32_t* order, float4* moments, cudaStream_t s);
cudaError_t launch_tile_order(const uint2* ranges, int n_tiles, uint32_t* counts, uint32_t* order,
                              cudaStream_t s);
cudaError_t launch_frag_stats(const ViewTable& vt, const float4* rec, const uint32_t* vals,
                              const uint2* ranges, unsigned long long* out, cudaStream_t s);
cudaError_t launch_adam(const mgs_gaussians_mut& p, const mgs_grads& g, const mgs_grads& m,
                        const mgs_grads& v, float lr, float b1, float b2, float eps, int step,
                        int zero_grads, cudaStream_t s);
cudaError_t launch_l1(const float* pred, const float* target, int64_t n, float scale, float* grad,
                      float* loss, cudaStream_t s);
struct MergeWs;
size_t merge_workspace_bytes(int64_t n, MergeWs* ws, char* base);
cudaError_t run_voxel_merge(const mgs_gaussians& in, float voxel, const mgs_merge_params& p,
                            const mgs_gaussians_mut& out, int32_t* partner, int32_t* vox, char* ws_base,
                            cudaStream_t s, int32_t** hdr_dev);

namespace {
thread_local std::string g_error;

mgs_status fail(mgs_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

// ---------------- render workspace ----------------
struct RenderLayout {
  int64_t N = 0, VN = 0, pixels = 0, tiles = 0, key_cap = 0;
  size_t hdr, rec, rects, touched, dkeys[2], dvals[2], offsets, tkeys[2], tvals[2], ranges,
      order, ocounts, tfinal, ncontrib, moments, plan, gmask, scratch, total;
};

bool cams_valid(const mgs_camera* cams, int nv, std::string* why) {
  if (!cams || nv < 1 || nv > MGS_MAX_VIEWS) {
    *why = "n_views must be in [1, MGS_MAX_VIEWS] with a camera array";
    return false;
  }
  for (int v = 0; v < nv; ++v) {
    const mgs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * MGS_TILE || c.height > 65535 * MGS_TILE ||
        !(c.fx > 0) || !(c.fy > 0) || !(c.near_z > 0) || !std::isfinite(c.cx) || !std::isfinite(c.cy)) {
      *why = "camera " + std::to_string(v) + ": need width, height, fx, fy, near_z > 0";
      return false;
    }
  }
  return true;
}

// Per-view item counts: the number of Gaussians of each view's map.
struct ViewItems {
  int64_t n[MGS_MAX_VIEWS];
};
ViewItems uniform_items(int64_t n, int nv) {
  ViewItems it{};
  for (int v = 0; v < nv && v < MGS_MAX_VIEWS; ++v) it.n[v] = n;
  return it;
}

RenderLayout render_layout(const ViewItems& items, const mgs_camera* cams, int nv, int64_t key_cap) {
  RenderLayout L;
  L.N = 0;
  L.VN = 0;
  for (int v = 0; v < nv; ++v) {
    L.N = std::max(L.N, items.n[v]);
    L.VN += items.n[v];
  }
  for (int v = 0; v < nv; ++v) {
    L.pixels += (int64_t)cams[v].width * cams[v].height;
    L.tiles += div_up(cams[v].width, MGS_TILE) * div_up(cams[v].height, MGS_TILE);
  }
  L.key_cap = key_cap;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(std::max<size_t>(bytes, 1)); return o; };
  const size_t vn = (size_t)std::max<int64_t>(L.VN, 1), kc = (size_t)std::max<int64_t>(key_cap, 1);
  L.hdr = take(256);
  L.rec = take(48 * vn);
  L.rects = take(8 * vn);
  L.touched = take(4 * vn);
  L.dkeys[0] = take(4 * vn);
  L.dkeys[1] = take(4 * vn);
  L.dvals[0] = take(4 * vn);
  L.dvals[1] = take(4 * vn);
  L.offsets = take(4 * vn);
  L.tkeys[0] = take(4 * kc);
  L.tkeys[1] = take(4 * kc);
  L.tvals[0] = take(4 * kc);
  L.tvals[1] = take(4 * kc);
  L.ranges = take(8 * (size_t)L.tiles);
  L.order = take(4 * (size_t)L.tiles);
  L.ocounts = take(512);
  L.tfinal = take(4 * (size_t)L.pixels);
  L.ncontrib = take(4 * (size_t)L.pixels);
  L.moments = take(48 * vn);
  L.plan = take(2 * kPlanCountWords * sizeof(uint32_t));
  L.gmask = take(8 * (size_t)std::max<int64_t>(L.N, 1));
  L.scratch = take(4 * (size_t)sort_scratch_words(std::max<int64_t>(L.VN, key_cap)));
  L.total = off;
  return L;
}

// Largest key capacity whose layout fits in `bytes` (-1 if not even zero keys fit).
int64_t key_capacity_for(const ViewItems& items, const mgs_camera* cams, int nv, size_t bytes) {
  if (render_layout(items, cams, nv, 0).total > bytes) return -1;
  int64_t lo = 0, hi = 1;
  while (render_layout(items, cams, nv, hi).total <= bytes && hi < (int64_t(1) << 40)) hi *= 2;
  while (hi - lo > 1) {
    int64_t mid = lo + (hi - lo) / 2;
    if (render_layout(items, cams, nv, mid).total <= bytes) lo = mid; else hi = mid;
  }
  return lo;
}

// Bits of a tile key: ids 0..tiles-1 plus the sentinel id `tiles`.
int tile_bits(int64_t tiles) {
  int b = 1;
  while ((int64_t(1) << b) < tiles + 1) ++b;
  return b;
}

template <class T>
T* at(void* base, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(base) + off); }

void fill_view(View& V, const mgs_camera& c) {
  std::memcpy(V.R, c.R, sizeof(V.R));
  std::memcpy(V.t, c.t, sizeof(V.t));
  V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy; V.near_z = c.near_z;
  // camera centre -R^T t in double, kept as a pair of floats: the viewing direction of
  // a Gaussian (the SH argument) is then as accurate as its mean allows
  for (int k = 0; k < 3; ++k) {
    const double Cd = -((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]);
    V.C[k] = (float)Cd;
    V.C_lo[k] = (float)(Cd - (double)V.C[k]);
  }
  V.limx = kFovClamp * (0.5f * (float)c.width / c.fx);
  V.limy = kFovClamp * (0.5f * (float)c.height / c.fy);
  V.width = c.width; V.height = c.height;
  V.tiles_x = (int)div_up(c.width, MGS_TILE);
  V.tiles_y = (int)div_up(c.height, MGS_TILE);
}

ViewTable make_table(const mgs_camera* cams, int nv, const RenderLayout& L, void* ws, const ViewItems& items) {
  ViewTable vt{};
  vt.n_views = nv;
  int tb = 0;
  int64_t pb = 0, ib = 0;
  for (int v = 0; v < nv; ++v) {
    View& V = vt.v[v];
    fill_view(V, cams[v]);
    V.tile_base = tb;
    V.item_base = ib;
    V.n_items = items.n[v];
    ib += items.n[v];
    tb += V.tiles_x * V.tiles_y;
    V.T_final = at<float>(ws, L.tfinal) + pb;
    V.n_contrib = at<uint32_t>(ws, L.ncontrib) + pb;
    pb += (int64_t)V.width * V.height;
  }
  vt.n_tiles = tb;
  return vt;
}

std::string check_gaussians(const mgs_gaussians* g, bool need_birth) {
  if (!g) return "gaussians pointer is NULL";
  if (g->n < 0) return "n < 0";
  if (g->sh_degree < 0 || g->sh_degree > 3) return "sh_degree must be 0..3";
  if (g->attr_dtype < MGS_F32 || g->attr_dtype > MGS_BF16) return "attr_dtype must be MGS_F32, MGS_F16 or MGS_BF16";
  if (g->geom_dtype < MGS_F32 || g->geom_dtype > MGS_BF16) return "geom_dtype must be MGS_F32, MGS_F16 or MGS_BF16";
  if (g->quat_dtype < MGS_F32 || g->quat_dtype > MGS_BF16) return "quat_dtype must be MGS_F32, MGS_F16 or MGS_BF16";
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->sh))
    return "parameter pointer is NULL";
  if (need_birth && g->n > 0 && !g->birth) return "birth is NULL";
  return "";
}

}  // namespace

void set_error(const std::string& msg) { g_error = msg; }
mgs_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return MGS_ERR_CUDA;
}

}  // namespace mgs

using namespace mgs;

extern "C" {

const char* mgs_last_error(void) { return g_error.c_str(); }
const char* mgs_version(void) { return "memgs 0.1 sm_103a"; }

size_t mgs_render_workspace_size(int64_t n, const mgs_camera* cams, int32_t n_views,
                                 int64_t key_capacity) {
  std::string why;
  if (n < 0 || key_capacity < 0 || !cams_valid(cams, n_views, &why)) return 0;
  return render_layout(uniform_items(n, n_views), cams, n_views, key_capacity).total;
}

// Render-plan of the asynchronous form: from the projection's counters, the number of
// drawn items and of keys the later launches process (both 0 when the keys exceed the
// workspace's capacity: then nothing is emitted, sorted or blended beyond empty
// tiles), and the status {keys, overflow} for the caller.
__global__ void k_render_plan(const unsigned long long* counters, unsigned long long cap, uint32_t* plan,
                              long long* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long nk = counters[0], nv = counters[1];
  const bool over = nk > cap || nk >= 0xffffffffull;
  plan[0] = over ? 0u : (uint32_t)nv;
  plan[1] = over ? 0u : (uint32_t)nk;
  status[0] = (long long)nk;
  status[1] = over ? 1 : 0;
}

static mgs_status render_impl(const mgs_gaussians* maps, int n_maps, const int32_t* map_of_view,
                              const mgs_camera* cams, int32_t n_views, const mgs_image* out, void* workspace,
                              size_t workspace_bytes, int64_t* n_keys_host, cudaStream_t s,
                              bool async = false, int64_t* status_pinned = nullptr) {
  std::string why;
  if (!cams_valid(cams, n_views, &why)) return fail(MGS_ERR_INVALID, why);
  if (!out || !workspace) return fail(MGS_ERR_INVALID, "out or workspace is NULL");
  ViewItems items{};
  int64_t total = 0;
  for (int v = 0; v < n_views; ++v) {
    if (!out[v].rgb || !out[v].depth || !out[v].alpha) return fail(MGS_ERR_INVALID, "image plane is NULL");
    const int m = map_of_view ? map_of_view[v] : 0;
    if (m < 0 || m >= n_maps) return fail(MGS_ERR_INVALID, "map_of_view out of range");
    items.n[v] = maps[m].n;
    total += maps[m].n;
  }
  if (total >= (int64_t)UINT32_MAX) return fail(MGS_ERR_UNSUPPORTED, "the views' maps hold 2^32 or more Gaussians in all");
  int64_t cap = key_capacity_for(items, cams, n_views, workspace_bytes);
  if (cap < 0) {
    if (n_keys_host) *n_keys_host = 0;
    return fail(MGS_ERR_WORKSPACE, "workspace smaller than the zero-key layout");
  }
  RenderLayout L = render_layout(items, cams, n_views, cap);
  ViewTable vt = make_table(cams, n_views, L, workspace, items);
  for (int v = 0; v < n_views; ++v) {
    vt.v[v].rgb = out[v].rgb;
    vt.v[v].depth = out[v].depth;
    vt.v[v].alpha = out[v].alpha;
  }
  auto* counters = at<unsigned long long>(workspace, L.hdr);
  auto* rec = at<float4>(workspace, L.rec);
  auto* rects = at<uint2>(workspace, L.rects);
  auto* touched = at<uint32_t>(workspace, L.touched);
  uint32_t* dk[2] = {at<uint32_t>(workspace, L.dkeys[0]), at<uint32_t>(workspace, L.dkeys[1])};
  uint32_t* dv[2] = {at<uint32_t>(workspace, L.dvals[0]), at<uint32_t>(workspace, L.dvals[1])};
  uint32_t* tk[2] = {at<uint32_t>(workspace, L.tkeys[0]), at<uint32_t>(workspace, L.tkeys[1])};
  uint32_t* tv[2] = {at<uint32_t>(workspace, L.tvals[0]), at<uint32_t>(workspace, L.tvals[1])};
  auto* offsets = at<uint32_t>(workspace, L.offsets);
  auto* ranges = at<uint2>(workspace, L.ranges);
  auto* scratch = at<uint32_t>(workspace, L.scratch);

  // a render of one map may be followed by the reverse pass: its projection clears the
  // drawn items' moments and leaves the masks and bucket counts of the reverse
  // projection's work plan
  FwdPlanOut fb{nullptr, nullptr, nullptr};
  if (!map_of_view)
    fb = FwdPlanOut{at<float4>(workspace, L.moments), at<uint2>(workspace, L.gmask),
                    at<uint32_t>(workspace, L.plan)};
  {
    ProfScope ps(kProfPreprocess, s);
    MGS_TRY_CUDA(cudaMemsetAsync(counters, 0, 256, s));
    if (fb.bcounts) MGS_TRY_CUDA(cudaMemsetAsync(fb.bcounts, 0, kPlanCountWords * sizeof(uint32_t), s));
    // one projection launch per run of consecutive views that share a map: each thread
    // projects one Gaussian into every view of the run (its items are consecutive)
    for (int v0 = 0; v0 < n_views;) {
      const int m = map_of_view ? map_of_view[v0] : 0;
      int v1 = v0 + 1;
      while (v1 < n_views && (map_of_view ? map_of_view[v1] : 0) == m) ++v1;
      ViewTable sub{};
      sub.n_views = v1 - v0;
      sub.n_tiles = vt.n_tiles;
      for (int v = v0; v < v1; ++v) sub.v[v - v0] = vt.v[v];
      const int64_t ib = vt.v[v0].item_base;
      MGS_TRY_CUDA(launch_preprocess(maps[m], sub, rec + 3 * ib, rects + ib, touched + ib, dk[0] + ib, counters,
                                     fb, s));
      v0 = v1;
    }
  }
  // Counts for the launches that follow: read on the host (one synchronisation), or
  // kept on the device (asynchronous form: launches sized for the workspace's capacity
  // read them from the plan).
  int64_t n_keys = cap, n_vis = L.VN;
  const uint32_t* vis_dev = nullptr;
  const uint32_t* keys_dev = nullptr;
  auto* plan = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(counters) + 128);
  auto* status = reinterpret_cast<long long*>(reinterpret_cast<char*>(counters) + 144);
  if (async) {
    k_render_plan<<<1, 32, 0, s>>>(counters, (unsigned long long)cap, plan, status);
    count_launch();
    MGS_TRY_CUDA(cudaGetLastError());
    vis_dev = plan;
    keys_dev = plan + 1;
  } else {
    unsigned long long cnt[2] = {0, 0};
    MGS_TRY_CUDA(cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    MGS_TRY_CUDA(cudaStreamSynchronize(s));
    n_keys = (int64_t)cnt[0];
    n_vis = (int64_t)cnt[1];
    if (n_keys_host) *n_keys_host = n_keys;
    if (n_keys >= (int64_t)UINT32_MAX) return fail(MGS_ERR_UNSUPPORTED, "more than 2^32-1 (Gaussian, tile) pairs");
    if (n_keys > cap)
      return fail(MGS_ERR_WORKSPACE, "workspace holds " + std::to_string(cap) + " keys, render needs " +
                                         std::to_string(n_keys));
  }
  cudaError_t e = cudaSuccess;
  int dcur = 0;
  if (L.VN > 0) {
    // front-to-back order of the drawn (view, Gaussian) items: float32 depth bits, then item
    // index; undrawn items (key kSortDrop) leave in the first pass
    ProfScope ps(kProfDepthSort, s);
    dcur = radix_sort_pairs(dk, dv, L.VN, 0, 32, true, scratch, s, &e, n_vis, nullptr, vis_dev);
    if (e != cudaSuccess) return cuda_status(e, "depth sort");
    MGS_TRY_CUDA(scan_exclusive_u32(touched, dv[dcur], offsets, n_vis, scratch, nullptr, s, vis_dev));
  }
  {
    ProfScope ps(kProfEmit, s);
    MGS_TRY_CUDA(launch_emit(n_vis, L.N, dv[dcur], offsets, touched, rects, rec, vt, tk[0], tv[0], s, vis_dev));
  }
  int tcur = 0;
  {
    ProfScope ps(kProfTileSort, s);
    // the last pass also writes each tile's [start, end) (sentinel keys, id n_tiles, left out)
    tcur = radix_sort_pairs(tk, tv, n_keys, 0, tile_bits(vt.n_tiles), false, scratch, s, &e, -1, keys_dev,
                            nullptr, ranges, (uint32_t)vt.n_tiles);
    if (e != cudaSuccess) return cuda_status(e, "tile sort");
    // the blend launches (forward, and the reverse pass on this workspace) take the tiles
    // longest list first
    MGS_TRY_CUDA(launch_tile_order(ranges, (int)vt.n_tiles, at<uint32_t>(workspace, L.ocounts),
                                   at<uint32_t>(workspace, L.order), s));
  }
  if (async && status_pinned)
    MGS_TRY_CUDA(cudaMemcpyAsync(status_pinned, status, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  {
    ProfScope ps(kProfBlendFwd, s);
    MGS_TRY_CUDA(launch_blend_fwd(vt, rec, tv[tcur], ranges, at<uint32_t>(workspace, L.order), s));
  }
  return MGS_OK;
}

mgs_status mgs_render(const mgs_gaussians* g, const mgs_camera* cams, int32_t n_views,
                      const mgs_image* out, void* workspace, size_t workspace_bytes,
                      int64_t* n_keys_host, void* stream) {
  set_error("");
  std::string why = check_gaussians(g, false);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  return render_impl(g, 1, nullptr, cams, n_views, out, workspace, workspace_bytes, n_keys_host,
                     (cudaStream_t)stream);
}

mgs_status mgs_render_async(const mgs_gaussians* g, const mgs_camera* cams, int32_t n_views,
                            const mgs_image* out, void* workspace, size_t workspace_bytes, int64_t* status_pinned,
                            void* stream) {
  set_error("");
  std::string why = check_gaussians(g, false);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  return render_impl(g, 1, nullptr, cams, n_views, out, workspace, workspace_bytes, nullptr, (cudaStream_t)stream,
                     true, status_pinned);
}

size_t mgs_render_multi_workspace_size(const mgs_gaussians* maps, int32_t n_maps, const int32_t* map_of_view,
                                       const mgs_camera* cams, int32_t n_views, int64_t key_capacity) {
  std::string why;
  if (!maps || !map_of_view || n_maps < 1 || key_capacity < 0 || !cams_valid(cams, n_views, &why)) return 0;
  ViewItems items{};
  for (int v = 0; v < n_views; ++v) {
    if (map_of_view[v] < 0 || map_of_view[v] >= n_maps || maps[map_of_view[v]].n < 0) return 0;
    items.n[v] = maps[map_of_view[v]].n;
  }
  return render_layout(items, cams, n_views, key_capacity).total;
}

mgs_status mgs_render_multi(const mgs_gaussians* maps, int32_t n_maps, const int32_t* map_of_view,
                            const mgs_camera* cams, int32_t n_views, const mgs_image* out, void* workspace,
                            size_t workspace_bytes, int64_t* n_keys_host, void* stream) {
  set_error("");
  if (!maps || n_maps < 1 || !map_of_view) return fail(MGS_ERR_INVALID, "need maps, n_maps >= 1 and map_of_view");
  for (int m = 0; m < n_maps; ++m) {
    std::string why = check_gaussians(&maps[m], false);
    if (!why.empty()) return fail(MGS_ERR_INVALID, "map " + std::to_string(m) + ": " + why);
  }
  return render_impl(maps, n_maps, map_of_view, cams, n_views, out, workspace, workspace_bytes, n_keys_host,
                     (cudaStream_t)stream);
}

mgs_status mgs_render_backward(const mgs_gaussians* g, const mgs_camera* cams, int32_t n_views,
                               const mgs_image* dL, void* workspace, size_t workspace_bytes,
                               const mgs_grads* grads, void* stream) {
  set_error("");
  cudaStream_t s = (cudaStream_t)stream;
  std::string why = check_gaussians(g, false);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  if (!cams_valid(cams, n_views, &why)) return fail(MGS_ERR_INVALID, why);
  if (!dL || !workspace || !grads) return fail(MGS_ERR_INVALID, "dL, workspace or grads is NULL");
  if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logit || !grads->sh))
    return fail(MGS_ERR_INVALID, "gradient pointer is NULL");
  const ViewItems items = uniform_items(g->n, n_views);
  int64_t cap = key_capacity_for(items, cams, n_views, workspace_bytes);
  if (cap < 0) return fail(MGS_ERR_WORKSPACE, "workspace smaller than the zero-key layout");
  RenderLayout L = render_layout(items, cams, n_views, cap);
  ViewTable vt = make_table(cams, n_views, L, workspace, items);
  for (int v = 0; v < n_views; ++v) {
    vt.v[v].g_rgb = dL[v].rgb;
    vt.v[v].g_depth = dL[v].depth;
    vt.v[v].g_alpha = dL[v].alpha;
  }
  uint32_t* tv[2] = {at<uint32_t>(workspace, L.tvals[0]), at<uint32_t>(workspace, L.tvals[1])};
  int tcur = radix_passes(0, tile_bits(vt.n_tiles)) & 1;
  auto* moments = at<float4>(workspace, L.moments);
  {
    ProfScope ps(kProfBlendBwd, s);
    // the forward cleared the drawn items' moments; a second reverse pass of the same
    // render clears the whole buffer first
    MGS_TRY_CUDA(launch_moments_clear(moments, 3 * L.VN, at<uint32_t>(workspace, L.plan) + kPlanDirtyWord, s));
    MGS_TRY_CUDA(launch_blend_bwd(vt, at<float4>(workspace, L.rec), tv[tcur], at<uint2>(workspace, L.ranges),
                                  at<uint32_t>(workspace, L.order),
                                  moments, s));
  }
  {
    ProfScope ps(kProfPreprocessBwd, s);
    // the plan lists take the depth-sort buffers, free once the forward has emitted its
    // keys (each holds 4 x VN >= 4 x N bytes)
    const BwdPlan pl{at<uint2>(workspace, L.gmask), at<uint32_t>(workspace, L.plan),
                     at<uint32_t>(workspace, L.dkeys[0]), at<uint32_t>(workspace, L.dkeys[1]),
                     at<uint32_t>(workspace, L.dvals[0])};
    MGS_TRY_CUDA(launch_preprocess_bwd(*g, vt, moments, pl, *grads, s));
  }
  return MGS_OK;
}

mgs_status mgs_render_stats(const mgs_gaussians* g, const mgs_camera* cams, int32_t n_views, void* workspace,
                            size_t workspace_bytes, uint64_t* stats, void* stream) {
  set_error("");
  cudaStream_t s = (cudaStream_t)stream;
  std::string why = check_gaussians(g, false);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  if (!cams_valid(cams, n_views, &why)) return fail(MGS_ERR_INVALID, why);
  if (!workspace || !stats) return fail(MGS_ERR_INVALID, "workspace or stats is NULL");
  const ViewItems items = uniform_items(g->n, n_views);
  int64_t cap = key_capacity_for(items, cams, n_views, workspace_bytes);
  if (cap < 0) return fail(MGS_ERR_WORKSPACE, "workspace smaller than the zero-key layout");
  RenderLayout L = render_layout(items, cams, n_views, cap);
  ViewTable vt = make_table(cams, n_views, L, workspace, items);
  uint32_t* tv[2] = {at<uint32_t>(workspace, L.tvals[0]), at<uint32_t>(workspace, L.tvals[1])};
  int tcur = radix_passes(0, tile_bits(vt.n_tiles)) & 1;
  auto* hdr = at<unsigned long long>(workspace, L.hdr);
  MGS_TRY_CUDA(cudaMemsetAsync(hdr + 8, 0, 8 * 8, s));
  MGS_TRY_CUDA(launch_frag_stats(vt, at<float4>(workspace, L.rec), tv[tcur], at<uint2>(workspace, L.ranges),
                                 hdr + 8, s));
  unsigned long long h[16];
  MGS_TRY_CUDA(cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  MGS_TRY_CUDA(cudaStreamSynchronize(s));
  stats[0] = h[8];
  stats[1] = h[9];
  stats[2] = h[10];
  stats[3] = h[0];
  stats[4] = h[11];
  stats[5] = h[12];
  stats[6] = h[13];
  stats[7] = h[14];
  stats[8] = h[1];
  return MGS_OK;
}

mgs_status mgs_project(const mgs_gaussians* g, const mgs_camera* cam, float* mean2d, float* conic,
                       float* rgb, float* depth, int32_t* radius, int32_t* rect, void* stream) {
  set_error("");
  std::string why = check_gaussians(g, false);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  if (!cams_valid(cam, 1, &why)) return fail(MGS_ERR_INVALID, why);
  View V{};
  fill_view(V, *cam);
  MGS_TRY_CUDA(launch_project_one(*g, V, mean2d, conic, rgb, depth, radius, rect, (cudaStream_t)stream));
  return MGS_OK;
}

size_t mgs_voxel_merge_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return merge_workspace_bytes(n, nullptr, nullptr);
}

static mgs_status merge_args(const mgs_gaussians* in, float voxel_size, const mgs_merge_params* p,
                             const mgs_gaussians_mut* out, void* workspace, size_t workspace_bytes) {
  std::string why = check_gaussians(in, true);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  if (!p || !out) return fail(MGS_ERR_INVALID, "params or out is NULL");
  if (!(voxel_size > 0) || !std::isfinite(voxel_size)) return fail(MGS_ERR_INVALID, "voxel_size must be > 0");
  if (!(p->chi2 > 0)) return fail(MGS_ERR_INVALID, "chi2 must be > 0");
  if (p->solver != 0 && p->solver != 1) return fail(MGS_ERR_INVALID, "solver must be 0 (closed form) or 1 (L-BFGS)");
  if (out->n < in->n || out->sh_degree != in->sh_degree || out->attr_dtype != in->attr_dtype ||
      out->geom_dtype != in->geom_dtype || out->quat_dtype != in->quat_dtype)
    return fail(MGS_ERR_INVALID, "out must have capacity >= n and the same sh_degree and storage types");
  if (in->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logit || !out->sh))
    return fail(MGS_ERR_INVALID, "output pointer is NULL");
  if (in->n >= (int64_t)INT32_MAX) return fail(MGS_ERR_UNSUPPORTED, "n must be < 2^31");
  if (!workspace || workspace_bytes < merge_workspace_bytes(in->n, nullptr, nullptr))
    return fail(MGS_ERR_WORKSPACE, "merge workspace too small");
  return MGS_OK;
}

mgs_status mgs_voxel_merge(const mgs_gaussians* in, float voxel_size, const mgs_merge_params* p,
                           const mgs_gaussians_mut* out, int32_t* partner, int32_t* voxel,
                           int64_t* n_out_host, void* workspace, size_t workspace_bytes, void* stream) {
  set_error("");
  if (!n_out_host) return fail(MGS_ERR_INVALID, "n_out_host is NULL");
  mgs_status st = merge_args(in, voxel_size, p, out, workspace, workspace_bytes);
  if (st != MGS_OK) return st;
  if (in->n == 0) {
    *n_out_host = 0;
    return MGS_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* hdr = nullptr;
  {
    ProfScope ps(kProfMerge, s);
    cudaError_t e = run_voxel_merge(*in, voxel_size, *p, *out, partner, voxel, static_cast<char*>(workspace), s, &hdr);
    if (e != cudaSuccess) return cuda_status(e, "voxel merge");
  }
  int32_t h[16];
  MGS_TRY_CUDA(cudaMemcpyAsync(h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
  MGS_TRY_CUDA(cudaStreamSynchronize(s));
  *n_out_host = (int64_t)(uint32_t)h[10];
  unsigned long long it = 0;
  std::memcpy(&it, h + 12, sizeof(it));
  last_merge_stats().pairs = (int64_t)(uint32_t)h[11];
  last_merge_stats().lbfgs_iterations = (int64_t)it;
  if (h[7] & 1) return fail(MGS_ERR_UNSUPPORTED, "voxel coordinate outside +-2^20 (nothing merged)");
  if (h[7] & 4) return fail(MGS_ERR_UNSUPPORTED, "occupied voxel box needs more than 31 key bits (nothing merged)");
  if (h[7] & 8) return fail(MGS_ERR_UNSUPPORTED, "voxel grouping table full");
  return MGS_OK;
}

mgs_status mgs_voxel_merge_async(const mgs_gaussians* in, float voxel_size, const mgs_merge_params* p,
                                 const mgs_gaussians_mut* out, int32_t* partner, int32_t* voxel,
                                 int32_t* status_pinned, void* workspace, size_t workspace_bytes, void* stream) {
  set_error("");
  mgs_status st = merge_args(in, voxel_size, p, out, workspace, workspace_bytes);
  if (st != MGS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (in->n == 0) {
    if (status_pinned) status_pinned[0] = status_pinned[1] = 0;
    return MGS_OK;
  }
  int32_t* hdr = nullptr;
  {
    ProfScope ps(kProfMerge, s);
    cudaError_t e = run_voxel_merge(*in, voxel_size, *p, *out, partner, voxel, static_cast<char*>(workspace), s, &hdr);
    if (e != cudaSuccess) return cuda_status(e, "voxel merge");
  }
  if (status_pinned) {
    MGS_TRY_CUDA(cudaMemcpyAsync(status_pinned, hdr + 10, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MGS_TRY_CUDA(cudaMemcpyAsync(status_pinned + 1, hdr + 7, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  return MGS_OK;
}

mgs_status mgs_adam_step(const mgs_gaussians_mut* params, const mgs_grads* grads, const mgs_grads* m,
                         const mgs_grads* v, float lr, float beta1, float beta2, float eps,
                         int32_t step, int32_t zero_grads, void* stream) {
  set_error("");
  if (!params || !grads || !m || !v) return fail(MGS_ERR_INVALID, "NULL argument");
  if (params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3 || step < 1)
    return fail(MGS_ERR_INVALID, "need n >= 0, sh_degree 0..3, step >= 1");
  if (params->attr_dtype < MGS_F32 || params->attr_dtype > MGS_BF16 || params->geom_dtype < MGS_F32 ||
      params->geom_dtype > MGS_BF16 || params->quat_dtype < MGS_F32 || params->quat_dtype > MGS_BF16)
    return fail(MGS_ERR_INVALID, "bad attr_dtype / geom_dtype / quat_dtype");
  if (!(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(MGS_ERR_INVALID, "need 0 <= beta < 1 and eps > 0");
  {
    // the kernel moves f32 arrays in 16-byte vectors: a misaligned view is an error here,
    // not a fault on the device
    auto mis = [](const void* q) { return q && (reinterpret_cast<uintptr_t>(q) & 15) != 0; };
    const void* f32s[] = {grads->means, grads->log_scales, grads->quats, grads->opacity_logit, grads->sh,
                          m->means, m->log_scales, m->quats, m->opacity_logit, m->sh,
                          v->means, v->log_scales, v->quats, v->opacity_logit, v->sh, params->means,
                          params->geom_dtype == MGS_F32 ? params->log_scales : nullptr,
                          params->quat_dtype == MGS_F32 ? params->quats : nullptr,
                          params->attr_dtype == MGS_F32 ? params->opacity_logit : nullptr,
                          params->attr_dtype == MGS_F32 ? params->sh : nullptr};
    for (const void* q : f32s)
      if (mis(q)) return fail(MGS_ERR_INVALID, "f32 parameter, gradient and moment arrays must be 16-byte aligned");
  }
  ProfScope ps(kProfAdam, (cudaStream_t)stream);
  MGS_TRY_CUDA(launch_adam(*params, *grads, *m, *v, lr, beta1, beta2, eps, step, zero_grads ? 1 : 0,
                           (cudaStream_t)stream));
  return MGS_OK;
}

mgs_status mgs_l1_loss_grad(const float* pred, const float* target, int64_t n, float scale,
                            float* grad, float* loss, void* stream) {
  set_error("");
  if (n < 0 || (n > 0 && (!pred || !target || !grad))) return fail(MGS_ERR_INVALID, "bad arguments");
  ProfScope ps(kProfLoss, (cudaStream_t)stream);
  MGS_TRY_CUDA(launch_l1(pred, target, n, scale, grad, loss, (cudaStream_t)stream));
  return MGS_OK;
}

static std::string pg_check(int32_t width, int32_t height, const mgs_pg_params* p) {
  if (!p) return "params is NULL";
  if (width <= 0 || height <= 0) return "width and height must be positive";
  if (p->patch <= 0 || p->grid <= 0 || p->grid > p->patch) return "need 0 < grid <= patch";
  if (p->min_keypoints < 0) return "min_keypoints must be >= 0";
  return "";
}

size_t mgs_patch_grid_workspace_size(int32_t width, int32_t height, const mgs_pg_params* p) {
  if (!pg_check(width, height, p).empty()) return 0;
  return pg_layout(width, height, p->patch, p->grid).bytes;
}

int64_t mgs_patch_grid_capacity(int32_t width, int32_t height, const mgs_pg_params* p) {
  if (!pg_check(width, height, p).empty()) return 0;
  return pg_layout(width, height, p->patch, p->grid).max_cand;
}

mgs_status mgs_patch_grid_sample(const mgs_camera* cam, int32_t n_keypoints, const float* kp_uv,
                                 const float* kp_depth, const float* depth_image, const mgs_pg_params* p,
                                 float* out, int32_t* source, int64_t capacity, int64_t* n_out_host,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  set_error("");
  if (!cam || !n_out_host) return fail(MGS_ERR_INVALID, "camera or n_out_host is NULL");
  std::string why = pg_check(cam->width, cam->height, p);
  if (!why.empty()) return fail(MGS_ERR_INVALID, why);
  if (n_keypoints < 0 || (n_keypoints > 0 && !kp_uv)) return fail(MGS_ERR_INVALID, "bad keypoints");
  if (capacity < 0 || (capacity > 0 && !out)) return fail(MGS_ERR_INVALID, "bad output");
  if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(MGS_ERR_INVALID, "focal lengths must be > 0");
  const PgLayout L = pg_layout(cam->width, cam->height, p->patch, p->grid);
  if (L.max_cand >= (int64_t)UINT32_MAX) return fail(MGS_ERR_UNSUPPORTED, "too many patches");
  if (!workspace || workspace_bytes < L.bytes) return fail(MGS_ERR_WORKSPACE, "patch-grid workspace too small");
  uint32_t n = 0;
  MGS_TRY_CUDA(launch_patch_grid(*cam, n_keypoints, kp_uv, kp_depth, depth_image, p->patch, p->min_keypoints,
                                 p->grid, L, (char*)workspace, out, source, capacity, &n, (cudaStream_t)stream));
  *n_out_host = (int64_t)n;
  if ((int64_t)n > capacity) return fail(MGS_ERR_WORKSPACE, "output capacity too small");
  return MGS_OK;
}

void mgs_merge_stats(int64_t out[2]) {
  if (!out) return;
  out[0] = last_merge_stats().pairs;
  out[1] = last_merge_stats().lbfgs_iterations;
}

size_t mgs_mapping_loss_workspace_size(int32_t n_views, int32_t width, int32_t height) {
  if (n_views < 1 || n_views > MGS_MAX_VIEWS || width <= 0 || height <= 0) return 0;
  return loss_layout(n_views, width, height).bytes;
}

mgs_status mgs_mapping_loss(int32_t n_views, int32_t width, int32_t height, const mgs_image* rendered,
                            const mgs_image* target, const mgs_image* grad, float lambda_ssim,
                            float w_depth, float* loss, void* workspace, size_t workspace_bytes,
                            void* stream) {
  set_error("");
  if (n_views < 1 || n_views > MGS_MAX_VIEWS) return fail(MGS_ERR_INVALID, "n_views must be in [1, 32]");
  if (width <= 0 || height <= 0) return fail(MGS_ERR_INVALID, "width and height must be positive");
  if (!rendered || !target || !grad || !loss) return fail(MGS_ERR_INVALID, "NULL argument");
  if (!(lambda_ssim >= 0.f && lambda_ssim <= 1.f)) return fail(MGS_ERR_INVALID, "lambda_ssim must be in [0, 1]");
  for (int v = 0; v < n_views; ++v) {
    if (!rendered[v].rgb || !target[v].rgb || !grad[v].rgb) return fail(MGS_ERR_INVALID, "NULL rgb plane");
    if (target[v].depth && !rendered[v].depth) return fail(MGS_ERR_INVALID, "target depth without rendered depth");
  }
  const LossLayout L = loss_layout(n_views, width, height);
  if (!workspace || workspace_bytes < L.bytes) return fail(MGS_ERR_WORKSPACE, "mapping-loss workspace too small");
  ProfScope ps(kProfLoss, (cudaStream_t)stream);
  MGS_TRY_CUDA(launch_mapping_loss(n_views, width, height, L, (char*)workspace, rendered, target, grad,
                                   lambda_ssim, w_depth, loss, (cudaStream_t)stream));
  return MGS_OK;
}

size_t mgs_iso_loss_workspace_size(int64_t n) { return n < 0 ? 0 : iso_workspace_bytes(n); }

mgs_status mgs_iso_loss(const mgs_gaussians* g, float w_iso, const mgs_grads* grads, float* loss,
                        void* workspace, size_t workspace_bytes, void* stream) {
  set_error("");
  if (!g || !loss || g->n < 0) return fail(MGS_ERR_INVALID, "bad arguments");
  if (g->n > 0 && !g->log_scales) return fail(MGS_ERR_INVALID, "NULL log_scales");
  if (g->geom_dtype < MGS_F32 || g->geom_dtype > MGS_BF16) return fail(MGS_ERR_INVALID, "bad geom_dtype");
  if (!workspace || workspace_bytes < iso_workspace_bytes(g->n)) return fail(MGS_ERR_WORKSPACE, "iso workspace too small");
  ProfScope ps(kProfLoss, (cudaStream_t)stream);
  MGS_TRY_CUDA(launch_iso_loss(*g, w_iso, grads ? grads->log_scales : nullptr, loss, (char*)workspace,
                               (cudaStream_t)stream));
  return MGS_OK;
}

size_t mgs_sort_workspace_size(int64_t n) {
  if (n < 0) return 0;
  size_t m = (size_t)std::max<int64_t>(n, 1);
  return 3 * align_up(4 * m) + align_up(4 * (size_t)sort_scratch_words(n));
}

mgs_status mgs_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* vals_out, int64_t n,
                          int32_t begin_bit, int32_t end_bit, void* workspace, size_t workspace_bytes,
                          void* stream) {
  set_error("");
  cudaStream_t s = (cudaStream_t)stream;
  if (n < 0 || begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit)
    return fail(MGS_ERR_INVALID, "need n >= 0 and 0 <= begin_bit < end_bit <= 32");
  if (n >= (int64_t)UINT32_MAX) return fail(MGS_ERR_UNSUPPORTED, "n must be < 2^32");
  if (n > 0 && (!keys || (!vals && !vals_out))) return fail(MGS_ERR_INVALID, "NULL keys or values");
  if (!workspace || workspace_bytes < mgs_sort_workspace_size(n)) return fail(MGS_ERR_WORKSPACE, "sort workspace too small");
  if (n == 0) return MGS_OK;
  size_t m = align_up(4 * (size_t)n);
  char* w = static_cast<char*>(workspace);
  uint32_t* kalt = reinterpret_cast<uint32_t*>(w);
  uint32_t* valt = reinterpret_cast<uint32_t*>(w + m);
  uint32_t* vtmp = reinterpret_cast<uint32_t*>(w + 2 * m);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(w + 3 * m);
  bool iota = vals == nullptr;
  uint32_t* vdst = iota ? vals_out : vals;
  uint32_t* K[2] = {keys, kalt};
  uint32_t* V[2] = {iota ? vtmp : vals, valt};
  cudaError_t e;
  int cur = radix_sort_pairs(K, V, n, begin_bit, end_bit, iota, scratch, s, &e);
  if (e != cudaSuccess) return cuda_status(e, "radix sort");
  if (cur == 1) MGS_TRY_CUDA(cudaMemcpyAsync(keys, kalt, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  if (V[cur] != vdst) MGS_TRY_CUDA(cudaMemcpyAsync(vdst, V[cur], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  return MGS_OK;
}

}  // extern "C"
