// Patch-Grid sampling (Sec. II-B), sm_103a: densify the patches of a keyframe that hold
// too few keypoints with evenly spaced samples, give each sample a depth (depth image,
// else the nearest keypoint with a depth) and back-project it to the world frame.
//
//   k_pg_count    keypoints -> per-patch counts (integer atomics: exact)
//   k_pg_flags    per patch: grid^2 candidate samples if count < min_keypoints
//   scan          candidate offsets (patch order)
//   k_pg_sample   per candidate: position, depth, world point, kept flag
//   scan          output offsets of the kept candidates
//   k_pg_compact  kept candidates -> output, in candidate order
// Decisions are taken in float32 exactly as written (explicit round-to-nearest
// operations), positions computed in double and rounded once, so that the oracle can
// take the same decisions.
#include "internal.h"

namespace mgs {
namespace {

constexpr int kPgTile = 256;

__global__ void k_pg_count(int n_kp, const float* __restrict__ kp, int W, int H, int patch, int PX,
                           uint32_t* __restrict__ count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_kp) return;
  const float u = kp[2 * k], v = kp[2 * k + 1];
  if (!(u >= 0.f && u < (float)W && v >= 0.f && v < (float)H)) return;
  atomicAdd(&count[((int)v / patch) * PX + (int)u / patch], 1u);
}

__global__ void k_pg_flags(int n_patch, const uint32_t* __restrict__ count, int min_kp, uint32_t per_patch,
                           uint32_t* __restrict__ flags) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n_patch) flags[p] = count[p] < (uint32_t)min_kp ? per_patch : 0u;
}

struct PgCam {
  float R[9], t[3];
  double fx, fy, cx, cy;
  int W, H;
};

// One thread per candidate sample; the block walks the keypoints in shared-memory tiles.
__global__ void __launch_bounds__(kPgTile) k_pg_sample(int n_patch, int PX, int patch, int grid,
                                                       const uint32_t* __restrict__ flags,
                                                       const uint32_t* __restrict__ cand_off,
                                                       const uint32_t* __restrict__ n_cand_p,
                                                       const PgCam cam, int n_kp, const float* __restrict__ kp,
                                                       const float* __restrict__ kd,
                                                       const float* __restrict__ depth_image,
                                                       float* __restrict__ cand, uint32_t* __restrict__ keep) {
  __shared__ float s_u[kPgTile], s_v[kPgTile], s_d[kPgTile];
  const uint32_t n_cand = *n_cand_p;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = c < n_cand;
  // which patch and which sample: binary search of the candidate offsets
  float u = 0.f, v = 0.f;
  float depth = -1.f;
  int src = 0;
  if (live) {
    int lo = 0, hi = n_patch - 1;
    while (lo < hi) {  // last patch with offset <= c and a non-zero count
      const int mid = (lo + hi + 1) >> 1;
      if (cand_off[mid] <= c) lo = mid;
      else hi = mid - 1;
    }
    // (an empty patch shares its offset with the next one, so the last match has samples)
    const int p = lo, q = (int)(c - cand_off[p]);
    const int px = p % PX, py = p / PX, a = q / grid, b = q % grid;
    const double x0 = (double)px * patch, y0 = (double)py * patch;
    const double pw = fmin((double)patch, cam.W - x0), ph = fmin((double)patch, cam.H - y0);
    u = (float)(x0 + (b + 0.5) * pw / grid);
    v = (float)(y0 + (a + 0.5) * ph / grid);
    if (depth_image) {
      const float di = depth_image[(size_t)(int)v * cam.W + (int)u];
      if (di > 0.f) depth = di;
    }
  }
  // nearest keypoint with a depth, by the float32 squared distance (ties: smaller index)
  const bool need = live && !(depth > 0.f) && kd;
  int best = -1;
  float bd = 0.f;
  if (__syncthreads_or(need)) {
    for (int t0 = 0; t0 < n_kp; t0 += kPgTile) {
      const int k = t0 + threadIdx.x;
      s_u[threadIdx.x] = k < n_kp ? kp[2 * k] : 0.f;
      s_v[threadIdx.x] = k < n_kp ? kp[2 * k + 1] : 0.f;
      s_d[threadIdx.x] = k < n_kp ? kd[k] : 0.f;
      __syncthreads();
      if (need) {
        const int m = min(kPgTile, n_kp - t0);
        for (int j = 0; j < m; ++j) {
          if (!(s_d[j] > 0.f)) continue;
          const float du = __fsub_rn(s_u[j], u), dv = __fsub_rn(s_v[j], v);
          const float d2 = __fadd_rn(__fmul_rn(du, du), __fmul_rn(dv, dv));
          if (best < 0 || d2 < bd) { best = t0 + j; bd = d2; }
        }
      }
      __syncthreads();
    }
  }
  if (!live) return;
  if (need && best >= 0) {
    depth = kd[best];
    src = 1;
  }
  const bool ok = depth > 0.f;
  keep[c] = ok ? 1u : 0u;
  float* o = cand + 7 * (size_t)c;
  if (!ok) return;
  const float xc = (float)(((double)u - cam.cx) / cam.fx) * depth;
  const float yc = (float)(((double)v - cam.cy) / cam.fy) * depth;
  const float pc[3] = {xc - cam.t[0], yc - cam.t[1], depth - cam.t[2]};
  o[0] = u;
  o[1] = v;
  o[2] = depth;
  for (int r = 0; r < 3; ++r) o[3 + r] = cam.R[r] * pc[0] + cam.R[3 + r] * pc[1] + cam.R[6 + r] * pc[2];
  o[6] = __int_as_float(src);
}

__global__ void k_pg_compact(const uint32_t* __restrict__ n_cand_p, const uint32_t* __restrict__ keep,
                             const uint32_t* __restrict__ pos, const float* __restrict__ cand, int64_t capacity,
                             float* __restrict__ out, int32_t* __restrict__ source) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= *n_cand_p || !keep[c]) return;
  const uint32_t w = pos[c];
  if ((int64_t)w >= capacity) return;  // the host reports the overflow
  for (int k = 0; k < 6; ++k) out[6 * (size_t)w + k] = cand[7 * (size_t)c + k];
  if (source) source[w] = __float_as_int(cand[7 * (size_t)c + 6]);
}

}  // namespace

PgLayout pg_layout(int width, int height, int patch, int grid) {
  PgLayout L{};
  L.PX = (int)div_up(width, patch);
  L.PY = (int)div_up(height, patch);
  L.n_patch = (int64_t)L.PX * L.PY;
  L.max_cand = L.n_patch * grid * grid;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  const int64_t m = std::max<int64_t>(std::max(L.n_patch, L.max_cand), 1);
  L.hdr = take(64);
  L.count = take(4 * (size_t)L.n_patch);
  L.flags = take(4 * (size_t)L.n_patch);
  L.cand_off = take(4 * (size_t)L.n_patch);
  L.cand = take(sizeof(float) * 7 * (size_t)std::max<int64_t>(L.max_cand, 1));
  L.keep = take(4 * (size_t)m);
  L.pos = take(4 * (size_t)m);
  L.scratch = take(4 * (size_t)sort_scratch_words(m));
  L.bytes = off;
  return L;
}

cudaError_t launch_patch_grid(const mgs_camera& c, int n_kp, const float* kp, const float* kd,
                              const float* depth_image, int patch, int min_kp, int grid, const PgLayout& L,
                              char* ws, float* out, int32_t* source, int64_t capacity, uint32_t* n_host,
                              cudaStream_t s) {
  uint32_t* hdr = reinterpret_cast<uint32_t*>(ws + L.hdr);
  uint32_t* count = reinterpret_cast<uint32_t*>(ws + L.count);
  uint32_t* flags = reinterpret_cast<uint32_t*>(ws + L.flags);
  uint32_t* cand_off = reinterpret_cast<uint32_t*>(ws + L.cand_off);
  float* cand = reinterpret_cast<float*>(ws + L.cand);
  uint32_t* keep = reinterpret_cast<uint32_t*>(ws + L.keep);
  uint32_t* pos = reinterpret_cast<uint32_t*>(ws + L.pos);
  uint32_t* scratch = reinterpret_cast<uint32_t*>(ws + L.scratch);
  cudaError_t e = cudaMemsetAsync(hdr, 0, 64, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, 4 * (size_t)L.n_patch, s);
  if (e != cudaSuccess) return e;
  if (n_kp > 0) {
    k_pg_count<<<(unsigned)div_up(n_kp, 256), 256, 0, s>>>(n_kp, kp, c.width, c.height, patch, L.PX, count);
    count_launch();
  }
  k_pg_flags<<<(unsigned)div_up(L.n_patch, 256), 256, 0, s>>>((int)L.n_patch, count, min_kp,
                                                               (uint32_t)(grid * grid), flags);
  count_launch();
  e = scan_exclusive_u32(flags, nullptr, cand_off, L.n_patch, scratch, hdr + 0, s);
  if (e != cudaSuccess) return e;
  PgCam cam;
  for (int k = 0; k < 9; ++k) cam.R[k] = c.R[k];
  for (int k = 0; k < 3; ++k) cam.t[k] = c.t[k];
  cam.fx = c.fx; cam.fy = c.fy; cam.cx = c.cx; cam.cy = c.cy;
  cam.W = c.width; cam.H = c.height;
  const int64_t mc = std::max<int64_t>(L.max_cand, 1);
  e = cudaMemsetAsync(keep, 0, 4 * (size_t)mc, s);  // candidates beyond the count stay 0
  if (e != cudaSuccess) return e;
  const unsigned gc = (unsigned)div_up(mc, kPgTile);
  k_pg_sample<<<gc, kPgTile, 0, s>>>((int)L.n_patch, L.PX, patch, grid, flags, cand_off, hdr + 0, cam, n_kp, kp,
                                     kd, depth_image, cand, keep);
  count_launch();
  e = scan_exclusive_u32(keep, nullptr, pos, mc, scratch, hdr + 1, s);
  if (e != cudaSuccess) return e;
  k_pg_compact<<<(unsigned)div_up(mc, 256), 256, 0, s>>>(hdr + 0, keep, pos, cand, capacity, out, source);
  count_launch();
  e = cudaMemcpyAsync(n_host, hdr + 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace mgs
