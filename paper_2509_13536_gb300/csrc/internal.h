// Host-side declarations shared by the translation units of libmemgs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace mgs {

// ---- error reporting (thread-local message behind mgs_last_error) ----
void set_error(const std::string& msg);
mgs_status cuda_status(cudaError_t e, const char* what);
#define MGS_TRY_CUDA(expr)                                 \
  do {                                                     \
    cudaError_t e_ = (expr);                               \
    if (e_ != cudaSuccess) return cuda_status(e_, #expr);  \
  } while (0)
#define MGS_CHECK_LAUNCH(what) MGS_TRY_CUDA(cudaGetLastError())

// ---- diagnostics (diag.cu) ----
void count_launch(int n = 1);
enum ProfKind { kProfPreprocess, kProfDepthSort, kProfEmit, kProfTileSort, kProfBlendFwd, kProfBlendBwd,
                kProfPreprocessBwd, kProfAdam, kProfLoss, kProfMerge, kProfKinds };
// Brackets a group of launches with CUDA events when profiling is on (no-op otherwise).
struct ProfScope {
  ProfScope(int kind, cudaStream_t s);
  ~ProfScope();
  int kind;
  cudaStream_t s;
  void* ev;
};

// ---- scan / radix sort (sort.cu) ----
constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 4096 items per block

inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// u32 words of scratch needed to sort or scan n items.
int64_t sort_scratch_words(int64_t n);

// Exclusive scan out[i] = sum_{k<i} in[gather ? gather[k] : k]; out may alias in.
// *total_dev (optional) receives the sum.  scratch: sort_scratch_words(n) words.
// n_dev (optional): the item count in device memory (<= n, which sizes the launch).
cudaError_t scan_exclusive_u32(const uint32_t* in, const uint32_t* gather, uint32_t* out,
                               int64_t n, uint32_t* scratch, uint32_t* total_dev,
                               cudaStream_t s, const uint32_t* n_dev = nullptr);

// Stable LSD radix sort of (k[0], v[0]) on bits [begin, end).  When vals_iota the input
// values are the positions 0..n-1 (v[0] is not read).  With n_keep >= 0 the first pass
// drops every pair whose key is kSortDrop, and n_keep (the number of other keys, known
// to the caller) pairs remain for the later passes and in the result.  Returns the index
// (0 or 1) of the buffer pair that holds the result.  n_dev (optional): the pair count
// in device memory (<= n, which sizes the launches); n_keep_dev (optional, with
// n_keep >= 0): the kept count in device memory, for the passes after the first.
// ranges (optional): filled with [start, end) of every key value < n_valid in the sorted
// keys ((0, 0) for absent values), by the last pass, which then writes the sorted values
// and not the keys (the result's key buffer is left as it was).
constexpr uint32_t kSortDrop = 0xffffffffu;
int radix_sort_pairs(uint32_t* k[2], uint32_t* v[2], int64_t n, int begin_bit, int end_bit,
                     bool vals_iota, uint32_t* scratch, cudaStream_t s, cudaError_t* err,
                     int64_t n_keep = -1, const uint32_t* n_dev = nullptr,
                     const uint32_t* n_keep_dev = nullptr, uint2* ranges = nullptr, uint32_t n_valid = 0);
inline int radix_passes(int begin_bit, int end_bit) {
  return end_bit > begin_bit ? (end_bit - begin_bit + 7) / 8 : 0;
}

// Work plan of the reverse projection (project.cu).  The forward projection of a render
// that a reverse pass may follow fills FwdPlanOut (all three null otherwise): it clears
// the drawn items' moment accumulators, leaves per Gaussian its drawing and gradient
// view masks (gmask, N entries) and adds the bucket sizes into bcounts (kPlanCountWords
// words, cleared by the caller; its last word, kPlanDirtyWord, is nonzero once a reverse
// pass has added into the moments since).  BwdPlan: those masks and counts, the
// scatter's cursors (the kPlanCountWords words after the counts, cleared by the launch)
// and three N-word buffers for the plan (Gaussian index, drawing views, gradient views).
constexpr int kPlanCountWords = 64;
constexpr int kPlanDirtyWord = kPlanCountWords - 1;
struct FwdPlanOut {
  float4* moments;
  uint2* gmask;
  uint32_t* bcounts;
};
struct BwdPlan {
  const uint2* gmask;
  uint32_t* counts;
  uint32_t* list;
  uint32_t* ldrawn;
  uint32_t* ltodo;
};
// Clears the n float4 moment accumulators if the word at `dirty` is nonzero.
cudaError_t launch_moments_clear(float4* moments, int64_t n, const uint32_t* dirty, cudaStream_t s);


// Patch-Grid sampling (pg.cu): workspace layout for one keyframe.
struct PgLayout {
  int PX, PY;
  int64_t n_patch, max_cand;
  size_t hdr, count, flags, cand_off, cand, keep, pos, scratch, bytes;
};
PgLayout pg_layout(int width, int height, int patch, int grid);
cudaError_t launch_patch_grid(const mgs_camera& c, int n_kp, const float* kp, const float* kd,
                              const float* depth_image, int patch, int min_kp, int grid, const PgLayout& L,
                              char* ws, float* out, int32_t* source, int64_t capacity, uint32_t* n_host,
                              cudaStream_t s);

// Counters of the calling thread's last mgs_voxel_merge (merge.cu).
struct MergeStats {
  int64_t pairs = 0, lbfgs_iterations = 0;
};
MergeStats& last_merge_stats();

// Mapping loss (loss.cu): workspace layout for n_views images of width x height.
struct LossLayout {
  int tiles_x, tiles_y, nb_ssim, nb_depth;
  size_t dmaps, part_ssim, part_depth, bytes;
};
LossLayout loss_layout(int n_views, int width, int height);
cudaError_t launch_mapping_loss(int n_views, int width, int height, const LossLayout& L, char* ws,
                                const mgs_image* rendered, const mgs_image* target, const mgs_image* grad,
                                float lambda, float w_depth, float* loss, cudaStream_t s);
size_t iso_workspace_bytes(int64_t n);
cudaError_t launch_iso_loss(const mgs_gaussians& g, float w_iso, float* grad_ls, float* loss, char* ws,
                            cudaStream_t s);

}  // namespace mgs
