// Launch counting and optional CUDA-event timing of the library's kernel groups.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace mgs {
namespace {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_mu;

const char* kNames[kProfKinds] = {"preprocess", "depth_sort", "emit", "tile_sort", "blend_fwd",
                                  "blend_bwd", "preprocess_bwd", "adam", "l1_loss", "voxel_merge"};

struct Pending {
  int kind;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[kProfKinds];
int64_t g_count[kProfKinds];

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void drain_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.kind] += ms;
      g_count[p.kind] += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

}  // namespace

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

ProfScope::ProfScope(int k, cudaStream_t st) : kind(k), s(st), ev(nullptr) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_pending.size() > 4096) drain_locked();
  cudaEvent_t a = get_event();
  cudaEventRecord(a, s);
  ev = a;
}

ProfScope::~ProfScope() {
  if (!ev) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  cudaEventRecord(b, s);
  g_pending.push_back(Pending{kind, (cudaEvent_t)ev, b});
}

}  // namespace mgs

extern "C" {

uint64_t mgs_launch_count(void) { return mgs::g_launches.load(); }

void mgs_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(mgs::g_mu);
  mgs::drain_locked();
  if (on) {
    std::memset(mgs::g_ms, 0, sizeof(mgs::g_ms));
    std::memset(mgs::g_count, 0, sizeof(mgs::g_count));
  }
  mgs::g_prof_on.store(on ? 1 : 0);
}

int32_t mgs_profile_read(int32_t max_kinds, char* names, double* ms_total, int64_t* launches) {
  std::lock_guard<std::mutex> lk(mgs::g_mu);
  mgs::drain_locked();
  int n = std::min<int>(max_kinds, mgs::kProfKinds);
  for (int k = 0; k < n; ++k) {
    if (names) {
      std::memset(names + 32 * k, 0, 32);
      std::strncpy(names + 32 * k, mgs::kNames[k], 31);
    }
    if (ms_total) ms_total[k] = mgs::g_ms[k];
    if (launches) launches[k] = mgs::g_count[k];
  }
  return mgs::kProfKinds;
}

}  // extern "C"
