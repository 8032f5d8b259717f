// Render-serving loop with continuous batching (host runtime, C++).
//
// Resident scene maps; requests (scene, camera, output planes) arrive at any time.  A
// dispatcher thread admits the oldest pending requests, of any scene and resolution, as
// soon as a worker slot is free: up to max_batch_views of them, as many as fit in free
// memory of the caller's device arena, go into one mgs_render_multi call (one
// projection launch per map, then one sort, one emission and one blend launch over all
// their (view, tile) items).  Each slot owns a CUDA stream and a worker thread, so
// admitted batches run concurrently on the device while new requests keep arriving.  The arena is carved first-fit; nothing is allocated on the
// device.  Workspace sizes are learnt per (scene, resolution) from the key counts of
// earlier renders; a render that reports a too-small workspace is retried once with the
// reported size if the arena has room, and otherwise goes back to the head of the queue.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Request {
  int64_t tag;
  int scene;
  mgs_camera cam;
  mgs_image out;
  double t_submit, t_start = 0, t_done = 0;
  mgs_status status = MGS_OK;
};

struct Arena {
  char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(void* b, size_t n) {
    base = static_cast<char*>(b);
    bytes = n;
    free_.clear();
    if (n) free_[0] = n;
  }
  // first fit, 256-byte aligned; returns SIZE_MAX when nothing fits
  size_t take(size_t n) {
    n = mgs::align_up(std::max<size_t>(n, 256));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        size_t off = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void give(size_t off, size_t n) {
    n = mgs::align_up(std::max<size_t>(n, 256));
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
};

struct Batch {
  std::vector<Request> reqs;
  std::vector<mgs_gaussians> maps;      // distinct maps of the batch, copied under the lock
  std::vector<int32_t> map_of_view;     // per request: index into maps
  size_t off = SIZE_MAX, bytes = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  std::thread th;
  bool busy = false;
  Batch work;
  bool has_work = false;
};

}  // namespace

struct mgs_server {
  mgs_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_disp, cv_work, cv_done;
  std::vector<mgs_gaussians> scenes;
  std::deque<Request> pending;
  std::vector<Request> done;
  std::vector<Slot> slots;
  Arena arena;
  std::map<std::pair<int, int64_t>, int64_t> keys_seen;  // (scene, w*65536+h) -> keys per view
  int64_t in_flight = 0;
  int64_t n_launches = 0, n_served = 0, max_views = 0, mixed_launches = 0;
  bool stop = false;
  std::thread dispatcher;
  std::string last_error;

  // keys of one view: learnt from earlier renders, else 8 per Gaussian
  int64_t raw_keys(int scene, const mgs_camera& c) {
    auto it = keys_seen.find({scene, (int64_t)c.width * 65536 + c.height});
    return it != keys_seen.end() ? it->second : 8 * scenes[scene].n;
  }
  int64_t est_keys(int scene, const mgs_camera& c) {
    const int64_t k = raw_keys(scene, c);
    return k + k / 4 + 1024;
  }
  // the batch's maps and views (call with the lock held)
  void bind_maps(Batch& b) {
    b.maps.clear();
    b.map_of_view.clear();
    std::vector<int> ids;
    for (auto& r : b.reqs) {
      int m = -1;
      for (size_t k = 0; k < ids.size(); ++k)
        if (ids[k] == r.scene) m = (int)k;
      if (m < 0) {
        m = (int)ids.size();
        ids.push_back(r.scene);
        b.maps.push_back(scenes[r.scene]);
      }
      b.map_of_view.push_back(m);
    }
  }
  size_t need_bytes(Batch& b) {
    bind_maps(b);
    std::vector<mgs_camera> cams;
    int64_t keys = 0;
    for (auto& r : b.reqs) {
      cams.push_back(r.cam);
      keys += est_keys(r.scene, r.cam);
    }
    return mgs_render_multi_workspace_size(b.maps.data(), (int)b.maps.size(), b.map_of_view.data(), cams.data(),
                                           (int)cams.size(), keys);
  }

  void dispatch_loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      int free_slot = -1;
      for (size_t i = 0; i < slots.size(); ++i)
        if (!slots[i].busy) { free_slot = (int)i; break; }
      if (pending.empty() || free_slot < 0) {
        cv_disp.wait(lk);
        continue;
      }
      // the oldest pending requests, any scene and resolution (up to the batch cap)
      Batch b;
      while (!pending.empty() && (int)b.reqs.size() < cfg.max_batch_views) {
        b.reqs.push_back(pending.front());
        pending.pop_front();
      }
      // admission by free arena memory: shrink the batch until it fits; if even the
      // oldest request alone does not fit, wait for running work to free memory
      while (true) {
        size_t need = need_bytes(b);
        size_t off = arena.take(need);
        if (off != SIZE_MAX) {
          b.off = off;
          b.bytes = need;
          break;
        }
        if (b.reqs.size() == 1) break;
        pending.push_front(b.reqs.back());
        b.reqs.pop_back();
      }
      bind_maps(b);
      if (b.off == SIZE_MAX) {
        for (auto it = b.reqs.rbegin(); it != b.reqs.rend(); ++it) pending.push_front(*it);
        if (in_flight == 0) {  // nothing will ever free memory: fail the request
          Request r = pending.front();
          pending.pop_front();
          r.status = MGS_ERR_WORKSPACE;
          r.t_start = r.t_done = now_s();
          done.push_back(r);
          cv_done.notify_all();
          continue;
        }
        cv_disp.wait(lk);
        continue;
      }
      double t0 = now_s();
      for (auto& r : b.reqs) r.t_start = t0;
      Slot& s = slots[free_slot];
      s.busy = true;
      s.work = std::move(b);
      s.has_work = true;
      in_flight += 1;
      cv_work.notify_all();
    }
  }

  void worker_loop(int idx) {
    Slot& s = slots[idx];
    cudaSetDevice(cfg.device);
    while (true) {
      Batch b;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || s.has_work; });
        if (stop && !s.has_work) return;
        b = std::move(s.work);
        s.has_work = false;
      }
      std::vector<mgs_camera> cams;
      std::vector<mgs_image> outs;
      for (auto& r : b.reqs) {
        cams.push_back(r.cam);
        outs.push_back(r.out);
      }
      // the batch's maps were copied by the dispatcher under the lock: no access to
      // `scenes` here, which add_scene may grow meanwhile
      const int nm = (int)b.maps.size();
      int64_t nk = 0;
      mgs_status st = mgs_render_multi(b.maps.data(), nm, b.map_of_view.data(), cams.data(), (int)cams.size(),
                                       outs.data(), arena.base + b.off, b.bytes, &nk, s.stream);
      if (st == MGS_ERR_WORKSPACE && nk > 0) {
        // learn the true size and retry once with a bigger block if the arena has room
        size_t need = mgs_render_multi_workspace_size(b.maps.data(), nm, b.map_of_view.data(), cams.data(),
                                                      (int)cams.size(), nk + nk / 8 + 1024);
        std::unique_lock<std::mutex> lk(mu);
        arena.give(b.off, b.bytes);
        size_t off = arena.take(need);
        if (off != SIZE_MAX) {
          b.off = off;
          b.bytes = need;
          lk.unlock();
          st = mgs_render_multi(b.maps.data(), nm, b.map_of_view.data(), cams.data(), (int)cams.size(),
                                outs.data(), arena.base + b.off, b.bytes, &nk, s.stream);
        } else {
          b.off = SIZE_MAX;
        }
      }
      if (st == MGS_OK && cudaStreamSynchronize(s.stream) != cudaSuccess) st = MGS_ERR_CUDA;
      double t1 = now_s();
      std::unique_lock<std::mutex> lk(mu);
      if (b.off != SIZE_MAX) arena.give(b.off, b.bytes);
      if ((st == MGS_OK || st == MGS_ERR_WORKSPACE) && nk > 0) {
        // the key count of the whole batch, shared out over its views in proportion to
        // what each view was expected to need
        double expect = 0;
        for (auto& r : b.reqs) expect += (double)raw_keys(r.scene, r.cam);
        const double ratio = expect > 0 ? (double)nk / expect : 1.0;
        for (auto& r : b.reqs) {
          const int64_t k = (int64_t)(ratio * (double)raw_keys(r.scene, r.cam)) + 1;
          keys_seen[{r.scene, (int64_t)r.cam.width * 65536 + r.cam.height}] = k;
        }
      }
      if (st == MGS_OK) {
        n_launches += 1;
        n_served += (int64_t)b.reqs.size();
        max_views = std::max<int64_t>(max_views, (int64_t)b.reqs.size());
        if (b.maps.size() > 1) mixed_launches += 1;
      }
      if (st == MGS_ERR_WORKSPACE && b.off == SIZE_MAX) {
        // too big for the arena right now: queue the requests again (sizes learnt above)
        for (auto it = b.reqs.rbegin(); it != b.reqs.rend(); ++it) pending.push_front(*it);
      } else {
        for (auto& r : b.reqs) {
          r.t_done = t1;
          r.status = st;
          done.push_back(r);
        }
        if (st != MGS_OK) last_error = mgs_last_error();
      }
      s.busy = false;
      in_flight -= 1;
      cv_disp.notify_all();
      cv_done.notify_all();
    }
  }
};

extern "C" {

mgs_status mgs_server_create(const mgs_server_config* cfg, mgs_server** out) {
  mgs::set_error("");
  if (!cfg || !out) {
    mgs::set_error("NULL argument");
    return MGS_ERR_INVALID;
  }
  if (cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->max_batch_views < 1 || cfg->max_batch_views > MGS_MAX_VIEWS ||
      !cfg->arena || cfg->arena_bytes < (1u << 20)) {
    mgs::set_error("need 1 <= n_slots <= 64, 1 <= max_batch_views <= MGS_MAX_VIEWS and an arena of >= 1 MiB");
    return MGS_ERR_INVALID;
  }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    mgs::set_error("cudaSetDevice failed");
    return MGS_ERR_CUDA;
  }
  auto* s = new mgs_server();
  s->cfg = *cfg;
  s->arena.init(cfg->arena, cfg->arena_bytes);
  s->slots.resize(cfg->n_slots);
  for (auto& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& x : s->slots)
        if (x.stream) cudaStreamDestroy(x.stream);
      delete s;
      mgs::set_error("cudaStreamCreate failed");
      return MGS_ERR_CUDA;
    }
  }
  for (int i = 0; i < cfg->n_slots; ++i) s->slots[i].th = std::thread([s, i] { s->worker_loop(i); });
  s->dispatcher = std::thread([s] { s->dispatch_loop(); });
  *out = s;
  return MGS_OK;
}

mgs_status mgs_server_add_scene(mgs_server* s, const mgs_gaussians* g, int32_t* scene_id) {
  mgs::set_error("");
  if (!s || !g || !scene_id || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) {
    mgs::set_error("bad arguments");
    return MGS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->scenes.push_back(*g);
  *scene_id = (int32_t)s->scenes.size() - 1;
  return MGS_OK;
}

mgs_status mgs_server_submit(mgs_server* s, int32_t scene_id, const mgs_camera* cam, const mgs_image* out,
                             int64_t tag, double t_submit) {
  mgs::set_error("");
  if (!s || !cam || !out || !out->rgb || !out->depth || !out->alpha || cam->width <= 0 || cam->height <= 0) {
    mgs::set_error("bad arguments");
    return MGS_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size()) {
    mgs::set_error("unknown scene id");
    return MGS_ERR_INVALID;
  }
  Request r;
  r.tag = tag;
  r.scene = scene_id;
  r.cam = *cam;
  r.out = *out;
  r.t_submit = t_submit > 0 ? t_submit : now_s();
  s->pending.push_back(r);
  s->cv_disp.notify_all();
  return MGS_OK;
}

int32_t mgs_server_poll(mgs_server* s, int32_t max, int64_t* tags, double* t_submit, double* t_start,
                        double* t_done, int32_t* status, double wait_s) {
  if (!s || max <= 0) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_s > 0)
    s->cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !s->done.empty(); });
  int n = std::min<int>(max, (int)s->done.size());
  for (int i = 0; i < n; ++i) {
    const Request& r = s->done[i];
    if (tags) tags[i] = r.tag;
    if (t_submit) t_submit[i] = r.t_submit;
    if (t_start) t_start[i] = r.t_start;
    if (t_done) t_done[i] = r.t_done;
    if (status) status[i] = r.status;
  }
  s->done.erase(s->done.begin(), s->done.begin() + n);
  return n;
}

double mgs_server_clock(void) { return now_s(); }

mgs_status mgs_server_stats(mgs_server* s, int64_t out[4]) {
  if (!s || !out) return MGS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->n_launches;
  out[1] = s->n_served;
  out[2] = s->max_views;
  out[3] = s->mixed_launches;
  return MGS_OK;
}

mgs_status mgs_server_destroy(mgs_server* s) {
  if (!s) return MGS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_disp.notify_all();
  s->cv_work.notify_all();
  s->dispatcher.join();
  for (auto& sl : s->slots) sl.th.join();
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
  }
  delete s;
  return MGS_OK;
}

}  // extern "C"
