// serve.cu -- continuous-batching render server (ssgi_serve_*).
//
// The method's real-time editing use (relighting and material edits, Sec. 4 "Editing") turned
// into a request loop.  One device arena (the HBM budget) is allocated at create and carved
// first-fit into per-request and per-scene blocks; max_slots CUDA streams carry admitted
// requests concurrently.  An engine thread admits queued requests in arrival order as soon as a
// slot is free and the arena has room for the head request (head-of-line order keeps large
// requests from starving); a host callback on the slot's stream retires the request when its
// copies and kernels are done, frees its block and wakes the engine.  Resident scenes keep a
// G-buffer and its Hi-Z pyramid on the device for many requests.  All waits are bounded on the
// host; nothing on the device waits for anything.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ssgi_internal.h"

namespace ssgi {
namespace serve {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;
inline size_t up(size_t n) { return (n + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing; host-side bookkeeping of the arena.
struct Arena {
  size_t size = 0, in_use = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t n) {
    size = n;
    free_.clear();
    if (n) free_[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    n = up(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, noff = it->first + n;
      free_.erase(it);
      if (rest) free_[noff] = rest;
      in_use += n;
      peak = std::max(peak, in_use);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = up(n);
    in_use -= n;
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
};

// Offsets (bytes) of a scene part (G-buffer + pyramid) and a request part (env, mips, c_d, c1,
// final) inside one arena block.
struct SceneLayout {
  size_t depth, normal, albedo, rough, metal, hiz, bytes;
};
struct ReqLayout {
  size_t env, mips, cd, c1, fin, bytes;
};

inline SceneLayout scene_layout(ssgi_dims d, int levels) {
  SceneLayout L;
  const size_t px = (size_t)d.views * d.height * d.width;
  size_t o = 0;
  L.depth = o; o += up(px * 4);
  L.normal = o; o += up(px * 12);
  L.albedo = o; o += up(px * 12);
  L.rough = o; o += up(px * 4);
  L.metal = o; o += up(px * 4);
  L.hiz = o; o += up(std::max<size_t>(ssgi_hiz_floats(d, levels), 1) * 4);
  L.bytes = o;
  return L;
}

inline ReqLayout req_layout(ssgi_dims d, int env_h, int env_w) {
  ReqLayout L;
  const size_t px = (size_t)d.views * d.height * d.width;
  size_t o = 0;
  L.env = o; o += up((size_t)env_h * env_w * 12);
  L.mips = o; o += up(ssgi_env_mip_floats(env_h, env_w) * 4);
  L.cd = o; o += up(px * 12);
  L.c1 = o; o += up(px * 12);
  L.fin = o; o += up(px * 12);
  L.bytes = o;
  return L;
}

enum State { kQueued, kRunning, kDone, kCancelled, kFailed };

struct Scene {
  ssgi_dims d;
  std::vector<ssgi_camera> cams;
  int levels;
  SceneLayout L;
  size_t off;
  int refs;
};

struct Request {
  ssgi_request r;
  std::vector<ssgi_camera> cams;
  Clock::time_point t_submit, t_done;
  State state = kQueued;
  size_t off = 0, bytes = 0;
  int slot = -1;
};

struct Server;

struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  uint64_t ticket = 0;
  Server* srv = nullptr;
};

struct Server {
  ssgi_serve_config cfg;
  int device = 0;
  char* base = nullptr;  // device arena
  float* lut = nullptr;  // device BRDF table
  int lut_n = 64;
  Arena arena;
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::map<int64_t, Scene> scenes;
  uint64_t next_ticket = 1;
  int64_t next_scene = 0;
  std::mutex mu;
  std::condition_variable cv_engine, cv_done;
  std::thread engine;
  bool stop = false;
  ssgi_serve_stats st{};
};

// Host callback run after a slot's stream finished a request's work (no CUDA calls here).
void CUDART_CB on_done(void* arg) {
  Slot* sl = static_cast<Slot*>(arg);
  Server* S = sl->srv;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(sl->ticket);
    if (it != S->reqs.end()) {
      Request& R = it->second;
      R.state = kDone;
      R.t_done = Clock::now();
      S->arena.release(R.off, R.bytes);
      if (R.r.scene >= 0) {
        auto sc = S->scenes.find(R.r.scene);
        if (sc != S->scenes.end()) --sc->second.refs;
      }
      ++S->st.completed;
      --S->st.in_flight;
    }
    sl->busy = false;
  }
  S->cv_engine.notify_one();
  S->cv_done.notify_all();
}

// Enqueue one admitted request's work on its slot's stream.  Called without the lock; the
// request, its block and the slot are reserved for it.
ssgi_status launch(Server* S, Request& R, Slot& sl, const Scene* sc) {
  cudaStream_t st = sl.stream;
  char* blk = S->base + R.off;
  const ssgi_request& q = R.r;
  ssgi_dims d;
  SceneLayout SL;
  char* sblk;
  const ssgi_camera* cams;
  int levels = q.params.hiz_levels;
  if (sc) {
    d = sc->d;
    SL = sc->L;
    sblk = S->base + sc->off;
    cams = sc->cams.data();
    levels = sc->levels;
  } else {
    d = q.d;
    SL = scene_layout(d, levels);
    sblk = blk;
    cams = R.cams.data();
    const size_t px = (size_t)d.views * d.height * d.width;
    const struct { const float* src; size_t off, n; } cp[5] = {
        {q.depth, SL.depth, px * 4}, {q.normal, SL.normal, px * 12}, {q.albedo, SL.albedo, px * 12},
        {q.rough, SL.rough, px * 4}, {q.metal, SL.metal, px * 4}};
    for (const auto& c : cp)
      if (cudaMemcpyAsync(sblk + c.off, c.src, c.n, cudaMemcpyHostToDevice, st) != cudaSuccess) return SSGI_ERR_CUDA;
    if (levels > 1) {
      const ssgi_status s1 = ssgi_build_hiz((const float*)(sblk + SL.depth), d, levels, (float*)(sblk + SL.hiz), st);
      if (s1 != SSGI_OK) return s1;
    }
  }
  const ReqLayout RL = req_layout(d, q.env_h, q.env_w);
  char* rblk = blk + (sc ? 0 : SL.bytes);
  if (cudaMemcpyAsync(rblk + RL.env, q.env, (size_t)q.env_h * q.env_w * 12, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SSGI_ERR_CUDA;
  ssgi_status s2 = ssgi_build_env_mips((const float*)(rblk + RL.env), q.env_h, q.env_w, (float*)(rblk + RL.mips), st);
  if (s2 != SSGI_OK) return s2;
  ssgi_gbuffer g;
  g.depth = (const float*)(sblk + SL.depth);
  g.normal = (const float*)(sblk + SL.normal);
  g.albedo = (const float*)(sblk + SL.albedo);
  g.rough = (const float*)(sblk + SL.rough);
  g.metal = (const float*)(sblk + SL.metal);
  g.d = d;
  ssgi_envmap e;
  e.mips = (const float*)(rblk + RL.mips);
  e.h = q.env_h;
  e.w = q.env_w;
  e.levels = ssgi_env_levels(q.env_h, q.env_w);
  s2 = ssgi_shade_direct(&g, cams, &e, S->lut, S->lut_n, (float*)(rblk + RL.cd), nullptr, (float*)(rblk + RL.c1), st);
  if (s2 != SSGI_OK) return s2;
  ssgi_trace_params p = q.params;
  p.hiz_levels = levels;
  s2 = ssgi_trace_indirect(&g, cams, levels > 1 ? (const float*)(sblk + SL.hiz) : nullptr, (const float*)(rblk + RL.c1),
                           (const float*)(rblk + RL.cd), &e, &p, nullptr, nullptr, (float*)(rblk + RL.fin), nullptr,
                           nullptr, st);
  if (s2 != SSGI_OK) return s2;
  const size_t px = (size_t)d.views * d.height * d.width;
  if (cudaMemcpyAsync(q.final_out, rblk + RL.fin, px * 12, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SSGI_ERR_CUDA;
  if (cudaLaunchHostFunc(st, on_done, &sl) != cudaSuccess) return SSGI_ERR_CUDA;
  return SSGI_OK;
}

void engine_main(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    if (S->stop) break;
    bool progressed = false;
    while (!S->queue.empty()) {
      int free_slot = -1;
      for (size_t i = 0; i < S->slots.size(); ++i)
        if (!S->slots[i].busy) {
          free_slot = (int)i;
          break;
        }
      if (free_slot < 0) break;
      const uint64_t t = S->queue.front();
      Request& R = S->reqs[t];
      if (!S->arena.alloc(R.bytes, &R.off)) break;  // head waits for memory
      S->queue.pop_front();
      Slot& sl = S->slots[free_slot];
      sl.busy = true;
      sl.ticket = t;
      R.state = kRunning;
      R.slot = free_slot;
      ++S->st.admitted;
      ++S->st.in_flight;
      const Scene* sc = nullptr;
      if (R.r.scene >= 0) sc = &S->scenes.at(R.r.scene);
      lk.unlock();
      const ssgi_status ls = launch(S, R, sl, sc);
      lk.lock();
      if (ls != SSGI_OK) {
        // the stream may hold part of the work: let it drain before the block is reused
        lk.unlock();
        cudaStreamSynchronize(sl.stream);
        lk.lock();
        R.state = kFailed;
        R.t_done = Clock::now();
        S->arena.release(R.off, R.bytes);
        if (sc) --S->scenes.at(R.r.scene).refs;
        sl.busy = false;
        --S->st.in_flight;
        S->cv_done.notify_all();
      }
      progressed = true;
    }
    if (!progressed) S->cv_engine.wait_for(lk, std::chrono::milliseconds(2));
  }
}

bool request_ok(const ssgi_request* q) {
  if (!q || !q->env || !q->final_out) return false;
  if (ssgi_env_levels(q->env_h, q->env_w) < 1) return false;
  if (trace_params_ok(&q->params) != SSGI_OK) return false;
  if (q->params.flags & SSGI_BRUTE_FORCE) return false;
  if (q->scene < 0) {
    if (!dims_ok(q->d) || !q->depth || !q->normal || !q->albedo || !q->rough || !q->metal || !q->cams) return false;
    Views vs;
    if (make_views(q->cams, q->d, &vs) != SSGI_OK) return false;
  }
  return true;
}

}  // namespace serve
}  // namespace ssgi

using namespace ssgi;
using namespace ssgi::serve;

extern "C" {

size_t ssgi_serve_request_bytes(ssgi_dims d, int32_t env_h, int32_t env_w, int32_t hiz_levels, int32_t resident) {
  if (!dims_ok(d) || ssgi_env_levels(env_h, env_w) < 1 || hiz_levels < 1 || hiz_levels > SSGI_MAX_HIZ_LEVELS) return 0;
  const size_t r = req_layout(d, env_h, env_w).bytes;
  return resident ? r : r + scene_layout(d, hiz_levels).bytes;
}

ssgi_status ssgi_serve_create(const ssgi_serve_config* cfg, ssgi_server** out) {
  if (!cfg || !out || cfg->hbm_budget_bytes < (1u << 20) || cfg->max_slots < 1 || cfg->max_slots > 64 ||
      cfg->queue_capacity < 1)
    return SSGI_ERR_INVALID_ARG;
  Server* S = new (std::nothrow) Server();
  if (!S) return SSGI_ERR_OOM;
  S->cfg = *cfg;
  S->lut_n = cfg->lut_n > 0 ? cfg->lut_n : 64;
  const int samples = cfg->lut_samples > 0 ? cfg->lut_samples : 4096;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return SSGI_ERR_CUDA;
  }
  if (cudaMalloc((void**)&S->base, cfg->hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return SSGI_ERR_OOM;
  }
  if (cudaMalloc((void**)&S->lut, (size_t)S->lut_n * S->lut_n * 2 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(S->base);
    delete S;
    return SSGI_ERR_OOM;
  }
  S->arena.init(cfg->hbm_budget_bytes);
  S->slots.resize(cfg->max_slots);
  for (auto& sl : S->slots) {
    sl.srv = S;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& s2 : S->slots)
        if (s2.stream) cudaStreamDestroy(s2.stream);
      cudaFree(S->lut);
      cudaFree(S->base);
      delete S;
      return SSGI_ERR_CUDA;
    }
  }
  if (ssgi_build_brdf_lut(S->lut_n, samples, S->lut, S->slots[0].stream) != SSGI_OK ||
      cudaStreamSynchronize(S->slots[0].stream) != cudaSuccess) {
    for (auto& s2 : S->slots) cudaStreamDestroy(s2.stream);
    cudaFree(S->lut);
    cudaFree(S->base);
    delete S;
    return SSGI_ERR_CUDA;
  }
  S->engine = std::thread(engine_main, S);
  *out = reinterpret_cast<ssgi_server*>(S);
  return SSGI_OK;
}

ssgi_status ssgi_serve_scene_add(ssgi_server* s, ssgi_dims d, const float* depth, const float* normal,
                                 const float* albedo, const float* rough, const float* metal,
                                 const ssgi_camera* cams, int32_t hiz_levels, int64_t* scene) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !scene || !dims_ok(d) || !depth || !normal || !albedo || !rough || !metal || !cams || hiz_levels < 1 ||
      hiz_levels > SSGI_MAX_HIZ_LEVELS)
    return SSGI_ERR_INVALID_ARG;
  Views vs;
  if (make_views(cams, d, &vs) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  Scene sc;
  sc.d = d;
  sc.cams.assign(cams, cams + d.views);
  sc.levels = hiz_levels;
  sc.L = scene_layout(d, hiz_levels);
  sc.refs = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->arena.alloc(sc.L.bytes, &sc.off)) return SSGI_ERR_BUDGET;
  }
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->arena.release(sc.off, sc.L.bytes);
    return SSGI_ERR_CUDA;
  }
  char* b = S->base + sc.off;
  const size_t px = (size_t)d.views * d.height * d.width;
  bool ok = cudaMemcpyAsync(b + sc.L.depth, depth, px * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b + sc.L.normal, normal, px * 12, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b + sc.L.albedo, albedo, px * 12, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b + sc.L.rough, rough, px * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(b + sc.L.metal, metal, px * 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (ok && hiz_levels > 1)
    ok = ssgi_build_hiz((const float*)(b + sc.L.depth), d, hiz_levels, (float*)(b + sc.L.hiz), st) == SSGI_OK;
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
  cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lk(S->mu);
  if (!ok) {
    S->arena.release(sc.off, sc.L.bytes);
    return SSGI_ERR_CUDA;
  }
  const int64_t id = S->next_scene++;
  S->scenes.emplace(id, std::move(sc));
  S->st.resident_scenes = (int32_t)S->scenes.size();
  *scene = id;
  return SSGI_OK;
}

ssgi_status ssgi_serve_scene_remove(ssgi_server* s, int64_t scene) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return SSGI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->scenes.find(scene);
  if (it == S->scenes.end()) return SSGI_ERR_INVALID_ARG;
  if (it->second.refs > 0) return SSGI_ERR_NOT_READY;
  S->arena.release(it->second.off, it->second.L.bytes);
  S->scenes.erase(it);
  S->st.resident_scenes = (int32_t)S->scenes.size();
  S->cv_engine.notify_one();
  return SSGI_OK;
}

ssgi_status ssgi_serve_submit(ssgi_server* s, const ssgi_request* req, uint64_t* ticket) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !ticket || !request_ok(req)) {
    if (S) {
      std::lock_guard<std::mutex> lk(S->mu);
      ++S->st.rejected;
    }
    return SSGI_ERR_INVALID_ARG;
  }
  Request R;
  R.r = *req;
  R.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  size_t bytes;
  if (req->scene >= 0) {
    auto it = S->scenes.find(req->scene);
    if (it == S->scenes.end()) {
      ++S->st.rejected;
      return SSGI_ERR_INVALID_ARG;
    }
    R.r.d = it->second.d;
    bytes = req_layout(it->second.d, req->env_h, req->env_w).bytes;
  } else {
    R.cams.assign(req->cams, req->cams + req->d.views);
    bytes = scene_layout(req->d, req->params.hiz_levels).bytes + req_layout(req->d, req->env_h, req->env_w).bytes;
  }
  if (up(bytes) > S->arena.size) {
    ++S->st.rejected;
    return SSGI_ERR_BUDGET;
  }
  if ((int)S->queue.size() >= S->cfg.queue_capacity) {
    ++S->st.rejected;
    return SSGI_ERR_QUEUE_FULL;
  }
  R.bytes = bytes;
  if (req->scene >= 0) ++S->scenes.at(req->scene).refs;
  const uint64_t t = S->next_ticket++;
  S->reqs.emplace(t, std::move(R));
  S->queue.push_back(t);
  ++S->st.submitted;
  *ticket = t;
  S->cv_engine.notify_one();
  return SSGI_OK;
}

static ssgi_status collect(Server* S, std::unordered_map<uint64_t, Request>::iterator it, double* latency_ms) {
  Request& R = it->second;
  ssgi_status rc = SSGI_OK;
  if (R.state == kCancelled) rc = SSGI_ERR_CANCELLED;
  if (R.state == kFailed) rc = SSGI_ERR_CUDA;
  if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(R.t_done - R.t_submit).count();
  S->reqs.erase(it);
  return rc;
}

ssgi_status ssgi_serve_poll(ssgi_server* s, uint64_t ticket, double* latency_ms) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return SSGI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return SSGI_ERR_INVALID_ARG;
  if (it->second.state == kQueued || it->second.state == kRunning) return SSGI_ERR_NOT_READY;
  return collect(S, it, latency_ms);
}

ssgi_status ssgi_serve_wait(ssgi_server* s, uint64_t ticket, uint32_t timeout_ms, double* latency_ms) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return SSGI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SSGI_ERR_INVALID_ARG;
    if (it->second.state != kQueued && it->second.state != kRunning) return collect(S, it, latency_ms);
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto jt = S->reqs.find(ticket);
      if (jt != S->reqs.end() && jt->second.state != kQueued && jt->second.state != kRunning)
        return collect(S, jt, latency_ms);
      return SSGI_ERR_TIMEOUT;
    }
  }
}

ssgi_status ssgi_serve_cancel(ssgi_server* s, uint64_t ticket) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return SSGI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return SSGI_ERR_INVALID_ARG;
  Request& R = it->second;
  if (R.state == kRunning) return SSGI_ERR_NOT_READY;
  if (R.state != kQueued) return SSGI_ERR_INVALID_ARG;
  S->queue.erase(std::find(S->queue.begin(), S->queue.end(), ticket));
  R.state = kCancelled;
  R.t_done = Clock::now();
  if (R.r.scene >= 0) --S->scenes.at(R.r.scene).refs;
  ++S->st.cancelled;
  S->cv_done.notify_all();
  S->cv_engine.notify_one();
  return SSGI_OK;
}

ssgi_status ssgi_serve_stats_get(ssgi_server* s, ssgi_serve_stats* out) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S || !out) return SSGI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->queued = (int32_t)S->queue.size();
  out->arena_bytes_in_use = S->arena.in_use;
  out->arena_bytes_peak = S->arena.peak;
  return SSGI_OK;
}

ssgi_status ssgi_serve_destroy(ssgi_server* s, uint32_t timeout_ms) {
  Server* S = reinterpret_cast<Server*>(s);
  if (!S) return SSGI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (uint64_t t : S->queue) {
      Request& R = S->reqs[t];
      R.state = kCancelled;
      R.t_done = Clock::now();
      if (R.r.scene >= 0) --S->scenes.at(R.r.scene).refs;
      ++S->st.cancelled;
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv_engine.notify_all();
  S->cv_done.notify_all();
  if (S->engine.joinable()) S->engine.join();
  // running requests: bounded wait for their streams
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  for (auto& sl : S->slots) {
    for (;;) {
      const cudaError_t q = cudaStreamQuery(sl.stream);
      if (q != cudaErrorNotReady) break;
      if (Clock::now() > deadline) {
        // restart the engine so the server stays usable; the caller may call destroy again
        S->stop = false;
        S->engine = std::thread(engine_main, S);
        return SSGI_ERR_TIMEOUT;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  // host callbacks of finished streams may still be running: take the lock once more
  { std::lock_guard<std::mutex> lk(S->mu); }
  for (auto& sl : S->slots) cudaStreamDestroy(sl.stream);
  cudaFree(S->lut);
  cudaFree(S->base);
  delete S;
  return SSGI_OK;
}

}  // extern "C"
