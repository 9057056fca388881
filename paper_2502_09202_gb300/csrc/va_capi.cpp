// extern "C" entry points of include/analyser.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>

#include "../../include/analyser.h"
#include "va_detect.h"
#include "va_engine.h"

struct analyser {
  std::unique_ptr<va::Engine> eng;
  va::Clip clip;
  va::ResultsBuf res;
  int status = ANALYSER_OK;
  std::string msg;
  bool offline = false;
};

struct server {
  analyser_params p{};
  unsigned long long budget = 0;
  unsigned long long used = 0;
  std::unique_ptr<va::Engine> eng;
  struct Req {
    std::unique_ptr<va::Clip> clip;
    const uint8_t* frames = nullptr;
    long long pitch = 0;
    int nframes = 0, uploaded = 0;
    bool admitted = false, done = false;
    double t_submit = 0, t_done = 0;
    va::ResultsBuf res;
    size_t bytes = 0;
  };
  std::map<long long, Req> reqs;
  std::deque<long long> queue;
  long long next_ticket = 1;
  int status = ANALYSER_OK;
  std::string msg;
};

namespace {

int fail(analyser* a, int code, const std::string& why) {
  a->status = code;
  a->msg = why;
  return code;
}

int fail_srv(server* s, int code, const std::string& why) {
  s->status = code;
  s->msg = why;
  return code;
}

// Run waves until the clip's detector is done (finish) or no more progress is
// possible without new frames.  Short of the end, it also returns for more
// frames once a quarter of the window is free, even with deep checks still
// requested: the next wave then carries those checks beside the new frames'
// adjacent pairs (fewer, fuller waves; every measure is the same whichever
// wave computes it).
int drive(analyser* a, bool to_end) {
  va::Engine& e = *a->eng;
  const int merge_slots = std::max(32, a->clip.cap / 4);
  for (;;) {
    const int rc = e.wave();
    if (rc < 0 || e.status) return fail(a, e.status ? e.status : rc, e.message);
    if (a->clip.done()) return ANALYSER_OK;
    if (rc == 0) {
      if (to_end) return fail(a, ANALYSER_ERR_STATE, "analysis stalled before the end of the clip");
      return ANALYSER_OK;
    }
    if (to_end) continue;
    const int free = e.free_slots(&a->clip);
    if ((free > 0 && a->clip.pending.empty()) || free >= merge_slots) return ANALYSER_OK;
  }
}

}  // namespace

extern "C" {

int analyser_default_params(analyser_params* p) {
  if (!p) return ANALYSER_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->block = 16;
  p->levels = 3;
  p->radius_coarse = 16;
  p->radius_refine = 2;
  p->mv_cost = 4;
  p->kmax = 8;
  p->jback = 2;
  p->fast_window = 8;
  p->fast_lambda = 2.0;
  p->fast_rise = 1.3;
  p->fast_tau = 0.5;
  p->deep_rho = 2.0;
  p->deep_tau = 0.5;
  p->done_eps = 0.25;
  p->steady_gamma = 1.2;
  p->steady_frames = 4;
  p->steady_span = 2;
  p->lag_rho = 1.5;
  p->blend_ratio = 0.6;
  p->pd_rho = 1.4;
  p->pd_gamma_new = 2.5;
  p->pd_gamma_old = 1.4;
  p->samp_max_frames = 20;
  p->static_amm_px = 0.5;
  p->comb_ratio = 0.65;
  p->unequal_ratio = 1.04;
  p->rep_ratio = 0.25;
  p->rep_probe = 5;
  p->pulldown_match = 0.8;
  p->kf_theta = 8.0;
  p->device = 0;
  p->window_frames = 0;
  p->mem_budget_bytes = 0;
  p->want_motion = 0;
  p->tile_x = 0;
  p->tile_y = 0;
  p->time_kernels = 0;
  p->step_frames = 32;
  p->kernel_mode = 0;
  p->want_histogram = 0;
  p->prefetch_frames = 256;
  p->wait_timeout_ms = 0.0;
  return ANALYSER_OK;
}

int analyser_create(int width, int height, double fps, const analyser_params* p, analyser** out) {
  if (!p || !out) return ANALYSER_ERR_INVALID_ARG;
  const double t0 = va::now_seconds();
  *out = nullptr;
  std::string why;
  int rc = va::validate_params(*p, why);
  if (!rc) rc = va::validate_size(width, height, *p, why);
  if (rc) return rc;
  if (!(fps > 0)) return ANALYSER_ERR_INVALID_ARG;
  {
    // the window's bytes are known from the sizes alone: refuse an over-budget
    // clip before touching the device
    va::Geometry g;
    g.init(width, height, p->levels);
    const int cap = p->window_frames > 0 ? p->window_frames : std::max(96, va::min_window(*p) + 2);
    if (p->mem_budget_bytes && va::Engine::ring_bytes(g, cap) > p->mem_budget_bytes) return ANALYSER_ERR_OOM;
  }
  analyser* a = new (std::nothrow) analyser();
  if (!a) return ANALYSER_ERR_OOM;
  a->eng.reset(new (std::nothrow) va::Engine(*p));
  if (!a->eng) { delete a; return ANALYSER_ERR_OOM; }
  rc = a->eng->init(why);
  if (rc) { delete a; return rc; }
  a->clip.geo.W = width;
  a->clip.geo.H = height;
  a->clip.fps = fps;
  rc = a->eng->add_clip(&a->clip, why);
  if (rc) {
    a->eng->clips.clear();
    delete a;
    return rc;
  }
  a->eng->host_setup_ms += 1e3 * (va::now_seconds() - t0);
  *out = a;
  return ANALYSER_OK;
}

int analyser_push_frames(analyser* a, const uint8_t* luma, long long pitch_bytes, int nframes) {
  if (!a) return ANALYSER_ERR_INVALID_ARG;
  if (a->status) return a->status;
  if (a->offline) return ANALYSER_ERR_STATE;
  if (a->clip.finished) return fail(a, ANALYSER_ERR_STATE, "push after analyser_finish");
  if (nframes < 0 || (nframes > 0 && !luma) || pitch_bytes < a->clip.geo.W) return ANALYSER_ERR_INVALID_ARG;
  if (a->clip.external_l0) return fail(a, ANALYSER_ERR_STATE, "host and device pushes cannot be mixed");
  va::Engine& e = *a->eng;
  // pipeline: keep every free slot of the window filled with copies in flight
  // (chunks of frames, one event each); launch a wave whenever resident frames
  // or requested pairs give work, and block on a copy only when nothing else
  // can run, so that copies and kernels overlap
  constexpr int kChunk = 16;
  constexpr int kMinWave = 64;   // new frames a wave waits for while copies stream in
  int done = 0;
  int stall = 0;
  for (;;) {
    if (done < nframes) {
      const int k = e.upload_async(&a->clip, luma + (size_t)done * a->clip.geo.H * pitch_bytes, pitch_bytes,
                                   nframes - done, kChunk);
      if (k < 0 || e.status) return fail(a, e.status ? e.status : ANALYSER_ERR_CUDA, e.message);
      done += k;
    }
    if (e.poll_uploads(&a->clip, false) < 0) return fail(a, e.status ? e.status : ANALYSER_ERR_CUDA, e.message);
    // every wave costs a host round trip: while copies are still landing and
    // the detectors ask for nothing, let a few chunks accumulate first
    if (!a->clip.up_chunks.empty() && a->clip.pending.empty() && a->clip.pushed - a->clip.pyr_done < kMinWave) {
      if (e.poll_uploads(&a->clip, true) < 0) return fail(a, e.status ? e.status : ANALYSER_ERR_CUDA, e.message);
      continue;
    }
    const int launched = e.wave_launch();
    if (launched < 0 || e.status) return fail(a, e.status ? e.status : launched, e.message);
    if (launched > 0) {
      const int rc = e.wave_complete();
      if (rc < 0 || e.status) return fail(a, e.status ? e.status : rc, e.message);
      stall = 0;
      continue;
    }
    if (!a->clip.up_chunks.empty()) {
      if (e.poll_uploads(&a->clip, true) < 0) return fail(a, e.status ? e.status : ANALYSER_ERR_CUDA, e.message);
      stall = 0;
      continue;
    }
    if (done >= nframes) break;
    if (++stall > 2) return fail(a, ANALYSER_ERR_STATE, "frame window cannot advance");
  }
  // every copy has completed: the caller may reuse its buffer
  return ANALYSER_OK;
}

int analyser_push_frames_device(analyser* a, const uint8_t* luma, long long pitch_bytes, long long frame_stride_bytes,
                                int nframes) {
  if (!a) return ANALYSER_ERR_INVALID_ARG;
  if (a->status) return a->status;
  if (a->offline) return ANALYSER_ERR_STATE;
  if (a->clip.finished) return fail(a, ANALYSER_ERR_STATE, "push after analyser_finish");
  // field views double the pitch, and the kernels' plane descriptors hold it in an int
  if (nframes < 0 || (nframes > 0 && !luma) || pitch_bytes < a->clip.geo.W || pitch_bytes % 16 ||
      pitch_bytes > INT_MAX / 2 || frame_stride_bytes % 16 || ((uintptr_t)luma % 16) ||
      frame_stride_bytes < pitch_bytes * a->clip.geo.H)
    return ANALYSER_ERR_INVALID_ARG;
  if (a->clip.pushed > 0 && !a->clip.external_l0)
    return fail(a, ANALYSER_ERR_STATE, "host and device pushes cannot be mixed");
  va::Engine& e = *a->eng;
  int done = 0;
  while (done < nframes) {
    const int k = e.attach_device(&a->clip, luma + (size_t)done * frame_stride_bytes, pitch_bytes, frame_stride_bytes,
                                  nframes - done);
    done += k;
    if (done < nframes) {
      const int rc = drive(a, false);
      if (rc) return rc;
      if (e.free_slots(&a->clip) == 0) {
        const int rc2 = e.wave();
        if (rc2 < 0) return fail(a, e.status, e.message);
        if (e.free_slots(&a->clip) == 0) return fail(a, ANALYSER_ERR_STATE, "frame window cannot advance");
      }
    }
  }
  return ANALYSER_OK;
}

int analyser_finish(analyser* a) {
  if (!a) return ANALYSER_ERR_INVALID_ARG;
  if (a->status) return a->status;
  if (a->offline) return ANALYSER_OK;
  a->clip.finished = true;
  const int rc = drive(a, true);
  if (rc) return rc;
  const cudaError_t e = a->eng->wait_stream(a->eng->stream);
  if (e == cudaErrorTimeout) return fail(a, ANALYSER_ERR_TIMEOUT, "analyser_finish: GPU work not complete in wait_timeout_ms");
  if (e != cudaSuccess) return fail(a, ANALYSER_ERR_CUDA, "cudaStreamSynchronize");
  return ANALYSER_OK;
}

int analyser_results(analyser* a, analyser_results_t* out) {
  if (!a || !out) return ANALYSER_ERR_INVALID_ARG;
  if (a->status) return a->status;
  if (!a->clip.done()) return ANALYSER_ERR_STATE;
  va::build_results(a->clip, a->res);
  *out = a->res.r;
  return ANALYSER_OK;
}

int analyser_last_error(const analyser* a, const char** message) {
  if (!a) return ANALYSER_ERR_INVALID_ARG;
  if (message) *message = a->msg.c_str();
  return a->status;
}

int analyser_stats(const analyser* a, long long* pairs, long long* waves, long long* launches) {
  if (!a) return ANALYSER_ERR_INVALID_ARG;
  if (pairs) *pairs = a->eng ? a->eng->n_pairs : 0;
  if (waves) *waves = a->eng ? a->eng->n_waves : 0;
  if (launches) *launches = a->eng ? a->eng->n_launches : 0;
  return ANALYSER_OK;
}

int analyser_profile(const analyser* a, analyser_profile_t* out) {
  if (!a || !out) return ANALYSER_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (a->eng) a->eng->profile(out);
  return ANALYSER_OK;
}

void analyser_destroy(analyser* a) {
  if (!a) return;
  if (a->eng) {
    a->eng->remove_clip(&a->clip);
    if (a->eng->stream) cudaStreamSynchronize(a->eng->stream);
  }
  delete a;
}

int analyser_measure_pairs(const analyser_params* p, int width, int height, const uint8_t* frames,
                           long long pitch_bytes, long long frame_stride_bytes, int nframes, const int* kinds,
                           const int* ia, const int* ib, int npairs, int64_t* records, int16_t* motion,
                           void* stream) {
  if (!p) return ANALYSER_ERR_INVALID_ARG;
  va::Engine e(*p);
  std::string why;
  int rc = e.init(why);
  if (rc) return rc;
  e.autotune = false;
  return e.measure_pairs(width, height, frames, pitch_bytes, frame_stride_bytes, nframes, kinds, ia, ib, npairs,
                         records, motion, (cudaStream_t)stream, why);
}

int analyser_detect_offline(const analyser_params* p, int width, int height, int nframes, analyser_measure_fn get,
                            void* ctx, analyser** out) {
  if (!p || !get || !out || nframes < 0) return ANALYSER_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = va::validate_params(*p, why);
  if (!rc) rc = va::validate_size(width, height, *p, why);
  if (rc) return rc;
  analyser* a = new (std::nothrow) analyser();
  if (!a) return ANALYSER_ERR_OOM;
  a->offline = true;
  va::Clip& c = a->clip;
  c.p = *p;
  c.geo.init(width, height, p->levels);
  c.pushed = nframes;
  c.finished = true;
  c.det.reset(*p, (int64_t)(width / c.geo.B0) * (height / c.geo.B0));
  auto fetch = [&](uint64_t key) -> int {
    int64_t rec[9];
    if (get(ctx, va::key_kind(key), va::key_a(key), va::key_b(key), rec)) return ANALYSER_ERR_INVALID_ARG;
    va::Measure m;
    for (int k = 0; k < 7; k++) m.s[k] = rec[k];
    m.n = rec[7];
    m.nb = rec[8];
    m.used = va::key_kind(key) == va::kFrame && va::key_b(key) == va::key_a(key) + 1;
    va::finalise_measure(m);
    c.store.map[key] = m;
    return ANALYSER_OK;
  };
  for (int t = 0; t + 1 < nframes; t++) {
    if (fetch(va::pair_key(va::kFrame, t, t + 1))) { delete a; return ANALYSER_ERR_INVALID_ARG; }
  }
  for (int guard = 0; guard < 10000000 && !c.det.done(); guard++) {
    std::vector<uint64_t> need;
    c.det.run(c.store, nframes, true, need);
    std::sort(need.begin(), need.end());
    need.erase(std::unique(need.begin(), need.end()), need.end());
    for (uint64_t k : need)
      if (!c.store.map.count(k) && fetch(k)) { delete a; return ANALYSER_ERR_INVALID_ARG; }
    if (need.empty() && !c.det.done()) { delete a; return ANALYSER_ERR_STATE; }
  }
  *out = a;
  return ANALYSER_OK;
}

// ---------------------------------------------------------------------------
// serving
// ---------------------------------------------------------------------------

int server_create(const analyser_params* p, unsigned long long budget_bytes, server** out) {
  if (!p || !out) return ANALYSER_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = va::validate_params(*p, why);
  if (rc) return rc;
  server* s = new (std::nothrow) server();
  if (!s) return ANALYSER_ERR_OOM;
  s->p = *p;
  s->budget = budget_bytes;
  s->eng.reset(new (std::nothrow) va::Engine(*p));
  if (!s->eng) { delete s; return ANALYSER_ERR_OOM; }
  rc = s->eng->init(why);
  // one tile shape for every clip (8x4 unless the parameters fix one): a wave's
  // pairs of all sizes then go out as one coarse and one refinement launch
  // (a tile changes the schedule only, never a result)
  s->eng->autotune = false;
  s->eng->max_chunks = 1;
  if (rc) { delete s; return rc; }
  *out = s;
  return ANALYSER_OK;
}

int server_submit(server* s, int width, int height, double fps, const uint8_t* frames, long long pitch_bytes,
                  int nframes, long long* ticket) {
  if (!s || !ticket || nframes < 0 || (nframes > 0 && !frames) || pitch_bytes < width || !(fps > 0))
    return ANALYSER_ERR_INVALID_ARG;
  if (s->status) return s->status;
  std::string why;
  int rc = va::validate_size(width, height, s->p, why);
  if (rc) return rc;
  const long long t = s->next_ticket++;
  server::Req& r = s->reqs[t];
  r.clip.reset(new (std::nothrow) va::Clip());
  if (!r.clip) { s->reqs.erase(t); return ANALYSER_ERR_OOM; }
  r.clip->id = t;
  r.clip->geo.W = width;
  r.clip->geo.H = height;
  r.clip->fps = fps;
  r.frames = frames;
  r.pitch = pitch_bytes;
  r.nframes = nframes;
  r.t_submit = va::now_seconds();
  r.clip->t_submit = r.t_submit;
  // window size is fixed at admission; estimate its bytes now for the budget
  va::Geometry g;
  g.init(width, height, s->p.levels);
  const int cap = s->p.window_frames > 0 ? s->p.window_frames : std::max(96, va::min_window(s->p) + 2);
  r.bytes = va::Engine::ring_bytes(g, cap);
  if (s->budget && r.bytes > s->budget) {
    s->reqs.erase(t);
    return ANALYSER_ERR_OOM;
  }
  s->queue.push_back(t);
  *ticket = t;
  return ANALYSER_OK;
}

int server_step(server* s, int* active) {
  if (!s) return ANALYSER_ERR_INVALID_ARG;
  if (s->status) return s->status;
  va::Engine& e = *s->eng;
  // admission in arrival order of every queued clip whose window fits what is
  // left of the budget: a clip too large for the space free now does not hold
  // back smaller ones behind it, unless it has waited kHeadWaitS already, in
  // which case nothing behind it is admitted until it is
  constexpr double kHeadWaitS = 0.5;
  const double now = va::now_seconds();
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    server::Req& r = s->reqs[*it];
    const bool head = it == s->queue.begin();
    bool admit = !(s->budget && s->used + r.bytes > s->budget);
    if (admit) {
      std::string why;
      const int rc = e.add_clip(r.clip.get(), why);
      if (rc == ANALYSER_ERR_OOM && !e.clips.empty()) admit = false;   // retry when memory frees up
      else if (rc) return fail_srv(s, rc, why);
    }
    if (admit) {
      r.admitted = true;
      s->used += r.bytes;
      it = s->queue.erase(it);
      continue;
    }
    if (head && now - r.t_submit > kHeadWaitS) break;
    ++it;
  }
  // top up every admitted clip's window with asynchronous chunked copies (at
  // most step_frames new frames per clip and step, so that short clips arriving
  // later are not queued behind long ones); frames join the analysis once their
  // copy has landed, so the wave below overlaps the copies issued here
  constexpr int kChunk = 16;
  for (auto& kv : s->reqs) {
    server::Req& r = kv.second;
    if (!r.admitted || r.done) continue;
    if (r.uploaded < r.nframes) {
      int n = r.nframes - r.uploaded;
      if (s->p.step_frames > 0 && n > s->p.step_frames) n = s->p.step_frames;
      const int k = e.upload_async(r.clip.get(), r.frames + (size_t)r.uploaded * r.clip->geo.H * r.pitch, r.pitch,
                                   n, kChunk);
      if (k < 0) return fail_srv(s, e.status, e.message);
      r.uploaded += k;
    }
  }
  auto land = [&](bool wait) -> int {
    bool waited = !wait;
    for (auto& kv : s->reqs) {
      server::Req& r = kv.second;
      if (!r.admitted || r.done) continue;
      const bool block = !waited && !r.clip->up_chunks.empty();
      if (e.poll_uploads(r.clip.get(), block) < 0) return -1;
      waited = waited || block;
      if (r.clip->pushed == r.nframes) r.clip->finished = true;
    }
    return 0;
  };
  if (land(false)) return fail_srv(s, e.status, e.message);
  // every wave costs a host round trip: while copies are still landing and no
  // detector waits for pairs, let at least kMinWave new frames (over all clips)
  // accumulate before launching
  constexpr int kMinWave = 1024;
  for (;;) {
    int fresh = 0, pending = 0;
    bool copying = false;
    for (va::Clip* c : e.clips) {
      fresh += c->pushed - c->pyr_done;
      pending += (int)c->pending.size();
      copying = copying || !c->up_chunks.empty();
    }
    if (!copying || pending > 0 || fresh >= kMinWave) break;
    if (land(true)) return fail_srv(s, e.status, e.message);
  }
  int rc = e.wave();
  if (rc < 0 || e.status) return fail_srv(s, e.status ? e.status : rc, e.message);
  bool in_flight = false;
  for (auto& kv : s->reqs)
    if (kv.second.admitted && !kv.second.done && !kv.second.clip->up_chunks.empty()) in_flight = true;
  if (rc == 0 && in_flight && land(true)) return fail_srv(s, e.status, e.message);   // nothing to compute yet
  // retire finished clips
  int n_active = (int)s->queue.size();
  for (auto& kv : s->reqs) {
    server::Req& r = kv.second;
    if (!r.admitted || r.done) continue;
    if (r.clip->done()) {
      va::build_results(*r.clip, r.res);
      r.t_done = r.clip->t_done > 0 ? r.clip->t_done : va::now_seconds();
      e.remove_clip(r.clip.get());
      s->used -= r.bytes;
      r.done = true;
      r.clip->store.map.clear();
    } else {
      n_active++;
      if (rc == 0 && !in_flight && r.uploaded == r.nframes && r.clip->pushed == r.nframes && r.clip->pending.empty())
        return fail_srv(s, ANALYSER_ERR_STATE, "a served clip stalled");
    }
  }
  if (active) *active = n_active;
  return ANALYSER_OK;
}

int server_drain(server* s) {
  if (!s) return ANALYSER_ERR_INVALID_ARG;
  for (;;) {
    int active = 0;
    const int rc = server_step(s, &active);
    if (rc) return rc;
    if (active == 0) return ANALYSER_OK;
  }
}

int server_poll(server* s, long long ticket, analyser_results_t* out) {
  if (!s || !out) return ANALYSER_ERR_INVALID_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return ANALYSER_ERR_INVALID_ARG;
  if (s->status) return s->status;
  if (!it->second.done) return ANALYSER_PENDING;
  *out = it->second.res.r;
  return ANALYSER_OK;
}

int server_profile(const server* s, analyser_profile_t* out) {
  if (!s || !out) return ANALYSER_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (s->eng) s->eng->profile(out);
  return ANALYSER_OK;
}

int server_latency(const server* s, long long ticket, double* seconds) {
  if (!s || !seconds) return ANALYSER_ERR_INVALID_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return ANALYSER_ERR_INVALID_ARG;
  if (!it->second.done) return ANALYSER_PENDING;
  *seconds = it->second.t_done - it->second.t_submit;
  return ANALYSER_OK;
}

int server_release(server* s, long long ticket) {
  if (!s) return ANALYSER_ERR_INVALID_ARG;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || !it->second.done) return ANALYSER_ERR_STATE;
  s->reqs.erase(it);
  return ANALYSER_OK;
}

void server_destroy(server* s) {
  if (!s) return;
  if (s->eng) {
    for (auto& kv : s->reqs)
      if (kv.second.admitted && !kv.second.done) s->eng->remove_clip(kv.second.clip.get());
  }
  delete s;
}

}  // extern "C"
