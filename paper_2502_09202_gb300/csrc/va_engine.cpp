// Runtime of the analyser (see va_engine.h).
#include "va_engine.h"
#include "va_pool.h"

#include <algorithm>
#include <cmath>
#include <chrono>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

namespace va {

#define VA_CUDA_TRY(call, why)                                                        \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      why = std::string(#call) + ": " + cudaGetErrorString(e_);                       \
      return ANALYSER_ERR_CUDA;                                                       \
    }                                                                                 \
  } while (0)

double now_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
static inline size_t round_up_sz(size_t v, size_t m) { return (v + m - 1) / m * m; }

// floor(sqrt(n)), digit-by-digit (binary restoring) method
static uint64_t isqrt_digits(uint64_t n) {
  uint64_t res = 0, bit = 1ull << 62;
  while (bit > n) bit >>= 2;
  while (bit) {
    if (n >= res + bit) {
      n -= res + bit;
      res = (res >> 1) + bit;
    } else {
      res >>= 1;
    }
    bit >>= 2;
  }
  return res;
}

// Q(k) = floor(sqrt(k) * 2^16) = isqrt(k * 2^32), k = 0..qmax
static void build_qtab(uint32_t* q, int qmax) {
  for (int k = 0; k <= qmax; k++) q[k] = (uint32_t)isqrt_digits((uint64_t)k << 32);
}

// Statistics of a frame's 256-bin histogram (n pixels): exact integer sums
// S1, S2, then mean = S1/n and std = sqrt((n*S2 - S1^2) / (n*n)) in FP64 with
// that operation order; lower median and lower median of |v - median|.
static void hist_stats(const uint32_t* bins, int64_t n, analyser_frame_hist& h) {
  int64_t s1 = 0, s2 = 0;
  for (int v = 0; v < 256; v++) {
    h.bins[v] = bins[v];
    s1 += (int64_t)v * bins[v];
    s2 += (int64_t)v * v * bins[v];
  }
  h.mean = (double)s1 / (double)n;
  h.std = std::sqrt((double)(n * s2 - s1 * s1) / ((double)n * (double)n));
  const int64_t k = (n - 1) / 2;   // index of the lower median in sorted order
  int64_t c = 0;
  int med = 255;
  for (int v = 0; v < 256; v++) {
    c += bins[v];
    if (c > k) { med = v; break; }
  }
  c = 0;
  int mad = 255;
  for (int d = 0; d < 256; d++) {
    const int64_t cnt = d == 0 ? bins[med]
                               : (int64_t)(med + d < 256 ? bins[med + d] : 0) + (med - d >= 0 ? bins[med - d] : 0);
    c += cnt;
    if (c > k) { mad = d; break; }
  }
  h.median = med;
  h.mad = mad;
}

int min_window(const analyser_params& p) {
  // frames a deep check at t can still touch: t - kmax .. t + kmax + steady_span + steady_frames,
  // and the oldest frame kept for the next check
  return 2 * p.kmax + p.steady_span + p.steady_frames + 4;
}

int validate_params(const analyser_params& p, std::string& why) {
  if (p.levels < 2 || p.levels > 3) { why = "levels must be 2 or 3"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.block != (kCoarseSide << (p.levels - 1))) {
    why = "block must equal 4 << (levels-1)";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.radius_coarse != 8 && p.radius_coarse != 16 && p.radius_coarse != 24) {
    why = "radius_coarse must be 8, 16 or 24";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.radius_refine < 0 || p.radius_refine > 4) { why = "radius_refine must be 0..4"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.mv_cost < 0 || p.mv_cost > 64) { why = "mv_cost must be 0..64"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.kmax < 1 || p.kmax > 16) { why = "kmax must be 1..16"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.jback < 1 || p.jback > 64) { why = "jback must be 1..64"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.fast_window < 1 || p.fast_window > 1024) { why = "fast_window must be 1..1024"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.samp_max_frames < 0 || p.samp_max_frames > 100000) { why = "samp_max_frames out of range"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.steady_frames < 1 || p.steady_frames > 64 || p.steady_span < 1 || p.steady_span > 8) {
    why = "steady_frames must be 1..64 and steady_span 1..8";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.rep_probe < 0 || p.rep_probe > 100000) { why = "rep_probe out of range"; return ANALYSER_ERR_INVALID_ARG; }
  if (p.prefetch_frames < 0 || p.prefetch_frames > 1000000) {
    why = "prefetch_frames out of range";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (!(p.fast_lambda >= 0) || !(p.fast_rise >= 0) || !(p.fast_tau >= 0) || !(p.deep_rho >= 0) || !(p.deep_tau >= 0) ||
      !(p.done_eps >= 0) || !(p.steady_gamma >= 0) || !(p.lag_rho >= 0) || !(p.blend_ratio >= 0) ||
      !(p.pd_rho >= 0) || !(p.pd_gamma_new >= 0) || !(p.pd_gamma_old >= 0) || !(p.rep_ratio >= 0) ||
      !(p.static_amm_px >= 0) || !(p.comb_ratio >= 0) || !(p.unequal_ratio >= 0) || !(p.pulldown_match >= 0) ||
      !(p.kf_theta >= 0) || !(p.wait_timeout_ms >= 0)) {
    why = "thresholds must be non-negative numbers";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if ((p.tile_x || p.tile_y) && !pair_tile_supported(p.radius_coarse, p.tile_x, p.tile_y)) {
    why = "tile_x x tile_y is not a compiled tile shape";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.want_histogram < 0 || p.want_histogram > 1) {
    why = "want_histogram must be 0 or 1";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.kernel_mode < 0 || p.kernel_mode > 1) {
    why = "kernel_mode must be 0 (split kernels for the default estimator) or 1 (fused kernel)";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.step_frames < 0) {
    why = "step_frames must be >= 0";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (p.window_frames != 0 && p.window_frames < min_window(p)) {
    why = "window_frames must be 0 (auto) or >= 2*kmax + steady_span + steady_frames + 4";
    return ANALYSER_ERR_INVALID_ARG;
  }
  return ANALYSER_OK;
}

int validate_size(int width, int height, const analyser_params& p, std::string& why) {
  (void)p;
  if (width < 64 || height < 64) { why = "width and height must be >= 64"; return ANALYSER_ERR_INVALID_ARG; }
  if (height % 2) { why = "height must be even (two equal fields)"; return ANALYSER_ERR_INVALID_ARG; }
  if ((long long)width * height > 11800000LL) {
    why = "width*height must be <= 11,800,000 (exact 64-bit correlation sums)";
    return ANALYSER_ERR_INVALID_ARG;
  }
  return ANALYSER_OK;
}

void Geometry::init(int width, int height, int levels, bool own_l0) {
  W = width; H = height; L = levels; B0 = kCoarseSide << (levels - 1);
  fw[0] = W; fh[0] = H; fp[0] = round_up(W, 64);
  gw[0] = W; gh[0] = H / 2; gp[0] = 2 * fp[0];
  for (int l = 1; l < L; l++) {
    fw[l] = fw[l - 1] / 2; fh[l] = fh[l - 1] / 2; fp[l] = round_up(std::max(fw[l], 4), 16);
    gw[l] = gw[l - 1] / 2; gh[l] = gh[l - 1] / 2; gp[l] = round_up(std::max(gw[l], 4), 16);
  }
  // level 0 of the slots is one contiguous array of frames (H * fp[0] bytes
  // apart), so a run of consecutive slots is a single copy target; the pyramid
  // levels of a slot follow in a second array
  l0_bytes = own_l0 ? (size_t)fh[0] * fp[0] : 0;
  size_t off = 0;
  for (int l = 1; l < L; l++) { off_f[l] = off; off += round_up_sz((size_t)fh[l] * fp[l] + 16, 256); }
  for (int l = 1; l < L; l++) { off_u[l] = off; off += round_up_sz((size_t)gh[l] * gp[l] + 16, 256); }
  for (int l = 1; l < L; l++) { off_l[l] = off; off += round_up_sz((size_t)gh[l] * gp[l] + 16, 256); }
  slot_bytes = round_up_sz(off, 256);
}

size_t Geometry::l0_region(int cap) const { return l0_bytes ? round_up_sz((size_t)cap * l0_bytes + 64, 256) : 0; }

Engine::Engine(const analyser_params& params) : p(params) {}

Engine::~Engine() {
  // nothing may still run on the engine's streams when their buffers return to the cache
  if (stream) cudaStreamSynchronize(stream);
  if (cstream) cudaStreamSynchronize(cstream);
  if (rstream) cudaStreamSynchronize(rstream);
  for (Clip* c : clips) {
    for (auto& u : c->up_chunks) pool_release_event(u.second);
    c->up_chunks.clear();
    pool_free(c->d_ring);
    pool_free(c->d_hist);
  }
  pool_free(d_status);
  pool_free_host(h_status);
  pool_free(d_pjobs);
  pool_free_host(h_pjobs);
  pool_free(d_djobs);
  pool_free_host(h_djobs);
  pool_free(d_pyjobs);
  pool_free_host(h_pyjobs);
  pool_free_host(h_hist);
  pool_free(d_rec);
  pool_free_host(h_rec);
  pool_free(d_vec);
  pool_free(d_cvec);
  for (cudaEvent_t& e : ev_) pool_release_event(e);
  pool_release_event(ev_chunk_);
  pool_release_event(ev_join_);
  pool_release_event(ev_wait_);
  pool_release_stream(rstream);
  pool_release_stream(cstream);
  pool_release_stream(stream);
}

void Engine::profile(analyser_profile_t* out) const {
  out->pairs = n_pairs;
  out->waves = n_waves;
  out->launches = n_launches;
  out->pair_launches = n_pair_launches;
  out->pyramid_launches = n_pyr_launches;
  out->pair_kernel_ms = pair_ms;
  out->pyramid_kernel_ms = pyr_ms;
  out->absdiff_ops = absdiff_ops;
  out->pyramid_bytes = pyr_bytes;
  out->h2d_bytes = h2d_bytes;
  out->d2h_bytes = d2h_bytes;
  out->host_gather_ms = host_gather_ms;
  out->host_wait_ms = host_wait_ms;
  out->host_results_ms = host_results_ms;
  out->host_setup_ms = host_setup_ms;
  out->host_copy_wait_ms = host_copy_wait_ms;
}

int Engine::init(std::string& why) {
  int rc = validate_params(p, why);
  if (rc) return rc;
  VA_CUDA_TRY(cudaSetDevice(p.device), why);
  VA_CUDA_TRY(pool_stream(&stream), why);
  VA_CUDA_TRY(pool_stream(&cstream), why);
  VA_CUDA_TRY(pool_stream(&rstream), why);
  VA_CUDA_TRY(pool_event(&ev_chunk_, false), why);
  VA_CUDA_TRY(pool_event(&ev_join_, false), why);
  VA_CUDA_TRY(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, p.device), why);
  // Q(k) = floor(sqrt(k) * 2^16) for every k = vx^2 + vy^2 the search can produce
  int vmax = p.radius_coarse;
  for (int l = p.levels - 2; l >= 0; l--) vmax = 2 * vmax + p.radius_refine;
  qmax = 2 * vmax * vmax;
  VA_CUDA_TRY(pool_qtab(qmax, build_qtab, &d_qtab), why);
  VA_CUDA_TRY(pool_malloc(reinterpret_cast<void**>(&d_status), sizeof(int)), why);
  VA_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), stream), why);
  VA_CUDA_TRY(pool_malloc_host(reinterpret_cast<void**>(&h_status), sizeof(int)), why);
  for (cudaEvent_t& ev : ev_) VA_CUDA_TRY(pool_event(&ev, true), why);
  return ANALYSER_OK;
}

size_t Engine::ring_bytes(const Geometry& g, int cap) { return g.l0_region(cap) + (size_t)cap * g.slot_bytes; }

int Engine::add_clip(Clip* c, std::string& why, bool enlist) {
  c->p = p;
  c->want_vec_ = c->want_vec_ || (!c->stateless_ && p.want_motion);
  c->geo.init(c->geo.W, c->geo.H, p.levels, !c->external_l0);
  if (c->cap <= 0) c->cap = p.window_frames > 0 ? p.window_frames : std::max(96, min_window(p) + 2);
  c->l0.assign(c->cap, nullptr);
  c->l0_pitch.assign(c->cap, 0);
  const size_t bytes = ring_bytes(c->geo, c->cap);
  if (p.mem_budget_bytes && bytes > p.mem_budget_bytes) {
    why = "rolling window exceeds mem_budget_bytes";
    return ANALYSER_ERR_OOM;
  }
  cudaError_t e = pool_malloc(reinterpret_cast<void**>(&c->d_ring), bytes);
  if (e != cudaSuccess) {
    why = std::string("cudaMalloc(window): ") + cudaGetErrorString(e);
    return ANALYSER_ERR_OOM;
  }
  if (p.want_histogram && !c->stateless_) {
    e = pool_malloc(reinterpret_cast<void**>(&c->d_hist), sizeof(uint32_t) * 256 * c->cap);
    if (e != cudaSuccess) {
      pool_free(c->d_ring);
      c->d_ring = nullptr;
      why = std::string("cudaMalloc(histograms): ") + cudaGetErrorString(e);
      return ANALYSER_ERR_OOM;
    }
  }
  c->pyr = c->d_ring + c->geo.l0_region(c->cap);
  for (int s = 0; s < c->cap; s++) {
    c->l0[s] = c->geo.l0_bytes ? c->d_ring + (size_t)s * c->geo.l0_bytes : nullptr;
    c->l0_pitch[s] = c->geo.fp[0];
  }
  const int nbx = c->geo.W / c->geo.B0, nby = c->geo.H / c->geo.B0;
  c->det.reset(p, (int64_t)nbx * nby);
  if (p.tile_x > 0) {
    c->tbx = p.tile_x;
    c->tby = p.tile_y;
  } else if (!c->stateless_) {
    choose_tile(c->geo.W, c->geo.H, &c->tbx, &c->tby);
  }
  if (enlist) clips.push_back(c);
  return ANALYSER_OK;
}

void Engine::remove_clip(Clip* c) {
  clips.erase(std::remove(clips.begin(), clips.end(), c), clips.end());
  if (!c->up_chunks.empty()) {
    cudaStreamSynchronize(cstream);
    for (auto& u : c->up_chunks) pool_release_event(u.second);
    c->up_chunks.clear();
  }
  if (c->d_ring) {
    // the window returns to the cache: nothing queued may still read or write
    // it.  The clip's own copies have all landed (its chunk list is empty), and
    // the copy stream's other work is other clips' frames, so only the compute
    // streams are waited for: with many clips in flight, waiting for the copy
    // stream would hold every retirement until all queued frames had landed.
    cudaStreamSynchronize(stream);
    cudaStreamSynchronize(rstream);
    pool_free(c->d_ring);
    c->d_ring = nullptr;
    pool_free(c->d_hist);
    c->d_hist = nullptr;
  }
}

cudaError_t Engine::wait_event(cudaEvent_t ev) {
  if (!(p.wait_timeout_ms > 0)) return cudaEventSynchronize(ev);
  // host watchdog: poll the event against a deadline instead of blocking in the driver
  const double deadline = now_seconds() + 1e-3 * p.wait_timeout_ms;
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) return e;
    cudaGetLastError();
    if (now_seconds() >= deadline) return cudaErrorTimeout;
    std::this_thread::yield();
  }
}

cudaError_t Engine::wait_stream(cudaStream_t st) {
  if (!(p.wait_timeout_ms > 0)) return cudaStreamSynchronize(st);
  if (!ev_wait_) {
    const cudaError_t e = pool_event(&ev_wait_, false);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaEventRecord(ev_wait_, st);
  if (e != cudaSuccess) return e;
  return wait_event(ev_wait_);
}

int Engine::upload_async(Clip* c, const uint8_t* frames, long long pitch, int nframes, int chunk) {
  const Geometry& g = c->geo;
  const int k = std::min(nframes, free_slots(c));
  int i = 0;
  while (i < k) {
    const int f0 = c->uploaded;
    const int s0 = c->slot_of(f0);
    const int run = std::min(std::min(k - i, chunk), c->cap - s0);
    const uint8_t* src = frames + (size_t)i * g.H * pitch;
    uint8_t* dst = c->d_ring + (size_t)s0 * g.l0_bytes;
    const size_t rows = (size_t)run * g.H;
    cudaError_t e = pitch == g.fp[0]
                        ? cudaMemcpyAsync(dst, src, (rows - 1) * (size_t)pitch + g.W, cudaMemcpyHostToDevice, cstream)
                        : cudaMemcpy2DAsync(dst, g.fp[0], src, (size_t)pitch, g.W, rows, cudaMemcpyHostToDevice, cstream);
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = pool_event(&ev, false);
    if (e == cudaSuccess) e = cudaEventRecord(ev, cstream);
    if (e != cudaSuccess) {
      pool_release_event(ev);
      status = ANALYSER_ERR_CUDA;
      message = std::string("cudaMemcpyAsync(frames): ") + cudaGetErrorString(e);
      return -1;
    }
    for (int j = 0; j < run; j++) {
      c->l0[s0 + j] = dst + (size_t)j * g.l0_bytes;
      c->l0_pitch[s0 + j] = g.fp[0];
    }
    c->uploaded += run;
    c->up_chunks.push_back({c->uploaded, ev});
    h2d_bytes += (long long)run * g.W * g.H;
    i += run;
  }
  return k;
}

int Engine::poll_uploads(Clip* c, bool wait) {
  const int before = c->pushed;
  while (!c->up_chunks.empty()) {
    cudaEvent_t ev = c->up_chunks.front().second;
    const bool block = wait && c->pushed == before;
    const double tq = block ? now_seconds() : 0.0;
    cudaError_t e = block ? wait_event(ev) : cudaEventQuery(ev);
    if (block) host_copy_wait_ms += 1e3 * (now_seconds() - tq);
    if (e == cudaErrorNotReady) {
      cudaGetLastError();
      break;
    }
    if (e == cudaErrorTimeout) {
      status = ANALYSER_ERR_TIMEOUT;
      message = "frame copy not complete within wait_timeout_ms";
      return -1;
    }
    if (e != cudaSuccess) {
      status = ANALYSER_ERR_CUDA;
      message = std::string("frame copy: ") + cudaGetErrorString(e);
      return -1;
    }
    c->pushed = c->up_chunks.front().first;
    pool_release_event(ev);
    c->up_chunks.pop_front();
  }
  return c->pushed - before;
}

int Engine::attach_device(Clip* c, const uint8_t* frames, long long pitch, long long stride, int nframes) {
  const int k = std::min(nframes, free_slots(c));
  for (int i = 0; i < k; i++) {
    const int f = c->pushed + i;
    const int s = c->slot_of(f);
    c->l0[s] = frames + (size_t)i * stride;
    c->l0_pitch[s] = (int)pitch;
  }
  c->external_l0 = true;
  c->pushed += k;
  return k;
}

// Tile choices are a property of the device and the size, shared by every
// engine of the process.
static std::mutex g_tune_mu;
static std::map<std::vector<int>, std::pair<int, int>> g_tune;

void Engine::choose_tile(int width, int height, int* tbx, int* tby) {
  if (!autotune) {   // the default shape, whatever other engines of the process tuned
    *tbx = 8;
    *tby = 4;
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const std::vector<int> gkey = {dev, width, height, p.levels, p.radius_coarse, p.radius_refine};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(gkey);
    if (it != g_tune.end()) {
      *tbx = it->second.first;
      *tby = it->second.second;
      return;
    }
  }
  for (size_t i = 0; i < tune_keys_.size(); i++)
    if (tune_keys_[i] == std::make_pair(width, height)) {
      *tbx = tune_vals_[i].first;
      *tby = tune_vals_[i].second;
      return;
    }
  int bx = 8, by = 4;
  if (autotune && stream) {
    // time every compiled tile shape on a batch of synthetic pairs of this size;
    // the tile changes the schedule only, never the result
    const int B0 = kCoarseSide << (p.levels - 1);
    const int nblk = std::max(1, (width / B0) * (height / B0));
    const int reps = std::max(4, std::min(32, 400000 / nblk + 1));
    const long long pitch = round_up(width, 64);
    const long long stride = pitch * height;
    const int nfr = reps + 1;
    uint8_t* d = nullptr;
    if (cudaMalloc(&d, (size_t)stride * nfr) == cudaSuccess) {
      std::vector<uint8_t> h((size_t)stride * nfr);
      uint32_t st = 12345;
      for (size_t i = 0; i < h.size(); i++) { st = st * 1664525u + 1013904223u; h[i] = (uint8_t)(st >> 24); }
      cudaMemcpy(d, h.data(), h.size(), cudaMemcpyHostToDevice);
      Clip c;
      c.geo.W = width;
      c.geo.H = height;
      c.cap = nfr;
      c.stateless_ = true;
      c.external_l0 = true;
      std::string why;
      if (add_clip(&c, why, false) == ANALYSER_OK) {
        attach_device(&c, d, pitch, stride, nfr);
        const int cand[5][2] = {{8, 4}, {4, 4}, {8, 2}, {16, 2}, {4, 8}};
        double best_s = 1e30, t84 = -1.0;
        for (auto& cd : cand) {
          if (!pair_tile_supported(p.radius_coarse, cd[0], cd[1])) continue;
          c.tbx = cd[0];
          c.tby = cd[1];
          double tsum = 0.0;
          bool ok = true;
          for (int it = 0; it < 3 && ok; it++) {
            c.store.map.clear();
            c.pyr_done = it == 0 ? 0 : c.pushed;
            for (int i = 0; i < reps; i++) c.pending.push_back(pair_key(kFrame, i, i + 1));
            const double t0 = now_seconds();
            if (run_alone(&c) < 0) ok = false;
            const double t1 = now_seconds();
            if (it > 0) tsum += t1 - t0;
          }
          if (ok && tsum < best_s) { best_s = tsum; bx = cd[0]; by = cd[1]; }
          if (ok && cd[0] == 8 && cd[1] == 4) t84 = tsum;
        }
        // the default shape unless another is clearly faster: clips of several
        // sizes then share one launch per wave
        if (t84 > 0.0 && t84 <= 1.03 * best_s) { bx = 8; by = 4; }
        cudaStreamSynchronize(stream);
        pool_free(c.d_ring);
        c.d_ring = nullptr;
      }
      cudaFree(d);
    }
    cudaGetLastError();
    status = ANALYSER_OK;
    message.clear();
  }
  tune_keys_.push_back({width, height});
  tune_vals_.push_back({bx, by});
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[gkey] = {bx, by};
  }
  *tbx = bx;
  *tby = by;
}

int Engine::run_alone(Clip* c) {
  std::vector<Clip*> saved;
  saved.swap(clips);
  clips.push_back(c);
  const int rc = wave();
  clips.swap(saved);
  return status ? status : rc;
}

int Engine::ensure_capacity(int npairs, int ndown, int npyr) {
  std::string why;
  if (npairs > cap_pairs) {
    // no wave is in flight here: the previous buffers are idle
    int nc = std::max(npairs, std::max(256, cap_pairs * 2));
    pool_free(d_pjobs);
    pool_free_host(h_pjobs);
    pool_free(d_rec);
    pool_free_host(h_rec);
    d_pjobs = nullptr; h_pjobs = nullptr; d_rec = nullptr; h_rec = nullptr;
    VA_CUDA_TRY(pool_malloc(reinterpret_cast<void**>(&d_pjobs), sizeof(PairJob) * nc), message);
    VA_CUDA_TRY(pool_malloc_host(reinterpret_cast<void**>(&h_pjobs), sizeof(PairJob) * nc), message);
    VA_CUDA_TRY(pool_malloc(reinterpret_cast<void**>(&d_rec), sizeof(unsigned long long) * kRecWords * nc), message);
    VA_CUDA_TRY(pool_malloc_host(reinterpret_cast<void**>(&h_rec), sizeof(unsigned long long) * kRecWords * nc),
                message);
    cap_pairs = nc;
  }
  if (ndown > cap_down) {
    int nc = std::max(ndown, std::max(256, cap_down * 2));
    pool_free(d_djobs);
    pool_free_host(h_djobs);
    d_djobs = nullptr; h_djobs = nullptr;
    VA_CUDA_TRY(pool_malloc(reinterpret_cast<void**>(&d_djobs), sizeof(DownJob) * nc), message);
    VA_CUDA_TRY(pool_malloc_host(reinterpret_cast<void**>(&h_djobs), sizeof(DownJob) * nc), message);
    cap_down = nc;
  }
  if (npyr > cap_pyr) {
    int nc = std::max(npyr, std::max(256, cap_pyr * 2));
    pool_free(d_pyjobs);
    pool_free_host(h_pyjobs);
    d_pyjobs = nullptr; h_pyjobs = nullptr;
    VA_CUDA_TRY(pool_malloc(reinterpret_cast<void**>(&d_pyjobs), sizeof(PyrJob) * nc), message);
    VA_CUDA_TRY(pool_malloc_host(reinterpret_cast<void**>(&h_pyjobs), sizeof(PyrJob) * nc), message);
    cap_pyr = nc;
  }
  return ANALYSER_OK;
}

int Engine::setup_pair_job(const Clip& c, uint64_t key, PairJob& pj, int item_begin, unsigned long long* rec,
                           short2* vec) {
  const Geometry& g = c.geo;
  const int kind = key_kind(key), a = key_a(key), b = key_b(key);
  const int sa = c.slot_of(a), sb = c.slot_of(b);
  const uint8_t* ra = c.pyr + (size_t)sa * g.slot_bytes;
  const uint8_t* rb = c.pyr + (size_t)sb * g.slot_bytes;
  const uint8_t* la = c.l0[sa];
  const uint8_t* lb = c.l0[sb];
  const int pa = c.l0_pitch[sa], pb = c.l0_pitch[sb];
  if (kind == kFrame) {
    pj.I[0] = {la, pa, g.W, g.H};
    pj.J[0] = {lb, pb, g.W, g.H};
    for (int l = 1; l < g.L; l++) {
      pj.I[l] = {ra + g.off_f[l], g.fp[l], g.fw[l], g.fh[l]};
      pj.J[l] = {rb + g.off_f[l], g.fp[l], g.fw[l], g.fh[l]};
    }
    pj.nbx = g.W / g.B0;
    pj.nby = g.H / g.B0;
  } else {
    // which field of a is I and which field of b is J
    const bool iu = kind == kUpperLower || kind == kUpperUpper;
    const bool ju = kind == kLowerUpper || kind == kUpperUpper;
    // level-0 fields are row-strided views of the frames
    pj.I[0] = {iu ? la : la + pa, 2 * pa, g.W, g.H / 2};
    pj.J[0] = {ju ? lb : lb + pb, 2 * pb, g.W, g.H / 2};
    for (int l = 1; l < g.L; l++) {
      pj.I[l] = {ra + (iu ? g.off_u[l] : g.off_l[l]), g.gp[l], g.gw[l], g.gh[l]};
      pj.J[l] = {rb + (ju ? g.off_u[l] : g.off_l[l]), g.gp[l], g.gw[l], g.gh[l]};
    }
    pj.nbx = g.W / g.B0;
    pj.nby = (g.H / 2) / g.B0;
  }
  pj.tiles_x = (pj.nbx + c.tbx - 1) / c.tbx;
  pj.tiles_y = (pj.nby + c.tby - 1) / c.tby;
  pj.item_begin = item_begin;
  pj.rec = rec;
  pj.vec = vec;
  return pj.tiles_x * pj.tiles_y;
}

int Engine::wave() {
  const int n = wave_launch();
  if (n <= 0) return n;
  return wave_complete();
}

int Engine::wave_launch() {
  if (status) return status;
  if (inflight_) return ANALYSER_ERR_STATE;
  const double tw0 = now_seconds();
  wp_.clear();
  // detectors with nothing queued may be able to move on (new frames, finish)
  for (Clip* c : clips) {
    if (c->status || c->stateless_ || c->done() || !c->pending.empty()) continue;
    std::vector<uint64_t> need;
    c->det.run(c->store, c->pushed, c->finished, need);
    std::sort(need.begin(), need.end());
    need.erase(std::unique(need.begin(), need.end()), need.end());
    c->pending = need;
    if (c->done() && c->t_done < 0) c->t_done = now_seconds();
  }
  // ---- gather ---------------------------------------------------------------
  std::vector<DownJob> down[kMaxLevels];
  pyr_.clear();
  hist_runs_.clear();
  int nhist = 0;
  for (Clip* c : clips) {
    if (c->status || c->done()) continue;
    const Geometry& g = c->geo;
    for (int f = c->pyr_done; f < c->pushed; f++) {
      const int s = c->slot_of(f);
      uint8_t* base = c->pyr + (size_t)s * g.slot_bytes;
      const uint8_t* l0 = c->l0[s];
      const int p0 = c->l0_pitch[s];
      if (g.L < 2) continue;
      // levels 1 and 2 of the frame and both fields from one read of level 0
      PyrJob pj;
      pj.l0 = l0;
      pj.l0_pitch = p0;
      pj.w = g.W;
      pj.h = g.H;
      const bool two = g.L >= 3;
      pj.out[0] = base + g.off_f[1]; pj.pitch[0] = g.fp[1];
      pj.out[2] = base + g.off_u[1]; pj.pitch[2] = g.gp[1];
      pj.out[4] = base + g.off_l[1]; pj.pitch[4] = g.gp[1];
      pj.out[1] = two ? base + g.off_f[2] : nullptr; pj.pitch[1] = two ? g.fp[2] : 0;
      pj.out[3] = two ? base + g.off_u[2] : nullptr; pj.pitch[3] = two ? g.gp[2] : 0;
      pj.out[5] = two ? base + g.off_l[2] : nullptr; pj.pitch[5] = two ? g.gp[2] : 0;
      pj.hist = nullptr;
      if (c->d_hist) {
        pj.hist = c->d_hist + (size_t)256 * s;
        HistRun* last = hist_runs_.empty() ? nullptr : &hist_runs_.back();
        if (last && last->clip == c && last->frame0 + last->n == f && last->slot0 + last->n == s) last->n++;
        else hist_runs_.push_back({c, f, s, 1, nhist});
        nhist++;
      }
      pyr_.push_back(pj);
      for (int l = 3; l < g.L; l++) {
        down[l].push_back({{base + g.off_f[l - 1], g.fp[l - 1], g.fw[l - 1], g.fh[l - 1]}, base + g.off_f[l], g.fp[l]});
        down[l].push_back({{base + g.off_u[l - 1], g.gp[l - 1], g.gw[l - 1], g.gh[l - 1]}, base + g.off_u[l], g.gp[l]});
        down[l].push_back({{base + g.off_l[l - 1], g.gp[l - 1], g.gw[l - 1], g.gh[l - 1]}, base + g.off_l[l], g.gp[l]});
      }
    }
    c->pyr_done = c->pushed;
    auto want = [&](uint64_t k) {
      if (c->store.map.count(k) || c->inflight.count(k)) return;
      c->inflight.insert(k);
      wp_.push_back({c, k, 0, c->tbx, c->tby});
    };
    if (!c->stateless_) {
      for (int t = c->aon_next; t < c->pushed - 1; t++) want(pair_key(kFrame, t, t + 1));
      c->aon_next = std::max(c->aon_next, c->pushed - 1);
    }
    for (uint64_t k : c->pending) want(k);
    c->pending.clear();
  }
  int ndown = 0;
  for (int l = 1; l < kMaxLevels; l++) ndown += (int)down[l].size();
  const int npyr = (int)pyr_.size();
  const int npairs = (int)wp_.size();
  if (npairs == 0 && ndown == 0 && npyr == 0) return 0;
  if (ensure_capacity(npairs, ndown, npyr)) { status = ANALYSER_ERR_CUDA; return status; }

  // ---- pair jobs, grouped by tile shape ---------------------------------------
  std::stable_sort(wp_.begin(), wp_.end(), [](const WavePair& x, const WavePair& y) {
    return x.tbx != y.tbx ? x.tbx < y.tbx : x.tby < y.tby;
  });
  size_t vec_total = 0;
  for (auto& w : wp_) {
    const int kind = key_kind(w.key);
    const bool aon = kind == kFrame && key_b(w.key) == key_a(w.key) + 1;
    const bool dump = w.clip->want_vec_ && (w.clip->stateless_ || aon);
    if (dump) {
      const Geometry& g = w.clip->geo;
      const int h0 = kind == kFrame ? g.H : g.H / 2;
      w.vec_off = vec_total + 1;
      vec_total += (size_t)(g.W / g.B0) * (h0 / g.B0);
    }
  }
  if (vec_total > cap_vec) {
    pool_free(d_vec);
    d_vec = nullptr;
    if (pool_malloc(reinterpret_cast<void**>(&d_vec), sizeof(short2) * vec_total) != cudaSuccess) {
      status = ANALYSER_ERR_OOM; message = "cudaMalloc(motion dump)"; return status;
    }
    cap_vec = vec_total;
  }
  // groups of pairs sharing a tile shape; with the split kernels a group is
  // also a chunk of the wave, so that chunk c's refinement runs beside chunk
  // c+1's coarse search
  const bool split = p.levels == 3 && p.radius_refine == 2 && p.kernel_mode == 0;
  // (four chunks for a large wave; a small one is not worth the launches)
  const int nchunks = split && npairs >= 256 ? std::max(1, max_chunks) : 1;
  const int chunk = split ? (npairs + nchunks - 1) / nchunks : npairs + 1;
  size_t cvec_total = 0;
  for (auto& w : wp_) {
    const Geometry& g = w.clip->geo;
    const int h0 = key_kind(w.key) == kFrame ? g.H : g.H / 2;
    cvec_total += (size_t)(g.W / g.B0) * (h0 / g.B0);
  }
  if (split && cvec_total > cap_cvec) {
    pool_free(d_cvec);
    d_cvec = nullptr;
    if (pool_malloc(reinterpret_cast<void**>(&d_cvec), sizeof(short2) * cvec_total) != cudaSuccess) {
      status = ANALYSER_ERR_OOM; message = "cudaMalloc(coarse vectors)"; return status;
    }
    cap_cvec = cvec_total;
  }
  struct Group { int first, count, items, tbx, tby; };
  std::vector<Group> groups;
  int items = 0;
  size_t cvec_off = 0;
  for (int i = 0; i < npairs; i++) {
    WavePair& w = wp_[i];
    if (groups.empty() || groups.back().tbx != w.tbx || groups.back().tby != w.tby || groups.back().count >= chunk) {
      groups.push_back({i, 0, 0, w.tbx, w.tby});
      items = 0;
    }
    short2* vp = w.vec_off ? d_vec + (w.vec_off - 1) : nullptr;
    const int n = setup_pair_job(*w.clip, w.key, h_pjobs[i], items, d_rec + (size_t)kRecWords * i, vp);
    h_pjobs[i].cvec = split ? d_cvec + cvec_off : nullptr;
    cvec_off += (size_t)h_pjobs[i].nbx * h_pjobs[i].nby;
    items += n;
    groups.back().count++;
    groups.back().items = items;
  }
  int di = 0;
  int dstart[kMaxLevels] = {0}, dcount[kMaxLevels] = {0}, dmaxh[kMaxLevels] = {0}, dmaxw[kMaxLevels] = {0};
  for (int l = 1; l < kMaxLevels; l++) {
    dstart[l] = di;
    for (const DownJob& j : down[l]) {
      h_djobs[di++] = j;
      dmaxh[l] = std::max(dmaxh[l], j.src.h / 2);
      dmaxw[l] = std::max(dmaxw[l], j.src.w / 2);
    }
    dcount[l] = (int)down[l].size();
  }

  // ---- launch -----------------------------------------------------------------
  const double tw1 = now_seconds();
  host_gather_ms += 1e3 * (tw1 - tw0);
  std::string& why = message;
  auto fail = [&](cudaError_t e, const char* what) {
    status = ANALYSER_ERR_CUDA;
    message = std::string(what) + ": " + cudaGetErrorString(e);
    return status;
  };
  cudaError_t e;
  (void)why;
  if (npairs) {
    // descriptors are read from page-locked memory by a kernel, not queued on a copy engine
    e = launch_copy_words(h_pjobs, d_pjobs, sizeof(PairJob) * npairs, stream);
    if (e) return fail(e, "copy(pair jobs)");
    n_launches++;
    e = cudaMemsetAsync(d_rec, 0, sizeof(unsigned long long) * kRecWords * npairs, stream);
    if (e) return fail(e, "cudaMemsetAsync(records)");
  }
  if (ndown) {
    e = launch_copy_words(h_djobs, d_djobs, sizeof(DownJob) * ndown, stream);
    if (e) return fail(e, "copy(pyramid jobs)");
    n_launches++;
  }
  int pmaxw = 0, pmaxh = 0;
  if (npyr) {
    for (int i = 0; i < npyr; i++) {
      h_pyjobs[i] = pyr_[i];
      pmaxw = std::max(pmaxw, pyr_[i].w);
      pmaxh = std::max(pmaxh, pyr_[i].h);
    }
    e = launch_copy_words(h_pyjobs, d_pyjobs, sizeof(PyrJob) * npyr, stream);
    if (e) return fail(e, "copy(pyramid jobs)");
    n_launches++;
  }
  // per-frame histograms: zero the new frames' bins (one run of consecutive slots at a time)
  if (nhist > cap_hist) {
    pool_free_host(h_hist);
    h_hist = nullptr;
    cap_hist = 0;
    e = pool_malloc_host(reinterpret_cast<void**>(&h_hist), sizeof(uint32_t) * 256 * std::max(nhist, 64));
    if (e) return fail(e, "cudaMallocHost(histograms)");
    cap_hist = std::max(nhist, 64);
  }
  for (const HistRun& r : hist_runs_) {
    e = cudaMemsetAsync(r.clip->d_hist + (size_t)256 * r.slot0, 0, sizeof(uint32_t) * 256 * r.n, stream);
    if (e) return fail(e, "cudaMemsetAsync(histograms)");
  }
  const bool timed = p.time_kernels != 0;
  if (timed && (ndown || npyr)) cudaEventRecord(ev_[0], stream);
  if (npyr) {
    e = launch_pyramid(d_pyjobs, npyr, pmaxw, pmaxh, nhist > 0, stream);
    if (e) return fail(e, "pyramid_kernel");
    n_launches += nhist > 0 ? 2 : 1;
    n_pyr_launches++;
    for (const HistRun& r : hist_runs_) {
      e = launch_copy_words(r.clip->d_hist + (size_t)256 * r.slot0, h_hist + (size_t)256 * r.off,
                            sizeof(uint32_t) * 256 * r.n, stream);
      if (e) return fail(e, "copy(histograms)");
      n_launches++;
    }
    for (const PyrJob& j : pyr_) {
      // read level 0 once, write levels 1-2 of the frame and both fields
      double b = (double)j.w * j.h + (double)(j.w / 2) * (j.h / 2) + 2.0 * (j.w / 2) * (j.h / 4);
      if (j.out[1]) b += (double)(j.w / 4) * (j.h / 4) + 2.0 * (j.w / 4) * (j.h / 8);
      pyr_bytes += b;
    }
  }
  for (int l = 1; l < kMaxLevels; l++) {
    if (!dcount[l]) continue;
    e = launch_downsample(d_djobs + dstart[l], dcount[l], dmaxh[l], dmaxw[l], stream);
    if (e) return fail(e, "downsample_kernel");
    n_launches++;
    n_pyr_launches++;
    for (const DownJob& j : down[l]) pyr_bytes += 2.0 * (j.src.h / 2) * (double)(2 * (j.src.w / 2)) * 1.25;
  }
  if (timed && (ndown || npyr)) cudaEventRecord(ev_[1], stream);
  if (timed && !groups.empty()) cudaEventRecord(ev_[2], stream);
  for (const Group& gr : groups) {
    PairBatch b;
    b.jobs = d_pjobs + gr.first;
    b.njobs = gr.count;
    b.nitems = gr.items;
    b.qtab = d_qtab;
    b.qmax = qmax;
    b.cfg = {p.levels, p.radius_coarse, p.radius_refine, p.mv_cost};
    b.status = d_status;
    if (split) {
      // coarse search on the main stream, refinement + sums on the second one
      e = launch_coarse(b, gr.tbx, gr.tby, stream);
      if (e) return fail(e, "coarse_kernel");
      e = cudaEventRecord(ev_chunk_, stream);
      if (!e) e = cudaStreamWaitEvent(rstream, ev_chunk_, 0);
      if (e) return fail(e, "cudaStreamWaitEvent(chunk)");
      e = launch_refine(b, gr.tbx, gr.tby, rstream);
      if (e) return fail(e, "refine_kernel");
      n_launches += 2;
      n_pair_launches += 2;
    } else {
      const int per_sm = pair_blocks_per_sm(p.radius_coarse, gr.tbx, gr.tby);
      const int grid = std::max(1, std::min(gr.items, sm_count * std::max(per_sm, 1)));
      e = launch_pairs(b, gr.tbx, gr.tby, grid, stream);
      if (e) return fail(e, "pair_kernel");
      n_launches++;
      n_pair_launches++;
    }
  }
  if (split && !groups.empty()) {
    e = cudaEventRecord(ev_join_, rstream);
    if (!e) e = cudaStreamWaitEvent(stream, ev_join_, 0);
    if (e) return fail(e, "cudaStreamWaitEvent(join)");
  }
  if (timed && !groups.empty()) cudaEventRecord(ev_[3], stream);
  if (npairs) {
    e = launch_copy_words(d_rec, h_rec, sizeof(unsigned long long) * kRecWords * npairs, stream);
    if (e) return fail(e, "copy(records)");
    n_launches++;
    if (vec_total) {
      h_vec.resize(vec_total);
      e = cudaMemcpyAsync(h_vec.data(), d_vec, sizeof(short2) * vec_total, cudaMemcpyDeviceToHost, stream);
      if (e) return fail(e, "cudaMemcpyAsync(motion)");
    }
  }
  e = launch_copy_words(d_status, h_status, sizeof(int), stream);
  if (e) return fail(e, "copy(status)");
  n_launches++;
  fl_npairs_ = npairs;
  fl_ndown_ = ndown + npyr;
  fl_vec_total_ = vec_total;
  fl_groups_ = !groups.empty();
  fl_t1_ = tw1;
  inflight_ = true;
  return npairs + ndown + npyr;
}

int Engine::wave_complete() {
  if (!inflight_) return 0;
  inflight_ = false;
  const int npairs = fl_npairs_, ndown = fl_ndown_;
  const size_t vec_total = fl_vec_total_;
  const bool any_groups = fl_groups_;
  const double tw1 = fl_t1_;
  const bool timed = p.time_kernels != 0;
  auto fail = [&](cudaError_t e, const char* what) {
    status = ANALYSER_ERR_CUDA;
    message = std::string(what) + ": " + cudaGetErrorString(e);
    return status;
  };
  cudaError_t e;
  const double tw2 = now_seconds();
  e = wait_stream(stream);
  if (e == cudaErrorTimeout) {
    status = ANALYSER_ERR_TIMEOUT;
    message = "wave not complete within wait_timeout_ms";
    return status;
  }
  if (e) return fail(e, "cudaStreamSynchronize(wave)");
  const double tw3 = now_seconds();
  host_wait_ms += 1e3 * (tw3 - tw2);
  host_gather_ms += 1e3 * (tw2 - tw1);
  const int dev_status = *h_status;
  h2d_bytes += (long long)(sizeof(PairJob) * npairs + sizeof(DownJob) * ndown);
  d2h_bytes += (long long)(sizeof(unsigned long long) * kRecWords * npairs + sizeof(short2) * vec_total + sizeof(int));
  if (timed) {
    float ms = 0.f;
    if (ndown && cudaEventElapsedTime(&ms, ev_[0], ev_[1]) == cudaSuccess) pyr_ms += ms;
    if (any_groups && cudaEventElapsedTime(&ms, ev_[2], ev_[3]) == cudaSuccess) pair_ms += ms;
  }
  // algorithmic block-search work: |a-b| accumulates per block over all levels
  {
    const int L = p.levels, B0 = kCoarseSide << (L - 1);
    const double cw = (double)(2 * p.radius_coarse + 1) * (2 * p.radius_coarse + 1);
    const double rw = (double)(2 * p.radius_refine + 1) * (2 * p.radius_refine + 1);
    double per_block = kCoarseSide * kCoarseSide * cw;
    for (int l = L - 2; l >= 0; l--) per_block += (double)(B0 >> l) * (B0 >> l) * rw;
    for (int i = 0; i < npairs; i++) absdiff_ops += per_block * h_pjobs[i].nbx * h_pjobs[i].nby;
  }
  if (dev_status) {
    status = ANALYSER_ERR_CUDA;
    message = "device-side check failed in pair_kernel (motion vector outside the AMM table)";
    return status;
  }
  n_waves++;
  n_pairs += npairs;

  // ---- results ------------------------------------------------------------------
  for (int i = 0; i < npairs; i++) {
    WavePair& w = wp_[i];
    Clip* c = w.clip;
    Measure m;
    for (int k = 0; k < kRecWords; k++) m.s[k] = (int64_t)h_rec[(size_t)kRecWords * i + k];
    const Geometry& g = c->geo;
    const int kind = key_kind(w.key);
    const int h0 = kind == kFrame ? g.H : g.H / 2;
    m.n = (int64_t)g.W * h0;
    m.nb = (int64_t)(g.W / g.B0) * (h0 / g.B0);
    m.used = kind == kFrame && key_b(w.key) == key_a(w.key) + 1;
    finalise_measure(m);
    c->store.map[w.key] = m;
    c->inflight.erase(w.key);
    if (w.vec_off) {
      const int a = key_a(w.key);
      const size_t nbk = (size_t)(g.W / g.B0) * (h0 / g.B0);
      if (c->stateless_) {
        c->vec_out_.push_back({w.key, std::vector<short2>(h_vec.begin() + (w.vec_off - 1),
                                                         h_vec.begin() + (w.vec_off - 1) + nbk)});
      } else if (key_b(w.key) == a + 1) {
        if (c->motion.size() < (size_t)(a + 1) * nbk * 2) c->motion.resize((size_t)(a + 1) * nbk * 2, 0);
        for (size_t q = 0; q < nbk; q++) {
          c->motion[(size_t)a * nbk * 2 + 2 * q] = h_vec[w.vec_off - 1 + q].x;
          c->motion[(size_t)a * nbk * 2 + 2 * q + 1] = h_vec[w.vec_off - 1 + q].y;
        }
      }
    }
  }
  // ---- per-frame histograms ---------------------------------------------------------------
  for (const HistRun& r : hist_runs_) {
    Clip* c = r.clip;
    if ((int)c->hist.size() < r.frame0 + r.n) c->hist.resize(r.frame0 + r.n);
    for (int i = 0; i < r.n; i++) {
      analyser_frame_hist& h = c->hist[r.frame0 + i];
      h.frame = r.frame0 + i;
      hist_stats(h_hist + (size_t)256 * (r.off + i), (int64_t)c->geo.W * c->geo.H, h);
    }
  }
  // ---- detectors and eviction ---------------------------------------------------------
  for (Clip* c : clips) {
    if (c->status || c->stateless_ || c->done()) continue;
    std::vector<uint64_t> need;
    c->det.run(c->store, c->pushed, c->finished, need);
    std::sort(need.begin(), need.end());
    need.erase(std::unique(need.begin(), need.end()), need.end());
    c->pending = need;
    if (c->done() && c->t_done < 0) c->t_done = now_seconds();
    const int keep = std::min(c->det.keep_from(), c->aon_next);
    if (c->done()) c->evicted = c->pushed;
    else c->evicted = std::max(c->evicted, std::min(keep, c->pushed));
  }
  host_results_ms += 1e3 * (now_seconds() - tw3);
  return npairs + ndown;
}

int Engine::measure_pairs(int width, int height, const uint8_t* frames, long long pitch, long long stride,
                          int nframes, const int* kinds, const int* ia, const int* ib, int npairs, int64_t* records,
                          int16_t* motion, cudaStream_t st, std::string& why) {
  int rc = validate_size(width, height, p, why);
  if (rc) return rc;
  if (!frames || nframes <= 0 || npairs < 0 || (npairs && (!kinds || !ia || !ib || !records))) {
    why = "null pointer or empty frame set";
    return ANALYSER_ERR_INVALID_ARG;
  }
  if (pitch < width || pitch % 16 || pitch > INT_MAX / 2 || ((uintptr_t)frames % 16) || stride % 16 ||
      stride < pitch * height) {
    why = "device frames need 16-byte aligned base, pitch and stride, width <= pitch <= INT_MAX/2";
    return ANALYSER_ERR_INVALID_ARG;
  }
  for (int i = 0; i < npairs; i++) {
    if (kinds[i] < 0 || kinds[i] >= kPairKinds || ia[i] < 0 || ib[i] < 0 || ia[i] >= nframes || ib[i] >= nframes) {
      why = "pair index or kind out of range";
      return ANALYSER_ERR_INVALID_ARG;
    }
  }
  Clip c;
  c.geo.W = width;
  c.geo.H = height;
  c.cap = nframes;
  c.stateless_ = true;
  c.external_l0 = true;
  c.want_vec_ = motion != nullptr;
  cudaStream_t saved = stream;
  if (st) stream = st;
  rc = add_clip(&c, why, false);
  if (rc) { stream = saved; return rc; }
  attach_device(&c, frames, pitch, stride, nframes);
  for (int i = 0; i < npairs; i++) c.pending.push_back(pair_key(kinds[i], ia[i], ib[i]));
  rc = run_alone(&c);
  if (c.d_ring) {
    cudaStreamSynchronize(stream);
    pool_free(c.d_ring);
    c.d_ring = nullptr;
  }
  stream = saved;
  if (rc < 0 || status) {
    why = message;
    int s = status ? status : rc;
    status = ANALYSER_OK;
    return s;
  }
  const int nbk = (width / c.geo.B0) * (height / c.geo.B0);
  const int nbk_f = (width / c.geo.B0) * ((height / 2) / c.geo.B0);
  size_t moff = 0;
  for (int i = 0; i < npairs; i++) {
    const uint64_t k = pair_key(kinds[i], ia[i], ib[i]);
    Measure* m = c.store.find(kinds[i], ia[i], ib[i]);
    for (int w = 0; w < kRecWords; w++) records[(size_t)kRecWords * i + w] = m->s[w];
    if (motion) {
      const int nb_here = kinds[i] == kFrame ? nbk : nbk_f;
      for (auto& vo : c.vec_out_)
        if (vo.first == k) {
          for (int q = 0; q < nb_here && q < (int)vo.second.size(); q++) {
            motion[moff + 2 * q] = vo.second[q].x;
            motion[moff + 2 * q + 1] = vo.second[q].y;
          }
          break;
        }
      moff += (size_t)2 * nb_here;
    }
  }
  return ANALYSER_OK;
}

void build_results(const Clip& c, ResultsBuf& out) {
  const Detector& d = c.det;
  out.cuts = d.cuts;
  out.dissolves = d.dissolves;
  out.keyframes = d.keyframes;
  out.shots.clear();
  for (const ShotOut& s : d.shots)
    out.shots.push_back({s.first, s.last, s.label, s.field_order, s.phase, s.analysed});
  std::map<uint64_t, const Measure*> ordered;
  for (auto& kv : c.store.map)
    if (kv.second.used) ordered[kv.first] = &kv.second;
  out.measures.clear();
  for (auto& kv : ordered) {
    const Measure& m = *kv.second;
    analyser_measure am;
    am.kind = key_kind(kv.first);
    am.a = key_a(kv.first);
    am.b = key_b(kv.first);
    am.si = m.s[0]; am.sj = m.s[1]; am.sii = m.s[2]; am.sjj = m.s[3]; am.sij = m.s[4]; am.sabs = m.s[5];
    am.samm = m.s[6];
    am.n = m.n; am.nb = m.nb;
    am.ncc = m.ncc; am.swr = m.swr; am.amm = m.amm; am.act = m.act;
    out.measures.push_back(am);
  }
  out.motion = c.motion;
  analyser_results_t& r = out.r;
  std::memset(&r, 0, sizeof(r));
  r.nframes = c.pushed;
  r.ncuts = (int)out.cuts.size(); r.cuts = out.cuts.data();
  r.ndissolves = (int)out.dissolves.size() / 2; r.dissolves = out.dissolves.data();
  r.nshots = (int)out.shots.size(); r.shots = out.shots.data();
  r.label = d.clip_label; r.field_order = d.clip_fo; r.pulldown_phase = d.clip_phase;
  r.nkeyframes = (int)out.keyframes.size(); r.keyframes = out.keyframes.data();
  r.nmeasures = (int)out.measures.size(); r.measures = out.measures.data();
  if (!out.motion.empty()) {
    r.motion_w = c.geo.W / c.geo.B0;
    r.motion_h = c.geo.H / c.geo.B0;
    r.motion = out.motion.data();
  }
  out.hist = c.hist;
  r.nhist = (int)out.hist.size();
  r.hist = out.hist.empty() ? nullptr : out.hist.data();
}

}  // namespace va
