/*
 * analyser.h -- C ABI of the GB300 video analyser (shot boundaries, sampling
 * structure, dynamic keyframes) of arXiv 2502.09202.
 *
 * The library computes the paper's per-frame measures on the GPU and runs its
 * detectors on the host:
 *   AMM(I,J)  average magnitude of the motion field between I and J   (Sec. III.A)
 *   SWR(I,J)  dissimilarity 1 - NCC of I and motion-compensated J      (Sec. III.A)
 *   ACT(I,J)  geometric mean sqrt(AMM * SWR)                           (Sec. III.A)
 *   ACT(I_t, I_t+1) for every t; every other measure on demand          (Sec. III.A)
 *   shot boundaries: fast check, then a deep check for K = 1..Kmax      (Sec. III.B)
 *   sampling structure from v0 = ACT(u_t,l_t), v1 = ACT(u_t,l_t+1),
 *     v2 = ACT(l_t,u_t+1), field order from beta = v1/v2                (Sec. III.C)
 *   dynamic keyframes by accumulated activity                           (Sec. III.D)
 *
 * Conventions for every call:
 *   - plain C types; every call that can fail returns an int status
 *     (ANALYSER_OK or a negative error code) and never throws or aborts;
 *   - errors are sticky per handle: after a failure the handle refuses further
 *     work with the same code (analyser_last_error reports it);
 *   - frames are 8-bit luma planes, row-major, `pitch_bytes` between rows;
 *   - "device" pointers are CUDA device pointers of the current device.
 */
#ifndef GB300_VIDEO_ANALYSER_H
#define GB300_VIDEO_ANALYSER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define ANALYSER_OK 0
#define ANALYSER_ERR_INVALID_ARG (-1) /* null pointer, bad size/pitch, unsupported parameters */
#define ANALYSER_ERR_OOM (-2)         /* device or host allocation failed, or budget exceeded */
#define ANALYSER_ERR_CUDA (-3)        /* a CUDA call failed (the message says which) */
#define ANALYSER_ERR_TIMEOUT (-4)     /* a bounded wait gave up (params.wait_timeout_ms) */
#define ANALYSER_ERR_STATE (-5)       /* call not allowed in this state (e.g. push after finish) */
#define ANALYSER_PENDING 1            /* server_poll: the request is not done yet */

/* ---- labels ---------------------------------------------------------------- */
#define ANALYSER_UNKNOWN 0
#define ANALYSER_PROGRESSIVE 1
#define ANALYSER_INTERLACED 2
#define ANALYSER_PULLDOWN 3
#define ANALYSER_FO_NONE 0
#define ANALYSER_FO_TFF 1 /* upper (even-row) field first */
#define ANALYSER_FO_BFF 2 /* lower (odd-row) field first */

/* ---- pair kinds of a measure record ----------------------------------------- */
#define ANALYSER_PAIR_FRAME 0       /* I = frame a, J = frame b */
#define ANALYSER_PAIR_UPPER_LOWER 1 /* I = upper field of a, J = lower field of b */
#define ANALYSER_PAIR_LOWER_UPPER 2 /* I = lower field of a, J = upper field of b */
/* Same-parity field pairs: an extension for repeated-field detection in the
 * spirit of Sec. III.C (the paper measures only v0, v1, v2).  The sampling
 * detector reads them for its voters to find the repeated fields of 3:2
 * pulldown; analyser_measure_pairs and analyser_measure_pair_noalloc take them
 * too. */
#define ANALYSER_PAIR_UPPER_UPPER 3 /* I = upper field of a, J = upper field of b */
#define ANALYSER_PAIR_LOWER_LOWER 4 /* I = lower field of a, J = lower field of b */

/*
 * Parameters.  The paper fixes none of the motion estimator's choices and none
 * of the thresholds (Sec. III); these defaults are the readings the library and
 * its tests use.  Fill with analyser_default_params() and change fields.
 */
typedef struct {
  /* motion estimator: integer block matching on a box-filter pyramid */
  int block;           /* level-0 block side B0 = 4 << (levels-1)          (16) */
  int levels;          /* pyramid depth L, 2 or 3                           (3) */
  int radius_coarse;   /* exhaustive radius R at the coarsest level: 8, 16, 24 (16) */
  int radius_refine;   /* refinement radius r at finer levels, 0..4          (2) */
  int mv_cost;         /* lambda: cost per pixel of |vx|+|vy| added to the SAD, 0..64 (4) */
  /* shot detector (Sec. III.B) */
  int kmax;            /* largest dissolve span K tested, 1..16              (8) */
  int jback;           /* J: predecessors compared in the deep check, and needed
                          in the shot before a fast check                    (2) */
  int fast_window;     /* median window W                                    (8) */
  double fast_lambda;  /* candidate iff a_t > max(fast_tau, fast_lambda*median) (2.0) */
  double fast_rise;    /* ... or a_t > max(fast_tau, fast_rise*median) and a_t < a_t+1 < a_t+2 (1.3) */
  double fast_tau;     /*                                                    (0.5) */
  double deep_rho;     /* x << y  iff  deep_rho*x + deep_tau < y             (2.0) */
  double deep_tau;     /*                                                    (0.5) */
  double done_eps;     /* transition complete at t+K: ACT(t,t+K+1) <= (1+done_eps)*ACT(t,t+K) (0.25) */
  double steady_gamma; /* dissolve K >= 2: a_t+K+d <= steady_gamma * max of the next
                          steady_frames values, d = 0..steady_span-1          (1.2) */
  int steady_frames;   /*                                                    (4) */
  int steady_span;     /*                                                    (2) */
  double lag_rho;      /* dissolve K >= 2: ACT(t,t+K) > lag_rho * ACT(t,t-K)  (1.5) */
  double blend_ratio;  /* dissolve K >= 2: ACT(t,t+K-1) >= blend_ratio * ACT(t,t+K) (0.6) */
  double pd_rho;       /* 3:2 pulldown shots: candidate and cut iff a_t > pd_rho * the same
                          cadence step one 5-frame unit earlier              (1.4) */
  double pd_gamma_new; /* ... and a_t+1 <= pd_gamma_new * a_t-4 (steady new shot) (2.5) */
  double pd_gamma_old; /* ... and a_t-1 <= pd_gamma_old * a_t-6 (t is no flash)  (1.4) */
  /* sampling structure (Sec. III.C) */
  int samp_max_frames;   /* frames analysed per shot (N_s)                    (20) */
  double static_amm_px;  /* frames with AMM(t,t+1) below this are skipped     (0.5) */
  double comb_ratio;     /* combed iff AMM(v0) > comb_ratio * min(AMM(v1), AMM(v2)) (0.65) */
  double unequal_ratio;  /* interlaced needs median(AMM(v1)/AMM(v2)) > this or < 1/this (1.04) */
  double rep_ratio;      /* repeated field: ACT(u_t,u_t+1) < rep_ratio * ACT(l_t,l_t+1), or
                            the same with the fields swapped                 (0.25) */
  int rep_probe;         /* voters that always read the same-parity pairs     (5) */
  double pulldown_match; /* fraction of voters matching the 3:2 repeated-field pattern (0.8) */
  /* dynamic keyframes (Sec. III.D) */
  double kf_theta;       /* keyframe when the accumulated activity exceeds this (8.0) */
  /* resources */
  int device;                          /* CUDA device ordinal                 (0) */
  int window_frames;                   /* rolling window of frames on the device: 0 = auto (max(96,
                                          2*kmax + steady_span + steady_frames + 6)), else at least
                                          2*kmax + steady_span + steady_frames + 4 */
  unsigned long long mem_budget_bytes; /* device memory cap for one analyser (0 = none) */
  int want_motion;                     /* keep level-0 motion fields of frame pairs (t,t+1) (0) */
  int tile_x, tile_y;                  /* pair-kernel tile in blocks (8x4, 4x4, 8x2, 16x2, 4x8);
                                          0 = autotuned per resolution (0, 0) */
  int time_kernels;                    /* record CUDA events around every kernel launch (0) */
  int step_frames;                     /* server: frames copied per clip per step (0 = fill the window) (32) */
  int kernel_mode;                     /* 0: split coarse / refine kernels on two streams for the default
                                          estimator (levels 3, radius_refine 2), fused otherwise;
                                          1: always the fused kernel (0) */
  int want_histogram;                  /* per-frame luma histogram and its statistics (0) */
  int prefetch_frames;                 /* when the detectors wait for pairs, a look-ahead over at most
                                          this many frames asks for the pairs they will read next
                                          (computed in the same wave; decisions unchanged) (256) */
  double wait_timeout_ms;              /* host watchdog: a wave or frame copy not complete after this
                                          many ms fails the call with ANALYSER_ERR_TIMEOUT (sticky);
                                          0 = wait without a limit (0) */
} analyser_params;

/* One measure of one pair, in the order of (kind, a, b). */
typedef struct {
  int kind, a, b;
  int64_t si, sj, sii, sjj, sij; /* exact sums of i, j, i^2, j^2, i*j over the pair's pixels */
  int64_t sabs;                  /* residual: sum of |i - j| (J motion-compensated) */
  int64_t samm;                  /* sum over blocks of floor(|v| * 65536) */
  int64_t n, nb;                 /* pixels and blocks of the pair */
  double ncc, swr, amm, act;
} analyser_measure;

typedef struct {
  int first, last;     /* frame range of the shot (inclusive) */
  int label;           /* ANALYSER_UNKNOWN / _PROGRESSIVE / _INTERLACED / _PULLDOWN */
  int field_order;     /* ANALYSER_FO_* (interlaced shots) */
  int pulldown_phase;  /* 0..4: a frame t with (t - phase) mod 5 == 0 shows fields A A; -1 if none */
  int analysed;        /* frames that voted */
} analyser_shot;

/*
 * Unary measure of one frame (Sec. III.A lists histogram measures among the
 * unary ones; this is their exact integer form): the 256-bin histogram of the
 * level-0 luma and statistics derived from it.  With n = width*height,
 * S1 = sum v, S2 = sum v^2 (exact integers): mean = S1 / n,
 * std = sqrt((n*S2 - S1^2) / (n*n)) in FP64 with that operation order,
 * median = lower median of the values (sorted index (n-1)/2) and mad = lower
 * median of |v - median|.  Not used by the detectors.
 */
typedef struct {
  int frame;
  uint32_t bins[256];
  double mean, std;
  int median, mad;
} analyser_frame_hist;

typedef struct {
  int nframes;
  int ncuts;      const int* cuts;            /* first frame of each new shot after a hardcut */
  int ndissolves; const int* dissolves;       /* pairs (t, K): last frame before, span */
  int nshots;     const analyser_shot* shots;
  int label, field_order, pulldown_phase;     /* clip-level verdict */
  int nkeyframes; const int* keyframes;
  int nmeasures;  const analyser_measure* measures;
  int motion_w, motion_h;                     /* block grid of the motion dumps (0 if none) */
  const int16_t* motion;                      /* (nframes-1) x motion_h x motion_w x 2 (vx, vy), or null */
  int nhist;      const analyser_frame_hist* hist;   /* one per frame when params.want_histogram, else 0 */
} analyser_results_t;

typedef struct analyser analyser;
typedef struct server server;

/* Defaults of every parameter (values in the comments above). */
int analyser_default_params(analyser_params* p);

/*
 * Create an analyser for a clip of width x height luma frames at `fps` frames/s.
 * Requirements: 64 <= width, 64 <= height, height even, width*height <= 11,800,000
 * (exact 64-bit correlation sums), parameters within the ranges above.
 * ANALYSER_ERR_OOM when the rolling window exceeds params.mem_budget_bytes
 * (checked before any device work) or its allocation fails.
 * On success *out owns the device buffers of the rolling frame window.
 */
int analyser_create(int width, int height, double fps, const analyser_params* p, analyser** out);

/*
 * Append `nframes` frames from HOST memory (frame k at luma + k*height*pitch_bytes,
 * rows pitch_bytes apart, pitch_bytes >= width).  The frames are copied; the
 * caller keeps ownership.  Runs GPU work as the window fills; returns when all
 * frames are copied.  A push after analyser_finish fails with ANALYSER_ERR_STATE,
 * and like every failure that code sticks to the handle.
 */
int analyser_push_frames(analyser* a, const uint8_t* luma, long long pitch_bytes, int nframes);

/*
 * Append `nframes` frames already resident in DEVICE memory (frame k at
 * luma + k*frame_stride_bytes; pitch_bytes a multiple of 16 and at most
 * INT_MAX/2, luma 16-byte aligned).  No copy is made: the buffer must stay valid and unchanged until
 * analyser_finish returns.
 */
int analyser_push_frames_device(analyser* a, const uint8_t* luma, long long pitch_bytes,
                                long long frame_stride_bytes, int nframes);

/* No more frames: runs the remaining work to the end of the clip. */
int analyser_finish(analyser* a);

/*
 * Results after analyser_finish (ANALYSER_ERR_STATE before it, without making
 * the handle fail).  Pointers are owned by the analyser and stay valid until
 * the next call on it or analyser_destroy.
 */
int analyser_results(analyser* a, analyser_results_t* out);

/* Last error code and a one-line message (owned by the analyser). */
int analyser_last_error(const analyser* a, const char** message);

/* Counters of the last run: pair measures computed, GPU waves, kernel launches. */
int analyser_stats(const analyser* a, long long* pairs, long long* waves, long long* launches);

/* Work and time counters (kernel times need params.time_kernels = 1). */
typedef struct {
  long long pairs, waves, launches;
  long long pair_launches, pyramid_launches;
  double pair_kernel_ms, pyramid_kernel_ms;  /* CUDA-event time on the library's stream */
  double absdiff_ops;                        /* algorithmic |a-b| accumulates of the block search */
  double pyramid_bytes;                      /* algorithmic bytes of the pyramid kernel (read + write) */
  long long h2d_bytes, d2h_bytes;            /* host<->device bytes moved by the library */
  double host_gather_ms;                     /* host time building wave descriptors */
  double host_wait_ms;                       /* host time waiting for wave completion */
  double host_results_ms;                    /* host time finalising records and running detectors */
  double host_setup_ms;                      /* host time creating the analyser (window allocation, tables) */
  double host_copy_wait_ms;                  /* host time blocked on frame copies from host memory */
} analyser_profile_t;
int analyser_profile(const analyser* a, analyser_profile_t* out);

void analyser_destroy(analyser* a);

/*
 * Stateless measure of `npairs` pairs on DEVICE frames, for tests and kernel
 * timing: pair k compares frame ia[k] with frame ib[k] of `frames` (frame f at
 * frames + f*frame_stride_bytes) with pair kind kinds[k] (ANALYSER_PAIR_FRAME ..
 * ANALYSER_PAIR_LOWER_LOWER; field kinds need an even height).  records receives
 * 7 int64 per pair (sum i, sum j, sum i^2, sum j^2, sum i*j, sum |i-j|, S_amm)
 * in HOST memory (pitch_bytes a multiple of 16 and at most INT_MAX/2, frames
 * 16-byte aligned); motion (optional, HOST) receives the level-0 field of every
 * pair, nby*nbx (vx, vy) int16 each.  `stream` is a cudaStream_t (0 = default).
 * Takes its pyramids and queues from the library's resource cache for the
 * duration of the call.
 */
int analyser_measure_pairs(const analyser_params* p, int width, int height, const uint8_t* frames,
                           long long pitch_bytes, long long frame_stride_bytes, int nframes,
                           const int* kinds, const int* ia, const int* ib, int npairs,
                           int64_t* records, int16_t* motion, void* stream);

/*
 * One pair measure that allocates no device memory: the same record as
 * analyser_measure_pairs (7 int64 written to HOST memory `record`) for frames
 * a and b in DEVICE memory (pitch_bytes a multiple of 16, 16-byte aligned
 * pointers) and pair kind `kind` (ANALYSER_PAIR_FRAME .. ANALYSER_PAIR_LOWER_LOWER).
 * The paper has no counterpart; it exists for
 * callers embedded in a host application that reserves all device memory up
 * front and forbids cudaMalloc/cudaFree while it runs (an allocation could
 * fail against that reservation, and both calls synchronise the device).
 * Its scratch (pyramids, descriptors, accumulators) is a fixed 5.5 MiB device
 * array inside this library, present on every device that loads it until the
 * process exits: 3840x2160 frames fit, larger scratch needs are rejected with
 * ANALYSER_ERR_INVALID_ARG, as is a pitch_bytes above INT_MAX/2.  Only params
 * levels = 3, block = 16.  The array is shared by all calls: calls whose GPU
 * work overlaps race on it.  The first call for a device (params.device) looks
 * up the array's device address with that device current; make that first
 * call before any stream capture.  Every call waits for `stream` and returns
 * once the record is in `record`; the calling thread's current device is the
 * same after the call as before it.
 */
int analyser_measure_pair_noalloc(const analyser_params* p, int width, int height, int kind,
                                  const uint8_t* frame_a, const uint8_t* frame_b, long long pitch_bytes,
                                  int64_t* record, void* stream);

/*
 * Host-only: run the detectors alone on measures supplied by `get`, without a
 * GPU.  get(ctx, kind, a, b, rec) fills rec[0..8] = sum i, sum j, sum i^2,
 * sum j^2, sum i*j, sum |i-j|, S_amm, n, nb for pair (kind, a, b) and returns 0
 * (nonzero aborts with ANALYSER_ERR_INVALID_ARG).  The FP64 finalisation and
 * every decision are the library's own.  *out is an analyser handle whose only
 * valid calls are analyser_results, analyser_last_error and analyser_destroy.
 */
typedef int (*analyser_measure_fn)(void* ctx, int kind, int a, int b, int64_t* rec);
int analyser_detect_offline(const analyser_params* p, int width, int height, int nframes,
                            analyser_measure_fn get, void* ctx, analyser** out);

/*
 * Throughput of the packed-byte SAD instruction the search kernels issue
 * (vabsdiff4 with accumulate) in a register-only loop over every SM, in
 * 10^12 |a-b| accumulates per second: the peak against which the pair
 * kernel's roofline fraction is reported.  Needs a GPU; runs ~50 ms.
 */
int analyser_measure_sad_peak(int device, double* tera_per_s);

/*
 * The same register-only loop timed for other packed |a-b| sequences (for
 * choosing the kernels' instruction): 0 vabsdiff4 with accumulate (as
 * analyser_measure_sad_peak), 1 the sum-of-absolute-differences intrinsic plus
 * an add, 2 per-byte absolute differences plus dp4a, 3 per-byte max minus min
 * plus dp4a, 4 half the chains as 0 and half as 2.  Same units and errors as
 * analyser_measure_sad_peak; a sequence outside 0..4 gives ANALYSER_ERR_INVALID_ARG.
 */
int analyser_measure_sad_sequence(int device, int sequence, double* tera_per_s);

/* ---- dense sub-pixel flow (alternative motion estimator) ---------------------- */

/*
 * Dense flow by inverse search, the estimator the paper names for its motion
 * field (Sec. III.A, reference [8]), as an alternative to the block-matching
 * field the analyser's measures use.  Steps, coarse to fine over the same box
 * pyramid: a grid of patch x patch patches of frame a (stride `stride`, the last
 * patch of a row or column flush with the border); per patch `iters`
 * inverse-compositional Gauss-Newton steps, H from the template's
 * central-difference gradients damped by damp_rel * trace(H) + damp_abs, the
 * residual J(x + u) - T(x) with frame b sampled bilinearly (clamp-to-edge); a
 * patch starts from the coarser level's dense flow at its centre, doubled;
 * densification weights each covering patch by 1 / max(1, |J(x + u) - I(x)|).
 * No step compares against a threshold.  The kernels compute in FP32, or in
 * FP64 with fp64 = 1 (the output is float either way).  Where a patch's
 * iteration does not converge, FP32 rounding can grow over the steps: the FP32
 * flow then differs from an FP64 evaluation by more than rounding at some
 * pixels.
 */
typedef struct analyser_flow_params {
  int levels;        /* pyramid levels, 1..3; width and height >= patch << (levels - 1) (3) */
  int patch;         /* patch side; this build supports 8 (8) */
  int stride;        /* patch grid step, 1..patch (4) */
  int iters;         /* Gauss-Newton steps per patch and level, 0..64 (8) */
  int fp64;          /* 0: the steps in FP32; 1: in FP64 (slower; element-wise reproducible) (0) */
  double damp_rel;   /* damping per unit of trace(H), >= 0 (0.01) */
  double damp_abs;   /* damping added to it, > 0 (1.0) */
} analyser_flow_params;

void analyser_default_flow_params(analyser_flow_params* p);

/*
 * The flow from frame a to frame b (frame b at x + U(x) matches frame a at x):
 * frame_a, frame_b: DEVICE 8-bit luma planes, width x height, rows pitch_bytes
 * apart (width <= pitch_bytes <= INT_MAX); flow: DEVICE buffer of width *
 * height * 2 floats, written row-major as (u, v) per pixel; all owned by the
 * caller.  Runs on `stream` (a cudaStream_t, or null) and returns once the flow
 * is written; device scratch comes from the resource cache.  Returns
 * ANALYSER_ERR_INVALID_ARG for null pointers or parameters or sizes outside
 * the ranges above, ANALYSER_ERR_OOM when scratch cannot be had,
 * ANALYSER_ERR_CUDA when a launch fails.
 */
int analyser_dense_flow(const analyser_flow_params* p, int width, int height, const uint8_t* frame_a,
                        const uint8_t* frame_b, long long pitch_bytes, float* flow, void* stream);

/*
 * The pair measures of Sec. III.A with the dense flow U of analyser_dense_flow
 * as the motion field: AMM = mean |U(x)| over the width * height pixels (px);
 * frame b warped by U, Jw(x) = J(x + U(x)) (bilinear, clamp-to-edge); NCC of
 * frame a and Jw = C / sqrt(Vi * Vj) with C = n S_ij - S_i S_j, Vi = n S_ii -
 * S_i^2, Vj = n S_jj - S_j^2 (both variances zero or below: 1, one of them: 0);
 * SWR = max(0, 1 - NCC); ACT = sqrt(AMM * SWR).  The sums are FP64, added in
 * a fixed order (the same value on every call); the per-pixel values are in
 * the flow's precision.  Arguments and errors as
 * analyser_dense_flow (scratch for the flow comes from the resource cache).
 */
typedef struct analyser_flow_measure_t {
  double amm, ncc, swr, act;
  double sums[6];   /* sum |U|, S_i, S_j, S_ii, S_jj, S_ij */
} analyser_flow_measure_t;

int analyser_flow_measure(const analyser_flow_params* p, int width, int height, const uint8_t* frame_a,
                          const uint8_t* frame_b, long long pitch_bytes, analyser_flow_measure_t* out, void* stream);

/*
 * Resource cache (the paper has no counterpart: this is library plumbing).
 * Device buffers, page-locked host buffers, streams and events that an
 * analyser, server or analyser_measure_pairs call releases go back to a
 * process-wide cache and are reused by the next one of the same size class,
 * which avoids cudaMalloc/cudaFree (and the device synchronisation cudaFree
 * implies) per clip.  analyser_trim_cache() returns the cached device and host
 * buffers to CUDA (buffers still owned by live analysers or servers are not
 * touched); analyser_cached_bytes() reports the device bytes held.  Both are
 * thread-safe and never fail.
 */
void analyser_trim_cache(void);
long long analyser_cached_bytes(void);

/* ---- serving: continuous batching of many clips on one GPU ------------------- */

/* A server admits clips while the device-memory budget allows.  Every clip of
 * a server uses one tile shape (params tile_x/tile_y, else 8x4; no autotune),
 * so that a wave's pairs of all sizes go out as one coarse and one refinement
 * launch; while frame copies are landing and no detector waits for pairs, a
 * step waits for 1024 new frames (over all clips) or the end of the copies
 * before it launches a wave. */
int server_create(const analyser_params* p, unsigned long long budget_bytes, server** out);

/*
 * Submit a whole clip from HOST memory (copied before return is NOT guaranteed:
 * the buffer must stay valid until server_poll reports the ticket done).
 * *ticket identifies the request.
 */
int server_submit(server* s, int width, int height, double fps, const uint8_t* frames,
                  long long pitch_bytes, int nframes, long long* ticket);

/* ANALYSER_PENDING while the clip is queued or running; ANALYSER_OK with the
 * results (owned by the server, valid until server_release or destroy). */
int server_poll(server* s, long long ticket, analyser_results_t* out);

/*
 * One scheduling step: admit queued clips while the budget allows, copy the
 * next frames of every admitted clip into its window, run one GPU wave over
 * all of them and retire finished clips.  Admission takes queued clips in
 * arrival order and admits every one whose window fits what is left of the
 * budget, so a large clip waiting for memory does not hold back smaller ones
 * behind it; once the oldest queued clip has waited 0.5 s, nothing behind it
 * is admitted before it.  *active (optional) receives the number of clips
 * admitted or queued after the step.
 */
int server_step(server* s, int* active);

/* Run server_step until every submitted clip is done. */
int server_drain(server* s);

/* Work and time counters of the server's engine. */
int server_profile(const server* s, analyser_profile_t* out);

/* Per-request timing: seconds from submit to results ready. */
int server_latency(const server* s, long long ticket, double* seconds);

/* Free one finished request's results. */
int server_release(server* s, long long ticket);

void server_destroy(server* s);

#ifdef __cplusplus
}
#endif
#endif /* GB300_VIDEO_ANALYSER_H */
