/*
 * seg.h -- C ABI of the B300 (sm_103a) per-frame path of Akamine, Fukuchi,
 * Kimura and Takagi, "Fully automatic extraction of salient objects from
 * videos in near real-time" (arXiv:1008.0502):
 *
 *   RGB8 frame --(Sec. 3, Sec. 7.2: Itti-style saliency map)--> saliency
 *     --(Sec. 5: saliency prior q; Sec. 6: sequential Kalman update with the
 *        previous segmentation)--> prior p-hat
 *     --(Sec. 4, Eqs. 1-4; Sec. 5: MRF data and smoothness terms)--> int32 graph
 *     --(Sec. 4: exact s-t minimum cut)--> mask, cut value.
 *
 * Conventions (all entry points):
 *  - Return SEG_OK (0) or a negative SEG_E* code; seg_strerror() names it.
 *  - "dev" pointers are CUDA device pointers on the context's device; "host"
 *    pointers are host memory (pinned memory gives asynchronous copies).
 *  - Images are row-major, pixel (y, x) at y*W + x.  RGB8 frames are
 *    interleaved H x W x 3 bytes.  Masks are H x W bytes, 1 = object (the
 *    source side of the cut), 0 = background.
 *  - Grid n-link capacities (ncap) are nbr/2 planes of H x W int32, ordered
 *    E (x+1, y), S (x, y+1), SE (x+1, y+1), SW (x-1, y+1); an entry whose
 *    neighbour lies outside the grid is ignored.  Each undirected n-link has
 *    the same capacity in both directions (Sec. 4 footnote: a pair of directed
 *    edges).  Every capacity must lie in [0, 2^24].
 *  - The caller owns every input/output buffer.  A context owns its workspace,
 *    allocated once in seg_create; per-frame calls allocate nothing.
 *  - Work is enqueued asynchronously on the context's stream; outputs are
 *    valid once that stream has been synchronised (seg_sync does it and also
 *    reports device-side failures).  A context is not thread-safe.
 *  - Cuts are exact: the returned mask is the unique minimal source set (the
 *    intersection of all minimum cuts), so equal-energy ties go to background.
 */
#ifndef SEG_H
#define SEG_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEG_OK 0
#define SEG_EINVAL (-1)        /* bad argument, size or parameter */
#define SEG_ENOMEM (-2)        /* device memory allocation failed */
#define SEG_ENOTCONVERGED (-3) /* the min-cut hit its cycle cap (max_cycles) */
#define SEG_ECUDA (-4)         /* a CUDA runtime call failed */
#define SEG_ETIMEOUT (-5)      /* a bounded device-side wait ran out (kernel returned early) */
#define SEG_ECAPACITY (-6)     /* an input capacity lies outside [0, 2^24] */

typedef struct seg_ctx seg_ctx;

/* Parameters of the method.  Defaults (seg_default_params) are the 640x480
 * reading: 9 pyramid images, centers c in 2..4, surrounds s = c + 3..4, an
 * 8-neighbour grid. */
typedef struct seg_params {
  int32_t levels;          /* pyramid images incl. base: sigma = 0 .. levels-1 (<= 16) */
  int32_t c_min, c_max;    /* center scales (1 <= c_min <= c_max) */
  int32_t d_min, d_max;    /* surround s = c + d, c_max + d_max <= levels-1 */
  int32_t n_orient;        /* Gabor orientations theta_k = k*pi/n_orient (1..8) */
  float gabor_lambda;      /* carrier wavelength in pixels of each level (4) */
  float gabor_sigma;       /* isotropic envelope sigma (2) */
  int32_t gabor_radius;    /* taps per axis = 2r+1 (6; <= 8) */
  int32_t norm_tile;       /* N(.) local-maximum tile side (8) */
  float norm_flat;         /* maps with range <= norm_flat normalise to 0 (1e-5) */
  float w[4];              /* channel weights I, RG, BY, O (1/3, 1/6, 1/6, 1/3) */
  int32_t cs_opponent_sum; /* 1: RG/BY center-surround |X(c) + up X(s)| (literal Itti), 0: |X(c) - up X(s)| */
  int32_t border_px;       /* frame-edge band with saliency prior eps (1) */
  double sigma1, sigma2;   /* Kalman noise std-devs (0.03, 0.035: Sec. 8.1) */
  float f_sigma;           /* Gaussian smoothing of the previous mask (2) */
  int32_t f_radius;        /* its radius (6; <= 8) */
  float eps;               /* clamp for logs and the border prior (1e-4) */
  double lambda_u;         /* colour-likelihood weight (1) */
  double lambda_p;         /* Potts constant xi_2 (0) */
  double lambda_s;         /* contrast weight of psi_2 (1.5) */
  double sigma_I;          /* contrast intensity scale (0.05) */
  double cap_scale;        /* K: capacity = min(2^24, floor(K*cost + 1/2)) (1000) */
  int32_t neighbourhood;   /* 4 or 8 */
  int32_t max_cycles;      /* min-cut cycle cap -> SEG_ENOTCONVERGED (20000) */
  int32_t global_relabel_every; /* min-cut cycles between global relabels (1) */
  int32_t local_iters;     /* push/relabel iterations per tile visit (12) */
  int32_t use_graph;       /* 1: seg_push_frame replays one captured CUDA graph per frame (when the
                              context's stream is not the legacy default stream); 0: eager launches */
  int32_t gmm_components;  /* Gaussians per label in the colour likelihood psi_1: 1 (closed form) or 3
                              (EM, Sec. 4 / Sec. 7.3; M = 3 in Sec. 8.1) */
  int32_t em_iters;        /* EM iterations when gmm_components > 1 (5) */
  int32_t warm_start;      /* 1: each stream's min cut starts from its previous frame's n-link flows
                              (dynamic graph cuts, Sec. 1 / Sec. 8.2 prior art); results are identical
                              to a cold start; 0: cold start every frame */
  int32_t barrier_timeout_us; /* time limit of every wait at a grid barrier of the min cut, in
                              microseconds (1 .. 60e6; 4e6): a CTA that waits longer records
                              SEG_ETIMEOUT, every CTA then returns at its next barrier, and the
                              context stays usable (failure detection; no wait is unbounded) */
  int32_t kmeans_iters;    /* Lloyd iterations of the k-means start of the EM (gmm_components > 1;
                              Sec. 7.3); the seeds are k-means++ taken in expectation (3; 0 .. 100) */
  int32_t gmm_update;      /* 1: a stream's EM starts from its previous frame's fitted mixtures (the
                              likelihood update of Sec. 2 / Sec. 6), the k-means start only on a
                              video's first frame; 0: every frame starts from the k-means start */
  int32_t relabel_frontier; /* min cut schedule (results identical): 1 = the third and later fixpoint
                              rounds of a global relabel (BFS from t) or of the final reach take
                              only the tiles next to a tile that changed, from a queue compacted
                              with warp ballots and spread over all CTAs; 0 = every CTA scans its
                              own tiles for changed neighbours (0) */
  int32_t cut_tile;        /* min cut tile shape (results identical; fixed for a context's life):
                              0 = 32x16, 1 = 32x8, 2 = 64x8 nodes, one thread a node (0) */
} seg_params;

/* Fills *p with the defaults above.  Returns SEG_EINVAL if p is NULL. */
int seg_default_params(seg_params* p);

/* Creates a context for H x W frames on the current CUDA device, enqueuing on
 * `stream` (a cudaStream_t; NULL = legacy default stream).  Allocates the whole
 * workspace (about 120 bytes per pixel).  Errors: SEG_EINVAL (H or W < 1,
 * H*W > 2^26, invalid params), SEG_ENOMEM, SEG_ECUDA.  *out is NULL on error. */
int seg_create(void* stream, int H, int W, const seg_params* p, seg_ctx** out);

/* A batch context: B independent video streams of the same size H x W, all
 * advanced by one seg_push_frame (one frame of every stream per call, one
 * launch per kernel for the whole batch).  Every per-frame input/output is B
 * frames back to back: rgb B x H x W x 3, saliency/prior B x H x W, mask
 * B x H x W, cut B int64.  Stream b's results equal those of a single context
 * fed the same frames.  The stage entry points seg_prior, seg_terms and
 * seg_mincut need B == 1.  seg_create(...) is seg_create_batch(..., 1, ...).
 * Errors as seg_create, plus SEG_EINVAL for B < 1 or B*H*W > 2^26. */
int seg_create_batch(void* stream, int B, int H, int W, const seg_params* p, seg_ctx** out);

/* Marks slot b of a batch context as holding a stream (on = 1, the state at
 * creation) or empty (on = 0).  The per-frame kernels skip an empty slot's
 * frame: no kernel reads or writes its rows (the stacked cut treats them as
 * outside the grid), its outputs are then undefined, and the slot's state
 * (previous mask, Kalman variance, warm-start flows, colour mixtures) keeps its
 * values, so a stream switched off and on again without seg_reset_stream
 * continues where it stopped.  Enqueued on the context's stream, so it
 * applies from the next seg_push_frame on, also inside captured graphs.  No
 * paper counterpart: continuous batching of many streams.  A single-stream
 * context always runs its frame.  Errors: SEG_EINVAL (ctx NULL, b out of
 * range, on not 0 or 1), SEG_ECUDA. */
int seg_set_stream_active(seg_ctx* ctx, int b, int on);

/* Device bytes seg_create_batch(B, H, W, p) would allocate for its workspace
 * (for admission control by HBM footprint).  Errors as seg_create_batch. */
int seg_workspace_bytes(int B, int H, int W, const seg_params* p, size_t* bytes);

/* Changes the min cut's grid-barrier time limit (seg_params.barrier_timeout_us)
 * of an existing context, e.g. a watchdog tightened after start-up.  Waits for
 * the context's stream and drops its captured CUDA graphs (the limit is a
 * kernel argument; the next seg_push_frame captures them again).  No
 * paper counterpart: failure detection of the device-side waits.
 * Errors: SEG_EINVAL (ctx NULL, us outside 1 .. 60e6), SEG_ECUDA. */
int seg_set_barrier_timeout(seg_ctx* ctx, int us);

/* Frees the context and its workspace (synchronises its stream first).
 * Errors: SEG_EINVAL (ctx NULL). */
int seg_destroy(seg_ctx* ctx);

/* Starts a new video: forgets the previous mask and the prior variance, so the
 * next frame is t = 0 (Sec. 6 with P_{-1} = +inf: p-hat = q).  Enqueued on the
 * context's stream.  Errors: SEG_EINVAL (ctx NULL), SEG_ECUDA. */
int seg_reset(seg_ctx* ctx);
/* seg_reset for stream b of a batch context only (a new video on that slot).
 * Errors: SEG_EINVAL (ctx NULL, b outside 0..B-1), SEG_ECUDA. */
int seg_reset_stream(seg_ctx* ctx, int b);

/* One frame of the whole method (Fig. 3; Secs. 3-6).
 *   rgb_dev      H*W*3 uint8 input frame (device).
 *   saliency_dev H*W float: the saliency map upsampled to frame size (device).
 *   prior_dev    H*W float: p-hat(A_x,t = 1) of Sec. 6 (device).
 *   mask_dev     H*W uint8: the minimum-cut segmentation (device).
 *   cut_dev      one int64: the minimum cut value of the integer graph (device).
 * Any output pointer except mask_dev may be NULL.  The mask is kept inside the
 * context as A_{t-1} of the next frame and the Kalman variance advances.
 * Errors found on the host return immediately; device-side failures (cycle
 * cap, wait timeout, capacity range) are reported by the next seg_sync. */
int seg_push_frame(seg_ctx* ctx, const uint8_t* rgb_dev, float* saliency_dev, float* prior_dev,
                   uint8_t* mask_dev, int64_t* cut_dev);

/* seg_push_frame with HOST buffers: copies the frame to the device, runs the
 * frame, copies mask and cut value (and saliency/prior when non-NULL) back,
 * then synchronises the stream.  The buffers hold B*H*W*3 bytes (rgb), B*H*W
 * bytes (mask), B*H*W floats (saliency, prior) and B int64 (cut); pinned memory
 * makes the copies asynchronous.  Returns the frame's device status, or
 * SEG_EINVAL (ctx, rgb_host or mask_host NULL) or SEG_ECUDA. */
int seg_push_frame_host(seg_ctx* ctx, const uint8_t* rgb_host, float* saliency_host,
                        float* prior_host, uint8_t* mask_host, int64_t* cut_host);

/* Synchronises the context's stream and returns the first device-side status
 * recorded since the last seg_sync (SEG_OK, SEG_ENOTCONVERGED, SEG_ETIMEOUT,
 * SEG_ECAPACITY), or SEG_ECUDA.  *cycles (nullable) receives the last min-cut's
 * cycle count. */
int seg_sync(seg_ctx* ctx, int* cycles);

/* The last CUDA runtime call of this library that failed on the calling host
 * thread (the call and CUDA's error name), "" if none: the detail behind
 * SEG_ECUDA.  Owned by the library; valid until the next failure on the
 * thread. */
const char* seg_last_cuda_error(void);

/* ---- groups: several contexts (e.g. batch contexts of different
 * resolutions) advanced by one CUDA graph launch per frame step (many streams
 * of uneven resolution in one launch; Sec. 7.1 processes one stream).
 *
 * seg_group_create captures every member's frame launch sequence (the one
 * seg_push_frame runs) as parallel branches of one graph, on the members'
 * own streams forked from and joined into `stream` (a cudaStream_t, not the
 * legacy default stream).  A step (seg_group_push) writes every member's
 * frame pointers through the graph's root node and launches the graph once on
 * `stream`.  Results equal those of seg_push_frame on each member.  Members
 * keep their state; their streams are ordered around every step, so
 * seg_reset_stream, seg_set_stream_active or seg_sync on a member between
 * steps apply in order.  The graph holds the members' parameters as at
 * creation: after seg_set_barrier_timeout on a member, create the group
 * again.  Destroy the group before its members; do not push frames to a
 * member directly while its group has steps in flight.  No paper
 * counterpart. */
#define SEG_GROUP_MAX 16
typedef struct seg_group seg_group;

/* One member's frame of a step: device pointers laid out as seg_push_frame
 * takes them for that member (rgb and mask required; sal, prior and cut
 * nullable). */
typedef struct seg_frame_io {
  const uint8_t* rgb;
  float* sal;
  float* prior;
  uint8_t* mask;
  int64_t* cut;
} seg_frame_io;

/* ctxs: n distinct contexts (1 <= n <= SEG_GROUP_MAX), each on a stream of its
 * own creation (not the legacy default stream), not pipelined, not profiling;
 * the caller keeps ownership.  Synchronises the members' streams first.
 * Errors: SEG_EINVAL, SEG_ENOMEM, SEG_ECUDA (capture or instantiation failed).
 * *out is NULL on error. */
int seg_group_create(void* stream, seg_ctx* const* ctxs, int n, seg_group** out);

/* One frame step of every member: io[i] is member i's frame.  Enqueued on the
 * group's stream after all work enqueued on the members' streams.  Errors:
 * SEG_EINVAL (g or io NULL, a required pointer NULL), SEG_ECUDA. */
int seg_group_push(seg_group* g, const seg_frame_io* io);

/* Synchronises the group's stream and every member (seg_sync); codes[i] and
 * cycles[i] (both nullable, n entries) receive each member's status and last
 * cycle count.  Returns the first non-zero member status, SEG_OK, or
 * SEG_EINVAL / SEG_ECUDA. */
int seg_group_sync(seg_group* g, int* codes, int* cycles);

/* Waits for the group's stream and frees the group (not its members).
 * Errors: SEG_EINVAL (g NULL). */
int seg_group_destroy(seg_group* g);

/* Temporal state (Sec. 6: A_{t-1} and sigma^2_xi1(t-1), plus the frame index)
 * as a byte string: a 16-byte header of four uint32 (0x53454732, H, W, B);
 * then per stream 16 bytes (int32 frame index t, int32 0, double variance
 * P_{t-1}); then the B previous masks, H*W bytes each (0/1).  Host byte
 * order.  seg_get_state with buf == NULL stores the needed size in *n.  Both
 * synchronise the stream; seg_set_state makes the next cut start cold (the
 * warm-start flows are not part of the state).  Errors: SEG_EINVAL (size,
 * header not matching the context). */
int seg_get_state(seg_ctx* ctx, void* buf, size_t* n);
int seg_set_state(seg_ctx* ctx, const void* buf, size_t n);

const char* seg_strerror(int code);

/* ---- stage entry points: the same kernels as seg_push_frame, one stage at a
 * time, with every input explicit.  They use the context's workspace and do
 * not touch its temporal state. ---- */

/* Sec. 3 / Sec. 7.2: saliency map of one frame into saliency_dev (H*W float,
 * B*H*W for a batch context).  Errors: SEG_EINVAL (NULL argument), SEG_ECUDA. */
int seg_saliency(seg_ctx* ctx, const uint8_t* rgb_dev, float* saliency_dev);

/* Sec. 3 / Sec. 7.2: standalone saliency map of one H x W RGB8 frame, without a
 * context: allocates and frees its own workspace (about 40 B/pixel), enqueues on
 * `stream` and synchronises it.  Errors as seg_create. */
int seg_saliency_grid(void* stream, int H, int W, const seg_params* p, const uint8_t* rgb_dev,
                      float* saliency_dev);

/* Sec. 5 + Sec. 6: p-hat = w_f * f(prev_mask) + (1 - w_f) * q(saliency), with
 * q = saliency / max(saliency) and eps on the border band.  prev_mask_dev may be
 * NULL when w_f == 0.  Errors: SEG_EINVAL (NULL ctx, saliency or prior; w_f
 * outside [0, 1]; prev_mask NULL with w_f != 0; a batch context), SEG_ECUDA. */
int seg_prior(seg_ctx* ctx, const float* saliency_dev, const uint8_t* prev_mask_dev, double w_f,
              float* prior_dev);

/* Sec. 4 Eqs. 1-4 + Sec. 5: int32 t-links cs = c(s,v), ct = c(v,t) (H*W each)
 * and n-links ncap (nbr/2 planes of H*W: E, S[, SE, SW]) from the frame and the
 * prior.  Errors: SEG_EINVAL (NULL argument, a batch context), SEG_ECUDA. */
int seg_terms(seg_ctx* ctx, const uint8_t* rgb_dev, const float* prior_dev, int32_t* cs_dev,
              int32_t* ct_dev, int32_t* ncap_dev);

/* Sec. 4: exact minimum cut of the context's H x W grid (its neighbourhood)
 * with the given capacities; writes mask and cut value (cut_dev may be NULL).
 * Errors: SEG_EINVAL (NULL ctx, capacity or mask pointer; a batch context),
 * SEG_ECUDA; device-side status (cycle cap, capacity range, wait timeout) is
 * reported by seg_sync. */
int seg_mincut(seg_ctx* ctx, const int32_t* cs_dev, const int32_t* ct_dev, const int32_t* ncap_dev,
               uint8_t* mask_dev, int64_t* cut_dev);

/* Sec. 4: standalone exact minimum cut of an H x W grid with neighbourhood nbr
 * (4 or 8).  Allocates and frees its own workspace, synchronises `stream`, and
 * returns the device status (SEG_ENOTCONVERGED after max_cycles cycles;
 * max_cycles <= 0 selects the default).  *cycles (nullable) receives the
 * number of cycles used. */
int seg_mincut_grid(void* stream, int H, int W, int nbr, const int32_t* cs_dev,
                    const int32_t* ct_dev, const int32_t* ncap_dev, uint8_t* mask_dev,
                    int64_t* cut_dev, int max_cycles, int* cycles);

/* seg_mincut_grid without any device allocation, for callers that are not
 * allowed to call cudaMalloc (code living under another framework's memory
 * pool, processes with a fixed device-memory quota, real-time loops that must
 * not allocate after start-up).  The paper has no counterpart.
 *   Same arguments, results and return codes as seg_mincut_grid, except that
 *   cut_dev must not be NULL and H*W may be at most
 *   SEG_MINCUT_STATIC_MAX_PIXELS (SEG_EINVAL otherwise).
 *   The workspace is one fixed device array inside the library (about 6 MB on
 *   every GPU that loads it, held until the process exits).  The first call on
 *   each device looks up that array's device address (cudaGetSymbolAddress)
 *   and keeps it for the life of the process, so make that first call before
 *   any stream capture; a cudaDeviceReset makes the kept address stale, and
 *   the entry point must not be used on that device afterwards.
 *   All calls share the one array: calls that overlap on the GPU (two streams,
 *   or two host threads on the same device) race and corrupt each other's
 *   results.  Every call waits for its cut: it synchronises `stream` and
 *   copies the device status word to the host before returning. */
#define SEG_MINCUT_STATIC_MAX_PIXELS 131072
int seg_mincut_grid_static(void* stream, int H, int W, int nbr, const int32_t* cs_dev,
                           const int32_t* ct_dev, const int32_t* ncap_dev, uint8_t* mask_dev,
                           int64_t* cut_dev, int max_cycles, int* cycles);

/* Copies an intermediate map of the last seg_saliency/seg_push_frame into
 * dst_host (float, n elements), for stage-by-stage parity checks:
 *   which 0: pyramid channel index / 16 (0 I, 1 RG, 2 BY) at level index % 16 (levels >= 1)
 *   which 1: orientation map theta = index / 16 at level index % 16
 *   which 2: normalised conspicuity map index (0 I, 1 RG, 2 BY, 3 O) at sigma_S = c_max
 *   which 3: S at sigma_S (index ignored)
 * Synchronises the stream.  Errors: SEG_EINVAL (unknown map or wrong n). */
int seg_debug_copy(seg_ctx* ctx, int which, int index, float* dst_host, size_t n);

/* Per-stage device timing of seg_push_frame (measurement support; the paper
 * reports per-stage times in Table 5).  seg_profile_enable(ctx, 1) starts a
 * fresh record: every following seg_push_frame records CUDA events on the
 * context's stream around its four stages (saliency, prior, terms, min cut)
 * and stores the min-cut's cycle count; up to 4096 frames are kept (later
 * frames are not recorded).  seg_profile_enable(ctx, 0) stops recording.
 * seg_profile_read synchronises the stream and returns, over the recorded
 * frames: stage_ms[4] summed stage times, *frames, *cycles summed min-cut
 * cycles, and (if frame_ms is non-NULL) each frame's first-to-last event time
 * in frame_ms[0 .. min(frames, max_frames)-1].  Errors: SEG_EINVAL, SEG_ENOMEM,
 * SEG_ECUDA. */
int seg_profile_enable(seg_ctx* ctx, int on);
int seg_profile_read(seg_ctx* ctx, double* stage_ms, int* frames, long long* cycles, float* frame_ms,
                     int max_frames);
/* seg_profile_read plus, per recorded frame f < max_frames (if mincut_stats is
 * non-NULL), seven int32 min-cut statistics in mincut_stats[7f .. 7f+6]:
 * cycles, global relabels, fixpoint rounds, then the time spent in
 * initialisation, global relabels, discharge cycles and the final reach pass
 * (units of 0.1 us, read from the device timer).  Errors as seg_profile_read. */
int seg_profile_read_ex(seg_ctx* ctx, double* stage_ms, int* frames, long long* cycles, float* frame_ms,
                        int* mincut_stats, int max_frames);

/* Pipelined frames.  A frame's saliency map (Sec. 3) does not depend on the
 * previous frame -- only its prior does (Sec. 6) -- so with pipelining on, the
 * saliency of frame t runs on an internal stream while frame t-1's prior, terms
 * and cut still run on a second internal stream (each frame's prior, terms and
 * cut start after the work enqueued on the context stream before the call, and
 * the context stream waits for them).  Results are identical to the
 * unpipelined path, frame order and temporal state are unchanged, and outputs
 * are valid once the context stream passes them, as for seg_push_frame.
 * seg_pipeline_enable(ctx, 1) allocates a second buffer for S and the saliency
 * maximum (even and odd frames alternate) plus the two internal streams;
 * seg_pipeline_enable(ctx, 0) synchronises and
 * releases them.  Profiled frames (seg_profile_enable) run unpipelined.
 * seg_push_frame_ev: as seg_push_frame, where the frame's saliency starts once
 * `rgb_ready` (a cudaEvent_t recorded after the RGB8 data was written) has
 * completed -- NULL: once the context stream reaches this call, which gives no
 * overlap.  The rgb buffer must stay unchanged until the context stream passes
 * the frame.  Errors as seg_push_frame; seg_pipeline_enable: SEG_ENOMEM,
 * SEG_ECUDA. */
int seg_pipeline_enable(seg_ctx* ctx, int on);
/* Host-buffer frames on a pipelined context, without waiting on the host: the
 * RGB8 frame (host, B x H x W x 3, pinned for overlap) is copied into a
 * three-frame device ring, pushed as by seg_push_frame_ev, and the mask (host,
 * B x H x W) and cut (host, B int64, or NULL) are copied back in frame order.
 * Results are complete after seg_sync; the host buffers must stay untouched until
 * then.  Errors: SEG_EINVAL (NULL rgb/mask, pipelining off), as seg_push_frame. */
int seg_push_frame_host_async(seg_ctx* ctx, const uint8_t* rgb_host, uint8_t* mask_host, int64_t* cut_host);
int seg_push_frame_ev(seg_ctx* ctx, const uint8_t* rgb_dev, float* saliency_dev, float* prior_dev,
                      uint8_t* mask_dev, int64_t* cut_dev, void* rgb_ready_event);

/* Size of pyramid level `level` along an n-pixel axis: ceil-halving (Sec. 7.2;
 * level 0 is n itself).  Pure host arithmetic; no error codes. */
int seg_level_dim(int n, int level);

/* ------------------------------------------------------------------------
 * Backward form: the saliency map (Sec. 3, Sec. 7.2) and the Kalman-updated
 * prior (Sec. 6) of B floating-point frames, differentiated with respect to
 * the frames, the four channel weights and the Kalman noise variances.
 *
 * theta (dev, 6 doubles) = (w_I, w_RG, w_BY, w_O, Q, R): the weights of
 * S = sum_k w_k N(C_k) (Sec. 3) and Q = sigma1^2, R = sigma2^2 of the
 * sequential update (Sec. 6); the context's params supply everything else
 * (their w, sigma1 and sigma2 are not used).
 *
 * Frames (dev, float, B x H x W x 3, values nominally in [0, 255]) are clip
 * times t0 .. t0+B-1 of one video: w_f(t) = Q / (Q + R + P(t-1)) with
 * P(t) = Q (R + P(t-1)) / (Q + R + P(t-1)) and P(-1) = inf, so w_f(0) = 0.
 * fmap (dev, float, B x H x W, or NULL for zeros) holds the previous masks
 * smoothed as in Sec. 6 (constants: no derivative is taken through them).
 *
 * Derivatives are those of the forward as written, with one-sided choices at
 * its kinks: N(.) through the first index (row-major) attaining the minimum,
 * the maximum and each tile maximum; |a| through sign(a), 0 at a = 0; max(0, a)
 * through a > 0; the hue-normalisation mask (10 (r+g+b) > max) held fixed.
 * The paper trains nothing and has no derivative; this form exists so that the
 * weights and variances can be fitted by gradient descent.
 * ------------------------------------------------------------------------ */
typedef struct seg_diff seg_diff;

/* Device bytes of a backward-form context.  Errors as seg_diff_create. */
int seg_diff_workspace_bytes(int B, int H, int W, const seg_params* p, size_t* bytes);

/* Allocates a context for batches of B frames of H x W on the current device;
 * its work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 * Errors: SEG_EINVAL (params as seg_create; B < 1; B*H*W > 2^26; more than 4096
 * N(.) tiles in a center-surround map or 1024 at sigma_S; W > 5120),
 * SEG_ENOMEM, SEG_ECUDA. */
int seg_diff_create(void* stream, int B, int H, int W, const seg_params* p, seg_diff** out);
int seg_diff_destroy(seg_diff* d);

/* Forward: saliency (dev, B x H x W, or NULL) and prior (dev, B x H x W) of the
 * frames at clip times t0 .. t0+B-1 (0 <= t0 <= 2^24).  Keeps what the backward
 * needs in the context (the pyramid, the Gabor responses, the accumulators and
 * conspicuity maps at sigma_S, w_f(t) and its derivatives).
 * Errors: SEG_EINVAL (NULL rgb/theta/prior, t0 out of range), SEG_ECUDA. */
int seg_diff_forward(seg_diff* d, const float* rgb_dev, const float* fmap_dev, const double* theta_dev, int t0,
                     float* saliency_dev, float* prior_dev);

/* Backward of the last seg_diff_forward (same rgb, fmap and theta):
 * L = sum_b <g_prior_b, prior_b> + <g_sal_b, saliency_b>; g_prior (dev,
 * B x H x W), g_sal (dev, B x H x W, or NULL for zeros).  Writes dL/dframes into
 * g_rgb (dev, B x H x W x 3) and dL/dtheta into g_theta (dev, 6 doubles).
 * Errors: SEG_EINVAL (NULL pointers; no forward yet), SEG_ECUDA. */
int seg_diff_backward(seg_diff* d, const float* rgb_dev, const float* fmap_dev, const double* theta_dev,
                      const float* g_prior_dev, const float* g_sal_dev, float* g_rgb_dev, double* g_theta_dev);

#ifdef __cplusplus
}
#endif
#endif
