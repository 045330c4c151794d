// seg_internal.cuh -- shared declarations of the CUDA path (sm_103a).
//
// The library is one shared object built from saliency.cu, prior_terms.cu,
// maxflow.cu and seg_api.cu.  This header holds the context layout, the
// kernel-argument structs and small device helpers.  Nothing here is shared
// with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/seg.h"

#define SEG_MAX_LEVELS 16
#define SEG_MAX_ORIENT 8
#define SEG_MAX_TAPS 17  // radius <= 8
#define SEG_MAX_PAIRS 64
#define SEG_MAX_MAPS (SEG_MAX_PAIRS * (3 + SEG_MAX_ORIENT))
#define SEG_INF_H 0x3fffffff

// Slots of a batch that hold no stream (on[fb] == 0) are skipped: a kernel's
// CTAs of such a frame return at once (on == nullptr: every frame is on).
#define SEG_SLOT_OFF(on, fb) ((on) != nullptr && !(on)[fb])

// Programmatic dependent launch: the frame's kernels are launched with
// programmatic stream serialisation, so each one is scheduled while its
// predecessor is still running.  Each such kernel first waits for its
// predecessor's completion and memory (griddepcontrol.wait: a no-op without a
// programmatic dependency), then lets its own successor be scheduled.
__device__ __forceinline__ void seg_pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline cudaError_t seg_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Records a failed CUDA call (its name and the call's text) for
// seg_last_cuda_error, per host thread.
void seg_note_cuda_error(cudaError_t e, const char* call);

#define SEG_CUDA_TRY(expr)                 \
  do {                                     \
    cudaError_t _e = (expr);               \
    if (_e != cudaSuccess) {               \
      seg_note_cuda_error(_e, #expr);      \
      return SEG_ECUDA;                    \
    }                                      \
  } while (0)

__device__ __forceinline__ int seg_clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Source coordinate of the half-pixel-centred resampling used by every
// across-scale interpolation: src = (dst + 0.5) * ns / nd - 0.5, clamped to
// [0, ns-1].  Computed from integers, so the cell index is exact and the
// fraction carries a single rounding.
__device__ __forceinline__ void seg_src_coord(int d, int ns, int nd, int& i0, int& i1, float& f) {
  int num = (2 * d + 1) * ns - nd;  // src = num / (2 nd)
  if (num <= 0) {
    i0 = 0;
    i1 = 0;
    f = 0.f;
    return;
  }
  int den = 2 * nd;
  int q = num / den;
  if (q >= ns - 1) {
    i0 = ns - 1;
    i1 = ns - 1;
    f = 0.f;
    return;
  }
  i0 = q;
  i1 = q + 1;
  f = (float)(num - q * den) / (float)den;
}

__device__ __forceinline__ float seg_bilinear(const float* src, int hs, int ws, int y, int x,
                                              int hd, int wd) {
  int y0, y1, x0, x1;
  float fy, fx;
  seg_src_coord(y, hs, hd, y0, y1, fy);
  seg_src_coord(x, ws, wd, x0, x1, fx);
  float top = (1.f - fx) * src[y0 * ws + x0] + fx * src[y0 * ws + x1];
  float bot = (1.f - fx) * src[y1 * ws + x0] + fx * src[y1 * ws + x1];
  return (1.f - fy) * top + fy * bot;
}

// Precomputed form of seg_src_coord for every output row/column of one
// resampling: .x packs i0 | i1 << 16, .y holds the fraction's bits.  Built on
// the host with the same integer arithmetic and one IEEE division, so a table
// lookup gives exactly what seg_src_coord computes.
__host__ __device__ inline int2 seg_rs_entry(int d, int ns, int nd) {
  int i0, i1;
  float f;
  int num = (2 * d + 1) * ns - nd;
  if (num <= 0) {
    i0 = i1 = 0;
    f = 0.f;
  } else {
    int den = 2 * nd, q = num / den;
    if (q >= ns - 1) {
      i0 = i1 = ns - 1;
      f = 0.f;
    } else {
      i0 = q;
      i1 = q + 1;
      f = (float)(num - q * den) / (float)den;
    }
  }
  int2 e;
  e.x = i0 | (i1 << 16);
  union {
    float f;
    int i;
  } u;
  u.f = f;
  e.y = u.i;
  return e;
}

// Bilinear sample (same arithmetic as seg_bilinear) from row/column tables.
__device__ __forceinline__ float seg_bilinear_t(const float* src, int ws, int2 ry, int2 rx) {
  const int y0 = ry.x & 0xffff, y1 = ry.x >> 16, x0 = rx.x & 0xffff, x1 = rx.x >> 16;
  const float fy = __int_as_float(ry.y), fx = __int_as_float(rx.y);
  float top = (1.f - fx) * src[y0 * ws + x0] + fx * src[y0 * ws + x1];
  float bot = (1.f - fx) * src[y1 * ws + x0] + fx * src[y1 * ws + x1];
  return (1.f - fy) * top + fy * bot;
}

// Order-preserving map from float to unsigned (so atomicMax works for any sign).
__device__ __forceinline__ unsigned f2key(float x) {
  unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Output rows (or columns) d of a bilinear up-sampling ns -> nd at which the
// interpolant can peak: the first and last samples of every source cell (within
// one cell the interpolant is bilinear, so its maximum over the cell's samples
// lies on those rows and columns), plus both ends.
__device__ __forceinline__ int seg_up_cell(int d, int ns, int nd) {
  int i0, i1;
  float f;
  seg_src_coord(d, ns, nd, i0, i1, f);
  return (i0 == i1) ? (i0 == 0 && d < nd / 2 ? -1 : ns) : i0;
}
__device__ __forceinline__ bool seg_up_candidate(int d, int ns, int nd) {
  int id = seg_up_cell(d, ns, nd);
  return d == 0 || d == nd - 1 || seg_up_cell(d - 1, ns, nd) != id || seg_up_cell(d + 1, ns, nd) != id;
}

__device__ __forceinline__ double seg_warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float seg_warp_max_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float seg_warp_min_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float seg_warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- saliency
// Separable factors of the zero-mean complex Gabor (rank 2 per orientation):
//   k_theta(u,v) = hx(u) vy(v) - kappa * g0(u) g0(v)
// with hx(u) = g(u) e^{i w u cos theta}/sum g, vy(v) = g(v) e^{i w v sin theta}/sum g,
// g0 = g / sum g and kappa = (sum hx)(sum vy).
struct GaborTaps {
  int R;
  int no;
  float g0[SEG_MAX_TAPS];
  float hx_re[SEG_MAX_ORIENT][SEG_MAX_TAPS], hx_im[SEG_MAX_ORIENT][SEG_MAX_TAPS];
  float vy_re[SEG_MAX_ORIENT][SEG_MAX_TAPS], vy_im[SEG_MAX_ORIENT][SEG_MAX_TAPS];
  float kap_re[SEG_MAX_ORIENT], kap_im[SEG_MAX_ORIENT];
};

// Per-context saliency workspace.  Level-0 feature planes are never stored:
// the first kernel fuses feature extraction with the first REDUCE.
struct SalWS {
  int B;  // frames of the batch (same size); every per-frame buffer holds B frames
  const uint8_t* on;  // [B] slots holding a stream (nullptr: all; batch contexts only)
  int light_ctas;  // sharing the GPU with a pipelined back half: smaller CTAs where that pays
  int H, W, L, c_min, c_max, d_min, d_max, no, s_max, sS, tile;
  int opp_sum;
  float flat;
  float w[4];
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  float* pyr[3][SEG_MAX_LEVELS];              // levels 1..L-1
  float* ori[SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // levels c_min..s_max
  float2* oc[SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // complex Gabor responses (backward form only, else null)
  int npairs, nch, nmaps;                      // nch = 3 + no channels, nmaps = npairs * nch
  int pair_c[SEG_MAX_PAIRS], pair_s[SEG_MAX_PAIRS];
  unsigned* mm;  // [nmaps][2]: min and max as float bits (maps are >= 0)
  float* tpart;  // [nbands_total]: per-band sums of tile maxima
  int nbands_total;
  float* acc[2];  // ping-pong channel accumulators at scale c (nch planes)
  float* acc_final;  // the accumulator holding scale c_max (sigma_S): acc[(c_max - c_min) & 1]
  float* consp;   // 4 planes at sigma_S: N(C_I), N(C_RG), N(C_BY), N(C_O)
  float* csum;    // scratch plane at sigma_S
  float* S;       // combined map at sigma_S
  unsigned* salmax;  // max of the upsampled saliency (float bits)
  int* smax;         // frame max of r+g+b
  int consp_staged;  // k_consp stages its maps in shared memory
  size_t consp_smem; // its dynamic shared memory
  int consp_cl;       // the four-CTA cluster form of k_consp runs instead
  size_t consp_cl_smem;
  GaborTaps taps;
  // row-staged up-sampling (k_upsample_rows): its dynamic shared memory (0: the
  // per-pixel kernel)
  size_t up_smem;
  // resampling tables (seg_rs_entry): per center-surround pair p, rows
  // hl[s]->hl[c] at rs + rs_row[p] and columns wl[s]->wl[c] at rs + rs_col[p];
  // the final up-sampling S -> H x W at rs + rs_frow / rs + rs_fcol
  int2* rs;
  int rs_row[SEG_MAX_PAIRS], rs_col[SEG_MAX_PAIRS], rs_frow, rs_fcol, rs_n;
};

// Frame-varying pointers of seg_push_frame, read by the kernels of the captured
// per-frame CUDA graph (a kernel argument that is nullptr is taken from here).
struct SegIO {
  const uint8_t* rgb;
  float* sal;
  float* prior;
  uint8_t* mask;
  long long* cut;
};

// ---------------------------------------------------------------- prior / terms
struct KalmanDev {
  double P;  // sigma^2_xi1(t-1)
  int t;     // frame index
  int pad;
};

struct GaussDev {
  double mu[2][3];
  double sw[2];      // total prior weight per label
  float muf[2][3];
  float linv[2][6];  // lower-triangular inverse Cholesky factor: l00 l10 l11 l20 l21 l22
  float lconst[2];   // 1/2 log det + 3/2 log 2 pi
  int degenerate;    // bit a: label a has zero total weight
};

// M-component colour model of one label of one frame (Sec. 4 / Sec. 7.3 EM).
#define SEG_MAX_GMM 3
struct GmmDev {
  float mu[SEG_MAX_GMM][3];
  float linv[SEG_MAX_GMM][6];  // inverse Cholesky factor, l00 l10 l11 l20 l21 l22
  float lc[SEG_MAX_GMM];       // log pi - 1/2 log det Sigma - 3/2 log 2 pi
  double logdet[SEG_MAX_GMM];  // log det Sigma (reused by components that stop moving)
};

// ---------------------------------------------------------------- max-flow
// Tile shapes of the min cut (seg_params.cut_tile), one compiled copy of
// maxflow.cu each: 0 = 32x16, 1 = 32x8, 2 = 64x8 nodes (one thread per node).
#define SEG_CUT_TILES 3

// Grid barrier words, one 128-byte line: the arrival counter (zeroed before
// every launch, never reset inside one) and the error word a CTA sets when its
// wait times out.
struct GridBar {
  unsigned int count;
  unsigned int err;
  unsigned int pad[30];
};

__device__ __forceinline__ long long seg_now() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch with a bounded wait.  Returns false
// (in every thread of the CTA) once the wait timed out here or in another CTA.
// Barrier k of a launch (k = 1, 2, ..; *epoch_smem counts them, thread 0 only)
// is passed once the counter reaches k * gridDim.x (modulo 2^32): every CTA adds 1 with a
// release reduction on arrival and polls the counter with acquire loads, so a
// barrier costs the reduction and one poll round trip (no generation word to
// read before arriving, no status word after).  The CTA barriers before and
// after carry the other threads' writes (release and acquire are cumulative).
// Every 8 polls the waiter reads the clock and the error word: on its own
// timeout it records SEG_ETIMEOUT in status[0] and sets the error word; a CTA
// that sees the error word set returns false too (a CTA that passed the barrier
// before the error was set sees it at its next barrier, where the CTA that timed
// out never arrives).  ok: a shared-memory word of the CTA.
__device__ __forceinline__ bool seg_grid_sync(GridBar* bar, int* status, long long timeout_ns, int* ok_smem,
                                              unsigned int* epoch_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = (*epoch_smem + 1u) * gridDim.x;
    *epoch_smem += 1u;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
    int ok = 1;
    const long long t0 = seg_now();
    for (unsigned int k = 0;; ++k) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((int)(cur - target) >= 0) break;  // (the count runs at most gridDim.x past target; wraps safely)
      if ((k & 7u) == 7u) {
        unsigned int e;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(e) : "l"(&bar->err) : "memory");
        if (e) {
          ok = 0;
          break;
        }
        if (seg_now() - t0 > timeout_ns) {
          atomicCAS(&status[0], 0, SEG_ETIMEOUT);
          asm volatile("st.relaxed.gpu.global.u32 [%0], 1;" ::"l"(&bar->err) : "memory");
          ok = 0;
          break;
        }
      }
    }
    *ok_smem = ok;
  }
  __syncthreads();
  return *ok_smem != 0;
}

struct MFArgs {
  int H, W, N, ndir;
  int nframes, frame_h;  // a batch of frames stacked vertically: H = nframes * frame_h
  int ntx, nty;
  const int32_t* cs;
  const int32_t* ct;
  const int32_t* ncap;
  int* e;
  int* h;
  int* rt;
  int* r;             // ndir planes of N residual capacities
  unsigned char* rm;  // residual bitmask per node
  unsigned char* z;   // reach flags
  uint8_t* mask_out;
  uint8_t* mask_state;  // nullable second copy of the mask
  long long* cut_out;   // nullable
  const SegIO* io;      // mask_out / cut_out == nullptr: take them from here
  int* flow;            // nullable: nbr/2 planes of n-link flows (warm start in, final out)
  unsigned char* warm;  // per frame: flow holds the previous frame's flows
  unsigned long long* cut_acc;
  unsigned int* flags;  // [3] rotating round counters
  int* tstamp;           // per tile: last round (epoch) in which a fixpoint changed it
  unsigned char* tact;   // per tile: may hold an active node
  GridBar* bar;
  int* status;  // [0] error code, [1] cycles, [2] global relabels, [3] fixpoint rounds,
               // [4..7] time in init / global relabel / discharge / reach, 0.1 us units
  int max_cycles, gr_every, local_iters;
  long long timeout_ns;
  int init_done;  // e, rt and r already hold the initial residual graph (formed by the terms kernel)
  const uint8_t* on;  // [nframes] nullable: 0 = an empty slot, its frame's rows are neither read nor written
  int frontier;       // 1: fixpoint rounds from the third on take their tiles from a compacted queue
  int* tq;            // [2][ntiles] the tile queues of consecutive rounds
  int* tqs;           // [ntiles] epoch of the round that last queued the tile
};

struct MFWS {
  int* e;
  int* h;
  int* rt;
  int* r;
  unsigned char* rm;
  unsigned char* z;
  unsigned long long* cut_acc;  // [nframes]
  unsigned int* flags;
  int* tstamp;
  unsigned char* tact;
  GridBar* bar;
  int* tq;   // [2][ntiles]
  int* tqs;  // [ntiles]
  int nframes;
};

// ---------------------------------------------------------------- context
struct seg_ctx {
  cudaStream_t stream;
  int device;
  int B;  // streams (frames per step) of the batch, all H x W
  int H, W, N;
  seg_params p;
  void* arena;
  SalWS sal;
  KalmanDev* kal;
  GaussDev* gauss;
  double* mom_part;
  unsigned* mom_counter;  // last-CTA counter of the moment passes (returns to 0)
  GmmDev* gmm;            // [B][2] colour mixtures (gmm_components > 1)
  int* gmm_valid;         // [B][2] the mixture is a fitted one (the next frame's EM may start from it)
  uint8_t* slot_on;       // [B] 1: the slot holds a stream (batch contexts: empty slots are skipped)
  double* em_part;        // [B][2][em partial doubles]
  unsigned* em_counter;   // [B][2]
  int mom_blocks;
  int* lut;  // [766][2] n-link capacities by |delta(r+g+b)| and diagonal flag
  uint8_t* prev_mask;
  int32_t *cs, *ct, *ncap;
  float *sal_buf, *prior_buf;
  uint8_t* mask_buf;
  int64_t* cut_buf;
  uint8_t* rgb_stage;
  MFWS mf;
  int mf_grid;
  // captured per-frame graph of seg_push_frame
  SegIO* io;
  int io_mode;       // launchers pass nullptr for frame pointers (graph capture)
  int graph_state;   // 0 not built, 1 ready, -1 unavailable (eager launches)
  cudaGraphExec_t gexec;
  int* status;       // device [8]
  int* status_host;  // pinned [8]
  int* flow;            // warm start: nbr/2 planes of B*N n-link flows
  unsigned char* warm;  // [B] flow valid for the stream
  // pipelined frames (seg_pipeline_enable): frame t+1's saliency on s_front
  // while frame t's prior, terms and cut run on s_back (captured graphs) or on
  // stream (eager launches); stream waits for every frame's back
  int pipe_on;
  cudaStream_t s_front, s_back;
  cudaEvent_t ev_front[2], ev_back[2], ev_in, ev_ctx;
  float* pS[2];           // S of even / odd frames ([0] is sal.S)
  unsigned* psalmax[2];   // saliency maxima of even / odd frames ([0] is sal.salmax)
  SegIO* io_front;        // the front's frame pointers (graph replays)
  void* pipe_mem;
  int pipe_graph;         // 0 not built, 1 ready, -1 eager launches
  cudaGraphExec_t gf[2], gb[2];
  unsigned long long pipe_t;
  uint8_t* ring[3];       // RGB8 staging ring of the asynchronous host-buffer entry point
  cudaEvent_t ev_ring[3]; // back of the frame that last read each slot
  unsigned long long ring_t;
  // optional per-stage timing (seg_profile_enable)
  int prof_on, prof_n, prof_cap;
  cudaEvent_t* prof_ev;  // 5 per frame
  int* prof_cycles;      // device [prof_cap]
};

// ---------------------------------------------------------------- launchers
int seg_check_params(const seg_params* p, int H, int W);
int sal_layout(SalWS& s, int B, int H, int W, const seg_params& p, size_t* bytes, bool keep_complex = false);
void sal_bind(SalWS& s, char* base);
int sal_upload_tables(const SalWS& s);
// upsample == false: stop at S and the saliency maximum (the prior kernel then
// evaluates the saliency map itself); nullptr + c->io_mode: pointers from c->io
int sal_launch(seg_ctx* c, const uint8_t* rgb, float* sal_out, bool upsample);
// The saliency pipeline on a workspace: rgb is RGB8 (rgb_f32 = false) or float
// RGB in [0, 255]; io supplies a null rgb / sal_out (RGB8 only); wdev, if set,
// holds the four channel weights (double) on the device.
int sal_run(SalWS& s, cudaStream_t st, const void* rgb, bool rgb_f32, const SegIO* io, const double* wdev,
            float* sal_out, bool upsample, bool smax_zeroed = false);

int pt_mom_blocks(int H, int W);
int pt_launch_salmax(seg_ctx* c, const float* sal);
// rgb_moments != nullptr: also run the first moment pass (and, with use_kalman,
// advance the Kalman variance) inside the prior kernel
// from_S: compute the saliency map from the context's S (writing it to sal when
// sal is non-null) instead of reading sal
int pt_launch_prior(seg_ctx* c, const float* sal, const uint8_t* prev_mask, int use_kalman,
                    double wf_host, float* prior, const uint8_t* rgb_moments, bool from_S = false);
int pt_launch_moments_terms(seg_ctx* c, const uint8_t* rgb, const float* prior, int first_pass,
                            int32_t* cs, int32_t* ct, int32_t* ncap, bool mf_init = false);
int pt_part_doubles(int H, int W);
int pt_launch_back(seg_ctx* c, const float* sal, float* prior, const uint8_t* rgb);
// The launch sequence of one frame of c (saliency, prior, moments + terms, min
// cut) on c->stream; with c->io_mode set every frame pointer is nullptr and the
// kernels read them from c->io (graph capture).
int seg_ctx_push_launches(seg_ctx* c, const uint8_t* rgb, float* s, float* pr, uint8_t* mask, int64_t* cut);
int pt_em_part_doubles(int H, int W);
void pt_fill_lut(const seg_params& p, int* lut_host);

// One min-cut launch.  H is the stacked height (nframes frames of H / nframes
// rows each, nframes from the workspace).
struct MFCall {
  cudaStream_t st = nullptr;
  int grid = 0, H = 0, W = 0, nbr = 8;
  const int32_t* cs = nullptr;  // the capacities (read unless init_done)
  const int32_t* ct = nullptr;
  const int32_t* ncap = nullptr;
  uint8_t* mask_out = nullptr;    // nullptr: io->mask
  uint8_t* mask_state = nullptr;  // nullable second copy of the mask
  long long* cut_out = nullptr;   // nullptr: io->cut (or none)
  int* status = nullptr;          // [8] error code, cycles, relabels, rounds, phase times
  int max_cycles = 1, gr_every = 1, local_iters = 1;
  long long timeout_ns = 0;       // grid-barrier wait limit
  const SegIO* io = nullptr;
  int* flow = nullptr;            // warm start: n-link flows in and out (nullable)
  unsigned char* warm = nullptr;  // per frame: flow holds the previous frame's flows
  bool words_zeroed = false;      // the caller zeroed cut sums, round flags and barrier
  bool init_done = false;         // the terms kernel formed the initial residual graph
  const uint8_t* on = nullptr;    // [nframes] slots holding a stream (nullable: all)
  int frontier = 0;               // seg_params.relabel_frontier
};

// The per-frame words a replay of a captured frame zeroes before its kernels
// accumulate into them: frame maxima of r+g+b (nullable), the min cut's
// per-frame cut sums, round flags and grid-barrier counter.
struct FrameWords {
  int* smax;
  int B;
  unsigned long long* cut_acc;
  unsigned int* flags;
  GridBar* bar;
};

// Dispatch on the tile shape (maxflow_shapes.cu); every other argument as in
// the shape's own copy.
size_t mf_bytes(int H, int W, int ndir, int nframes, int shape);
void mf_bind(MFWS& m, char* base, int H, int W, int ndir, int nframes, int shape);
int mf_grid_size(int H, int W, int shape, int* grid);
int mf_launch(const MFWS& m, const MFCall& c, int shape);

static inline size_t seg_align(size_t x) { return (x + 255) & ~(size_t)255; }
