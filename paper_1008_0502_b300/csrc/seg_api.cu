// seg_api.cu -- the extern "C" entry points declared in include/seg.h.
//
// A context owns one device arena, carved into the saliency workspace, the
// prior/terms buffers and the min-cut state at creation; no entry point below
// allocates device memory except seg_create and the standalone
// seg_mincut_grid.
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include "seg_internal.cuh"

static void prof_free(seg_ctx* c);

extern "C" int seg_level_dim(int n, int level) {
  for (int l = 0; l < level; ++l) n = (n + 1) / 2;
  return n;
}

extern "C" int seg_default_params(seg_params* p) {
  if (!p) return SEG_EINVAL;
  memset(p, 0, sizeof(*p));
  p->levels = 9;
  p->c_min = 2;
  p->c_max = 4;
  p->d_min = 3;
  p->d_max = 4;
  p->n_orient = 4;
  p->gabor_lambda = 4.0f;
  p->gabor_sigma = 2.0f;
  p->gabor_radius = 6;
  p->norm_tile = 8;
  p->norm_flat = 1e-5f;
  p->w[0] = 1.0f / 3.0f;
  p->w[1] = 1.0f / 6.0f;
  p->w[2] = 1.0f / 6.0f;
  p->w[3] = 1.0f / 3.0f;
  p->cs_opponent_sum = 1;
  p->border_px = 1;
  p->sigma1 = 0.03;
  p->sigma2 = 0.035;
  p->f_sigma = 2.0f;
  p->f_radius = 6;
  p->eps = 1e-4f;
  p->lambda_u = 1.0;
  p->lambda_p = 0.0;
  p->lambda_s = 1.5;
  p->sigma_I = 0.05;
  p->cap_scale = 1000.0;
  p->neighbourhood = 8;
  p->max_cycles = 20000;
  p->global_relabel_every = 1;
  p->local_iters = 12;
  p->use_graph = 1;
  p->gmm_components = 1;
  p->em_iters = 5;
  p->warm_start = 1;
  p->barrier_timeout_us = 4000000;
  p->kmeans_iters = 3;
  p->gmm_update = 1;
  p->relabel_frontier = 0;
  p->cut_tile = 0;
  return SEG_OK;
}

static thread_local char g_last_cuda_error[256];

void seg_note_cuda_error(cudaError_t e, const char* call) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s in %s", cudaGetErrorName(e), call);
}

extern "C" const char* seg_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" const char* seg_strerror(int code) {
  switch (code) {
    case SEG_OK: return "ok";
    case SEG_EINVAL: return "invalid argument";
    case SEG_ENOMEM: return "device memory allocation failed";
    case SEG_ENOTCONVERGED: return "min-cut did not converge within max_cycles";
    case SEG_ECUDA: return "CUDA runtime error";
    case SEG_ETIMEOUT: return "device-side wait timed out";
    case SEG_ECAPACITY: return "capacity outside [0, 2^24]";
    default: return "unknown error";
  }
}

int seg_check_params(const seg_params* p, int H, int W) {
  if (!p) return SEG_EINVAL;
  if (H < 1 || W < 1 || (long long)H * W > (1LL << 26)) return SEG_EINVAL;
  if (p->levels < 2 || p->levels > SEG_MAX_LEVELS) return SEG_EINVAL;
  if (p->c_min < 1 || p->c_max < p->c_min || p->d_min < 1 || p->d_max < p->d_min) return SEG_EINVAL;
  if (p->c_max + p->d_max > p->levels - 1) return SEG_EINVAL;
  if ((p->c_max - p->c_min + 1) * (p->d_max - p->d_min + 1) > SEG_MAX_PAIRS) return SEG_EINVAL;
  if (p->n_orient < 1 || p->n_orient > SEG_MAX_ORIENT) return SEG_EINVAL;
  if (p->gabor_radius < 0 || p->gabor_radius > 8 || !(p->gabor_sigma > 0) || !(p->gabor_lambda > 0))
    return SEG_EINVAL;
  if (p->f_radius < 0 || p->f_radius > 8 || !(p->f_sigma > 0)) return SEG_EINVAL;
  if (p->norm_tile < 1 || p->border_px < 0) return SEG_EINVAL;
  if (p->neighbourhood != 4 && p->neighbourhood != 8) return SEG_EINVAL;
  if (!(p->sigma1 >= 0) || !(p->sigma2 >= 0) || !(p->sigma_I > 0) || !(p->cap_scale > 0)) return SEG_EINVAL;
  if (!(p->eps > 0) || !(p->eps < 0.5f)) return SEG_EINVAL;
  if (p->max_cycles < 1 || p->global_relabel_every < 1 || p->local_iters < 1) return SEG_EINVAL;
  if (p->barrier_timeout_us < 1 || p->barrier_timeout_us > 60000000) return SEG_EINVAL;
  if (p->kmeans_iters < 0 || p->kmeans_iters > 100 || (p->gmm_update != 0 && p->gmm_update != 1)) return SEG_EINVAL;
  if (p->relabel_frontier != 0 && p->relabel_frontier != 1) return SEG_EINVAL;
  if (p->cut_tile < 0 || p->cut_tile >= SEG_CUT_TILES) return SEG_EINVAL;
  if (p->gmm_components < 1 || p->gmm_components > SEG_MAX_GMM || p->em_iters < 0 || p->em_iters > 100)
    return SEG_EINVAL;
  return SEG_OK;
}

// Byte offsets of every buffer in a context's single device arena.
struct ArenaLayout {
  size_t kal, gauss, mom, lut, cnt, prev, cs, ct, ncap, sal, prior, mask, cut, rgb, status, io, flow, warm, mf;
  size_t gmm, empart, emcnt, gvalid, slots;
  size_t total;
};

static int arena_layout(SalWS& sal, int B, int H, int W, const seg_params& p, ArenaLayout& L) {
  size_t sal_bytes = 0;
  int rc = sal_layout(sal, B, H, W, p, &sal_bytes);
  if (rc) return rc;
  const size_t BN = (size_t)H * W * B;
  const int nk = p.neighbourhood / 2;
  size_t off = seg_align(sal_bytes);
  auto take = [&](size_t b) {
    size_t o = off;
    off += seg_align(b);
    return o;
  };
  L.kal = take(B * sizeof(KalmanDev));
  L.gauss = take(B * sizeof(GaussDev));
  L.mom = take((size_t)B * sizeof(double) * pt_part_doubles(H, W));
  L.lut = take(sizeof(int) * 766 * 2);
  L.cnt = take(B * sizeof(unsigned));
  L.prev = take(BN);
  L.cs = take(4 * BN);
  L.ct = take(4 * BN);
  L.ncap = take(4 * BN * nk);
  L.sal = take(4 * BN);
  L.prior = take(4 * BN);
  L.mask = take(BN);
  L.cut = take(8 * B);
  L.rgb = take(3 * BN);
  L.status = take(32);
  L.io = take(sizeof(SegIO));
  L.flow = take(4 * BN * nk);
  L.warm = take(B);
  L.mf = take(mf_bytes(B * H, W, p.neighbourhood, B, p.cut_tile));
  L.gmm = take((size_t)B * 2 * sizeof(GmmDev));
  L.empart = take((size_t)B * 2 * sizeof(double) * pt_em_part_doubles(H, W));
  L.emcnt = take((size_t)B * 2 * sizeof(unsigned));
  L.gvalid = take((size_t)B * 2 * sizeof(int));
  L.slots = take((size_t)B);
  L.total = off;
  return SEG_OK;
}

extern "C" int seg_workspace_bytes(int B, int H, int W, const seg_params* p, size_t* bytes) {
  if (!bytes) return SEG_EINVAL;
  int rc = seg_check_params(p, H, W);
  if (rc) return rc;
  if (B < 1 || (long long)B * H * W > (1LL << 26)) return SEG_EINVAL;
  SalWS sal;
  ArenaLayout L;
  rc = arena_layout(sal, B, H, W, *p, L);
  if (rc) return rc;
  *bytes = L.total;
  return SEG_OK;
}

extern "C" int seg_create(void* stream, int H, int W, const seg_params* p, seg_ctx** out) {
  return seg_create_batch(stream, 1, H, W, p, out);
}

extern "C" int seg_create_batch(void* stream, int B, int H, int W, const seg_params* p, seg_ctx** out) {
  if (!out) return SEG_EINVAL;
  *out = nullptr;
  int rc = seg_check_params(p, H, W);
  if (rc) return rc;
  if (B < 1 || (long long)B * H * W > (1LL << 26)) return SEG_EINVAL;
  seg_ctx* c = (seg_ctx*)calloc(1, sizeof(seg_ctx));
  if (!c) return SEG_ENOMEM;
  c->stream = (cudaStream_t)stream;
  c->B = B;
  c->H = H;
  c->W = W;
  c->N = H * W;
  c->p = *p;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    free(c);
    return SEG_ECUDA;
  }
  ArenaLayout L;
  rc = arena_layout(c->sal, B, H, W, *p, L);
  if (rc) {
    free(c);
    return rc;
  }
  const size_t N = (size_t)c->N, BN = N * B;
  c->mom_blocks = pt_mom_blocks(H, W);
  const size_t off = L.total;
  size_t o_kal = L.kal, o_gauss = L.gauss, o_mom = L.mom, o_lut = L.lut, o_cnt = L.cnt, o_prev = L.prev;
  size_t o_cs = L.cs, o_ct = L.ct, o_ncap = L.ncap, o_sal = L.sal, o_prior = L.prior, o_mask = L.mask;
  size_t o_cut = L.cut, o_rgb = L.rgb, o_status = L.status, o_io = L.io, o_flow = L.flow, o_warm = L.warm;
  size_t o_mf = L.mf;
  char* base = nullptr;
  if (cudaMalloc((void**)&base, off) != cudaSuccess) {
    free(c);
    return SEG_ENOMEM;
  }
  c->arena = base;
  sal_bind(c->sal, base);
  c->kal = (KalmanDev*)(base + o_kal);
  c->gauss = (GaussDev*)(base + o_gauss);
  c->mom_part = (double*)(base + o_mom);
  c->mom_counter = (unsigned*)(base + o_cnt);
  c->lut = (int*)(base + o_lut);
  c->prev_mask = (uint8_t*)(base + o_prev);
  c->cs = (int32_t*)(base + o_cs);
  c->ct = (int32_t*)(base + o_ct);
  c->ncap = (int32_t*)(base + o_ncap);
  c->sal_buf = (float*)(base + o_sal);
  c->prior_buf = (float*)(base + o_prior);
  c->mask_buf = (uint8_t*)(base + o_mask);
  c->cut_buf = (int64_t*)(base + o_cut);
  c->rgb_stage = (uint8_t*)(base + o_rgb);
  c->status = (int*)(base + o_status);
  c->io = (SegIO*)(base + o_io);
  c->flow = (int*)(base + o_flow);
  c->gmm = (GmmDev*)(base + L.gmm);
  c->em_part = (double*)(base + L.empart);
  c->em_counter = (unsigned*)(base + L.emcnt);
  c->gmm_valid = (int*)(base + L.gvalid);
  c->slot_on = (uint8_t*)(base + L.slots);
  c->sal.on = B > 1 ? c->slot_on : nullptr;  // (a single stream is always on)
  c->warm = (unsigned char*)(base + o_warm);
  mf_bind(c->mf, base + o_mf, B * H, W, p->neighbourhood, B, p->cut_tile);
  int* lut = (int*)malloc(sizeof(int) * 766 * 2);
  if (!lut) {
    cudaFree(base);
    free(c);
    return SEG_ENOMEM;
  }
  pt_fill_lut(*p, lut);
  bool ok = cudaMemcpy(c->lut, lut, sizeof(int) * 766 * 2, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && sal_upload_tables(c->sal) == SEG_OK;
  free(lut);
  ok = ok && cudaMemset(c->kal, 0, B * sizeof(KalmanDev)) == cudaSuccess;
  ok = ok && cudaMemset(c->prev_mask, 0, BN) == cudaSuccess;
  ok = ok && cudaMemset(c->status, 0, 32) == cudaSuccess;
  ok = ok && cudaMemset(c->mom_counter, 0, B * sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMemset(c->warm, 0, B) == cudaSuccess;
  ok = ok && cudaMemset(c->em_counter, 0, (size_t)B * 2 * sizeof(unsigned)) == cudaSuccess;
  ok = ok && cudaMemset(c->gmm_valid, 0, (size_t)B * 2 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaMemset(c->slot_on, 1, (size_t)B) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&c->status_host, 32) == cudaSuccess;
  ok = ok && mf_grid_size(B * H, W, p->cut_tile, &c->mf_grid) == SEG_OK;
  if (!ok) {
    if (c->status_host) cudaFreeHost(c->status_host);
    cudaFree(base);
    free(c);
    return SEG_ECUDA;
  }
  *out = c;
  return SEG_OK;
}

static void pipe_free(seg_ctx* c);

extern "C" int seg_destroy(seg_ctx* c) {
  if (!c) return SEG_EINVAL;
  cudaStreamSynchronize(c->stream);
  pipe_free(c);
  if (c->graph_state == 1) cudaGraphExecDestroy(c->gexec);
  prof_free(c);
  cudaFree(c->arena);
  cudaFreeHost(c->status_host);
  free(c);
  return SEG_OK;
}

extern "C" int seg_set_barrier_timeout(seg_ctx* c, int us) {
  if (!c || us < 1 || us > 60000000) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->s_front) SEG_CUDA_TRY(cudaStreamSynchronize(c->s_front));
  if (c->s_back) SEG_CUDA_TRY(cudaStreamSynchronize(c->s_back));
  c->p.barrier_timeout_us = us;
  // the limit is baked into the captured graphs' kernel arguments: capture again
  if (c->graph_state == 1) cudaGraphExecDestroy(c->gexec);
  if (c->graph_state != 0) c->graph_state = 0;
  if (c->pipe_graph == 1)
    for (int k = 0; k < 2; ++k) {
      cudaGraphExecDestroy(c->gf[k]);
      cudaGraphExecDestroy(c->gb[k]);
    }
  if (c->pipe_graph != 0) c->pipe_graph = 0;
  return SEG_OK;
}

extern "C" int seg_set_stream_active(seg_ctx* c, int b, int on) {
  if (!c || b < 0 || b >= c->B || (on != 0 && on != 1)) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaMemsetAsync(c->slot_on + b, on, 1, c->stream));
  if (c->pipe_on) {  // the next frame's saliency (on the front stream) comes after the change too
    cudaEvent_t e;
    SEG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, c->stream);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(c->s_front, e, 0);
    cudaEventDestroy(e);
    SEG_CUDA_TRY(r);
  }
  return SEG_OK;
}

extern "C" int seg_reset(seg_ctx* c) {
  if (!c) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaMemsetAsync(c->kal, 0, c->B * sizeof(KalmanDev), c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->prev_mask, 0, (size_t)c->B * c->N, c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->warm, 0, c->B, c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->gmm_valid, 0, (size_t)c->B * 2 * sizeof(int), c->stream));
  return SEG_OK;
}

extern "C" int seg_reset_stream(seg_ctx* c, int b) {
  if (!c || b < 0 || b >= c->B) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaMemsetAsync(c->kal + b, 0, sizeof(KalmanDev), c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->prev_mask + (size_t)b * c->N, 0, c->N, c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->warm + b, 0, 1, c->stream));
  SEG_CUDA_TRY(cudaMemsetAsync(c->gmm_valid + 2 * b, 0, 2 * sizeof(int), c->stream));
  return SEG_OK;
}

// The B frames of a batch form one (B*H) x W grid for the min cut: links that
// would join two frames have capacity 0 (the terms kernel writes 0 for every
// neighbour outside the frame), so the stacked cut is the B cuts side by side.
static int run_mincut(seg_ctx* c, const int32_t* cs, const int32_t* ct, const int32_t* ncap,
                      uint8_t* mask, uint8_t* mask_state, int64_t* cut, bool init_done = false) {
  // the per-stream path (mask_state set) warm-starts from the stream's last cut
  MFCall m;
  m.st = c->stream;
  m.grid = c->mf_grid;
  m.H = c->B * c->H;
  m.W = c->W;
  m.nbr = c->p.neighbourhood;
  m.cs = cs;
  m.ct = ct;
  m.ncap = ncap;
  m.mask_state = mask_state;
  m.status = c->status;
  m.max_cycles = c->p.max_cycles;
  m.gr_every = c->p.global_relabel_every;
  m.local_iters = c->p.local_iters;
  m.timeout_ns = 1000LL * c->p.barrier_timeout_us;
  m.flow = (mask_state && c->p.warm_start) ? c->flow : nullptr;
  m.warm = m.flow ? c->warm : nullptr;
  m.init_done = init_done;
  m.on = c->sal.on;
  m.frontier = c->p.relabel_frontier;
  if (c->io_mode) {  // mask and cut come from the frame's SegIO; k_set_io zeroed the words
    m.io = c->io;
    m.words_zeroed = true;
  } else {
    m.mask_out = mask;
    m.cut_out = (long long*)(cut ? cut : c->cut_buf);
  }
  return mf_launch(c->mf, m, c->p.cut_tile);
}

// The launch sequence of one frame.  With c->io_mode set (graph capture) every
// frame pointer is nullptr and the kernels read them from c->io.
int seg_ctx_push_launches(seg_ctx* c, const uint8_t* rgb, float* s, float* pr, uint8_t* mask, int64_t* cut) {
  int rc = sal_launch(c, rgb, s, false);
  if (!rc) rc = pt_launch_back(c, s, pr, rgb);
  if (!rc) rc = run_mincut(c, c->cs, c->ct, c->ncap, mask, c->prev_mask, cut, true);
  return rc;
}

// Starts a replay of the captured frame: records the frame's pointers and zeroes
// the per-frame words the graph's kernels accumulate into (FrameWords), in place
// of memset nodes inside the graph.
__global__ void k_set_io(SegIO* io, SegIO v, FrameWords w) {
  const int t = threadIdx.x;
  if (t == 0) {
    *io = v;
    w.bar->count = 0u;
    w.bar->err = 0u;
  }
  if (t < 4) w.flags[t] = 0u;
  for (int b = t; b < w.B; b += blockDim.x) {
    if (w.smax) w.smax[b] = 0;  // (null: the pipelined front zeroes them)
    w.cut_acc[b] = 0ull;
  }
}

// Front of a pipelined frame: its RGB8 pointer and zeroed frame maxima.
__global__ void k_set_front(SegIO* io, const uint8_t* rgb, int* smax, int B) {
  if (threadIdx.x == 0) io->rgb = rgb;
  for (int b = threadIdx.x; b < B; b += blockDim.x) smax[b] = 0;
}

// Captures push_launches once into a CUDA graph (needs a stream that can be
// captured, i.e. not the legacy default stream).  On any failure the context
// stays on eager launches.
static void build_graph(seg_ctx* c) {
  c->graph_state = -1;
  if (!c->p.use_graph || c->stream == nullptr) return;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c->io_mode = 1;
  int rc = seg_ctx_push_launches(c, nullptr, nullptr, nullptr, nullptr, nullptr);
  c->io_mode = 0;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (rc || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return;
  }
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  c->graph_state = 1;
}

static void prof_mark(seg_ctx* c, int k) {
  if (c->prof_on && c->prof_n < c->prof_cap) cudaEventRecord(c->prof_ev[5 * c->prof_n + k], c->stream);
}

extern "C" int seg_push_frame_ev(seg_ctx* c, const uint8_t* rgb, float* sal, float* prior, uint8_t* mask,
                                 int64_t* cut, void* rgb_ready);

extern "C" int seg_push_frame(seg_ctx* c, const uint8_t* rgb, float* sal, float* prior, uint8_t* mask,
                              int64_t* cut) {
  if (!c || !rgb || !mask) return SEG_EINVAL;
  if (c->pipe_on && !c->prof_on) return seg_push_frame_ev(c, rgb, sal, prior, mask, cut, nullptr);
  float* s = sal ? sal : c->sal_buf;
  float* pr = prior ? prior : c->prior_buf;
  if (!c->prof_on) {
    if (c->graph_state == 0) build_graph(c);
    if (c->graph_state == 1) {
      SegIO v = {rgb, s, pr, mask, (long long*)(cut ? cut : c->cut_buf)};
      FrameWords w = {c->sal.smax, c->B, c->mf.cut_acc, c->mf.flags, c->mf.bar};
      k_set_io<<<1, 32, 0, c->stream>>>(c->io, v, w);
      SEG_CUDA_TRY(cudaGetLastError());
      SEG_CUDA_TRY(cudaGraphLaunch(c->gexec, c->stream));
      return SEG_OK;
    }
  }
  prof_mark(c, 0);
  int rc = sal_launch(c, rgb, s, false);
  prof_mark(c, 1);
  if (!rc) rc = pt_launch_prior(c, s, c->prev_mask, 1, 0.0, pr, rgb, true);
  prof_mark(c, 2);
  if (!rc) rc = pt_launch_moments_terms(c, rgb, pr, 0, c->cs, c->ct, c->ncap, true);
  prof_mark(c, 3);
  if (!rc) rc = run_mincut(c, c->cs, c->ct, c->ncap, mask, c->prev_mask, cut, true);
  prof_mark(c, 4);
  if (!rc && c->prof_on && c->prof_n < c->prof_cap) {
    SEG_CUDA_TRY(cudaMemcpyAsync(c->prof_cycles + 7 * c->prof_n, c->status + 1, 7 * sizeof(int),
                                 cudaMemcpyDeviceToDevice, c->stream));
    c->prof_n++;
  }
  return rc;
}

static void prof_free(seg_ctx* c) {
  if (c->prof_ev) {
    for (int i = 0; i < 5 * c->prof_cap; ++i) cudaEventDestroy(c->prof_ev[i]);
    free(c->prof_ev);
    c->prof_ev = nullptr;
  }
  if (c->prof_cycles) cudaFree(c->prof_cycles);
  c->prof_cycles = nullptr;
  c->prof_cap = 0;
}

extern "C" int seg_profile_enable(seg_ctx* c, int on) {
  if (!c) return SEG_EINVAL;
  c->prof_on = 0;
  c->prof_n = 0;
  if (!on) return SEG_OK;
  if (!c->prof_ev) {
    const int cap = 4096;
    c->prof_ev = (cudaEvent_t*)calloc(5 * cap, sizeof(cudaEvent_t));
    if (!c->prof_ev) return SEG_ENOMEM;
    c->prof_cap = cap;
    for (int i = 0; i < 5 * cap; ++i)
      if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) {
        prof_free(c);
        return SEG_ECUDA;
      }
    if (cudaMalloc((void**)&c->prof_cycles, 7 * sizeof(int) * cap) != cudaSuccess) {
      prof_free(c);
      return SEG_ENOMEM;
    }
  }
  c->prof_on = 1;
  return SEG_OK;
}

extern "C" int seg_profile_read(seg_ctx* c, double* stage_ms, int* frames, long long* cycles,
                                float* frame_ms, int max_frames) {
  return seg_profile_read_ex(c, stage_ms, frames, cycles, frame_ms, nullptr, max_frames);
}

extern "C" int seg_profile_read_ex(seg_ctx* c, double* stage_ms, int* frames, long long* cycles,
                                   float* frame_ms, int* mincut_stats, int max_frames) {
  if (!c || !stage_ms || !frames || !cycles) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 4; ++k) stage_ms[k] = 0.0;
  *frames = c->prof_n;
  *cycles = 0;
  if (c->prof_n == 0) return SEG_OK;
  int* cyc = (int*)malloc(7 * sizeof(int) * c->prof_n);
  if (!cyc) return SEG_ENOMEM;
  if (cudaMemcpy(cyc, c->prof_cycles, 7 * sizeof(int) * c->prof_n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    free(cyc);
    return SEG_ECUDA;
  }
  for (int f = 0; f < c->prof_n; ++f) {
    *cycles += cyc[7 * f];
    if (mincut_stats && f < max_frames)
      for (int k = 0; k < 7; ++k) mincut_stats[7 * f + k] = cyc[7 * f + k];
    bool ok = true;
    for (int k = 0; k < 4 && ok; ++k) {
      float ms = 0.f;
      ok = cudaEventElapsedTime(&ms, c->prof_ev[5 * f + k], c->prof_ev[5 * f + k + 1]) == cudaSuccess;
      stage_ms[k] += ms;
    }
    if (ok && frame_ms && f < max_frames) {
      float ms = 0.f;
      ok = cudaEventElapsedTime(&ms, c->prof_ev[5 * f], c->prof_ev[5 * f + 4]) == cudaSuccess;
      frame_ms[f] = ms;
    }
    if (!ok) {
      free(cyc);
      return SEG_ECUDA;
    }
  }
  free(cyc);
  return SEG_OK;
}

extern "C" int seg_sync(seg_ctx* c, int* cycles) {
  if (!c) return SEG_EINVAL;
  if (c->pipe_on) SEG_CUDA_TRY(cudaStreamSynchronize(c->s_front));
  if (c->pipe_on) SEG_CUDA_TRY(cudaStreamSynchronize(c->s_back));
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  SEG_CUDA_TRY(cudaMemcpy(c->status_host, c->status, 32, cudaMemcpyDeviceToHost));
  if (cycles) *cycles = c->status_host[1];
  int code = c->status_host[0];
  if (code) SEG_CUDA_TRY(cudaMemset(c->status, 0, sizeof(int)));
  return code;
}

// ---------------------------------------------------------------- pipelined frames
// Frame t's saliency map does not depend on frame t-1 (only its prior does), so
// it runs on an internal stream ("front") while the context stream finishes
// frame t-1's prior, terms and min cut ("back").  Even and odd frames write their
// S and saliency maximum into separate buffers; the front of frame t waits for
// the back of frame t-2, the last reader of its buffer.
static void pipe_free(seg_ctx* c) {
  c->sal.light_ctas = 0;
  if (!c->pipe_mem && !c->s_front && !c->s_back) return;
  if (c->s_front) cudaStreamSynchronize(c->s_front);
  if (c->s_back) cudaStreamSynchronize(c->s_back);
  for (int k = 0; k < 2; ++k) {
    if (c->pipe_graph == 1) {
      cudaGraphExecDestroy(c->gf[k]);
      cudaGraphExecDestroy(c->gb[k]);
    }
    if (c->ev_front[k]) cudaEventDestroy(c->ev_front[k]);
    if (c->ev_back[k]) cudaEventDestroy(c->ev_back[k]);
    c->ev_front[k] = c->ev_back[k] = nullptr;
  }
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  c->ev_in = nullptr;
  if (c->ev_ctx) cudaEventDestroy(c->ev_ctx);
  c->ev_ctx = nullptr;
  for (int j = 0; j < 3; ++j) {
    if (c->ev_ring[j]) cudaEventDestroy(c->ev_ring[j]);
    c->ev_ring[j] = nullptr;
    c->ring[j] = nullptr;
  }
  if (c->s_front) cudaStreamDestroy(c->s_front);
  c->s_front = nullptr;
  if (c->s_back) cudaStreamDestroy(c->s_back);
  c->s_back = nullptr;
  if (c->pipe_mem) cudaFree(c->pipe_mem);
  c->pipe_mem = nullptr;
  c->pipe_on = 0;
  c->pipe_graph = 0;
  c->sal.S = c->pS[0] ? c->pS[0] : c->sal.S;
  c->sal.salmax = c->psalmax[0] ? c->psalmax[0] : c->sal.salmax;
}

extern "C" int seg_pipeline_enable(seg_ctx* c, int on) {
  if (!c) return SEG_EINVAL;
  if (!on) {
    SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
    pipe_free(c);
    return SEG_OK;
  }
  if (c->pipe_on) return SEG_OK;
  c->sal.light_ctas = 1;  // (the pipelined graphs are captured with it)
  const size_t nS = (size_t)c->sal.hl[c->sal.sS] * c->sal.wl[c->sal.sS] * c->B;
  const size_t o_salmax = seg_align(nS * sizeof(float)), o_io = o_salmax + seg_align(c->B * sizeof(unsigned));
  const size_t o_ring = o_io + seg_align(sizeof(SegIO)), ring_bytes = seg_align((size_t)3 * c->N * c->B);
  char* m = nullptr;
  if (cudaMalloc((void**)&m, o_ring + 3 * ring_bytes) != cudaSuccess) return SEG_ENOMEM;
  for (int j = 0; j < 3; ++j) c->ring[j] = (uint8_t*)(m + o_ring + j * ring_bytes);
  c->ring_t = 0;
  c->pipe_mem = m;
  c->pS[0] = c->sal.S;
  c->psalmax[0] = c->sal.salmax;
  c->pS[1] = (float*)m;
  c->psalmax[1] = (unsigned*)(m + o_salmax);
  c->io_front = (SegIO*)(m + o_io);
  // the front and the back half run on two internal streams created one after the
  // other (the runtime then gives them different hardware queues whatever streams
  // the caller made before)
  bool ok = cudaStreamCreateWithFlags(&c->s_front, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&c->s_back, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k)
    ok = cudaEventCreateWithFlags(&c->ev_front[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_back[k], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_ctx, cudaEventDisableTiming) == cudaSuccess;
  for (int j = 0; j < 3 && ok; ++j)
    ok = cudaEventCreateWithFlags(&c->ev_ring[j], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    pipe_free(c);
    return SEG_ECUDA;
  }
  c->pipe_on = 1;
  c->pipe_graph = 0;
  c->pipe_t = 0;
  return SEG_OK;
}

static void pipe_select(seg_ctx* c, int k) {
  c->sal.S = c->pS[k];
  c->sal.salmax = c->psalmax[k];
}

// Captures the front and back of even and odd frames (four graphs); on any
// failure the context stays on eager launches.
static void pipe_build_graphs(seg_ctx* c) {
  c->pipe_graph = -1;
  if (!c->p.use_graph || c->stream == nullptr) return;
  cudaGraph_t g[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ok = true;
  SegIO* io_back = c->io;
  for (int k = 0; k < 2 && ok; ++k) {
    pipe_select(c, k);
    c->io_mode = 1;
    c->io = c->io_front;
    ok = cudaStreamBeginCapture(c->s_front, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = ok ? sal_run(c->sal, c->s_front, nullptr, false, c->io_front, nullptr, nullptr, false, true) : 0;
    ok = cudaStreamEndCapture(c->s_front, &g[2 * k]) == cudaSuccess && ok && !rc && g[2 * k];
    c->io = io_back;
    if (ok) ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      rc = pt_launch_back(c, nullptr, nullptr, nullptr);
      if (!rc) rc = run_mincut(c, c->cs, c->ct, c->ncap, nullptr, c->prev_mask, nullptr, true);
      ok = cudaStreamEndCapture(c->stream, &g[2 * k + 1]) == cudaSuccess && !rc && g[2 * k + 1];
    }
    c->io_mode = 0;
  }
  int built = 0;
  for (int k = 0; k < 2 && ok; ++k) {
    ok = cudaGraphInstantiate(&c->gf[k], g[2 * k], 0) == cudaSuccess;
    if (ok) {
      ++built;
      ok = cudaGraphInstantiate(&c->gb[k], g[2 * k + 1], 0) == cudaSuccess;
      if (!ok) cudaGraphExecDestroy(c->gf[k]);
      else ++built;
    }
  }
  for (int i = 0; i < 4; ++i)
    if (g[i]) cudaGraphDestroy(g[i]);
  pipe_select(c, 0);
  if (!ok) {
    for (int k = 0; 2 * k + 1 < built; ++k) {
      cudaGraphExecDestroy(c->gf[k]);
      cudaGraphExecDestroy(c->gb[k]);
    }
    cudaGetLastError();
    return;
  }
  c->pipe_graph = 1;
}

extern "C" int seg_push_frame_ev(seg_ctx* c, const uint8_t* rgb, float* sal, float* prior, uint8_t* mask,
                                 int64_t* cut, void* rgb_ready) {
  if (!c || !rgb || !mask) return SEG_EINVAL;
  if (!c->pipe_on || c->prof_on) {
    if (rgb_ready) SEG_CUDA_TRY(cudaStreamWaitEvent(c->stream, (cudaEvent_t)rgb_ready, 0));
    return seg_push_frame(c, rgb, sal, prior, mask, cut);
  }
  float* s = sal ? sal : c->sal_buf;
  float* pr = prior ? prior : c->prior_buf;
  int64_t* ct = cut ? cut : c->cut_buf;
  if (c->pipe_graph == 0) pipe_build_graphs(c);
  const int k = (int)(c->pipe_t & 1);
  // front: after the frame's data and after the back of frame t-2 (last reader of buffer k)
  if (rgb_ready) {
    SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_front, (cudaEvent_t)rgb_ready, 0));
  } else {
    SEG_CUDA_TRY(cudaEventRecord(c->ev_in, c->stream));
    SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_front, c->ev_in, 0));
  }
  SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_front, c->ev_back[k], 0));
  int rc = SEG_OK;
  if (c->pipe_graph == 1) {
    k_set_front<<<1, 32, 0, c->s_front>>>(c->io_front, rgb, c->sal.smax, c->B);
    SEG_CUDA_TRY(cudaGetLastError());
    SEG_CUDA_TRY(cudaGraphLaunch(c->gf[k], c->s_front));
  } else {
    pipe_select(c, k);
    rc = sal_run(c->sal, c->s_front, rgb, false, nullptr, nullptr, nullptr, false, false);
  }
  if (rc) {
    pipe_select(c, 0);
    return rc;
  }
  SEG_CUDA_TRY(cudaEventRecord(c->ev_front[k], c->s_front));
  if (c->pipe_graph == 1) {
    // back, in frame order on the internal back stream, after the frame's front
    // and after the work enqueued on the context stream so far (readers of the
    // output buffers, slot and stream resets); the context stream then waits for
    // it, so the outputs are valid once the context stream passes them
    SEG_CUDA_TRY(cudaEventRecord(c->ev_ctx, c->stream));
    SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_back, c->ev_ctx, 0));
    SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_back, c->ev_front[k], 0));
    SegIO v = {rgb, s, pr, mask, (long long*)ct};
    FrameWords w = {nullptr, c->B, c->mf.cut_acc, c->mf.flags, c->mf.bar};
    k_set_io<<<1, 32, 0, c->s_back>>>(c->io, v, w);
    SEG_CUDA_TRY(cudaGetLastError());
    SEG_CUDA_TRY(cudaGraphLaunch(c->gb[k], c->s_back));
    SEG_CUDA_TRY(cudaEventRecord(c->ev_back[k], c->s_back));
    SEG_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_back[k], 0));
    c->pipe_t++;
    return SEG_OK;
  }
  // eager launches: back, in frame order on the context stream
  SEG_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_front[k], 0));
  {
    pipe_select(c, k);
    rc = pt_launch_back(c, s, pr, rgb);
    if (!rc) rc = run_mincut(c, c->cs, c->ct, c->ncap, mask, c->prev_mask, (int64_t*)ct, true);
    pipe_select(c, 0);
    if (rc) return rc;
  }
  SEG_CUDA_TRY(cudaEventRecord(c->ev_back[k], c->stream));
  c->pipe_t++;
  return SEG_OK;
}

// Asynchronous host-buffer frames (pipelined contexts): the RGB8 frame is copied
// into a slot of a three-frame device ring on the front stream (after the back
// of the frame that last used the slot), the frame is pushed pipelined, and the
// mask and cut are copied back on the context stream.  Nothing waits on the
// host; the host buffers must stay untouched until seg_sync.
extern "C" int seg_push_frame_host_async(seg_ctx* c, const uint8_t* rgb_host, uint8_t* mask_host,
                                         int64_t* cut_host) {
  if (!c || !rgb_host || !mask_host) return SEG_EINVAL;
  if (!c->pipe_on) return SEG_EINVAL;
  const size_t N = (size_t)c->N * c->B;
  const int j = (int)(c->ring_t % 3);
  SEG_CUDA_TRY(cudaStreamWaitEvent(c->s_front, c->ev_ring[j], 0));
  SEG_CUDA_TRY(cudaMemcpyAsync(c->ring[j], rgb_host, 3 * N, cudaMemcpyHostToDevice, c->s_front));
  SEG_CUDA_TRY(cudaEventRecord(c->ev_in, c->s_front));
  int rc = seg_push_frame_ev(c, c->ring[j], c->sal_buf, c->prior_buf, c->mask_buf, c->cut_buf, c->ev_in);
  if (rc) return rc;
  SEG_CUDA_TRY(cudaEventRecord(c->ev_ring[j], c->stream));
  SEG_CUDA_TRY(cudaMemcpyAsync(mask_host, c->mask_buf, N, cudaMemcpyDeviceToHost, c->stream));
  if (cut_host) SEG_CUDA_TRY(cudaMemcpyAsync(cut_host, c->cut_buf, 8 * c->B, cudaMemcpyDeviceToHost, c->stream));
  c->ring_t++;
  return SEG_OK;
}

extern "C" int seg_push_frame_host(seg_ctx* c, const uint8_t* rgb_host, float* sal_host,
                                   float* prior_host, uint8_t* mask_host, int64_t* cut_host) {
  if (!c || !rgb_host || !mask_host) return SEG_EINVAL;
  cudaStream_t st = c->stream;
  size_t N = (size_t)c->N * c->B;
  SEG_CUDA_TRY(cudaMemcpyAsync(c->rgb_stage, rgb_host, 3 * N, cudaMemcpyHostToDevice, st));
  int rc = seg_push_frame(c, c->rgb_stage, c->sal_buf, c->prior_buf, c->mask_buf, c->cut_buf);
  if (rc) return rc;
  SEG_CUDA_TRY(cudaMemcpyAsync(mask_host, c->mask_buf, N, cudaMemcpyDeviceToHost, st));
  if (cut_host) SEG_CUDA_TRY(cudaMemcpyAsync(cut_host, c->cut_buf, 8 * c->B, cudaMemcpyDeviceToHost, st));
  if (sal_host) SEG_CUDA_TRY(cudaMemcpyAsync(sal_host, c->sal_buf, 4 * N, cudaMemcpyDeviceToHost, st));
  if (prior_host)
    SEG_CUDA_TRY(cudaMemcpyAsync(prior_host, c->prior_buf, 4 * N, cudaMemcpyDeviceToHost, st));
  return seg_sync(c, nullptr);
}

#define SEG_STATE_MAGIC 0x53454732u  // "SEG2"

// Byte layout: {magic, H, W, B} (4 x u32), then per stream {t (i32), pad, P (f64)},
// then the B previous masks (B*H*W bytes).
static size_t state_bytes(const seg_ctx* c) { return 16 + 16 * (size_t)c->B + (size_t)c->B * c->N; }

extern "C" int seg_get_state(seg_ctx* c, void* buf, size_t* n) {
  if (!c || !n) return SEG_EINVAL;
  size_t need = state_bytes(c);
  if (!buf) {
    *n = need;
    return SEG_OK;
  }
  if (*n < need) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  char* b = (char*)buf;
  uint32_t hdr[4] = {SEG_STATE_MAGIC, (uint32_t)c->H, (uint32_t)c->W, (uint32_t)c->B};
  memcpy(b, hdr, 16);
  for (int i = 0; i < c->B; ++i) {
    KalmanDev k;
    SEG_CUDA_TRY(cudaMemcpy(&k, c->kal + i, sizeof(k), cudaMemcpyDeviceToHost));
    int32_t rec[2] = {k.t, 0};
    memcpy(b + 16 + 16 * i, rec, 8);
    memcpy(b + 16 + 16 * i + 8, &k.P, 8);
  }
  SEG_CUDA_TRY(cudaMemcpy(b + 16 + 16 * (size_t)c->B, c->prev_mask, (size_t)c->B * c->N, cudaMemcpyDeviceToHost));
  *n = need;
  return SEG_OK;
}

extern "C" int seg_set_state(seg_ctx* c, const void* buf, size_t n) {
  if (!c || !buf || n != state_bytes(c)) return SEG_EINVAL;
  const char* b = (const char*)buf;
  uint32_t hdr[4];
  memcpy(hdr, b, 16);
  if (hdr[0] != SEG_STATE_MAGIC || hdr[1] != (uint32_t)c->H || hdr[2] != (uint32_t)c->W ||
      hdr[3] != (uint32_t)c->B)
    return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->B; ++i) {
    KalmanDev k;
    memset(&k, 0, sizeof(k));
    int32_t rec[2];
    memcpy(rec, b + 16 + 16 * i, 8);
    k.t = rec[0];
    memcpy(&k.P, b + 16 + 16 * i + 8, 8);
    SEG_CUDA_TRY(cudaMemcpy(c->kal + i, &k, sizeof(k), cudaMemcpyHostToDevice));
  }
  SEG_CUDA_TRY(cudaMemcpy(c->prev_mask, b + 16 + 16 * (size_t)c->B, (size_t)c->B * c->N, cudaMemcpyHostToDevice));
  SEG_CUDA_TRY(cudaMemset(c->warm, 0, c->B));  // flows are not part of the state: next cut starts cold
  // nor are the colour mixtures: the next frame's EM starts from the k-means start
  SEG_CUDA_TRY(cudaMemset(c->gmm_valid, 0, (size_t)c->B * 2 * sizeof(int)));
  return SEG_OK;
}

extern "C" int seg_saliency(seg_ctx* c, const uint8_t* rgb, float* sal) {
  if (!c || !rgb || !sal) return SEG_EINVAL;
  return sal_launch(c, rgb, sal, true);
}

extern "C" int seg_saliency_grid(void* stream, int H, int W, const seg_params* p, const uint8_t* rgb,
                                 float* sal) {
  if (!rgb || !sal) return SEG_EINVAL;
  int rc = seg_check_params(p, H, W);
  if (rc) return rc;
  SalWS s;
  size_t bytes = 0;
  rc = sal_layout(s, 1, H, W, *p, &bytes);
  if (rc) return rc;
  char* base = nullptr;
  if (cudaMalloc((void**)&base, bytes) != cudaSuccess) return SEG_ENOMEM;
  sal_bind(s, base);
  cudaStream_t st = (cudaStream_t)stream;
  rc = sal_upload_tables(s);
  if (!rc) rc = sal_run(s, st, rgb, false, nullptr, nullptr, sal, true);
  if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = SEG_ECUDA;
  cudaFree(base);
  return rc;
}

extern "C" int seg_prior(seg_ctx* c, const float* sal, const uint8_t* prev_mask, double w_f,
                         float* prior) {
  if (!c || !sal || !prior || !(w_f >= 0.0 && w_f <= 1.0) || c->B != 1) return SEG_EINVAL;
  if (w_f != 0.0 && !prev_mask) return SEG_EINVAL;
  int rc = pt_launch_salmax(c, sal);  // q = saliency / max(saliency) of THIS map
  return rc ? rc : pt_launch_prior(c, sal, prev_mask, 0, w_f, prior, nullptr);
}

extern "C" int seg_terms(seg_ctx* c, const uint8_t* rgb, const float* prior, int32_t* cs, int32_t* ct,
                         int32_t* ncap) {
  if (!c || !rgb || !prior || !cs || !ct || !ncap || c->B != 1) return SEG_EINVAL;
  return pt_launch_moments_terms(c, rgb, prior, 1, cs, ct, ncap);
}

extern "C" int seg_mincut(seg_ctx* c, const int32_t* cs, const int32_t* ct, const int32_t* ncap,
                          uint8_t* mask, int64_t* cut) {
  if (!c || !cs || !ct || !ncap || !mask || c->B != 1) return SEG_EINVAL;
  return run_mincut(c, cs, ct, ncap, mask, nullptr, cut);
}

extern "C" int seg_mincut_grid(void* stream, int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                               const int32_t* ncap, uint8_t* mask, int64_t* cut, int max_cycles,
                               int* cycles) {
  if (H < 1 || W < 1 || (long long)H * W > (1LL << 26) || (nbr != 4 && nbr != 8)) return SEG_EINVAL;
  if (!cs || !ct || !ncap || !mask) return SEG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  seg_params d;
  seg_default_params(&d);
  int grid = 0;
  int rc = mf_grid_size(H, W, d.cut_tile, &grid);
  if (rc) return rc;
  size_t mfb = mf_bytes(H, W, nbr, 1, d.cut_tile);
  char* base = nullptr;
  if (cudaMalloc((void**)&base, seg_align(mfb) + 256) != cudaSuccess) return SEG_ENOMEM;
  MFWS m;
  mf_bind(m, base, H, W, nbr, 1, d.cut_tile);
  int* status = (int*)(base + seg_align(mfb));
  long long* cut_tmp = (long long*)(base + seg_align(mfb) + 128);
  rc = SEG_OK;
  if (cudaMemsetAsync(status, 0, 32, st) != cudaSuccess) rc = SEG_ECUDA;
  if (!rc) {
    MFCall k;
    k.st = st;
    k.grid = grid;
    k.H = H;
    k.W = W;
    k.nbr = nbr;
    k.cs = cs;
    k.ct = ct;
    k.ncap = ncap;
    k.mask_out = mask;
    k.cut_out = cut ? (long long*)cut : cut_tmp;
    k.status = status;
    k.max_cycles = max_cycles > 0 ? max_cycles : d.max_cycles;
    k.gr_every = d.global_relabel_every;
    k.local_iters = d.local_iters;
    k.timeout_ns = 1000LL * d.barrier_timeout_us;
    k.frontier = d.relabel_frontier;
    rc = mf_launch(m, k, d.cut_tile);
  }
  int hs[4] = {0, 0, 0, 0};
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = SEG_ECUDA;
  if (!rc && cudaMemcpy(hs, status, 16, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SEG_ECUDA;
  cudaFree(base);
  if (rc) return rc;
  if (cycles) *cycles = hs[1];
  return hs[0];
}

extern "C" int seg_debug_copy(seg_ctx* c, int which, int index, float* dst, size_t n) {
  if (!c || !dst) return SEG_EINVAL;
  const SalWS& s = c->sal;
  const float* src = nullptr;
  size_t cnt = 0;
  int sS = s.sS;
  if (which == 0) {
    int ch = index / 16, l = index % 16;
    if (ch < 0 || ch > 2 || l < 1 || l >= s.L) return SEG_EINVAL;
    src = s.pyr[ch][l];
    cnt = (size_t)s.hl[l] * s.wl[l];
  } else if (which == 1) {
    int k = index / 16, l = index % 16;
    if (k < 0 || k >= s.no || l < s.c_min || l > s.s_max) return SEG_EINVAL;
    src = s.ori[k][l];
    cnt = (size_t)s.hl[l] * s.wl[l];
  } else if (which == 2) {
    if (index < 0 || index > 3) return SEG_EINVAL;
    cnt = (size_t)s.hl[sS] * s.wl[sS];
    src = s.consp + index * cnt;
  } else if (which == 3) {
    src = s.S;
    cnt = (size_t)s.hl[sS] * s.wl[sS];
  } else {
    return SEG_EINVAL;
  }
  if (n != cnt) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(c->stream));
  SEG_CUDA_TRY(cudaMemcpy(dst, src, cnt * sizeof(float), cudaMemcpyDeviceToHost));
  return SEG_OK;
}
