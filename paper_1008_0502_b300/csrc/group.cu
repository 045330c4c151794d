// group.cu -- seg_group: several contexts (batch contexts of different
// resolutions, say) advanced by one CUDA graph launch per frame step.
//
// At creation the group captures every member's frame launch sequence (the one
// seg_push_frame runs) as parallel branches of one graph, behind a root kernel
// that writes each member's frame pointers and zeroes its per-frame words (what
// k_set_io does before a member's own graph).  A step updates the root's
// arguments on the instantiated graph and launches it once.  The members' state
// (previous masks, Kalman variances, flows, slot flags) stays in the members;
// their streams are ordered with the group's around every step, so calls on a
// member between steps (seg_reset_stream, seg_set_stream_active, seg_sync)
// apply in order.
#include <stdlib.h>
#include <string.h>

#include "seg_internal.cuh"

struct GroupSetIo {
  SegIO* io;
  SegIO v;
  FrameWords w;
};

struct GroupSetIoArgs {
  int n;
  GroupSetIo e[SEG_GROUP_MAX];
};

// One CTA per member: its frame pointers, and its per-frame words zeroed.
__global__ void k_group_set_io(const __grid_constant__ GroupSetIoArgs a) {
  const GroupSetIo& m = a.e[blockIdx.x];
  const int t = threadIdx.x;
  if (t == 0) {
    *m.io = m.v;
    m.w.bar->count = 0u;
    m.w.bar->err = 0u;
  }
  if (t < 4) m.w.flags[t] = 0u;
  for (int b = t; b < m.w.B; b += blockDim.x) {
    if (m.w.smax) m.w.smax[b] = 0;
    m.w.cut_acc[b] = 0ull;
  }
}

struct seg_group {
  cudaStream_t stream;
  int n;
  seg_ctx* ctx[SEG_GROUP_MAX];
  cudaGraph_t graph;       // kept while the group lives: set_node is a node of it
  cudaGraphExec_t gexec;
  cudaGraphNode_t set_node;
  GroupSetIoArgs args;
  cudaEvent_t ev_in[SEG_GROUP_MAX];  // per step: a member's work so far
  cudaEvent_t ev_done;               // per step: the step's end
};

static void group_free(seg_group* g) {
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (int i = 0; i < g->n; ++i)
    if (g->ev_in[i]) cudaEventDestroy(g->ev_in[i]);
  if (g->ev_done) cudaEventDestroy(g->ev_done);
  free(g);
}

static void fill_entry(GroupSetIo& e, seg_ctx* c, const seg_frame_io* f) {
  e.io = c->io;
  memset(&e.v, 0, sizeof(e.v));
  if (f) {
    e.v.rgb = f->rgb;
    e.v.sal = f->sal ? f->sal : c->sal_buf;
    e.v.prior = f->prior ? f->prior : c->prior_buf;
    e.v.mask = f->mask;
    e.v.cut = (long long*)(f->cut ? f->cut : c->cut_buf);
  }
  e.w.smax = c->sal.smax;
  e.w.B = c->B;
  e.w.cut_acc = c->mf.cut_acc;
  e.w.flags = c->mf.flags;
  e.w.bar = c->mf.bar;
}

static cudaKernelNodeParams set_params(seg_group* g, void** kargs) {
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_group_set_io;
  kp.gridDim = dim3(g->n);
  kp.blockDim = dim3(32);
  kp.sharedMemBytes = 0;
  kargs[0] = &g->args;
  kp.kernelParams = kargs;
  kp.extra = nullptr;
  return kp;
}

// Captures the members' frame launches on their own streams, forked from and
// joined back into the group's stream, then adds the root kernel in front.
static int group_build(seg_group* g) {
  // events of the capture only (an event last recorded in a capturing stream
  // cannot be waited on outside it)
  cudaEvent_t ev[SEG_GROUP_MAX + 1] = {};
  for (int i = 0; i <= g->n; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      return SEG_ECUDA;
    }
  cudaGraph_t graph = nullptr;
  int rc = SEG_OK;
  cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (cudaEventRecord(ev[g->n], g->stream) != cudaSuccess) rc = SEG_ECUDA;
    for (int i = 0; i < g->n && !rc; ++i) {
      seg_ctx* c = g->ctx[i];
      if (cudaStreamWaitEvent(c->stream, ev[g->n], 0) != cudaSuccess) {
        rc = SEG_ECUDA;
        break;
      }
      c->io_mode = 1;
      rc = seg_ctx_push_launches(c, nullptr, nullptr, nullptr, nullptr, nullptr);
      c->io_mode = 0;
      if (!rc && (cudaEventRecord(ev[i], c->stream) != cudaSuccess ||
                  cudaStreamWaitEvent(g->stream, ev[i], 0) != cudaSuccess))
        rc = SEG_ECUDA;
    }
    e = cudaStreamEndCapture(g->stream, &graph);
  }
  for (int i = 0; i <= g->n; ++i) cudaEventDestroy(ev[i]);
  if (rc || e != cudaSuccess || !graph) {
    if (e != cudaSuccess) seg_note_cuda_error(e, "group capture");
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : SEG_ECUDA;
  }
  size_t nroots = 0;
  cudaGraphNode_t* roots = nullptr;
  bool ok = cudaGraphGetRootNodes(graph, nullptr, &nroots) == cudaSuccess && nroots > 0;
  if (ok) {
    roots = (cudaGraphNode_t*)malloc(nroots * sizeof(cudaGraphNode_t));
    ok = roots && cudaGraphGetRootNodes(graph, roots, &nroots) == cudaSuccess;
  }
  void* kargs[1];
  for (int i = 0; i < g->n; ++i) fill_entry(g->args.e[i], g->ctx[i], nullptr);
  g->args.n = g->n;
  cudaKernelNodeParams kp = set_params(g, kargs);
  ok = ok && cudaGraphAddKernelNode(&g->set_node, graph, nullptr, 0, &kp) == cudaSuccess;
  if (ok) {
    cudaGraphNode_t* from = (cudaGraphNode_t*)malloc(nroots * sizeof(cudaGraphNode_t));
    ok = from != nullptr;
    for (size_t k = 0; ok && k < nroots; ++k) from[k] = g->set_node;
    ok = ok && cudaGraphAddDependencies(graph, from, roots, nullptr, nroots) == cudaSuccess;
    free(from);
  }
  free(roots);
  if (ok) {
    e = cudaGraphInstantiate(&g->gexec, graph, 0);
    if (e != cudaSuccess) seg_note_cuda_error(e, "cudaGraphInstantiate (group)");
    ok = e == cudaSuccess;
  } else {
    seg_note_cuda_error(cudaGetLastError(), "group graph root node");
  }
  if (!ok) {
    cudaGraphDestroy(graph);
    g->gexec = nullptr;
    cudaGetLastError();
    return SEG_ECUDA;
  }
  g->graph = graph;  // (the exec's root node is addressed through it)
  return SEG_OK;
}

extern "C" int seg_group_create(void* stream, seg_ctx* const* ctxs, int n, seg_group** out) {
  if (!out) return SEG_EINVAL;
  *out = nullptr;
  if (!ctxs || n < 1 || n > SEG_GROUP_MAX || !stream) return SEG_EINVAL;
  for (int i = 0; i < n; ++i) {
    seg_ctx* c = ctxs[i];
    if (!c || !c->stream || c->pipe_on || c->prof_on) return SEG_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return SEG_EINVAL;
  }
  seg_group* g = (seg_group*)calloc(1, sizeof(seg_group));
  if (!g) return SEG_ENOMEM;
  g->stream = (cudaStream_t)stream;
  g->n = n;
  for (int i = 0; i < n; ++i) g->ctx[i] = ctxs[i];
  bool ok = cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i) ok = cudaEventCreateWithFlags(&g->ev_in[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    group_free(g);
    return SEG_ECUDA;
  }
  // nothing a member has enqueued may run inside the capture
  for (int i = 0; i < n; ++i)
    if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) {
      group_free(g);
      return SEG_ECUDA;
    }
  int rc = group_build(g);
  if (rc) {
    group_free(g);
    return rc;
  }
  *out = g;
  return SEG_OK;
}

extern "C" int seg_group_push(seg_group* g, const seg_frame_io* io) {
  if (!g || !io) return SEG_EINVAL;
  for (int i = 0; i < g->n; ++i)
    if (!io[i].rgb || !io[i].mask) return SEG_EINVAL;
  for (int i = 0; i < g->n; ++i) fill_entry(g->args.e[i], g->ctx[i], &io[i]);
  void* kargs[1];
  cudaKernelNodeParams kp = set_params(g, kargs);
  SEG_CUDA_TRY(cudaGraphExecKernelNodeSetParams(g->gexec, g->set_node, &kp));
  for (int i = 0; i < g->n; ++i) {  // after what the members have enqueued
    SEG_CUDA_TRY(cudaEventRecord(g->ev_in[i], g->ctx[i]->stream));
    SEG_CUDA_TRY(cudaStreamWaitEvent(g->stream, g->ev_in[i], 0));
  }
  SEG_CUDA_TRY(cudaGraphLaunch(g->gexec, g->stream));
  SEG_CUDA_TRY(cudaEventRecord(g->ev_done, g->stream));
  for (int i = 0; i < g->n; ++i) SEG_CUDA_TRY(cudaStreamWaitEvent(g->ctx[i]->stream, g->ev_done, 0));
  return SEG_OK;
}

extern "C" int seg_group_sync(seg_group* g, int* codes, int* cycles) {
  if (!g) return SEG_EINVAL;
  SEG_CUDA_TRY(cudaStreamSynchronize(g->stream));
  int first = SEG_OK;
  for (int i = 0; i < g->n; ++i) {
    int cyc = 0;
    const int code = seg_sync(g->ctx[i], &cyc);
    if (codes) codes[i] = code;
    if (cycles) cycles[i] = cyc;
    if (code && !first) first = code;
  }
  return first;
}

extern "C" int seg_group_destroy(seg_group* g) {
  if (!g) return SEG_EINVAL;
  cudaStreamSynchronize(g->stream);
  group_free(g);
  return SEG_OK;
}
