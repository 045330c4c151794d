// diff.cu -- the backward form on sm_103a: the saliency map (Sec. 3 / Sec. 7.2)
// and the Kalman-updated prior (Sec. 6) of B floating-point frames, and the
// reverse pass of
//     L = sum_b <g_prior_b, prior_b> + <g_sal_b, saliency_b>
// with respect to the frames, the four channel weights w and the Kalman noise
// variances Q = sigma1^2, R = sigma2^2 (theta = (w_I, w_RG, w_BY, w_O, Q, R)).
//
// Frame b of a batch is clip time t0 + b.  The variance recursion of Sec. 6 does
// not depend on the data, so the frames of a clip are independent given w_f(t),
// and a clip is one batch.  The previous masks enter through the smoothed maps f
// (stop-gradient constants).
//
// Checkpointing: the forward keeps the pyramid levels, the Gabor responses
// (complex), the across-scale accumulators at sigma_S, the conspicuity maps and S;
// the reverse pass recomputes every center-surround map and its N(.) statistics
// from those.  Piecewise-linear parts take the one-sided derivative: N(.) through
// the first index attaining the minimum, the maximum and each tile maximum,
// |a| through sign(a) (0 at 0), max(0, a) through a > 0, the hue mask as fixed.
//
// Reverse-pass kernels, in launch order (every output element is written by one
// thread, so results are deterministic):
//   k_db_rows      dL/dsaliency per pixel, fused with the transposed bilinear
//                  up-sampling along x; partial sums of dL/dw_f and of the
//                  saliency-maximum term
//   k_db_top       one CTA per frame at sigma_S: transposed up-sampling along y,
//                  the maximum's term, dL/dw, dL/dQ, dL/dR
//   k_db_nbwd      N(.)^T of the four conspicuity maps, then of the orientation
//                  accumulators (one CTA per map and frame)
//   k_db_reduceT   transposed REDUCE (across-scale sums, then the pyramid)
//   k_db_cs_stats  per center-surround map: N(.) statistics of the recomputed map
//                  and the reductions its derivative needs
//   k_db_cs_apply  dL/dmap per pixel -> center level (+ sign), surround field
//   k_db_surT      transposed up-sampling of the surround fields
//   k_db_gaborT    transposed complex Gabor filter (separable, clamped borders)
//   k_db_feat      level 1 -> level 0 transposed REDUCE fused with the features'
//                  derivative: dL/dframe
//   k_db_final     per-frame parameter gradients summed over the batch
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "seg_internal.cuh"

typedef unsigned long long u64;

#define DB_MAXT 4096    // N(.) tiles per center-surround map
#define DB_MAXT_S 1024  // N(.) tiles per map at sigma_S (the forward's limit as well)
#define DB_RB 2       // frame rows per CTA of k_db_rows
#define DB_TX 32
#define DB_TY 16
#define GB_MAXR_T 8  // largest Gabor radius (taps <= 17)
#define SURT_CAP 8192  // floats of the row-transposed surround field staged per chunk

__constant__ float c_kb[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};

struct DiffPart {  // N(.) statistics of one band of T rows of a center-surround map
  u64 kmin, kmax;
  double sg, sgv, st;
};

struct DiffCoef {
  float aG, at, smin, smax;  // dN^T: aG g_i + at [i tile argmax] + smin [i = argmin] + smax [i = argmax]
  int amin, amax, flat, pad;
};

struct seg_diff {
  cudaStream_t stream;
  int device, B, H, W;
  seg_params p;
  char* arena;
  size_t bytes;
  SalWS sal;
  double* kal;  // [B][3]: w_f, dw_f/dQ, dw_f/dR
  float* Tx;    // [B][H][wS]
  double* part; // [B][nbx][2]
  int nbx;
  float* gS;    // [B][nS]
  float* gC3;   // [B][nS]
  float* G[SEG_MAX_LEVELS];  // scales c_min..c_max: [B][nch][hl*wl]
  DiffCoef* coef;            // [B][nmaps]
  DiffPart* dpart;           // [B][bands of all center-surround maps]
  int* targ;                 // [B][ntarg]
  int ntarg;
  int targ_off[SEG_MAX_PAIRS];
  float* hsur;  // [B][nhsur]
  size_t nhsur;
  size_t hsur_off[SEG_MAX_PAIRS];
  float* gpyr[3][SEG_MAX_LEVELS];
  float* gori[SEG_MAX_ORIENT][SEG_MAX_LEVELS];
  char* grad_base;
  size_t grad_bytes;
  double* gpar;  // [B][6]
  int2* rsT;     // transposed resampling ranges {first, last + 1}
  int* rt_lo;    // transposed REDUCE tables, per level l -> l+1: rows then columns
  float4* rt_w;
  int rt_row[SEG_MAX_LEVELS], rt_col[SEG_MAX_LEVELS], rt_n;
  int rsT_row[SEG_MAX_PAIRS], rsT_col[SEG_MAX_PAIRS], rsT_frow, rsT_fcol, rsT_n;
  int forward_done;
};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ u64 key_max(float v, int i) {
  return ((u64)f2key(v) << 32) | (u64)(0xffffffffu - (unsigned)i);  // larger value, then smaller index
}
__device__ __forceinline__ u64 key_min(float v, int i) {
  return ((u64)f2key(v) << 32) | (u64)(unsigned)i;  // smaller value, then smaller index
}
__device__ __forceinline__ float key_val(u64 k) { return key2f((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_max_idx(u64 k) { return (int)(0xffffffffu - (unsigned)(k & 0xffffffffu)); }
__device__ __forceinline__ int key_min_idx(u64 k) { return (int)(unsigned)(k & 0xffffffffu); }

__device__ __forceinline__ u64 warp_min_u64(u64 v) {
  for (int o = 16; o > 0; o >>= 1) {
    u64 w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
__device__ __forceinline__ u64 warp_max_u64(u64 v) {
  for (int o = 16; o > 0; o >>= 1) {
    u64 w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Block-wide reductions (every thread gets the result).  red must hold 32
// entries of the reduced type; the call ends with a barrier.  Sums take one float
// per thread (each thread's share is a few terms): float within a warp, the warp
// partials added in double by one thread -- the FP64 pipe of this part is narrow.
__device__ double block_sum_d(float v, double* red) {
  v = seg_warp_sum_f(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  float* rf = (float*)(red + 1);  // 31 doubles of room: 62 floats >= 32 warps
  if (lane == 0) rf[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += rf[w];  // fixed order: deterministic
    red[0] = t;
  }
  __syncthreads();
  const double t = red[0];
  __syncthreads();
  return t;
}
__device__ u64 block_min_u64(u64 v, u64* red) {
  v = warp_min_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  u64 t = red[0];
  for (int w = 1; w < nw; ++w) t = red[w] < t ? red[w] : t;
  __syncthreads();
  return t;
}
__device__ u64 block_max_u64(u64 v, u64* red) {
  v = warp_max_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  u64 t = red[0];
  for (int w = 1; w < nw; ++w) t = red[w] > t ? red[w] : t;
  __syncthreads();
  return t;
}

// Coefficients of N(.)^T (the reading of N(.): v' = (v - min)/D, D = max - min,
// mbar = (sum of tile maxima of v' - 1)/(nt - 1), N = v' (1 - mbar)^2; flat maps,
// D <= flat, give N = 0) from the map's statistics and the two reductions
// sum g and sum g v of the incoming derivative g:
//   dN^T g = (F/D) g + (dm/D) [tile argmax] + smin [argmin] + smax [argmax],
//   F = (1 - mbar)^2, dm = -2 (1 - mbar) sum(g v') / (nt - 1).
__device__ DiffCoef norm_coef(u64 kmin, u64 kmax, double sum_tmax, int nt, double sg, double sgv, float flat) {
  DiffCoef c;
  memset(&c, 0, sizeof(c));
  const double mn = key_val(kmin), mx = key_val(kmax), D = mx - mn;
  c.amin = key_min_idx(kmin);
  c.amax = key_max_idx(kmax);
  if (!(D > (double)flat)) {
    c.flat = 1;
    return c;
  }
  const double st = (sum_tmax - nt * mn) / D;  // sum of the rescaled tile maxima
  const double mbar = nt > 1 ? (st - 1.0) / (nt - 1) : 0.0;
  const double F = (1.0 - mbar) * (1.0 - mbar);
  const double sgvp = (sgv - mn * sg) / D;  // sum g v'
  const double dm = nt > 1 ? sgvp * (-2.0 * (1.0 - mbar)) / (nt - 1) : 0.0;
  const double sgp_v = F * sgvp + dm * st;  // sum gp v', gp = F g + dm [tile argmax]
  const double sgp = F * sg + dm * nt;
  c.aG = (float)(F / D);
  c.at = (float)(dm / D);
  c.smin = (float)((sgp_v - sgp) / D);
  c.smax = (float)(-sgp_v / D);
  return c;
}

__device__ __forceinline__ float coef_apply(const DiffCoef& c, float g, int i, int targ_i) {
  if (c.flat) return 0.f;
  float r = c.aG * g;
  if (targ_i == i) r += c.at;
  if (i == c.amin) r += c.smin;
  if (i == c.amax) r += c.smax;
  return r;
}

// ------------------------------------------------------------------ forward-only kernels
// Sec. 6 with forward-mode derivatives: w_f(t) = Q / (Q + R + P(t-1)),
// P(t) = Q (R + P(t-1)) / (Q + R + P(t-1)), P(-1) = inf (w_f(0) = 0, P(0) = Q).
__global__ void k_df_kalman(const double* __restrict__ theta, int t0, int B, double* __restrict__ kal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double Q = theta[4], R = theta[5];
  double P = 0, dPq = 0, dPr = 0;
  for (int t = 0; t < t0 + B; ++t) {
    double w = 0, wq = 0, wr = 0, Pn = Q, Pq = 1, Pr = 0;
    if (t > 0) {
      const double den = Q + R + P, dq = 1 + dPq, dr = 1 + dPr, num = Q * (R + P);
      const double inv = 1.0 / den, inv2 = inv * inv;  // one division per step
      w = Q * inv;
      wq = (den - Q * dq) * inv2;
      wr = -Q * dr * inv2;
      Pn = num * inv;
      Pq = ((R + P + Q * dPq) * den - num * dq) * inv2;
      Pr = (Q * dr * den - num * dr) * inv2;
    }
    if (t >= t0) {
      kal[3 * (t - t0)] = w;
      kal[3 * (t - t0) + 1] = wq;
      kal[3 * (t - t0) + 2] = wr;
    }
    P = Pn;
    dPq = Pq;
    dPr = Pr;
  }
}

// Secs. 5-6: saliency = S up-sampled; q = saliency / max inside the frame, eps on
// the border; prior = w_f f + (1 - w_f) q.
__global__ void __launch_bounds__(256) k_df_prior(const float* __restrict__ S, int hs, int ws, int H, int W,
                                                  const int2* __restrict__ frow, const int2* __restrict__ fcol,
                                                  const unsigned* __restrict__ salmax,
                                                  const double* __restrict__ kal, const float* __restrict__ fmap,
                                                  int border, float eps, float* __restrict__ sal,
                                                  float* __restrict__ prior) {
  const int b = blockIdx.z;
  const int x = blockIdx.x * 64 + (threadIdx.x & 63), y = blockIdx.y * 4 + (threadIdx.x >> 6);
  if (x >= W || y >= H) return;
  const size_t i = (size_t)b * H * W + (size_t)y * W + x;
  const float v = seg_bilinear_t(S + (size_t)b * hs * ws, ws, frow[y], fcol[x]);
  const float mx = __uint_as_float(salmax[b]);
  const bool edge = y < border || y >= H - border || x < border || x >= W - border;
  const float q = edge ? eps : (mx > 0.f ? v / mx : 0.f);
  const float wf = (float)kal[3 * b];
  const float f = fmap ? fmap[i] : 0.f;
  if (sal) sal[i] = v;
  prior[i] = wf * f + (1.f - wf) * q;
}

// ------------------------------------------------------------------ reverse pass
// dL/dsaliency for DB_RB frame rows (all columns) of one frame, then its
// transposed up-sampling along x into Tx[y][X]; partial sums of
// dL/dw_f = sum g_prior (f - q) and of sum g_q saliency (the maximum's term).
__global__ void __launch_bounds__(256) k_db_rows(const float* __restrict__ S, int hs, int ws, int H, int W,
                                                 const int2* __restrict__ frow, const int2* __restrict__ fcol,
                                                 const int2* __restrict__ fcolT,
                                                 const unsigned* __restrict__ salmax,
                                                 const double* __restrict__ kal, const float* __restrict__ fmap,
                                                 const float* __restrict__ g_prior, const float* __restrict__ g_sal,
                                                 int border, float eps, float* __restrict__ Tx,
                                                 double* __restrict__ part) {
  extern __shared__ float sg[];  // [DB_RB][W]
  __shared__ double red[32];
  const int b = blockIdx.y, Y0 = blockIdx.x * DB_RB;
  const float mx = __uint_as_float(salmax[b]);
  const float wf = (float)kal[3 * b];
  const float* Sb = S + (size_t)b * hs * ws;
  float a_wf = 0.f, a_m = 0.f;  // a few pixels per thread; the block sums are double
  for (int k = threadIdx.x; k < DB_RB * W; k += blockDim.x) {
    const int r = k / W, x = k - r * W, y = Y0 + r;
    if (y >= H) continue;
    const size_t i = (size_t)b * H * W + (size_t)y * W + x;
    const float v = seg_bilinear_t(Sb, ws, frow[y], fcol[x]);
    const bool edge = y < border || y >= H - border || x < border || x >= W - border;
    const float q = edge ? eps : (mx > 0.f ? v / mx : 0.f);
    const float gp = g_prior[i];
    const float f = fmap ? fmap[i] : 0.f;
    a_wf += gp * (f - q);
    float gs = g_sal ? g_sal[i] : 0.f;
    if (!edge && mx > 0.f) {
      const float gq = gp * (1.f - wf);
      gs += gq / mx;
      a_m += gq * v;
    }
    sg[r * W + x] = gs;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < DB_RB * ws; k += blockDim.x) {
    const int r = k / ws, X = k - r * ws, y = Y0 + r;
    if (y >= H) continue;
    const int2 rg = fcolT[X];
    float acc = 0.f;
    for (int x = rg.x; x < rg.y; ++x) {
      const int2 e = fcol[x];
      const int x0 = e.x & 0xffff, x1 = e.x >> 16;
      const float fx = __int_as_float(e.y);
      float w = 0.f;
      if (x0 == X) w += 1.f - fx;
      if (x1 == X) w += fx;
      acc += w * sg[r * W + x];
    }
    Tx[((size_t)b * H + y) * ws + X] = acc;
  }
  const double s_wf = block_sum_d(a_wf, red), s_m = block_sum_d(a_m, red);
  if (threadIdx.x == 0) {
    part[2 * ((size_t)b * gridDim.x + blockIdx.x)] = s_wf;
    part[2 * ((size_t)b * gridDim.x + blockIdx.x) + 1] = s_m;
  }
}

// N(.)^T of one map of n = h*w values held in global memory (one CTA): out =
// dN^T (scale * g).  tk holds DB_MAXT keys.
__device__ void block_norm_bwd(const float* v, const float* g, float scale, float* out, int h, int w, int T,
                               float flat, u64* tk, double* redd, u64* redk) {
  const int n = h * w, ntx = (w + T - 1) / T, nt = ntx * ((h + T - 1) / T);
  for (int t = threadIdx.x; t < nt; t += blockDim.x) tk[t] = 0ull;
  __syncthreads();
  u64 kmin = ~0ull, kmax = 0ull;
  float sg = 0.f, sgv = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x = v[i], gi = scale * g[i];
    const int yy = i / w, xx = i - yy * w;
    const u64 kx = key_max(x, i), kn = key_min(x, i);
    kmin = kn < kmin ? kn : kmin;
    kmax = kx > kmax ? kx : kmax;
    atomicMax(&tk[(yy / T) * ntx + xx / T], kx);
    sg += gi;
    sgv += gi * x;
  }
  kmin = block_min_u64(kmin, redk);
  kmax = block_max_u64(kmax, redk);
  const double sgd = block_sum_d(sg, redd), sgvd = block_sum_d(sgv, redd);
  float st = 0.f;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) st += key_val(tk[t]);
  const double std_ = block_sum_d(st, redd);
  const DiffCoef c = norm_coef(kmin, kmax, std_, nt, sgd, sgvd, flat);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int yy = i / w, xx = i - yy * w;
    out[i] = coef_apply(c, scale * g[i], i, key_max_idx(tk[(yy / T) * ntx + xx / T]));
  }
  __syncthreads();
}

struct TopArgs {
  const float* Tx;
  const double* part;
  int nbx;
  int H, W, hs, ws, nch, tile;
  float flat;
  const int2* frow;
  const int2* fcol;
  const int2* frowT;
  const unsigned* salmax;
  const float* S;
  const float* consp;
  const float* acc;   // accumulators at sigma_S: [B][nch][nS]
  const float* csum;  // orientation conspicuity C_O: [B][nS]
  const double* kal;
  const double* theta;
  float* gS;
  float* gC3;
  float* gacc;  // [B][nch][nS]
  double* gpar;
};

// One CTA per frame, at sigma_S.
__global__ void __launch_bounds__(1024) k_db_top(TopArgs a) {
  __shared__ double redd[32];
  __shared__ u64 redk[32];
  __shared__ int crow[2048], ccol[2048];
  __shared__ int nr, nc;
  const int b = blockIdx.x, nS = a.hs * a.ws;
  const float mx = __uint_as_float(a.salmax[b]);
  const float* Sb = a.S + (size_t)b * nS;
  float* gS = a.gS + (size_t)b * nS;
  // sums of the row partials (fixed order)
  if (threadIdx.x == 0) {  // row partials in order (one thread: deterministic)
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < a.nbx; ++k) {
      s0 += a.part[2 * ((size_t)b * a.nbx + k)];
      s1 += a.part[2 * ((size_t)b * a.nbx + k) + 1];
    }
    redd[0] = s0;
    redd[1] = s1;
  }
  __syncthreads();
  const double gwf = redd[0], gmq = redd[1];
  __syncthreads();
  // transposed up-sampling along y
  const float* Tx = a.Tx + (size_t)b * a.H * a.ws;
  for (int k = threadIdx.x; k < nS; k += blockDim.x) {
    const int Y = k / a.ws, X = k - Y * a.ws;
    const int2 rg = a.frowT[Y];
    float acc = 0.f;
    for (int y = rg.x; y < rg.y; ++y) {
      const int2 e = a.frow[y];
      const int y0 = e.x & 0xffff, y1 = e.x >> 16;
      const float fy = __int_as_float(e.y);
      float w = 0.f;
      if (y0 == Y) w += 1.f - fy;
      if (y1 == Y) w += fy;
      acc += w * Tx[(size_t)y * a.ws + X];
    }
    gS[k] = acc;
  }
  // the maximum's term: q = saliency / max, d max / d saliency = [first argmax]
  if (mx > 0.f && gmq != 0.0) {
    if (threadIdx.x == 0) nr = nc = 0;
    __syncthreads();
    for (int y = threadIdx.x; y < a.H; y += blockDim.x)
      if (seg_up_candidate(y, a.hs, a.H)) crow[atomicAdd(&nr, 1)] = y;
    for (int x = threadIdx.x; x < a.W; x += blockDim.x)
      if (seg_up_candidate(x, a.ws, a.W)) ccol[atomicAdd(&nc, 1)] = x;
    __syncthreads();
    u64 best = 0ull;
    for (int k = threadIdx.x; k < nr * nc; k += blockDim.x) {
      const int y = crow[k / nc], x = ccol[k % nc];
      const u64 key = key_max(seg_bilinear_t(Sb, a.ws, a.frow[y], a.fcol[x]), y * a.W + x);
      best = key > best ? key : best;
    }
    best = block_max_u64(best, redk);
    if (threadIdx.x == 0) {
      const int i = key_max_idx(best), y = i / a.W, x = i - y * a.W;
      const float gm = (float)(-gmq / ((double)mx * mx));
      const int2 ey = a.frow[y], ex = a.fcol[x];
      const int y0 = ey.x & 0xffff, y1 = ey.x >> 16, x0 = ex.x & 0xffff, x1 = ex.x >> 16;
      const float fy = __int_as_float(ey.y), fx = __int_as_float(ex.y);
      gS[y0 * a.ws + x0] += gm * (1.f - fy) * (1.f - fx);
      gS[y0 * a.ws + x1] += gm * (1.f - fy) * fx;
      gS[y1 * a.ws + x0] += gm * fy * (1.f - fx);
      gS[y1 * a.ws + x1] += gm * fy * fx;
    }
  }
  __syncthreads();
  // dL/dw_k = <gS, N(C_k)>; dL/dQ, dL/dR through w_f(t)
  const float* consp = a.consp + (size_t)b * 4 * nS;
  for (int k = 0; k < 4; ++k) {
    float sf = 0.f;
    for (int i = threadIdx.x; i < nS; i += blockDim.x) sf += gS[i] * consp[(size_t)k * nS + i];
    const double s = block_sum_d(sf, redd);
    if (threadIdx.x == 0) a.gpar[6 * b + k] = s;
  }
  if (threadIdx.x == 0) {
    a.gpar[6 * b + 4] = gwf * a.kal[3 * b + 1];
    a.gpar[6 * b + 5] = gwf * a.kal[3 * b + 2];
  }
}

// N(.)^T at sigma_S, one CTA per (map, frame).  stage 0: S = sum_k w_k N(C_k)
// with C_I, C_RG, C_BY the accumulators and C_O = csum (map k = blockIdx.x);
// stage 1: C_O = sum_theta N(accumulator_theta) (theta = blockIdx.x).
__global__ void __launch_bounds__(512) k_db_nbwd(TopArgs a, int stage) {
  __shared__ u64 tk[DB_MAXT_S];
  __shared__ double redd[32];
  __shared__ u64 redk[32];
  const int b = blockIdx.y, nS = a.hs * a.ws, k = blockIdx.x;
  const float* acc = a.acc + (size_t)b * a.nch * nS;
  float* gacc = a.gacc + (size_t)b * a.nch * nS;
  float* gC3 = a.gC3 + (size_t)b * nS;
  if (stage == 0) {
    const float* v = k < 3 ? acc + (size_t)k * nS : a.csum + (size_t)b * nS;
    float* out = k < 3 ? gacc + (size_t)k * nS : gC3;
    block_norm_bwd(v, a.gS + (size_t)b * nS, (float)a.theta[k], out, a.hs, a.ws, a.tile, a.flat, tk, redd, redk);
  } else {
    const int f = 3 + k;
    block_norm_bwd(acc + (size_t)f * nS, gC3, 1.f, gacc + (size_t)f * nS, a.hs, a.ws, a.tile, a.flat, tk, redd,
                   redk);
  }
}

// Transposed REDUCE (5x5 binomial, clamp-to-edge, even samples): out (+)= R^T in,
// with in at (h2, w2) = ((h+1)/2, (w+1)/2).  Plane z: pointer slot z % K, plane
// z / K of that slot.
struct RTArgs {
  const float* in[3];
  float* out[3];
  int K, h, w, h2, w2, accumulate;
  const int* lo_y;  // per output row: first level-(l+1) row reaching it
  const float4* w_y;  // its four weights (0 past the level)
  const int* lo_x;
  const float4* w_x;
};

// sum_{j,i < 4} wy[j] wx[i] in[lo_y + j][lo_x + i] (zero-weight taps past the
// level are read at a clamped address)
__device__ __forceinline__ float rt_apply(const float* in, int w2, int h2, int ylo, float4 wy, int xlo, float4 wx) {
  const float wya[4] = {wy.x, wy.y, wy.z, wy.w}, wxa[4] = {wx.x, wx.y, wx.z, wx.w};
  int xs[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) xs[i] = min(xlo + i, w2 - 1);
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float* row = in + (size_t)min(ylo + j, h2 - 1) * w2;
    acc += wya[j] * (wxa[0] * row[xs[0]] + wxa[1] * row[xs[1]] + wxa[2] * row[xs[2]] + wxa[3] * row[xs[3]]);
  }
  return acc;
}

__global__ void __launch_bounds__(256) k_db_reduceT(RTArgs a) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= a.w || y >= a.h) return;
  const int slot = blockIdx.z % a.K, pl = blockIdx.z / a.K;
  // (select the slot without indexing the parameter arrays at run time)
  const float* in = (slot == 0 ? a.in[0] : slot == 1 ? a.in[1] : a.in[2]) + (size_t)pl * a.h2 * a.w2;
  float* out = (slot == 0 ? a.out[0] : slot == 1 ? a.out[1] : a.out[2]) + (size_t)pl * a.h * a.w;
  const float acc = rt_apply(in, a.w2, a.h2, a.lo_y[y], a.w_y[y], a.lo_x[x], a.w_x[x]);
  const size_t o = (size_t)y * a.w + x;
  out[o] = a.accumulate ? out[o] + acc : acc;
}

// Arguments shared by the center-surround kernels of the reverse pass.
struct DCSArgs {
  const float* X[3 + SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // forward channel planes
  float* GX[3 + SEG_MAX_ORIENT][SEG_MAX_LEVELS];       // their gradients
  const float* G[SEG_MAX_LEVELS];                      // dL/d(sum of N(maps)) at scale c: [B][nch][n]
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  int pair_c[SEG_MAX_PAIRS], pair_s[SEG_MAX_PAIRS];
  int npairs, nch, nmaps, tile, opp_sum;
  float flat;
  const int2* rs;
  int rs_row[SEG_MAX_PAIRS], rs_col[SEG_MAX_PAIRS];
  const int2* rsT;
  int rsT_row[SEG_MAX_PAIRS], rsT_col[SEG_MAX_PAIRS];
  DiffCoef* coef;
  int* targ;
  int ntarg;
  int targ_off[SEG_MAX_PAIRS];
  float* hsur;
  size_t nhsur;
  size_t hsur_off[SEG_MAX_PAIRS];
  int slist[SEG_MAX_LEVELS], nsl;  // distinct surround scales
  int band_off[SEG_MAX_PAIRS + 1];  // prefix of (channels x bands of T rows) per pair
  int nbands_total;
  DiffPart* dpart;  // [B][nbands_total]
};

__device__ __forceinline__ float cs_signed(const DCSArgs& a, int p, int f, int b, int y, int x) {
  const int c = a.pair_c[p], sv = a.pair_s[p];
  const int wc = a.wl[c], hs = a.hl[sv], ws = a.wl[sv];
  const float u = seg_bilinear_t(a.X[f][sv] + (size_t)b * hs * ws, ws, a.rs[a.rs_row[p] + y], a.rs[a.rs_col[p] + x]);
  const float v0 = a.X[f][c][(size_t)b * a.hl[c] * wc + (size_t)y * wc + x];
  return (a.opp_sum && (f == 1 || f == 2)) ? v0 + u : v0 - u;
}

// One CTA per (band of T rows of a center-surround map, frame): the N(.)
// statistics of the recomputed map |a| over the band and the reductions of its
// incoming derivative; warps take the band's T x T tiles in turn and reduce
// each tile's maximum (value, first index) with shuffles.
__global__ void __launch_bounds__(256) k_db_cs_stats(DCSArgs a) {
  __shared__ double redd[32];
  __shared__ u64 redk[32];
  int bx = blockIdx.x, p = 0;
  while (p < a.npairs - 1 && bx >= a.band_off[p + 1]) ++p;
  const int b = blockIdx.y, c = a.pair_c[p], hc = a.hl[c], wc = a.wl[c], T = a.tile;
  const int nb = (hc + T - 1) / T, ntx = (wc + T - 1) / T, nt = ntx * nb;
  const int rem = bx - a.band_off[p], f = rem / nb, band = rem - f * nb;
  const float* G = a.G[c] + ((size_t)b * a.nch + f) * hc * wc;
  int* targ = a.targ + (size_t)b * a.ntarg + a.targ_off[p] + (size_t)f * nt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int y0 = band * T, rows = min(T, hc - y0);
  u64 kmin = ~0ull, kmax = 0ull;
  float sg = 0.f, sgv = 0.f, st = 0.f;
  for (int tx = wid; tx < ntx; tx += nw) {
    const int x0 = tx * T, cols = min(T, wc - x0);
    u64 kt = 0ull;
    float sgt = 0.f, sgvt = 0.f;
    for (int k = lane; k < rows * cols; k += 32) {
      const int yy = k / cols, y = y0 + yy, x = x0 + (k - yy * cols), i = y * wc + x;
      const float v = fabsf(cs_signed(a, p, f, b, y, x)), g = G[i];
      const u64 kn = key_min(v, i), kx = key_max(v, i);
      kmin = kn < kmin ? kn : kmin;
      kt = kx > kt ? kx : kt;
      sgt += g;
      sgvt += g * v;
    }
    sg += sgt;
    sgv += sgvt;
    kt = warp_max_u64(kt);
    kmax = kt > kmax ? kt : kmax;
    if (lane == 0) {
      targ[band * ntx + tx] = key_max_idx(kt);
      st += key_val(kt);
    }
  }
  kmin = block_min_u64(kmin, redk);
  kmax = block_max_u64(kmax, redk);
  const double sgd = block_sum_d(sg, redd), sgvd = block_sum_d(sgv, redd), std_ = block_sum_d(st, redd);
  if (threadIdx.x == 0) {
    DiffPart q;
    q.kmin = kmin;
    q.kmax = kmax;
    q.sg = sgd;
    q.sgv = sgvd;
    q.st = std_;
    a.dpart[(size_t)b * a.nbands_total + bx] = q;
  }
}

// N(.)^T coefficients of every center-surround map from its band statistics
// (bands summed in order: deterministic).
__global__ void k_db_cs_coef(DCSArgs a, int B) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.nmaps * B) return;
  const int b = j / a.nmaps, m = j - b * a.nmaps, p = m / a.nch, f = m - p * a.nch;
  const int c = a.pair_c[p], T = a.tile, nb = (a.hl[c] + T - 1) / T, nt = nb * ((a.wl[c] + T - 1) / T);
  const DiffPart* q = a.dpart + (size_t)b * a.nbands_total + a.band_off[p] + f * nb;
  u64 kmin = ~0ull, kmax = 0ull;
  double sg = 0.0, sgv = 0.0, st = 0.0;
  for (int i = 0; i < nb; ++i) {
    kmin = q[i].kmin < kmin ? q[i].kmin : kmin;
    kmax = q[i].kmax > kmax ? q[i].kmax : kmax;
    sg += q[i].sg;
    sgv += q[i].sgv;
    st += q[i].st;
  }
  a.coef[(size_t)b * a.nmaps + m] = norm_coef(kmin, kmax, st, nt, sg, sgv, a.flat);
}

// dL/dmap per pixel of scale c: the center level receives sign(a) times it, the
// surround field h = -/+ sign(a) times it waits for k_db_surT.
__global__ void __launch_bounds__(256) k_db_cs_apply(DCSArgs a, int c) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int hc = a.hl[c], wc = a.wl[c], n = hc * wc, T = a.tile;
  if (x >= wc || y >= hc) return;
  const int f = blockIdx.z % a.nch, b = blockIdx.z / a.nch;
  const int i = y * wc + x, ntx = (wc + T - 1) / T, nt = ntx * ((hc + T - 1) / T), tile = (y / T) * ntx + x / T;
  const float G = a.G[c][((size_t)b * a.nch + f) * n + i];
  float gsum = 0.f;
  for (int p = 0; p < a.npairs; ++p) {
    if (a.pair_c[p] != c) continue;
    const int m = p * a.nch + f;
    const DiffCoef cf = a.coef[(size_t)b * a.nmaps + m];
    const int ti = a.targ[(size_t)b * a.ntarg + a.targ_off[p] + (size_t)f * nt + tile];
    const float gv = coef_apply(cf, G, i, ti);
    const float s = cs_signed(a, p, f, b, y, x);
    const float sg = s > 0.f ? 1.f : (s < 0.f ? -1.f : 0.f);
    gsum += gv * sg;
    const bool opp = a.opp_sum && (f == 1 || f == 2);
    a.hsur[(size_t)b * a.nhsur + a.hsur_off[p] + (size_t)f * n + i] = opp ? gv * sg : -gv * sg;
  }
  float* gx = a.GX[f][c] + (size_t)b * n + i;
  *gx += gsum;
}

// Transposed bilinear up-sampling of the surround fields, one CTA per (surround
// scale s, channel f, frame b), over every pair whose surround scale is s:
// separably, T1[y][X] = sum_x wx(x, X) h[y][x] for the rows y a chunk of output
// rows needs (shared memory), then out[Y][X] += sum_y wy(y, Y) T1[y][X].
__global__ void __launch_bounds__(256) k_db_surT(DCSArgs a) {
  __shared__ float sT[SURT_CAP];
  const int s = a.slist[blockIdx.x], f = blockIdx.y, b = blockIdx.z;
  const int hs = a.hl[s], ws = a.wl[s];
  float* gx = a.GX[f][s] + (size_t)b * hs * ws;
  for (int p = 0; p < a.npairs; ++p) {
    if (a.pair_s[p] != s) continue;
    const int c = a.pair_c[p], hc = a.hl[c], wc = a.wl[c];
    const float* h = a.hsur + (size_t)b * a.nhsur + a.hsur_off[p] + (size_t)f * hc * wc;
    const int2* rT = a.rsT + a.rsT_row[p];
    const int2* cT = a.rsT + a.rsT_col[p];
    const int2* trow = a.rs + a.rs_row[p];
    const int2* tcol = a.rs + a.rs_col[p];
    for (int Y0 = 0; Y0 < hs;) {
      const int ya = rT[Y0].x;
      int Y1 = Y0 + 1;
      while (Y1 < hs && (rT[Y1].y - ya) * ws <= SURT_CAP) ++Y1;
      const int yb = max(ya, rT[Y1 - 1].y);
      for (int k = threadIdx.x; k < (yb - ya) * ws; k += blockDim.x) {
        const int y = ya + k / ws, X = k % ws;
        const int2 rg = cT[X];
        const float* row = h + (size_t)y * wc;
        float r = 0.f;
        for (int x = rg.x; x < rg.y; ++x) {
          const int2 ex = tcol[x];
          const float fx = __int_as_float(ex.y);
          float wx = 0.f;
          if ((ex.x & 0xffff) == X) wx += 1.f - fx;
          if ((ex.x >> 16) == X) wx += fx;
          r += wx * row[x];
        }
        sT[k] = r;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < (Y1 - Y0) * ws; k += blockDim.x) {
        const int Y = Y0 + k / ws, X = k % ws;
        const int2 rg = rT[Y];
        float acc = 0.f;
        for (int y = rg.x; y < rg.y; ++y) {
          const int2 ey = trow[y];
          const float fy = __int_as_float(ey.y);
          float wy = 0.f;
          if ((ey.x & 0xffff) == Y) wy += 1.f - fy;
          if ((ey.x >> 16) == Y) wy += fy;
          acc += wy * sT[(y - ya) * ws + X];
        }
        gx[(size_t)Y * ws + X] += acc;
      }
      __syncthreads();
      Y0 = Y1;
    }
  }
}

// Weight of input sample x in output X of the transposed clamped correlation
// with taps t[0..2R] (u = -R..R) on an axis of n samples: the sum of t(u) over
// the u with clamp(x + u) = X; cum = prefix sums of t.
__device__ __forceinline__ float tap_T(const float* t, const float* cum, int R, int n, int X, int x) {
  if (n == 1) return cum[2 * R];
  if (X == 0) {
    const int k = R - x;  // u <= -x
    return k < 0 ? 0.f : cum[min(k, 2 * R)];
  }
  if (X == n - 1) {
    const int k0 = n - 1 - x + R;  // u >= n - 1 - x
    if (k0 > 2 * R) return 0.f;
    return k0 <= 0 ? cum[2 * R] : cum[2 * R] - cum[k0 - 1];
  }
  const int u = X - x;
  return (u >= -R && u <= R) ? t[u + R] : 0.f;
}

struct GTArgs {
  const float* g[SEG_MAX_ORIENT][SEG_MAX_LEVELS];    // dL/d|response|
  const float* mag[SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // |response|
  const float2* z[SEG_MAX_ORIENT][SEG_MAX_LEVELS];   // response
  float* gin[SEG_MAX_LEVELS];                        // dL/d intensity level (accumulated)
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  int lvl_first, lvl_last;
  int blk_off[SEG_MAX_LEVELS + 1];
};

// Reverse of the Gabor magnitude (Sec. 7.2): with gz = g (re, im)/|z| and the
// filter K = hx (x) vy - kappa g0 (x) g0, dL/din = Re[K^T conj(gz)], computed
// separably (x then y) on a tile with an R-sample halo.
__global__ void __launch_bounds__(256) k_db_gaborT(GTArgs a, GaborTaps t) {
  __shared__ float sGr[DB_TY + 2 * GB_MAXR_T][DB_TX + 2 * GB_MAXR_T];
  __shared__ float sGi[DB_TY + 2 * GB_MAXR_T][DB_TX + 2 * GB_MAXR_T];
  __shared__ float sAr[DB_TY + 2 * GB_MAXR_T][DB_TX], sAi[DB_TY + 2 * GB_MAXR_T][DB_TX];
  __shared__ float sBr[DB_TY + 2 * GB_MAXR_T][DB_TX], sBi[DB_TY + 2 * GB_MAXR_T][DB_TX];
  __shared__ float cg0[SEG_MAX_TAPS], chr[SEG_MAX_TAPS], chi[SEG_MAX_TAPS], cvr[SEG_MAX_TAPS], cvi[SEG_MAX_TAPS];
  int blk = blockIdx.x, l = a.lvl_first;
  while (l < a.lvl_last && blk >= a.blk_off[l - a.lvl_first + 1]) ++l;
  blk -= a.blk_off[l - a.lvl_first];
  const int h = a.hl[l], w = a.wl[l], b = blockIdx.y;
  const size_t fo = (size_t)b * h * w;
  const int ntx = (w + DB_TX - 1) / DB_TX;
  const int X0 = (blk % ntx) * DB_TX, Y0 = (blk / ntx) * DB_TY;
  const int R = t.R, K = 2 * R + 1;
  const int iny = DB_TY + 2 * R, inx = DB_TX + 2 * R;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads, two output rows each
  float out[2] = {0.f, 0.f};
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int u = 0; u < K; ++u) cg0[u] = (s += t.g0[u]);
  }
  for (int k = 0; k < t.no; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
      for (int u = 0; u < K; ++u) {
        chr[u] = (s1 += t.hx_re[k][u]);
        chi[u] = (s2 += t.hx_im[k][u]);
        cvr[u] = (s3 += t.vy_re[k][u]);
        cvi[u] = (s4 += t.vy_im[k][u]);
      }
    }
    const float* g = a.g[k][l] + fo;
    const float* mg = a.mag[k][l] + fo;
    const float2* z = a.z[k][l] + fo;
    for (int i = threadIdx.x; i < iny * inx; i += blockDim.x) {
      const int ry = i / inx, rx = i - ry * inx, y = Y0 - R + ry, x = X0 - R + rx;
      float gr = 0.f, gi = 0.f;
      if (y >= 0 && y < h && x >= 0 && x < w) {
        const size_t o = (size_t)y * w + x;
        const float m = mg[o];
        if (m > 0.f) {
          const float2 zz = z[o];
          const float s = g[o] / m;
          gr = s * zz.x;
          gi = s * zz.y;
        }
      }
      sGr[ry][rx] = gr;
      sGi[ry][rx] = gi;
    }
    __syncthreads();
    // along x: A = Hx^T conj(gz) (complex), B = G0^T (gr, gi)
    for (int i = threadIdx.x; i < iny * DB_TX; i += blockDim.x) {
      const int ry = i / DB_TX, lx = i - ry * DB_TX, X = X0 + lx;
      float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
      if (X > 0 && X < w - 1) {
        // interior output: plain correlation with the reversed taps (samples
        // outside the level are staged as zeros)
        const float* pr = &sGr[ry][lx + R];
        const float* pi = &sGi[ry][lx + R];
        for (int u = -R; u <= R; ++u) {
          const float whr = t.hx_re[k][u + R], whi = t.hx_im[k][u + R], w0 = t.g0[u + R];
          const float gr = pr[-u], gi = pi[-u];
          ar += whr * gr + whi * gi;  // (whr + i whi)(gr - i gi)
          ai += whi * gr - whr * gi;
          br += w0 * gr;
          bi += w0 * gi;
        }
      } else if (X < w) {
        const int xlo = max(0, X - R), xhi = min(w - 1, X + R);
        for (int x = xlo; x <= xhi; ++x) {
          const float whr = tap_T(t.hx_re[k], chr, R, w, X, x), whi = tap_T(t.hx_im[k], chi, R, w, X, x);
          const float w0 = tap_T(t.g0, cg0, R, w, X, x);
          const float gr = sGr[ry][x - X0 + R], gi = sGi[ry][x - X0 + R];
          ar += whr * gr + whi * gi;
          ai += whi * gr - whr * gi;
          br += w0 * gr;
          bi += w0 * gi;
        }
      }
      sAr[ry][lx] = ar;
      sAi[ry][lx] = ai;
      sBr[ry][lx] = br;
      sBi[ry][lx] = bi;
    }
    __syncthreads();
    // along y: Re[Vy^T A] - G0^T (kr B_r + ki B_i)
    const float kr = t.kap_re[k], ki = t.kap_im[k];
    for (int j = 0; j < 2; ++j) {
      const int Y = Y0 + ty + 8 * j, X = X0 + tx;
      if (Y >= h || X >= w) continue;
      float acc = 0.f;
      if (Y > 0 && Y < h - 1) {
        // rows outside the level hold zeros (staged as zero gradients)
        const int ry0 = Y - Y0 + R;
        for (int v = -R; v <= R; ++v) {
          const int ry = ry0 - v;
          acc += t.vy_re[k][v + R] * sAr[ry][tx] - t.vy_im[k][v + R] * sAi[ry][tx] -
                 t.g0[v + R] * (kr * sBr[ry][tx] + ki * sBi[ry][tx]);
        }
      } else {
        const int ylo = max(0, Y - R), yhi = min(h - 1, Y + R);
        for (int y = ylo; y <= yhi; ++y) {
          const int ry = y - Y0 + R;
          const float wvr = tap_T(t.vy_re[k], cvr, R, h, Y, y), wvi = tap_T(t.vy_im[k], cvi, R, h, Y, y);
          const float w0 = tap_T(t.g0, cg0, R, h, Y, y);
          acc += wvr * sAr[ry][tx] - wvi * sAi[ry][tx] - w0 * (kr * sBr[ry][tx] + ki * sBi[ry][tx]);
        }
      }
      out[j] += acc;
    }
  }
  for (int j = 0; j < 2; ++j) {
    const int Y = Y0 + ty + 8 * j, X = X0 + tx;
    if (Y < h && X < w) a.gin[l][fo + (size_t)Y * w + X] += out[j];
  }
}

__device__ __noinline__ bool pos3_exact(float a, float b, float c) {
  return 2.0 * (double)a - (double)b - (double)c > 0.0;
}

// Exact test 2a - b - c > 0 for floats a, b, c (the double evaluation is a call, so
// that it runs only on the rare operands near the kink).
__device__ __forceinline__ bool pos3(float a, float b, float c) {
  const float f = 2.f * a - b - c;
  // two roundings, each within 2^-24 of a partial sum bounded by 2|a| + |b| + |c|
  if (fabsf(f) > 1e-6f * (2.f * fabsf(a) + fabsf(b) + fabsf(c))) return f > 0.f;
  return pos3_exact(a, b, c);
}

// Level 1 -> level 0 transposed REDUCE of the three feature gradients, fused with
// the derivative of the features (Sec. 7.2 step 1):
//   I = s/765, s = r+g+b; where 10 s > max s: rn = 3r/s (gn, bn likewise),
//   R = max(0, rn - (gn+bn)/2), G, B likewise, Y = max(0, (rn+gn)/2 - |rn-gn|/2 - bn),
//   RG = R - G, BY = B - Y.
__global__ void __launch_bounds__(256) k_db_feat(const float* __restrict__ rgb, const int* __restrict__ smax_p,
                                                 const float* __restrict__ gI1, const float* __restrict__ gRG1,
                                                 const float* __restrict__ gBY1, int H, int W, int h1, int w1,
                                                 const int* __restrict__ lo_y, const float4* __restrict__ w_y,
                                                 const int* __restrict__ lo_x, const float4* __restrict__ w_x,
                                                 float* __restrict__ g_rgb) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  const int b = blockIdx.z;
  const size_t o1 = (size_t)b * h1 * w1;
  const int ylo = lo_y[y], xlo = lo_x[x];
  const float4 wy = w_y[y], wx = w_x[x];
  const float gI = rt_apply(gI1 + o1, w1, h1, ylo, wy, xlo, wx);
  const float gRG = rt_apply(gRG1 + o1, w1, h1, ylo, wy, xlo, wx);
  const float gBY = rt_apply(gBY1 + o1, w1, h1, ylo, wy, xlo, wx);
  const size_t p = ((size_t)b * H + y) * W + x;
  const float r = rgb[3 * p], g = rgb[3 * p + 1], bl = rgb[3 * p + 2], s = r + g + bl;
  const float smax = __int_as_float(smax_p[b]);
  float gs = gI / 765.f, gr = gs, gg = gs, gb = gs;
  if (10.f * s > smax) {
    // the clamps' decisions are signs of linear forms of (r, g, b) (s > 0 scales
    // out), evaluated exactly in double: R > 0 iff 2r - g - b > 0, Y > 0 iff
    // min(r, g) > b, sign(rn - gn) = sign(r - g)
    // (a 3-term form in float is re-evaluated in double only when it lies within
    // its rounding bound of zero; min(r, g) > b and r > g are exact comparisons)
    const float inv = 3.f / s;
    const float aR = pos3(r, g, bl), aG = pos3(g, r, bl), aB = pos3(bl, r, g);
    const float aY = fminf(r, g) > bl;
    const float sd = r > g ? 1.f : (r < g ? -1.f : 0.f);
    const float dR = gRG, dG = -gRG, dB = gBY, dY = -gBY;
    const float grn = dR * aR - 0.5f * dG * aG - 0.5f * dB * aB + dY * aY * (0.5f - 0.5f * sd);
    const float ggn = -0.5f * dR * aR + dG * aG - 0.5f * dB * aB + dY * aY * (0.5f + 0.5f * sd);
    const float gbn = -0.5f * dR * aR - 0.5f * dG * aG + dB * aB - dY * aY;
    const float tt = (grn * r + ggn * g + gbn * bl) * inv / s;  // rn = 3 r / s
    gr += grn * inv - tt;
    gg += ggn * inv - tt;
    gb += gbn * inv - tt;
  }
  g_rgb[3 * p] = gr;
  g_rgb[3 * p + 1] = gg;
  g_rgb[3 * p + 2] = gb;
}

__global__ void k_db_final(const double* __restrict__ gpar, int B, double* __restrict__ g_theta) {
  const int j = threadIdx.x;
  if (j >= 6) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += gpar[6 * b + j];
  g_theta[j] = s;
}

// ------------------------------------------------------------------ host side
struct DiffLayout {
  size_t kal, Tx, part, gS, gC3, G[SEG_MAX_LEVELS], coef, dpart, targ, hsur, grad, gpar, rsT, rtlo, rtw, total;
  size_t gpyr[3][SEG_MAX_LEVELS], gori[SEG_MAX_ORIENT][SEG_MAX_LEVELS], grad_bytes;
};

static int diff_layout(seg_diff* d, int B, int H, int W, const seg_params& p, DiffLayout& L) {
  size_t sal_bytes = 0;
  int rc = sal_layout(d->sal, B, H, W, p, &sal_bytes, true);
  if (rc) return rc;
  SalWS& s = d->sal;
  const int T = s.tile;
  const int hS = s.hl[s.sS], wS = s.wl[s.sS], nS = hS * wS;
  if (((hS + T - 1) / T) * ((wS + T - 1) / T) > DB_MAXT_S) return SEG_EINVAL;
  for (int q = 0; q < s.npairs; ++q) {
    const int c = s.pair_c[q];
    if (((s.hl[c] + T - 1) / T) * ((s.wl[c] + T - 1) / T) > DB_MAXT) return SEG_EINVAL;
  }
  if ((size_t)DB_RB * W * sizeof(float) > 40 * 1024) return SEG_EINVAL;  // W <= 5120
  for (int q = 0; q < s.npairs; ++q) {  // one surround row's transposed field fits a chunk
    const int d = s.pair_s[q] - s.pair_c[q];
    if ((long long)((1 << d) + 3) * s.wl[s.pair_s[q]] > SURT_CAP) return SEG_EINVAL;
  }
  size_t off = seg_align(sal_bytes);
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += seg_align(bytes);
    return o;
  };
  const size_t Bz = B;
  d->nbx = (H + DB_RB - 1) / DB_RB;
  L.kal = take(Bz * 3 * sizeof(double));
  L.Tx = take(Bz * H * wS * sizeof(float));
  L.part = take(Bz * d->nbx * 2 * sizeof(double));
  L.gS = take(Bz * nS * sizeof(float));
  L.gC3 = take(Bz * nS * sizeof(float));
  for (int c = s.c_min; c <= s.c_max; ++c) L.G[c] = take(Bz * s.nch * s.hl[c] * s.wl[c] * sizeof(float));
  L.coef = take(Bz * s.nmaps * sizeof(DiffCoef));
  L.dpart = take(Bz * s.nbands_total * sizeof(DiffPart));
  d->ntarg = 0;
  d->nhsur = 0;
  for (int q = 0; q < s.npairs; ++q) {
    const int c = s.pair_c[q];
    d->targ_off[q] = d->ntarg;
    d->ntarg += s.nch * ((s.hl[c] + T - 1) / T) * ((s.wl[c] + T - 1) / T);
    d->hsur_off[q] = d->nhsur;
    d->nhsur += (size_t)s.nch * s.hl[c] * s.wl[c];
  }
  L.targ = take(Bz * d->ntarg * sizeof(int));
  L.hsur = take(Bz * d->nhsur * sizeof(float));
  // gradients of the pyramid and Gabor levels: one contiguous block (zeroed per call)
  L.grad = off;
  for (int ch = 0; ch < 3; ++ch)
    for (int l = 1; l < s.L; ++l) L.gpyr[ch][l] = take(Bz * s.hl[l] * s.wl[l] * sizeof(float));
  for (int k = 0; k < s.no; ++k)
    for (int l = s.c_min; l <= s.s_max; ++l) L.gori[k][l] = take(Bz * s.hl[l] * s.wl[l] * sizeof(float));
  L.grad_bytes = off - L.grad;
  L.gpar = take(Bz * 6 * sizeof(double));
  int n = 0;
  for (int q = 0; q < s.npairs; ++q) {
    d->rsT_row[q] = n;
    n += s.hl[s.pair_s[q]];
    d->rsT_col[q] = n;
    n += s.wl[s.pair_s[q]];
  }
  d->rsT_frow = n;
  n += hS;
  d->rsT_fcol = n;
  n += wS;
  d->rsT_n = n;
  L.rsT = take(n * sizeof(int2));
  int nr = 0;
  for (int l = 0; l + 1 < s.L; ++l) {
    d->rt_row[l] = nr;
    nr += s.hl[l];
    d->rt_col[l] = nr;
    nr += s.wl[l];
  }
  d->rt_n = nr;
  L.rtlo = take(nr * sizeof(int));
  L.rtw = take(nr * sizeof(float4));
  L.total = off;
  return SEG_OK;
}

// ranges[i] = {first, last + 1} of the output samples whose bilinear taps (of the
// resampling ns -> nd) include source sample i.
static void transposed_ranges(int ns, int nd, int2* ranges) {
  for (int i = 0; i < ns; ++i) ranges[i] = make_int2(nd, 0);
  for (int dd = 0; dd < nd; ++dd) {
    const int2 e = seg_rs_entry(dd, ns, nd);
    const int i0 = e.x & 0xffff, i1 = e.x >> 16;
    for (int i : {i0, i1}) {
      ranges[i].x = std::min(ranges[i].x, dd);
      ranges[i].y = std::max(ranges[i].y, dd + 1);
    }
  }
  for (int i = 0; i < ns; ++i)
    if (ranges[i].y == 0) ranges[i] = make_int2(0, 0);
}

// Transposed REDUCE along one axis (n samples -> n2 = ceil(n/2)): output sample
// y receives level-(l+1) samples Y = lo + j (j < 4) with weight
// sum_t k(t) [clamp(2Y + t, 0, n-1) = y], k = [1 4 6 4 1]/16.
static void reduceT_table(int n, int n2, int* lo, float4* w) {
  static const float kb[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
  for (int y = 0; y < n; ++y) {
    lo[y] = std::max(0, y / 2 - 1);
    float ws[4];
    for (int j = 0; j < 4; ++j) {
      const int Y = lo[y] + j;
      float acc = 0.f;
      for (int t = -2; t <= 2 && Y < n2; ++t)
        if (std::min(std::max(2 * Y + t, 0), n - 1) == y) acc += kb[t + 2];
      ws[j] = acc;
    }
    w[y] = make_float4(ws[0], ws[1], ws[2], ws[3]);
  }
}

extern "C" int seg_diff_workspace_bytes(int B, int H, int W, const seg_params* p, size_t* bytes) {
  if (!bytes || !p) return SEG_EINVAL;
  int rc = seg_check_params(p, H, W);
  if (rc) return rc;
  if (B < 1 || (long long)B * H * W > (1LL << 26)) return SEG_EINVAL;
  seg_diff* d = (seg_diff*)calloc(1, sizeof(seg_diff));
  if (!d) return SEG_ENOMEM;
  DiffLayout L;
  rc = diff_layout(d, B, H, W, *p, L);
  if (!rc) *bytes = L.total;
  free(d);
  return rc;
}

extern "C" int seg_diff_create(void* stream, int B, int H, int W, const seg_params* p, seg_diff** out) {
  if (!out) return SEG_EINVAL;
  *out = nullptr;
  int rc = seg_check_params(p, H, W);
  if (rc) return rc;
  if (B < 1 || (long long)B * H * W > (1LL << 26)) return SEG_EINVAL;
  seg_diff* d = (seg_diff*)calloc(1, sizeof(seg_diff));
  if (!d) return SEG_ENOMEM;
  d->stream = (cudaStream_t)stream;
  d->B = B;
  d->H = H;
  d->W = W;
  d->p = *p;
  DiffLayout L;
  rc = diff_layout(d, B, H, W, *p, L);
  if (rc || cudaGetDevice(&d->device) != cudaSuccess) {
    free(d);
    return rc ? rc : SEG_ECUDA;
  }
  char* base = nullptr;
  if (cudaMalloc((void**)&base, L.total) != cudaSuccess) {
    free(d);
    return SEG_ENOMEM;
  }
  d->arena = base;
  d->bytes = L.total;
  sal_bind(d->sal, base);
  SalWS& s = d->sal;
  d->kal = (double*)(base + L.kal);
  d->Tx = (float*)(base + L.Tx);
  d->part = (double*)(base + L.part);
  d->gS = (float*)(base + L.gS);
  d->gC3 = (float*)(base + L.gC3);
  for (int c = s.c_min; c <= s.c_max; ++c) d->G[c] = (float*)(base + L.G[c]);
  d->coef = (DiffCoef*)(base + L.coef);
  d->dpart = (DiffPart*)(base + L.dpart);
  d->targ = (int*)(base + L.targ);
  d->hsur = (float*)(base + L.hsur);
  for (int ch = 0; ch < 3; ++ch)
    for (int l = 1; l < s.L; ++l) d->gpyr[ch][l] = (float*)(base + L.gpyr[ch][l]);
  for (int k = 0; k < s.no; ++k)
    for (int l = s.c_min; l <= s.s_max; ++l) d->gori[k][l] = (float*)(base + L.gori[k][l]);
  d->grad_base = base + L.grad;
  d->grad_bytes = L.grad_bytes;
  d->gpar = (double*)(base + L.gpar);
  d->rsT = (int2*)(base + L.rsT);
  d->rt_lo = (int*)(base + L.rtlo);
  d->rt_w = (float4*)(base + L.rtw);
  rc = sal_upload_tables(s);
  if (!rc) {
    std::vector<int2> t(d->rsT_n);
    for (int q = 0; q < s.npairs; ++q) {
      const int c = s.pair_c[q], sv = s.pair_s[q];
      transposed_ranges(s.hl[sv], s.hl[c], &t[d->rsT_row[q]]);
      transposed_ranges(s.wl[sv], s.wl[c], &t[d->rsT_col[q]]);
    }
    transposed_ranges(s.hl[s.sS], H, &t[d->rsT_frow]);
    transposed_ranges(s.wl[s.sS], W, &t[d->rsT_fcol]);
    if (cudaMemcpy(d->rsT, t.data(), sizeof(int2) * d->rsT_n, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = SEG_ECUDA;
    std::vector<int> lo(d->rt_n);
    std::vector<float4> wt(d->rt_n);
    for (int l = 0; l + 1 < s.L; ++l) {
      reduceT_table(s.hl[l], s.hl[l + 1], &lo[d->rt_row[l]], &wt[d->rt_row[l]]);
      reduceT_table(s.wl[l], s.wl[l + 1], &lo[d->rt_col[l]], &wt[d->rt_col[l]]);
    }
    if (!rc && (cudaMemcpy(d->rt_lo, lo.data(), sizeof(int) * d->rt_n, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(d->rt_w, wt.data(), sizeof(float4) * d->rt_n, cudaMemcpyHostToDevice) != cudaSuccess))
      rc = SEG_ECUDA;
  }
  if (rc) {
    cudaFree(base);
    free(d);
    return rc;
  }
  *out = d;
  return SEG_OK;
}

extern "C" int seg_diff_destroy(seg_diff* d) {
  if (!d) return SEG_EINVAL;
  cudaFree(d->arena);
  free(d);
  return SEG_OK;
}

extern "C" int seg_diff_forward(seg_diff* d, const float* rgb, const float* fmap, const double* theta, int t0,
                                float* saliency, float* prior) {
  if (!d || !rgb || !theta || !prior || t0 < 0 || t0 > (1 << 24)) return SEG_EINVAL;
  SalWS& s = d->sal;
  cudaStream_t st = d->stream;
  k_df_kalman<<<1, 32, 0, st>>>(theta, t0, d->B, d->kal);
  int rc = sal_run(s, st, rgb, true, nullptr, theta, nullptr, false);
  if (rc) return rc;
  dim3 g((d->W + 63) / 64, (d->H + 3) / 4, d->B);
  k_df_prior<<<g, 256, 0, st>>>(s.S, s.hl[s.sS], s.wl[s.sS], d->H, d->W, s.rs + s.rs_frow, s.rs + s.rs_fcol,
                                s.salmax, d->kal, fmap, d->p.border_px, d->p.eps, saliency, prior);
  SEG_CUDA_TRY(cudaGetLastError());
  d->forward_done = 1;
  return SEG_OK;
}

static void fill_dcs(const seg_diff* d, DCSArgs& a) {
  const SalWS& s = d->sal;
  memset(&a, 0, sizeof(a));
  for (int l = 0; l < s.L; ++l) {
    a.hl[l] = s.hl[l];
    a.wl[l] = s.wl[l];
    for (int ch = 0; ch < 3; ++ch) {
      a.X[ch][l] = l >= 1 ? s.pyr[ch][l] : nullptr;
      a.GX[ch][l] = l >= 1 ? d->gpyr[ch][l] : nullptr;
    }
    for (int k = 0; k < s.no; ++k) {
      const bool in = l >= s.c_min && l <= s.s_max;
      a.X[3 + k][l] = in ? s.ori[k][l] : nullptr;
      a.GX[3 + k][l] = in ? d->gori[k][l] : nullptr;
    }
  }
  for (int c = s.c_min; c <= s.c_max; ++c) a.G[c] = d->G[c];
  a.npairs = s.npairs;
  a.nch = s.nch;
  a.nmaps = s.nmaps;
  a.tile = s.tile;
  a.opp_sum = s.opp_sum;
  a.flat = s.flat;
  a.rs = s.rs;
  a.rsT = d->rsT;
  for (int q = 0; q < s.npairs; ++q) {
    a.pair_c[q] = s.pair_c[q];
    a.pair_s[q] = s.pair_s[q];
    a.rs_row[q] = s.rs_row[q];
    a.rs_col[q] = s.rs_col[q];
    a.rsT_row[q] = d->rsT_row[q];
    a.rsT_col[q] = d->rsT_col[q];
    a.targ_off[q] = d->targ_off[q];
    a.hsur_off[q] = d->hsur_off[q];
  }
  a.coef = d->coef;
  a.targ = d->targ;
  a.ntarg = d->ntarg;
  a.hsur = d->hsur;
  a.nhsur = d->nhsur;
  int off = 0;
  for (int q = 0; q < s.npairs; ++q) {
    a.band_off[q] = off;
    off += s.nch * ((s.hl[s.pair_c[q]] + s.tile - 1) / s.tile);
  }
  a.band_off[s.npairs] = off;
  a.nbands_total = off;
  a.dpart = d->dpart;
  a.nsl = 0;
  for (int sv = 0; sv < s.L; ++sv) {
    bool any = false;
    for (int q = 0; q < s.npairs; ++q) any |= s.pair_s[q] == sv;
    if (any) a.slist[a.nsl++] = sv;
  }
}

extern "C" int seg_diff_backward(seg_diff* d, const float* rgb, const float* fmap, const double* theta,
                                 const float* g_prior, const float* g_sal, float* g_rgb, double* g_theta) {
  if (!d || !rgb || !theta || !g_prior || !g_rgb || !g_theta) return SEG_EINVAL;
  if (!d->forward_done) return SEG_EINVAL;
  SalWS& s = d->sal;
  cudaStream_t st = d->stream;
  const int B = d->B, H = d->H, W = d->W;
  const int hS = s.hl[s.sS], wS = s.wl[s.sS];
  SEG_CUDA_TRY(cudaMemsetAsync(d->grad_base, 0, d->grad_bytes, st));
  k_db_rows<<<dim3(d->nbx, B), 256, DB_RB * W * sizeof(float), st>>>(
      s.S, hS, wS, H, W, s.rs + s.rs_frow, s.rs + s.rs_fcol, d->rsT + d->rsT_fcol, s.salmax, d->kal, fmap, g_prior,
      g_sal, d->p.border_px, d->p.eps, d->Tx, d->part);
  TopArgs ta;
  ta.Tx = d->Tx;
  ta.part = d->part;
  ta.nbx = d->nbx;
  ta.H = H;
  ta.W = W;
  ta.hs = hS;
  ta.ws = wS;
  ta.nch = s.nch;
  ta.tile = s.tile;
  ta.flat = s.flat;
  ta.frow = s.rs + s.rs_frow;
  ta.fcol = s.rs + s.rs_fcol;
  ta.frowT = d->rsT + d->rsT_frow;
  ta.salmax = s.salmax;
  ta.S = s.S;
  ta.consp = s.consp;
  ta.acc = s.acc_final;
  ta.csum = s.csum;
  ta.kal = d->kal;
  ta.theta = theta;
  ta.gS = d->gS;
  ta.gC3 = d->gC3;
  ta.gacc = d->G[s.c_max];
  ta.gpar = d->gpar;
  k_db_top<<<B, 1024, 0, st>>>(ta);
  k_db_nbwd<<<dim3(4, B), 512, 0, st>>>(ta, 0);
  k_db_nbwd<<<dim3(s.no, B), 512, 0, st>>>(ta, 1);
  // across-scale sums: G_c = REDUCE^T G_{c+1}
  for (int c = s.c_max - 1; c >= s.c_min; --c) {
    RTArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.in[0] = d->G[c + 1];
    ra.out[0] = d->G[c];
    ra.K = 1;
    ra.h = s.hl[c];
    ra.w = s.wl[c];
    ra.h2 = s.hl[c + 1];
    ra.w2 = s.wl[c + 1];
    ra.accumulate = 0;
    ra.lo_y = d->rt_lo + d->rt_row[c];
    ra.w_y = d->rt_w + d->rt_row[c];
    ra.lo_x = d->rt_lo + d->rt_col[c];
    ra.w_x = d->rt_w + d->rt_col[c];
    k_db_reduceT<<<dim3((ra.w + 31) / 32, (ra.h + 7) / 8, s.nch * B), 256, 0, st>>>(ra);
  }
  DCSArgs ca;
  fill_dcs(d, ca);
  k_db_cs_stats<<<dim3(ca.nbands_total, B), 256, 0, st>>>(ca);
  k_db_cs_coef<<<(s.nmaps * B + 127) / 128, 128, 0, st>>>(ca, B);
  for (int c = s.c_min; c <= s.c_max; ++c)
    k_db_cs_apply<<<dim3((s.wl[c] + 31) / 32, (s.hl[c] + 7) / 8, s.nch * B), 256, 0, st>>>(ca, c);
  k_db_surT<<<dim3(ca.nsl, s.nch, B), 256, 0, st>>>(ca);
  GTArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.lvl_first = s.c_min;
  ga.lvl_last = s.s_max;
  int tot = 0;
  for (int l = s.c_min; l <= s.s_max; ++l) {
    for (int k = 0; k < s.no; ++k) {
      ga.g[k][l] = d->gori[k][l];
      ga.mag[k][l] = s.ori[k][l];
      ga.z[k][l] = s.oc[k][l];
    }
    ga.gin[l] = d->gpyr[0][l];
    ga.hl[l] = s.hl[l];
    ga.wl[l] = s.wl[l];
    ga.blk_off[l - s.c_min] = tot;
    tot += ((s.wl[l] + DB_TX - 1) / DB_TX) * ((s.hl[l] + DB_TY - 1) / DB_TY);
  }
  ga.blk_off[s.s_max - s.c_min + 1] = tot;
  k_db_gaborT<<<dim3(tot, B), 256, 0, st>>>(ga, s.taps);
  // pyramid: level l -> l-1, from the top
  for (int l = s.L - 1; l >= 2; --l) {
    RTArgs ra;
    memset(&ra, 0, sizeof(ra));
    for (int ch = 0; ch < 3; ++ch) {
      ra.in[ch] = d->gpyr[ch][l];
      ra.out[ch] = d->gpyr[ch][l - 1];
    }
    ra.K = 3;
    ra.h = s.hl[l - 1];
    ra.w = s.wl[l - 1];
    ra.h2 = s.hl[l];
    ra.w2 = s.wl[l];
    ra.accumulate = 1;
    ra.lo_y = d->rt_lo + d->rt_row[l - 1];
    ra.w_y = d->rt_w + d->rt_row[l - 1];
    ra.lo_x = d->rt_lo + d->rt_col[l - 1];
    ra.w_x = d->rt_w + d->rt_col[l - 1];
    k_db_reduceT<<<dim3((ra.w + 31) / 32, (ra.h + 7) / 8, 3 * B), 256, 0, st>>>(ra);
  }
  k_db_feat<<<dim3((W + 31) / 32, (H + 7) / 8, B), 256, 0, st>>>(
      rgb, s.smax, d->gpyr[0][1], d->gpyr[1][1], d->gpyr[2][1], H, W, s.hl[1], s.wl[1], d->rt_lo + d->rt_row[0],
      d->rt_w + d->rt_row[0], d->rt_lo + d->rt_col[0], d->rt_w + d->rt_col[0], g_rgb);
  k_db_final<<<1, 32, 0, st>>>(d->gpar, B, g_theta);
  SEG_CUDA_TRY(cudaGetLastError());
  return SEG_OK;
}
