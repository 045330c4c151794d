// prior_terms.cu -- saliency prior, Kalman update and MRF terms on sm_103a.
//
//   k_prior      Sec. 5 + Sec. 6: q = saliency / max (eps on the border band),
//                f = separable Gaussian of the previous mask (shared-memory halo
//                tile), p-hat = w_f f + (1 - w_f) q.  w_f comes from the device
//                Kalman state, so a frame needs no host round trip.
//                In seg_push_frame it also runs the first pass of the
//                prior-weighted colour moments (Sec. 5: all pixels, weighted by
//                p-hat for the object and 1 - p-hat for the background); its last
//                CTA reduces the per-CTA partials in a fixed order into the means
//                and advances the Kalman variance (Sec. 6 equations).
//   k_mom1       the same first pass alone (stage entry seg_terms)
//   k_mom2       second pass: centred weighted second moments (no cancellation);
//                its last CTA forms covariance + 1e-4 I, the Cholesky factor,
//                its inverse and the log-determinant
//   k_terms      Eqs. 1-4: t-links from D(a) = lambda_u psi_1(a) + xi_1(a),
//                shifted by min_a D(a) and quantised; n-links from a host-built
//                FP64 table indexed by |delta(r+g+b)| and the diagonal flag.
#include <math.h>
#include <string.h>

#include "seg_internal.cuh"

#define PR_TX 32
#define PR_TY 16
#define PR_MAXR 8
#define MOM_PX 4  // pixels per thread in the moment passes (2: twice the CTAs, which crowded the concurrent
                  // saliency of the next frame -- pipelined 640x480 ~6085 against ~6285 frames/s)

struct PriorArgs {
  float* sal;      // input map, or (from_S) the saliency output (nullable)
  const float* S;  // from_S: the combined map at sigma_S, hS x wS per frame
  int hS, wS, from_S;
  const int2* frow;  // from_S: up-sampling tables S -> H x W
  const int2* fcol;
  const unsigned* salmax;
  const uint8_t* prev;
  const KalmanDev* kal;  // nullable: use wf_host
  double wf_host;
  double a, b;  // sigma1^2, sigma2^2
  int H, W, border;
  float eps;
  int fR;
  float ftap[2 * PR_MAXR + 1];
  float* prior;
  // fused first moment pass (rgb == nullptr: off)
  const uint8_t* rgb;
  float* part;
  int part_stride;     // partials per frame
  unsigned* counter;
  GaussDev* gauss;
  KalmanDev* kal_adv;  // nullable: advance the variance recursion
  const SegIO* io;     // sal / prior / rgb == nullptr: take them from here
  const uint8_t* on;   // [B] slots holding a stream (nullptr: all)
};

struct MomFinArgs {
  float* part;
  int part_stride;  // partials per frame
  unsigned* counter;
  GaussDev* gauss;
  KalmanDev* kal;  // nullable: advance the variance recursion
  double a, b;
  const SegIO* io;  // rgb / prior == nullptr: take them from here
  const uint8_t* on;
};

__device__ __forceinline__ void mom1_add_rgb(float p, int r8, int g8, int b8, float* s) {
  float r = r8 / 255.f, g = g8 / 255.f, b = b8 / 255.f;
  float w0 = 1.f - p;
  s[0] += w0;
  s[1] += w0 * r;
  s[2] += w0 * g;
  s[3] += w0 * b;
  s[4] += p;
  s[5] += p * r;
  s[6] += p * g;
  s[7] += p * b;
}
__device__ __forceinline__ void mom1_add(float p, const uint8_t* px, float* s) { mom1_add_rgb(p, px[0], px[1], px[2], s); }

// Centred second moments about the label means muf[label][channel] (Sec. 5):
// rr, gr, gg, br, bg, bb for the background (weight 1 - p), then the object (p).
__device__ __forceinline__ void mom2_add(float p, const uint8_t* px, const float* muf, float* s) {
  float r = px[0] / 255.f, g = px[1] / 255.f, b = px[2] / 255.f;
  float w0 = 1.f - p;
  float dr = r - muf[0], dg = g - muf[1], db = b - muf[2];
  s[0] += w0 * dr * dr;
  s[1] += w0 * dg * dr;
  s[2] += w0 * dg * dg;
  s[3] += w0 * db * dr;
  s[4] += w0 * db * dg;
  s[5] += w0 * db * db;
  dr = r - muf[3];
  dg = g - muf[4];
  db = b - muf[5];
  s[6] += p * dr * dr;
  s[7] += p * dg * dr;
  s[8] += p * dg * dg;
  s[9] += p * db * dr;
  s[10] += p * db * dg;
  s[11] += p * db * db;
}

// Finalisation arithmetic (one or two threads while the rest of the grid has
// finished).  FP64 divide, square root and log are long dependent sequences on
// this part's narrow FP64 pipe (hundreds to thousands of cycles each), so they
// are formed by Newton's iteration from a float seed: reciprocal r <- r (2 - x r)
// and reciprocal square root y <- y (3 - x y^2) / 2 each square the relative
// error per step, so two steps take the ~1e-7 seed below the double rounding.
#define LOG_2PI 1.8378770664093453
__device__ __forceinline__ double nr_rcp(double x) {
  if (!(fabs(x) > 1e-30 && fabs(x) < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double nr_rsqrt(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  const double h = 0.5 * x;
  double y = (double)rsqrtf((float)x);
  y = y * fma(-h * y, y, 1.5);
  return y * fma(-h * y, y, 1.5);
}
// log x to float accuracy (the results are stored as float): logf of the float
// rounding xf plus the first-order term of log(x / xf), |x / xf - 1| < 2^-24.
__device__ __forceinline__ double log_f(double x) {
  if (!(x > 1e-30 && x < 1e30)) return log(x);
  const float xf = (float)x;
  return (double)logf(xf) + (x - (double)xf) * (double)__frcp_rn(xf);
}

template <int NV>
__device__ void reduce_parts(const float* part, int nblocks, double* out);
template <int NV>
__device__ bool block_partial_last(const float* v, float* part, unsigned* counter, int bid,
                                   int nblocks);
__device__ void finalize_means(const double* tot, GaussDev* g, KalmanDev* kal, double a, double b);

// Pointers of frame fb of a batch (and, when captured, the frame's I/O).
__device__ __forceinline__ void prior_frame(PriorArgs& a, int fb) {
  if (a.io) {
    if (!a.sal) a.sal = a.io->sal;
    if (!a.prior) a.prior = a.io->prior;
    if (!a.rgb) a.rgb = a.io->rgb;
  }
  const size_t n = (size_t)a.H * a.W;
  if (a.sal) a.sal += fb * n;
  if (a.from_S) a.S += (size_t)fb * a.hS * a.wS;
  a.prior += fb * n;
  if (a.prev) a.prev += fb * n;
  if (a.rgb) a.rgb += fb * 3 * n;
  a.salmax += fb;
  if (a.kal) a.kal += fb;
  if (a.kal_adv) a.kal_adv += fb;
  a.gauss += fb;
  a.part += (size_t)fb * a.part_stride;
  a.counter += fb;
}

// Thread 0: the blur taps into shared memory (indexed by a runtime tap, so not
// read from the parameter block) and, Sec. 6, the weight on f(A_{t-1}).
__device__ __forceinline__ void prior_setup(const PriorArgs& a, float* sTap, float* s_wf) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int u = 0; u < 2 * PR_MAXR + 1; ++u) sTap[u] = a.ftap[u];
    double wf = a.wf_host;
    if (a.kal) {
      int t = a.kal->t;
      double P = a.kal->P;
      wf = t == 0 ? 0.0 : a.a * nr_rcp(a.a + a.b + P);
    }
    *s_wf = (float)wf;
  }
}

typedef float PrTileM[PR_TX + 2 * PR_MAXR];
typedef float PrTileH[PR_TX];

// The previous mask on a tile and its halo, into sM (no barrier).
__device__ __forceinline__ void prior_tile_mask(const PriorArgs& a, int X0, int Y0, PrTileM* sM) {
  const int R = a.fR, iny = PR_TY + 2 * R, inx = PR_TX + 2 * R;
  for (int i = threadIdx.x; i < iny * inx; i += blockDim.x) {
    int ry = i / inx, rx = i - ry * inx;
    int gy = seg_clampi(Y0 - R + ry, 0, a.H - 1), gx = seg_clampi(X0 - R + rx, 0, a.W - 1);
    sM[ry][rx] = (float)a.prev[(size_t)gy * a.W + gx];
  }
}

// The prior on one PR_TX x PR_TY tile (whole CTA, any block size), adding the
// first-moment sums of its pixels to ms when a.rgb is set.  Consecutive calls
// may reuse sM / sH: each call's barriers order them.  mask_loaded: sM already
// holds the tile's mask (prior_tile_mask, before a barrier).  A thread's two
// pixels (i, i + blockDim.x) issue all their loads before any store.
__device__ __forceinline__ void prior_tile(const PriorArgs& a, int X0, int Y0, float wff, bool use_f, float mx,
                                           const float* sTap, PrTileM* sM, PrTileH* sH, float* ms,
                                           bool mask_loaded = false) {
  const int R = a.fR, iny = PR_TY + 2 * R;
  if (use_f) {
    if (!mask_loaded) {
      prior_tile_mask(a, X0, Y0, sM);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < iny * PR_TX; i += blockDim.x) {
      int ry = i / PR_TX, x = i - ry * PR_TX;
      float acc = 0.f;
      for (int u = 0; u <= 2 * R; ++u) acc += sTap[u] * sM[ry][x + u];
      sH[ry][x] = acc;
    }
    __syncthreads();
  }
  for (int i0 = threadIdx.x; i0 < PR_TY * PR_TX; i0 += 2 * blockDim.x) {
    float sv[2], fv[2];
    int px[2][3];
    bool ok[2], edge[2];
    size_t gg[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = i0 + u * blockDim.x;
      const int y = i / PR_TX, x = i - y * PR_TX;
      const int gy = Y0 + y, gx = X0 + x;
      ok[u] = i < PR_TY * PR_TX && gy < a.H && gx < a.W;
      gg[u] = ok[u] ? (size_t)gy * a.W + gx : 0;
      edge[u] = gy < a.border || gy >= a.H - a.border || gx < a.border || gx >= a.W - a.border;
      sv[u] = 0.f;
      fv[u] = 0.f;
      px[u][0] = px[u][1] = px[u][2] = 0;
      if (ok[u]) {
        // the saliency map at this pixel (from_S: bilinear up-sampling of S)
        sv[u] = a.from_S ? seg_bilinear_t(a.S, a.wS, a.frow[gy], a.fcol[gx]) : a.sal[gg[u]];
        if (use_f) {
          float f = 0.f;
          for (int v = 0; v <= 2 * R; ++v) f += sTap[v] * sH[y + v][x];
          fv[u] = f;
        }
        if (a.rgb) {
          const uint8_t* q = a.rgb + 3 * gg[u];
          px[u][0] = q[0];
          px[u][1] = q[1];
          px[u][2] = q[2];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!ok[u]) continue;
      if (a.from_S && a.sal) a.sal[gg[u]] = sv[u];
      float q = edge[u] ? a.eps : (mx > 0.f ? sv[u] / mx : 0.f);
      float p = (1.f - wff) * q;
      if (use_f) p += wff * fv[u];
      a.prior[gg[u]] = p;
      if (a.rgb) mom1_add_rgb(p, px[u][0], px[u][1], px[u][2], ms);
    }
  }
}

__global__ void __launch_bounds__(256) k_prior(PriorArgs a) {
  __shared__ float sM[PR_TY + 2 * PR_MAXR][PR_TX + 2 * PR_MAXR];
  __shared__ float sH[PR_TY + 2 * PR_MAXR][PR_TX];
  __shared__ float s_wf;
  __shared__ float sTap[2 * PR_MAXR + 1];
  // Before waiting for the preceding kernel (the saliency's last, which writes S
  // and its maximum): the I/O pointers, the Kalman state and the previous mask
  // tile, none of which it writes (the mask tile is unused when w_f = 0).
  if (SEG_SLOT_OFF(a.on, blockIdx.z)) return;
  prior_frame(a, blockIdx.z);
  prior_setup(a, sTap, &s_wf);
  if (a.prev) prior_tile_mask(a, blockIdx.x * PR_TX, blockIdx.y * PR_TY, sM);
  seg_pdl_enter();
  const float mx = __uint_as_float(*a.salmax);
  __syncthreads();
  const float wff = s_wf;
  const bool use_f = wff != 0.f && a.prev != nullptr;
  float ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  prior_tile(a, blockIdx.x * PR_TX, blockIdx.y * PR_TY, wff, use_f, mx, sTap, sM, sH, ms, true);
  if (a.rgb) {
    const int nb = gridDim.x * gridDim.y;
    if (block_partial_last<8>(ms, a.part, a.counter, blockIdx.y * gridDim.x + blockIdx.x, nb)) {
      __shared__ double tot[8];
      reduce_parts<8>(a.part, nb, tot);
      if (threadIdx.x == 0) finalize_means(tot, a.gauss, a.kal_adv, a.a, a.b);
    }
  }
}

// Writes this CTA's NV partial sums to part[k * nblocks + bid] (value-major, so
// the final sum reads them coalesced) and returns true in every thread of
// exactly one CTA, the last to finish (threadfence reduction).
// A CTA covers at most a few thousand pixels, so its sums are plain FP32; the
// sum across CTAs (reduce_parts) is an error-free float-float sum, which keeps
// about 44 bits without the FP64 pipe (narrow on this part).
template <int NV>
__device__ void block_partial_write(const float* v, float* part, int bid, int nblocks) {
  __shared__ float red[32][NV];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float s = seg_warp_sum_f(v[k]);
    if (lane == 0) red[wid][k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][k];
    part[k * nblocks + bid] = s;
    __threadfence();  // (only the writers need to fence)
  }
  __syncthreads();
}

template <int NV>
__device__ bool block_partial_last(const float* v, float* part, unsigned* counter, int bid, int nblocks) {
  __shared__ int is_last;
  block_partial_write<NV>(v, part, bid, nblocks);
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    is_last = prev == (unsigned)nblocks - 1u;
    if (is_last) *counter = 0u;  // ready for the next launch
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last != 0;
}

// (hi, lo) float pairs: two_sum gives s + e = a + b exactly (Knuth).
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
  const float s = x.x + y.x, bb = s - x.x;
  float e = (x.x - (s - bb)) + (y.x - bb);
  e += x.y + y.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// Deterministic fixed-order float-float sums of the NV per-CTA partials (one CTA):
// warp w sums values w, w + nw, .. (G of them in one pass, so their loads are in
// flight together), lanes striding over the CTAs, then a shuffle tree;
// out[k] = hi + lo.
template <int NV>
__device__ void reduce_parts(const float* part, int nblocks, double* out) {
  constexpr int G = NV <= 8 ? 1 : NV <= 16 ? 2 : 4;
  constexpr int U = G >= 4 ? 8 : 16;  // loads in flight per value (the sum order is b order either way)
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5, wid = threadIdx.x >> 5;
  for (int k0 = wid; k0 < NV; k0 += G * nw) {
    float2 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float2(0.f, 0.f);
    for (int b0 = lane; b0 < nblocks; b0 += 32 * U) {
      // L2 reads (other CTAs' partials are not in this L1), U x G in flight
      float v[G][U];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int k = k0 + g * nw;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int b = b0 + 32 * u;
          v[g][u] = k < NV && b < nblocks ? __ldcg(part + (size_t)k * nblocks + b) : 0.f;
        }
      }
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int u = 0; u < U; ++u) acc[g] = ff_add(acc[g], make_float2(v[g][u], 0.f));
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float2 other;
        other.x = __shfl_xor_sync(0xffffffffu, acc[g].x, o);
        other.y = __shfl_xor_sync(0xffffffffu, acc[g].y, o);
        acc[g] = lane < (lane ^ o) ? ff_add(acc[g], other) : ff_add(other, acc[g]);  // same order in both lanes
      }
      const int k = k0 + g * nw;
      if (lane == 0 && k < NV) out[k] = (double)acc[g].x + (double)acc[g].y;
    }
  }
  __syncthreads();
}

// Weighted means per label; advances sigma^2_xi1 (Sec. 6):
// P_t = a (b + P) / (a + b + P), and at t = 0 (P_{-1} = inf) P_0 = a.
__device__ void finalize_means(const double* tot, GaussDev* g, KalmanDev* kal, double a, double b) {
  g->degenerate = 0;
  for (int lab = 0; lab < 2; ++lab) {
    const double sw = tot[4 * lab];
    if (!(sw > 0.0)) g->degenerate |= 1 << lab;
    const double rsw = sw > 0.0 ? nr_rcp(sw) : 0.0;
    for (int k = 0; k < 3; ++k) {
      const double m = tot[4 * lab + 1 + k] * rsw;
      g->mu[lab][k] = m;
      g->muf[lab][k] = (float)m;
    }
    g->sw[lab] = sw;
  }
  if (kal) {
    double P = kal->P;
    kal->P = kal->t == 0 ? a : a * (b + P) * nr_rcp(a + b + P);
    kal->t += 1;
  }
}

// Cholesky factor of a 3x3 covariance (+ 1e-4 I already added), written as
// the inverse factor L^-1 (6 floats), and log det.  Pivots come from
// reciprocal square roots (L^-1 is what the data term needs): i_jj = 1/l_jj.
__device__ double chol_inv(double c00, double c10, double c11, double c20, double c21, double c22, float* li) {
  const double i00 = nr_rsqrt(c00);
  const double l10 = c10 * i00, l20 = c20 * i00;
  const double i11 = nr_rsqrt(c11 - l10 * l10);
  const double l21 = (c21 - l20 * l10) * i11;
  const double i22 = nr_rsqrt(c22 - l20 * l20 - l21 * l21);
  const double i10 = -l10 * i00 * i11;
  const double i21 = -l21 * i11 * i22;
  const double i20 = -(l20 * i00 + l21 * i10) * i22;
  li[0] = (float)i00;
  li[1] = (float)i10;
  li[2] = (float)i11;
  li[3] = (float)i20;
  li[4] = (float)i21;
  li[5] = (float)i22;
  return -2.0 * log_f(i00 * i11 * i22);  // log det = 2 log(l00 l11 l22)
}

// Covariance + 1e-4 I, Cholesky factor L, L^-1 and 1/2 log det + 3/2 log 2 pi.
__device__ void finalize_cov(const double* tot, GaussDev* g, int lab) {
  if (g->degenerate & (1 << lab)) {  // no pixel carries weight: psi_1 = 0 for this label
    for (int k = 0; k < 6; ++k) g->linv[lab][k] = 0.f;
    g->lconst[lab] = 0.f;
    return;
  }
  const double rsw = nr_rcp(g->sw[lab]);
  const double* m = tot + 6 * lab;  // rr, gr, gg, br, bg, bb
  const double c00 = m[0] * rsw + 1e-4, c10 = m[1] * rsw, c11 = m[2] * rsw + 1e-4;
  const double c20 = m[3] * rsw, c21 = m[4] * rsw, c22 = m[5] * rsw + 1e-4;
  const double ld = chol_inv(c00, c10, c11, c20, c21, c22, g->linv[lab]);
  g->lconst[lab] = (float)(0.5 * ld + 1.5 * LOG_2PI);
}

__global__ void __launch_bounds__(256) k_mom1(const uint8_t* __restrict__ rgb,
                                              const float* __restrict__ prior, int N, MomFinArgs f) {
  seg_pdl_enter();
  const int fb = blockIdx.y;  // frame of the batch
  if (SEG_SLOT_OFF(f.on, fb)) return;
  rgb += (size_t)fb * 3 * N;
  prior += (size_t)fb * N;
  f.part += (size_t)fb * f.part_stride;
  f.counter += fb;
  f.gauss += fb;
  if (f.kal) f.kal += fb;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    mom1_add(prior[i], rgb + 3 * (size_t)i, s);
  if (block_partial_last<8>(s, f.part, f.counter, blockIdx.x, gridDim.x)) {
    __shared__ double tot[8];
    reduce_parts<8>(f.part, gridDim.x, tot);
    if (threadIdx.x == 0) finalize_means(tot, f.gauss, f.kal, f.a, f.b);
  }
}

__global__ void __launch_bounds__(256) k_mom2(const uint8_t* __restrict__ rgb,
                                              const float* __restrict__ prior, int N, MomFinArgs f) {
  seg_pdl_enter();
  if (!rgb) rgb = f.io->rgb;
  if (!prior) prior = f.io->prior;
  const int fb = blockIdx.y;  // frame of the batch
  if (SEG_SLOT_OFF(f.on, fb)) return;
  rgb += (size_t)fb * 3 * N;
  prior += (size_t)fb * N;
  f.part += (size_t)fb * f.part_stride;
  f.counter += fb;
  f.gauss += fb;
  float s[12];
  for (int k = 0; k < 12; ++k) s[k] = 0.f;
  float muf[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) muf[k] = f.gauss->muf[k / 3][k % 3];
  int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) mom2_add(prior[i], rgb + 3 * (size_t)i, muf, s);
  if (block_partial_last<12>(s, f.part, f.counter, blockIdx.x, gridDim.x)) {
    __shared__ double tot[12];
    reduce_parts<12>(f.part, gridDim.x, tot);
    if (threadIdx.x < 2)  // one thread per label
      finalize_cov(tot, f.gauss, threadIdx.x);
  }
}

// ------------------------------------------------------------------ EM (M components)
#define EM_NV 30  // per component: weight, 3 shifted first moments, 6 shifted second moments

struct EMArgs {
  const uint8_t* rgb;
  const float* prior;
  int N, M;
  GmmDev* gmm;        // [frame][label]
  const GaussDev* gauss;
  float* part;        // [frame][label][blocks * EM_NV]
  int part_stride;
  unsigned* counter;  // [frame][label]
  const SegIO* io;
  const uint8_t* on;
};

// One EM iteration for label a of frame fb (blockIdx.y = 2 fb + a): E-step
// responsibilities from the current mixture, moments of every component about
// its current mean (so the update has no large cancellation); the last CTA
// forms pi, mu, Sigma (+ 1e-4 I) per component.  Components whose weight is
// below 1e-6 of the label's total keep their mean and covariance.
template <int M>
__global__ void __launch_bounds__(256) k_em_step(EMArgs a) {
  seg_pdl_enter();
  const int lab = blockIdx.y & 1, fb = blockIdx.y >> 1;
  if (SEG_SLOT_OFF(a.on, fb)) return;
  const GaussDev* gd = a.gauss + fb;
  if (gd->degenerate & (1 << lab)) return;  // uniform over the grid: no partials, no finalise
  const uint8_t* rgb = (a.rgb ? a.rgb : a.io->rgb) + (size_t)fb * 3 * a.N;
  const float* prior = (a.prior ? a.prior : a.io->prior) + (size_t)fb * a.N;
  GmmDev* g = a.gmm + 2 * fb + lab;
  float mu[M][3], li[M][6], lc[M];
  for (int m = 0; m < M; ++m) {
    for (int k = 0; k < 3; ++k) mu[m][k] = g->mu[m][k];
    for (int k = 0; k < 6; ++k) li[m][k] = g->linv[m][k];
    lc[m] = g->lc[m];
  }
  float s[EM_NV];
#pragma unroll
  for (int k = 0; k < EM_NV; ++k) s[k] = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
    float p = prior[i];
    float w = lab ? p : 1.f - p;
    float c[3] = {rgb[3 * (size_t)i] / 255.f, rgb[3 * (size_t)i + 1] / 255.f, rgb[3 * (size_t)i + 2] / 255.f};
    float lp[M], d[M][3], mx = -3.0e38f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
      for (int k = 0; k < 3; ++k) d[m][k] = c[k] - mu[m][k];
      float y0 = li[m][0] * d[m][0];
      float y1 = li[m][1] * d[m][0] + li[m][2] * d[m][1];
      float y2 = li[m][3] * d[m][0] + li[m][4] * d[m][1] + li[m][5] * d[m][2];
      lp[m] = lc[m] - 0.5f * (y0 * y0 + y1 * y1 + y2 * y2);
      mx = fmaxf(mx, lp[m]);
    }
    float z = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      lp[m] = expf(lp[m] - mx);
      z += lp[m];
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float wr = w * lp[m] / z;
      float* t = s + 10 * m;
      t[0] += wr;
      t[1] += wr * d[m][0];
      t[2] += wr * d[m][1];
      t[3] += wr * d[m][2];
      t[4] += wr * d[m][0] * d[m][0];
      t[5] += wr * d[m][1] * d[m][0];
      t[6] += wr * d[m][1] * d[m][1];
      t[7] += wr * d[m][2] * d[m][0];
      t[8] += wr * d[m][2] * d[m][1];
      t[9] += wr * d[m][2] * d[m][2];
    }
  }
  float* part = a.part + (size_t)(2 * fb + lab) * a.part_stride;
  if (block_partial_last<EM_NV>(s, part, a.counter + 2 * fb + lab, blockIdx.x, gridDim.x)) {
    __shared__ double tot[EM_NV];
    reduce_parts<EM_NV>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
      double ntot = 0.0;
      for (int m = 0; m < M; ++m) ntot += tot[10 * m];
      const double rtot = nr_rcp(ntot);
      for (int m = 0; m < M; ++m) {
        const double* t = tot + 10 * m;
        const double nm = t[0], pim = nm * rtot;
        double ld = g->logdet[m];
        if (nm >= 1e-6 * ntot) {
          const double rn = nr_rcp(nm);
          double dx = t[1] * rn, dy = t[2] * rn, dz = t[3] * rn;
          for (int k = 0; k < 3; ++k) g->mu[m][k] = (float)((double)mu[m][k] + (k == 0 ? dx : k == 1 ? dy : dz));
          ld = chol_inv(t[4] * rn - dx * dx + 1e-4, t[5] * rn - dy * dx, t[6] * rn - dy * dy + 1e-4,
                        t[7] * rn - dz * dx, t[8] * rn - dz * dy, t[9] * rn - dz * dz + 1e-4, g->linv[m]);
          g->logdet[m] = ld;
        }
        g->lc[m] = (float)(log_f(pim) - 0.5 * ld - 1.5 * LOG_2PI);
      }
    }
  }
}

// ------------------------------------------------------------------ k-means start of the EM
// Sec. 7.3: the EM starts from a k-means partition of the label's prior-weighted
// colours.  Reading (the paper's CPU k-means is not specified): seeds by
// k-means++ taken in expectation -- c_1 = the weighted mean (the M = 1 fit's),
// c_m = the mean weighted by w D^2, D the distance to the nearest earlier seed;
// then Lloyd iterations (nearest center, lowest index on equal distances; a
// center whose cluster carries >= 1e-6 of the weight moves to its weighted
// mean); the mixture is the final partition's weight shares, means and
// covariances (+ 1e-4 I), a (nearly) empty cluster keeping its center and the
// label's covariance.  Sec. 2 / Sec. 6 likelihood update: with gmm_update a
// label that already holds a fitted mixture (the previous frame's) skips these
// passes and its EM continues from that mixture; valid[frame][label] records
// it (cleared when a stream starts a new video).  One pass per launch, grid
// (blocks, 2 frames) like the EM; partial sums through the EM's buffers.
enum { KM_SEED = 0, KM_LLOYD = 1, KM_MIX = 2 };
struct KMArgs {
  const uint8_t* rgb;
  const float* prior;
  int N;
  GmmDev* gmm;  // [frame][label]: centers in mu during the passes, then the mixture
  const GaussDev* gauss;
  float* part;
  int part_stride;
  unsigned* counter;
  int* valid;  // [frame][label] (nullable: the stateless stage entry point)
  int update;
  int mseed;   // KM_SEED: seeds already placed (the pass places seed mseed)
  const SegIO* io;
  const uint8_t* on;
};

template <int M, int MODE>
__global__ void __launch_bounds__(256) k_km_pass(KMArgs a) {
  constexpr int NV = MODE == KM_SEED ? 4 : MODE == KM_LLOYD ? 4 * M : 10 * M;
  seg_pdl_enter();
  const int lab = blockIdx.y & 1, fb = blockIdx.y >> 1;
  if (SEG_SLOT_OFF(a.on, fb)) return;
  const GaussDev* gd = a.gauss + fb;
  if (gd->degenerate & (1 << lab)) return;  // no weight: no mixture to start
  if (a.update && a.valid && a.valid[2 * fb + lab]) return;  // EM continues from the previous frame's mixture
  const uint8_t* rgb = (a.rgb ? a.rgb : a.io->rgb) + (size_t)fb * 3 * a.N;
  const float* prior = (a.prior ? a.prior : a.io->prior) + (size_t)fb * a.N;
  GmmDev* g = a.gmm + 2 * fb + lab;
  float ctr[M][3];
  const int nc = MODE == KM_SEED ? a.mseed : M;
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < 3; ++k) ctr[m][k] = (m == 0 && MODE == KM_SEED) ? gd->muf[lab][k] : g->mu[m][k];
  float s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += gridDim.x * blockDim.x) {
    const float p = prior[i];
    const float w = lab ? p : 1.f - p;
    const float c[3] = {rgb[3 * (size_t)i] / 255.f, rgb[3 * (size_t)i + 1] / 255.f, rgb[3 * (size_t)i + 2] / 255.f};
    float bd = 3.0e38f;
    int best = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      if (m >= nc) break;
      const float d0 = c[0] - ctr[m][0], d1 = c[1] - ctr[m][1], d2 = c[2] - ctr[m][2];
      const float d = d0 * d0 + d1 * d1 + d2 * d2;
      if (d < bd) {
        bd = d;
        best = m;
      }
    }
    if (MODE == KM_SEED) {
      const float wd = w * bd;
      s[0] += wd;
      s[1] += wd * c[0];
      s[2] += wd * c[1];
      s[3] += wd * c[2];
    } else if (MODE == KM_LLOYD) {
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (m == best) {
          s[4 * m] += w;
          s[4 * m + 1] += w * c[0];
          s[4 * m + 2] += w * c[1];
          s[4 * m + 3] += w * c[2];
        }
    } else {
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (m == best) {  // moments about the center (no large cancellation)
          const float d0 = c[0] - ctr[m][0], d1 = c[1] - ctr[m][1], d2 = c[2] - ctr[m][2];
          float* t = s + 10 * m;
          t[0] += w;
          t[1] += w * d0;
          t[2] += w * d1;
          t[3] += w * d2;
          t[4] += w * d0 * d0;
          t[5] += w * d1 * d0;
          t[6] += w * d1 * d1;
          t[7] += w * d2 * d0;
          t[8] += w * d2 * d1;
          t[9] += w * d2 * d2;
        }
    }
  }
  float* part = a.part + (size_t)(2 * fb + lab) * a.part_stride;
  if (block_partial_last<NV>(s, part, a.counter + 2 * fb + lab, blockIdx.x, gridDim.x)) {
    __shared__ double tot[NV];
    reduce_parts<NV>(part, gridDim.x, tot);
    if (threadIdx.x == 0) {
      if (MODE == KM_SEED) {
        if (a.mseed == 1)
          for (int k = 0; k < 3; ++k) g->mu[0][k] = gd->muf[lab][k];
        const bool ok = tot[0] > 0.0;
        const double r = ok ? nr_rcp(tot[0]) : 0.0;
        for (int k = 0; k < 3; ++k) g->mu[a.mseed][k] = ok ? (float)(tot[1 + k] * r) : gd->muf[lab][k];
      } else if (MODE == KM_LLOYD) {
        double sw = 0.0;
        for (int m = 0; m < M; ++m) sw += tot[4 * m];
        for (int m = 0; m < M; ++m)
          if (tot[4 * m] >= 1e-6 * sw) {
            const double r = nr_rcp(tot[4 * m]);
            for (int k = 0; k < 3; ++k) g->mu[m][k] = (float)(tot[4 * m + 1 + k] * r);
          }
      } else {
        double sw = 0.0;
        for (int m = 0; m < M; ++m) sw += tot[10 * m];
        const double rsw = nr_rcp(sw);
        for (int m = 0; m < M; ++m) {
          const double* t = tot + 10 * m;
          const double pim = t[0] * rsw;
          double ld;
          if (t[0] >= 1e-6 * sw) {
            const double rn = nr_rcp(t[0]);
            const double dx = t[1] * rn, dy = t[2] * rn, dz = t[3] * rn;
            g->mu[m][0] = (float)((double)ctr[m][0] + dx);
            g->mu[m][1] = (float)((double)ctr[m][1] + dy);
            g->mu[m][2] = (float)((double)ctr[m][2] + dz);
            ld = chol_inv(t[4] * rn - dx * dx + 1e-4, t[5] * rn - dy * dx, t[6] * rn - dy * dy + 1e-4,
                          t[7] * rn - dz * dx, t[8] * rn - dz * dy, t[9] * rn - dz * dz + 1e-4, g->linv[m]);
          } else {  // (nearly) empty: its center and the label's covariance
            for (int k = 0; k < 6; ++k) g->linv[m][k] = gd->linv[lab][k];
            ld = 2.0 * ((double)gd->lconst[lab] - 1.5 * LOG_2PI);
          }
          g->logdet[m] = ld;
          g->lc[m] = (float)(log_f(pim) - 0.5 * ld - 1.5 * LOG_2PI);
        }
        if (a.valid) a.valid[2 * fb + lab] = 1;
      }
    }
  }
}

struct TermsArgs {
  const uint8_t* rgb;
  const float* prior;
  const GaussDev* gauss;
  const int* lut;
  int H, W, nk, B;
  float eps, lambda_u, K;
  int32_t* cs;
  int32_t* ct;
  int32_t* ncap;
  const SegIO* io;  // rgb / prior == nullptr: take them from here
  const GmmDev* gmm;  // M > 1: [frame][label] colour mixtures
  int M;
  // the min cut's initial residual graph, formed here (seg_push_frame; nullptr:
  // off): residual planes e, rt and r[2 nk] over the stacked grid (plane stride
  // N B); flow / warm: the warm start's previous n-link flows and per-frame flag
  int* mf_e;
  int* mf_rt;
  int* mf_r;
  const int* flow;
  const unsigned char* warm;
  const uint8_t* on;  // [B] slots holding a stream (nullptr: all); an empty slot is not written
};

__device__ __forceinline__ int32_t quant_cap(float K, float x) {
  float v = floorf(K * x + 0.5f);
  v = fminf(v, 16777216.f);
  return (int32_t)fmaxf(v, 0.f);
}

// What the terms of one pixel read: its colour, its prior and r + g + b of its
// forward neighbours (-1 outside the frame).
struct TermsIn {
  int r8, g8, b8;
  float pr;
  int nsum[4];
  int bsum[4];  // (fused initialisation) r + g + b of the backward neighbours W, N, NW, NE, -1 outside
  int fl[8];    // (fused warm start) the flows of the eight links, forward ones first
};

__device__ __forceinline__ void terms_load(const TermsArgs& a, int x, int y, TermsIn& t) {
  const size_t g = (size_t)y * a.W + x;
  const uint8_t* p = a.rgb + 3 * g;
  t.r8 = p[0];
  t.g8 = p[1];
  t.b8 = p[2];
  t.pr = __ldcg(a.prior + g);  // (L2: in the fused kernel other CTAs wrote it)
  // neighbour k: (+1, 0), (0, +1), (+1, +1), (-1, +1); k >= 2 diagonal
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    t.nsum[k] = -1;
    if (k >= a.nk) continue;
    const int xx = x + (k == 1 ? 0 : k == 3 ? -1 : 1), yy = y + (k == 0 ? 0 : 1);
    if (xx >= 0 && xx < a.W && yy < a.H) {
      const uint8_t* q = a.rgb + 3 * ((size_t)yy * a.W + xx);
      t.nsum[k] = q[0] + q[1] + q[2];
    }
  }
  if (a.mf_r) {
    // backward neighbour k: W (-1, 0), N (0, -1), NW (-1, -1), NE (+1, -1)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      t.bsum[k] = -1;
      if (k >= a.nk) continue;
      const int xx = x + (k == 1 ? 0 : k == 3 ? 1 : -1), yy = y - (k == 0 ? 0 : 1);
      if (xx >= 0 && xx < a.W && yy >= 0) {
        const uint8_t* q = a.rgb + 3 * ((size_t)yy * a.W + xx);
        t.bsum[k] = q[0] + q[1] + q[2];
      }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) t.fl[d] = 0;
    if (a.flow) {
      // forward link k of this node, and the backward one: forward link k of the
      // neighbour it comes from (its plane k)
      const size_t NB = (size_t)a.H * a.W * a.B;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= a.nk) continue;
        if (t.nsum[k] >= 0) t.fl[k] = a.flow[k * NB + g];
        const int xx = x + (k == 1 ? 0 : k == 3 ? 1 : -1), yy = y - (k == 0 ? 0 : 1);
        if (t.bsum[k] >= 0) t.fl[4 + k] = a.flow[k * NB + (size_t)yy * a.W + xx];
      }
    }
  }
}

// t-links and n-links of pixel (x, y) of one frame from what terms_load read:
// rgb, prior, cs, ct and ncap point at the frame, NB is the plane stride of the
// stacked n-link planes, lut the n-link table (shared memory), gs / gmm the
// frame's colour model.
__device__ __forceinline__ void terms_store(const TermsArgs& a, const GaussDev& gs, const GmmDev* gmm, size_t NB,
                                            const int* lut, int x, int y, const TermsIn& t) {
  const size_t g = (size_t)y * a.W + x;
  const float C[3] = {t.r8 / 255.f, t.g8 / 255.f, t.b8 / 255.f};
  const float pr = t.pr;
  float D[2];
#pragma unroll
  for (int lab = 0; lab < 2; ++lab) {
    float psi;
    if (a.M > 1 && !(gs.degenerate & (1 << lab))) {  // -log sum_m pi_m N_m(C)
      const GmmDev& q = gmm[lab];
      float lp[SEG_MAX_GMM], mx = -3.0e38f;
#pragma unroll
      for (int m = 0; m < SEG_MAX_GMM; ++m) {
        if (m >= a.M) break;
        const float* li = q.linv[m];
        float d0 = C[0] - q.mu[m][0], d1 = C[1] - q.mu[m][1], d2 = C[2] - q.mu[m][2];
        float y0 = li[0] * d0;
        float y1 = li[1] * d0 + li[2] * d1;
        float y2 = li[3] * d0 + li[4] * d1 + li[5] * d2;
        lp[m] = q.lc[m] - 0.5f * (y0 * y0 + y1 * y1 + y2 * y2);
        mx = fmaxf(mx, lp[m]);
      }
      float z = 0.f;
#pragma unroll
      for (int m = 0; m < SEG_MAX_GMM; ++m) {
        if (m >= a.M) break;
        z += expf(lp[m] - mx);
      }
      psi = -(mx + logf(z));
    } else {
      const float* li = gs.linv[lab];
      float d0 = C[0] - gs.muf[lab][0], d1 = C[1] - gs.muf[lab][1], d2 = C[2] - gs.muf[lab][2];
      float y0 = li[0] * d0;
      float y1 = li[1] * d0 + li[2] * d1;
      float y2 = li[3] * d0 + li[4] * d1 + li[5] * d2;
      psi = 0.5f * (y0 * y0 + y1 * y1 + y2 * y2) + gs.lconst[lab];
    }
    float pl = lab ? pr : 1.f - pr;
    float xi = -logf(fminf(fmaxf(pl, a.eps), 1.f - a.eps));
    D[lab] = a.lambda_u * psi + xi;
  }
  const float m = fminf(D[0], D[1]);
  const int32_t csq = quant_cap(a.K, D[0] - m), ctq = quant_cap(a.K, D[1] - m);
  a.cs[g] = csq;  // c(s, v) = D(0): paid when v is background
  a.ct[g] = ctq;  // c(v, t) = D(1): paid when v is object
  const int s0 = t.r8 + t.g8 + t.b8;
  int cf[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= a.nk) break;
    cf[k] = t.nsum[k] < 0 ? 0 : lut[2 * abs(s0 - t.nsum[k]) + (k >= 2)];
    a.ncap[k * NB + g] = cf[k];
  }
  if (a.mf_r) {
    // the min cut's initial state (its init pass, done here): residuals of the
    // eight directed links from the capacities (a backward link's capacity is the
    // neighbour's forward one, the same table entry) and, warm, the previous
    // flows clamped to them; source arcs saturated and s->v->t flow cancelled.
    // Directions E W S N SE NW SW NE: forward link k is direction 2k, and
    // backward link k (from W, N, NW, NE) direction 2k + 1.
    const bool warm = a.flow != nullptr && a.warm[0];
    auto clampf = [](int f, int c) { return f > c ? c : (f < -c ? -c : f); };
    int net_out = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= a.nk) break;
      const int cb = t.bsum[k] < 0 ? 0 : lut[2 * abs(s0 - t.bsum[k]) + (k >= 2)];
      const int ff = warm ? clampf(t.fl[k], cf[k]) : 0, fb = warm ? clampf(t.fl[4 + k], cb) : 0;
      a.mf_r[(2 * k) * NB + g] = cf[k] - ff;
      a.mf_r[(2 * k + 1) * NB + g] = cb + fb;
      net_out += ff - fb;
    }
    int e0 = csq - net_out, cte = ctq;
    if (e0 < 0) {  // deficit
      cte = ctq - e0;
      e0 = 0;
    }
    const int m = min(e0, cte);
    a.mf_e[g] = e0 - m;
    a.mf_rt[g] = cte - m;
  }
}

// Frame fb's pointers (and, when captured, the frame's I/O).  The frame's n-link
// planes are rows fb*H .. fb*H+H-1 of the stacked (B*H) x W grid the min cut
// sees; links leaving the frame stay 0.
__device__ __forceinline__ void terms_frame(TermsArgs& a, int fb) {
  if (!a.rgb) a.rgb = a.io->rgb;
  if (!a.prior) a.prior = a.io->prior;
  const size_t N = (size_t)a.H * a.W;
  a.rgb += fb * 3 * N;
  a.prior += fb * N;
  a.gauss += fb;
  a.cs += fb * N;
  a.ct += fb * N;
  a.ncap += fb * N;
  a.gmm += 2 * fb;
  if (a.mf_r) {
    a.mf_e += fb * N;
    a.mf_rt += fb * N;
    a.mf_r += fb * N;
    if (a.flow) {
      a.flow += fb * N;
      a.warm += fb;
    }
  }
}

__global__ void __launch_bounds__(256) k_terms(TermsArgs a) {
  // (Loading the inputs the preceding kernel does not write before waiting for
  // it took 3 us off this kernel alone but slowed pipelined frames: its early
  // CTAs' loads competed with the next frame's saliency.)
  seg_pdl_enter();
  __shared__ int sLut[766 * 2];
  for (int i = threadIdx.x; i < 766 * 2; i += blockDim.x) sLut[i] = a.lut[i];
  __syncthreads();
  terms_frame(a, blockIdx.z);
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= a.W || y >= a.H) return;
  if (SEG_SLOT_OFF(a.on, blockIdx.z)) return;  // no stream in the slot: the cut skips its rows
  TermsIn t;
  terms_load(a, x, y, t);
  terms_store(a, *a.gauss, a.gmm, (size_t)a.H * a.W * a.B, sLut, x, y, t);
}

// ------------------------------------------------------------------ host side
// n-link capacity table, FP64 on the host so the integer capacities are exact:
// lut[2*ds + diag] = min(2^24, floor(K (lambda_p + lambda_s exp(-(ds/765)^2 /
// (2 sigma_I^2)) / |x-y|) + 1/2)), |x-y| = 1 or sqrt 2 (Eq. 2 with the contrast
// term of Sec. 4).
void pt_fill_lut(const seg_params& p, int* lut) {
  for (int ds = 0; ds <= 765; ++ds)
    for (int diag = 0; diag < 2; ++diag) {
      double dI = ds / 765.0;
      double dist = diag ? sqrt(2.0) : 1.0;
      double c = p.lambda_p + p.lambda_s * exp(-dI * dI / (2.0 * p.sigma_I * p.sigma_I)) / dist;
      double v = floor(p.cap_scale * c + 0.5);
      if (v > 16777216.0) v = 16777216.0;
      if (v < 0) v = 0;
      lut[2 * ds + diag] = (int)v;
    }
}

int pt_mom_blocks(int H, int W) {
  int n = H * W;
  int b = (n + 256 * MOM_PX - 1) / (256 * MOM_PX);
  return b < 1 ? 1 : (b > 2048 ? 2048 : b);
}

__global__ void k_map_max(const float* __restrict__ v, int n, unsigned* out) {
  seg_pdl_enter();
  float m = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmaxf(m, v[i]);
  m = seg_warp_max_f(m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// max of a non-negative saliency map (float bits order like the values)
int pt_launch_salmax(seg_ctx* c, const float* sal) {
  SEG_CUDA_TRY(cudaMemsetAsync(c->sal.salmax, 0, sizeof(unsigned), c->stream));
  int nb = (c->N + 1023) / 1024;
  nb = nb > 1184 ? 1184 : nb;
  SEG_CUDA_TRY(seg_launch(k_map_max, nb, 256, 0, c->stream, sal, c->N, c->sal.salmax));
  SEG_CUDA_TRY(cudaGetLastError());
  return SEG_OK;
}

static void prior_args(seg_ctx* c, const float* sal, const uint8_t* prev_mask, int use_kalman, double wf_host,
                       float* prior, const uint8_t* rgb_moments, bool from_S, PriorArgs& a) {
  const seg_params& p = c->p;
  memset(&a, 0, sizeof(a));
  a.sal = const_cast<float*>(sal);
  a.from_S = from_S ? 1 : 0;
  a.S = c->sal.S;
  a.hS = c->sal.hl[c->sal.sS];
  a.wS = c->sal.wl[c->sal.sS];
  a.frow = c->sal.rs + c->sal.rs_frow;
  a.fcol = c->sal.rs + c->sal.rs_fcol;
  a.salmax = c->sal.salmax;
  a.prev = prev_mask;
  a.kal = use_kalman ? c->kal : nullptr;
  a.wf_host = wf_host;
  a.a = p.sigma1 * p.sigma1;
  a.b = p.sigma2 * p.sigma2;
  a.H = c->H;
  a.W = c->W;
  a.border = p.border_px;
  a.eps = p.eps;
  a.fR = p.f_radius;
  double g[2 * PR_MAXR + 1], sg = 0;
  for (int u = -p.f_radius; u <= p.f_radius; ++u) {
    g[u + p.f_radius] = exp(-(double)(u * u) / (2.0 * p.f_sigma * p.f_sigma));
    sg += g[u + p.f_radius];
  }
  for (int u = 0; u <= 2 * p.f_radius; ++u) a.ftap[u] = (float)(g[u] / sg);
  a.prior = prior;
  a.rgb = rgb_moments;
  a.part = (float*)c->mom_part;
  a.counter = c->mom_counter;
  a.gauss = c->gauss;
  a.part_stride = pt_part_doubles(c->H, c->W);
  a.kal_adv = (use_kalman && (rgb_moments || c->io_mode)) ? c->kal : nullptr;
  a.io = c->io_mode ? c->io : nullptr;
  a.on = c->sal.on;
}

int pt_launch_prior(seg_ctx* c, const float* sal, const uint8_t* prev_mask, int use_kalman,
                    double wf_host, float* prior, const uint8_t* rgb_moments, bool from_S) {
  PriorArgs a;
  prior_args(c, sal, prev_mask, use_kalman, wf_host, prior, rgb_moments, from_S, a);
  dim3 grid((c->W + PR_TX - 1) / PR_TX, (c->H + PR_TY - 1) / PR_TY, c->B);
  SEG_CUDA_TRY(seg_launch(k_prior, grid, 256, 0, c->stream, a));
  SEG_CUDA_TRY(cudaGetLastError());
  return SEG_OK;
}

static void terms_args(seg_ctx* c, const uint8_t* rgb, const float* prior, int32_t* cs, int32_t* ct, int32_t* ncap,
                       TermsArgs& ta, bool mf_init);

int pt_launch_moments_terms(seg_ctx* c, const uint8_t* rgb, const float* prior, int first_pass,
                            int32_t* cs, int32_t* ct, int32_t* ncap, bool mf_init) {
  const seg_params& p = c->p;
  cudaStream_t st = c->stream;
  int N = c->N;
  MomFinArgs fa;
  fa.part = (float*)c->mom_part;
  fa.part_stride = pt_part_doubles(c->H, c->W);
  fa.counter = c->mom_counter;
  fa.gauss = c->gauss;
  fa.kal = nullptr;
  fa.a = p.sigma1 * p.sigma1;
  fa.b = p.sigma2 * p.sigma2;
  fa.io = c->io_mode ? c->io : nullptr;
  fa.on = c->sal.on;
  const int M = p.gmm_components;
  if (first_pass) SEG_CUDA_TRY(seg_launch(k_mom1, dim3(c->mom_blocks, c->B), 256, 0, st, rgb, prior, N, fa));
  SEG_CUDA_TRY(seg_launch(k_mom2, dim3(c->mom_blocks, c->B), 256, 0, st, rgb, prior, N, fa));
  if (M > 1) {  // Sec. 4 / Sec. 7.3: EM of the M-component colour mixtures
    EMArgs ea;
    ea.rgb = rgb;
    ea.prior = prior;
    ea.N = N;
    ea.M = M;
    ea.gmm = c->gmm;
    ea.gauss = c->gauss;
    ea.part = (float*)c->em_part;
    ea.part_stride = pt_em_part_doubles(c->H, c->W);
    ea.counter = c->em_counter;
    ea.io = c->io_mode ? c->io : nullptr;
    ea.on = c->sal.on;
    KMArgs ka;
    ka.rgb = rgb;
    ka.prior = prior;
    ka.N = N;
    ka.gmm = c->gmm;
    ka.gauss = c->gauss;
    ka.part = (float*)c->em_part;
    ka.part_stride = pt_em_part_doubles(c->H, c->W);
    ka.counter = c->em_counter;
    // the stage entry point (first_pass) is stateless: always the k-means start, and the
    // stream's mixtures are not marked as the next frame's start
    ka.valid = first_pass ? nullptr : c->gmm_valid;
    ka.update = first_pass ? 0 : p.gmm_update;
    ka.io = ea.io;
    ka.on = c->sal.on;
    const dim3 gk(c->mom_blocks, 2 * c->B);
    for (int m = 1; m < M; ++m) {
      ka.mseed = m;
      if (M == 2)
        SEG_CUDA_TRY(seg_launch(k_km_pass<2, KM_SEED>, gk, 256, 0, st, ka));
      else
        SEG_CUDA_TRY(seg_launch(k_km_pass<3, KM_SEED>, gk, 256, 0, st, ka));
    }
    for (int it = 0; it < p.kmeans_iters; ++it) {
      if (M == 2)
        SEG_CUDA_TRY(seg_launch(k_km_pass<2, KM_LLOYD>, gk, 256, 0, st, ka));
      else
        SEG_CUDA_TRY(seg_launch(k_km_pass<3, KM_LLOYD>, gk, 256, 0, st, ka));
    }
    if (M == 2)
      SEG_CUDA_TRY(seg_launch(k_km_pass<2, KM_MIX>, gk, 256, 0, st, ka));
    else
      SEG_CUDA_TRY(seg_launch(k_km_pass<3, KM_MIX>, gk, 256, 0, st, ka));
    for (int it = 0; it < p.em_iters; ++it) {
      if (M == 2)
        SEG_CUDA_TRY(seg_launch(k_em_step<2>, dim3(c->mom_blocks, 2 * c->B), 256, 0, st, ea));
      else
        SEG_CUDA_TRY(seg_launch(k_em_step<3>, dim3(c->mom_blocks, 2 * c->B), 256, 0, st, ea));
    }
  }
  TermsArgs ta;
  terms_args(c, rgb, prior, cs, ct, ncap, ta, mf_init);
  dim3 grid((c->W + 31) / 32, (c->H + 7) / 8, c->B);
  SEG_CUDA_TRY(seg_launch(k_terms, grid, 256, 0, st, ta));
  SEG_CUDA_TRY(cudaGetLastError());
  return SEG_OK;
}

static void terms_args(seg_ctx* c, const uint8_t* rgb, const float* prior, int32_t* cs, int32_t* ct, int32_t* ncap,
                       TermsArgs& ta, bool mf_init) {
  const seg_params& p = c->p;
  ta.mf_e = mf_init ? c->mf.e : nullptr;
  ta.mf_rt = mf_init ? c->mf.rt : nullptr;
  ta.mf_r = mf_init ? c->mf.r : nullptr;
  ta.flow = mf_init && p.warm_start ? c->flow : nullptr;
  ta.warm = mf_init && p.warm_start ? c->warm : nullptr;
  ta.rgb = rgb;
  ta.prior = prior;
  ta.gauss = c->gauss;
  ta.lut = c->lut;
  ta.H = c->H;
  ta.W = c->W;
  ta.nk = p.neighbourhood / 2;
  ta.B = c->B;
  ta.eps = p.eps;
  ta.lambda_u = (float)p.lambda_u;
  ta.K = (float)p.cap_scale;
  ta.cs = cs;
  ta.ct = ct;
  ta.ncap = ncap;
  ta.io = c->io_mode ? c->io : nullptr;
  ta.gmm = c->gmm;
  ta.M = p.gmm_components;
  ta.on = c->sal.on;
}

// A frame's prior, first moments (fused into k_prior), second moments and
// terms, the terms kernel also forming the min cut's initial residual graph
// (the cut then runs with init_done): the launches of one frame's back half
// before the cut.
int pt_launch_back(seg_ctx* c, const float* sal, float* prior, const uint8_t* rgb) {
  int rc = pt_launch_prior(c, sal, c->prev_mask, 1, 0.0, prior, rgb, true);
  return rc ? rc : pt_launch_moments_terms(c, rgb, prior, 0, c->cs, c->ct, c->ncap, true);
}

int pt_em_part_doubles(int H, int W) { return EM_NV * pt_mom_blocks(H, W); }

int pt_part_doubles(int H, int W) {
  int prior_blocks = ((W + PR_TX - 1) / PR_TX) * ((H + PR_TY - 1) / PR_TY);
  int mb = pt_mom_blocks(H, W);
  return 12 * (prior_blocks > mb ? prior_blocks : mb);
}
