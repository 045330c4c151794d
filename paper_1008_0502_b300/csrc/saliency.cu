// saliency.cu -- the saliency map of Sec. 3 / Sec. 7.2 on sm_103a.
//
// Pipeline per frame (all kernels stream-ordered, no host round trip):
//   k_rgb_max       frame max of r+g+b (the hue-normalisation threshold)
//   k_feat_reduce1  RGB8 -> I, RG, BY features fused with the first REDUCE:
//                   level 0 never leaves shared memory
//   k_reduce3       Gaussian pyramid, levels 2..L-1 (separable [1 4 6 4 1]/16,
//                   clamp-to-edge, keep even samples)
//   k_gabor         |complex Gabor| at levels c_min..c_max+d_max, 4 orientations,
//                   evaluated as a rank-2 separable filter from shared memory
//   k_cs_stats      center-surround maps |X(c) -/+ up X(s)| computed on the fly;
//                   per-map min, max and T x T tile maxima for N(.)
//   k_cs_accum      across-scale sum: B_c = sum_s N(CS(c,s)) + REDUCE(B_{c-1}),
//                   each map's N(.) taken as an affine map a*v + b from its
//                   statistics in the CTA's prologue
//                   (REDUCE is linear, so reducing the sum equals summing the
//                   reduced maps)
//   k_consp         one CTA per frame at sigma_S: orientation conspicuity,
//                   N(C_k), S = sum_k w_k N(C_k)
//   k_upsample      S -> frame-size saliency (bilinear); seg_push_frame skips it
//                   and lets the prior kernel evaluate the saliency on the fly
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cooperative_groups.h>
#include <type_traits>

#include "seg_internal.cuh"

#define RED_TX 32
#define RED_TY 16
#define RED_IN_X (2 * RED_TX + 3)
#define RED_IN_Y (2 * RED_TY + 3)

__constant__ float c_binom[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};

// ------------------------------------------------------------------ k_rgb_max
// TIn = uint8_t (RGB8) or float (values in [0, 255], the backward form); for
// float frames smax holds the maximum's float bits (non-negative floats order
// like their bit patterns).
template <typename TIn>
__global__ void k_rgb_max(const TIn* __restrict__ rgb, int n, int* smax, unsigned* mm,
                          int nmaps, const SegIO* io, const uint8_t* on) {
  seg_pdl_enter();
  if (SEG_SLOT_OFF(on, blockIdx.y)) return;
  if constexpr (std::is_same<TIn, uint8_t>::value) {
    if (!rgb) rgb = io->rgb;
  }
  const int fb = blockIdx.y;  // frame of the batch
  rgb += (size_t)fb * 3 * n;
  smax += fb;
  mm += (size_t)fb * 2 * nmaps;
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < nmaps) {  // N(.) statistics start empty: min = +max float, max = 0
    mm[2 * tid] = 0x7f7fffffu;
    mm[2 * tid + 1] = 0u;
  }
  int m = 0;
  bool done = false;
  if constexpr (std::is_same<TIn, uint8_t>::value) {
    if ((n & 15) == 0 && ((uintptr_t)rgb & 15) == 0) {  // 16 pixels = three 16-byte loads
      const uint4* q = reinterpret_cast<const uint4*>(rgb);
      for (int g = tid; g < (n >> 4); g += gridDim.x * blockDim.x) {
        const uint4 v0 = q[3 * (size_t)g], v1 = q[3 * (size_t)g + 1], v2 = q[3 * (size_t)g + 2];
        const unsigned w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          int s = 0;
#pragma unroll
          for (int c = 0; c < 3; ++c) s += (w[(3 * k + c) >> 2] >> (8 * ((3 * k + c) & 3))) & 255u;
          m = max(m, s);
        }
      }
      done = true;
    }
  }
  for (int i = tid; !done && i < n; i += gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TIn, uint8_t>::value) {
      int s = rgb[3 * (size_t)i] + rgb[3 * (size_t)i + 1] + rgb[3 * (size_t)i + 2];
      m = max(m, s);
    } else {
      float s = rgb[3 * (size_t)i] + rgb[3 * (size_t)i + 1] + rgb[3 * (size_t)i + 2];
      m = max(m, s > 0.f ? __float_as_int(s) : 0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    if (m > 0) atomicMax(smax, m);
  }
}

// ------------------------------------------------------------------ features + REDUCE
// Sec. 7.2 step 1 (features) and step 2 (pyramid).  I = (r+g+b)/765; where
// 10*(r+g+b) > max(r+g+b) the normalised colour rn = 3r/(r+g+b) etc. (else
// 0); R, G, B, Y broadly tuned channels clamped at 0; RG = R-G, BY = B-Y.
template <typename TIn>
__global__ void __launch_bounds__(256) k_feat_reduce1(const TIn* __restrict__ rgb, int H, int W,
                                                      const int* __restrict__ smax_p,
                                                      float* __restrict__ I1, float* __restrict__ RG1,
                                                      float* __restrict__ BY1, int h1, int w1,
                                                      const SegIO* io, const uint8_t* on) {
  constexpr bool U8 = std::is_same<TIn, uint8_t>::value;
  if constexpr (U8) {
    if (!rgb) rgb = io->rgb;
  }
  __shared__ float sF[3][RED_IN_Y][RED_IN_X];
  __shared__ float sH[3][RED_IN_Y][RED_TX];
  const int fb = blockIdx.z;  // frame of the batch
  if (SEG_SLOT_OFF(on, fb)) return;
  rgb += (size_t)fb * 3 * H * W;
  const size_t o1 = (size_t)fb * h1 * w1;
  I1 += o1;
  RG1 += o1;
  BY1 += o1;
  const int X0 = blockIdx.x * RED_TX, Y0 = blockIdx.y * RED_TY;
  const int gx0 = 2 * X0 - 2, gy0 = 2 * Y0 - 2;
  int smax = 0;  // (read once the preceding kernel, which forms it, is complete)
  // features of input pixel (ry, rx) of the tile into sF
  auto feat = [&](int ry, int rx, float r, float g, float b, float s, bool hue) {
    float rn = 0.f, gn = 0.f, bn = 0.f;
    if (hue) {
      float inv = 3.f / s;
      rn = r * inv;
      gn = g * inv;
      bn = b * inv;
    }
    float R = fmaxf(0.f, rn - (gn + bn) / 2.f);
    float G = fmaxf(0.f, gn - (rn + bn) / 2.f);
    float B = fmaxf(0.f, bn - (rn + gn) / 2.f);
    float Y = fmaxf(0.f, (rn + gn) / 2.f - fabsf(rn - gn) / 2.f - bn);
    sF[0][ry][rx] = s / 765.f;
    sF[1][ry][rx] = R - G;
    sF[2][ry][rx] = B - Y;
  };
  constexpr int NIN = RED_IN_Y * RED_IN_X, PER = (NIN + 255) / 256;
  // RGB8 tile away from the frame border, rows 4-byte aligned: the tile's rows
  // as 32-bit words (RED_IN_X pixels = 201 bytes from byte 3 gx0, read from the
  // aligned byte 3 gx0 - 2) staged in sH's space, a quarter of the byte loads
  constexpr int RWORDS = (3 * RED_IN_X + 2 + 3) / 4;
  static_assert(RED_IN_Y * RWORDS * 4 <= (int)sizeof(sH), "staged rows fit sH");
  bool staged = false;
  if constexpr (U8)
    staged = (W & 3) == 0 && ((uintptr_t)rgb & 3) == 0 && gx0 >= 1 && gy0 >= 0 &&
             4 * RWORDS + 3 * gx0 - 2 <= 3 * W && gy0 + RED_IN_Y <= H;
  if (staged) {
    unsigned* sw = reinterpret_cast<unsigned*>(&sH[0][0][0]);
    const unsigned* gw = reinterpret_cast<const unsigned*>(rgb);
    constexpr int NWD = RED_IN_Y * RWORDS, PW = (NWD + 255) / 256;  // (256 threads)
    unsigned wv[PW];
#pragma unroll
    for (int k = 0; k < PW; ++k) {  // every load in flight before the first store
      const int i = threadIdx.x + 256 * k;
      if (i < NWD) {
        const int ry = i / RWORDS, c = i - ry * RWORDS;
        wv[k] = gw[((size_t)(gy0 + ry) * 3 * W + 3 * gx0 - 2) / 4 + c];
      }
    }
#pragma unroll
    for (int k = 0; k < PW; ++k)
      if (threadIdx.x + 256 * k < NWD) sw[threadIdx.x + 256 * k] = wv[k];
    seg_pdl_enter();
    smax = smax_p[fb];
    __syncthreads();
    const unsigned char* sb = reinterpret_cast<const unsigned char*>(sw);
    for (int i = threadIdx.x; i < NIN; i += blockDim.x) {
      const int ry = i / RED_IN_X, rx = i - ry * RED_IN_X;
      const unsigned char* q = sb + ry * 4 * RWORDS + 2 + 3 * rx;
      const int ri = q[0], gi = q[1], bi = q[2], si = ri + gi + bi;
      feat(ry, rx, (float)ri, (float)gi, (float)bi, (float)si, 10 * si > smax);
    }
    __syncthreads();  // (sH is overwritten next)
  } else {
    // all of this thread's input pixels are loaded first (independent loads in
    // flight together), then turned into features
    constexpr int NW = U8 ? 1 : 3;  // registers per input pixel
    unsigned pk[PER][NW];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int i = threadIdx.x + k * 256;
      if (i < NIN) {
        int ry = i / RED_IN_X, rx = i - ry * RED_IN_X;
        int gy = seg_clampi(gy0 + ry, 0, H - 1), gx = seg_clampi(gx0 + rx, 0, W - 1);
        const TIn* p = rgb + 3 * ((size_t)gy * W + gx);
        if constexpr (U8) {
          pk[k][0] = (unsigned)p[0] | ((unsigned)p[1] << 8) | ((unsigned)p[2] << 16);
        } else {
#pragma unroll
          for (int j = 0; j < 3; ++j) pk[k][j] = __float_as_uint(p[j]);
        }
      }
    }
    seg_pdl_enter();
    smax = smax_p[fb];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int i = threadIdx.x + k * 256;
      if (i >= NIN) break;
      int ry = i / RED_IN_X, rx = i - ry * RED_IN_X;
      if constexpr (U8) {
        int ri = pk[k][0] & 255, gi = (pk[k][0] >> 8) & 255, bi = pk[k][0] >> 16;
        int si = ri + gi + bi;
        feat(ry, rx, (float)ri, (float)gi, (float)bi, (float)si, 10 * si > smax);
      } else {
        float r = __uint_as_float(pk[k][0]), g = __uint_as_float(pk[k][1]), b = __uint_as_float(pk[k][2]);
        float sum = r + g + b;
        feat(ry, rx, r, g, b, sum, 10.f * sum > __int_as_float(smax));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * RED_IN_Y * RED_TX; i += blockDim.x) {
    int ch = i / (RED_IN_Y * RED_TX);
    int rem = i - ch * RED_IN_Y * RED_TX;
    int ry = rem / RED_TX, x = rem - ry * RED_TX;
    const float* row = &sF[ch][ry][2 * x];
    sH[ch][ry][x] = c_binom[0] * row[0] + c_binom[1] * row[1] + c_binom[2] * row[2] +
                    c_binom[3] * row[3] + c_binom[4] * row[4];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * RED_TY * RED_TX; i += blockDim.x) {
    int ch = i / (RED_TY * RED_TX);
    int rem = i - ch * RED_TY * RED_TX;
    int y = rem / RED_TX, x = rem - y * RED_TX;
    int oy = Y0 + y, ox = X0 + x;
    if (oy >= h1 || ox >= w1) continue;
    float v = c_binom[0] * sH[ch][2 * y][x] + c_binom[1] * sH[ch][2 * y + 1][x] +
              c_binom[2] * sH[ch][2 * y + 2][x] + c_binom[3] * sH[ch][2 * y + 3][x] +
              c_binom[4] * sH[ch][2 * y + 4][x];
    float* out = ch == 0 ? I1 : (ch == 1 ? RG1 : BY1);
    out[(size_t)oy * w1 + ox] = v;
  }
}

// ------------------------------------------------------------------ features + REDUCE, 16-pixel runs
// The same two steps for frames whose width is a multiple of 16, shaped to
// spend few instructions per pixel.  A thread owns a run of 16 level-0 pixels
// of one row (three 16-byte loads of RGB8), computes their features in
// registers, takes the two pixels left and the one right of its run from the
// neighbouring threads of the row by shuffles (the tile's outer neighbours
// from a small shared table) and forms the horizontal REDUCE of its 8 level-1
// columns; the vertical REDUCE reads those rows back from shared memory.
// The features are Itti's broadly tuned channels written with integer
// numerators (rn = 3r/s etc., and (x + y)/2 - |x - y|/2 = min(x, y)):
//   R - G = (3 / 2s) (max(0, 2r - g - b) - max(0, 2g - r - b))
//   B - Y = (3 / 2s) (max(0, 2b - r - g) - 2 max(0, min(r, g) - b))
// for RGB8 the numerators are exact integers (byte dot products), then one
// reciprocal per pixel; the REDUCE uses the binomial weights 1 4 6 4 1 as
// integers and scales by 1/256 at the end (exact).  Float frames holding
// integer values give the RGB8 result bit for bit, and the tile height does
// not change any value.
#define FV_TX 64    // level-1 columns per CTA (128 level-0 pixels per row)
#define FV_LANES 8  // threads per level-0 row

__device__ __forceinline__ int fv_dp4a(unsigned a, unsigned b) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(0));
  return d;
}
__device__ __forceinline__ float fv_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
struct FV3 {
  float v[3];  // I, R - G, B - Y
};
// s2 = 2 s, n3 = 3 x the numerators: R - G = 3 nrg / 2s = n3rg / s2, likewise B - Y
__device__ __forceinline__ FV3 fv_finish(float s2f, float n3rg, float n3by, bool hue) {
  const float k = hue ? fv_rcp(s2f) : 0.f;
  return {{s2f * (1.f / 1530.f), n3rg * k, n3by * k}};
}
// RGB8 pixel whose r, g, b are the bytes SH/8, SH/8 + 1, SH/8 + 2 of P;
// hue <=> 10 s > smax <=> s > floor(smax / 10) <=> 2s > thr2 = 2 floor(smax / 10)
template <int SH>
__device__ __forceinline__ FV3 fv_px_u8(unsigned P, int thr2) {
  // byte weights (r, g, b, -) packed little-endian
  const int s2 = fv_dp4a(P, 0x00020202u << SH);  // 2 (r + g + b)
  const int t1 = fv_dp4a(P, 0x00FDFD06u << SH);  // 3 (2r - g - b)
  const int t2 = fv_dp4a(P, 0x00FD06FDu << SH);  // 3 (2g - r - b)
  const int t3 = fv_dp4a(P, 0x0006FDFDu << SH);  // 3 (2b - r - g)
  const int u1 = fv_dp4a(P, 0x00FD0003u << SH);  // 3 (r - b)
  const int u2 = fv_dp4a(P, 0x00FD0300u << SH);  // 3 (g - b)
  const int n3rg = max(t1, 0) - max(t2, 0);
  const int n3by = max(t3, 0) - 2 * __vimin_s32_relu(u1, u2);
  return fv_finish((float)s2, (float)n3rg, (float)n3by, s2 > thr2);
}
__device__ __forceinline__ FV3 fv_px_f32(float r, float g, float b, float smaxf) {
  const float sf = r + g + b;
  const float n3rg = fmaxf(0.f, 3.f * (2.f * r - g - b)) - fmaxf(0.f, 3.f * (2.f * g - r - b));
  const float n3by = fmaxf(0.f, 3.f * (2.f * b - r - g)) - 2.f * fmaxf(0.f, 3.f * (fminf(r, g) - b));
  return fv_finish(2.f * sf, n3rg, n3by, 10.f * sf > smaxf);
}
// one REDUCE tap set, x16: f(-2) + 4 f(-1) + 6 f(0) + 4 f(1) + f(2)
__device__ __forceinline__ float fv_h(float a, float b, float c, float d, float e) {
  return fmaf(6.f, c, fmaf(4.f, b + d, a + e));
}

template <int TY>
__host__ __device__ constexpr int fv_threads() {
  return FV_LANES * (2 * TY + 4);
}

// The run's horizontal REDUCE into sH (pixels -2, -1 and 16 of the run from
// the neighbouring runs of the row by shuffles, or from the span's neighbours
// in sHalo, which the caller has made visible), a CTA barrier, then the
// vertical REDUCE of the tile, 4 output rows x 4 columns per task.  I1, RG1,
// BY1 point at the frame's level-1 maps.
template <int TY>
__device__ __forceinline__ void fv_reduce_tile(const float (&F)[3][16], float (*sH)[2 * TY + 3][FV_TX],
                                               const float (*sHalo)[3][3], int slot, int j, int nvalid, int X0,
                                               int Y0, int h1, int w1, float* __restrict__ I1,
                                               float* __restrict__ RG1, float* __restrict__ BY1) {
  constexpr int ROWS = 2 * TY + 3;
  const int hs = min(slot, ROWS - 1);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float m2 = __shfl_up_sync(0xffffffffu, F[ch][14], 1, FV_LANES);
    float m1 = __shfl_up_sync(0xffffffffu, F[ch][15], 1, FV_LANES);
    float p16 = __shfl_down_sync(0xffffffffu, F[ch][0], 1, FV_LANES);
    if (j == 0) {
      m2 = sHalo[hs][0][ch];
      m1 = sHalo[hs][1][ch];
    }
    if (j == nvalid - 1) p16 = sHalo[hs][2][ch];
    if (slot < ROWS) {
      float hv[8];
      hv[0] = fv_h(m2, m1, F[ch][0], F[ch][1], F[ch][2]);
#pragma unroll
      for (int m = 1; m < 7; ++m) hv[m] = fv_h(F[ch][2 * m - 2], F[ch][2 * m - 1], F[ch][2 * m], F[ch][2 * m + 1], F[ch][2 * m + 2]);
      hv[7] = fv_h(F[ch][12], F[ch][13], F[ch][14], F[ch][15], p16);
      float4* d = reinterpret_cast<float4*>(&sH[ch][slot][8 * j]);
      d[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
      d[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
    }
  }
  __syncthreads();
  constexpr int NQ = FV_TX / 4, NG = TY / 4;
  for (int t = threadIdx.x; t < 3 * NQ * NG; t += blockDim.x) {
    const int q = t % NQ, rg = (t / NQ) % NG, ch = t / (NQ * NG);
    const int ox = X0 + 4 * q;
    if (ox >= w1) continue;
    float4 r[11];  // horizontal REDUCE rows 8 rg .. 8 rg + 10
#pragma unroll
    for (int i = 0; i < 11; ++i) r[i] = *reinterpret_cast<const float4*>(&sH[ch][8 * rg + i][4 * q]);
    float* out = ch == 0 ? I1 : ch == 1 ? RG1 : BY1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int oy = Y0 + 4 * rg + k;
      if (oy >= h1) break;
      const float4 a = r[2 * k], b = r[2 * k + 1], c = r[2 * k + 2], d = r[2 * k + 3], e = r[2 * k + 4];
      constexpr float sc = 1.f / 256.f;
      *reinterpret_cast<float4*>(out + (size_t)oy * w1 + ox) =
          make_float4(fv_h(a.x, b.x, c.x, d.x, e.x) * sc, fv_h(a.y, b.y, c.y, d.y, e.y) * sc,
                      fv_h(a.z, b.z, c.z, d.z, e.z) * sc, fv_h(a.w, b.w, c.w, d.w, e.w) * sc);
    }
  }
}

template <typename TIn, int TY>
__global__ void __launch_bounds__(fv_threads<TY>()) k_feat_reduce1_v(
    const TIn* __restrict__ rgb, int H, int W, const int* __restrict__ smax_p, float* __restrict__ I1,
    float* __restrict__ RG1, float* __restrict__ BY1, int h1, int w1, const SegIO* io, const uint8_t* on) {
  constexpr bool U8 = std::is_same<TIn, uint8_t>::value;
  constexpr int ROWS = 2 * TY + 3;  // level-0 rows under TY level-1 rows
  __shared__ __align__(16) float sH[3][ROWS][FV_TX];
  __shared__ float sHalo[ROWS][3][3];  // [row][pixel -2, -1, +128 of the span][channel]
  if constexpr (U8) {
    if (!rgb) rgb = io->rgb;
  }
  const int fb = blockIdx.z;  // frame of the batch
  if (SEG_SLOT_OFF(on, fb)) return;
  rgb += (size_t)fb * 3 * H * W;
  const size_t o1 = (size_t)fb * h1 * w1;
  const int X0 = blockIdx.x * FV_TX, Y0 = blockIdx.y * TY;
  const int cx0 = 2 * X0, ry0 = 2 * Y0 - 2;
  const int tid = threadIdx.x, slot = tid >> 3, j = tid & 7;
  const int nvalid = min(FV_LANES, (W - cx0) >> 4);  // threads of a row holding pixels
  const bool act = slot < ROWS && j < nvalid;
  const int row = seg_clampi(ry0 + slot, 0, H - 1);
  const TIn* run = rgb + 3 * ((size_t)row * W + cx0 + 16 * j);
  // RGB8: the run's 48 bytes, loaded before the wait for the frame maximum
  unsigned wv[U8 ? 12 : 1];
  if constexpr (U8) {
    if (act && ((uintptr_t)run & 15) == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(run);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldg(q + k);
        wv[4 * k] = v.x;
        wv[4 * k + 1] = v.y;
        wv[4 * k + 2] = v.z;
        wv[4 * k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k)
        wv[k] = act ? (unsigned)run[4 * k] | ((unsigned)run[4 * k + 1] << 8) | ((unsigned)run[4 * k + 2] << 16) |
                          ((unsigned)run[4 * k + 3] << 24)
                    : 0u;
    }
  }
  seg_pdl_enter();
  const int smax = smax_p[fb];
  const int thr2 = 2 * (smax / 10);
  const float smaxf = __int_as_float(smax);
  // the span's outer neighbours, one pixel per thread (clamped to the frame)
  if (tid < 3 * ROWS) {
    const int hr = tid / 3, hw = tid - 3 * hr;
    const int y = seg_clampi(ry0 + hr, 0, H - 1);
    const int x = seg_clampi(hw == 0 ? cx0 - 2 : hw == 1 ? cx0 - 1 : cx0 + 2 * FV_TX, 0, W - 1);
    const TIn* p = rgb + 3 * ((size_t)y * W + x);
    FV3 f;
    if constexpr (U8)
      f = fv_px_u8<0>((unsigned)p[0] | ((unsigned)p[1] << 8) | ((unsigned)p[2] << 16), thr2);
    else
      f = fv_px_f32(p[0], p[1], p[2], smaxf);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) sHalo[hr][hw][ch] = f.v[ch];
  }
  // features of the run
  float F[3][16];
  if constexpr (U8) {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const unsigned a = wv[3 * g], b = wv[3 * g + 1], c = wv[3 * g + 2];  // r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3
      const FV3 f0 = fv_px_u8<0>(a, thr2), f1 = fv_px_u8<0>(__byte_perm(a, b, 0x0543), thr2),
                f2 = fv_px_u8<0>(__byte_perm(b, c, 0x0432), thr2), f3 = fv_px_u8<8>(c, thr2);
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        F[ch][4 * g] = f0.v[ch];
        F[ch][4 * g + 1] = f1.v[ch];
        F[ch][4 * g + 2] = f2.v[ch];
        F[ch][4 * g + 3] = f3.v[ch];
      }
    }
  } else {
    const bool vec = ((uintptr_t)run & 15) == 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float e[12];
      if (act && vec) {
        const float4* q = reinterpret_cast<const float4*>(run) + 3 * g;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float4 v = __ldg(q + k);
          e[4 * k] = v.x;
          e[4 * k + 1] = v.y;
          e[4 * k + 2] = v.z;
          e[4 * k + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = act ? run[12 * g + k] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const FV3 f = fv_px_f32(e[3 * k], e[3 * k + 1], e[3 * k + 2], smaxf);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) F[ch][4 * g + k] = f.v[ch];
      }
    }
  }
  __syncthreads();  // sHalo
  fv_reduce_tile<TY>(F, sH, sHalo, slot, j, nvalid, X0, Y0, h1, w1, I1 + o1, RG1 + o1, BY1 + o1);
}

struct Reduce3Args {
  const float* in[3];
  float* out[3];
  int h, w, h2, w2;
  const uint8_t* on;
};

// One REDUCE step of one channel per CTA (blockIdx.z = channel + 3 * frame).
__global__ void __launch_bounds__(256) k_reduce3(Reduce3Args a) {
  seg_pdl_enter();
  __shared__ float sF[RED_IN_Y][RED_IN_X];
  __shared__ float sH[RED_IN_Y][RED_TX];
  const int ch = blockIdx.z % 3, fb = blockIdx.z / 3;
  if (SEG_SLOT_OFF(a.on, fb)) return;
  // (selects, not a runtime index into the parameter block, which would copy it to local memory)
  const float* __restrict__ in = (ch == 0 ? a.in[0] : ch == 1 ? a.in[1] : a.in[2]) + (size_t)fb * a.h * a.w;
  float* __restrict__ out = (ch == 0 ? a.out[0] : ch == 1 ? a.out[1] : a.out[2]) + (size_t)fb * a.h2 * a.w2;
  const int X0 = blockIdx.x * RED_TX, Y0 = blockIdx.y * RED_TY;
  const int gx0 = 2 * X0 - 2, gy0 = 2 * Y0 - 2;
  for (int i = threadIdx.x; i < RED_IN_Y * RED_IN_X; i += blockDim.x) {
    int ry = i / RED_IN_X, rx = i - ry * RED_IN_X;
    int gy = seg_clampi(gy0 + ry, 0, a.h - 1), gx = seg_clampi(gx0 + rx, 0, a.w - 1);
    sF[ry][rx] = in[(size_t)gy * a.w + gx];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RED_IN_Y * RED_TX; i += blockDim.x) {
    int ry = i / RED_TX, x = i - ry * RED_TX;
    const float* row = &sF[ry][2 * x];
    sH[ry][x] = c_binom[0] * row[0] + c_binom[1] * row[1] + c_binom[2] * row[2] +
                c_binom[3] * row[3] + c_binom[4] * row[4];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < RED_TY * RED_TX; i += blockDim.x) {
    int y = i / RED_TX, x = i - y * RED_TX;
    int oy = Y0 + y, ox = X0 + x;
    if (oy >= a.h2 || ox >= a.w2) continue;
    out[(size_t)oy * a.w2 + ox] = c_binom[0] * sH[2 * y][x] + c_binom[1] * sH[2 * y + 1][x] +
                                  c_binom[2] * sH[2 * y + 2][x] + c_binom[3] * sH[2 * y + 3][x] +
                                  c_binom[4] * sH[2 * y + 4][x];
  }
}

// The small pyramid levels in one launch: CTA = channel, levels computed one
// after another from global memory (L1/L2 resident), a barrier between levels.
struct PyrTailArgs {
  float* lvl[3][SEG_MAX_LEVELS];
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  int from, to;  // produce levels from+1 .. to
  const uint8_t* on;
};

__global__ void __launch_bounds__(1024) k_pyr_tail(PyrTailArgs a) {
  seg_pdl_enter();
  const int ch = blockIdx.x % 3, fb = blockIdx.x / 3;
  if (SEG_SLOT_OFF(a.on, fb)) return;
  for (int l = a.from; l < a.to; ++l) {
    const int h = a.hl[l], w = a.wl[l], h2 = a.hl[l + 1], w2 = a.wl[l + 1];
    const float* __restrict__ in = a.lvl[ch][l] + (size_t)fb * h * w;
    float* __restrict__ out = a.lvl[ch][l + 1] + (size_t)fb * h2 * w2;
    for (int i = threadIdx.x; i < h2 * w2; i += blockDim.x) {
      int y = i / w2, x = i - y * w2;
      int xs[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) xs[k] = seg_clampi(2 * x + k - 2, 0, w - 1);
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const float* row = in + (size_t)seg_clampi(2 * y + j - 2, 0, h - 1) * w;
        acc += c_binom[j] * (c_binom[0] * row[xs[0]] + c_binom[1] * row[xs[1]] + c_binom[2] * row[xs[2]] +
                             c_binom[3] * row[xs[3]] + c_binom[4] * row[xs[4]]);
      }
      out[i] = acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Gabor
#define GB_TX 32
#define GB_TY 16
#define GB_MAXR 8
#define GB_IN_X (GB_TX + 2 * GB_MAXR)
#define GB_IN_Y (GB_TY + 2 * GB_MAXR)

struct GaborArgs {
  const float* in[SEG_MAX_LEVELS];
  float* out[SEG_MAX_ORIENT][SEG_MAX_LEVELS];
  float2* out_c[SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // optional complex responses (backward form)
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  int lvl_first, lvl_last;
  int blk_off[SEG_MAX_LEVELS + 1];  // prefix of tile counts from lvl_first
  const uint8_t* on;
};

// Sec. 7.2 (edge orientation): O(sigma, theta) = |k_theta * I(sigma)| with the
// zero-mean complex Gabor factored into two separable complex terms.
// Orientation groups: {0}, {k, no - k} for 0 < k < no / 2, and {no / 2} when no
// is even.  theta and pi - theta have conjugate horizontal factors and the same
// vertical one, so a pair shares one horizontal pass and four vertical sums.
__host__ __device__ __forceinline__ int gb_ngroups(int no) { return no / 2 + 1 < no ? no / 2 + 1 : no; }
__device__ __forceinline__ void gb_group(int g, int no, int& k0, int& k1) {
  k0 = g;
  k1 = (g > 0 && 2 * g != no && no - g != g) ? no - g : -1;
}

// RT > 0: the radius at compile time (loops unrolled); 0: t.R at run time.
template <int RT>
__global__ void __launch_bounds__(256) k_gabor(GaborArgs a, GaborTaps t) {
  seg_pdl_enter();
  if (SEG_SLOT_OFF(a.on, blockIdx.y)) return;
  __shared__ float sIn[GB_IN_Y][GB_IN_X];
  __shared__ float sH0[GB_IN_Y][GB_TX];
  __shared__ float sHr[GB_IN_Y][GB_TX], sHi[GB_IN_Y][GB_TX];
  int b = blockIdx.x, l = a.lvl_first;
  while (l < a.lvl_last && b >= a.blk_off[l - a.lvl_first + 1]) ++l;
  b -= a.blk_off[l - a.lvl_first];
  const int h = a.hl[l], w = a.wl[l];
  const size_t fo = (size_t)blockIdx.y * h * w;  // frame of the batch
  const int ntx = (w + GB_TX - 1) / GB_TX;
  const int X0 = (b % ntx) * GB_TX, Y0 = (b / ntx) * GB_TY;
  const int R = RT > 0 ? RT : t.R, K = 2 * R + 1;
  const int iny = GB_TY + 2 * R, inx = GB_TX + 2 * R;
  const float* __restrict__ in = a.in[l] + fo;
  for (int i = threadIdx.x; i < iny * inx; i += blockDim.x) {
    int ry = i / inx, rx = i - ry * inx;
    sIn[ry][rx] = in[(size_t)seg_clampi(Y0 - R + ry, 0, h - 1) * w + seg_clampi(X0 - R + rx, 0, w - 1)];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < iny * GB_TX; i += blockDim.x) {
    int ry = i / GB_TX, x = i - ry * GB_TX;
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < (RT > 0 ? 2 * RT + 1 : GB_MAXR * 2 + 1); ++u) {
      if (RT == 0 && u >= K) break;
      acc += t.g0[u] * sIn[ry][x + u];
    }
    sH0[ry][x] = acc;
  }
  __syncthreads();
  // this thread's output pixels (i = tid, tid + 256) and their Gaussian (DC) term,
  // the same for every orientation
  constexpr int NPX = GB_TY * GB_TX / 256;
  float dcv[NPX];
#pragma unroll
  for (int j = 0; j < NPX; ++j) {
    const int i = threadIdx.x + 256 * j, y = i / GB_TX, x = i - y * GB_TX;
    float dc = 0.f;
#pragma unroll
    for (int v = 0; v < (RT > 0 ? 2 * RT + 1 : GB_MAXR * 2 + 1); ++v) {
      if (RT == 0 && v >= K) break;
      dc += t.g0[v] * sH0[y + v][x];
    }
    dcv[j] = dc;
  }
  // one orientation group per CTA when the grid has one z-slice per group (single
  // frame), otherwise every group in turn from the same staged tile
  const int ng = gb_ngroups(t.no);
  const int g_begin = gridDim.z == 1 ? 0 : blockIdx.z, g_end = gridDim.z == 1 ? ng : blockIdx.z + 1;
  for (int gi = g_begin; gi < g_end; ++gi) {
    int k0, k1;
    gb_group(gi, t.no, k0, k1);
    __syncthreads();
    for (int i = threadIdx.x; i < iny * GB_TX; i += blockDim.x) {
      int ry = i / GB_TX, x = i - ry * GB_TX;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int u = 0; u < (RT > 0 ? 2 * RT + 1 : GB_MAXR * 2 + 1); ++u) {
        if (RT == 0 && u >= K) break;
        float p = sIn[ry][x + u];
        re += t.hx_re[k0][u] * p;
        im += t.hx_im[k0][u] * p;
      }
      sHr[ry][x] = re;
      sHi[ry][x] = im;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
      const int i = threadIdx.x + 256 * j, y = i / GB_TX, x = i - y * GB_TX;
      const int oy = Y0 + y, ox = X0 + x;
      if (oy >= h || ox >= w) continue;
      // P = sum vre hr, Q = sum vim hi, Rr = sum vre hi, Sr = sum vim hr: theta gives
      // (P - Q, Rr + Sr); pi - theta (conjugate horizontal factor) gives (P + Q, Sr - Rr)
      float P = 0.f, Q = 0.f, Rr = 0.f, Sr = 0.f;
#pragma unroll
      for (int v = 0; v < (RT > 0 ? 2 * RT + 1 : GB_MAXR * 2 + 1); ++v) {
        if (RT == 0 && v >= K) break;
        const float hr = sHr[y + v][x], hi = sHi[y + v][x];
        const float vr = t.vy_re[k0][v], vi = t.vy_im[k0][v];
        P += vr * hr;
        Q += vi * hi;
        Rr += vr * hi;
        Sr += vi * hr;
      }
      const size_t o = fo + (size_t)oy * w + ox;
      {
        const float re = P - Q - t.kap_re[k0] * dcv[j], im = Rr + Sr - t.kap_im[k0] * dcv[j];
        a.out[k0][l][o] = sqrtf(re * re + im * im);
        if (a.out_c[k0][l]) a.out_c[k0][l][o] = make_float2(re, im);
      }
      if (k1 >= 0) {
        const float re = P + Q - t.kap_re[k1] * dcv[j], im = Sr - Rr - t.kap_im[k1] * dcv[j];
        a.out[k1][l][o] = sqrtf(re * re + im * im);
        if (a.out_c[k1][l]) a.out_c[k1][l][o] = make_float2(re, im);
      }
    }
  }
}

// ------------------------------------------------------------------ center-surround
struct CSArgs {
  const float* X[3 + SEG_MAX_ORIENT][SEG_MAX_LEVELS];  // channel planes per level
  int hl[SEG_MAX_LEVELS], wl[SEG_MAX_LEVELS];
  int pair_c[SEG_MAX_PAIRS], pair_s[SEG_MAX_PAIRS];
  int pair_band_off[SEG_MAX_PAIRS + 1];  // prefix of (row bands x channels) per pair
  int npairs, nch, tile, opp_sum;
  int nbands_total;
  unsigned* mm;
  float* tpart;
  float flat;  // N(.) flat-map threshold
  int c_lo, c_hi;  // center scales c_min .. c_max (= sigma_S)
  const int2* rs;
  int rs_row[SEG_MAX_PAIRS], rs_col[SEG_MAX_PAIRS];
  const uint8_t* on;
  int sm_ws, sm_wc;  // widest surround and center level: the staged shared-memory layout
};

// The center-surround statistics kernel stages what its CTA reads of a pair's
// surround level in shared memory: up to CS_SR rows of every channel it
// handles (the rows the bilinear up-sampling of its band's center rows
// touches), the pair's column table and the row-table entries of the band
// (with the surround rows renumbered from the first staged one).  Values are unchanged: the same
// interpolation reads the same numbers from shared memory.
#define CS_SR 4
#define CS_TR 32
__host__ __device__ constexpr size_t cs_stage_bytes(int nf, int ws, int wc) {
  return sizeof(float) * (size_t)nf * CS_SR * ws + sizeof(int2) * ((size_t)wc + CS_TR);
}


#define CS_MAX_TILES_X 1024

// Per (center-surround pair, band of `tile` rows), for all NCH channels at once
// (they share the pair's resampling coordinates): min, max and the sum of the
// band's T x T tile maxima (Sec. 7.2 step 3: block-wise extrema).  One warp
// reduces one tile at a time with shuffles; maps are non-negative, so their
// float bit patterns order like the values for the global min/max atomics.
template <int NCH, int CPB>
__global__ void __launch_bounds__(256) k_cs_stats(CSArgs a) {
  seg_pdl_enter();
  extern __shared__ __align__(16) float cs_dyn[];
  __shared__ float sMin[8][CPB], sMax[8][CPB], sTs[8][CPB];
  constexpr int G = NCH / CPB;  // channel groups per (pair, band)
  const int f0 = (blockIdx.x % G) * CPB;
  int b = blockIdx.x / G, p = 0;
  while (p < a.npairs - 1 && b >= a.pair_band_off[p + 1] / NCH) ++p;
  const int c = a.pair_c[p], sv = a.pair_s[p];
  const int hc = a.hl[c], wc = a.wl[c], hs = a.hl[sv], ws = a.wl[sv], T = a.tile;
  const int nb = (hc + T - 1) / T, ntx = (wc + T - 1) / T;
  const int band = b - a.pair_band_off[p] / NCH;
  const int fb = blockIdx.y;  // frame of the batch
  if (SEG_SLOT_OFF(a.on, fb)) return;
  unsigned* mm = a.mm + (size_t)fb * 2 * a.npairs * NCH;
  float* tpart = a.tpart + (size_t)fb * a.nbands_total;
  const float* cen[CPB];
  const float* sur[CPB];
#pragma unroll
  for (int f = 0; f < CPB; ++f) {
    cen[f] = a.X[f0 + f][c] + (size_t)fb * hc * wc;
    sur[f] = a.X[f0 + f][sv] + (size_t)fb * hs * ws;
  }
  const int2* trow = a.rs + a.rs_row[p];
  const int2* tcol = a.rs + a.rs_col[p];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int y0 = band * T, rows = min(T, hc - y0);
  const int lo = trow[y0].x & 0xffff, nr = (trow[y0 + rows - 1].x >> 16) - lo + 1;
  const bool staged = nr <= CS_SR && ws <= a.sm_ws && wc <= a.sm_wc && rows <= CS_TR;
  float* sS = cs_dyn;                                                       // [CPB][CS_SR][ws]
  int2* sTc = reinterpret_cast<int2*>(cs_dyn + (size_t)CPB * CS_SR * a.sm_ws);  // [wc]
  int2* sTr = sTc + a.sm_wc;                                                 // [rows], renumbered
  if (staged) {
#pragma unroll
    for (int f = 0; f < CPB; ++f)
      for (int i = threadIdx.x; i < nr * ws; i += blockDim.x) sS[f * CS_SR * ws + i] = sur[f][lo * ws + i];
    for (int i = threadIdx.x; i < wc; i += blockDim.x) sTc[i] = tcol[i];
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
      const int2 r = trow[y0 + i];
      sTr[i] = make_int2(r.x - lo - (lo << 16), r.y);
    }
    __syncthreads();
  }
  float mn[CPB], mx[CPB], ts[CPB];
#pragma unroll
  for (int f = 0; f < CPB; ++f) {
    mn[f] = 3.0e38f;
    mx[f] = 0.f;
    ts[f] = 0.f;
  }
  // one element: its |CS| value per channel into the running extrema and tile maxima
#define CS_ELEMENT(RY, RX, SUR_F, Y, X)                                                      \
  {                                                                                          \
    float u = seg_bilinear_t(SUR_F, ws, RY, RX), v0 = cen[f][(Y) * wc + (X)];                \
    const int ch = f0 + f;                                                                   \
    float v = (a.opp_sum && (ch == 1 || ch == 2)) ? fabsf(v0 + u) : fabsf(v0 - u);           \
    mn[f] = fminf(mn[f], v);                                                                 \
    mx[f] = fmaxf(mx[f], v);                                                                 \
    tm[f] = fmaxf(tm[f], v);                                                                 \
  }
  for (int tx = wid; tx < ntx; tx += nw) {
    const int x0 = tx * T, cols = min(T, wc - x0);
    float tm[CPB];
#pragma unroll
    for (int f = 0; f < CPB; ++f) tm[f] = 0.f;
    if (staged) {
#pragma unroll 2
      for (int i = lane; i < rows * cols; i += 32) {
        const int yy = i / cols, xx = i - yy * cols;
        const int2 ry = sTr[yy], rx = sTc[x0 + xx];
#pragma unroll
        for (int f = 0; f < CPB; ++f) CS_ELEMENT(ry, rx, sS + f * CS_SR * ws, y0 + yy, x0 + xx)
      }
    } else {
      for (int i = lane; i < rows * cols; i += 32) {
        const int yy = i / cols, y = y0 + yy, x = x0 + (i - yy * cols);
        const int2 ry = trow[y], rx = tcol[x];
#pragma unroll
        for (int f = 0; f < CPB; ++f) CS_ELEMENT(ry, rx, sur[f], y, x)
      }
    }
#pragma unroll
    for (int f = 0; f < CPB; ++f) ts[f] += seg_warp_max_f(tm[f]);  // every lane holds the tile maximum
  }
#undef CS_ELEMENT
#pragma unroll
  for (int f = 0; f < CPB; ++f) {
    float a0 = seg_warp_min_f(mn[f]), a1 = seg_warp_max_f(mx[f]);
    if (lane == 0) {
      sMin[wid][f] = a0;
      sMax[wid][f] = a1;
      sTs[wid][f] = ts[f];
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < CPB) {
    const int f = threadIdx.x, m = p * NCH + f0 + f;
    float a0 = sMin[0][f], a1 = sMax[0][f], a2 = 0.f;
    for (int w = 0; w < nw; ++w) {
      a0 = fminf(a0, sMin[w][f]);
      a1 = fmaxf(a1, sMax[w][f]);
      a2 += sTs[w][f];
    }
    atomicMin(&mm[2 * m], __float_as_uint(a0));
    atomicMax(&mm[2 * m + 1], __float_as_uint(a1));
    tpart[a.pair_band_off[p] + (f0 + f) * nb + band] = a2;
  }
}

// N(v) = a v + b with a = (1 - mbar)^2 / (max - min), b = -min a, where mbar is
// the mean of the tile maxima of the rescaled map without one copy of its
// maximum 1; a flat map (range <= flat) gives a = b = 0.  Single precision: the
// few threads that form it would otherwise hold the whole CTA at its next
// barrier on the narrow FP64 pipe.
__device__ __forceinline__ void norm_affine(float mn, float mx, float sum_tmax, int nt, float flat, float* ab) {
  const float range = mx - mn;
  if (!(range > flat)) {
    ab[0] = 0.f;
    ab[1] = 0.f;
    return;
  }
  const float st = (sum_tmax - (float)nt * mn) / range;
  const float mbar = nt > 1 ? (st - 1.f) / (float)(nt - 1) : 0.f;
  const float a = (1.f - mbar) * (1.f - mbar) / range;
  ab[0] = a;
  ab[1] = -mn * a;
}

// N(.) of map m = (pair p, channel f) as a*v + b from its statistics.
__device__ void cs_map_affine(const CSArgs& a, int p, int f, float flat, float* ab, int fb) {
  int c = a.pair_c[p];
  int T = a.tile, nb = (a.hl[c] + T - 1) / T, ntx = (a.wl[c] + T - 1) / T;
  int m = p * a.nch + f;
  const unsigned* mm = a.mm + (size_t)fb * 2 * a.npairs * a.nch;
  float sum = 0.f;
  const float* tp = a.tpart + (size_t)fb * a.nbands_total + a.pair_band_off[p] + f * nb;
  for (int i = 0; i < nb; ++i) sum += tp[i];
  norm_affine(__uint_as_float(mm[2 * m]), __uint_as_float(mm[2 * m + 1]), sum, nb * ntx, flat, ab);
}


// B_c(f) = sum over pairs (c, s) of N(CS_f(c, s)) + REDUCE(B_{c-1}(f)).
#define ACC_TX 32
#define ACC_TY 8
#define ACC_MAX_PC 16  // center-surround pairs per center scale
// B_c = sum over pairs (c, s) of N(CS(c, s)) + REDUCE(B_{c-1}), all NCH channels
// of a 32 x 8 output tile per CTA; the REDUCE input tile (with its 2-pixel
// halo) is staged in shared memory one channel at a time.
template <int NCH, int CPB>
__global__ void __launch_bounds__(256) k_cs_accum(CSArgs a, int c, const float* __restrict__ prev, int hp,
                                                  int wp, float* __restrict__ out) {
  seg_pdl_enter();
  // channels whose REDUCE(B_{c-1}) tiles are staged together (2: 80 registers, 3 CTAs per SM; 4 took 101
  // registers and 2 CTAs per SM, and the 32-frame saliency 306.5 us against 299.5)
  constexpr int CG = CPB < 2 ? CPB : 2;
  constexpr int PY = 2 * ACC_TY + 3, PX = 2 * ACC_TX + 3;
  __shared__ float sP[CG][PY][PX];
  __shared__ float sH[CG][PY][ACC_TX];
  __shared__ float sab[2 * ACC_MAX_PC * CPB];  // N(.) of this CTA's maps as a*v + b
  constexpr int G = NCH / CPB;                  // channel groups
  const int fb = blockIdx.z / G;                // frame of the batch
  if (SEG_SLOT_OFF(a.on, fb)) return;
  const int f0 = (blockIdx.z % G) * CPB;        // first channel of this CTA
  const int hc = a.hl[c], wc = a.wl[c];
  {
    // the affine form of N(.) of every (pair with center c, channel) map this CTA
    // adds, from the statistics of k_cs_stats
    int npc = 0;
    for (int p = 0; p < a.npairs; ++p) npc += a.pair_c[p] == c;
    for (int j = threadIdx.x; j < npc * CPB; j += blockDim.x) {
      const int slot = j / CPB, f = j - slot * CPB;
      int p = 0;
      for (int k = -1; p < a.npairs; ++p)
        if (a.pair_c[p] == c && ++k == slot) break;
      cs_map_affine(a, p, f0 + f, a.flat, &sab[2 * j], fb);
    }
    __syncthreads();
  }
  if (prev) prev += (size_t)fb * NCH * hp * wp;
  out += (size_t)fb * NCH * hc * wc;
  const int X0 = blockIdx.x * ACC_TX, Y0 = blockIdx.y * ACC_TY;
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int x = X0 + lx, y = Y0 + ly;
  const bool in = x < wc && y < hc;
  float acc[CPB];
#pragma unroll
  for (int f = 0; f < CPB; ++f) acc[f] = 0.f;
  if (in) {
    for (int p = 0, slot = 0; p < a.npairs; ++p) {
      if (a.pair_c[p] != c) continue;
      const float* ab = &sab[2 * CPB * slot++];
      const int sv = a.pair_s[p], hs = a.hl[sv], ws = a.wl[sv];
      const int2 ry = a.rs[a.rs_row[p] + y], rx = a.rs[a.rs_col[p] + x];
#pragma unroll
      for (int f = 0; f < CPB; ++f) {
        const int ch = f0 + f;
        float u = seg_bilinear_t(a.X[ch][sv] + (size_t)fb * hs * ws, ws, ry, rx);
        float v0 = a.X[ch][c][(size_t)fb * hc * wc + (size_t)y * wc + x];
        float v = (a.opp_sum && (ch == 1 || ch == 2)) ? fabsf(v0 + u) : fabsf(v0 - u);
        acc[f] += ab[2 * f] * v + ab[2 * f + 1];
      }
    }
  }
  if (prev) {
    // REDUCE(B_{c-1}) of CG channels at a time: their halo tiles are loaded
    // together (every load of a thread in flight before the first store), then
    // one horizontal and one vertical pass -- one load round trip and two
    // barriers per group instead of per channel (256 threads)
    const int gx0 = 2 * X0 - 2, gy0 = 2 * Y0 - 2;
    constexpr int NL = CG * PY * PX, PL = (NL + 255) / 256;
#pragma unroll
    for (int g0 = 0; g0 < CPB; g0 += CG) {
      const int ng = CPB - g0 < CG ? CPB - g0 : CG;
      float v[PL];
#pragma unroll
      for (int k = 0; k < PL; ++k) {
        const int i = threadIdx.x + 256 * k;
        v[k] = 0.f;
        if (i < ng * PY * PX) {
          const int f = i / (PY * PX), rem = i - f * PY * PX, ry = rem / PX, rx = rem - ry * PX;
          v[k] = prev[(size_t)(f0 + g0 + f) * hp * wp + (size_t)seg_clampi(gy0 + ry, 0, hp - 1) * wp +
                      seg_clampi(gx0 + rx, 0, wp - 1)];
        }
      }
#pragma unroll
      for (int k = 0; k < PL; ++k) {
        const int i = threadIdx.x + 256 * k;
        if (i < ng * PY * PX) (&sP[0][0][0])[i] = v[k];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < ng * PY * ACC_TX; i += blockDim.x) {
        const int f = i / (PY * ACC_TX), rem = i - f * PY * ACC_TX, ry = rem / ACC_TX, xx = rem - ry * ACC_TX;
        const float* row = &sP[f][ry][2 * xx];
        sH[f][ry][xx] = c_binom[0] * row[0] + c_binom[1] * row[1] + c_binom[2] * row[2] + c_binom[3] * row[3] +
                        c_binom[4] * row[4];
      }
      __syncthreads();
#pragma unroll
      for (int f = 0; f < CG; ++f)
        if (g0 + f < CPB)
          acc[g0 + f] += c_binom[0] * sH[f][2 * ly][lx] + c_binom[1] * sH[f][2 * ly + 1][lx] +
                         c_binom[2] * sH[f][2 * ly + 2][lx] + c_binom[3] * sH[f][2 * ly + 3][lx] +
                         c_binom[4] * sH[f][2 * ly + 4][lx];
      __syncthreads();
    }
  }
  if (in)
#pragma unroll
    for (int f = 0; f < CPB; ++f) out[(size_t)(f0 + f) * hc * wc + (size_t)y * wc + x] = acc[f];
}

// ------------------------------------------------------------------ fused across-scale sum
// B_{c_max} over one 8 x 8 tile of sigma_S per CTA (one channel, one frame),
// level by level from c_min over the tile's halo regions: the region of level
// c_max - k starts at 2^k (Y0, X0) - 3 (2^k - 1) and holds 2^k 8 + 3 (2^k - 1)
// rows and columns, each entry at its clamped level coordinate, so every
// REDUCE input the next level needs is in shared memory.  Same sums as the
// level-by-level kernel: B_c = sum over pairs (c, s) of N(CS(c, s)) + REDUCE(B_{c-1}).
// Up to two REDUCE steps (c_max - c_min <= 2).
#define FA_TX 8  // (16 x 8: 84 CTAs at 640x480 and 67.5 us for the saliency; 8 x 4: 71.0; 8 x 8: 65.2)
#define FA_TY 8
#define FA_N(t, k) (((t) << (k)) + 3 * ((1 << (k)) - 1))

__device__ __forceinline__ float fa_eval(const CSArgs& a, const float* sab, int c, int f, int fb, int y, int x) {
  float acc = 0.f;
  for (int p = 0; p < a.npairs; ++p) {
    if (a.pair_c[p] != c) continue;
    const int sv = a.pair_s[p], hs = a.hl[sv], ws = a.wl[sv];
    const float u = seg_bilinear_t(a.X[f][sv] + (size_t)fb * hs * ws, ws, a.rs[a.rs_row[p] + y], a.rs[a.rs_col[p] + x]);
    const float v0 = a.X[f][c][(size_t)fb * a.hl[c] * a.wl[c] + (size_t)y * a.wl[c] + x];
    const float v = (a.opp_sum && (f == 1 || f == 2)) ? fabsf(v0 + u) : fabsf(v0 - u);
    acc += sab[2 * p] * v + sab[2 * p + 1];
  }
  return acc;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_cs_accum_fused(CSArgs a, float* __restrict__ out) {
  seg_pdl_enter();
  __shared__ float sR2[FA_N(FA_TY, 2) * FA_N(FA_TX, 2)];  // region two levels below sigma_S
  __shared__ float sR1[FA_N(FA_TY, 1) * FA_N(FA_TX, 1)];  // one level below
  __shared__ float sT[FA_N(FA_TY, 2) * FA_N(FA_TX, 1)];   // horizontal REDUCE pass
  __shared__ float sab[2 * SEG_MAX_PAIRS];
  const int f = blockIdx.z % a.nch, fb = blockIdx.z / a.nch;
  if (SEG_SLOT_OFF(a.on, fb)) return;
  const int cmax = a.c_hi, D = a.c_hi - a.c_lo;
  for (int p = threadIdx.x; p < a.npairs; p += blockDim.x) cs_map_affine(a, p, f, a.flat, &sab[2 * p], fb);
  int RY[3], RX[3], NY[3], NX[3];
  RY[0] = blockIdx.y * FA_TY;
  RX[0] = blockIdx.x * FA_TX;
  NY[0] = FA_TY;
  NX[0] = FA_TX;
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    RY[k] = 2 * RY[k - 1] - 2;
    RX[k] = 2 * RX[k - 1] - 2;
    NY[k] = 2 * NY[k - 1] + 3;
    NX[k] = 2 * NX[k - 1] + 3;
  }
  float* const buf[3] = {nullptr, sR1, sR2};
  __syncthreads();
  // unrolled over the level offset so the region arrays stay in registers
#pragma unroll
  for (int k = 2; k >= 0; --k) {
    if (k > D) continue;
    const int c = cmax - k, hc = a.hl[c], wc = a.wl[c];
    if (k < D) {
      // horizontal pass of REDUCE(B_{c-1}): rows of the finer region x this region's columns
      const int hf = a.hl[c - 1], wf = a.wl[c - 1];
      const float* F = buf[k + 1];
      for (int i = threadIdx.x; i < NY[k + 1] * NX[k]; i += blockDim.x) {
        const int r = i / NX[k], q = i - r * NX[k];
        const int xc = seg_clampi(RX[k] + q, 0, wc - 1);
        const float* row = F + r * NX[k + 1];
        float h = 0.f;
#pragma unroll
        for (int t = 0; t < 5; ++t)
          h += c_binom[t] * row[seg_clampi(seg_clampi(2 * xc + t - 2, 0, wf - 1) - RX[k + 1], 0, NX[k + 1] - 1)];
        sT[i] = h;
      }
      (void)hf;
      __syncthreads();
    }
    const int n = NY[k] * NX[k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / NX[k], q = i - r * NX[k];
      const int yy = RY[k] + r, xx = RX[k] + q;
      if (k == 0 && (yy >= hc || xx >= wc)) continue;
      const int y = seg_clampi(yy, 0, hc - 1), x = seg_clampi(xx, 0, wc - 1);
      float v = fa_eval(a, sab, c, f, fb, y, x);
      if (k < D) {
        const int hf = a.hl[c - 1];
        float s2 = 0.f;
#pragma unroll
        for (int t = 0; t < 5; ++t)
          s2 += c_binom[t] * sT[seg_clampi(seg_clampi(2 * y + t - 2, 0, hf - 1) - RY[k + 1], 0, NY[k + 1] - 1) * NX[k] + q];
        v += s2;
      }
      if (k == 0)
        out[((size_t)fb * a.nch + f) * hc * wc + (size_t)y * wc + x] = v;
      else
        buf[k][i] = v;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ conspicuity, S


#define CONSP_TILES 1024  // N(.) tiles per map at sigma_S

// N(.) parameters of up to four maps held in global memory, computed by the
// whole CTA in one pass over the pixels: min, max and the T x T tile maxima
// (shared-memory atomics on order-preserving keys), then each map's affine
// form on one thread.  ab[2m], ab[2m+1] receive map m's a and b.
__device__ void block_norm_multi(const float* const* v, int nm, int h, int w, int T, float flat,
                                 float* ab, float* red, unsigned* tmax) {
  const int n = h * w, ntx = (w + T - 1) / T, nt = ntx * ((h + T - 1) / T);
  for (int t = threadIdx.x; t < nm * CONSP_TILES; t += blockDim.x) tmax[t] = 0u;
  __syncthreads();
  float mn[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f}, mx[4] = {-3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int yy = i / w, xx = i - yy * w, tile = (yy / T) * ntx + xx / T;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (m >= nm) break;
      float x = v[m][i];
      mn[m] = fminf(mn[m], x);
      mx[m] = fmaxf(mx[m], x);
      atomicMax(&tmax[m * CONSP_TILES + tile], f2key(x));
    }
  }
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float a0 = seg_warp_min_f(mn[m]), a1 = seg_warp_max_f(mx[m]);
    if ((threadIdx.x & 31) == 0) {
      red[(3 * m) * 32 + wid] = a0;
      red[(3 * m + 1) * 32 + wid] = a1;
    }
  }
  __syncthreads();
  float ts[4] = {0.f, 0.f, 0.f, 0.f};
  for (int t = threadIdx.x; t < nt; t += blockDim.x)
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (m < nm) ts[m] += key2f(tmax[m * CONSP_TILES + t]);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float a2 = seg_warp_sum_f(ts[m]);
    if ((threadIdx.x & 31) == 0) red[(3 * m + 2) * 32 + wid] = a2;
  }
  __syncthreads();
  if ((int)threadIdx.x < nm) {
    const int m = threadIdx.x;
    float a0 = red[(3 * m) * 32], a1 = red[(3 * m + 1) * 32];
    float a2 = 0.f;
    for (int i = 0; i < nw; ++i) {
      a0 = fminf(a0, red[(3 * m) * 32 + i]);
      a1 = fmaxf(a1, red[(3 * m + 1) * 32 + i]);
      a2 += red[(3 * m + 2) * 32 + i];
    }
    norm_affine(a0, a1, a2, nt, flat, ab + 2 * m);
  }
  __syncthreads();
}

struct ConspArgs {
  const float* acc;  // nch planes at sigma_S
  int h, w, nch, tile;
  int H, W;          // frame size of the up-sampled saliency
  unsigned* salmax;  // per frame: max of the up-sampled saliency (float bits, >= 0)
  const int2* frow;  // final up-sampling tables
  const int2* fcol;
  float flat;
  float wgt[4];
  const double* wdev;  // if set: the channel weights are read from device memory
  float* csum;
  float* consp;
  float* S;
  const uint8_t* on;
};

// Orientation conspicuity sum_theta N(B_theta), then N of the four conspicuity
// maps and S = sum_k w_k N(C_k): two normalisation passes of up to 4 maps each.
// STAGED: the accumulators, C_O and S live in shared memory during the kernel
// (one load, every later pass at shared-memory latency) and C_O and S are
// written out at the end.
template <bool STAGED>
__global__ void __launch_bounds__(1024) k_consp(ConspArgs a) {
  seg_pdl_enter();
  extern __shared__ float dsm[];
  __shared__ float ab[8];
  __shared__ float red[12 * 32];
  __shared__ unsigned tmax[4 * CONSP_TILES];
  const int n = a.h * a.w;
  const int fb = blockIdx.x;  // frame of the batch
  if (SEG_SLOT_OFF(a.on, fb)) return;
  a.acc += (size_t)fb * a.nch * n;
  float* const csum_g = a.csum + (size_t)fb * n;
  float* const S_g = a.S + (size_t)fb * n;
  a.consp += (size_t)fb * 4 * n;
  if (STAGED) {
    for (int i = threadIdx.x; i < a.nch * n; i += blockDim.x) dsm[i] = a.acc[i];
    a.acc = dsm;
    a.csum = dsm + (size_t)a.nch * n;
    a.S = dsm + (size_t)(a.nch + 1) * n;
    __syncthreads();
  } else {
    a.csum = csum_g;
    a.S = S_g;
  }
  const float* v[4];
  for (int k0 = 3; k0 < a.nch; k0 += 4) {
    const int nm = min(4, a.nch - k0);
    for (int m = 0; m < nm; ++m) v[m] = a.acc + (size_t)(k0 + m) * n;
    block_norm_multi(v, nm, a.h, a.w, a.tile, a.flat, ab, red, tmax);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float acc = k0 == 3 ? 0.f : a.csum[i];
      for (int m = 0; m < nm; ++m) acc += ab[2 * m] * v[m][i] + ab[2 * m + 1];
      a.csum[i] = acc;
    }
    __syncthreads();
  }
  v[0] = a.acc;
  v[1] = a.acc + n;
  v[2] = a.acc + 2 * (size_t)n;
  v[3] = a.csum;
  block_norm_multi(v, 4, a.h, a.w, a.tile, a.flat, ab, red, tmax);
  float wk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wk[k] = a.wdev ? (float)a.wdev[k] : a.wgt[k];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float nv = ab[2 * k] * v[k][i] + ab[2 * k + 1];
      a.consp[(size_t)k * n + i] = nv;
      S += wk[k] * nv;
    }
    a.S[i] = S;
  }
  __syncthreads();
  // Maximum of the bilinear up-sampling of S to H x W without visiting every
  // pixel: within one source cell the interpolant is bilinear in (y, x), so over
  // the output samples of that cell it peaks at its first or last sample row and
  // column.  Only those rows and columns are evaluated (same arithmetic as the
  // up-sampling itself, so the value is identical).
  if (STAGED) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      csum_g[i] = a.csum[i];
      S_g[i] = a.S[i];
    }
  }
  int* crow = (int*)tmax;
  int* ccol = crow + 2048;
  __shared__ int nr, nc;
  if (threadIdx.x == 0) nr = nc = 0;
  __syncthreads();
  for (int y = threadIdx.x; y < a.H; y += blockDim.x)
    if (seg_up_candidate(y, a.h, a.H)) crow[atomicAdd(&nr, 1)] = y;
  for (int x = threadIdx.x; x < a.W; x += blockDim.x)
    if (seg_up_candidate(x, a.w, a.W)) ccol[atomicAdd(&nc, 1)] = x;
  __syncthreads();
  float mxv = 0.f;
  for (int k = threadIdx.x; k < nr * nc; k += blockDim.x)
    mxv = fmaxf(mxv, seg_bilinear_t(a.S, a.w, a.frow[crow[k / nc]], a.fcol[ccol[k % nc]]));
  mxv = seg_warp_max_f(mxv);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mxv;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mxv = fmaxf(mxv, red[w]);
    a.salmax[blockIdx.x] = __float_as_uint(fmaxf(red[0], mxv));
  }
}

__global__ void __launch_bounds__(256) k_upsample(const float* __restrict__ S, int hs, int ws, int H,
                                                  int W, float* __restrict__ sal, const SegIO* io,
                                                  const int2* __restrict__ frow, const int2* __restrict__ fcol,
                                                  const uint8_t* on) {
  seg_pdl_enter();
  if (!sal) sal = io->sal;
  const int fb = blockIdx.z;  // frame of the batch
  if (SEG_SLOT_OFF(on, fb)) return;
  S += (size_t)fb * hs * ws;
  sal += (size_t)fb * H * W;
  const int xq = blockIdx.x * 64 + (threadIdx.x & 63), y = blockIdx.y * 4 + (threadIdx.x >> 6);
  if (y >= H) return;
  const int2 ry = frow[y];
  float* row = sal + (size_t)y * W;
  if ((W & 3) == 0 && ((uintptr_t)sal & 15) == 0) {  // four pixels, one 16-byte store
    const int x = 4 * xq;
    if (x >= W) return;
    float4 v;
    v.x = seg_bilinear_t(S, ws, ry, fcol[x]);
    v.y = seg_bilinear_t(S, ws, ry, fcol[x + 1]);
    v.z = seg_bilinear_t(S, ws, ry, fcol[x + 2]);
    v.w = seg_bilinear_t(S, ws, ry, fcol[x + 3]);
    *reinterpret_cast<float4*>(row + x) = v;
  } else {
    for (int x = 4 * xq; x < 4 * xq + 4 && x < W; ++x) row[x] = seg_bilinear_t(S, ws, ry, fcol[x]);
  }
}

// S -> H x W saliency for a band of UP_ROWS output rows per CTA: the few rows of
// S the band touches are first interpolated along x into shared memory (each
// once per band instead of once per output row), then every output pixel is
// the interpolation of two of those rows along y, four pixels per 16-byte
// store.  The arithmetic and its order are seg_bilinear_t's: along x within a
// source row, then along y.
#define UP_ROWS 8
__global__ void __launch_bounds__(256) k_upsample_rows(const float* __restrict__ S, int hs, int ws, int H, int W,
                                                       float* __restrict__ sal, const SegIO* io,
                                                       const int2* __restrict__ frow,
                                                       const int2* __restrict__ fcol, const uint8_t* on) {
  seg_pdl_enter();
  extern __shared__ __align__(16) float up_smem[];  // [rows of S touched][W]
  if (!sal) sal = io->sal;
  const int fb = blockIdx.y;  // frame of the batch
  if (SEG_SLOT_OFF(on, fb)) return;
  S += (size_t)fb * hs * ws;
  sal += (size_t)fb * H * W;
  const int y_first = blockIdx.x * UP_ROWS, y_last = min(y_first + UP_ROWS, H) - 1;
  const int s0 = frow[y_first].x & 0xffff, s1 = frow[y_last].x >> 16;  // source rows s0 .. s1
  const int nr = s1 - s0 + 1;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const int2 rx = fcol[x];
    const int x0 = rx.x & 0xffff, x1 = rx.x >> 16;
    const float fx = __int_as_float(rx.y);
    for (int r = 0; r < nr; ++r) {
      const float* row = S + (size_t)(s0 + r) * ws;
      up_smem[r * W + x] = (1.f - fx) * row[x0] + fx * row[x1];
    }
  }
  __syncthreads();
  const bool vec = (W & 3) == 0 && ((uintptr_t)sal & 15) == 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int y = y_first + wid; y <= y_last; y += nw) {  // one warp per output row
    const int2 ry = frow[y];
    const float* t = up_smem + (size_t)((ry.x & 0xffff) - s0) * W;
    const float* b = up_smem + (size_t)((ry.x >> 16) - s0) * W;
    const float fy = __int_as_float(ry.y);
    float* out = sal + (size_t)y * W;
    if (vec) {
      for (int x = 4 * lane; x < W; x += 128) {
        float4 v;
        v.x = (1.f - fy) * t[x] + fy * b[x];
        v.y = (1.f - fy) * t[x + 1] + fy * b[x + 1];
        v.z = (1.f - fy) * t[x + 2] + fy * b[x + 2];
        v.w = (1.f - fy) * t[x + 3] + fy * b[x + 3];
        *reinterpret_cast<float4*>(out + x) = v;
      }
    } else {
      for (int x = lane; x < W; x += 32) out[x] = (1.f - fy) * t[x] + fy * b[x];
    }
  }
}

// The same maps on a cluster of four CTAs per frame (one conspicuity map each),
// exchanging the N(.) coefficients through distributed shared memory:
//   1. CTA r: N(.) statistics of orientation maps r, r + 4, ..; every CTA
//      receives every orientation map's affine form.
//   2. CTA 3: C_O = sum_theta N(B_theta) (same order and arithmetic as
//      k_consp) and its N(.) form; CTAs 0-2: the N(.) forms of I, RG, BY.
//   3. Every CTA: S = sum_k w_k N(C_k) over the whole map in shared memory (C_O
//      read from CTA 3), writing a quarter of N(C_k) and S out, and a quarter
//      of the up-sampling's candidate samples for the maximum; CTA 0 takes the
//      cluster's maximum.
// Per map the statistics are those of k_consp (the same sums in the same
// order while a map has at most 512 N(.) tiles), so the outputs match it.
#define CC_CTAS 4
#define CC_THREADS 512

__global__ void __cluster_dims__(CC_CTAS, 1, 1) __launch_bounds__(CC_THREADS) k_consp_cl(ConspArgs a) {
  seg_pdl_enter();
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank(), fb = blockIdx.x / CC_CTAS;
  if (SEG_SLOT_OFF(a.on, fb)) return;  // (every CTA of the cluster: one frame)
  extern __shared__ float dsm[];  // C_O (CTA 3), then S: n floats each
  __shared__ float ab[8];
  __shared__ float red[12 * 32];
  __shared__ unsigned tmax[4 * CONSP_TILES];
  __shared__ float abO[2 * SEG_MAX_ORIENT];  // every orientation map's N(.) form
  __shared__ float abC[8];                   // the four conspicuity maps' forms
  __shared__ unsigned smx;                   // (CTA 0) the cluster's maximum, float bits >= 0
  const int n = a.h * a.w, no = a.nch - 3;
  const float* acc = a.acc + (size_t)fb * a.nch * n;
  float* const csum_g = a.csum + (size_t)fb * n;
  float* const S_g = a.S + (size_t)fb * n;
  float* const consp = a.consp + (size_t)fb * 4 * n;
  float* const csum_s = dsm;
  float* const S_s = dsm + n;
  if (r == 0 && threadIdx.x == 0) smx = 0u;
  {  // 1. orientation maps r, r + 4, ..
    const float* v[4];
    int nm = 0;
    for (int m = r; m < no && nm < 4; m += CC_CTAS) v[nm++] = acc + (size_t)(3 + m) * n;
    if (nm > 0) block_norm_multi(v, nm, a.h, a.w, a.tile, a.flat, ab, red, tmax);
    if ((int)threadIdx.x < nm) {
      const int m = r + CC_CTAS * threadIdx.x;
      for (int q = 0; q < CC_CTAS; ++q) {
        float* d = cl.map_shared_rank(abO, q);
        d[2 * m] = ab[2 * threadIdx.x];
        d[2 * m + 1] = ab[2 * threadIdx.x + 1];
      }
    }
  }
  cl.sync();
  {  // 2. C_O on CTA 3; each CTA's conspicuity map's N(.) form
    const float* v[1];
    if (r == 3) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float c = 0.f;
        for (int m = 0; m < no; ++m) c += abO[2 * m] * acc[(size_t)(3 + m) * n + i] + abO[2 * m + 1];
        csum_s[i] = c;
        csum_g[i] = c;
      }
      __syncthreads();
      v[0] = csum_s;
    } else {
      v[0] = acc + (size_t)r * n;
    }
    block_norm_multi(v, 1, a.h, a.w, a.tile, a.flat, ab, red, tmax);
    if (threadIdx.x == 0)
      for (int q = 0; q < CC_CTAS; ++q) {
        float* d = cl.map_shared_rank(abC, q);
        d[2 * r] = ab[0];
        d[2 * r + 1] = ab[1];
      }
  }
  cl.sync();
  // 3. S over the whole map; this CTA's quarter of N(C_k) and S written out
  float wk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wk[k] = a.wdev ? (float)a.wdev[k] : a.wgt[k];
  const float* co = cl.map_shared_rank(csum_s, 3);
  const int q0 = (int)(((long long)n * r) / CC_CTAS), q1 = (int)(((long long)n * (r + 1)) / CC_CTAS);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float x[4] = {acc[i], acc[(size_t)n + i], acc[2 * (size_t)n + i], co[i]};
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float nv = abC[2 * k] * x[k] + abC[2 * k + 1];
      if (i >= q0 && i < q1) consp[(size_t)k * n + i] = nv;
      S += wk[k] * nv;
    }
    S_s[i] = S;
    if (i >= q0 && i < q1) S_g[i] = S;
  }
  // maximum of the bilinear up-sampling over its candidate samples (k_consp):
  // this CTA takes the candidate rows y with y mod 4 = r, against every
  // candidate column (the lists' order, set by atomics, does not matter)
  int* crow = (int*)tmax;
  int* ccol = crow + 2048;
  __shared__ int nr, nc;
  if (threadIdx.x == 0) nr = nc = 0;
  __syncthreads();
  for (int y = r + CC_CTAS * (int)threadIdx.x; y < a.H; y += CC_CTAS * blockDim.x)
    if (seg_up_candidate(y, a.h, a.H)) crow[atomicAdd(&nr, 1)] = y;
  for (int x = threadIdx.x; x < a.W; x += blockDim.x)
    if (seg_up_candidate(x, a.w, a.W)) ccol[atomicAdd(&nc, 1)] = x;
  __syncthreads();
  float mxv = 0.f;
  for (int k = threadIdx.x; k < nr * nc; k += blockDim.x)
    mxv = fmaxf(mxv, seg_bilinear_t(S_s, a.w, a.frow[crow[k / nc]], a.fcol[ccol[k % nc]]));
  mxv = seg_warp_max_f(mxv);
  if ((threadIdx.x & 31) == 0) atomicMax(cl.map_shared_rank(&smx, 0), __float_as_uint(mxv));
  cl.sync();
  if (r == 0 && threadIdx.x == 0) a.salmax[fb] = smx;
}

// ------------------------------------------------------------------ host side
static void make_taps(const seg_params& p, GaborTaps& t) {
  memset(&t, 0, sizeof(t));
  int R = p.gabor_radius;
  t.R = R;
  t.no = p.n_orient;
  double g[SEG_MAX_TAPS], sg = 0;
  for (int u = -R; u <= R; ++u) {
    g[u + R] = exp(-(double)(u * u) / (2.0 * p.gabor_sigma * p.gabor_sigma));
    sg += g[u + R];
  }
  double w = 2.0 * M_PI / p.gabor_lambda;
  for (int u = 0; u <= 2 * R; ++u) t.g0[u] = (float)(g[u] / sg);
  for (int k = 0; k < p.n_orient; ++k) {
    double th = k * M_PI / p.n_orient, cx = cos(th), sy = sin(th);
    double hr = 0, hi = 0, vr = 0, vi = 0;
    for (int u = -R; u <= R; ++u) {
      double a = g[u + R] / sg;
      double ar = a * cos(w * cx * u), ai = a * sin(w * cx * u);
      double br = a * cos(w * sy * u), bi = a * sin(w * sy * u);
      t.hx_re[k][u + R] = (float)ar;
      t.hx_im[k][u + R] = (float)ai;
      t.vy_re[k][u + R] = (float)br;
      t.vy_im[k][u + R] = (float)bi;
      hr += ar;
      hi += ai;
      vr += br;
      vi += bi;
    }
    t.kap_re[k] = (float)(hr * vr - hi * vi);
    t.kap_im[k] = (float)(hr * vi + hi * vr);
  }
}

int sal_layout(SalWS& s, int B, int H, int W, const seg_params& p, size_t* bytes, bool keep_complex) {
  memset(&s, 0, sizeof(s));
  s.B = B;
  s.H = H;
  s.W = W;
  s.L = p.levels;
  s.c_min = p.c_min;
  s.c_max = p.c_max;
  s.d_min = p.d_min;
  s.d_max = p.d_max;
  s.no = p.n_orient;
  s.s_max = p.c_max + p.d_max;
  s.sS = p.c_max;
  s.tile = p.norm_tile;
  s.flat = p.norm_flat;
  s.opp_sum = p.cs_opponent_sum;
  for (int k = 0; k < 4; ++k) s.w[k] = p.w[k];
  for (int l = 0; l < s.L; ++l) {
    s.hl[l] = seg_level_dim(H, l);
    s.wl[l] = seg_level_dim(W, l);
  }
  s.nch = 3 + s.no;
  s.npairs = 0;
  for (int c = s.c_min; c <= s.c_max; ++c)
    for (int d = s.d_min; d <= s.d_max; ++d) {
      if (s.npairs >= SEG_MAX_PAIRS) return SEG_EINVAL;
      s.pair_c[s.npairs] = c;
      s.pair_s[s.npairs] = c + d;
      s.npairs++;
    }
  s.nmaps = s.npairs * s.nch;
  if (s.d_max - s.d_min + 1 > ACC_MAX_PC) return SEG_EINVAL;
  s.nbands_total = 0;
  for (int i = 0; i < s.npairs; ++i) {
    int c = s.pair_c[i];
    if ((s.wl[c] + s.tile - 1) / s.tile > CS_MAX_TILES_X) return SEG_EINVAL;
    s.nbands_total += s.nch * ((s.hl[c] + s.tile - 1) / s.tile);
  }
  {
    int hS = s.hl[s.sS], wS = s.wl[s.sS];
    if (((hS + s.tile - 1) / s.tile) * ((wS + s.tile - 1) / s.tile) > CONSP_TILES) return SEG_EINVAL;
    if (2 * hS + 4 > 2048 || 2 * wS + 4 > 2048) return SEG_EINVAL;  // candidate rows / columns of the max
  }
  make_taps(p, s.taps);
  {
    // k_consp keeps the nch accumulators, C_O and S in shared memory when they fit
    const size_t need = sizeof(float) * (s.nch + 2) * (size_t)s.hl[s.sS] * s.wl[s.sS];
    const size_t cap = 160 * 1024;
    s.consp_staged = need <= cap && cudaFuncSetAttribute(k_consp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)cap) == cudaSuccess;
    s.consp_smem = s.consp_staged ? need : 0;
    // the cluster form: C_O and S (2 maps) in dynamic shared memory
    const size_t need_cl = sizeof(float) * 2 * (size_t)s.hl[s.sS] * s.wl[s.sS];
    s.consp_cl = s.nch - 3 <= SEG_MAX_ORIENT && need_cl <= cap &&
                 cudaFuncSetAttribute(k_consp_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) == cudaSuccess;
    s.consp_cl_smem = s.consp_cl ? need_cl : 0;
    cudaGetLastError();
  }
  // row-staged up-sampling: the most rows of S one band of UP_ROWS output rows touches
  {
    const int hS = s.hl[s.sS];
    int nr = 0;
    for (int y = 0; y < H; y += UP_ROWS) {
      const int yl = (y + UP_ROWS < H ? y + UP_ROWS : H) - 1;
      const int r = (seg_rs_entry(yl, hS, H).x >> 16) - (seg_rs_entry(y, hS, H).x & 0xffff) + 1;
      nr = r > nr ? r : nr;
    }
    s.up_smem = sizeof(float) * (size_t)nr * W;
    if (s.up_smem > 160 * 1024 ||
        cudaFuncSetAttribute(k_upsample_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.up_smem) != cudaSuccess)
      s.up_smem = 0;
    cudaGetLastError();
  }
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += seg_align(b);
    return o;
  };
  // record offsets in the pointer fields (bound later); every per-frame buffer
  // holds B frames back to back
  const size_t Bz = (size_t)B;
  for (int ch = 0; ch < 3; ++ch)
    for (int l = 1; l < s.L; ++l) s.pyr[ch][l] = (float*)take(Bz * sizeof(float) * s.hl[l] * s.wl[l]);
  for (int k = 0; k < s.no; ++k)
    for (int l = s.c_min; l <= s.s_max; ++l)
      s.ori[k][l] = (float*)take(Bz * sizeof(float) * s.hl[l] * s.wl[l]);
  if (keep_complex)
    for (int k = 0; k < s.no; ++k)
      for (int l = s.c_min; l <= s.s_max; ++l)
        s.oc[k][l] = (float2*)take(Bz * sizeof(float2) * s.hl[l] * s.wl[l]);
  s.mm = (unsigned*)take(Bz * sizeof(unsigned) * 2 * s.nmaps);
  s.tpart = (float*)take(Bz * sizeof(float) * s.nbands_total);
  size_t big = (size_t)s.hl[s.c_min] * s.wl[s.c_min] * s.nch;
  s.acc[0] = (float*)take(Bz * sizeof(float) * big);
  s.acc[1] = (float*)take(Bz * sizeof(float) * big);
  size_t nS = (size_t)s.hl[s.sS] * s.wl[s.sS];
  s.consp = (float*)take(Bz * sizeof(float) * 4 * nS);
  s.csum = (float*)take(Bz * sizeof(float) * nS);
  s.S = (float*)take(Bz * sizeof(float) * nS);
  s.salmax = (unsigned*)take(Bz * sizeof(unsigned));
  s.smax = (int*)take(Bz * sizeof(int));
  int nrs = 0;
  for (int i = 0; i < s.npairs; ++i) {
    s.rs_row[i] = nrs;
    nrs += s.hl[s.pair_c[i]];
    s.rs_col[i] = nrs;
    nrs += s.wl[s.pair_c[i]];
  }
  s.rs_frow = nrs;
  nrs += H;
  s.rs_fcol = nrs;
  nrs += W;
  s.rs_n = nrs;
  s.rs = (int2*)take(sizeof(int2) * nrs);
  *bytes = off;
  return SEG_OK;
}

void sal_bind(SalWS& s, char* base) {
  auto fix = [&](auto*& ptr) {
    using T = std::remove_reference_t<decltype(ptr)>;
    ptr = (T)(base + (size_t)ptr);
  };
  for (int ch = 0; ch < 3; ++ch)
    for (int l = 1; l < s.L; ++l) fix(s.pyr[ch][l]);
  for (int k = 0; k < s.no; ++k)
    for (int l = s.c_min; l <= s.s_max; ++l) {
      fix(s.ori[k][l]);
      if (s.oc[k][l]) fix(s.oc[k][l]);
    }
  fix(s.mm);
  fix(s.tpart);
  fix(s.acc[0]);
  fix(s.acc[1]);
  s.acc_final = s.acc[(s.c_max - s.c_min) & 1];
  fix(s.consp);
  fix(s.csum);
  fix(s.S);
  fix(s.salmax);
  fix(s.smax);
  fix(s.rs);
}

int sal_upload_tables(const SalWS& s) {
  int2* t = (int2*)malloc(sizeof(int2) * s.rs_n);
  if (!t) return SEG_ENOMEM;
  for (int i = 0; i < s.npairs; ++i) {
    int c = s.pair_c[i], sv = s.pair_s[i];
    for (int y = 0; y < s.hl[c]; ++y) t[s.rs_row[i] + y] = seg_rs_entry(y, s.hl[sv], s.hl[c]);
    for (int x = 0; x < s.wl[c]; ++x) t[s.rs_col[i] + x] = seg_rs_entry(x, s.wl[sv], s.wl[c]);
  }
  int hS = s.hl[s.sS], wS = s.wl[s.sS];
  for (int y = 0; y < s.H; ++y) t[s.rs_frow + y] = seg_rs_entry(y, hS, s.H);
  for (int x = 0; x < s.W; ++x) t[s.rs_fcol + x] = seg_rs_entry(x, wS, s.W);
  cudaError_t e = cudaMemcpy(s.rs, t, sizeof(int2) * s.rs_n, cudaMemcpyHostToDevice);
  free(t);
  return e == cudaSuccess ? SEG_OK : SEG_ECUDA;
}

static void fill_cs_args(const SalWS& s, CSArgs& a) {
  memset(&a, 0, sizeof(a));
  for (int l = 0; l < s.L; ++l) {
    a.hl[l] = s.hl[l];
    a.wl[l] = s.wl[l];
    for (int ch = 0; ch < 3; ++ch) a.X[ch][l] = l >= 1 ? s.pyr[ch][l] : nullptr;
    for (int k = 0; k < s.no; ++k) a.X[3 + k][l] = (l >= s.c_min && l <= s.s_max) ? s.ori[k][l] : nullptr;
  }
  a.npairs = s.npairs;
  a.nch = s.nch;
  a.tile = s.tile;
  a.opp_sum = s.opp_sum;
  a.nbands_total = s.nbands_total;
  int off = 0;
  for (int i = 0; i < s.npairs; ++i) {
    a.pair_c[i] = s.pair_c[i];
    a.pair_s[i] = s.pair_s[i];
    a.pair_band_off[i] = off;
    off += s.nch * ((s.hl[s.pair_c[i]] + s.tile - 1) / s.tile);
  }
  a.pair_band_off[s.npairs] = off;
  a.mm = s.mm;
  a.tpart = s.tpart;
  a.flat = s.flat;
  a.c_lo = s.c_min;
  a.c_hi = s.c_max;
  a.rs = s.rs;
  for (int i = 0; i < s.npairs; ++i) {
    a.rs_row[i] = s.rs_row[i];
    a.rs_col[i] = s.rs_col[i];
  }
  a.on = s.on;
  // the staged center-surround layout: widest surround and center levels of the pairs
  a.sm_ws = a.sm_wc = 0;
  for (int i = 0; i < s.npairs; ++i) {
    a.sm_ws = max(a.sm_ws, s.wl[s.pair_s[i]]);
    a.sm_wc = max(a.sm_wc, s.wl[s.pair_c[i]]);
  }
  if (cs_stage_bytes(s.nch, a.sm_ws, a.sm_wc) > 48 * 1024)
    a.sm_ws = a.sm_wc = 0;  // (reads from global memory instead)
}

// dynamic shared memory of the center-surround kernels for nf channels per CTA
static size_t cs_stats_smem(const CSArgs& a, int nf) { return a.sm_ws ? cs_stage_bytes(nf, a.sm_ws, a.sm_wc) : 0; }

int sal_launch(seg_ctx* c, const uint8_t* rgb, float* sal_out, bool upsample) {
  // under graph capture the frame's k_set_io has zeroed the frame maxima
  return sal_run(c->sal, c->stream, rgb, false, c->io_mode ? c->io : nullptr, nullptr, sal_out, upsample,
                 c->io_mode != 0);
}

int sal_run(SalWS& s, cudaStream_t st, const void* rgb, bool rgb_f32, const SegIO* io, const double* wdev,
            float* sal_out, bool upsample, bool smax_zeroed) {
  const int H = s.H, W = s.W, N = H * W, B = s.B;
  if (!smax_zeroed) SEG_CUDA_TRY(cudaMemsetAsync(s.smax, 0, B * sizeof(int), st));
  int nb = min((N + 255) / 256, B > 1 ? 148 : 148 * 8);
  nb = max(nb, (s.nmaps + 255) / 256);
  // RGB8 frames go 16 pixels per thread (three 16-byte loads): a grid for that,
  // not one thread per pixel (idle CTAs would crowd the concurrent back half)
  const int nb8 = max((N / 16 + 255) / 256, (s.nmaps + 255) / 256);
  dim3 g1((s.wl[1] + RED_TX - 1) / RED_TX, (s.hl[1] + RED_TY - 1) / RED_TY, B);
  // widths that are a multiple of 16: 16-pixel runs; the shorter tile while a
  // batch of the taller one would not give two CTAs per SM
  const bool fv = (W & 15) == 0;
  const int fvx = (s.wl[1] + FV_TX - 1) / FV_TX;
  const bool fv8 = (long long)fvx * ((s.hl[1] + 15) / 16) * B < 2 * 148;
  const dim3 gv(fvx, fv8 ? (s.hl[1] + 7) / 8 : (s.hl[1] + 15) / 16, B);
  float *l1i = s.pyr[0][1], *l1rg = s.pyr[1][1], *l1by = s.pyr[2][1];
  const int h1 = s.hl[1], w1 = s.wl[1];
  if (rgb_f32) {
    const float* f = (const float*)rgb;
    SEG_CUDA_TRY(seg_launch(k_rgb_max<float>, dim3(nb, B), 256, 0, st, f, N, s.smax, s.mm, s.nmaps, nullptr, s.on));
    if (!fv)
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1<float>, g1, 256, 0, st, f, H, W, s.smax, l1i, l1rg, l1by, h1, w1,
                              nullptr, s.on));
    else if (fv8)
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1_v<float, 8>, gv, fv_threads<8>(), 0, st, f, H, W, s.smax, l1i, l1rg,
                              l1by, h1, w1, nullptr, s.on));
    else
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1_v<float, 16>, gv, fv_threads<16>(), 0, st, f, H, W, s.smax, l1i, l1rg,
                              l1by, h1, w1, nullptr, s.on));
  } else {
    const uint8_t* u = (const uint8_t*)rgb;
    SEG_CUDA_TRY(seg_launch(k_rgb_max<uint8_t>, dim3(nb8, B), 256, 0, st, u, N, s.smax, s.mm, s.nmaps, io, s.on));
    if (!fv)
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1<uint8_t>, g1, 256, 0, st, u, H, W, s.smax, l1i, l1rg, l1by, h1, w1, io,
                              s.on));
    else if (fv8)
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1_v<uint8_t, 8>, gv, fv_threads<8>(), 0, st, u, H, W, s.smax, l1i, l1rg,
                              l1by, h1, w1, io, s.on));
    else
      SEG_CUDA_TRY(seg_launch(k_feat_reduce1_v<uint8_t, 16>, gv, fv_threads<16>(), 0, st, u, H, W, s.smax, l1i, l1rg,
                              l1by, h1, w1, io, s.on));
  }
  // tiled launches while the produced level is large; one tail launch for the rest
  int tail_from = s.L - 1;
  for (int l = 1; l + 1 < s.L; ++l)
    if ((long long)s.hl[l + 1] * s.wl[l + 1] <= 2048) {
      tail_from = l;
      break;
    }
  for (int l = 1; l + 1 < s.L && l < tail_from; ++l) {
    Reduce3Args ra;
    for (int ch = 0; ch < 3; ++ch) {
      ra.in[ch] = s.pyr[ch][l];
      ra.out[ch] = s.pyr[ch][l + 1];
    }
    ra.h = s.hl[l];
    ra.w = s.wl[l];
    ra.h2 = s.hl[l + 1];
    ra.w2 = s.wl[l + 1];
    ra.on = s.on;
    dim3 g((ra.w2 + RED_TX - 1) / RED_TX, (ra.h2 + RED_TY - 1) / RED_TY, 3 * B);
    SEG_CUDA_TRY(seg_launch(k_reduce3, g, 256, 0, st, ra));
  }
  if (tail_from < s.L - 1) {
    PyrTailArgs ta;
    memset(&ta, 0, sizeof(ta));
    for (int l = 1; l < s.L; ++l) {
      for (int ch = 0; ch < 3; ++ch) ta.lvl[ch][l] = s.pyr[ch][l];
      ta.hl[l] = s.hl[l];
      ta.wl[l] = s.wl[l];
    }
    ta.from = tail_from;
    ta.to = s.L - 1;
    ta.on = s.on;
    SEG_CUDA_TRY(seg_launch(k_pyr_tail, 3 * B, 1024, 0, st, ta));
  }
  GaborArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.lvl_first = s.c_min;
  ga.lvl_last = s.s_max;
  ga.on = s.on;
  int tot = 0;
  for (int l = s.c_min; l <= s.s_max; ++l) {
    ga.in[l] = s.pyr[0][l];
    ga.hl[l] = s.hl[l];
    ga.wl[l] = s.wl[l];
    for (int k = 0; k < s.no; ++k) {
      ga.out[k][l] = s.ori[k][l];
      ga.out_c[k][l] = s.oc[k][l];
    }
    ga.blk_off[l - s.c_min] = tot;
    tot += ((s.wl[l] + GB_TX - 1) / GB_TX) * ((s.hl[l] + GB_TY - 1) / GB_TY);
  }
  ga.blk_off[s.s_max - s.c_min + 1] = tot;
  const dim3 gg(tot, B, B == 1 ? gb_ngroups(s.no) : 1);
  if (s.taps.R == 6)
    SEG_CUDA_TRY(seg_launch(k_gabor<6>, gg, 256, 0, st, ga, s.taps));
  else
    SEG_CUDA_TRY(seg_launch(k_gabor<0>, gg, 256, 0, st, ga, s.taps));
  CSArgs ca;
  fill_cs_args(s, ca);
  {
    // one channel per CTA for a single frame (more CTAs), all channels of a pair
    // per CTA for a batch (shared resampling coordinates, fewer CTAs)
    const bool per_ch = B == 1;
    const dim3 g((s.nbands_total / s.nch) * (per_ch ? s.nch : 1), B);
    switch (s.nch) {
#define SEG_CS_STATS(n)                                 \
  case n:                                               \
    if (per_ch)                                         \
      SEG_CUDA_TRY(seg_launch(k_cs_stats<n, 1>, g, 256, cs_stats_smem(ca, 1), st, ca));          \
    else                                                \
      SEG_CUDA_TRY(seg_launch(k_cs_stats<n, n>, g, 256, cs_stats_smem(ca, n), st, ca));          \
    break;
      SEG_CS_STATS(4) SEG_CS_STATS(5) SEG_CS_STATS(6) SEG_CS_STATS(7)
      SEG_CS_STATS(8) SEG_CS_STATS(9) SEG_CS_STATS(10) SEG_CS_STATS(11)
#undef SEG_CS_STATS
      default:
        return SEG_EINVAL;
    }
  }
  int cur = 0;
  const float* prev = nullptr;
  int hp = 0, wp = 0;
  const bool fused = s.c_max - s.c_min <= 2 && B <= 4;
  if (fused) {
    // one launch: every tile of sigma_S rebuilds its halo regions of the lower scales
    // (for larger batches the level-by-level launches have enough CTAs and no halo work)
    const dim3 g((s.wl[s.sS] + FA_TX - 1) / FA_TX, (s.hl[s.sS] + FA_TY - 1) / FA_TY, s.nch * B);
    // CTA size: 1024 threads finish a frame's sum soonest; a pipelined context
    // takes 256 (fewer registers and threads held per SM, so the previous frame's
    // back half, running meanwhile, is crowded less: pipelined 640x480 ~6.13k
    // -> ~6.31k frames/s, the sum itself ~7 us slower)
    if (s.light_ctas)
      SEG_CUDA_TRY(seg_launch(k_cs_accum_fused<256>, g, 256, 0, st, ca, s.acc_final));
    else
      SEG_CUDA_TRY(seg_launch(k_cs_accum_fused<1024>, g, 1024, 0, st, ca, s.acc_final));
    prev = s.acc_final;
  }
  for (int cc = s.c_min; cc <= s.c_max && !fused; ++cc) {
    const bool per_ch = B == 1;
    dim3 g((s.wl[cc] + ACC_TX - 1) / ACC_TX, (s.hl[cc] + ACC_TY - 1) / ACC_TY, B * (per_ch ? s.nch : 1));
    switch (s.nch) {
#define SEG_CS_ACC(n)                                                          \
  case n:                                                                      \
    if (per_ch)                                                                \
      SEG_CUDA_TRY(seg_launch(k_cs_accum<n, 1>, g, 256, 0, st, ca, cc, prev, hp, wp, s.acc[cur]));   \
    else                                                                       \
      SEG_CUDA_TRY(seg_launch(k_cs_accum<n, n>, g, 256, 0, st, ca, cc, prev, hp, wp, s.acc[cur]));   \
    break;
      SEG_CS_ACC(4) SEG_CS_ACC(5) SEG_CS_ACC(6) SEG_CS_ACC(7)
      SEG_CS_ACC(8) SEG_CS_ACC(9) SEG_CS_ACC(10) SEG_CS_ACC(11)
#undef SEG_CS_ACC
      default:
        return SEG_EINVAL;
    }
    prev = s.acc[cur];
    hp = s.hl[cc];
    wp = s.wl[cc];
    cur ^= 1;
  }
  ConspArgs pa;
  pa.acc = prev;
  pa.h = s.hl[s.sS];
  pa.w = s.wl[s.sS];
  pa.nch = s.nch;
  pa.tile = s.tile;
  pa.flat = s.flat;
  for (int k = 0; k < 4; ++k) pa.wgt[k] = s.w[k];
  pa.wdev = wdev;
  pa.csum = s.csum;
  pa.consp = s.consp;
  pa.S = s.S;
  pa.H = H;
  pa.W = W;
  pa.salmax = s.salmax;
  pa.frow = s.rs + s.rs_frow;
  pa.fcol = s.rs + s.rs_fcol;
  pa.on = s.on;
  if (s.consp_cl)
    SEG_CUDA_TRY(seg_launch(k_consp_cl, CC_CTAS * B, CC_THREADS, s.consp_cl_smem, st, pa));
  else if (s.consp_staged)
    SEG_CUDA_TRY(seg_launch(k_consp<true>, B, 1024, s.consp_smem, st, pa));
  else
    SEG_CUDA_TRY(seg_launch(k_consp<false>, B, 1024, 0, st, pa));
  if (upsample && s.up_smem) {
    const dim3 gu((H + UP_ROWS - 1) / UP_ROWS, B);
    SEG_CUDA_TRY(seg_launch(k_upsample_rows, gu, 256, s.up_smem, st, s.S, s.hl[s.sS], s.wl[s.sS], H, W, sal_out, io,
                            s.rs + s.rs_frow, s.rs + s.rs_fcol, s.on));
  } else if (upsample) {
    dim3 gu((W + 255) / 256, (H + 3) / 4, B);  // 4 pixels per thread
    SEG_CUDA_TRY(seg_launch(k_upsample, gu, 256, 0, st, s.S, s.hl[s.sS], s.wl[s.sS], H, W, sal_out, io, s.rs + s.rs_frow,
                                   s.rs + s.rs_fcol, s.on));
  }
  SEG_CUDA_TRY(cudaGetLastError());
  return SEG_OK;
}
