/*
 * oracle.c -- plain, slow FP64 CPU reference ("the oracle") for the per-frame
 * path of Akamine et al., "Fully automatic extraction of salient objects from
 * videos in near real-time" (arXiv:1008.0502).
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load or run it.  It shares no code with the
 * CUDA path.  Every function follows one step of the method in the order the
 * paper (and, where the paper defers to it, the Itti-Koch saliency model it
 * cites in Sec. 3) states it, with no blocking, fusion or reordering: direct
 * 2-D convolutions, one map at a time, two-pass moments, textbook max-flow.
 *
 * Where the paper is silent, garbled or self-contradictory the reading taken
 * is named in the comment ("Reading: ...").
 *
 * Parity status: every function below is pinned by tests against closed
 * forms, invariants, library routines or brute force.  The composition of
 * the saliency map from its pyramids (orc_saliency_compose) is pinned on
 * hand-built pyramids whose conspicuity maps and S follow in closed form
 * (single and double peaks, two center scales, per-orientation N(.), the
 * source of each surround); the paper prints no worked example.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static double maxd(double a, double b) { return a > b ? a : b; }
static double mind(double a, double b) { return a < b ? a : b; }

int orc_level_dim(int n, int level) {
  /* Each pyramid level keeps the even samples: size ceil(n / 2). */
  for (int l = 0; l < level; ++l) n = (n + 1) / 2;
  return n;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3 / Sec. 7.2 step 1: fundamental features (intensity, colour opponents).
 * Reading (Itti-Koch model cited in Sec. 3): I = (r+g+b)/765; hue is
 * normalised only where the intensity exceeds a tenth of the frame maximum,
 * decided exactly on integers: 10*(r+g+b) > max(r+g+b).  There rn = 3r/(r+g+b)
 * (and gn, bn likewise), elsewhere 0; broadly tuned channels
 *   R = rn-(gn+bn)/2, G = gn-(rn+bn)/2, B = bn-(rn+gn)/2,
 *   Y = (rn+gn)/2 - |rn-gn|/2 - bn, each clamped at 0;
 * opponents RG = R-G, BY = B-Y. */
void orc_features(int H, int W, const uint8_t* rgb, double* I, double* RG, double* BY) {
  int n = H * W;
  int smax = 0;
  for (int i = 0; i < n; ++i) {
    int s = rgb[3 * i] + rgb[3 * i + 1] + rgb[3 * i + 2];
    if (s > smax) smax = s;
  }
  for (int i = 0; i < n; ++i) {
    int r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
    int s = r + g + b;
    I[i] = s / 765.0;
    double rn = 0, gn = 0, bn = 0;
    if (10 * s > smax) {
      rn = 3.0 * r / s;
      gn = 3.0 * g / s;
      bn = 3.0 * b / s;
    }
    double R = maxd(0.0, rn - (gn + bn) / 2.0);
    double G = maxd(0.0, gn - (rn + bn) / 2.0);
    double B = maxd(0.0, bn - (rn + gn) / 2.0);
    double Y = maxd(0.0, (rn + gn) / 2.0 - fabs(rn - gn) / 2.0 - bn);
    RG[i] = R - G;
    BY[i] = B - Y;
  }
}

/* Sec. 7.2 step 2: Gaussian pyramid.  One REDUCE step = 5x5 binomial
 * [1 4 6 4 1]^T [1 4 6 4 1] / 256 with clamp-to-edge borders, then keep the
 * even samples.  Written as the direct 2-D convolution.
 * Reading: the paper's filter listing pads with zeros and skips row/column 0
 * (an off-by-one); clamp-to-edge is used instead. */
void orc_reduce(int h, int w, const double* in, double* out) {
  static const double k[5] = {1.0, 4.0, 6.0, 4.0, 1.0};
  int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
  for (int y = 0; y < h2; ++y)
    for (int x = 0; x < w2; ++x) {
      double acc = 0.0;
      for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) {
          int yy = clampi(2 * y + j, 0, h - 1), xx = clampi(2 * x + i, 0, w - 1);
          acc += k[j + 2] * k[i + 2] / 256.0 * in[yy * w + xx];
        }
      out[y * w2 + x] = acc;
    }
}

/* Sec. 3 / Sec. 7.2: edge-orientation feature.
 * Reading: complex Gabor with an isotropic Gaussian envelope
 *   G(u,v) = exp(-(u^2+v^2) / (2 sigma^2)),  |u|,|v| <= radius,
 *   carrier exp(i 2 pi (u cos theta + v sin theta) / lambda),
 * made exactly zero-mean on its support by subtracting kappa*G with
 * kappa = sum(G e^{i phase}) / sum(G), and scaled by 1/sum(G).
 * u runs along x (columns), v along y (rows).  Layout k[(v+R)*(2R+1) + (u+R)]. */
void orc_gabor_kernel(double theta, double lambda, double sigma, int radius, double* kre,
                      double* kim) {
  int n = 2 * radius + 1;
  double sg = 0, kr = 0, ki = 0;
  for (int v = -radius; v <= radius; ++v)
    for (int u = -radius; u <= radius; ++u) {
      double g = exp(-(u * u + v * v) / (2.0 * sigma * sigma));
      double ph = 2.0 * M_PI * (u * cos(theta) + v * sin(theta)) / lambda;
      sg += g;
      kr += g * cos(ph);
      ki += g * sin(ph);
    }
  kr /= sg;
  ki /= sg;
  for (int v = -radius; v <= radius; ++v)
    for (int u = -radius; u <= radius; ++u) {
      double g = exp(-(u * u + v * v) / (2.0 * sigma * sigma));
      double ph = 2.0 * M_PI * (u * cos(theta) + v * sin(theta)) / lambda;
      kre[(v + radius) * n + (u + radius)] = g * (cos(ph) - kr) / sg;
      kim[(v + radius) * n + (u + radius)] = g * (sin(ph) - ki) / sg;
    }
}

/* O = | sum_{u,v} k(u,v) * in(x+u, y+v) |, clamp-to-edge. */
void orc_gabor(int h, int w, const double* in, const double* kre, const double* kim, int radius,
               double* out) {
  int n = 2 * radius + 1;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      double re = 0, im = 0;
      for (int v = -radius; v <= radius; ++v)
        for (int u = -radius; u <= radius; ++u) {
          double p = in[clampi(y + v, 0, h - 1) * w + clampi(x + u, 0, w - 1)];
          re += kre[(v + radius) * n + (u + radius)] * p;
          im += kim[(v + radius) * n + (u + radius)] * p;
        }
      out[y * w + x] = sqrt(re * re + im * im);
    }
}

/* Across-scale interpolation used by the center-surround difference and the
 * final saliency map.  Reading: bilinear with half-pixel centres,
 * src = (dst + 0.5) * n_src / n_dst - 0.5, clamped to [0, n_src - 1]. */
void orc_upsample(int hs, int ws, const double* src, int hd, int wd, double* dst) {
  for (int y = 0; y < hd; ++y) {
    double sy = mind(maxd((y + 0.5) * hs / (double)hd - 0.5, 0.0), hs - 1.0);
    int y0 = (int)floor(sy);
    int y1 = y0 + 1 < hs ? y0 + 1 : hs - 1;
    double fy = sy - y0;
    for (int x = 0; x < wd; ++x) {
      double sx = mind(maxd((x + 0.5) * ws / (double)wd - 0.5, 0.0), ws - 1.0);
      int x0 = (int)floor(sx);
      int x1 = x0 + 1 < ws ? x0 + 1 : ws - 1;
      double fx = sx - x0;
      double top = (1 - fx) * src[y0 * ws + x0] + fx * src[y0 * ws + x1];
      double bot = (1 - fx) * src[y1 * ws + x0] + fx * src[y1 * ws + x1];
      dst[y * wd + x] = (1 - fy) * top + fy * bot;
    }
  }
}

/* Sec. 7.2 step 3: the normalisation N(.) "using global and local extrema".
 * Reading: rescale by the global range to [0, 1] (M = 1); the local maxima are
 * the maxima of fixed tile x tile blocks (partial edge blocks included, as the
 * block-wise min/max search of Sec. 7.2 produces); mbar = mean of those block
 * maxima without one copy of the global maximum; N(v) = v' * (1 - mbar)^2.
 * A map whose range is <= flat is treated as constant: N = 0. */
void orc_normalize(int h, int w, const double* v, int tile, double flat, double* out) {
  int n = h * w;
  double mn = DBL_MAX, mx = -DBL_MAX;
  for (int i = 0; i < n; ++i) {
    mn = mind(mn, v[i]);
    mx = maxd(mx, v[i]);
  }
  if (!(mx - mn > flat)) {
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    return;
  }
  for (int i = 0; i < n; ++i) out[i] = (v[i] - mn) / (mx - mn);
  int nty = (h + tile - 1) / tile, ntx = (w + tile - 1) / tile;
  double sum = 0.0;
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx) {
      double m = 0.0;
      for (int y = ty * tile; y < h && y < (ty + 1) * tile; ++y)
        for (int x = tx * tile; x < w && x < (tx + 1) * tile; ++x) m = maxd(m, out[y * w + x]);
      sum += m;
    }
  int nt = nty * ntx;
  double mbar = nt > 1 ? (sum - 1.0) / (nt - 1) : 0.0;
  double f = (1.0 - mbar) * (1.0 - mbar);
  for (int i = 0; i < n; ++i) out[i] *= f;
}

/* Sec. 3 / Sec. 7.2 steps 4-6, the composition of the saliency map from its
 * feature pyramids (the Itti-Koch model cited in Sec. 3; Sec. 7.2 calls the
 * last step "weighted addition" of normalised maps):
 *   4. center-surround maps at scale c for every (c, s = c + d):
 *      |X(c) - up X(s)| for I and for each O(theta) (the surround of O(theta)
 *      is O(s, theta)); |X(c) + up X(s)| for RG and BY (Itti's (R-G)(c)
 *      minus (G-R)(s));
 *   5. N(.) of every center-surround map;
 *   6. REDUCE every normalised map down to sigma_S = c_max and add per
 *      channel: C_I, C_RG, C_BY; the orientation conspicuity is
 *      C_O = sum_theta N(sum_{c,s} N(O(c, s, theta)));
 *      S = sum_k w_k N(C_k) over k = I, RG, BY, O.
 * Inputs use the layout of orc_saliency_debug: pyr holds the three channels'
 * levels 0..levels-1 back to back, ori holds n_orient blocks of the levels
 * c_min..c_max+d_max; level l of an H x W frame is orc_level_dim(H, l) x
 * orc_level_dim(W, l).  Outputs: consp (4 maps N(C_k) at sigma_S, may be
 * NULL) and S (the map at sigma_S). */
void orc_saliency_compose(const orc_params* P, int H, int W, const double* pyr, const double* ori,
                          double* consp, double* S) {
  int L = P->levels, s_max = P->c_max + P->d_max, no = P->n_orient;
  int hl[64], wl[64];
  for (int l = 0; l < L; ++l) {
    hl[l] = orc_level_dim(H, l);
    wl[l] = orc_level_dim(W, l);
  }
  const double* X[3][64];
  const double* Ot[16][64];
  size_t off = 0;
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < L; ++l) {
      X[c][l] = pyr + off;
      off += (size_t)hl[l] * wl[l];
    }
  off = 0;
  for (int k = 0; k < no; ++k)
    for (int l = P->c_min; l <= s_max; ++l) {
      Ot[k][l] = ori + off;
      off += (size_t)hl[l] * wl[l];
    }

  int sS = P->c_max;
  int hS = hl[sS], wS = wl[sS], nS = hS * wS;
  int nacc = 3 + no;
  double* acc = (double*)calloc((size_t)nacc * nS, sizeof(double));
  int big = hl[P->c_min] * wl[P->c_min];
  double* up = (double*)malloc(sizeof(double) * big);
  double* map = (double*)malloc(sizeof(double) * big);
  double* nm = (double*)malloc(sizeof(double) * big);
  double* tmp = (double*)malloc(sizeof(double) * big);
  for (int c = P->c_min; c <= P->c_max; ++c)
    for (int d = P->d_min; d <= P->d_max; ++d) {
      int s = c + d;
      int nc = hl[c] * wl[c];
      for (int f = 0; f < nacc; ++f) {
        const double* cen = f < 3 ? X[f][c] : Ot[f - 3][c];
        const double* sur = f < 3 ? X[f][s] : Ot[f - 3][s];
        orc_upsample(hl[s], wl[s], sur, hl[c], wl[c], up);
        int opp = (f == 1 || f == 2) && P->cs_opponent_sum;
        for (int i = 0; i < nc; ++i) map[i] = fabs(opp ? cen[i] + up[i] : cen[i] - up[i]);
        orc_normalize(hl[c], wl[c], map, P->norm_tile, P->norm_flat, nm);
        for (int l = c; l < sS; ++l) {
          orc_reduce(hl[l], wl[l], nm, tmp);
          memcpy(nm, tmp, sizeof(double) * hl[l + 1] * wl[l + 1]);
        }
        for (int i = 0; i < nS; ++i) acc[(size_t)f * nS + i] += nm[i];
      }
    }
  double* C[4];
  for (int k = 0; k < 4; ++k) C[k] = (double*)calloc(nS, sizeof(double));
  memcpy(C[0], acc, sizeof(double) * nS);
  memcpy(C[1], acc + nS, sizeof(double) * nS);
  memcpy(C[2], acc + 2 * (size_t)nS, sizeof(double) * nS);
  for (int k = 0; k < no; ++k) {
    orc_normalize(hS, wS, acc + (size_t)(3 + k) * nS, P->norm_tile, P->norm_flat, tmp);
    for (int i = 0; i < nS; ++i) C[3][i] += tmp[i];
  }
  for (int i = 0; i < nS; ++i) S[i] = 0.0;
  for (int k = 0; k < 4; ++k) {
    orc_normalize(hS, wS, C[k], P->norm_tile, P->norm_flat, tmp);
    if (consp) memcpy(consp + (size_t)k * nS, tmp, sizeof(double) * nS);
    for (int i = 0; i < nS; ++i) S[i] += P->w[k] * tmp[i];
  }
  for (int k = 0; k < 4; ++k) free(C[k]);
  free(acc);
  free(up);
  free(map);
  free(nm);
  free(tmp);
}

/* Sec. 3 / Sec. 7.2: the saliency map.
 *   1. features at level 0; 2. pyramids of I, RG, BY; 3. Gabor orientation
 *   maps O(sigma, theta) on the intensity pyramid, sigma in [c_min, c_max +
 *   d_max]; 4-6. the composition above (center-surround, N(.), weighted
 *   addition) gives S at sigma_S; the saliency map is S upsampled to the
 *   frame size. */
void orc_saliency_ex(const orc_params* P, int H, int W, const uint8_t* rgb, double* saliency,
                     orc_saliency_debug* dbg) {
  int L = P->levels, s_max = P->c_max + P->d_max, no = P->n_orient;
  int hl[64], wl[64];
  size_t lev_off[65], ori_area = 0;
  lev_off[0] = 0;
  for (int l = 0; l < L; ++l) {
    hl[l] = orc_level_dim(H, l);
    wl[l] = orc_level_dim(W, l);
    lev_off[l + 1] = lev_off[l] + (size_t)hl[l] * wl[l];
    if (l >= P->c_min && l <= s_max) ori_area += (size_t)hl[l] * wl[l];
  }
  size_t pyr_area = lev_off[L];
  /* pyr: channel c, level l at c * pyr_area + lev_off[l] */
  double* pyr = (double*)malloc(sizeof(double) * 3 * pyr_area);
  orc_features(H, W, rgb, pyr, pyr + pyr_area, pyr + 2 * pyr_area);
  for (int c = 0; c < 3; ++c)
    for (int l = 1; l < L; ++l)
      orc_reduce(hl[l - 1], wl[l - 1], pyr + c * pyr_area + lev_off[l - 1], pyr + c * pyr_area + lev_off[l]);

  /* ori: orientation k, level l at k * ori_area + (lev_off[l] - lev_off[c_min]) */
  int R = P->gabor_radius, kn = 2 * R + 1;
  double* ori = (double*)malloc(sizeof(double) * (no > 0 ? no : 1) * (ori_area > 0 ? ori_area : 1));
  double* kre = (double*)malloc(sizeof(double) * kn * kn);
  double* kim = (double*)malloc(sizeof(double) * kn * kn);
  for (int k = 0; k < no; ++k) {
    orc_gabor_kernel(k * M_PI / no, P->gabor_lambda, P->gabor_sigma, R, kre, kim);
    for (int l = P->c_min; l <= s_max; ++l)
      orc_gabor(hl[l], wl[l], pyr + lev_off[l], kre, kim, R,
                ori + k * ori_area + (lev_off[l] - lev_off[P->c_min]));
  }
  free(kre);
  free(kim);

  int nS = hl[P->c_max] * wl[P->c_max];
  double* S = (double*)malloc(sizeof(double) * nS);
  orc_saliency_compose(P, H, W, pyr, ori, dbg ? dbg->consp : NULL, S);
  if (dbg && dbg->S) memcpy(dbg->S, S, sizeof(double) * nS);
  orc_upsample(hl[P->c_max], wl[P->c_max], S, H, W, saliency);

  if (dbg && dbg->pyr) memcpy(dbg->pyr, pyr, sizeof(double) * 3 * pyr_area);
  if (dbg && dbg->ori) memcpy(dbg->ori, ori, sizeof(double) * no * ori_area);
  free(pyr);
  free(ori);
  free(S);
}

void orc_saliency(const orc_params* P, int H, int W, const uint8_t* rgb, double* saliency) {
  orc_saliency_ex(P, H, W, rgb, saliency, NULL);
}

/* ------------------------------------------------------------------------ */
/* Sec. 6: sequential prior update (the two equations of Sec. 6, as printed).
 * a = sigma1^2, b = sigma2^2, P = sigma^2_xi1(t-1):
 *   weight on f:  w_f = a / (a + b + P)
 *   P_t = a (b + P) / (a + b + P).
 * Reading: at t = 0 there is no previous segmentation; P_{-1} = +inf, whose
 * limit gives w_f = 0 and P_0 = a. */
double orc_kalman_step(int t, double P_prev, double sigma1, double sigma2, double* w_f) {
  double a = sigma1 * sigma1, b = sigma2 * sigma2;
  if (t == 0) {
    *w_f = 0.0;
    return a;
  }
  *w_f = a / (a + b + P_prev);
  return a * (b + P_prev) / (a + b + P_prev);
}

/* Sec. 6: f(A_{t-1}, x) -- the previous binary segmentation turned into a grey
 * image by Gaussian smoothing (the form Sec. 7.3 implements).  Direct 2-D
 * normalised Gaussian on the (2r+1)^2 support, clamp-to-edge. */
void orc_smooth_mask(int H, int W, const uint8_t* mask, double sigma, int radius, double* f) {
  double sg = 0;
  for (int v = -radius; v <= radius; ++v)
    for (int u = -radius; u <= radius; ++u) sg += exp(-(u * u + v * v) / (2 * sigma * sigma));
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double acc = 0;
      for (int v = -radius; v <= radius; ++v)
        for (int u = -radius; u <= radius; ++u)
          acc += exp(-(u * u + v * v) / (2 * sigma * sigma)) / sg *
                 mask[clampi(y + v, 0, H - 1) * W + clampi(x + u, 0, W - 1)];
      f[y * W + x] = acc;
    }
}

/* Sec. 5 + Sec. 6: the saliency prior q and the updated prior p-hat.
 * Reading: q = saliency / max(saliency) (0 when the max is 0) stands in for
 * the attention-density GMM of Sec. 5; the frame edge gets q = eps ("the prior
 * on the edge of each frame is assumed to be approximately 0", Sec. 5), a band
 * of border_px pixels.  p-hat = w_f f + (1 - w_f) q (Sec. 6). */
void orc_prior(const orc_params* P, int H, int W, const double* saliency, const uint8_t* prev_mask,
               double w_f, double* q, double* prior) {
  int n = H * W;
  double mx = 0;
  for (int i = 0; i < n; ++i) mx = maxd(mx, saliency[i]);
  double* f = NULL;
  if (prev_mask && w_f != 0.0) {
    f = (double*)malloc(sizeof(double) * n);
    orc_smooth_mask(H, W, prev_mask, P->f_sigma, P->f_radius, f);
  }
  int b = P->border_px;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int i = y * W + x;
      int edge = y < b || y >= H - b || x < b || x >= W - b;
      double qi = edge ? P->eps : (mx > 0 ? saliency[i] / mx : 0.0);
      q[i] = qi;
      prior[i] = (f ? w_f * f[i] : 0.0) + (1.0 - w_f) * qi;
    }
  free(f);
}

/* ------------------------------------------------------------------------ */
/* Sec. 5: colour likelihood p(C|A) estimated from ALL pixels weighted by the
 * prior (weight p-hat for the object label 1, 1 - p-hat for background 0).
 * Reading: one Gaussian per label (the M = 1 case of the GMM), C = RGB/255,
 * two-pass weighted mean and covariance, plus 1e-4 I.  Returns a bitmask of
 * labels whose total weight is zero (no model: psi_1 = 0 for that label). */
int orc_colour_models(const double* prior, const uint8_t* rgb, int n, double mu[2][3],
                      double cov[2][3][3]) {
  int degenerate = 0;
  for (int a = 0; a < 2; ++a) {
    double sw = 0, m[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
      double w = a ? prior[i] : 1.0 - prior[i];
      sw += w;
      for (int k = 0; k < 3; ++k) m[k] += w * (rgb[3 * i + k] / 255.0);
    }
    if (!(sw > 0)) {
      degenerate |= 1 << a;
      for (int k = 0; k < 3; ++k) {
        mu[a][k] = 0;
        for (int j = 0; j < 3; ++j) cov[a][k][j] = k == j;
      }
      continue;
    }
    for (int k = 0; k < 3; ++k) mu[a][k] = m[k] / sw;
    double c[3][3] = {{0}};
    for (int i = 0; i < n; ++i) {
      double w = a ? prior[i] : 1.0 - prior[i];
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = rgb[3 * i + k] / 255.0 - mu[a][k];
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) c[k][j] += w * d[k] * d[j];
    }
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) cov[a][k][j] = c[k][j] / sw + (k == j ? 1e-4 : 0.0);
  }
  return degenerate;
}

static double det3(double m[3][3]) {
  return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
         m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
         m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

static void inv3(double m[3][3], double out[3][3]) {
  double d = det3(m);
  out[0][0] = (m[1][1] * m[2][2] - m[1][2] * m[2][1]) / d;
  out[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) / d;
  out[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) / d;
  out[1][0] = (m[1][2] * m[2][0] - m[1][0] * m[2][2]) / d;
  out[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) / d;
  out[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) / d;
  out[2][0] = (m[1][0] * m[2][1] - m[1][1] * m[2][0]) / d;
  out[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) / d;
  out[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) / d;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4 + Sec. 7.3: the colour likelihood p(C|A) as a Gaussian mixture of M
 * components per label, fitted by EM to all pixels weighted by the prior
 * (Sec. 5).  M = 3 in the paper's experiments (Sec. 8.1).
 * Reading (the paper initialises EM by k-means on the CPU, unspecified): a
 * deterministic initialisation without any argmax -- the means start on the
 * grey axis g = (1,1,1)/sqrt3 through the weighted mean, at (m - (M-1)/2) * 1.5
 * sigma_g with sigma_g^2 = g^T Sigma g; every covariance starts at the weighted
 * global covariance (+ 1e-4 I), every weight at 1/M.  Then a fixed number of
 * EM iterations: E-step responsibilities r_m = pi_m N_m / sum_k pi_k N_k;
 * M-step with the pixel weights w: N_m = sum w r_m, pi_m = N_m / sum_k N_k,
 * mu_m = sum w r_m C / N_m, Sigma_m = sum w r_m (C - mu_m)(C - mu_m)^T / N_m
 * + 1e-4 I.  A component with N_m < 1e-6 sum(w) keeps its parameters. */
static void gmm_pdf_terms(const orc_gmm* g, const double c[3], double* logp) {
  for (int m = 0; m < g->M; ++m) {
    double A[3][3], Ai[3][3];
    memcpy(A, g->cov[m], sizeof(A));
    double d = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
               A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
    Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
    Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
    Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
    Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
    Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
    Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
    Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
    Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
    double q = 0, dv[3];
    for (int k = 0; k < 3; ++k) dv[k] = c[k] - g->mu[m][k];
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) q += dv[k] * Ai[k][j] * dv[j];
    logp[m] = log(g->pi[m]) - 0.5 * q - 0.5 * log(d) - 1.5 * log(2.0 * M_PI);
  }
}

/* log sum_m pi_m N(c; mu_m, Sigma_m) */
double orc_gmm_logpdf(const orc_gmm* g, const double c[3]) {
  double lp[3], mx = -DBL_MAX, s = 0;
  gmm_pdf_terms(g, c, lp);
  for (int m = 0; m < g->M; ++m) mx = maxd(mx, lp[m]);
  for (int m = 0; m < g->M; ++m) s += exp(lp[m] - mx);
  return mx + log(s);
}

/* Sec. 7.3: EM of the colour mixtures starts from a k-means partition.
 * Reading (the paper names a CPU k-means but not its start): the seeds are
 * k-means++ taken in expectation instead of drawn at random -- c_1 is the
 * weighted mean of the colours, c_m (m > 1) the mean of the colours weighted by
 * w_i D_i^2, D_i the distance of C_i to its nearest earlier seed (the expected
 * position of a k-means++ draw, which picks C_i with probability proportional
 * to w_i D_i^2).  Then km_iters weighted Lloyd iterations: every pixel joins its
 * nearest center (the lowest index on equal distances), every center whose
 * cluster carries at least 1e-6 of the weight moves to its cluster's weighted
 * mean.  The mixture is the final partition's: pi_m = cluster weight / total,
 * mu_m and Sigma_m (+ 1e-4 I) the cluster's weighted mean and covariance; a
 * cluster below 1e-6 of the weight keeps its center, the label's covariance and
 * its (tiny or zero) weight. */
static int nearest_center(const double c[3], const double (*ctr)[3], int M) {
  int best = 0;
  double bd = DBL_MAX;
  for (int m = 0; m < M; ++m) {
    double d = 0;
    for (int k = 0; k < 3; ++k) d += (c[k] - ctr[m][k]) * (c[k] - ctr[m][k]);
    if (d < bd) {
      bd = d;
      best = m;
    }
  }
  return best;
}

void orc_gmm_init(const uint8_t* rgb, const double* w, int n, int M, int km_iters, orc_gmm* g) {
  double sw = 0, mu[3] = {0, 0, 0}, cv[3][3] = {{0}};
  for (int i = 0; i < n; ++i) {
    sw += w[i];
    for (int k = 0; k < 3; ++k) mu[k] += w[i] * (rgb[3 * i + k] / 255.0);
  }
  for (int k = 0; k < 3; ++k) mu[k] /= sw;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j)
        cv[k][j] += w[i] * (rgb[3 * i + k] / 255.0 - mu[k]) * (rgb[3 * i + j] / 255.0 - mu[j]);
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) cv[k][j] = cv[k][j] / sw + (k == j ? 1e-4 : 0.0);
  /* seeds */
  double ctr[3][3];
  memcpy(ctr[0], mu, sizeof(mu));
  for (int m = 1; m < M; ++m) {
    double s = 0, acc[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
      double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
      double d2 = DBL_MAX;
      for (int j = 0; j < m; ++j) {
        double d = 0;
        for (int k = 0; k < 3; ++k) d += (c[k] - ctr[j][k]) * (c[k] - ctr[j][k]);
        d2 = mind(d2, d);
      }
      s += w[i] * d2;
      for (int k = 0; k < 3; ++k) acc[k] += w[i] * d2 * c[k];
    }
    for (int k = 0; k < 3; ++k) ctr[m][k] = s > 0 ? acc[k] / s : mu[k];
  }
  /* Lloyd iterations */
  for (int it = 0; it < km_iters; ++it) {
    double W[3] = {0, 0, 0}, S[3][3] = {{0}};
    for (int i = 0; i < n; ++i) {
      double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
      int m = nearest_center(c, (const double(*)[3])ctr, M);
      W[m] += w[i];
      for (int k = 0; k < 3; ++k) S[m][k] += w[i] * c[k];
    }
    for (int m = 0; m < M; ++m)
      if (W[m] >= 1e-6 * sw)
        for (int k = 0; k < 3; ++k) ctr[m][k] = S[m][k] / W[m];
  }
  /* the mixture of the final partition (two passes per cluster) */
  double W[3] = {0, 0, 0}, S[3][3] = {{0}};
  int* lab = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
    lab[i] = nearest_center(c, (const double(*)[3])ctr, M);
    W[lab[i]] += w[i];
    for (int k = 0; k < 3; ++k) S[lab[i]][k] += w[i] * c[k];
  }
  g->M = M;
  for (int m = 0; m < M; ++m) {
    g->pi[m] = W[m] / sw;
    if (!(W[m] >= 1e-6 * sw)) {
      memcpy(g->mu[m], ctr[m], sizeof(ctr[m]));
      memcpy(g->cov[m], cv, sizeof(cv));
      continue;
    }
    double cm[3];
    for (int k = 0; k < 3; ++k) cm[k] = S[m][k] / W[m];
    double cc[3][3] = {{0}};
    for (int i = 0; i < n; ++i) {
      if (lab[i] != m) continue;
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
          cc[k][j] += w[i] * (rgb[3 * i + k] / 255.0 - cm[k]) * (rgb[3 * i + j] / 255.0 - cm[j]);
    }
    for (int k = 0; k < 3; ++k) {
      g->mu[m][k] = cm[k];
      for (int j = 0; j < 3; ++j) g->cov[m][k][j] = cc[k][j] / W[m] + (k == j ? 1e-4 : 0.0);
    }
  }
  free(lab);
}

double orc_gmm_loglik(const uint8_t* rgb, const double* w, int n, const orc_gmm* g) {
  double L = 0;
  for (int i = 0; i < n; ++i) {
    double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
    L += w[i] * orc_gmm_logpdf(g, c);
  }
  return L;
}

void orc_gmm_em_step(const uint8_t* rgb, const double* w, int n, orc_gmm* g) {
  int M = g->M;
  double* r = (double*)malloc(sizeof(double) * (size_t)n * M);
  double Nm[3] = {0, 0, 0}, sw = 0;
  for (int i = 0; i < n; ++i) {  /* E-step */
    double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
    double lp[3], mx = -DBL_MAX, s = 0;
    gmm_pdf_terms(g, c, lp);
    for (int m = 0; m < M; ++m) mx = maxd(mx, lp[m]);
    for (int m = 0; m < M; ++m) s += exp(lp[m] - mx);
    for (int m = 0; m < M; ++m) {
      r[(size_t)i * M + m] = exp(lp[m] - mx) / s;
      Nm[m] += w[i] * r[(size_t)i * M + m];
    }
    sw += w[i];
  }
  double Ntot = 0;
  for (int m = 0; m < M; ++m) Ntot += Nm[m];
  for (int m = 0; m < M; ++m) {  /* M-step, two passes per component */
    g->pi[m] = Nm[m] / Ntot;
    if (!(Nm[m] >= 1e-6 * sw)) continue;
    double mu[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k) mu[k] += w[i] * r[(size_t)i * M + m] * (rgb[3 * i + k] / 255.0);
    for (int k = 0; k < 3; ++k) mu[k] /= Nm[m];
    double cv[3][3] = {{0}};
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j)
          cv[k][j] += w[i] * r[(size_t)i * M + m] * (rgb[3 * i + k] / 255.0 - mu[k]) * (rgb[3 * i + j] / 255.0 - mu[j]);
    for (int k = 0; k < 3; ++k) {
      g->mu[m][k] = mu[k];
      for (int j = 0; j < 3; ++j) g->cov[m][k][j] = cv[k][j] / Nm[m] + (k == j ? 1e-4 : 0.0);
    }
  }
  free(r);
}

void orc_gmm_fit(const uint8_t* rgb, const double* w, int n, int M, int km_iters, int iters, orc_gmm* g) {
  orc_gmm_init(rgb, w, n, M, km_iters, g);
  for (int it = 0; it < iters; ++it) orc_gmm_em_step(rgb, w, n, g);
}

static int32_t quantize(double K, double x) {
  /* Reading: integer capacity = min(2^24, floor(K x + 1/2)). */
  double v = floor(K * x + 0.5);
  if (v > 16777216.0) v = 16777216.0;
  if (v < 0) v = 0;
  return (int32_t)v;
}

/* Sec. 4: n-link cost c(x,y) = psi_2 + xi_2 (Eq. 2).
 * Reading: xi_2 = lambda_p (Potts constant) and the contrast term with the
 * positive sign of Boykov-Jolly, lambda_s exp(-dI^2 / (2 sigma_I^2)) / |x-y|
 * (the printed minus sign would make cuts cheaper between similar pixels);
 * dI = (sum_x - sum_y) / 765 with sum = r+g+b; |x-y| = 1 or sqrt(2). */
int32_t orc_ncap_value(const orc_params* P, int dsum, int diagonal) {
  double dI = dsum / 765.0;
  double dist = diagonal ? sqrt(2.0) : 1.0;
  double c = P->lambda_p + P->lambda_s * exp(-dI * dI / (2.0 * P->sigma_I * P->sigma_I)) / dist;
  return quantize(P->cap_scale, c);
}

/* Sec. 4, Eqs. 1-4: graph capacities.
 *   xi_1(a) = -log p(A = a) with p(A=1) = p-hat, clamped to [eps, 1-eps];
 *   psi_1(a) = -log N(C; mu_a, Sigma_a)
 *            = 1/2 d^T Sigma_a^-1 d + 1/2 log det Sigma_a + 3/2 log 2 pi;
 *   D(a) = lambda_u psi_1(a) + xi_1(a);
 *   t-links c(s,v) = D(0) (Eq. 3), c(v,t) = D(1) (Eq. 4).
 * Reading: the source side is the object (label 1): a source-side pixel pays
 * c(v,t) = D(1), a sink-side pixel c(s,v) = D(0) (the paper's label-to-terminal
 * sentence is the reverse of its capacity equations).  Both t-links are
 * shifted by min(D(0), D(1)), a per-pixel constant that leaves every minimum
 * cut unchanged, then quantised. */
/* mix (nullable): the two labels' colour mixtures carried between frames.  With
 * from_mix the EM of a label starts from mix[a] (Sec. 2 / Sec. 6: feature
 * likelihoods updated to reflect the dominant feature components of the previous
 * segmentation; reading: the previous frame's fitted mixture is the current
 * frame's EM start, and the k-means start runs only on a video's first frame);
 * the fitted mixtures are written back to mix. */
void orc_terms_ex(const orc_params* P, int H, int W, const uint8_t* rgb, const double* prior,
                  int32_t* cs, int32_t* ct, int32_t* ncap, double* D0, double* D1, orc_gmm* mix, int from_mix) {
  int n = H * W;
  double mu[2][3], cov[2][3][3], icov[2][3][3], lconst[2];
  int degenerate = orc_colour_models(prior, rgb, n, mu, cov);
  orc_gmm gm[2];
  if (P->gmm_components > 1) {  /* Sec. 4 / Sec. 7.3: M-component EM per label */
    double* w = (double*)malloc(sizeof(double) * n);
    for (int a = 0; a < 2; ++a) {
      if (degenerate & (1 << a)) continue;
      for (int i = 0; i < n; ++i) w[i] = a ? prior[i] : 1.0 - prior[i];
      if (from_mix && mix && mix[a].M == P->gmm_components) {
        gm[a] = mix[a];
        for (int it = 0; it < P->em_iters; ++it) orc_gmm_em_step(rgb, w, n, &gm[a]);
      } else {
        orc_gmm_fit(rgb, w, n, P->gmm_components, P->kmeans_iters, P->em_iters, &gm[a]);
      }
      if (mix) mix[a] = gm[a];
    }
    free(w);
  }
  for (int a = 0; a < 2; ++a) {
    inv3(cov[a], icov[a]);
    lconst[a] = 0.5 * log(det3(cov[a])) + 1.5 * log(2.0 * M_PI);
  }
  double eps = P->eps;
  for (int i = 0; i < n; ++i) {
    double D[2];
    for (int a = 0; a < 2; ++a) {
      double p = a ? prior[i] : 1.0 - prior[i];
      double xi = -log(mind(maxd(p, eps), 1.0 - eps));
      double psi = 0.0;
      if (!(degenerate & (1 << a)) && P->gmm_components > 1) {
        double c[3] = {rgb[3 * i] / 255.0, rgb[3 * i + 1] / 255.0, rgb[3 * i + 2] / 255.0};
        psi = -orc_gmm_logpdf(&gm[a], c);
      } else if (!(degenerate & (1 << a))) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = rgb[3 * i + k] / 255.0 - mu[a][k];
        double q = 0;
        for (int k = 0; k < 3; ++k)
          for (int j = 0; j < 3; ++j) q += d[k] * icov[a][k][j] * d[j];
        psi = 0.5 * q + lconst[a];
      }
      D[a] = P->lambda_u * psi + xi;
    }
    double m = mind(D[0], D[1]);
    cs[i] = quantize(P->cap_scale, D[0] - m);
    ct[i] = quantize(P->cap_scale, D[1] - m);
    if (D0) D0[i] = D[0];
    if (D1) D1[i] = D[1];
  }
  if (!ncap) return;
  static const int dx[4] = {1, 0, 1, -1}, dy[4] = {0, 1, 1, 1};
  int nk = P->neighbourhood / 2;
  for (int k = 0; k < nk; ++k)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int xx = x + dx[k], yy = y + dy[k];
        int32_t c = 0;
        if (xx >= 0 && xx < W && yy < H) {
          int i = y * W + x, j = yy * W + xx;
          int s1 = rgb[3 * i] + rgb[3 * i + 1] + rgb[3 * i + 2];
          int s2 = rgb[3 * j] + rgb[3 * j + 1] + rgb[3 * j + 2];
          c = orc_ncap_value(P, s1 - s2, k >= 2);
        }
        ncap[(size_t)k * n + y * W + x] = c;
      }
}

void orc_terms(const orc_params* P, int H, int W, const uint8_t* rgb, const double* prior,
               int32_t* cs, int32_t* ct, int32_t* ncap, double* D0, double* D1) {
  orc_terms_ex(P, H, W, rgb, prior, cs, ct, ncap, D0, D1, NULL, 0);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: the MAP labelling is the minimum s-t cut of the graph of Fig. 5.
 * The grid graph: node y*W+x; an undirected n-link of capacity ncap gives two
 * directed arcs of that capacity ("a pair of mutually connected directed
 * edges", Sec. 4 footnote). */
static const int NB_DX[4] = {1, 0, 1, -1}, NB_DY[4] = {0, 1, 1, 1};

typedef struct {
  int n;          /* nodes incl. terminals when present */
  int m, mcap;    /* arcs */
  int* first;
  int* next;
  int* head;
  int64_t* r;     /* residual capacity */
} graph;

static void g_init(graph* g, int n, int mcap) {
  g->n = n;
  g->m = 0;
  g->mcap = mcap;
  g->first = (int*)malloc(sizeof(int) * n);
  for (int i = 0; i < n; ++i) g->first[i] = -1;
  g->next = (int*)malloc(sizeof(int) * mcap);
  g->head = (int*)malloc(sizeof(int) * mcap);
  g->r = (int64_t*)malloc(sizeof(int64_t) * mcap);
}

static void g_free(graph* g) {
  free(g->first);
  free(g->next);
  free(g->head);
  free(g->r);
}

/* adds u->v (cap c_uv) and v->u (cap c_vu) as arcs 2k and 2k+1 (sisters: a^1) */
static void g_add(graph* g, int u, int v, int64_t c_uv, int64_t c_vu) {
  int a = g->m++, b = g->m++;
  g->head[a] = v;
  g->r[a] = c_uv;
  g->next[a] = g->first[u];
  g->first[u] = a;
  g->head[b] = u;
  g->r[b] = c_vu;
  g->next[b] = g->first[v];
  g->first[v] = b;
}

static void g_add_grid(graph* g, int H, int W, int nbr, const int32_t* ncap) {
  int n = H * W;
  for (int k = 0; k < nbr / 2; ++k)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int xx = x + NB_DX[k], yy = y + NB_DY[k];
        if (xx < 0 || xx >= W || yy >= H) continue;
        int64_t c = ncap[(size_t)k * n + y * W + x];
        g_add(g, y * W + x, yy * W + xx, c, c);
      }
}

/* Edmonds-Karp: shortest augmenting paths by BFS from s until t is unreachable.
 * mask = nodes reachable from s in the final residual graph = the minimal
 * source set of the minimum cut (intersection of all minimum cuts). */
int64_t orc_maxflow_ek(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask) {
  int n = H * W, s = n, t = n + 1;
  graph g;
  g_init(&g, n + 2, 2 * (n * (nbr / 2) + 2 * n) + 8);
  g_add_grid(&g, H, W, nbr, ncap);
  for (int v = 0; v < n; ++v) {
    g_add(&g, s, v, cs[v], 0);
    g_add(&g, v, t, ct[v], 0);
  }
  int* par = (int*)malloc(sizeof(int) * (n + 2));
  int* q = (int*)malloc(sizeof(int) * (n + 2));
  int64_t flow = 0;
  for (;;) {
    for (int i = 0; i < n + 2; ++i) par[i] = -2;
    par[s] = -1;
    int qh = 0, qt = 0;
    q[qt++] = s;
    while (qh < qt && par[t] == -2) {
      int u = q[qh++];
      for (int a = g.first[u]; a >= 0; a = g.next[a])
        if (g.r[a] > 0 && par[g.head[a]] == -2) {
          par[g.head[a]] = a;
          q[qt++] = g.head[a];
        }
    }
    if (par[t] == -2) break;
    int64_t delta = INT64_MAX;
    for (int v = t; v != s; v = g.head[par[v] ^ 1]) delta = g.r[par[v]] < delta ? g.r[par[v]] : delta;
    for (int v = t; v != s; v = g.head[par[v] ^ 1]) {
      g.r[par[v]] -= delta;
      g.r[par[v] ^ 1] += delta;
    }
    flow += delta;
  }
  /* residual reachability from s (par != -2 after the last, failed BFS) */
  for (int v = 0; v < n; ++v) mask[v] = par[v] != -2;
  free(par);
  free(q);
  g_free(&g);
  return flow;
}

/* Boykov-Kolmogorov max-flow (search trees S and T grown from the terminals,
 * augmentation along the path where they meet, adoption of orphans).  Written
 * from the published algorithm; terminal arcs are kept as one signed residual
 * per node (tr > 0: residual from s, tr < 0: residual to t). */
enum { BK_FREE = 0, BK_S = 1, BK_T = 2 };
#define BK_TERMINAL (-2)
#define BK_ORPHAN (-3)
#define BK_NONE (-1)

int64_t orc_maxflow_bk(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask) {
  int n = H * W;
  graph g;
  g_init(&g, n, 2 * n * (nbr / 2) + 8);
  g_add_grid(&g, H, W, nbr, ncap);
  int64_t* tr = (int64_t*)malloc(sizeof(int64_t) * n);
  int* tree = (int*)malloc(sizeof(int) * n);
  int* parent = (int*)malloc(sizeof(int) * n); /* arc from node to its parent */
  int* ts = (int*)malloc(sizeof(int) * n);
  char* queued = (char*)malloc(n);
  int* active = (int*)malloc(sizeof(int) * (size_t)(n + 1)); /* circular FIFO */
  int* orphans = (int*)malloc(sizeof(int) * (size_t)n);
  int ah = 0, at = 0, acount = 0;
  int64_t flow = 0;
#define BK_PUSH_ACTIVE(v)                \
  do {                                   \
    if (!queued[v]) {                    \
      queued[v] = 1;                     \
      active[at] = (v);                  \
      at = (at + 1) % (n + 1);           \
      acount++;                          \
    }                                    \
  } while (0)
  for (int v = 0; v < n; ++v) {
    int64_t m = cs[v] < ct[v] ? cs[v] : ct[v];
    flow += m; /* s -> v -> t directly */
    tr[v] = (int64_t)cs[v] - ct[v];
    queued[v] = 0;
    ts[v] = 0;
    if (tr[v] > 0) {
      tree[v] = BK_S;
      parent[v] = BK_TERMINAL;
      BK_PUSH_ACTIVE(v);
    } else if (tr[v] < 0) {
      tree[v] = BK_T;
      parent[v] = BK_TERMINAL;
      BK_PUSH_ACTIVE(v);
    } else {
      tree[v] = BK_FREE;
      parent[v] = BK_NONE;
    }
  }
  int TIME = 0;
  while (acount > 0) {
    int i = active[ah];
    ah = (ah + 1) % (n + 1);
    acount--;
    queued[i] = 0;
    if (tree[i] == BK_FREE) continue;
    /* growth */
    int mid = -1; /* arc from an S node to a T node */
    for (int a = g.first[i]; a >= 0; a = g.next[a]) {
      int j = g.head[a];
      if (tree[i] == BK_S) {
        if (g.r[a] <= 0) continue;
        if (tree[j] == BK_FREE) {
          tree[j] = BK_S;
          parent[j] = a ^ 1; /* j -> i */
          ts[j] = ts[i];
          BK_PUSH_ACTIVE(j);
        } else if (tree[j] == BK_T) {
          mid = a;
          break;
        }
      } else {
        if (g.r[a ^ 1] <= 0) continue; /* need residual j -> i */
        if (tree[j] == BK_FREE) {
          tree[j] = BK_T;
          parent[j] = a ^ 1;
          ts[j] = ts[i];
          BK_PUSH_ACTIVE(j);
        } else if (tree[j] == BK_S) {
          mid = a ^ 1;
          break;
        }
      }
    }
    if (mid < 0) continue;
    BK_PUSH_ACTIVE(i); /* it may still have unexplored arcs after the augmentation */
    /* augmentation */
    int u = g.head[mid ^ 1], v = g.head[mid];
    int64_t delta = g.r[mid];
    int x;
    for (x = u; parent[x] != BK_TERMINAL; x = g.head[parent[x]])
      if (g.r[parent[x] ^ 1] < delta) delta = g.r[parent[x] ^ 1];
    if (tr[x] < delta) delta = tr[x];
    for (x = v; parent[x] != BK_TERMINAL; x = g.head[parent[x]])
      if (g.r[parent[x]] < delta) delta = g.r[parent[x]];
    if (-tr[x] < delta) delta = -tr[x];
    g.r[mid] -= delta;
    g.r[mid ^ 1] += delta;
    int no = 0;
    for (x = u;;) {
      if (parent[x] == BK_TERMINAL) {
        tr[x] -= delta;
        if (tr[x] == 0) {
          parent[x] = BK_ORPHAN;
          orphans[no++] = x;
        }
        break;
      }
      int a = parent[x], nx = g.head[a];
      g.r[a ^ 1] -= delta;
      g.r[a] += delta;
      if (g.r[a ^ 1] == 0) {
        parent[x] = BK_ORPHAN;
        orphans[no++] = x;
      }
      x = nx;
    }
    for (x = v;;) {
      if (parent[x] == BK_TERMINAL) {
        tr[x] += delta;
        if (tr[x] == 0) {
          parent[x] = BK_ORPHAN;
          orphans[no++] = x;
        }
        break;
      }
      int a = parent[x], nx = g.head[a];
      g.r[a] -= delta;
      g.r[a ^ 1] += delta;
      if (g.r[a] == 0) {
        parent[x] = BK_ORPHAN;
        orphans[no++] = x;
      }
      x = nx;
    }
    flow += delta;
    /* adoption */
    TIME++;
    while (no > 0) {
      int j = orphans[--no];
      int tj = tree[j];
      int found = -1;
      for (int a = g.first[j]; a >= 0 && found < 0; a = g.next[a]) {
        int k = g.head[a];
        if (tree[k] != tj) continue;
        if (tj == BK_S ? g.r[a ^ 1] <= 0 : g.r[a] <= 0) continue;
        /* does k trace back to its terminal without meeting an orphan? */
        int y = k, ok = 0;
        for (;;) {
          if (ts[y] == TIME) { ok = 1; break; }
          if (parent[y] == BK_TERMINAL) { ok = 1; break; }
          if (parent[y] == BK_ORPHAN || parent[y] == BK_NONE) break;
          y = g.head[parent[y]];
        }
        if (!ok) continue;
        for (y = k; ts[y] != TIME && parent[y] != BK_TERMINAL; y = g.head[parent[y]]) ts[y] = TIME;
        ts[y] = TIME;
        found = a;
      }
      if (found >= 0) {
        parent[j] = found;
        ts[j] = TIME;
        continue;
      }
      /* no valid parent: j leaves its tree */
      tree[j] = BK_FREE;
      parent[j] = BK_NONE;
      for (int a = g.first[j]; a >= 0; a = g.next[a]) {
        int k = g.head[a];
        if (tree[k] != tj) continue;
        if (tj == BK_S ? g.r[a ^ 1] > 0 : g.r[a] > 0) BK_PUSH_ACTIVE(k);
        if (parent[k] >= 0 && g.head[parent[k]] == j) {
          parent[k] = BK_ORPHAN;
          orphans[no++] = k;
        }
      }
    }
  }
#undef BK_PUSH_ACTIVE
  /* minimal source set: residual reachability from s (explicit BFS) */
  int* q = orphans;
  int qh = 0, qt = 0;
  for (int v = 0; v < n; ++v) {
    mask[v] = tr[v] > 0;
    if (mask[v]) q[qt++] = v;
  }
  while (qh < qt) {
    int u = q[qh++];
    for (int a = g.first[u]; a >= 0; a = g.next[a])
      if (g.r[a] > 0 && !mask[g.head[a]]) {
        mask[g.head[a]] = 1;
        q[qt++] = g.head[a];
      }
  }
  free(tr);
  free(tree);
  free(parent);
  free(ts);
  free(queued);
  free(active);
  free(orphans);
  g_free(&g);
  return flow;
}

/* Eq. 1 on the integer graph: cost of the cut whose source side is mask = 1. */
int64_t orc_cut_energy(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, const uint8_t* mask) {
  int n = H * W;
  int64_t e = 0;
  for (int v = 0; v < n; ++v) e += mask[v] ? ct[v] : cs[v];
  for (int k = 0; k < nbr / 2; ++k)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int xx = x + NB_DX[k], yy = y + NB_DY[k];
        if (xx < 0 || xx >= W || yy >= H) continue;
        if (mask[y * W + x] != mask[yy * W + xx]) e += ncap[(size_t)k * n + y * W + x];
      }
  return e;
}

/* Every labelling of a tiny grid (n <= 24): the minimum energy, and the
 * intersection of all minimisers (the minimal minimum-cut source set). */
int64_t orc_bruteforce(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask_min, int32_t* n_argmin) {
  int n = H * W;
  if (n > 24) return -1;
  uint8_t* m = (uint8_t*)malloc(n ? n : 1);
  int64_t best = INT64_MAX;
  uint32_t inter = 0;
  int count = 0;
  for (uint32_t bits = 0; bits < (1u << n); ++bits) {
    for (int v = 0; v < n; ++v) m[v] = (bits >> v) & 1;
    int64_t e = orc_cut_energy(H, W, nbr, cs, ct, ncap, m);
    if (e < best) {
      best = e;
      inter = bits;
      count = 1;
    } else if (e == best) {
      inter &= bits;
      count++;
    }
  }
  for (int v = 0; v < n; ++v) mask_min[v] = (inter >> v) & 1;
  if (n_argmin) *n_argmin = count;
  free(m);
  return best;
}

/* ------------------------------------------------------------------------ */
/* One frame of the method (Fig. 3): saliency (Sec. 3) -> prior q (Sec. 5) ->
 * sequential update with the previous segmentation (Sec. 6) -> MRF graph
 * (Sec. 4, Eqs. 1-4) -> minimum cut (Sec. 4).  The mask becomes A_{t-1} of the
 * next frame.  Returns the cut value. */
int64_t orc_push_frame(const orc_params* P, int H, int W, orc_state* st, const uint8_t* rgb,
                       double* saliency, double* prior, uint8_t* mask) {
  int n = H * W;
  double* q = (double*)malloc(sizeof(double) * n);
  orc_saliency(P, H, W, rgb, saliency);
  double w_f;
  double Pt = orc_kalman_step(st->t, st->P, P->sigma1, P->sigma2, &w_f);
  orc_prior(P, H, W, saliency, st->t > 0 ? st->prev_mask : NULL, w_f, q, prior);
  int nk = P->neighbourhood / 2;
  int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* ct = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* nc = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * nk);
  orc_terms_ex(P, H, W, rgb, prior, cs, ct, nc, NULL, NULL, st->gmm,
               P->gmm_update && st->gmm_valid && st->t > 0);
  if (P->gmm_components > 1) st->gmm_valid = 1;
  int64_t cut = orc_maxflow_bk(H, W, P->neighbourhood, cs, ct, nc, mask);
  memcpy(st->prev_mask, mask, n);
  st->P = Pt;
  st->t += 1;
  free(q);
  free(cs);
  free(ct);
  free(nc);
  return cut;
}
