/*
 * oracle_grad.c -- FP64 reverse-mode derivative ("adjoint") of the oracle's
 * saliency map and Kalman-updated prior, for the backward form of the path.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oracle.c): it shares no code with the
 * CUDA path.  The forward here is oracle.c's method restated on a floating-point
 * frame (RGB values in [0, 255], so that the frame can be differentiated), with
 * every intermediate kept; the backward walks the same steps in reverse:
 *
 *   prior = w_f f + (1 - w_f) q,  w_f = Q / (Q + R + P)       (Sec. 6, Q = sigma1^2, R = sigma2^2)
 *   P(t) = Q (R + P(t-1)) / (Q + R + P(t-1)), P(-1) = +inf      (Sec. 6; its Q, R derivatives forward mode)
 *   q = sal / max(sal) inside the frame, eps on the border     (Sec. 5)
 *   sal = up(S),  S = sum_k w_k N(C_k)                          (Sec. 3 / Sec. 7.2)
 *   C_k = sum over scales of REDUCE^(sigma_S - c) N(CS(c, s)), C_O = sum_theta N(.)
 *   CS = |X(c) -/+ up X(s)|, X = pyramids of I, RG, BY and Gabor magnitudes of I
 *
 * Piecewise parts take their one-sided (sub)gradient: N(.) through its min, max
 * and tile maxima at the first index attaining them, |.| and max(0, .) through
 * the sign at the point, the hue-normalisation mask (10 (r+g+b) > max) as fixed.
 * The previous mask (through f) is a constant.
 *
 * Parity unpinned? No: pinned by central finite differences of the forward in
 * tests/test_oracle_grad.py at points away from those kinks.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int ci(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static const double KB[5] = {1 / 16., 4 / 16., 6 / 16., 4 / 16., 1 / 16.};

/* ---------------- primitives and their adjoints ---------------- */
static void reduce_fw(int h, int w, const double* in, double* out) {
  int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
  for (int y = 0; y < h2; ++y)
    for (int x = 0; x < w2; ++x) {
      double a = 0;
      for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) a += KB[j + 2] * KB[i + 2] * in[ci(2 * y + j, 0, h - 1) * w + ci(2 * x + i, 0, w - 1)];
      out[y * w2 + x] = a;
    }
}
/* g_in += REDUCE^T g_out */
static void reduce_bw(int h, int w, const double* g_out, double* g_in) {
  int h2 = (h + 1) / 2, w2 = (w + 1) / 2;
  for (int y = 0; y < h2; ++y)
    for (int x = 0; x < w2; ++x)
      for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i)
          g_in[ci(2 * y + j, 0, h - 1) * w + ci(2 * x + i, 0, w - 1)] += KB[j + 2] * KB[i + 2] * g_out[y * w2 + x];
}

static void up_coord(int d, int ns, int nd, int* i0, int* i1, double* f) {
  double s = (d + 0.5) * ns / (double)nd - 0.5;
  if (s < 0) s = 0;
  if (s > ns - 1) s = ns - 1;
  *i0 = (int)floor(s);
  *i1 = *i0 + 1 < ns ? *i0 + 1 : ns - 1;
  *f = s - *i0;
}
static void up_fw(int hs, int ws, const double* src, int hd, int wd, double* dst) {
  for (int y = 0; y < hd; ++y) {
    int y0, y1;
    double fy;
    up_coord(y, hs, hd, &y0, &y1, &fy);
    for (int x = 0; x < wd; ++x) {
      int x0, x1;
      double fx;
      up_coord(x, ws, wd, &x0, &x1, &fx);
      dst[y * wd + x] = (1 - fy) * ((1 - fx) * src[y0 * ws + x0] + fx * src[y0 * ws + x1]) +
                        fy * ((1 - fx) * src[y1 * ws + x0] + fx * src[y1 * ws + x1]);
    }
  }
}
/* g_src += up^T g_dst */
static void up_bw(int hs, int ws, double* g_src, int hd, int wd, const double* g_dst) {
  for (int y = 0; y < hd; ++y) {
    int y0, y1;
    double fy;
    up_coord(y, hs, hd, &y0, &y1, &fy);
    for (int x = 0; x < wd; ++x) {
      int x0, x1;
      double fx;
      up_coord(x, ws, wd, &x0, &x1, &fx);
      double g = g_dst[y * wd + x];
      g_src[y0 * ws + x0] += (1 - fy) * (1 - fx) * g;
      g_src[y0 * ws + x1] += (1 - fy) * fx * g;
      g_src[y1 * ws + x0] += fy * (1 - fx) * g;
      g_src[y1 * ws + x1] += fy * fx * g;
    }
  }
}

/* N(.) with the quantities its derivative needs */
typedef struct {
  int flat, nt, amin, amax;
  double mn, mx, mbar, F;
  int* targ; /* per tile: first index of its maximum */
} nstat;

/* Near-tie census (test support): decisions of the forward whose margin,
 * relative to the map's range, is below g_tie_delta: [0] minimum / maximum of an
 * N(.) map, [1] a tile maximum, [2] the sign of a center-surround value. */
static double g_tie_delta = 0.0;
static long g_ties[3];

static void count_ties(int h, int w, const double* v, int T, const nstat* st) {
  if (!(g_tie_delta > 0) || st->flat) return;
  int n = h * w, ntx = (w + T - 1) / T;
  double D = st->mx - st->mn, lim = g_tie_delta * D;
  for (int i = 0; i < n; ++i) {
    if (i != st->amin && v[i] - st->mn < lim) g_ties[0]++;
    if (i != st->amax && st->mx - v[i] < lim) g_ties[0]++;
    int y = i / w, x = i - y * w, t = (y / T) * ntx + x / T;
    if (i != st->targ[t] && v[st->targ[t]] - v[i] < lim) g_ties[1]++;
  }
}

static void norm_fw(int h, int w, const double* v, int T, double flat, double* out, nstat* st) {
  int n = h * w, ntx = (w + T - 1) / T, nty = (h + T - 1) / T;
  st->nt = ntx * nty;
  st->targ = (int*)malloc(sizeof(int) * st->nt);
  st->amin = st->amax = 0;
  for (int i = 1; i < n; ++i) {
    if (v[i] < v[st->amin]) st->amin = i;
    if (v[i] > v[st->amax]) st->amax = i;
  }
  st->mn = v[st->amin];
  st->mx = v[st->amax];
  st->flat = !(st->mx - st->mn > flat);
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx) {
      int best = -1;
      for (int y = ty * T; y < h && y < (ty + 1) * T; ++y)
        for (int x = tx * T; x < w && x < (tx + 1) * T; ++x)
          if (best < 0 || v[y * w + x] > v[best]) best = y * w + x;
      st->targ[ty * ntx + tx] = best;
    }
  if (st->flat) {
    for (int i = 0; i < n; ++i) out[i] = 0;
    st->mbar = 0;
    st->F = 0;
    return;
  }
  double D = st->mx - st->mn, sum = 0;
  for (int t = 0; t < st->nt; ++t) sum += (v[st->targ[t]] - st->mn) / D;
  st->mbar = st->nt > 1 ? (sum - 1.0) / (st->nt - 1) : 0.0;
  st->F = (1 - st->mbar) * (1 - st->mbar);
  for (int i = 0; i < n; ++i) out[i] = (v[i] - st->mn) / D * st->F;
  count_ties(h, w, v, T, st);
}
/* g_v += N^T g_out */
static void norm_bw(int h, int w, const double* v, const nstat* st, const double* g_out, double* g_v) {
  if (st->flat) return;
  int n = h * w;
  double D = st->mx - st->mn;
  double* gp = (double*)malloc(sizeof(double) * n); /* dL/dv' */
  double sgv = 0;
  for (int i = 0; i < n; ++i) {
    gp[i] = g_out[i] * st->F;
    sgv += g_out[i] * (v[i] - st->mn) / D;
  }
  if (st->nt > 1) {
    double dm = sgv * (-2.0 * (1 - st->mbar)) / (st->nt - 1); /* dL/dmbar / (nt-1) */
    for (int t = 0; t < st->nt; ++t) gp[st->targ[t]] += dm;
  }
  double smin = 0, smax = 0;
  for (int i = 0; i < n; ++i) {
    double vp = (v[i] - st->mn) / D;
    g_v[i] += gp[i] / D;
    smin += gp[i] * (vp - 1) / D;
    smax += gp[i] * (-vp) / D;
  }
  g_v[st->amin] += smin;
  g_v[st->amax] += smax;
  free(gp);
}

/* ---------------- forward with intermediates ---------------- */
typedef struct {
  const orc_params* P;
  int H, W, L, no, sS, hl[16], wl[16], smax_mask;
  double *pyr[3][16], *ore[16][8], *oim[16][8], *ori[16][8];
  double *I0, *RG0, *BY0;
  double* acc[11];
  nstat nC[4], nT[8];
  double *C[4], *NC[4], *NT[8], *S, *sal;
  double salmx;
  int salarg;
  double smax;
} fwd_t;

static void gabor_fw(int h, int w, const double* in, const double* kre, const double* kim, int R, double* ore,
                     double* oim, double* out) {
  int n = 2 * R + 1;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      double re = 0, im = 0;
      for (int v = -R; v <= R; ++v)
        for (int u = -R; u <= R; ++u) {
          double p = in[ci(y + v, 0, h - 1) * w + ci(x + u, 0, w - 1)];
          re += kre[(v + R) * n + (u + R)] * p;
          im += kim[(v + R) * n + (u + R)] * p;
        }
      ore[y * w + x] = re;
      oim[y * w + x] = im;
      out[y * w + x] = sqrt(re * re + im * im);
    }
}
static void gabor_bw(int h, int w, const double* kre, const double* kim, int R, const double* ore, const double* oim,
                     const double* g_out, double* g_in) {
  int n = 2 * R + 1;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      double m = sqrt(ore[y * w + x] * ore[y * w + x] + oim[y * w + x] * oim[y * w + x]);
      if (!(m > 0)) continue;
      double gr = g_out[y * w + x] * ore[y * w + x] / m, gi = g_out[y * w + x] * oim[y * w + x] / m;
      for (int v = -R; v <= R; ++v)
        for (int u = -R; u <= R; ++u)
          g_in[ci(y + v, 0, h - 1) * w + ci(x + u, 0, w - 1)] +=
              kre[(v + R) * n + (u + R)] * gr + kim[(v + R) * n + (u + R)] * gi;
    }
}

/* features of a floating-point frame (hue mask decided on the values) */
static void features_fw(int H, int W, const double* rgb, double smax, double* I, double* RG, double* BY) {
  for (int i = 0; i < H * W; ++i) {
    double r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2], s = r + g + b;
    I[i] = s / 765.0;
    double rn = 0, gn = 0, bn = 0;
    if (10 * s > smax) {
      rn = 3 * r / s;
      gn = 3 * g / s;
      bn = 3 * b / s;
    }
    double Rr = fmax(0, rn - (gn + bn) / 2), G = fmax(0, gn - (rn + bn) / 2), B = fmax(0, bn - (rn + gn) / 2);
    double Y = fmax(0, (rn + gn) / 2 - fabs(rn - gn) / 2 - bn);
    RG[i] = Rr - G;
    BY[i] = B - Y;
  }
}
static void features_bw(int H, int W, const double* rgb, double smax, const double* gI, const double* gRG,
                        const double* gBY, double* grgb) {
  for (int i = 0; i < H * W; ++i) {
    double r = rgb[3 * i], g = rgb[3 * i + 1], b = rgb[3 * i + 2], s = r + g + b;
    double gs = gI[i] / 765.0, gr = gs, gg = gs, gb = gs;
    if (10 * s > smax) {
      /* the clamps' decisions: s > 0 scales out of every sign, so they are the signs
       * of linear forms of (r, g, b) (e.g. R > 0 iff 2r - g - b > 0), taken on
       * those forms, which are exact for single-precision inputs */
      double aR = 2 * r - g - b > 0, aG = 2 * g - r - b > 0, aB = 2 * b - r - g > 0;
      double aY = fmin(r, g) - b > 0; /* (rn + gn)/2 - |rn - gn|/2 = min(rn, gn) */
      double sg = r > g ? 1.0 : (r < g ? -1.0 : 0.0);
      double gR = gRG[i], gG = -gRG[i], gB = gBY[i], gY = -gBY[i];
      double grn = gR * aR - 0.5 * gG * aG - 0.5 * gB * aB + gY * aY * (0.5 - 0.5 * sg);
      double ggn = -0.5 * gR * aR + gG * aG - 0.5 * gB * aB + gY * aY * (0.5 + 0.5 * sg);
      double gbn = -0.5 * gR * aR - 0.5 * gG * aG + gB * aB - gY * aY;
      /* rn = 3 r / s etc. */
      double t = (grn * r + ggn * g + gbn * b) * 3.0 / (s * s);
      gr += grn * 3.0 / s - t;
      gg += ggn * 3.0 / s - t;
      gb += gbn * 3.0 / s - t;
    }
    grgb[3 * i] += gr;
    grgb[3 * i + 1] += gg;
    grgb[3 * i + 2] += gb;
  }
}

/* forward: saliency (H*W) and prior (H*W) from a floating-point frame.
 * Q = sigma1^2, R = sigma2^2, P = sigma^2_xi1(t-1) (t >= 1), w = channel weights. */
static void fwd_run(fwd_t* F, const orc_params* P, int H, int W, const double* rgb) {
  memset(F, 0, sizeof(*F));
  F->P = P;
  F->H = H;
  F->W = W;
  F->L = P->levels;
  F->no = P->n_orient;
  F->sS = P->c_max;
  for (int l = 0; l < F->L; ++l) {
    F->hl[l] = orc_level_dim(H, l);
    F->wl[l] = orc_level_dim(W, l);
  }
  double smax = 0;
  for (int i = 0; i < H * W; ++i) smax = fmax(smax, rgb[3 * i] + rgb[3 * i + 1] + rgb[3 * i + 2]);
  F->smax = smax;
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < F->L; ++l) F->pyr[c][l] = (double*)malloc(sizeof(double) * F->hl[l] * F->wl[l]);
  features_fw(H, W, rgb, smax, F->pyr[0][0], F->pyr[1][0], F->pyr[2][0]);
  for (int c = 0; c < 3; ++c)
    for (int l = 1; l < F->L; ++l) reduce_fw(F->hl[l - 1], F->wl[l - 1], F->pyr[c][l - 1], F->pyr[c][l]);
  int R = P->gabor_radius, kn = 2 * R + 1, smx = P->c_max + P->d_max;
  double* kre = (double*)malloc(sizeof(double) * kn * kn);
  double* kim = (double*)malloc(sizeof(double) * kn * kn);
  for (int k = 0; k < F->no; ++k) {
    orc_gabor_kernel(k * M_PI / F->no, P->gabor_lambda, P->gabor_sigma, R, kre, kim);
    for (int l = P->c_min; l <= smx; ++l) {
      int n = F->hl[l] * F->wl[l];
      F->ore[l][k] = (double*)malloc(sizeof(double) * n);
      F->oim[l][k] = (double*)malloc(sizeof(double) * n);
      F->ori[l][k] = (double*)malloc(sizeof(double) * n);
      gabor_fw(F->hl[l], F->wl[l], F->pyr[0][l], kre, kim, R, F->ore[l][k], F->oim[l][k], F->ori[l][k]);
    }
  }
  free(kre);
  free(kim);
  int hS = F->hl[F->sS], wS = F->wl[F->sS], nS = hS * wS, nch = 3 + F->no;
  for (int f = 0; f < nch; ++f) F->acc[f] = (double*)calloc(nS, sizeof(double));
  int big = F->hl[P->c_min] * F->wl[P->c_min];
  double *up = (double*)malloc(sizeof(double) * big), *map = (double*)malloc(sizeof(double) * big);
  double *nm = (double*)malloc(sizeof(double) * big), *tmp = (double*)malloc(sizeof(double) * big);
  for (int c = P->c_min; c <= P->c_max; ++c)
    for (int d = P->d_min; d <= P->d_max; ++d)
      for (int f = 0; f < nch; ++f) {
        int s = c + d, nc = F->hl[c] * F->wl[c];
        const double* cen = f < 3 ? F->pyr[f][c] : F->ori[c][f - 3];
        const double* sur = f < 3 ? F->pyr[f][s] : F->ori[s][f - 3];
        up_fw(F->hl[s], F->wl[s], sur, F->hl[c], F->wl[c], up);
        int opp = (f == 1 || f == 2) && P->cs_opponent_sum;
        for (int i = 0; i < nc; ++i) map[i] = fabs(opp ? cen[i] + up[i] : cen[i] - up[i]);
        nstat st;
        norm_fw(F->hl[c], F->wl[c], map, P->norm_tile, P->norm_flat, nm, &st);
        if (g_tie_delta > 0 && !st.flat)
          for (int i = 0; i < nc; ++i)
            if (map[i] > 0 && map[i] < g_tie_delta * (st.mx - st.mn)) g_ties[2]++;
        free(st.targ);
        for (int l = c; l < F->sS; ++l) {
          reduce_fw(F->hl[l], F->wl[l], nm, tmp);
          memcpy(nm, tmp, sizeof(double) * F->hl[l + 1] * F->wl[l + 1]);
        }
        for (int i = 0; i < nS; ++i) F->acc[f][i] += nm[i];
      }
  free(up);
  free(map);
  free(nm);
  free(tmp);
  for (int k = 0; k < 4; ++k) {
    F->C[k] = (double*)calloc(nS, sizeof(double));
    F->NC[k] = (double*)malloc(sizeof(double) * nS);
  }
  for (int k = 0; k < 3; ++k) memcpy(F->C[k], F->acc[k], sizeof(double) * nS);
  for (int k = 0; k < F->no; ++k) {
    F->NT[k] = (double*)malloc(sizeof(double) * nS);
    norm_fw(hS, wS, F->acc[3 + k], P->norm_tile, P->norm_flat, F->NT[k], &F->nT[k]);
    for (int i = 0; i < nS; ++i) F->C[3][i] += F->NT[k][i];
  }
  F->S = (double*)calloc(nS, sizeof(double));
  for (int k = 0; k < 4; ++k) {
    norm_fw(hS, wS, F->C[k], P->norm_tile, P->norm_flat, F->NC[k], &F->nC[k]);
    for (int i = 0; i < nS; ++i) F->S[i] += P->w[k] * F->NC[k][i];
  }
  F->sal = (double*)malloc(sizeof(double) * H * W);
  up_fw(hS, wS, F->S, H, W, F->sal);
  F->salarg = 0;
  for (int i = 1; i < H * W; ++i)
    if (F->sal[i] > F->sal[F->salarg]) F->salarg = i;
  F->salmx = F->sal[F->salarg] > 0 ? F->sal[F->salarg] : 0.0;
}

static void fwd_free(fwd_t* F) {
  const orc_params* P = F->P;
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < F->L; ++l) free(F->pyr[c][l]);
  for (int k = 0; k < F->no; ++k)
    for (int l = P->c_min; l <= P->c_max + P->d_max; ++l) {
      free(F->ore[l][k]);
      free(F->oim[l][k]);
      free(F->ori[l][k]);
    }
  for (int f = 0; f < 3 + F->no; ++f) free(F->acc[f]);
  for (int k = 0; k < 4; ++k) {
    free(F->C[k]);
    free(F->NC[k]);
    free(F->nC[k].targ);
  }
  for (int k = 0; k < F->no; ++k) {
    free(F->NT[k]);
    free(F->nT[k].targ);
  }
  free(F->S);
  free(F->sal);
}

/* q and the prior from the saliency (Secs. 5-6) */
static void prior_fw(const orc_params* P, const fwd_t* F, const double* fmap, double wf, double* q, double* prior) {
  int H = F->H, W = F->W, b = P->border_px;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int i = y * W + x, edge = y < b || y >= H - b || x < b || x >= W - b;
      q[i] = edge ? P->eps : (F->salmx > 0 ? F->sal[i] / F->salmx : 0.0);
      prior[i] = wf * fmap[i] + (1 - wf) * q[i];
    }
}

/* Sec. 6 recursion with its derivatives (forward mode) with respect to Q = sigma1^2
 * and R = sigma2^2, from P_{-1} = +inf (w_f = 0 and P_0 = Q at t = 0):
 *   w_f(t) = Q / (Q + R + P(t-1)),   P(t) = Q (R + P(t-1)) / (Q + R + P(t-1)).
 * Fills w_f, dw_f/dQ and dw_f/dR for t = t0 .. t0 + T - 1. */
void orc_kalman_chain(int t0, int T, double Q, double R, double* wf, double* dwf_dQ, double* dwf_dR) {
  double P = 0, dPq = 0, dPr = 0;
  for (int t = 0; t < t0 + T; ++t) {
    double w = 0, wq = 0, wr = 0, Pn, Pq, Pr;
    if (t == 0) {
      Pn = Q;
      Pq = 1;
      Pr = 0;
    } else {
      double den = Q + R + P, dq = 1 + dPq, dr = 1 + dPr;
      w = Q / den;
      wq = (den - Q * dq) / (den * den);
      wr = -Q * dr / (den * den);
      double num = Q * (R + P);
      Pn = num / den;
      Pq = ((R + P + Q * dPq) * den - num * dq) / (den * den);
      Pr = (Q * dr * den - num * dr) / (den * den);
    }
    if (t >= t0) {
      wf[t - t0] = w;
      dwf_dQ[t - t0] = wq;
      dwf_dR[t - t0] = wr;
    }
    P = Pn;
    dPq = Pq;
    dPr = Pr;
  }
}

/* Public (test support): counts of the forward's near-tie decisions over the
 * frames, margin below delta times the map's range (see g_ties). */
void orc_prior_clip_ties(const orc_params* P, int T, int H, int W, const double* rgb, double delta, long* ties) {
  size_t n = (size_t)H * W;
  g_tie_delta = delta;
  g_ties[0] = g_ties[1] = g_ties[2] = 0;
  for (int t = 0; t < T; ++t) {
    fwd_t F;
    fwd_run(&F, P, H, W, rgb + 3 * n * t);
    fwd_free(&F);
  }
  for (int k = 0; k < 3; ++k) ties[k] = g_ties[k];
  g_tie_delta = 0.0;
}

/* Public: saliency and prior of T consecutive floating-point frames (clip times
 * t0 .. t0 + T - 1), each (H, W, 3) in [0, 255]; fmap = the smoothed previous
 * masks (T, H, W), or NULL for none. */
void orc_prior_clip_f(const orc_params* P, int T, int t0, int H, int W, const double* rgb, const double* fmap,
                      double Q, double R, double* saliency, double* prior) {
  size_t n = (size_t)H * W;
  double *wf = (double*)malloc(sizeof(double) * T), *a = (double*)malloc(sizeof(double) * T),
         *b = (double*)malloc(sizeof(double) * T);
  double* zero = (double*)calloc(n, sizeof(double));
  double* q = (double*)malloc(sizeof(double) * n);
  orc_kalman_chain(t0, T, Q, R, wf, a, b);
  for (int t = 0; t < T; ++t) {
    fwd_t F;
    fwd_run(&F, P, H, W, rgb + 3 * n * t);
    prior_fw(P, &F, fmap ? fmap + n * t : zero, wf[t], q, prior + n * t);
    if (saliency) memcpy(saliency + n * t, F.sal, sizeof(double) * n);
    fwd_free(&F);
  }
  free(wf);
  free(a);
  free(b);
  free(zero);
  free(q);
}

/* One frame of the reverse pass: L = <g_prior, prior> + <g_sal, saliency> at a
 * fixed w_f.  Returns dL/dw_f; accumulates dL/dw into gw and writes dL/drgb. */
static double frame_grad(const orc_params* P, int H, int W, const double* rgb, const double* fmap, double wf,
                         const double* g_prior, const double* g_sal, double* grgb, double* gw) {
  fwd_t F;
  fwd_run(&F, P, H, W, rgb);
  int n = H * W, b = P->border_px;
  double* q = (double*)malloc(sizeof(double) * n);
  double* pr = (double*)malloc(sizeof(double) * n);
  prior_fw(P, &F, fmap, wf, q, pr);
  /* prior = wf f + (1 - wf) q */
  double gwf = 0;
  double* gsal = (double*)calloc(n, sizeof(double));
  for (int i = 0; i < n; ++i) gwf += g_prior[i] * (fmap[i] - q[i]);
  /* q = sal / max(sal) inside the border */
  if (F.salmx > 0) {
    double gm = 0;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int i = y * W + x;
        if (y < b || y >= H - b || x < b || x >= W - b) continue;
        double gq = g_prior[i] * (1 - wf);
        gsal[i] += gq / F.salmx;
        gm -= gq * F.sal[i] / (F.salmx * F.salmx);
      }
    gsal[F.salarg] += gm;
  }
  if (g_sal)
    for (int i = 0; i < n; ++i) gsal[i] += g_sal[i];
  int hS = F.hl[F.sS], wS = F.wl[F.sS], nS = hS * wS, nch = 3 + F.no;
  double* gS = (double*)calloc(nS, sizeof(double));
  up_bw(hS, wS, gS, H, W, gsal);
  /* S = sum_k w_k N(C_k) */
  double* gC[4];
  for (int k = 0; k < 4; ++k) {
    double* gN = (double*)malloc(sizeof(double) * nS);
    for (int i = 0; i < nS; ++i) {
      gw[k] += gS[i] * F.NC[k][i];
      gN[i] = P->w[k] * gS[i];
    }
    gC[k] = (double*)calloc(nS, sizeof(double));
    norm_bw(hS, wS, F.C[k], &F.nC[k], gN, gC[k]);
    free(gN);
  }
  double* gacc[11];
  for (int f = 0; f < nch; ++f) gacc[f] = (double*)calloc(nS, sizeof(double));
  for (int k = 0; k < 3; ++k) memcpy(gacc[k], gC[k], sizeof(double) * nS);
  for (int k = 0; k < F.no; ++k) norm_bw(hS, wS, F.acc[3 + k], &F.nT[k], gC[3], gacc[3 + k]);
  /* across-scale sums and center-surround maps */
  double* gpyr[3][16];
  double* gori[16][8];
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < F.L; ++l) gpyr[c][l] = (double*)calloc(F.hl[l] * F.wl[l], sizeof(double));
  int smx = P->c_max + P->d_max;
  for (int k = 0; k < F.no; ++k)
    for (int l = P->c_min; l <= smx; ++l) gori[l][k] = (double*)calloc(F.hl[l] * F.wl[l], sizeof(double));
  int big = F.hl[P->c_min] * F.wl[P->c_min];
  double *up = (double*)malloc(sizeof(double) * big), *map = (double*)malloc(sizeof(double) * big);
  double *nm = (double*)malloc(sizeof(double) * big), *gl = (double*)malloc(sizeof(double) * big);
  double *gt = (double*)malloc(sizeof(double) * big), *gv = (double*)malloc(sizeof(double) * big);
  for (int c = P->c_min; c <= P->c_max; ++c)
    for (int d = P->d_min; d <= P->d_max; ++d)
      for (int f = 0; f < nch; ++f) {
        int s = c + d, nc = F.hl[c] * F.wl[c];
        const double* cen = f < 3 ? F.pyr[f][c] : F.ori[c][f - 3];
        const double* sur = f < 3 ? F.pyr[f][s] : F.ori[s][f - 3];
        up_fw(F.hl[s], F.wl[s], sur, F.hl[c], F.wl[c], up);
        int opp = (f == 1 || f == 2) && P->cs_opponent_sum;
        for (int i = 0; i < nc; ++i) map[i] = fabs(opp ? cen[i] + up[i] : cen[i] - up[i]);
        nstat st;
        norm_fw(F.hl[c], F.wl[c], map, P->norm_tile, P->norm_flat, nm, &st);
        /* gradient of the map's contribution at sigma_S, back down to scale c */
        memcpy(gl, gacc[f], sizeof(double) * nS);
        for (int l = F.sS - 1; l >= c; --l) {
          memset(gt, 0, sizeof(double) * F.hl[l] * F.wl[l]);
          reduce_bw(F.hl[l], F.wl[l], gl, gt);
          memcpy(gl, gt, sizeof(double) * F.hl[l] * F.wl[l]);
        }
        memset(gv, 0, sizeof(double) * nc);
        norm_bw(F.hl[c], F.wl[c], map, &st, gl, gv);
        free(st.targ);
        double* gcen = f < 3 ? gpyr[f][c] : gori[c][f - 3];
        double* gsur = f < 3 ? gpyr[f][s] : gori[s][f - 3];
        for (int i = 0; i < nc; ++i) {
          double a = opp ? cen[i] + up[i] : cen[i] - up[i];
          double sg = a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0);
          gcen[i] += gv[i] * sg;
          gt[i] = gv[i] * sg * (opp ? 1.0 : -1.0);
        }
        up_bw(F.hl[s], F.wl[s], gsur, F.hl[c], F.wl[c], gt);
      }
  /* Gabor magnitudes -> intensity pyramid */
  int Rg = P->gabor_radius, kn = 2 * Rg + 1;
  double* kre = (double*)malloc(sizeof(double) * kn * kn);
  double* kim = (double*)malloc(sizeof(double) * kn * kn);
  for (int k = 0; k < F.no; ++k) {
    orc_gabor_kernel(k * M_PI / F.no, P->gabor_lambda, P->gabor_sigma, Rg, kre, kim);
    for (int l = P->c_min; l <= smx; ++l)
      gabor_bw(F.hl[l], F.wl[l], kre, kim, Rg, F.ore[l][k], F.oim[l][k], gori[l][k], gpyr[0][l]);
  }
  /* pyramid, top level down to the base */
  for (int c = 0; c < 3; ++c)
    for (int l = F.L - 1; l >= 1; --l) reduce_bw(F.hl[l - 1], F.wl[l - 1], gpyr[c][l], gpyr[c][l - 1]);
  memset(grgb, 0, sizeof(double) * 3 * n);
  features_bw(H, W, rgb, F.smax, gpyr[0][0], gpyr[1][0], gpyr[2][0], grgb);
  free(kre);
  free(kim);
  free(up);
  free(map);
  free(nm);
  free(gl);
  free(gt);
  free(gv);
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < F.L; ++l) free(gpyr[c][l]);
  for (int k = 0; k < F.no; ++k)
    for (int l = P->c_min; l <= smx; ++l) free(gori[l][k]);
  for (int f = 0; f < nch; ++f) free(gacc[f]);
  for (int k = 0; k < 4; ++k) free(gC[k]);
  free(gS);
  free(gsal);
  free(q);
  free(pr);
  fwd_free(&F);
  return gwf;
}

/* Public: gradient of L = sum_t <g_prior_t, prior_t> + <g_sal_t, saliency_t> over the
 * clip of orc_prior_clip_f with respect to the frames (grgb, T*H*W*3; NULL to skip
 * nothing: it is always written), the channel weights (gw[4]), Q and R (through
 * w_f(t) and the whole variance recursion). */
void orc_prior_clip_grad(const orc_params* P, int T, int t0, int H, int W, const double* rgb, const double* fmap,
                         double Q, double R, const double* g_prior, const double* g_sal, double* grgb, double* gw,
                         double* gQ, double* gR) {
  size_t n = (size_t)H * W;
  double *wf = (double*)malloc(sizeof(double) * T), *a = (double*)malloc(sizeof(double) * T),
         *b = (double*)malloc(sizeof(double) * T);
  double* zero = (double*)calloc(n, sizeof(double));
  orc_kalman_chain(t0, T, Q, R, wf, a, b);
  for (int k = 0; k < 4; ++k) gw[k] = 0;
  *gQ = *gR = 0;
  for (int t = 0; t < T; ++t) {
    double gwf = frame_grad(P, H, W, rgb + 3 * n * t, fmap ? fmap + n * t : zero, wf[t], g_prior + n * t,
                            g_sal ? g_sal + n * t : NULL, grgb + 3 * n * t, gw);
    *gQ += gwf * a[t];
    *gR += gwf * b[t];
  }
  free(wf);
  free(a);
  free(b);
  free(zero);
}
