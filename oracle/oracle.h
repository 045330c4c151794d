/*
 * oracle.h -- plain, slow FP64 CPU reference ("the oracle") for the per-frame
 * path of Akamine, Fukuchi, Kimura and Takagi, "Fully automatic extraction of
 * salient objects from videos in near real-time" (arXiv:1008.0502).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or helper with the CUDA path and includes no GPU header.
 *
 * Images are row-major, pixel (y, x) at index y*W + x.  RGB8 frames are
 * interleaved H x W x 3.  Grid n-link capacities are nbr/2 planes of H x W
 * int32, ordered E (x+1), S (y+1), SE (x+1, y+1), SW (x-1, y+1); entries whose
 * neighbour falls outside the grid are ignored.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  int levels;          /* pyramid images incl. the base (sigma = 0 .. levels-1) */
  int c_min, c_max;    /* center scales */
  int d_min, d_max;    /* surround s = c + d */
  int n_orient;        /* Gabor orientations theta_k = k*pi/n_orient */
  double gabor_lambda; /* carrier wavelength (px at each level) */
  double gabor_sigma;  /* isotropic envelope sigma (px) */
  int gabor_radius;    /* taps = 2*radius+1 per axis */
  int norm_tile;       /* N(.) local-maximum tile side */
  double norm_flat;    /* a map whose range is <= this is treated as flat: N = 0 */
  double w[4];         /* channel weights: I, RG, BY, O */
  int cs_opponent_sum; /* 1: |RG(c) + up RG(s)| (literal opponent form), 0: |RG(c) - up RG(s)| */
  int border_px;       /* frame-edge band where the saliency prior is eps */
  double sigma1, sigma2; /* Kalman noise std-devs (Sec. 6, values of Sec. 8.1) */
  double f_sigma;      /* Gaussian smoothing of the previous mask */
  int f_radius;
  double eps;          /* clamp for the logs and the border prior */
  double lambda_u;     /* weight of the colour likelihood psi_1 */
  double lambda_p;     /* Potts constant xi_2 */
  double lambda_s;     /* contrast term psi_2 weight */
  double sigma_I;      /* contrast term intensity scale */
  double cap_scale;    /* K: integer capacity = round(K * cost) */
  int neighbourhood;   /* 4 or 8 */
  int gmm_components;  /* Gaussians per label in the colour likelihood: 1 or 3 */
  int em_iters;        /* EM iterations when gmm_components > 1 */
  int kmeans_iters;    /* Lloyd iterations of the k-means start of the EM */
  int gmm_update;      /* 1: a frame's EM starts from the previous frame's mixtures */
} orc_params;

/* A prior-weighted Gaussian mixture over C = RGB/255 (one label). */
typedef struct orc_gmm {
  int M;
  double pi[3];
  double mu[3][3];
  double cov[3][3][3];
} orc_gmm;

/* Debug outputs of orc_saliency_ex (any pointer may be NULL). */
typedef struct orc_saliency_debug {
  double* pyr;   /* 3 channels (I, RG, BY) x sum over levels of level area */
  double* ori;   /* n_orient x sum over sigma in [c_min, c_max+d_max] of level area */
  double* consp; /* 4 x (area at sigma_S = c_max): N(C_I), N(C_RG), N(C_BY), N(C_O) */
  double* S;     /* area at sigma_S: the combined saliency map before upsampling */
} orc_saliency_debug;

int orc_level_dim(int n, int level);

/* --- Sec. 3 / Sec. 7.2: saliency map --- */
void orc_features(int H, int W, const uint8_t* rgb, double* I, double* RG, double* BY);
void orc_reduce(int h, int w, const double* in, double* out);
void orc_gabor_kernel(double theta, double lambda, double sigma, int radius, double* kre, double* kim);
void orc_gabor(int h, int w, const double* in, const double* kre, const double* kim, int radius,
               double* out);
void orc_upsample(int hs, int ws, const double* src, int hd, int wd, double* dst);
void orc_normalize(int h, int w, const double* v, int tile, double flat, double* out);
/* Steps 4-6 (center-surround, N(.), weighted addition) on given pyramids laid out as
 * orc_saliency_debug's pyr and ori; writes the four N(C_k) maps (consp, may be NULL) and S at
 * sigma_S = c_max. */
void orc_saliency_compose(const orc_params* P, int H, int W, const double* pyr, const double* ori,
                          double* consp, double* S);
void orc_saliency_ex(const orc_params* P, int H, int W, const uint8_t* rgb, double* saliency,
                     orc_saliency_debug* dbg);
void orc_saliency(const orc_params* P, int H, int W, const uint8_t* rgb, double* saliency);

/* --- Sec. 5 / Sec. 6: saliency prior and its Kalman update --- */
double orc_kalman_step(int t, double P_prev, double sigma1, double sigma2, double* w_f);
void orc_smooth_mask(int H, int W, const uint8_t* mask, double sigma, int radius, double* f);
void orc_prior(const orc_params* P, int H, int W, const double* saliency, const uint8_t* prev_mask,
               double w_f, double* q, double* prior);

/* --- Sec. 4 / Sec. 5: MRF terms and graph capacities (Eqs. 1-4) --- */
int orc_colour_models(const double* prior, const uint8_t* rgb, int n, double mu[2][3],
                      double cov[2][3][3]);
void orc_terms(const orc_params* P, int H, int W, const uint8_t* rgb, const double* prior,
               int32_t* cs, int32_t* ct, int32_t* ncap, double* D0, double* D1);
void orc_gmm_init(const uint8_t* rgb, const double* w, int n, int M, int km_iters, orc_gmm* g);
double orc_gmm_loglik(const uint8_t* rgb, const double* w, int n, const orc_gmm* g);
void orc_gmm_em_step(const uint8_t* rgb, const double* w, int n, orc_gmm* g);
void orc_gmm_fit(const uint8_t* rgb, const double* w, int n, int M, int km_iters, int iters, orc_gmm* g);
void orc_terms_ex(const orc_params* P, int H, int W, const uint8_t* rgb, const double* prior,
                  int32_t* cs, int32_t* ct, int32_t* ncap, double* D0, double* D1, orc_gmm* mix, int from_mix);
double orc_gmm_logpdf(const orc_gmm* g, const double c[3]);
int32_t orc_ncap_value(const orc_params* P, int dsum, int diagonal);

/* --- Sec. 4: exact s-t min cut on the grid graph --- */
int64_t orc_maxflow_ek(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask);
int64_t orc_maxflow_bk(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask);
int64_t orc_cut_energy(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, const uint8_t* mask);
int64_t orc_bruteforce(int H, int W, int nbr, const int32_t* cs, const int32_t* ct,
                       const int32_t* ncap, uint8_t* mask_min, int32_t* n_argmin);

/* --- backward form (oracle_grad.c): float frames in [0, 255], Q = sigma1^2, R = sigma2^2 --- */
void orc_kalman_chain(int t0, int T, double Q, double R, double* wf, double* dwf_dQ, double* dwf_dR);
void orc_prior_clip_f(const orc_params* P, int T, int t0, int H, int W, const double* rgb, const double* fmap,
                      double Q, double R, double* saliency, double* prior);
void orc_prior_clip_ties(const orc_params* P, int T, int H, int W, const double* rgb, double delta, long* ties);
void orc_prior_clip_grad(const orc_params* P, int T, int t0, int H, int W, const double* rgb, const double* fmap,
                         double Q, double R, const double* g_prior, const double* g_sal, double* grgb, double* gw,
                         double* gQ, double* gR);

/* --- one frame of the whole method --- */
typedef struct orc_state {
  int t;               /* frame index */
  double P;            /* sigma^2_xi1(t-1) */
  uint8_t* prev_mask;  /* H*W, caller-owned */
  int gmm_valid;       /* gmm holds the previous frame's colour mixtures */
  orc_gmm gmm[2];      /* labels 0 and 1 */
} orc_state;

int64_t orc_push_frame(const orc_params* P, int H, int W, orc_state* st, const uint8_t* rgb,
                       double* saliency, double* prior, uint8_t* mask);

#ifdef __cplusplus
}
#endif
#endif
