"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It never imports the
CUDA path and the CUDA path never imports it.

Each wrapper takes and returns numpy arrays; parameter sets are plain dicts of
the ``orc_params`` fields (see :data:`CONFIG_SMALL` / :data:`CONFIG_VGA`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("c_min", C.c_int), ("c_max", C.c_int), ("d_min", C.c_int),
        ("d_max", C.c_int), ("n_orient", C.c_int), ("gabor_lambda", C.c_double),
        ("gabor_sigma", C.c_double), ("gabor_radius", C.c_int), ("norm_tile", C.c_int),
        ("norm_flat", C.c_double), ("w", C.c_double * 4), ("cs_opponent_sum", C.c_int),
        ("border_px", C.c_int), ("sigma1", C.c_double), ("sigma2", C.c_double),
        ("f_sigma", C.c_double), ("f_radius", C.c_int), ("eps", C.c_double),
        ("lambda_u", C.c_double), ("lambda_p", C.c_double), ("lambda_s", C.c_double),
        ("sigma_I", C.c_double), ("cap_scale", C.c_double), ("neighbourhood", C.c_int),
        ("gmm_components", C.c_int), ("em_iters", C.c_int), ("kmeans_iters", C.c_int), ("gmm_update", C.c_int),
    ]


class OrcGmm(C.Structure):
    _fields_ = [("M", C.c_int), ("pi", C.c_double * 3), ("mu", (C.c_double * 3) * 3),
                ("cov", ((C.c_double * 3) * 3) * 3)]


class OrcDebug(C.Structure):
    _fields_ = [("pyr", C.c_void_p), ("ori", C.c_void_p), ("consp", C.c_void_p), ("S", C.c_void_p)]


class OrcState(C.Structure):
    _fields_ = [("t", C.c_int), ("P", C.c_double), ("prev_mask", C.c_void_p), ("gmm_valid", C.c_int),
                ("gmm", OrcGmm * 2)]


# The 640x480 workload's parameters (9 images, centers 2..4, surrounds c+3..c+4,
# 8-neighbour grid) and the 160x120 one's (6 images, centers 1..2, c+2..c+3,
# 4-neighbour grid).  sigma1 = 0.03 and sigma2 = 0.035 are the paper's (Sec. 8.1).
CONFIG_VGA = dict(levels=9, c_min=2, c_max=4, d_min=3, d_max=4, n_orient=4, gabor_lambda=4.0,
                  gabor_sigma=2.0, gabor_radius=6, norm_tile=8, norm_flat=1e-5,
                  w=(1 / 3, 1 / 6, 1 / 6, 1 / 3), cs_opponent_sum=1, border_px=1, sigma1=0.03,
                  sigma2=0.035, f_sigma=2.0, f_radius=6, eps=1e-4, lambda_u=1.0, lambda_p=0.0,
                  lambda_s=1.5, sigma_I=0.05, cap_scale=1000.0, neighbourhood=8, gmm_components=1,
                  em_iters=5, kmeans_iters=3, gmm_update=1)
CONFIG_SMALL = dict(CONFIG_VGA, levels=6, c_min=1, c_max=2, d_min=2, d_max=3, neighbourhood=4)


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB_OVERRIDE: a separately built copy of the oracle (the planted-mistake
        # test builds copies with one deliberate slip each and checks that the pins fail)
        path = os.environ.get("ORACLE_LIB_OVERRIDE") or _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        vp = C.c_void_p
        L.orc_level_dim.argtypes = [C.c_int, C.c_int]
        L.orc_level_dim.restype = C.c_int
        for name, args in {
            "orc_features": [C.c_int, C.c_int, vp, vp, vp, vp],
            "orc_reduce": [C.c_int, C.c_int, vp, vp],
            "orc_gabor_kernel": [C.c_double, C.c_double, C.c_double, C.c_int, vp, vp],
            "orc_gabor": [C.c_int, C.c_int, vp, vp, vp, C.c_int, vp],
            "orc_upsample": [C.c_int, C.c_int, vp, C.c_int, C.c_int, vp],
            "orc_normalize": [C.c_int, C.c_int, vp, C.c_int, C.c_double, vp],
            "orc_saliency_ex": [P(OrcParams), C.c_int, C.c_int, vp, vp, P(OrcDebug)],
            "orc_saliency_compose": [P(OrcParams), C.c_int, C.c_int, vp, vp, vp, vp],
            "orc_smooth_mask": [C.c_int, C.c_int, vp, C.c_double, C.c_int, vp],
            "orc_prior": [P(OrcParams), C.c_int, C.c_int, vp, vp, C.c_double, vp, vp],
            "orc_terms": [P(OrcParams), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp],
            "orc_terms_ex": [P(OrcParams), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int],
        }.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = None
        L.orc_kalman_step.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, P(C.c_double)]
        L.orc_kalman_step.restype = C.c_double
        L.orc_colour_models.argtypes = [vp, vp, C.c_int, vp, vp]
        L.orc_colour_models.restype = C.c_int
        L.orc_ncap_value.argtypes = [P(OrcParams), C.c_int, C.c_int]
        L.orc_ncap_value.restype = C.c_int32
        for name in ("orc_maxflow_ek", "orc_maxflow_bk", "orc_cut_energy"):
            getattr(L, name).argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
            getattr(L, name).restype = C.c_int64
        L.orc_bruteforce.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, P(C.c_int32)]
        L.orc_bruteforce.restype = C.c_int64
        for name in ("orc_gmm_init", "orc_gmm_fit"):
            getattr(L, name).restype = None
        L.orc_gmm_init.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, P(OrcGmm)]
        L.orc_gmm_fit.argtypes = [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, P(OrcGmm)]
        L.orc_gmm_em_step.argtypes = [vp, vp, C.c_int, P(OrcGmm)]
        L.orc_gmm_em_step.restype = None
        L.orc_gmm_loglik.argtypes = [vp, vp, C.c_int, P(OrcGmm)]
        L.orc_gmm_loglik.restype = C.c_double
        L.orc_gmm_logpdf.argtypes = [P(OrcGmm), vp]
        L.orc_gmm_logpdf.restype = C.c_double
        L.orc_kalman_chain.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, vp, vp, vp]
        L.orc_kalman_chain.restype = None
        L.orc_prior_clip_f.argtypes = [P(OrcParams), C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, C.c_double,
                                       C.c_double, vp, vp]
        L.orc_prior_clip_f.restype = None
        L.orc_prior_clip_grad.argtypes = [P(OrcParams), C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, C.c_double,
                                          C.c_double, vp, vp, vp, vp, P(C.c_double), P(C.c_double)]
        L.orc_prior_clip_grad.restype = None
        L.orc_prior_clip_ties.argtypes = [P(OrcParams), C.c_int, C.c_int, C.c_int, vp, C.c_double, vp]
        L.orc_prior_clip_ties.restype = None
        L.orc_push_frame.argtypes = [P(OrcParams), C.c_int, C.c_int, P(OrcState), vp, vp, vp, vp]
        L.orc_push_frame.restype = C.c_int64
        _lib = L
    return _lib


def params(cfg: dict | None = None, **over) -> OrcParams:
    d = dict(CONFIG_VGA if cfg is None else cfg)
    d.update(over)
    p = OrcParams()
    for k, v in d.items():
        if k == "w":
            p.w = (C.c_double * 4)(*v)
        else:
            setattr(p, k, v)
    return p


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def level_dim(n: int, level: int) -> int:
    return lib().orc_level_dim(n, level)


def features(rgb):
    rgb = _c(rgb, np.uint8)
    H, W = rgb.shape[:2]
    I, RG, BY = (np.empty((H, W)) for _ in range(3))
    lib().orc_features(H, W, _p(rgb), _p(I), _p(RG), _p(BY))
    return I, RG, BY


def reduce(img):
    img = _c(img, np.float64)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2))
    lib().orc_reduce(h, w, _p(img), _p(out))
    return out


def gabor_kernel(theta, lam=4.0, sigma=2.0, radius=6):
    n = 2 * radius + 1
    kre, kim = np.empty((n, n)), np.empty((n, n))
    lib().orc_gabor_kernel(theta, lam, sigma, radius, _p(kre), _p(kim))
    return kre + 1j * kim


def gabor(img, theta, lam=4.0, sigma=2.0, radius=6):
    img = _c(img, np.float64)
    k = gabor_kernel(theta, lam, sigma, radius)
    kre, kim = _c(k.real, np.float64), _c(k.imag, np.float64)
    out = np.empty_like(img)
    lib().orc_gabor(img.shape[0], img.shape[1], _p(img), _p(kre), _p(kim), radius, _p(out))
    return out


def upsample(src, hd, wd):
    src = _c(src, np.float64)
    out = np.empty((hd, wd))
    lib().orc_upsample(src.shape[0], src.shape[1], _p(src), hd, wd, _p(out))
    return out


def normalize(v, tile=8, flat=1e-5):
    v = _c(v, np.float64)
    out = np.empty_like(v)
    lib().orc_normalize(v.shape[0], v.shape[1], _p(v), tile, flat, _p(out))
    return out


def saliency(rgb, cfg=None, debug=False, **over):
    """Saliency map (H x W, FP64).  With debug=True also returns a dict of the
    pyramid levels, orientation maps, normalised conspicuity maps and S."""
    rgb = _c(rgb, np.uint8)
    H, W = rgb.shape[:2]
    P = params(cfg, **over)
    out = np.empty((H, W))
    dbg = None
    bufs = {}
    if debug:
        dims = [(level_dim(H, l), level_dim(W, l)) for l in range(P.levels)]
        area = [h * w for h, w in dims]
        s_max = P.c_max + P.d_max
        bufs["pyr"] = np.zeros(3 * sum(area))
        bufs["ori"] = np.zeros(P.n_orient * sum(area[P.c_min:s_max + 1]))
        hS, wS = dims[P.c_max]
        bufs["consp"] = np.zeros(4 * hS * wS)
        bufs["S"] = np.zeros(hS * wS)
        dbg = OrcDebug(_p(bufs["pyr"]).value, _p(bufs["ori"]).value, _p(bufs["consp"]).value,
                       _p(bufs["S"]).value)
    lib().orc_saliency_ex(C.byref(P), H, W, _p(rgb), _p(out), C.byref(dbg) if dbg else None)
    if not debug:
        return out
    res = {"pyr": [[None] * P.levels for _ in range(3)], "ori": [dict() for _ in range(P.n_orient)]}
    off = 0
    for c in range(3):
        for l, (h, w) in enumerate(dims):
            res["pyr"][c][l] = bufs["pyr"][off:off + h * w].reshape(h, w)
            off += h * w
    off = 0
    for k in range(P.n_orient):
        for l in range(P.c_min, s_max + 1):
            h, w = dims[l]
            res["ori"][k][l] = bufs["ori"][off:off + h * w].reshape(h, w)
            off += h * w
    res["consp"] = bufs["consp"].reshape(4, hS, wS)
    res["S"] = bufs["S"].reshape(hS, wS)
    return out, res


def saliency_compose(pyr, ori, H, W, cfg=None, **over):
    """Steps 4-6 of the saliency map on given pyramids: pyr[c][l] (c = I, RG, BY; every level
    0..levels-1 of an H x W frame) and ori[k][l] (orientation k, levels c_min..c_max+d_max).
    Returns (consp (4, hS, wS): N(C_I), N(C_RG), N(C_BY), N(C_O); S (hS, wS))."""
    P = params(cfg, **over)
    dims = [(level_dim(H, l), level_dim(W, l)) for l in range(P.levels)]
    s_max = P.c_max + P.d_max
    flat_p = np.concatenate([np.asarray(pyr[c][l], np.float64).reshape(dims[l]).ravel()
                             for c in range(3) for l in range(P.levels)])
    flat_o = np.concatenate([np.asarray(ori[k][l], np.float64).reshape(dims[l]).ravel()
                             for k in range(P.n_orient) for l in range(P.c_min, s_max + 1)])
    hS, wS = dims[P.c_max]
    consp, S = np.empty((4, hS, wS)), np.empty((hS, wS))
    lib().orc_saliency_compose(C.byref(P), H, W, _p(flat_p), _p(flat_o), _p(consp), _p(S))
    return consp, S


def kalman_step(t, P_prev, sigma1=0.03, sigma2=0.035):
    wf = C.c_double()
    Pt = lib().orc_kalman_step(t, P_prev, sigma1, sigma2, C.byref(wf))
    return Pt, wf.value


def smooth_mask(mask, sigma=2.0, radius=6):
    mask = _c(mask, np.uint8)
    f = np.empty(mask.shape)
    lib().orc_smooth_mask(mask.shape[0], mask.shape[1], _p(mask), sigma, radius, _p(f))
    return f


def prior(sal, prev_mask, w_f, cfg=None, **over):
    sal = _c(sal, np.float64)
    H, W = sal.shape
    P = params(cfg, **over)
    q, pr = np.empty((H, W)), np.empty((H, W))
    pm = _c(prev_mask, np.uint8) if prev_mask is not None else None
    lib().orc_prior(C.byref(P), H, W, _p(sal), _p(pm) if pm is not None else None, w_f, _p(q), _p(pr))
    return q, pr


def kalman_chain(T, Q, R, t0=0):
    """w_f(t) and its derivatives dw_f/dQ, dw_f/dR for t = t0 .. t0+T-1 (Sec. 6, from
    P(-1) = inf), Q = sigma1^2, R = sigma2^2."""
    wf, dq, dr = np.empty(T), np.empty(T), np.empty(T)
    lib().orc_kalman_chain(t0, T, Q, R, _p(wf), _p(dq), _p(dr))
    return wf, dq, dr


def prior_clip(rgb, Q, R, fmap=None, t0=0, cfg=None, **over):
    """Backward form's forward (Secs. 3, 5, 6): saliency and Kalman-updated prior of
    T floating-point frames (T, H, W, 3) in [0, 255] at clip times t0..t0+T-1;
    fmap = smoothed previous masks (T, H, W) or None.  Returns (saliency, prior)."""
    rgb = _c(rgb, np.float64)
    T, H, W = rgb.shape[:3]
    fm = _c(fmap, np.float64) if fmap is not None else None
    P = params(cfg, **over)
    sal, pr = np.empty((T, H, W)), np.empty((T, H, W))
    lib().orc_prior_clip_f(C.byref(P), T, t0, H, W, _p(rgb), _p(fm) if fm is not None else None, Q, R,
                           _p(sal), _p(pr))
    return sal, pr


def prior_clip_ties(rgb, delta, cfg=None, **over):
    """Near-tie census of the forward on frames (T, H, W, 3): counts of decisions with
    margin below delta times the map's range -- N(.) minimum/maximum, tile maxima,
    center-surround signs (test support: FP32 and FP64 can disagree on those)."""
    rgb = _c(rgb, np.float64)
    T, H, W = rgb.shape[:3]
    P = params(cfg, **over)
    out = np.zeros(3, dtype=np.int64)
    lib().orc_prior_clip_ties(C.byref(P), T, H, W, _p(rgb), delta, _p(out))
    return out


def prior_clip_grad(rgb, Q, R, g_prior, g_sal=None, fmap=None, t0=0, cfg=None, **over):
    """Gradient of L = sum_t <g_prior_t, prior_t> + <g_sal_t, saliency_t> with respect to
    the frames, the four channel weights w, Q and R.  Returns (g_rgb, g_w (4,), g_Q, g_R)."""
    rgb = _c(rgb, np.float64)
    T, H, W = rgb.shape[:3]
    fm = _c(fmap, np.float64) if fmap is not None else None
    gp = _c(g_prior, np.float64)
    gs = _c(g_sal, np.float64) if g_sal is not None else None
    P = params(cfg, **over)
    grgb, gw = np.empty((T, H, W, 3)), np.empty(4)
    gQ, gR = C.c_double(), C.c_double()
    lib().orc_prior_clip_grad(C.byref(P), T, t0, H, W, _p(rgb), _p(fm) if fm is not None else None, Q, R,
                              _p(gp), _p(gs) if gs is not None else None, _p(grgb), _p(gw), C.byref(gQ),
                              C.byref(gR))
    return grgb, gw, gQ.value, gR.value


def colour_models(prior_map, rgb):
    prior_map = _c(prior_map, np.float64)
    rgb = _c(rgb, np.uint8)
    mu, cov = np.empty((2, 3)), np.empty((2, 3, 3))
    deg = lib().orc_colour_models(_p(prior_map), _p(rgb), prior_map.size, _p(mu), _p(cov))
    return mu, cov, deg


def terms(rgb, prior_map, cfg=None, **over):
    """Integer graph of one frame: (cs, ct, ncap[nbr/2], D0, D1)."""
    rgb = _c(rgb, np.uint8)
    prior_map = _c(prior_map, np.float64)
    H, W = prior_map.shape
    P = params(cfg, **over)
    cs, ct = np.empty((H, W), np.int32), np.empty((H, W), np.int32)
    nc = np.empty((P.neighbourhood // 2, H, W), np.int32)
    D0, D1 = np.empty((H, W)), np.empty((H, W))
    lib().orc_terms(C.byref(P), H, W, _p(rgb), _p(prior_map), _p(cs), _p(ct), _p(nc), _p(D0), _p(D1))
    return cs, ct, nc, D0, D1


def terms_from(rgb, prior_map, mix=None, cfg=None, **over):
    """terms() with the colour mixtures carried between frames: the EM of each label starts
    from mix (a pair of OrcGmm, e.g. the previous frame's) when it is given, else from the
    k-means start.  Returns (cs, ct, ncap, mixtures fitted here)."""
    rgb = _c(rgb, np.uint8)
    prior_map = _c(prior_map, np.float64)
    H, W = prior_map.shape
    P = params(cfg, **over)
    cs, ct = np.empty((H, W), np.int32), np.empty((H, W), np.int32)
    nc = np.empty((P.neighbourhood // 2, H, W), np.int32)
    out = (OrcGmm * 2)()
    if mix is not None:
        out[0], out[1] = mix[0], mix[1]
    lib().orc_terms_ex(C.byref(P), H, W, _p(rgb), _p(prior_map), _p(cs), _p(ct), _p(nc), None, None, out,
                       1 if mix is not None else 0)
    return cs, ct, nc, (out[0], out[1])


def _gmm_out(g):
    M = g.M
    return (np.array(g.pi[:M]), np.array([[g.mu[m][k] for k in range(3)] for m in range(M)]),
            np.array([[[g.cov[m][k][j] for j in range(3)] for k in range(3)] for m in range(M)]))


def gmm_fit(rgb, w, M=3, iters=5, km_iters=3):
    """Prior-weighted GMM over C = RGB/255: returns (pi, mu, cov)."""
    rgb = _c(rgb, np.uint8).reshape(-1, 3)
    w = _c(w, np.float64).ravel()
    g = OrcGmm()
    lib().orc_gmm_fit(_p(rgb), _p(w), w.size, M, km_iters, iters, C.byref(g))
    return _gmm_out(g)


def gmm_init(rgb, w, M=3, km_iters=3):
    """The EM's k-means start (seeds, Lloyd iterations, mixture of the partition): (pi, mu, cov)."""
    rgb = _c(rgb, np.uint8).reshape(-1, 3)
    w = _c(w, np.float64).ravel()
    g = OrcGmm()
    lib().orc_gmm_init(_p(rgb), _p(w), w.size, M, km_iters, C.byref(g))
    return _gmm_out(g)


def gmm_em_trace(rgb, w, M=3, iters=5, km_iters=3):
    """Weighted log-likelihood after init and after each EM step."""
    rgb = _c(rgb, np.uint8).reshape(-1, 3)
    w = _c(w, np.float64).ravel()
    g = OrcGmm()
    lib().orc_gmm_init(_p(rgb), _p(w), w.size, M, km_iters, C.byref(g))
    out = [lib().orc_gmm_loglik(_p(rgb), _p(w), w.size, C.byref(g))]
    for _ in range(iters):
        lib().orc_gmm_em_step(_p(rgb), _p(w), w.size, C.byref(g))
        out.append(lib().orc_gmm_loglik(_p(rgb), _p(w), w.size, C.byref(g)))
    return out


def gmm_em_from(rgb, w, pi, mu, cov, iters=1):
    """iters EM steps from the mixture (pi, mu, cov): returns (pi, mu, cov)."""
    rgb = _c(rgb, np.uint8).reshape(-1, 3)
    w = _c(w, np.float64).ravel()
    g = OrcGmm()
    g.M = len(pi)
    for m in range(g.M):
        g.pi[m] = pi[m]
        for k in range(3):
            g.mu[m][k] = mu[m][k]
            for j in range(3):
                g.cov[m][k][j] = cov[m][k][j]
    for _ in range(iters):
        lib().orc_gmm_em_step(_p(rgb), _p(w), w.size, C.byref(g))
    return _gmm_out(g)


def gmm_logpdf(pi, mu, cov, c):
    g = OrcGmm()
    g.M = len(pi)
    for m in range(g.M):
        g.pi[m] = pi[m]
        for k in range(3):
            g.mu[m][k] = mu[m][k]
            for j in range(3):
                g.cov[m][k][j] = cov[m][k][j]
    c = _c(c, np.float64)
    return lib().orc_gmm_logpdf(C.byref(g), _p(c))


def ncap_value(dsum, diagonal, cfg=None, **over):
    P = params(cfg, **over)
    return lib().orc_ncap_value(C.byref(P), int(dsum), int(diagonal))


def _graph_args(cs, ct, ncap):
    cs, ct, ncap = _c(cs, np.int32), _c(ct, np.int32), _c(ncap, np.int32)
    H, W = cs.shape
    return cs, ct, ncap, H, W, 2 * ncap.shape[0]


def maxflow(cs, ct, ncap, method="bk"):
    """Max-flow value and minimal source set (mask, 1 = source side = object)."""
    cs, ct, ncap, H, W, nbr = _graph_args(cs, ct, ncap)
    mask = np.empty((H, W), np.uint8)
    fn = {"bk": lib().orc_maxflow_bk, "ek": lib().orc_maxflow_ek}[method]
    v = fn(H, W, nbr, _p(cs), _p(ct), _p(ncap), _p(mask))
    return int(v), mask


def cut_energy(cs, ct, ncap, mask):
    cs, ct, ncap, H, W, nbr = _graph_args(cs, ct, ncap)
    mask = _c(mask, np.uint8)
    return int(lib().orc_cut_energy(H, W, nbr, _p(cs), _p(ct), _p(ncap), _p(mask)))


def bruteforce(cs, ct, ncap):
    cs, ct, ncap, H, W, nbr = _graph_args(cs, ct, ncap)
    mask = np.empty((H, W), np.uint8)
    cnt = C.c_int32()
    v = lib().orc_bruteforce(H, W, nbr, _p(cs), _p(ct), _p(ncap), _p(mask), C.byref(cnt))
    return int(v), mask, cnt.value


class Segmenter:
    """The oracle's whole per-frame method with its temporal state."""

    def __init__(self, H, W, cfg=None, **over):
        self.H, self.W = H, W
        self.P = params(cfg, **over)
        self.prev = np.zeros((H, W), np.uint8)
        self.st = OrcState(0, 0.0, _p(self.prev).value)

    def push(self, rgb):
        rgb = _c(rgb, np.uint8)
        sal, pr = np.empty((self.H, self.W)), np.empty((self.H, self.W))
        mask = np.empty((self.H, self.W), np.uint8)
        cut = lib().orc_push_frame(C.byref(self.P), self.H, self.W, C.byref(self.st), _p(rgb),
                                   _p(sal), _p(pr), _p(mask))
        return sal, pr, mask, int(cut)

    def set_state(self, t, P_var, prev_mask):
        """Temporal state of Sec. 6 (frame index, variance P_{t-1}, previous mask)."""
        self.prev[:] = _c(prev_mask, np.uint8).reshape(self.H, self.W)
        self.st.t = int(t)
        self.st.P = float(P_var)

    @property
    def t(self):
        return self.st.t

    @property
    def P_var(self):
        return self.st.P
