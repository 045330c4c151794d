"""Pins of the FP64 oracle against things other than itself.

Each test fixes one function of the oracle with a closed form, an invariant,
an independent library routine (scipy / numpy) or brute force, so that a
plausible slip in the oracle (dropped term, wrong sign or index, transposed
operand) fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy import ndimage, stats
from scipy.sparse.csgraph import maximum_flow

import oracle as O
from paper_1008_0502_b300 import synth

BINOM = np.array([1, 4, 6, 4, 1], float) / 16.0


# ---------------------------------------------------------------- features
def test_features_closed_forms():
    px = np.array([[[255, 0, 0], [255, 255, 0], [0, 0, 255], [0, 255, 0], [90, 90, 90],
                    [5, 5, 5]]], np.uint8)
    I, RG, BY = O.features(px)
    assert np.allclose(I[0], px[0].sum(1) / 765.0, rtol=0, atol=1e-15)
    # pure red: rn=3 -> R=3, G=0, B=0, Y=0
    assert RG[0, 0] == 3.0 and BY[0, 0] == 0.0
    # pure yellow: rn=gn=1.5 -> R=G=0.75, Y=1.5, B=0
    assert RG[0, 1] == 0.0 and BY[0, 1] == -1.5
    # pure blue: B=3, Y=0
    assert RG[0, 2] == 0.0 and BY[0, 2] == 3.0
    # pure green: G=3 -> RG=-3; Y = (0+3)/2 - 3/2 - 0 = 0
    assert RG[0, 3] == -3.0 and BY[0, 3] == 0.0
    # grey gives exactly zero opponents; a pixel at or below a tenth of the
    # maximum intensity (15 <= 76.5) gets no hue at all
    assert RG[0, 4] == 0.0 and BY[0, 4] == 0.0
    assert RG[0, 5] == 0.0 and BY[0, 5] == 0.0


def test_features_hue_threshold_is_integer_exact():
    # max sum = 765; a pixel with sum 76 is below a tenth, 77 is above
    px = np.array([[[255, 255, 255], [76, 0, 0], [77, 0, 0]]], np.uint8)
    _, RG, _ = O.features(px)
    assert RG[0, 1] == 0.0 and RG[0, 2] == 3.0
    # the boundary itself: max sum 300, a pixel with sum exactly 30 (10 x 30 = 300) is
    # not above a tenth, so it gets no hue (the test is strict); sum 31 does
    px = np.array([[[100, 100, 100], [30, 0, 0], [0, 31, 0], [0, 0, 30]]], np.uint8)
    _, RG, BY = O.features(px)
    assert RG[0, 1] == 0.0 and BY[0, 1] == 0.0
    assert RG[0, 2] == -3.0
    assert RG[0, 3] == 0.0 and BY[0, 3] == 0.0


def test_grey_image_has_no_colour_opponents():
    g = synth.noise_background(np.random.default_rng(3), 40, 50)
    rgb = np.repeat(g[:, :, None], 3, 2)
    _, RG, BY = O.features(rgb)
    assert not RG.any() and not BY.any()


# ---------------------------------------------------------------- pyramid
def test_reduce_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    for h, w in [(17, 23), (8, 8), (5, 3), (1, 7), (2, 2)]:
        img = rng.random((h, w))
        ref = ndimage.correlate(img, np.outer(BINOM, BINOM), mode="nearest")[::2, ::2]
        assert O.reduce(img).shape == ((h + 1) // 2, (w + 1) // 2)
        np.testing.assert_allclose(O.reduce(img), ref, rtol=0, atol=1e-14)


def test_reduce_impulse_closed_form():
    img = np.zeros((20, 20))
    img[8, 10] = 1.0  # even position -> taps 1,6,1 per axis
    out = O.reduce(img)
    exp = np.zeros((10, 10))
    exp[3:6, 4:7] = np.outer([1, 6, 1], [1, 6, 1]) / 256.0
    np.testing.assert_allclose(out, exp, atol=1e-16)
    img = np.zeros((20, 20))
    img[9, 11] = 1.0  # odd position -> taps 4,4 per axis
    out = O.reduce(img)
    exp = np.zeros((10, 10))
    exp[4:6, 5:7] = 16 / 256.0
    np.testing.assert_allclose(out, exp, atol=1e-16)


def test_reduce_constant_and_linear():
    c = np.full((13, 9), 0.37)
    np.testing.assert_allclose(O.reduce(c), 0.37, rtol=0, atol=1e-15)
    a, b = np.random.default_rng(1).random((2, 11, 14))
    np.testing.assert_allclose(O.reduce(2 * a - 3 * b), 2 * O.reduce(a) - 3 * O.reduce(b), atol=1e-14)


def test_level_dims_ceil_halving():
    assert [O.level_dim(640, l) for l in range(9)] == [640, 320, 160, 80, 40, 20, 10, 5, 3]
    assert [O.level_dim(480, l) for l in range(9)] == [480, 240, 120, 60, 30, 15, 8, 4, 2]


# ---------------------------------------------------------------- Gabor
@pytest.mark.parametrize("k", range(4))
def test_gabor_kernel_zero_mean_rank2_normalised(k):
    th = k * np.pi / 4
    g = O.gabor_kernel(th)
    assert abs(g.sum()) < 1e-15
    sv = np.linalg.svd(g, compute_uv=False)
    assert sv[2] < 1e-12 * sv[0]              # rank 2: modulated Gaussian minus DC Gaussian
    # envelope: |k| + DC part equals the normalised Gaussian times |carrier| = 1
    u = np.arange(-6, 7)
    G = np.exp(-(u[None, :] ** 2 + u[:, None] ** 2) / 8.0)
    kappa = (G * np.exp(1j * np.pi / 2 * (u[None, :] * np.cos(th) + u[:, None] * np.sin(th)))).sum() / G.sum()
    np.testing.assert_allclose(np.abs(g + kappa * G / G.sum()), G / G.sum(), atol=1e-15)


def test_gabor_matches_scipy_correlate_and_constant_is_zero():
    rng = np.random.default_rng(2)
    img = rng.random((31, 27))
    for k in range(4):
        th = k * np.pi / 4
        g = O.gabor_kernel(th)
        re = ndimage.correlate(img, g.real, mode="nearest")
        im = ndimage.correlate(img, g.imag, mode="nearest")
        np.testing.assert_allclose(O.gabor(img, th), np.hypot(re, im), atol=1e-13)
        assert np.abs(O.gabor(np.full((20, 20), 0.8), th)).max() < 1e-14


def test_gabor_orientation_selectivity_and_transpose():
    y, x = np.mgrid[0:48, 0:48]
    grating = 0.5 + 0.5 * np.cos(2 * np.pi * x / 4.0)  # varies along x: theta = 0
    r0 = O.gabor(grating, 0.0)[16:32, 16:32].mean()
    r90 = O.gabor(grating, np.pi / 2)[16:32, 16:32].mean()
    assert r0 > 50 * r90
    img = np.random.default_rng(5).random((24, 24))
    np.testing.assert_allclose(O.gabor(img.T, np.pi / 2), O.gabor(img, 0.0).T, atol=1e-13)
    np.testing.assert_allclose(O.gabor(img.T, np.pi / 4), O.gabor(img, np.pi / 4).T, atol=1e-13)
    np.testing.assert_allclose(O.gabor(img.T, 3 * np.pi / 4), O.gabor(img, 3 * np.pi / 4).T, atol=1e-13)


# ---------------------------------------------------------------- upsample
def test_upsample_matches_map_coordinates():
    rng = np.random.default_rng(4)
    src = rng.random((5, 7))
    for hd, wd in [(9, 13), (20, 28), (5, 7), (3, 4)]:
        sy = np.clip((np.arange(hd) + 0.5) * 5 / hd - 0.5, 0, 4)
        sx = np.clip((np.arange(wd) + 0.5) * 7 / wd - 0.5, 0, 6)
        yy, xx = np.meshgrid(sy, sx, indexing="ij")
        ref = ndimage.map_coordinates(src, [yy, xx], order=1, mode="nearest")
        np.testing.assert_allclose(O.upsample(src, hd, wd), ref, atol=1e-14)
    np.testing.assert_allclose(O.upsample(src, 5, 7), src, atol=1e-15)


# ---------------------------------------------------------------- N(.)
def test_normalize_single_peak_and_two_peaks():
    v = np.zeros((16, 24))  # 2 x 3 tiles of 8
    v[3, 3] = 5.0
    np.testing.assert_allclose(O.normalize(v), v / 5.0)  # mbar = 0
    v[12, 20] = 5.0  # second equal peak in another tile: mbar = 1/5
    np.testing.assert_allclose(O.normalize(v), v / 5.0 * (1 - 1 / 5) ** 2)


def test_normalize_matches_numpy_tiles_and_is_affine_invariant():
    rng = np.random.default_rng(6)
    for h, w in [(30, 40), (15, 20), (8, 8), (3, 2), (1, 1)]:
        v = rng.random((h, w))
        mn, mx = v.min(), v.max()
        ref = np.zeros_like(v)
        if mx > mn:
            vp = (v - mn) / (mx - mn)
            pad = np.zeros((-(-h // 8) * 8, -(-w // 8) * 8))
            pad[:h, :w] = vp
            tm = pad.reshape(pad.shape[0] // 8, 8, pad.shape[1] // 8, 8).max(axis=(1, 3))
            nt = tm.size
            mbar = (tm.sum() - 1) / (nt - 1) if nt > 1 else 0.0
            ref = vp * (1 - mbar) ** 2
        np.testing.assert_allclose(O.normalize(v), ref, atol=1e-14)
        np.testing.assert_allclose(O.normalize(3.5 * v + 1.25), O.normalize(v), atol=1e-12)


def test_normalize_flat_map_is_zero():
    assert not O.normalize(np.full((9, 9), 2.0)).any()
    v = np.full((9, 9), 2.0)
    v[0, 0] += 1e-7  # range below the flat threshold
    assert not O.normalize(v, flat=1e-5).any()
    # just above the threshold the map is normalised: its single peak rescales to 1, the
    # other three 8x8 tiles have maximum 0, so mbar = 0 and the peak keeps N = 1
    v = np.full((9, 9), 2.0)
    v[4, 4] += 2e-5
    n = O.normalize(v, flat=1e-5)
    assert n[4, 4] == pytest.approx(1.0) and np.count_nonzero(n) == 1


# ---------------------------------------------------------------- saliency map
def test_saliency_constant_frame_is_zero():
    for rgb in [(97, 97, 97), (200, 30, 60)]:
        f = synth.constant_frame(48, 64, rgb)
        s = O.saliency(f, O.CONFIG_SMALL)
        assert np.abs(s).max() == 0.0


def test_saliency_grey_frame_has_no_colour_conspicuity():
    g = synth.noise_background(np.random.default_rng(8), 120, 160)
    rgb = np.repeat(g[:, :, None], 3, 2)
    _, dbg = O.saliency(rgb, O.CONFIG_SMALL, debug=True)
    assert not dbg["consp"][1].any() and not dbg["consp"][2].any()
    assert dbg["consp"][0].max() > 0 and dbg["consp"][3].max() > 0


def test_opponent_center_surround_makes_a_uniform_red_region_conspicuous():
    # Itti's RG center-surround is (R-G)(c) minus (G-R)(s), i.e. |RG(c) + RG(s)|: inside a
    # uniform red region both terms are the same positive value, so the whole region is
    # conspicuous in the RG channel, and a grey region is not.  With a plain difference
    # |RG(c) - RG(s)| the interior cancels and only the boundary remains.
    H, W = 120, 160
    img = np.full((H, W, 3), 120, np.uint8)
    img[:, :W // 2] = (200, 50, 50)
    _, d = O.saliency(img, O.CONFIG_SMALL, debug=True)
    rg = d["consp"][1]
    wS = rg.shape[1]
    red_inside, grey_inside = rg[:, : wS // 2 - 6], rg[:, wS // 2 + 8:]
    assert red_inside.min() >= 0.95 * rg.max() and grey_inside.max() <= 0.05 * rg.max()
    _, d = O.saliency(img, O.CONFIG_SMALL, debug=True, cs_opponent_sum=0)
    rg = d["consp"][1]
    assert rg[:, : wS // 2 - 8].max() <= 0.05 * rg.max()
    assert wS // 2 - 4 <= int(np.argmax(rg.max(0))) <= wS // 2 + 4


def test_saliency_transpose_equivariance():
    rgb = synth.random_frame(64, 64, 11)
    a = O.saliency(rgb, O.CONFIG_SMALL)
    b = O.saliency(np.ascontiguousarray(rgb.transpose(1, 0, 2)), O.CONFIG_SMALL)
    np.testing.assert_allclose(b, a.T, atol=1e-12)


def test_saliency_debug_pyramid_consistent():
    frames, _ = synth.clip_small(2)
    sal, dbg = O.saliency(frames[1], O.CONFIG_SMALL, debug=True)
    I, RG, BY = O.features(frames[1])
    np.testing.assert_array_equal(dbg["pyr"][0][0], I)
    np.testing.assert_allclose(dbg["pyr"][1][2], O.reduce(O.reduce(RG)), atol=1e-15)
    np.testing.assert_allclose(dbg["ori"][1][3], O.gabor(dbg["pyr"][0][3], np.pi / 4), atol=1e-15)
    np.testing.assert_allclose(O.upsample(dbg["S"], 120, 160), sal, atol=1e-15)
    w = O.CONFIG_SMALL["w"]
    np.testing.assert_allclose(sum(w[k] * dbg["consp"][k] for k in range(4)), dbg["S"], atol=1e-14)


# ---------------------------------------------------------------- saliency composition
# Steps 4-6 of the saliency map (center-surround, N(.), weighted addition; Itti's model as
# cited in Sec. 3, "weighted addition" of normalised maps in Sec. 7.2) on hand-built
# pyramids whose conspicuity maps follow in closed form.  The 160x120 configuration's
# scales are used on a 128x128 frame: centers c in {1, 2} (64x64, 32x32), surrounds
# s = c + {2, 3} in {3, 4, 5}, disjoint from the centers; sigma_S = 2 (32x32, 4x4 tiles of
# 8).  With zero surrounds a center map that is a single positive peak normalises to the
# unit impulse (rescaled peak 1, every other tile maximum 0, so mbar = 0).
_CW = (0.1, 0.2, 0.3, 0.4)
_CCFG = dict(O.CONFIG_SMALL, w=_CW)
_CN = 128
_NT = 16  # tiles of 8x8 at sigma_S


def _cpyr():
    dims = [(O.level_dim(_CN, l),) * 2 for l in range(6)]
    pyr = [[np.zeros(dims[l]) for l in range(6)] for _ in range(3)]
    ori = [{l: np.zeros(dims[l]) for l in range(1, 6)} for _ in range(4)]
    return pyr, ori


def _delta(*pts, shape=(32, 32)):
    d = np.zeros(shape)
    for p in pts:
        d[p] = 1.0
    return d


def _reduced_impulse(y, x, shape=(32, 32)):
    # REDUCE of a unit impulse at the even position (2y, 2x): only the taps at even
    # offsets -2, 0, 2 of [1 4 6 4 1]/16 reach the kept samples, so the result is the
    # outer product of [1 6 1]/16 with itself centred at (y, x)
    r = np.zeros(shape)
    r[y - 1:y + 2, x - 1:x + 2] = np.outer([1, 6, 1], [1, 6, 1]) / 256.0
    return r


@pytest.mark.parametrize("k", range(4))
def test_compose_single_peak_in_one_channel(k):
    # one channel, one peak at sigma_S: each of its two center-surround maps normalises to
    # the impulse, their sum 2 delta normalises back to delta; every other map is zero
    # (flat, N = 0), so S = w_k delta
    pyr, ori = _cpyr()
    p = (13, 18)
    if k < 3:
        pyr[k][2][p] = 0.7
    else:
        ori[2][2][p] = 0.7
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    for j in range(4):
        np.testing.assert_allclose(consp[j], _delta(p) if j == k else 0.0, atol=1e-15)
    np.testing.assert_allclose(S, _CW[k] * _delta(p), atol=1e-15)


@pytest.mark.parametrize("k", range(3))
def test_compose_two_equal_peaks(k):
    # two equal peaks in different tiles: every N(.) keeps them equal and scales by
    # (1 - mbar)^2 with mbar = (2 - 1) / (n_tiles - 1); the two center-surround maps add to
    # 2g(delta_p + delta_q) and the conspicuity N(.) maps that back to g(delta_p + delta_q)
    pyr, ori = _cpyr()
    p, q = (3, 4), (27, 20)
    pyr[k][2][p] = pyr[k][2][q] = 0.25
    g = (1 - 1 / (_NT - 1)) ** 2
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    np.testing.assert_allclose(consp[k], g * _delta(p, q), atol=1e-15)
    np.testing.assert_allclose(S, _CW[k] * g * _delta(p, q), atol=1e-15)


@pytest.mark.parametrize("k", range(3))
def test_compose_two_center_scales(k):
    # a peak of height 3 at level 1 (even position) and one of height 0.5 at sigma_S = 2:
    # each center-surround map is normalised before it is REDUCEd, so the level-1 map
    # reaches sigma_S as the REDUCEd unit impulse r (peak 36/256), whatever its height; the
    # sum is 2(r + delta); its N(.) has maximum 1 at delta and tile maxima {1, 36/256, 0..}
    pyr, ori = _cpyr()
    (y1, x1), p2 = (5, 6), (22, 25)
    pyr[k][1][2 * y1, 2 * x1] = 3.0
    pyr[k][2][p2] = 0.5
    r = _reduced_impulse(y1, x1)
    mbar = (36 / 256) / (_NT - 1)
    want = (r + _delta(p2)) * (1 - mbar) ** 2
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    np.testing.assert_allclose(consp[k], want, atol=1e-15)
    np.testing.assert_allclose(S, _CW[k] * want, atol=1e-15)


def test_compose_each_orientation_normalised_before_the_sum():
    # orientation 0 has a peak at sigma_S only, orientation 1 a peak at level 1 only: the
    # orientation conspicuity takes N(.) of each orientation's sum first, so both reach the
    # sum over theta with peak 1 (delta and r / (36/256)); then two tiles hold maximum 1
    pyr, ori = _cpyr()
    (y1, x1), p2 = (9, 10), (24, 27)
    ori[0][2][p2] = 0.9
    ori[1][1][2 * y1, 2 * x1] = 0.2
    rhat = _reduced_impulse(y1, x1) / (36 / 256)
    want = (_delta(p2) + rhat) * (1 - 1 / (_NT - 1)) ** 2
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    np.testing.assert_allclose(consp[3], want, atol=1e-15)
    assert not consp[:3].any()
    np.testing.assert_allclose(S, _CW[3] * want, atol=1e-15)


def test_compose_surround_sources():
    # the surround of O(c, theta) is O(s, theta) of the same orientation and the surround
    # of X(c) is X(s) of the same channel.  A constant surround k larger than a center peak
    # a makes the map k everywhere except k - a at the peak: rescaled, every tile maximum
    # is 1, mbar = 1 and N = 0.  Intensity surrounds of 0.8 must not reach the
    # orientation maps (their own surrounds are 0), and an orientation-0 surround of 0.8
    # must leave orientation 2 alone.
    pyr, ori = _cpyr()
    p = (14, 9)
    for s in (3, 4, 5):
        pyr[0][s][:] = 0.8
        ori[0][s][:] = 0.8
    ori[2][2][p] = 0.3
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    np.testing.assert_allclose(consp[3], _delta(p), atol=1e-15)
    assert not consp[:3].any()
    # the same peak in orientation 0, whose own surrounds are 0.8: everything is flat
    ori[2][2][p] = 0.0
    ori[0][2][p] = 0.3
    consp, S = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    assert not consp.any() and not S.any()
    # colour opponents: the surround enters with its sign flipped (|X(c) + X(s)|), so a
    # surround of -0.8 under a center peak of 0.3 gives the flat case, +0.8 the impulse
    pyr, ori = _cpyr()
    pyr[1][2][p] = 0.3
    for s in (3, 4, 5):
        pyr[1][s][:] = -0.8
    consp, _ = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    assert not consp.any()
    for s in (3, 4, 5):
        pyr[1][s][:] = 0.8
    consp, _ = O.saliency_compose(pyr, ori, _CN, _CN, _CCFG)
    np.testing.assert_allclose(consp[1], _delta(p), atol=1e-15)


def test_compose_is_the_saliency_maps_last_steps():
    # orc_saliency_ex's S is the composition of its own pyramids (wiring of steps 1-3 to 4-6)
    frames, _ = synth.clip_small(2)
    _, d = O.saliency(frames[1], O.CONFIG_SMALL, debug=True)
    ori = [{l: d["ori"][k][l] for l in range(1, 6)} for k in range(4)]
    consp, S = O.saliency_compose(d["pyr"], ori, 120, 160, O.CONFIG_SMALL)
    np.testing.assert_array_equal(S, d["S"])
    np.testing.assert_array_equal(consp, d["consp"])


def test_saliency_finds_the_red_disk():
    frames, gt = synth.clip_small(3)
    for t in range(3):
        s = O.saliency(frames[t], O.CONFIG_SMALL)
        assert gt[t][np.unravel_index(np.argmax(s), s.shape)] == 1


# ---------------------------------------------------------------- Kalman prior
def test_paper_parameters_golden():
    txt = open(__file__.replace("test_oracle_pins.py", "golden/paper_parameters.txt")).read()
    vals = dict(l.split("=") for l in txt.splitlines() if "=" in l and not l.startswith("#"))
    assert float(vals["sigma1"]) == O.CONFIG_VGA["sigma1"] == 0.03
    assert float(vals["sigma2"]) == O.CONFIG_VGA["sigma2"] == 0.035


def test_kalman_is_the_product_of_two_gaussians():
    # the update combines f (variance sigma2^2 + P) and q (variance sigma1^2) by
    # precision weighting: 1/P_t = 1/V_f + 1/V_q, weight on f = (1/V_f) P_t
    s1, s2 = 0.03, 0.035
    P = float("inf")
    for t in range(30):
        Pt, wf = O.kalman_step(t, P, s1, s2)
        if t == 0:
            assert wf == 0.0 and Pt == pytest.approx(s1 * s1, rel=1e-15)
        else:
            Vf, Vq = s2 * s2 + P, s1 * s1
            Pp = 1.0 / (1.0 / Vf + 1.0 / Vq)
            assert Pt == pytest.approx(Pp, rel=1e-13)
            assert wf == pytest.approx(Pp / Vf, rel=1e-13)
        P = Pt


def test_kalman_steady_state_closed_form():
    a, b = 0.03 ** 2, 0.035 ** 2
    Pstar = (-b + math.sqrt(b * b + 4 * a * b)) / 2
    P = float("inf")
    seq = []
    for t in range(200):
        P, wf = O.kalman_step(t, P, 0.03, 0.035)
        seq.append(P)
    assert P == pytest.approx(Pstar, rel=1e-12)
    assert wf == pytest.approx(a / (a + b + Pstar), rel=1e-12)
    assert Pstar == pytest.approx(6.030888e-4, rel=1e-6) and wf == pytest.approx(0.329901, rel=1e-5)
    assert all(x > y for x, y in zip(seq[:5], seq[1:6]))  # monotone decrease from sigma1^2


def test_kalman_limits():
    # sigma1 -> 0: the prior is the saliency prior q; sigma2 -> 0 with P = 0: it is f
    _, wf = O.kalman_step(3, 1e-4, 1e-9, 0.035)
    assert wf < 1e-12
    _, wf = O.kalman_step(3, 0.0, 0.03, 0.0)
    assert wf == 1.0


def test_smooth_mask_matches_scipy():
    m = (np.random.default_rng(9).random((30, 41)) > 0.7).astype(np.uint8)
    u = np.arange(-6, 7)
    g = np.exp(-u ** 2 / 8.0)
    g2 = np.outer(g, g) / np.outer(g, g).sum()
    ref = ndimage.correlate(m.astype(float), g2, mode="nearest")
    np.testing.assert_allclose(O.smooth_mask(m), ref, atol=1e-14)


def test_prior_convex_and_border():
    rng = np.random.default_rng(10)
    sal = rng.random((20, 30)) * 3
    prev = (rng.random((20, 30)) > 0.5).astype(np.uint8)
    q, pr = O.prior(sal, prev, 0.3)
    assert (q[0] == 1e-4).all() and (q[:, -1] == 1e-4).all()
    np.testing.assert_allclose(q[1:-1, 1:-1], sal[1:-1, 1:-1] / sal.max(), atol=1e-15)
    np.testing.assert_allclose(pr, 0.3 * O.smooth_mask(prev) + 0.7 * q, atol=1e-15)
    assert pr.min() >= 0 and pr.max() <= 1
    q0, pr0 = O.prior(sal, None, 0.0)
    np.testing.assert_array_equal(pr0, q0)


# ---------------------------------------------------------------- MRF terms
def test_colour_models_match_numpy_weighted_cov():
    rng = np.random.default_rng(12)
    rgb = rng.integers(0, 256, (25, 31, 3)).astype(np.uint8)
    pr = rng.random((25, 31))
    mu, cov, deg = O.colour_models(pr, rgb)
    assert deg == 0
    C = rgb.reshape(-1, 3) / 255.0
    for a, w in [(1, pr.ravel()), (0, 1 - pr.ravel())]:
        np.testing.assert_allclose(mu[a], np.average(C, axis=0, weights=w), atol=1e-14)
        ref = np.cov(C.T, aweights=w, bias=True) + 1e-4 * np.eye(3)
        np.testing.assert_allclose(cov[a], ref, atol=1e-14)


def test_terms_match_scipy_logpdf():
    rng = np.random.default_rng(13)
    rgb = rng.integers(0, 256, (12, 17, 3)).astype(np.uint8)
    pr = rng.random((12, 17))
    cs, ct, nc, D0, D1 = O.terms(rgb, pr, O.CONFIG_SMALL)
    mu, cov, _ = O.colour_models(pr, rgb)
    C = rgb.reshape(-1, 3) / 255.0
    eps = 1e-4
    for a, D in [(0, D0), (1, D1)]:
        p = pr.ravel() if a else 1 - pr.ravel()
        ref = -stats.multivariate_normal(mu[a], cov[a]).logpdf(C) - np.log(np.clip(p, eps, 1 - eps))
        np.testing.assert_allclose(D.ravel(), ref, rtol=1e-12, atol=1e-12)
    m = np.minimum(D0, D1)
    np.testing.assert_array_equal(cs, np.floor(1000 * (D0 - m) + 0.5).astype(np.int32))
    np.testing.assert_array_equal(ct, np.floor(1000 * (D1 - m) + 0.5).astype(np.int32))
    assert (np.minimum(cs, ct) == 0).all()


def test_ncap_closed_form():
    assert O.ncap_value(0, 0) == 1500
    assert O.ncap_value(0, 1) == round(1500 / math.sqrt(2))
    assert O.ncap_value(765, 0) == 0
    d = 20
    assert O.ncap_value(d, 0) == O.ncap_value(-d, 0) == math.floor(
        1500 * math.exp(-(d / 765) ** 2 / (2 * 0.05 ** 2)) + 0.5)
    assert O.ncap_value(0, 0, lambda_p=0.25) == 1750


def test_capacities_are_capped_at_2_pow_24():
    # integer capacities are min(2^24, floor(K cost + 1/2)): a huge Potts constant or
    # capacity scale saturates at exactly 2^24, never beyond
    assert O.ncap_value(0, 0, lambda_p=1e5) == 1 << 24
    assert O.ncap_value(0, 1, lambda_p=1e5) == 1 << 24
    rng = np.random.default_rng(15)
    rgb = rng.integers(0, 256, (6, 7, 3)).astype(np.uint8)
    cs, ct, nc, _, _ = O.terms(rgb, rng.uniform(0.01, 0.99, (6, 7)), O.CONFIG_VGA, cap_scale=1e9)
    assert max(cs.max(), ct.max(), nc.max()) == 1 << 24 and min(cs.min(), ct.min(), nc.min()) >= 0


def test_terms_ncap_layout():
    rng = np.random.default_rng(14)
    # low contrast, so that every n-link is well above zero and a straight link and
    # a diagonal one of the same colour step differ (high contrast quantises to 0)
    rgb = rng.integers(100, 106, (6, 7, 3)).astype(np.uint8)
    _, _, nc, _, _ = O.terms(rgb, np.full((6, 7), 0.5), O.CONFIG_VGA)
    s = rgb.astype(int).sum(2)
    assert nc.shape == (4, 6, 7)
    assert nc[0, :, :6].min() > 1000 and nc[2, :5, :6].min() > 700
    assert nc[0, 2, 3] == O.ncap_value(s[2, 3] - s[2, 4], 0)
    assert nc[1, 2, 3] == O.ncap_value(s[2, 3] - s[3, 3], 0)
    assert nc[2, 2, 3] == O.ncap_value(s[2, 3] - s[3, 4], 1)
    assert nc[3, 2, 3] == O.ncap_value(s[2, 3] - s[3, 2], 1)
    assert not nc[0, :, 6].any() and not nc[1, 5].any() and not nc[3, :, 0].any()


# ---------------------------------------------------------------- min cut
def _scipy_flow(cs, ct, nc):
    H, W = cs.shape
    n = H * W
    s, t = n, n + 1
    rows, cols, vals = [], [], []
    for v in range(n):
        rows += [s, v]
        cols += [v, t]
        vals += [int(cs.flat[v]), int(ct.flat[v])]
    dx, dy = [1, 0, 1, -1], [0, 1, 1, 1]
    for k in range(nc.shape[0]):
        for y in range(H):
            for x in range(W):
                xx, yy = x + dx[k], y + dy[k]
                if 0 <= xx < W and yy < H:
                    c = int(nc[k, y, x])
                    rows += [y * W + x, yy * W + xx]
                    cols += [yy * W + xx, y * W + x]
                    vals += [c, c]
    A = sp.coo_array((np.array(vals, np.int32), (rows, cols)), shape=(n + 2, n + 2)).tocsr()
    A.sum_duplicates()
    return maximum_flow(A, s, t).flow_value


@pytest.mark.parametrize("nbr", [4, 8])
def test_bruteforce_equals_bk_and_ek(nbr):
    for seed in range(40):
        h, w = [(4, 4), (3, 5), (2, 2), (1, 6), (4, 3)][seed % 5]
        cs, ct, nc = synth.random_grid_caps(h, w, nbr, seed, tmax=60, nmax=40, p_zero=0.2)
        e, m, cnt = O.bruteforce(cs, ct, nc)
        assert O.cut_energy(cs, ct, nc, m) == e  # the intersection of minimisers is a minimiser
        for method in ("bk", "ek"):
            v, mm = O.maxflow(cs, ct, nc, method)
            assert v == e
            np.testing.assert_array_equal(mm, m)


@pytest.mark.parametrize("nbr", [4, 8])
def test_maxflow_value_matches_scipy_and_duality(nbr):
    for seed in range(6):
        cs, ct, nc = synth.random_grid_caps(13, 19, nbr, 100 + seed, tmax=500, nmax=200)
        vb, mb = O.maxflow(cs, ct, nc, "bk")
        ve, me = O.maxflow(cs, ct, nc, "ek")
        assert vb == ve == _scipy_flow(cs, ct, nc)
        assert O.cut_energy(cs, ct, nc, mb) == vb
        np.testing.assert_array_equal(mb, me)


def test_maxflow_blob_grids_bk_equals_ek():
    for nbr in (4, 8):
        cs, ct, nc = synth.blob_grid_caps(40, 50, nbr, 7)
        vb, mb = O.maxflow(cs, ct, nc, "bk")
        ve, me = O.maxflow(cs, ct, nc, "ek")
        assert vb == ve == O.cut_energy(cs, ct, nc, mb)
        np.testing.assert_array_equal(mb, me)


def test_maxflow_no_nlinks_closed_form():
    cs, ct, nc = synth.random_grid_caps(9, 11, 8, 21, tmax=9)
    nc[:] = 0
    v, m = O.maxflow(cs, ct, nc)
    assert v == int(np.minimum(cs, ct).sum())
    np.testing.assert_array_equal(m, (cs > ct).astype(np.uint8))  # ties go to background


def test_maxflow_chain_matches_dynamic_programming():
    # a 1 x N 4-neighbour chain is solvable exactly by a two-state Viterbi pass
    rng = np.random.default_rng(22)
    for _ in range(5):
        N = 200
        cs = rng.integers(0, 100, (1, N)).astype(np.int32)
        ct = rng.integers(0, 100, (1, N)).astype(np.int32)
        nc = np.zeros((2, 1, N), np.int32)
        nc[0, 0, :-1] = rng.integers(0, 60, N - 1)
        cost = [int(cs[0, 0]), int(ct[0, 0])]  # label 0 pays cs, label 1 pays ct
        for i in range(1, N):
            w = int(nc[0, 0, i - 1])
            cost = [min(cost[0], cost[1] + w) + int(cs[0, i]), min(cost[1], cost[0] + w) + int(ct[0, i])]
        v, _ = O.maxflow(cs, ct, nc)
        assert v == min(cost)


def test_maxflow_edge_cases():
    z = np.zeros((1, 1), np.int32)
    assert O.maxflow(z, z, np.zeros((2, 1, 1), np.int32))[0] == 0
    big = np.full((3, 3), 1 << 24, np.int32)
    nc = np.full((4, 3, 3), 1 << 24, np.int32)
    nc[0, :, 2] = nc[1, 2] = nc[2, 2] = nc[2, :, 2] = nc[3, 2] = nc[3, :, 0] = 0
    v, m = O.maxflow(big, big, nc)
    assert v == 9 * (1 << 24) and not m.any()


# ---------------------------------------------------------------- regression guard
@pytest.mark.parametrize("cfg", [O.CONFIG_SMALL, O.CONFIG_VGA], ids=["4-neighbour", "8-neighbour"])
def test_frame_sequence_carries_mask_and_variance(cfg):
    # Sec. 6 wiring of the per-frame method: frame t's prior is built from frame t's
    # saliency, the mask the method returned for frame t-1 and the Kalman weight of
    # step t; the cut is the exact cut of the terms of that prior (each part pinned
    # on its own above)
    frames, _ = synth.clip_small(4, seed=synth.SEED_BASE + 9)
    H, W = frames.shape[1:3]
    sg = O.Segmenter(H, W, cfg)
    P, prev = 0.0, None
    for t in range(4):
        sal, pr, mask, cut = sg.push(frames[t])
        P, wf = O.kalman_step(t, P)
        assert sg.t == t + 1 and sg.P_var == P
        np.testing.assert_array_equal(sal, O.saliency(frames[t], cfg))
        _, pr_ref = O.prior(sal, prev if t else None, wf, cfg)
        np.testing.assert_array_equal(pr, pr_ref)
        cs, ct, nc, _, _ = O.terms(frames[t], pr_ref, cfg)
        v, m = O.maxflow(cs, ct, nc)
        assert cut == v
        np.testing.assert_array_equal(mask, m)
        if t:
            assert wf > 0 and prev.any()  # the previous mask really enters from the second frame on
        prev = mask.copy()


def test_frame_sequence_updates_the_colour_mixtures():
    # Sec. 2 / Sec. 6 likelihood update (reading: a frame's EM starts from the previous
    # frame's fitted mixtures; the k-means start runs on the first frame only), composed
    # from separately pinned parts; with gmm_update = 0 every frame starts afresh
    cfg = dict(O.CONFIG_SMALL, gmm_components=3, em_iters=3)
    frames, _ = synth.clip_small(3, seed=synth.SEED_BASE + 11)
    H, W = frames.shape[1:3]
    for update in (1, 0):
        sg = O.Segmenter(H, W, cfg, gmm_update=update)
        P, prev, mix = 0.0, None, None
        for t in range(3):
            sal, pr, mask, cut = sg.push(frames[t])
            P, wf = O.kalman_step(t, P)
            _, pr_ref = O.prior(sal, prev if t else None, wf, cfg)
            np.testing.assert_array_equal(pr, pr_ref)
            cs, ct, nc, fitted = O.terms_from(frames[t], pr_ref, mix if update else None, cfg)
            if t and update:  # the carried start really leads elsewhere than a fresh one
                _, _, _, fresh = O.terms_from(frames[t], pr_ref, None, cfg)
                d = max(abs(fresh[a].mu[m][k] - fitted[a].mu[m][k]) for a in range(2) for m in range(3)
                        for k in range(3))
                assert d > 1e-6
            v, m = O.maxflow(cs, ct, nc)
            assert cut == v
            np.testing.assert_array_equal(mask, m)
            for a in range(2):  # the mixtures the method carries are the ones composed here
                assert [sg.st.gmm[a].pi[k] for k in range(3)] == [fitted[a].pi[k] for k in range(3)]
                assert all(sg.st.gmm[a].mu[k][j] == fitted[a].mu[k][j] for k in range(3) for j in range(3))
            prev, mix = mask.copy(), fitted


def test_small_clip_regression_golden():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_small_clip.json")))
    frames, gt = synth.clip_small()
    sg = O.Segmenter(120, 160, O.CONFIG_SMALL)
    for row in g["frames"]:
        sal, pr, mask, cut = sg.push(frames[row["t"]])
        assert cut == row["cut"] and int(mask.sum()) == row["mask_area"]
        assert float(sal.sum()) == pytest.approx(row["saliency_sum"], rel=1e-12)
        assert float(pr.sum()) == pytest.approx(row["prior_sum"], rel=1e-12)


# ---------------------------------------------------------------- M-component colour model (EM)
def _clustered_rgb(seed, n=3000):
    rng = np.random.default_rng(seed)
    centers = np.array([[50, 50, 50], [128, 128, 128], [210, 190, 170]], float)
    lab = rng.integers(0, 3, n)
    x = centers[lab] + rng.normal(0, 6, (n, 3))
    return np.clip(np.rint(x), 0, 255).astype(np.uint8), lab, centers


def test_em_single_component_is_the_weighted_gaussian():
    rng = np.random.default_rng(31)
    rgb = rng.integers(0, 256, (40, 50, 3)).astype(np.uint8)
    w = rng.random((40, 50))
    pi, mu, cov = O.gmm_fit(rgb, w, M=1, iters=4)
    mu1, cov1, _ = O.colour_models(w, rgb)
    np.testing.assert_allclose(pi, [1.0])
    np.testing.assert_allclose(mu[0], mu1[1], atol=1e-13)
    np.testing.assert_allclose(cov[0], cov1[1], atol=1e-13)


def test_em_loglik_never_decreases_and_weight_scale_invariant():
    rgb, _, _ = _clustered_rgb(32)
    w = np.random.default_rng(33).random(rgb.shape[0])
    trace = O.gmm_em_trace(rgb, w, M=3, iters=8)
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(trace, trace[1:]))
    a = O.gmm_fit(rgb, w, 3, 5)
    b = O.gmm_fit(rgb, 3.7 * w, 3, 5)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-10, atol=1e-13)


def test_em_recovers_separated_clusters():
    rgb, lab, centers = _clustered_rgb(34)
    pi, mu, cov = O.gmm_fit(rgb, np.ones(rgb.shape[0]), M=3, iters=30)
    order = np.argsort(mu[:, 0])
    np.testing.assert_allclose(mu[order] * 255, centers, atol=1.0)
    np.testing.assert_allclose(pi[order], np.bincount(lab) / lab.size, atol=0.01)


def test_em_components_are_the_weighted_cluster_gaussians():
    # clusters 13 standard deviations apart: at convergence every responsibility is 0
    # or 1 to FP64 precision, so each component must be its cluster's prior-weighted
    # Gaussian (numpy, from the known membership) with the 1e-4 ridge, and its weight
    # the cluster's share of the total pixel weight
    rgb, lab, _ = _clustered_rgb(35)
    w = np.random.default_rng(36).uniform(0.2, 1.0, lab.size)
    pi, mu, cov = O.gmm_fit(rgb, w, M=3, iters=40)
    order = np.argsort(mu[:, 0])
    c = rgb.astype(float) / 255.0
    for m, k in zip(order, range(3)):
        sel = lab == k
        np.testing.assert_allclose(mu[m], np.average(c[sel], axis=0, weights=w[sel]), rtol=1e-9)
        ref = np.cov(c[sel].T, aweights=w[sel], bias=True) + 1e-4 * np.eye(3)
        np.testing.assert_allclose(cov[m], ref, rtol=1e-6, atol=1e-12)
        assert pi[m] == pytest.approx(w[sel].sum() / w.sum(), rel=1e-9)


def test_kmeans_start_seed_is_the_expected_kmeanspp_draw():
    # Two point masses a = 0 (weight 0.6) and b = 1 (weight 0.4) on the red axis: the
    # first seed is the weighted mean 0.4; a k-means++ draw picks a point with
    # probability w D^2, so its expected position is (wa D_a^2 a + wb D_b^2 b) /
    # (wa D_a^2 + wb D_b^2) = (wb a + wa b) / W = 0.6.  With no Lloyd iteration a light
    # probe pixel joins the seed it is nearer to: below the midpoint 0.5 the first one
    # (with a), above it the second (with b).
    for probe, with_a in [(125, True), (130, False)]:
        rgb = np.array([[0, 0, 0], [255, 0, 0], [probe, 0, 0]], np.uint8)
        w = np.array([0.6, 0.4, 1e-6])
        pi, mu, cov = O.gmm_init(rgb, w, M=2, km_iters=0)
        ia = int(np.argmin(mu[:, 0]))
        members_a = [0, 2] if with_a else [0]
        c = rgb.astype(float) / 255.0
        np.testing.assert_allclose(mu[ia], np.average(c[members_a], axis=0, weights=w[members_a]), atol=1e-15)
        assert pi[ia] == pytest.approx(w[members_a].sum() / w.sum(), rel=1e-12)


def test_kmeans_start_single_component_and_weight_scale():
    rng = np.random.default_rng(41)
    rgb = rng.integers(0, 256, (30, 40, 3)).astype(np.uint8)
    w = rng.random((30, 40))
    pi, mu, cov = O.gmm_init(rgb, w, M=1, km_iters=3)
    mu1, cov1, _ = O.colour_models(w, rgb)
    np.testing.assert_allclose(pi, [1.0])
    np.testing.assert_allclose(mu[0], mu1[1], atol=1e-13)
    np.testing.assert_allclose(cov[0], cov1[1], atol=1e-13)
    a, b = O.gmm_init(rgb, w, M=3, km_iters=3), O.gmm_init(rgb, 2.5 * w, M=3, km_iters=3)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-10, atol=1e-13)


def test_kmeans_start_partitions_separated_clusters():
    # three well-separated clusters of unequal weight: the seeds reach every cluster and
    # a few Lloyd iterations settle on the true partition, so the start is already each
    # cluster's weighted Gaussian (numpy, from the known membership) with the 1e-4 ridge
    rgb, lab, _ = _clustered_rgb(42)
    w = np.random.default_rng(43).uniform(0.2, 1.0, lab.size) * np.array([1.0, 0.3, 0.6])[lab]
    pi, mu, cov = O.gmm_init(rgb, w, M=3, km_iters=3)
    order = np.argsort(mu[:, 0])
    c = rgb.astype(float) / 255.0
    for m, k in zip(order, range(3)):
        sel = lab == k
        np.testing.assert_allclose(mu[m], np.average(c[sel], axis=0, weights=w[sel]), rtol=1e-12)
        ref = np.cov(c[sel].T, aweights=w[sel], bias=True) + 1e-4 * np.eye(3)
        np.testing.assert_allclose(cov[m], ref, rtol=1e-9, atol=1e-14)
        assert pi[m] == pytest.approx(w[sel].sum() / w.sum(), rel=1e-12)


def test_em_step_matches_its_definition_on_overlapping_clusters():
    # one EM step from a given mixture, written from its definition: responsibilities by
    # Bayes' rule from scipy's Gaussian densities, then each component's prior-weighted
    # share, mean and covariance (numpy) plus the 1e-4 ridge.  Overlapping clusters keep
    # the responsibilities fractional.
    rng = np.random.default_rng(44)
    centers = np.array([[90, 90, 90], [120, 110, 100], [150, 140, 120]], float)
    lab = rng.integers(0, 3, 2000)
    rgb = np.clip(np.rint(centers[lab] + rng.normal(0, 18, (2000, 3))), 0, 255).astype(np.uint8)
    w = rng.uniform(0.1, 1.0, 2000)
    pi0 = np.array([0.5, 0.3, 0.2])
    mu0 = centers / 255.0 + 0.01
    cov0 = np.stack([np.eye(3) * s for s in (0.004, 0.006, 0.005)])
    pi, mu, cov = O.gmm_em_from(rgb, w, pi0, mu0, cov0, iters=1)
    c = rgb.astype(float) / 255.0
    dens = np.stack([pi0[m] * stats.multivariate_normal(mu0[m], cov0[m]).pdf(c) for m in range(3)], 1)
    r = dens / dens.sum(1, keepdims=True)
    assert 0.05 < r.max(1).mean() < 0.95  # fractional responsibilities
    for m in range(3):
        wr = w * r[:, m]
        assert pi[m] == pytest.approx(wr.sum() / w.sum(), rel=1e-10)
        np.testing.assert_allclose(mu[m], np.average(c, axis=0, weights=wr), rtol=1e-10)
        ref = np.cov(c.T, aweights=wr, bias=True) + 1e-4 * np.eye(3)
        np.testing.assert_allclose(cov[m], ref, rtol=1e-8, atol=1e-14)


def test_gmm_logpdf_and_terms_match_scipy():
    from scipy.special import logsumexp
    rgb, _, _ = _clustered_rgb(35, n=1200)
    img = rgb.reshape(30, 40, 3)
    pr = np.random.default_rng(36).random((30, 40))
    cfg = dict(O.CONFIG_SMALL, gmm_components=3, em_iters=5)
    cs, ct, nc, D0, D1 = O.terms(img, pr, cfg)
    C = img.reshape(-1, 3) / 255.0
    for a, D in [(0, D0), (1, D1)]:
        w = pr.ravel() if a else 1 - pr.ravel()
        pi, mu, cov = O.gmm_fit(img, w.reshape(30, 40), 3, 5)
        lp = logsumexp([np.log(pi[m]) + stats.multivariate_normal(mu[m], cov[m]).logpdf(C) for m in range(3)],
                       axis=0)
        assert O.gmm_logpdf(pi, mu, cov, C[7]) == pytest.approx(lp[7], rel=1e-12)
        ref = -lp - np.log(np.clip(w, 1e-4, 1 - 1e-4))
        np.testing.assert_allclose(D.ravel(), ref, rtol=1e-11, atol=1e-11)
