"""GPU path vs the FP64 oracle, through the C-ABI.

Tolerances (floating point): saliency, prior and every intermediate map within
max|gpu - oracle| / max|oracle| <= 1e-4 per map; integer n-links bit-exact;
t-link capacities within 2 + 2e-6 * cap (they are FP32 costs quantised at
K = 1000, so a cost that differs by FP32 rounding can land one unit off);
min cuts on identical int32 capacities bit-exact (value and mask); end-to-end
masks on >= 99.9% of pixels.  In a frame sequence the prior of frame t depends
on the mask of frame t-1 through the mask smoothing f (radius f_radius), so
the prior is compared outside that radius around pixels where the two previous
masks differ (everywhere when they agree).
"""
import base64
import itertools
import json
import os
import zlib

import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_0502_b300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def S(cuda_ok):
    from paper_1008_0502_b300 import build
    build.build()
    from paper_1008_0502_b300 import seg
    return seg


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / den if den > 0 else np.abs(a).max()


def seg_params(S, cfg, **over):
    return S.params_from({k: v for k, v in cfg.items()}, **over)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def prior_err(pr, opr, prev_gpu, prev_orc, radius):
    """rel_err of the prior outside the f-radius of previous-mask differences."""
    diff = np.asarray(prev_gpu) != np.asarray(prev_orc)
    keep = np.ones(diff.shape, bool)
    if diff.any():
        from scipy import ndimage
        keep = ~ndimage.binary_dilation(diff, np.ones((2 * radius + 1,) * 2, bool))
    pr, opr = np.asarray(pr, np.float64), np.asarray(opr, np.float64)
    return np.abs(pr - opr)[keep].max(initial=0.0) / np.abs(opr).max(), float(keep.mean())


def state_blob(t, P_var, prev_mask):
    """seg_set_state's byte string (include/seg.h) for one stream."""
    H, W = prev_mask.shape
    hdr = np.array([0x53454732, H, W, 1], np.uint32).tobytes()
    rec = np.array([t, 0], np.int32).tobytes() + np.array([P_var], np.float64).tobytes()
    return hdr + rec + np.ascontiguousarray(prev_mask, np.uint8).tobytes()


def golden_vga_state(t_start):
    d = json.load(open(os.path.join(GOLDEN, f"oracle_vga_state_f{t_start}.json")))
    bits = np.frombuffer(zlib.decompress(base64.b64decode(d["prev_mask_packbits_zlib_b64"])), np.uint8)
    mask = np.unpackbits(bits)[:d["H"] * d["W"]].reshape(d["H"], d["W"])
    return d["t"], float.fromhex(d["P_hex"]), mask


def host(t):
    return t.cpu().numpy()


# ---------------------------------------------------------------- saliency
@pytest.mark.parametrize("cfg_name,H,W", [("small", 120, 160), ("small", 97, 131), ("vga", 480, 640),
                                          ("vga", 301, 403)])
def test_saliency_stages_match_oracle(S, cfg_name, H, W):
    cfg = O.CONFIG_SMALL if cfg_name == "small" else O.CONFIG_VGA
    if (H, W) == (120, 160):
        rgb = synth.clip_small(2)[0][1]
    elif (H, W) == (480, 640):
        rgb = next(synth.clip_vga_frames(1))[0]
    else:
        rgb = synth.random_frame(H, W, 5 + H)
    ref, dbg = O.saliency(rgb, cfg, debug=True)
    sg = S.Segmenter(H, W, seg_params(S, cfg))
    sal = host(sg.saliency(dev(rgb)))
    assert rel_err(sal, ref) <= REL
    L = cfg["levels"]
    for ch in range(3):
        for l in range(1, L):
            h, w = dbg["pyr"][ch][l].shape
            got = sg.debug_copy(0, ch * 16 + l, (h, w)).numpy()
            assert rel_err(got, dbg["pyr"][ch][l]) <= REL, (ch, l)
    for k in range(cfg["n_orient"]):
        for l in range(cfg["c_min"], cfg["c_max"] + cfg["d_max"] + 1):
            ref_o = dbg["ori"][k][l]
            got = sg.debug_copy(1, k * 16 + l, ref_o.shape).numpy()
            # absolute bound relative to the largest orientation response of the level
            scale = max(np.abs(dbg["ori"][j][l]).max() for j in range(cfg["n_orient"]))
            assert np.abs(got - ref_o).max() <= REL * max(scale, 1e-3), (k, l)
    for k in range(4):
        got = sg.debug_copy(2, k, dbg["consp"][k].shape).numpy()
        assert np.abs(got - dbg["consp"][k]).max() <= REL * max(np.abs(dbg["consp"]).max(), 1e-12), k
    got = sg.debug_copy(3, 0, dbg["S"].shape).numpy()
    assert rel_err(got, dbg["S"]) <= REL
    sg.close()


def test_saliency_constant_and_grey_frames(S):
    sg = S.Segmenter(64, 80, seg_params(S, O.CONFIG_SMALL))
    for rgb in [synth.constant_frame(64, 80, (97, 97, 97)), synth.constant_frame(64, 80, (200, 30, 60))]:
        assert float(sg.saliency(dev(rgb)).abs().max()) == 0.0
    g = synth.noise_background(np.random.default_rng(8), 64, 80)
    grey = np.repeat(g[:, :, None], 3, 2)
    sg.saliency(dev(grey))
    hS, wS = S.level_dim(64, 2), S.level_dim(80, 2)
    assert not sg.debug_copy(2, 1, (hS, wS)).numpy().any()
    assert not sg.debug_copy(2, 2, (hS, wS)).numpy().any()
    sg.close()


# ---------------------------------------------------------------- prior
@pytest.mark.parametrize("w_f", [0.0, 0.329901, 1.0])
def test_prior_matches_oracle(S, w_f):
    H, W = 97, 130
    rng = np.random.default_rng(3)
    sal = (rng.random((H, W)) ** 3).astype(np.float32)
    prev = (rng.random((H, W)) > 0.6).astype(np.uint8)
    sg = S.Segmenter(H, W, seg_params(S, O.CONFIG_SMALL))
    got = host(sg.prior(dev(sal), dev(prev), w_f))
    _, ref = O.prior(sal.astype(np.float64), prev, w_f, O.CONFIG_SMALL)
    assert np.abs(got - ref).max() <= 1e-6
    sg.close()


# ---------------------------------------------------------------- terms
@pytest.mark.parametrize("cfg_name,M", [("small", 1), ("vga", 1), ("small", 3), ("vga", 3)])
def test_terms_match_oracle(S, cfg_name, M):
    """M = 3: the paper's EM colour mixtures (Sec. 4, Sec. 7.3), same tolerance."""
    cfg = dict(O.CONFIG_SMALL if cfg_name == "small" else O.CONFIG_VGA, gmm_components=M, em_iters=5)
    if cfg_name == "small":
        rgb = synth.clip_small(2)[0][1]
    else:  # a real 640x480 frame: 600 CTAs of moment partials summed across CTAs
        rgb = [f for f, _ in synth.clip_vga_frames(3)][2]
    H, W = rgb.shape[:2]
    sal = O.saliency(rgb, cfg)
    _, pr = O.prior(sal, None, 0.0, cfg)
    pr32 = pr.astype(np.float32)
    cs, ct, nc, D0, D1 = O.terms(rgb, pr32.astype(np.float64), cfg)
    sg = S.Segmenter(H, W, seg_params(S, cfg))
    gcs, gct, gnc = (host(t) for t in sg.terms(dev(rgb), dev(pr32)))
    np.testing.assert_array_equal(gnc, nc)
    for g, r in [(gcs, cs), (gct, ct)]:
        assert (np.abs(g.astype(np.int64) - r) <= 2 + 2e-6 * np.abs(r)).all()
    assert (np.minimum(gcs, gct) == 0).all()
    sg.close()


# ---------------------------------------------------------------- min cut, bit-exact
CUT_CASES = [(1, 1, 4), (1, 37, 4), (29, 1, 8), (4, 4, 8), (16, 32, 4), (17, 33, 8), (33, 65, 4),
             (50, 70, 8), (120, 160, 4), (121, 161, 8)]


@pytest.mark.parametrize("H,W,nbr", CUT_CASES)
def test_mincut_random_grids_bit_exact(S, H, W, nbr):
    for seed in range(3):
        cs, ct, nc = synth.random_grid_caps(H, W, nbr, 1000 * H + W + seed, tmax=800, nmax=300,
                                            p_zero=0.1 * seed)
        v, m = O.maxflow(cs, ct, nc)
        mask, cut, code, cyc = S.mincut_grid(dev(cs), dev(ct), dev(nc))
        assert code == 0
        assert int(cut.item()) == v
        np.testing.assert_array_equal(host(mask), m)


@pytest.mark.parametrize("H,W,nbr", [(64, 96, 4), (97, 131, 8), (240, 320, 8), (480, 640, 8)])
def test_mincut_blob_grids_bit_exact(S, H, W, nbr):
    cs, ct, nc = synth.blob_grid_caps(H, W, nbr, H + W)
    v, m = O.maxflow(cs, ct, nc)
    mask, cut, code, cyc = S.mincut_grid(dev(cs), dev(ct), dev(nc))
    assert code == 0 and int(cut.item()) == v
    np.testing.assert_array_equal(host(mask), m)


def test_mincut_extreme_capacities(S):
    H, W = 20, 40
    big = np.full((H, W), 1 << 24, np.int32)
    nc = np.full((4, H, W), 1 << 24, np.int32)
    v, m = O.maxflow(big, np.zeros_like(big), nc)
    mask, cut, code, _ = S.mincut_grid(dev(big), dev(np.zeros_like(big)), dev(nc))
    assert code == 0 and int(cut.item()) == v == 0 and host(mask).all()
    z = np.zeros((H, W), np.int32)
    mask, cut, code, _ = S.mincut_grid(dev(z), dev(z), dev(np.zeros((2, H, W), np.int32)))
    assert code == 0 and int(cut.item()) == 0 and not host(mask).any()


def test_mincut_frame_graphs_bit_exact(S):
    frames, _ = synth.clip_small(3)
    for t in range(3):
        sal = O.saliency(frames[t], O.CONFIG_SMALL)
        _, pr = O.prior(sal, None, 0.0, O.CONFIG_SMALL)
        cs, ct, nc, _, _ = O.terms(frames[t], pr, O.CONFIG_SMALL)
        v, m = O.maxflow(cs, ct, nc)
        mask, cut, code, _ = S.mincut_grid(dev(cs), dev(ct), dev(nc))
        assert code == 0 and int(cut.item()) == v
        np.testing.assert_array_equal(host(mask), m)
    f = next(synth.clip_vga_frames(1))[0]
    sal = O.saliency(f, O.CONFIG_VGA)
    _, pr = O.prior(sal, None, 0.0, O.CONFIG_VGA)
    cs, ct, nc, _, _ = O.terms(f, pr, O.CONFIG_VGA)
    v, m = O.maxflow(cs, ct, nc)
    mask, cut, code, _ = S.mincut_grid(dev(cs), dev(ct), dev(nc))
    assert code == 0 and int(cut.item()) == v
    np.testing.assert_array_equal(host(mask), m)


def test_mincut_errors_are_reported_and_context_survives(S):
    cs, ct, nc = synth.blob_grid_caps(64, 96, 8, 3)
    _, _, code, cyc = S.mincut_grid(dev(cs), dev(ct), dev(nc), max_cycles=1)
    assert code == S.SEG_ENOTCONVERGED and cyc == 1
    bad = cs.copy()
    bad[3, 4] = (1 << 24) + 1
    _, _, code, _ = S.mincut_grid(dev(bad), dev(ct), dev(nc))
    assert code == S.SEG_ECAPACITY
    neg = nc.copy()
    neg[1, 5, 5] = -3
    _, _, code, _ = S.mincut_grid(dev(cs), dev(ct), dev(neg))
    assert code == S.SEG_ECAPACITY
    v, m = O.maxflow(cs, ct, nc)
    mask, cut, code, _ = S.mincut_grid(dev(cs), dev(ct), dev(nc))
    assert code == 0 and int(cut.item()) == v
    np.testing.assert_array_equal(host(mask), m)


# ---------------------------------------------------------------- end to end
def _run_clip(S, frames, cfg, check_every=1, state=None, cut_on_oracle_caps=False):
    """Both sides through the same frames (optionally from the same oracle-made temporal
    state): saliency and prior within REL, mask agreement per frame; with
    cut_on_oracle_caps the GPU cut of the oracle's own capacities must equal the
    oracle's mask and cut value bit for bit.  Returns (agreement list, GPU cycle counts)."""
    H, W = frames.shape[1:3]
    sg = S.Segmenter(H, W, seg_params(S, cfg))
    orc = O.Segmenter(H, W, cfg)
    prev_g = prev_o = np.zeros((H, W), np.uint8)
    if state is not None:
        t0, P0, m0 = state
        orc.set_state(t0, P0, m0)
        sg.set_state(state_blob(t0, P0, m0))
        prev_g = prev_o = m0
    agree, cycles = [], []
    for t in range(len(frames)):
        sal, pr, mask, cut = sg.push_frame(dev(frames[t]))
        code, cyc = sg.sync()
        assert code == 0
        cycles.append(cyc)
        osal, opr, omask, ocut = orc.push(frames[t])
        hm = host(mask)
        if t % check_every == 0:
            assert rel_err(host(sal), osal) <= REL, t
            err, kept = prior_err(host(pr), opr, prev_g, prev_o, cfg["f_radius"])
            assert err <= REL and kept >= 0.9, (t, err, kept)
            agree.append((hm == omask).mean())
            if (hm == omask).all():
                assert int(cut.item()) == pytest.approx(ocut, rel=1e-3, abs=50)
            if cut_on_oracle_caps:
                cs, ct, nc, _, _ = O.terms(frames[t], opr, cfg)
                gm, gc, gcode, _ = S.mincut_grid(dev(cs), dev(ct), dev(nc))
                assert gcode == 0 and int(gc.item()) == ocut, t
                np.testing.assert_array_equal(host(gm), omask)
        prev_g, prev_o = hm, omask
    sg.close()
    return agree, cycles


def test_end_to_end_small_clip(S):
    frames, _ = synth.clip_small(10)
    agree, _ = _run_clip(S, frames, O.CONFIG_SMALL, cut_on_oracle_caps=True)
    assert min(agree) >= 0.999, agree


def test_end_to_end_small_clip_gmm3(S):
    frames, _ = synth.clip_small(10)
    agree, _ = _run_clip(S, frames, dict(O.CONFIG_SMALL, gmm_components=3, em_iters=5))
    assert min(agree) >= 0.999, agree


def test_end_to_end_vga_clip_gmm3(S):
    """The paper's M = 3 colour mixtures at 640x480 (Sec. 8.1): the k-means start on the first
    frame, then each frame's EM from the previous frame's mixtures (both sides)."""
    frames = np.stack([f for f, _ in synth.clip_vga_frames(4)])
    agree, _ = _run_clip(S, frames, dict(O.CONFIG_VGA, gmm_components=3, em_iters=5))
    assert min(agree) >= 0.999, agree


def test_gmm_update_and_reset(S):
    """With gmm_update a frame's EM starts from the previous frame's mixtures (so frame 1
    differs from a fresh start on the same prior); a reset returns to the k-means start, so
    the first frame of the new video equals a fresh context's, bit for bit."""
    cfg = dict(O.CONFIG_SMALL, gmm_components=3, em_iters=2)
    frames, _ = synth.clip_small(3, seed=synth.SEED_BASE + 21)
    H, W = frames.shape[1:3]
    a = S.Segmenter(H, W, seg_params(S, cfg))
    outs_a = [tuple(t.clone() for t in a.push_frame(dev(f))) for f in frames[:2]]
    a.sync()
    a.reset()
    again = a.push_frame(dev(frames[0]))
    fresh = S.Segmenter(H, W, seg_params(S, cfg))
    f0 = fresh.push_frame(dev(frames[0]))
    a.sync()
    fresh.sync()
    for x, y in zip(again, f0):
        assert torch.equal(x, y)
    for x, y in zip(outs_a[0], f0):
        assert torch.equal(x, y)
    a.close()
    fresh.close()


def test_end_to_end_vga_clip(S):
    frames = np.stack([f for f, _ in synth.clip_vga_frames(12)])
    agree, _ = _run_clip(S, frames, O.CONFIG_VGA, cut_on_oracle_caps=True)
    assert min(agree) >= 0.999, agree


def test_end_to_end_vga_ambiguous_frames(S):
    """Frames 195-250 of the 640x480 clip, where the fading disk melts into the
    background and its labelling flips (the cuts there need several push-relabel
    cycles).  Both sides start from the oracle's own state after frames 0..194
    (tests/golden, written by the oracle alone)."""
    t0, P0, m0 = golden_vga_state(195)
    assert t0 == 195
    # frames of the 300-frame clip (a clip's frames depend on its length)
    frames = np.stack([f for f, _ in itertools.islice(synth.clip_vga_frames(300), 251)][195:])
    agree, cycles = _run_clip(S, frames, O.CONFIG_VGA, state=(t0, P0, m0), cut_on_oracle_caps=True)
    assert min(agree) >= 0.999, agree
    assert max(cycles) >= 3, cycles  # the window does reach the multi-cycle cuts


@pytest.mark.parametrize("H,W", [(720, 1280), (1080, 1920)])
def test_end_to_end_hd_frames(S, H, W):
    """The larger resolutions of the mixed and serving workloads (same parameters as
    640x480): two frames through seg_push_frame (the second with the Kalman update and
    the previous mask), saliency and prior against the oracle, the cut of the oracle's
    capacities bit-exact."""
    frames = np.stack([f for f, _ in synth.clip_vga_frames(2, H, W, seed=synth.SEED_BASE + 4)])
    agree, _ = _run_clip(S, frames, O.CONFIG_VGA, cut_on_oracle_caps=True)
    assert min(agree) >= 0.999, agree


def test_host_entry_point_and_state_roundtrip(S):
    frames, _ = synth.clip_small(4)
    H, W = frames.shape[1:3]
    p = seg_params(S, O.CONFIG_SMALL)
    a, b = S.Segmenter(H, W, p), S.Segmenter(H, W, p)
    for t in range(2):
        _, _, ma, ca = a.push_frame(dev(frames[t]))
        mh = torch.empty(H, W, dtype=torch.uint8).pin_memory()
        ch = torch.empty(1, dtype=torch.int64).pin_memory()
        b.push_frame_host(torch.from_numpy(frames[t]).pin_memory(), mh, ch)
        a.sync()
        assert torch.equal(ma.cpu(), mh) and int(ca.item()) == int(ch.item())
    st = a.get_state()
    c = S.Segmenter(H, W, p)
    c.set_state(st)
    _, pa, ma, _ = a.push_frame(dev(frames[2]))
    _, pc, mc, _ = c.push_frame(dev(frames[2]))
    a.sync()
    c.sync()
    assert torch.equal(ma, mc) and torch.equal(pa, pc)
    a.reset()
    _, p0, _, _ = a.push_frame(dev(frames[0]))
    fresh = S.Segmenter(H, W, p)
    _, p1, _, _ = fresh.push_frame(dev(frames[0]))
    a.sync()
    fresh.sync()
    assert torch.equal(p0, p1)
    for s in (a, b, c, fresh):
        s.close()


def test_graph_replay_equals_eager_launches(S):
    """seg_push_frame replays a captured CUDA graph; it must give exactly what
    eager launches of the same kernels give (same workspace, same order)."""
    frames, _ = synth.clip_small(5)
    H, W = frames.shape[1:3]
    g = S.Segmenter(H, W, seg_params(S, O.CONFIG_SMALL))
    e = S.Segmenter(H, W, seg_params(S, O.CONFIG_SMALL, use_graph=0))
    for t in range(5):
        outs_g = g.push_frame(dev(frames[t]))
        outs_e = e.push_frame(dev(frames[t]))
        g.sync()
        e.sync()
        for a, b in zip(outs_g, outs_e):
            assert torch.equal(a, b), t
    g.close()
    e.close()


@pytest.mark.parametrize("start", [0, 232])
def test_warm_start_equals_cold_start(S, start):
    """Dynamic graph cuts: starting each cut from the previous frame's n-link flows
    must give exactly the cold-start result (mask, cut value, and so prior)."""
    frames = np.stack([f for f, _ in synth.clip_vga_frames(start + 10)])[start:]
    warm = S.Segmenter(480, 640, seg_params(S, O.CONFIG_VGA))
    cold = S.Segmenter(480, 640, seg_params(S, O.CONFIG_VGA, warm_start=0))
    assert warm.params.warm_start == 1
    for t in range(len(frames)):
        ow = warm.push_frame(dev(frames[t]))
        oc = cold.push_frame(dev(frames[t]))
        assert warm.sync()[0] == 0 and cold.sync()[0] == 0
        for a, b in zip(ow, oc):
            assert torch.equal(a, b), t
    warm.close()
    cold.close()


def test_saliency_grid_equals_context_saliency(S):
    """The context-free saliency entry point runs the same kernels."""
    frames, _ = synth.clip_small(2, seed=synth.SEED_BASE + 77)
    p = S.params_from(O.CONFIG_SMALL)
    sg = S.Segmenter(120, 160, p)
    for f in frames:
        x = torch.from_numpy(f).cuda()
        a = sg.saliency(x)
        b = S.saliency_grid(x, p)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    sg.close()
