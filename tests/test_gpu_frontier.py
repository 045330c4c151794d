"""The min cut's frontier schedule (seg_params.relabel_frontier = 1).

From the third fixpoint round of a global relabel (the BFS from t) or of the
final reach on, the tiles to visit come from a queue: a tile whose fixpoint moved
a rim node appends the neighbour tiles whose halo holds that node, each tile at
most once a round, with warp-ballot compaction, and the CTAs share the queue.
The schedule changes the order of work only: the cut value and the minimal
source set must equal the oracle's Boykov-Kolmogorov result bit for bit, and
whole frames must equal the default schedule's, on the ambiguous stretch of the
clip (frames 195-250, up to ten push-relabel cycles) as on easy frames, warm or
cold, alone or in a batch with an empty slot.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_0502_b300 import synth

pytestmark = pytest.mark.gpu

CUT_CASES = [(1, 1, 4), (1, 37, 4), (29, 1, 8), (4, 4, 8), (16, 32, 4), (17, 33, 8), (33, 65, 4),
             (50, 70, 8), (120, 160, 4), (121, 161, 8)]


@pytest.fixture(scope="module")
def S(cuda_ok):
    from paper_1008_0502_b300 import build
    build.build()
    from paper_1008_0502_b300 import seg
    return seg


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cut_ctx(S, H, W, nbr):
    p = S.params_from(O.CONFIG_SMALL, neighbourhood=nbr, relabel_frontier=1)
    return S.Segmenter(H, W, p)


@pytest.mark.parametrize("H,W,nbr", CUT_CASES)
def test_frontier_cut_random_grids_bit_exact(S, H, W, nbr):
    sg = _cut_ctx(S, H, W, nbr)
    for seed in range(3):
        cs, ct, nc = synth.random_grid_caps(H, W, nbr, 1000 * H + W + seed, tmax=800, nmax=300,
                                            p_zero=0.1 * seed)
        v, m = O.maxflow(cs, ct, nc)
        mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
        code, cycles = sg.sync(check=False)
        assert code == 0 and cycles >= 1
        assert int(cut.item()) == v
        np.testing.assert_array_equal(mask.cpu().numpy(), m)
    sg.close()


@pytest.mark.parametrize("H,W,nbr", [(64, 96, 4), (97, 131, 8), (480, 640, 8)])
def test_frontier_cut_blob_grids_bit_exact(S, H, W, nbr):
    cs, ct, nc = synth.blob_grid_caps(H, W, nbr, H + W)
    v, m = O.maxflow(cs, ct, nc)
    sg = _cut_ctx(S, H, W, nbr)
    mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
    assert sg.sync(check=False)[0] == 0
    assert int(cut.item()) == v
    np.testing.assert_array_equal(mask.cpu().numpy(), m)
    sg.close()


def test_frontier_cut_frame_graph_bit_exact(S):
    f = next(synth.clip_vga_frames(1))[0]
    sal = O.saliency(f, O.CONFIG_VGA)
    _, pr = O.prior(sal, None, 0.0, O.CONFIG_VGA)
    cs, ct, nc, _, _ = O.terms(f, pr, O.CONFIG_VGA)
    v, m = O.maxflow(cs, ct, nc)
    sg = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA, relabel_frontier=1))
    mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
    assert sg.sync(check=False)[0] == 0
    assert int(cut.item()) == v
    np.testing.assert_array_equal(mask.cpu().numpy(), m)
    sg.close()


@pytest.mark.parametrize("warm", [1, 0])
def test_frontier_frames_equal_default_schedule_on_ambiguous_frames(S, warm):
    """Clip frames 195-250, where the fading disk melts into the background and
    cuts need up to ten cycles (several relabels of many rounds each)."""
    frames = np.stack([f for f, _ in synth.clip_vga_frames(300)][:251])
    a = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA, relabel_frontier=1, warm_start=warm))
    b = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA, relabel_frontier=0, warm_start=warm))
    cyc = []
    for t in range(251):
        x = _dev(frames[t])
        oa = a.push_frame(x)
        ob = b.push_frame(x)
        if t >= 195:
            ca, na = a.sync(check=False)
            cb, _ = b.sync(check=False)
            assert ca == 0 and cb == 0
            cyc.append(na)
            for u, w in zip(oa, ob):
                assert torch.equal(u, w), t
    assert max(cyc) >= 3  # the stretch exercises multi-relabel cuts
    a.close()
    b.close()


def test_frontier_batch_with_empty_slot_equals_solo(S):
    """The frontier schedule together with an empty slot (the cut instantiation that
    leaves frames out): the other slots equal their streams run alone."""
    params = S.params_from(O.CONFIG_SMALL, relabel_frontier=1)
    clips = [_dev(synth.clip_small(3, seed=synth.SEED_BASE + 90 + k)[0]) for k in range(3)]
    sg = S.Segmenter(120, 160, params, batch=3)
    outs = sg.empty_outputs()
    sg.set_stream_active(1, False)
    got = []
    for t in range(3):
        _, pr, m, c = sg.push_frame(torch.stack([clips[0][t], clips[0][t], clips[2][t]]), *outs)
        got.append((m.clone(), c.clone()))
    assert sg.sync()[0] == 0
    for k in (0, 2):
        solo = S.Segmenter(120, 160, params)
        for t in range(3):
            _, _, m, c = solo.push_frame(clips[k][t])
            assert torch.equal(got[t][0][k], m) and int(got[t][1][k]) == int(c.item()), (k, t)
        solo.close()
    sg.close()
