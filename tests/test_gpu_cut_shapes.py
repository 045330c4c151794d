"""The min cut's tile shapes (seg_params.cut_tile: 0 = 32x16, 1 = 32x8, 2 = 64x8).

Each shape is its own compiled copy of the cut (one thread a node; 256-thread
CTAs for 32x8).  The shape changes which nodes a region discharge and a fixpoint
round see together, never the result: cut values and minimal source sets must
equal the oracle's Boykov-Kolmogorov max-flow bit for bit, on random, ragged,
blob and real frame graphs, and whole frames must equal those of the default
shape on the ambiguous stretch of the clip, also with the frontier schedule and
in a batch with an empty slot.
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


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("H,W,nbr", CUT_CASES)
def test_shape_cut_random_grids_bit_exact(S, shape, H, W, nbr):
    sg = S.Segmenter(H, W, S.params_from(O.CONFIG_SMALL, neighbourhood=nbr, cut_tile=shape))
    for seed in range(2):
        cs, ct, nc = synth.random_grid_caps(H, W, nbr, 1000 * H + W + seed + 7, tmax=800, nmax=300,
                                            p_zero=0.15 * seed)
        v, m = O.maxflow(cs, ct, nc)
        mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
        assert sg.sync(check=False)[0] == 0
        assert int(cut.item()) == v
        np.testing.assert_array_equal(mask.cpu().numpy(), m)
    sg.close()


@pytest.mark.parametrize("shape", [1, 2])
def test_shape_cut_blob_and_frame_graphs_bit_exact(S, shape):
    for H, W, nbr in ((97, 131, 8), (480, 640, 8), (64, 96, 4)):
        cs, ct, nc = synth.blob_grid_caps(H, W, nbr, H + W)
        v, m = O.maxflow(cs, ct, nc)
        sg = S.Segmenter(H, W, S.params_from(O.CONFIG_SMALL, neighbourhood=nbr, cut_tile=shape))
        mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
        assert sg.sync(check=False)[0] == 0 and int(cut.item()) == v
        np.testing.assert_array_equal(mask.cpu().numpy(), m)
        sg.close()
    f = next(synth.clip_vga_frames(1))[0]
    sal = O.saliency(f, O.CONFIG_VGA)
    _, pr = O.prior(sal, None, 0.0, O.CONFIG_VGA)
    cs, ct, nc, _, _ = O.terms(f, pr, O.CONFIG_VGA)
    v, m = O.maxflow(cs, ct, nc)
    sg = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA, cut_tile=shape))
    mask, cut = sg.mincut(_dev(cs), _dev(ct), _dev(nc))
    assert sg.sync(check=False)[0] == 0 and int(cut.item()) == v
    np.testing.assert_array_equal(mask.cpu().numpy(), m)
    sg.close()


@pytest.mark.parametrize("shape,frontier", [(1, 0), (2, 0), (1, 1)])
def test_shape_frames_equal_default_shape_on_ambiguous_frames(S, shape, frontier):
    frames = np.stack([f for f, _ in synth.clip_vga_frames(300)][:251])
    a = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA, cut_tile=shape, relabel_frontier=frontier))
    b = S.Segmenter(480, 640, S.params_from(O.CONFIG_VGA))
    for t in range(251):
        x = _dev(frames[t])
        oa = a.push_frame(x)
        ob = b.push_frame(x)
        if t >= 195:
            assert a.sync(check=False)[0] == 0 and b.sync(check=False)[0] == 0
            for u, w in zip(oa, ob):
                assert torch.equal(u, w), t
    a.close()
    b.close()


@pytest.mark.parametrize("shape", [1, 2])
def test_shape_batch_with_empty_slot_equals_solo(S, shape):
    params = S.params_from(O.CONFIG_SMALL, cut_tile=shape)
    clips = [_dev(synth.clip_small(3, seed=synth.SEED_BASE + 95 + k)[0]) for k in range(3)]
    sg = S.Segmenter(120, 160, params, batch=3)
    outs = sg.empty_outputs()
    sg.set_stream_active(1, False)
    got = []
    for t in range(3):
        _, pr, m, c = sg.push_frame(torch.stack([clips[0][t], clips[0][t], clips[2][t]]), *outs)
        got.append((m.clone(), c.clone()))
    assert sg.sync()[0] == 0
    for k in (0, 2):
        solo = S.Segmenter(120, 160, S.params_from(O.CONFIG_SMALL))
        for t in range(3):
            _, _, m, c = solo.push_frame(clips[k][t])
            assert torch.equal(got[t][0][k], m) and int(got[t][1][k]) == int(c.item()), (k, t)
        solo.close()
    sg.close()


def test_cut_tile_is_validated(S):
    with pytest.raises(S.SegError):
        S.Segmenter(64, 64, S.params_from(O.CONFIG_SMALL, cut_tile=3))
    with pytest.raises(S.SegError):
        S.Segmenter(64, 64, S.params_from(O.CONFIG_SMALL, cut_tile=-1))
