"""Multi-stream batching: B same-size video streams advanced by one call.

Every stream of a batch must give exactly (bit for bit: saliency, prior, mask,
cut value) what a single-stream context gives on the same frames, because the
per-frame kernels index frames independently and the stacked min cut is the
B independent cuts side by side.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_0502_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S(cuda_ok):
    from paper_1008_0502_b300 import build
    build.build()
    from paper_1008_0502_b300 import seg
    return seg


def _clips_small(n_streams, n_frames):
    return [synth.clip_small(n_frames, seed=synth.SEED_BASE + 1 + 17 * k)[0] for k in range(n_streams)]


def _run_single(S, params, frames):
    H, W = frames.shape[1:3]
    sg = S.Segmenter(H, W, params)
    outs = []
    for f in frames:
        sal, pr, m, c = sg.push_frame(torch.from_numpy(f).cuda())
        outs.append((sal.clone(), pr.clone(), m.clone(), c.clone()))
    sg.sync()
    sg.close()
    return outs


def _run_batch(S, params, clips):
    B = len(clips)
    H, W = clips[0].shape[1:3]
    sg = S.Segmenter(H, W, params, batch=B)
    outs = []
    for t in range(clips[0].shape[0]):
        x = torch.from_numpy(np.stack([c[t] for c in clips])).cuda()
        sal, pr, m, c = sg.push_frame(x if B > 1 else x[0])
        outs.append((sal.clone(), pr.clone(), m.clone(), c.clone()))
    code, _ = sg.sync()
    assert code == 0
    sg.close()
    return outs


@pytest.mark.parametrize("cfg_name,B", [("small", 3), ("small", 1), ("vga", 2), ("small_gmm3", 2)])
def test_batch_streams_equal_single_streams(S, cfg_name, B):
    """small_gmm3: the M = 3 colour mixtures, each stream carrying its own from frame to frame."""
    if cfg_name == "small":
        cfg, clips = O.CONFIG_SMALL, _clips_small(B, 4)
    elif cfg_name == "small_gmm3":
        cfg, clips = dict(O.CONFIG_SMALL, gmm_components=3, em_iters=3), _clips_small(B, 4)
    else:
        cfg = O.CONFIG_VGA
        allf = np.stack([f for f, _ in synth.clip_vga_frames(110)])
        clips = [allf[0:3], allf[100:103]][:B]
    p = S.params_from(cfg)
    batch = _run_batch(S, p, clips)
    for k in range(B):
        single = _run_single(S, p, clips[k])
        for t in range(len(single)):
            bs, bp, bm, bc = batch[t]
            ss, sp, sm, sc = single[t]
            if B > 1:
                bs, bp, bm = bs[k], bp[k], bm[k]
            assert torch.equal(bs, ss), (k, t)
            assert torch.equal(bp, sp), (k, t)
            assert torch.equal(bm, sm), (k, t)
            assert int(bc[k]) == int(sc[0]), (k, t)


def test_batch_matches_oracle_per_stream(S):
    clips = _clips_small(2, 3)
    outs = _run_batch(S, S.params_from(O.CONFIG_SMALL), clips)
    for k in range(2):
        ref = O.Segmenter(120, 160, O.CONFIG_SMALL)
        for t in range(3):
            osal, opr, omask, ocut = ref.push(clips[k][t])
            sal, pr, m, c = outs[t]
            assert np.abs(sal[k].cpu().numpy() - osal).max() <= 1e-4 * np.abs(osal).max()
            assert (m[k].cpu().numpy() == omask).mean() >= 0.999


def test_reset_one_stream_and_state_roundtrip(S):
    clips = _clips_small(2, 4)
    p = S.params_from(O.CONFIG_SMALL)
    sg = S.Segmenter(120, 160, p, batch=2)
    for t in range(2):
        sg.push_frame(torch.from_numpy(np.stack([clips[0][t], clips[1][t]])).cuda())
    state = sg.get_state()
    sg.reset(stream_index=1)  # stream 1 starts a new video with clips[1][2:]
    _, pr, m, _ = sg.push_frame(torch.from_numpy(np.stack([clips[0][2], clips[1][2]])).cuda())
    single0 = _run_single(S, p, clips[0][:3])
    single1 = _run_single(S, p, clips[1][2:3])
    assert torch.equal(pr[0], single0[2][1]) and torch.equal(m[0], single0[2][2])
    assert torch.equal(pr[1], single1[0][1]) and torch.equal(m[1], single1[0][2])
    other = S.Segmenter(120, 160, p, batch=2)
    other.set_state(state)
    _, pr2, m2, _ = other.push_frame(torch.from_numpy(np.stack([clips[0][2], clips[1][2]])).cuda())
    assert torch.equal(pr2[0], single0[2][1])
    assert not torch.equal(pr2[1], pr[1])  # restored stream 1 still had its history
    sg.close()
    other.close()
