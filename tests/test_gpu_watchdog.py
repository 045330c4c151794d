"""Failure detection of the min cut's device-side waits (no GPU is faulted or hung).

Every wait of the persistent min-cut kernel at a grid barrier is bounded by the
context's barrier_timeout_us.  With a limit of one microsecond some CTA of a
multi-CTA cut waits longer than that at one of its barriers: it records
SEG_ETIMEOUT, every CTA returns at its next barrier, and the host reads the
status.  The kernel has finished (the stream synchronises), and the same context
then gives the exact cut again at the default limit.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_barrier_time_limit_reports_timeout_and_context_recovers(S):
    H, W = 480, 640
    cs, ct, nc = synth.blob_grid_caps(H, W, 8, H + W)
    o_cut, o_mask = O.maxflow(cs, ct, nc, "bk")
    sg = S.Segmenter(H, W, S.params_from(O.CONFIG_VGA))
    dcs, dct, dnc = _dev(cs), _dev(ct), _dev(nc)

    mask, cut = sg.mincut(dcs, dct, dnc)
    code, cycles = sg.sync(check=False)
    assert code == S.SEG_OK and cycles >= 1
    assert int(cut.item()) == o_cut and np.array_equal(mask.cpu().numpy(), o_mask)

    sg.set_barrier_timeout(1)
    for _ in range(2):  # and a second time on the context the timeout left behind
        sg.mincut(dcs, dct, dnc)
        code, _ = sg.sync(check=False)
        assert code == S.SEG_ETIMEOUT

    sg.set_barrier_timeout(4_000_000)
    mask, cut = sg.mincut(dcs, dct, dnc)
    code, _ = sg.sync(check=False)
    assert code == S.SEG_OK
    assert int(cut.item()) == o_cut and np.array_equal(mask.cpu().numpy(), o_mask)
    sg.close()


def test_timeout_in_a_captured_frame_then_exact_frames(S):
    """The same through seg_push_frame's captured graph: a frame whose cut times out
    reports SEG_ETIMEOUT from seg_sync; after the limit is restored (the graph is
    captured again) a reset stream segments its frames exactly as a fresh context."""
    frames, _ = synth.clip_small(3)
    H, W = frames.shape[1:3]
    p = S.params_from(dict(O.CONFIG_SMALL, barrier_timeout_us=1))
    sg = S.Segmenter(H, W, p)
    sg.push_frame(_dev(frames[0]))
    assert sg.sync(check=False)[0] in (S.SEG_OK, S.SEG_ETIMEOUT)  # a 4-CTA cut may not wait long
    sg.set_barrier_timeout(4_000_000)
    sg.reset()
    fresh = S.Segmenter(H, W, S.params_from(O.CONFIG_SMALL))
    for t in range(3):
        a = sg.push_frame(_dev(frames[t]))
        b = fresh.push_frame(_dev(frames[t]))
        assert sg.sync()[0] == S.SEG_OK and fresh.sync()[0] == S.SEG_OK
        for x, y in zip(a, b):
            assert torch.equal(x, y), t
    sg.close()
    fresh.close()


def test_barrier_time_limit_is_validated(S):
    with pytest.raises(S.SegError):
        S.Segmenter(64, 64, S.params_from(O.CONFIG_SMALL, barrier_timeout_us=0))
    sg = S.Segmenter(64, 64, S.params_from(O.CONFIG_SMALL))
    for bad in (0, -5, 60_000_001):
        with pytest.raises(S.SegError):
            sg.set_barrier_timeout(bad)
    sg.close()
