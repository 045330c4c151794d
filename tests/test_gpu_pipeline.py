"""Pipelined frames: a frame's saliency overlaps the previous frame's prior, terms
and cut.  The results must equal the unpipelined path bit for bit (same kernels,
same frame order, same temporal state)."""
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


def _run(S, p, frames, B, pipeline):
    H, W = frames.shape[-3:-1]
    sg = S.Segmenter(H, W, p, batch=B, pipeline=pipeline)
    outs = []
    dev = torch.from_numpy(frames).cuda()
    for t in range(frames.shape[0]):
        o = sg.empty_outputs()
        sg.push_frame(dev[t], *o)
        outs.append(o)
    sg.outputs_ready()
    code, _ = sg.sync()
    assert code == 0
    sg.close()
    return [[x.cpu() for x in o] for o in outs]


@pytest.mark.parametrize("case", ["vga", "small_b3", "small_eager"])
def test_pipelined_equals_unpipelined(S, case):
    if case == "vga":
        p = S.params_from(O.CONFIG_VGA)
        frames = np.stack([f for f, _ in synth.clip_vga_frames(9)])
        B = 1
    else:
        p = S.params_from(O.CONFIG_SMALL, use_graph=0 if case == "small_eager" else 1)
        clips = [synth.clip_small(7, seed=synth.SEED_BASE + 3 + 11 * k)[0] for k in range(3)]
        B = 3 if case == "small_b3" else 1
        frames = np.stack(clips, axis=1) if B == 3 else clips[0]
    a = _run(S, p, frames, B, False)
    b = _run(S, p, frames, B, True)
    for t, (x, y) in enumerate(zip(a, b)):
        for u, v in zip(x, y):
            assert torch.equal(u, v), t


def test_async_host_frames_equal_device_frames(S):
    p = S.params_from(O.CONFIG_SMALL)
    frames = synth.clip_small(8, seed=synth.SEED_BASE + 21)[0]
    ref = _run(S, p, frames, 1, False)
    sg = S.Segmenter(120, 160, p, pipeline=True)
    rgb_h = torch.from_numpy(frames).pin_memory()
    masks = torch.empty(len(frames), 120, 160, dtype=torch.uint8).pin_memory()
    cuts = torch.empty(len(frames), 1, dtype=torch.int64).pin_memory()
    for t in range(len(frames)):
        sg.push_frame_host_async(rgb_h[t], masks[t], cuts[t])
    code, _ = sg.sync()
    assert code == 0
    for t in range(len(frames)):
        assert torch.equal(masks[t], ref[t][2]), t
        assert int(cuts[t][0]) == int(ref[t][3][0]), t
    sg.close()


def test_context_stream_orders_reused_outputs(S):
    """One set of output buffers for every frame, each frame's outputs copied on the
    context stream right after the call: with pipelining the prior, terms and cut run
    on an internal stream, yet the context stream must pass a frame's outputs only
    once they are complete, and the next frame must not overwrite them before the
    work enqueued on the context stream has read them.  Both the plain C call
    (seg_push_frame, no input event) and seg_push_frame_ev are checked against the
    unpipelined path."""
    import ctypes as C
    p = S.params_from(O.CONFIG_SMALL)
    frames = synth.clip_small(8, seed=synth.SEED_BASE + 23)[0]
    ref = _run(S, p, frames, 1, False)
    dev = torch.from_numpy(frames).cuda()
    torch.cuda.synchronize()  # (the frames are on the device before any context stream reads them)
    for use_ev in (False, True):
        sg = S.Segmenter(120, 160, p, pipeline=True)
        sal, pr, mask, cut = sg.empty_outputs()
        got = []
        for t in range(len(frames)):
            if use_ev:
                sg.push_frame(dev[t], sal, pr, mask, cut)
            else:
                with torch.cuda.stream(sg.stream):
                    code = S.lib.seg_push_frame(sg.handle, C.c_void_p(dev[t].data_ptr()), C.c_void_p(sal.data_ptr()),
                                                C.c_void_p(pr.data_ptr()), C.c_void_p(mask.data_ptr()),
                                                C.c_void_p(cut.data_ptr()))
                assert code == 0
            with torch.cuda.stream(sg.stream):
                got.append([x.clone() for x in (sal, pr, mask, cut)])
        code, _ = sg.sync()
        assert code == 0
        for t in range(len(frames)):
            for u, v in zip(got[t], ref[t]):
                assert torch.equal(u.cpu(), v), (use_ev, t)
        sg.close()
