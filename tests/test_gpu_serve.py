"""Continuous-batching server: streams of mixed resolutions arriving while
others run, admission by HBM footprint (a full group makes later arrivals wait),
slot reuse.  Every served stream must equal the same stream run alone, bit for
bit (mask, prior, cut value), whatever slot, group or mix it ran in."""
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
    from paper_1008_0502_b300 import seg, serve
    return seg, serve


def _solo(seg, params, frames):
    H, W = frames.shape[1:3]
    sg = seg.Segmenter(H, W, params)
    out = []
    for t in range(frames.shape[0]):
        _, pr, m, c = sg.push_frame(frames[t])
        out.append((m.clone(), pr.clone(), int(c.item())))
    sg.sync()
    sg.close()
    return out


@pytest.mark.parametrize("pipeline", [False, True])
def test_served_streams_equal_solo_runs(S, pipeline):
    """Streams arriving over several steps, waiting for slots, finishing at different
    steps (their slots switched off, then reset for the next stream): each served
    stream equals the same stream run alone, with groups pipelined or not."""
    seg, serve = S
    params = seg.params_from(O.CONFIG_SMALL)
    specs = [  # (sid, H, W, n_frames, arrival step)
        (0, 120, 160, 5, 0), (1, 120, 160, 4, 0), (2, 90, 120, 6, 1), (3, 120, 160, 3, 2), (4, 120, 160, 4, 2),
        (5, 90, 120, 3, 4)]
    clips = {}
    for sid, H, W, n, _ in specs:
        f, _ = synth.clip_small(n, H=H, W=W, seed=synth.SEED_BASE + 50 + sid, radius=min(15, H // 5))
        clips[sid] = torch.from_numpy(f).cuda()
    budget = seg.workspace_bytes(2, 120, 160, params) + seg.workspace_bytes(2, 90, 120, params)
    if pipeline:
        budget = sum(serve.Server(params, 0, slots=2, pipeline=True).group_bytes(h, w) for h, w in ((120, 160),
                                                                                              (90, 120)))
    srv = serve.Server(params, budget, slots=2, keep_outputs=True, pipeline=pipeline)
    reqs = [serve.Request(sid, clips[sid], n, arr) for sid, H, W, n, arr in specs]
    stats = srv.run(reqs, clock="steps")
    assert stats["groups"] == 2 and stats["frames"] == sum(s[3] for s in specs)
    # the two 120x160 slots were busy when streams 3 and 4 arrived: they waited
    assert srv.results[3].admitted > 2 and srv.results[4].admitted > 2
    assert srv.rejected_groups > 0
    for sid, H, W, n, _ in specs:
        r = srv.results[sid]
        solo = _solo(seg, params, clips[sid])
        assert len(r.masks) == n
        for t in range(n):
            assert torch.equal(r.masks[t], solo[t][0]), (sid, t)
            assert torch.equal(r.priors[t], solo[t][1]), (sid, t)
            assert r.cuts[t] == solo[t][2], (sid, t)
    srv.close()


def test_empty_slots_are_skipped_and_streams_unchanged(S):
    """A batch slot marked empty is skipped (no kernel touches its rows); the other
    slots give what they give alone, bit for bit, and the slot turned on again starts a new
    video exactly as a fresh context."""
    seg, _ = S
    params = seg.params_from(O.CONFIG_SMALL)
    clips = [torch.from_numpy(synth.clip_small(4, seed=synth.SEED_BASE + 60 + k)[0]).cuda() for k in range(3)]
    sg = seg.Segmenter(120, 160, params, batch=3)
    outs = sg.empty_outputs()
    sg.set_stream_active(1, False)
    got = []
    for t in range(4):
        if t == 2:  # slot 1 receives stream 1 from its first frame on
            sg.reset(stream_index=1)
            sg.set_stream_active(1, True)
        x = torch.stack([clips[0][t], clips[1][t - 2 if t >= 2 else 0], clips[2][t]])
        sal, pr, m, c = sg.push_frame(x, *outs)
        got.append((m.clone(), pr.clone(), c.clone()))
    assert sg.sync()[0] == 0
    for k in (0, 2):
        solo = _solo(seg, params, clips[k])
        for t in range(4):
            assert torch.equal(got[t][0][k], solo[t][0]) and torch.equal(got[t][1][k], solo[t][1])
            assert int(got[t][2][k]) == solo[t][2]
    solo1 = _solo(seg, params, clips[1][:2])
    for t in (2, 3):
        assert torch.equal(got[t][0][1], solo1[t - 2][0]) and int(got[t][2][1]) == solo1[t - 2][2]
    sg.close()


def test_paused_slot_resumes_where_it_stopped(S):
    """A slot switched off keeps its stream's state (previous mask, Kalman variance,
    warm-start flows, colour mixtures): switched on again without a reset, the stream
    continues as if the skipped steps had not happened.  120-row frames stack so that
    16-row tiles straddle the paused frame and its neighbours."""
    seg, _ = S
    params = seg.params_from(O.CONFIG_SMALL)
    clips = [torch.from_numpy(synth.clip_small(6, seed=synth.SEED_BASE + 70 + k)[0]).cuda() for k in range(3)]
    sg = seg.Segmenter(120, 160, params, batch=3)
    outs = sg.empty_outputs()
    plan1 = [0, 1, None, None, 2, 3]  # slot 1's frame at each step (None: paused)
    got = []
    for t in range(6):
        if t in (2, 4):
            sg.set_stream_active(1, plan1[t] is not None)
        f1 = clips[1][plan1[t] if plan1[t] is not None else 0]
        x = torch.stack([clips[0][t], f1, clips[2][t]])
        _, pr, m, c = sg.push_frame(x, *outs)
        got.append((m.clone(), pr.clone(), c.clone()))
    assert sg.sync()[0] == 0
    for k in (0, 2):
        solo = _solo(seg, params, clips[k])
        for t in range(6):
            assert torch.equal(got[t][0][k], solo[t][0]) and torch.equal(got[t][1][k], solo[t][1]), (k, t)
            assert int(got[t][2][k]) == solo[t][2]
    solo1 = _solo(seg, params, clips[1][:4])
    for t, f in enumerate(plan1):
        if f is None:
            continue
        assert torch.equal(got[t][0][1], solo1[f][0]) and torch.equal(got[t][1][1], solo1[f][1]), (t, f)
        assert int(got[t][2][1]) == solo1[f][2]
    sg.close()


def test_one_slot_groups_equal_solo_runs(S):
    """slots = 1 (the plain per-stream launch the server is compared with): every stream
    in a context of its own, the same results."""
    seg, serve = S
    params = seg.params_from(O.CONFIG_SMALL)
    clips = {k: torch.from_numpy(synth.clip_small(3, seed=synth.SEED_BASE + 80 + k)[0]).cuda() for k in range(2)}
    srv = serve.Server(params, 1 << 34, slots=1, keep_outputs=True)
    srv.run([serve.Request(k, clips[k], 3, float(k)) for k in range(2)], clock="steps")
    assert len(srv.groups) == 2
    for k in range(2):
        solo = _solo(seg, params, clips[k])
        for t in range(3):
            assert torch.equal(srv.results[k].masks[t], solo[t][0]) and srv.results[k].cuts[t] == solo[t][2]
    srv.close()


def test_served_latency_is_submission_to_mask(S):
    seg, serve = S
    params = seg.params_from(O.CONFIG_SMALL)
    f = torch.from_numpy(synth.clip_small(6, seed=synth.SEED_BASE + 70)[0]).cuda()
    srv = serve.Server(params, 1 << 34, slots=4)
    stats = srv.run([serve.Request(k, f, 6, 0.0) for k in range(3)], clock="steps")
    lat = [x for r in srv.results.values() for x in r.frame_ms]
    assert len(lat) == 18 and min(lat) > 0 and stats["latency_ms"]["p99"] >= stats["latency_ms"]["p50"] > 0
    assert all(r.done > 0 for r in srv.results.values())
    srv.close()
