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


def test_served_streams_equal_solo_runs(S):
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
    srv = serve.Server(params, budget, slots=2, keep_outputs=True)
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
