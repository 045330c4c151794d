"""The min-cut schedule autotuner: every candidate gives the same cut (the tuner
checks it), and it returns the fastest candidate's parameters."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1008_0502_b300 import synth

pytestmark = pytest.mark.gpu


def test_autotune_returns_a_candidate_and_equal_cuts(cuda_ok):
    from paper_1008_0502_b300 import build
    build.build()
    from paper_1008_0502_b300 import seg, tune
    frames = torch.from_numpy(synth.clip_small(6, seed=synth.SEED_BASE + 9)[0]).cuda()
    cands = ((16, 2), (8, 1), (4, 2))
    r = tune.autotune_mincut(frames, seg.params_from(O.CONFIG_SMALL), candidates=cands)
    assert (r.local_iters, r.global_relabel_every) in cands
    assert set(r.ms_per_frame) == set(cands)
    assert r.params.local_iters == r.local_iters and r.params.global_relabel_every == r.global_relabel_every


def test_autotune_over_tile_shapes_and_schedules(cuda_ok):
    """Candidates that change the compiled tile shape (32x16, 32x8, 64x8) and the
    relabel schedule; the tuner checks every one gives the same masks and cuts, on
    a 2-stream batch, and returns the fastest one's parameters."""
    from paper_1008_0502_b300 import build
    build.build()
    from paper_1008_0502_b300 import seg, tune
    clip = synth.clip_small(7, seed=synth.SEED_BASE + 10)[0]
    frames = torch.from_numpy(np.stack([clip[t:t + 2] for t in range(5)])).cuda()
    cands = ({}, {"cut_tile": 1}, {"cut_tile": 2, "local_iters": 16}, {"relabel_frontier": 1})
    r = tune.autotune_mincut(frames, seg.params_from(O.CONFIG_SMALL), candidates=cands, batch=2)
    assert r.best in [dict(c) for c in cands]
    assert len(r.ms_per_frame) == 4 and all(v > 0 for v in r.ms_per_frame.values())
    for f in tune.TUNED_FIELDS:
        want = r.best.get(f, getattr(seg.params_from(O.CONFIG_SMALL), f))
        assert getattr(r.params, f) == want
    with pytest.raises(ValueError):
        tune.autotune_mincut(frames, candidates=({"levels": 5},), batch=2)
