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
