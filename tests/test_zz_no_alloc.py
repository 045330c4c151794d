"""seg_mincut_grid_static, the min cut for callers that may not allocate device
memory (they run under another framework's memory pool, a fixed device-memory
quota, or a real-time loop that forbids allocation after start-up).

It must give exactly the result of the allocating entry point seg_mincut_grid
and of the oracle's Boykov-Kolmogorov max-flow (min cuts are compared bit-exact
everywhere in these tests), on two calls in a row: the second call reuses the
scratch array the first one left behind.  This file sorts last so a
stop-at-first-failure run has already run every other test.
"""
import ctypes as C

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


def test_static_scratch_matches_allocating_entry_point_twice(S):
    cases = [synth.blob_grid_caps(240, 320, 8, 11),            # 76800 px, 8-neighbour
             synth.random_grid_caps(97, 131, 4, 12, tmax=700, nmax=250)]  # ragged, 4-neighbour
    for cs, ct, nc in cases:
        o_cut, o_mask = O.maxflow(cs, ct, nc, "bk")
        ref_mask, ref_cut, ref_code, _ = S.mincut_grid(_dev(cs), _dev(ct), _dev(nc))
        assert ref_code == S.SEG_OK
        assert int(ref_cut.item()) == o_cut and np.array_equal(ref_mask.cpu().numpy(), o_mask)
        H, W = cs.shape
        mask = torch.empty(H, W, dtype=torch.uint8, device="cuda")
        cut = torch.empty(1, dtype=torch.int64, device="cuda")
        mask, cut, code, cycles = S.mincut_grid_static(_dev(cs), _dev(ct), _dev(nc), mask=mask, cut=cut)
        assert code == S.SEG_OK and cycles >= 1
        assert int(cut.item()) == int(ref_cut.item())
        assert torch.equal(mask, ref_mask)


def test_static_scratch_rejects_oversize_grids(S):
    H, W = 512, 257  # 131584 > SEG_MINCUT_STATIC_MAX_PIXELS
    assert H * W > S.SEG_MINCUT_STATIC_MAX_PIXELS
    z = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    nc = torch.zeros(2, H, W, dtype=torch.int32, device="cuda")
    mask = torch.empty(H, W, dtype=torch.uint8, device="cuda")
    cut = torch.empty(1, dtype=torch.int64, device="cuda")
    code = S.lib.seg_mincut_grid_static(None, H, W, 4, C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()),
                                        C.c_void_p(nc.data_ptr()), C.c_void_p(mask.data_ptr()),
                                        C.c_void_p(cut.data_ptr()), 0, None)
    assert code == S.SEG_EINVAL
    # a grid within the limit but without a cut buffer is refused the same way
    H, W = 64, 64
    z = torch.zeros(H, W, dtype=torch.int32, device="cuda")
    nc = torch.zeros(2, H, W, dtype=torch.int32, device="cuda")
    mask = torch.empty(H, W, dtype=torch.uint8, device="cuda")
    code = S.lib.seg_mincut_grid_static(None, H, W, 4, C.c_void_p(z.data_ptr()), C.c_void_p(z.data_ptr()),
                                        C.c_void_p(nc.data_ptr()), C.c_void_p(mask.data_ptr()), None, 0, None)
    assert code == S.SEG_EINVAL
