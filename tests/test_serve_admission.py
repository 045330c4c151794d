"""Admission and slot reuse of the continuous-batching server, on the host.

The server's groups hold a batch context on the GPU; here a stand-in group
records the same slot bookkeeping so the admission rules run without a GPU:
arrival order, one group per resolution filled slot by slot, a new group only
while its workspace (seg_workspace_bytes, a host-side computation) fits the HBM
budget, and a freed slot going to the next waiting stream as a fresh video."""
import pytest

from paper_1008_0502_b300 import seg, serve


class _FakeFrames:
    def __init__(self, H, W):
        self.shape = (H, W, 3)


class _FakeGroup:
    def __init__(self, H, W, slots, params):
        self.H, self.W, self.B = H, W, slots
        self.sid = [None] * slots
        self.pos = [0] * slots
        self.fresh = [False] * slots

    free_slot = serve._Group.free_slot
    active = serve._Group.active


def _req(sid, H, W, arrival, n=5):
    return serve.Request(sid=sid, frames=lambda t, H=H, W=W: _FakeFrames(H, W), n_frames=n, arrival=arrival)


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(serve, "_Group", _FakeGroup)
    p = seg.default_params()
    one = seg.workspace_bytes(2, 120, 160, p)
    # room for two groups of 160x120 streams, not for a third
    s = serve.Server(p, hbm_budget_bytes=2 * one + one // 2, slots=2)
    return s, one


def test_same_resolution_fills_slots_then_opens_a_group(server):
    s, one = server
    for i in range(3):
        s.submit(_req(i, 120, 160, arrival=0.0))
    s._admit(now=0.0)
    assert s.queue == []
    assert len(s.groups) == 2 and s.used == 2 * one
    assert s.groups[0].sid == [0, 1] and s.groups[1].sid == [2, None]
    assert all(s.results[i].admitted == 0.0 for i in range(3))
    assert s.groups[0].fresh == [True, True]


def test_future_arrivals_wait_and_order_is_by_arrival(server):
    s, _ = server
    s.submit(_req(7, 120, 160, arrival=2.0))
    s.submit(_req(8, 120, 160, arrival=1.0))
    s._admit(now=0.5)
    assert [r.sid for r in s.queue] == [8, 7]  # kept in arrival order
    assert s.groups == []
    s._admit(now=1.5)
    assert [r.sid for r in s.queue] == [7]
    assert s.groups[0].sid == [8, None]
    s._admit(now=2.5)
    assert s.queue == [] and s.groups[0].sid == [8, 7]


def test_budget_refuses_a_group_until_a_slot_frees(server):
    s, one = server
    for i in range(4):
        s.submit(_req(i, 120, 160, arrival=0.0))
    s._admit(now=0.0)
    assert len(s.groups) == 2 and s.queue == []
    # a fifth stream of the same size: both groups full, a third does not fit the budget
    s.submit(_req(4, 120, 160, arrival=0.0))
    s._admit(now=1.0)
    assert [r.sid for r in s.queue] == [4] and s.rejected_groups == 1 and len(s.groups) == 2
    assert s.used == 2 * one
    # a different resolution is refused too (its group would not fit either)
    s.submit(_req(5, 240, 320, arrival=0.0))
    s._admit(now=1.0)
    assert sorted(r.sid for r in s.queue) == [4, 5] and len(s.groups) == 2
    # stream 1 finishes: its slot goes to the next waiting stream of that size, as a new video
    g = s.groups[0]
    g.sid[1] = None
    g.fresh[1] = False
    g.pos[1] = 3
    s._admit(now=2.0)
    assert g.sid[1] == 4 and g.fresh[1] and g.pos[1] == 0
    assert s.results[4].admitted == 2.0
    assert [r.sid for r in s.queue] == [5]
    assert s.used == 2 * one


def test_workspace_grows_with_slots_and_pixels():
    p = seg.default_params()
    a = seg.workspace_bytes(1, 120, 160, p)
    assert seg.workspace_bytes(2, 120, 160, p) > a
    assert seg.workspace_bytes(1, 240, 320, p) > 3 * a
