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
    fail_allocs = 0  # the next n creations fail as a device allocation would (host-side fault injection)
    closed = []

    def __init__(self, H, W, slots, params, pipeline=False):
        if _FakeGroup.fail_allocs > 0:
            _FakeGroup.fail_allocs -= 1
            raise seg.SegError(seg.SEG_ENOMEM, "seg_create_batch")
        self.H, self.W, self.B = H, W, slots
        self.bytes = 0
        self.sid = [None] * slots
        self.pos = [0] * slots
        self.fresh = [False] * slots
        self.inflight = []  # (no step is ever launched here)

    free_slot = serve._Group.free_slot
    active = serve._Group.active

    def close(self):
        _FakeGroup.closed.append((self.H, self.W))


def _req(sid, H, W, arrival, n=5):
    return serve.Request(sid=sid, frames=lambda t, H=H, W=W: _FakeFrames(H, W), n_frames=n, arrival=arrival)


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(serve, "_Group", _FakeGroup)
    _FakeGroup.fail_allocs = 0
    _FakeGroup.closed = []
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
    # a different resolution waits too (its group would not fit beside the two running ones)
    s.submit(_req(5, 90, 120, arrival=0.0))
    s._admit(now=1.0)
    assert sorted(r.sid for r in s.queue) == [4, 5] and len(s.groups) == 2 and s.results[5].refused == ""
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


def _finish(g, b):
    g.sid[b] = None


def test_a_group_that_can_never_fit_is_refused_not_queued(server):
    s, one = server
    big = seg.workspace_bytes(2, 480, 640, s.params)
    assert big > s.budget
    s.submit(_req(0, 480, 640, arrival=0.0))
    s._admit(now=0.0)
    assert s.queue == [] and s.groups == [] and s.used == 0
    assert "exceeds" in s.results[0].refused and s.results[0].admitted < 0


def test_idle_groups_are_freed_for_a_new_resolution(server):
    s, one = server
    other = seg.workspace_bytes(2, 90, 120, s.params)
    for i in range(4):
        s.submit(_req(i, 120, 160, arrival=0.0))
    s._admit(now=0.0)
    assert len(s.groups) == 2
    # a 90x120 stream cannot get a group while both 160x120 groups run
    s.submit(_req(9, 90, 120, arrival=0.0))
    s._admit(now=1.0)
    assert [r.sid for r in s.queue] == [9] and s.evicted_groups == 0
    # group 2 goes idle: freeing it makes room, group 1 keeps running
    g0, g1 = s.groups
    _finish(g1, 0)
    _finish(g1, 1)
    s._admit(now=2.0)
    assert s.queue == [] and s.evicted_groups == 1 and _FakeGroup.closed == [(120, 160)]
    assert s.groups[0] is g0 and (s.groups[1].H, s.groups[1].W) == (90, 120)
    assert s.used == one + other and s.results[9].admitted == 2.0


def test_no_group_is_freed_when_that_would_not_make_room(server):
    s, one = server
    for i in range(4):
        s.submit(_req(i, 120, 160, arrival=0.0))
    s._admit(now=0.0)
    g0, g1 = s.groups
    _finish(g1, 0)
    _finish(g1, 1)
    # a resolution whose group fits the budget, but not beside the running group even
    # with the idle one freed: the idle group stays and the stream waits
    H, W = next((h, w) for h, w in [(150, 200), (160, 200), (180, 220), (200, 240)]
                if s.budget - one < seg.workspace_bytes(2, h, w, s.params) <= s.budget)
    s.submit(_req(9, H, W, arrival=0.0))
    s._admit(now=1.0)
    assert [r.sid for r in s.queue] == [9] and s.results[9].refused == ""
    assert s.groups == [g0, g1] and s.evicted_groups == 0 and _FakeGroup.closed == []
    # once the running group goes idle too, both are freed and the stream is admitted
    _finish(g0, 0)
    _finish(g0, 1)
    s._admit(now=2.0)
    assert s.queue == [] and s.evicted_groups == 2 and [(g.H, g.W) for g in s.groups] == [(H, W)]


def test_allocation_failure_waits_while_others_run_and_is_refused_otherwise(server):
    s, one = server
    s.submit(_req(0, 120, 160, arrival=0.0, n=3))
    s._admit(now=0.0)
    assert len(s.groups) == 1
    # a second resolution: the device allocation fails while group 1 runs -> it waits
    _FakeGroup.fail_allocs = 2
    s.submit(_req(1, 90, 120, arrival=0.0))
    s._admit(now=1.0)
    assert [r.sid for r in s.queue] == [1] and s.rejected_groups == 1 and s.results[1].refused == ""
    # group 1 finishes; the allocation fails again, is retried once with the idle group
    # freed, and succeeds
    _finish(s.groups[0], 0)
    _FakeGroup.fail_allocs = 1
    s._admit(now=2.0)
    assert s.queue == [] and s.evicted_groups == 1 and [(g.H, g.W) for g in s.groups] == [(90, 120)]
    assert s.used == seg.workspace_bytes(2, 90, 120, s.params)
    # nothing running and every allocation failing: refused instead of waiting forever
    _finish(s.groups[0], 0)
    _FakeGroup.fail_allocs = 5
    s.submit(_req(2, 240, 320, arrival=0.0))
    s.budget = 10 ** 12
    s._admit(now=3.0)
    assert s.queue == [] and "allocation failed" in s.results[2].refused


def test_auto_slots_size_groups_by_resolution(monkeypatch):
    """slots="auto": a group holds as many frames as fit the pixel budget (1 to 8), so
    small frames batch and a frame that fills the GPU alone runs alone; the workspace
    charged to the budget is that of the group's own slot count."""
    monkeypatch.setattr(serve, "_Group", _FakeGroup)
    _FakeGroup.fail_allocs = 0
    p = seg.default_params()
    s = serve.Server(p, hbm_budget_bytes=1 << 40, slots="auto", group_pixels=2_600_000)
    assert [s.slots_for(h, w) for h, w in ((240, 320), (480, 640), (720, 1280), (1080, 1920), (2160, 3840))] == \
        [8, 8, 2, 1, 1]
    for i, (h, w) in enumerate(((480, 640), (720, 1280), (1080, 1920))):
        s.submit(_req(i, h, w, arrival=0.0))
    s._admit(now=0.0)
    assert [g.B for g in s.groups] == [8, 2, 1]
    assert s.used == sum(seg.workspace_bytes(g.B, g.H, g.W, p) for g in s.groups)
    assert serve.Server(p, 1 << 40, slots=3).slots_for(1080, 1920) == 3
