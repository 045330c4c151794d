"""Continuous-batching server for many video streams on one GPU.

Streams of the same resolution share a batch context (``seg_create_batch``):
its B slots are B independent streams advanced together by one
``seg_push_frame`` (one CUDA-graph replay) per step.  Each resolution group runs
on a CUDA stream of its own, so the groups' work overlaps on the device.

* Admission by HBM footprint: a request whose resolution has a free slot takes
  it; otherwise a new group is created if its workspace
  (``seg_workspace_bytes``) fits the remaining budget, after freeing idle
  groups (no stream in any slot) when that makes it fit; otherwise the request
  waits in the queue.  A request whose group could never fit the budget, or
  whose group's device allocation fails while no other group is running (so
  nothing here will free memory), is refused (``StreamResult.refused``)
  instead of waiting forever.
* Continuous batching: requests are admitted at every step as slots and memory
  free up, while the other streams keep running; a finished stream frees its
  slot, and the next stream admitted there starts a new video
  (``seg_reset_stream``: previous mask, Kalman variance and warm-start flows
  of that slot only).
* Per-stream state (previous mask, Kalman variance, the last cut's flows for the
  warm start) stays on the device in the slot.

A stream's results do not depend on which slot or group it runs in or on the
other streams of the batch: every per-frame kernel treats the frames of a batch
independently, so a served stream equals the same stream run alone.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable

import numpy as np
import torch

from . import seg


@dataclasses.dataclass
class Request:
    sid: int
    frames: Callable[[int], torch.Tensor] | torch.Tensor  # frame t (H, W, 3) uint8 on the device
    n_frames: int
    arrival: float  # seconds (clock="wall") or steps (clock="steps")

    @property
    def shape(self):
        f = self.frame(0)
        return int(f.shape[0]), int(f.shape[1])

    def frame(self, t: int) -> torch.Tensor:
        return self.frames(t) if callable(self.frames) else self.frames[t]


@dataclasses.dataclass
class StreamResult:
    sid: int
    arrival: float
    admitted: float = -1.0
    done: float = -1.0
    frame_ms: list = dataclasses.field(default_factory=list)
    masks: list = dataclasses.field(default_factory=list)
    priors: list = dataclasses.field(default_factory=list)
    cuts: list = dataclasses.field(default_factory=list)
    refused: str = ""  # why the stream was never admitted ("" once admitted or while waiting)


class _Group:
    def __init__(self, H, W, slots, params):
        self.H, self.W, self.B = H, W, slots
        self.bytes = 0  # its workspace, charged to the server's budget
        self.stream = torch.cuda.Stream()
        self.ctx = seg.Segmenter(H, W, params, stream=self.stream, batch=slots)
        self.inbuf = torch.zeros(slots, H, W, 3, dtype=torch.uint8, device="cuda")
        self.outs = self.ctx.empty_outputs()
        self.sid = [None] * slots
        self.pos = [0] * slots
        self.fresh = [False] * slots

    def free_slot(self):
        for b in range(self.B):
            if self.sid[b] is None:
                return b
        return None

    def active(self):
        return any(s is not None for s in self.sid)

    def close(self):
        self.ctx.close()


class Server:
    def __init__(self, params: seg.seg_params, hbm_budget_bytes: int, slots: int = 8, keep_outputs: bool = False):
        self.params = params
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.slots = slots
        self.keep = keep_outputs
        self.groups: list[_Group] = []
        self.queue: list[Request] = []
        self.requests: dict[int, Request] = {}
        self.results: dict[int, StreamResult] = {}
        self.steps = 0
        self.rejected_groups = 0  # times a new group could not be created (the request waited)
        self.evicted_groups = 0

    # -- admission
    def submit(self, req: Request):
        self.queue.append(req)
        self.requests[req.sid] = req
        self.results[req.sid] = StreamResult(req.sid, req.arrival)

    def _admit(self, now: float):
        waiting = []
        for req in sorted(self.queue, key=lambda r: r.arrival):
            if req.arrival > now:
                waiting.append(req)
                continue
            H, W = req.shape
            slot = None
            for g in self.groups:
                if (g.H, g.W) == (H, W):
                    b = g.free_slot()
                    if b is not None:
                        slot = (g, b)
                        break
            if slot is None:
                need = seg.workspace_bytes(self.slots, H, W, self.params)
                if need > self.budget:
                    self.results[req.sid].refused = "its group's workspace exceeds the HBM budget"
                    continue
                if self.used + need > self.budget:
                    self._evict_idle(need)
                g = self._new_group(H, W, need) if self.used + need <= self.budget else None
                if g is None and self.used + need <= self.budget and not any(x.active() for x in self.groups):
                    self.results[req.sid].refused = "device allocation failed with no other group running"
                    continue
                if g is not None:
                    slot = (g, 0)
                else:
                    self.rejected_groups += 1
            if slot is None:
                waiting.append(req)
                continue
            g, b = slot
            g.sid[b] = req.sid
            g.pos[b] = 0
            g.fresh[b] = True
            self.results[req.sid].admitted = now
        self.queue = waiting

    def _evict_idle(self, need: int):
        """Frees idle groups, oldest first, if that lets a new group of `need`
        bytes fit the budget; frees none otherwise."""
        idle = [g for g in self.groups if not g.active()]
        if self.used - sum(g.bytes for g in idle) + need > self.budget:
            return
        for g in idle:
            if self.used + need <= self.budget:
                break
            self._drop(g)

    def _drop(self, g: _Group):
        g.close()
        self.groups.remove(g)
        self.used -= g.bytes
        self.evicted_groups += 1

    def _new_group(self, H: int, W: int, need: int):
        """A new group, or None when its device allocation fails (after one retry
        with the idle groups freed)."""
        for attempt in range(2):
            try:
                g = _Group(H, W, self.slots, self.params)
            except seg.SegError as e:
                if e.code != seg.SEG_ENOMEM:
                    raise
                idle = [x for x in self.groups if not x.active()]
                if attempt or not idle:
                    return None
                for x in idle:
                    self._drop(x)
                continue
            g.bytes = need
            self.groups.append(g)
            self.used += need
            return g
        return None

    # -- one step of every group with an active slot
    def step(self, now: float):
        self._admit(now)
        outer = torch.cuda.current_stream()
        launched = []
        for g in self.groups:
            if not g.active():
                continue
            g.stream.wait_stream(outer)  # frames produced on the caller's stream are ready
            with torch.cuda.stream(g.stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                for b in range(g.B):
                    sid = g.sid[b]
                    if sid is None:
                        continue
                    if g.fresh[b]:
                        g.ctx.reset(stream_index=b)
                        g.fresh[b] = False
                    g.inbuf[b].copy_(self.requests[sid].frame(g.pos[b]), non_blocking=True)
                e0.record(g.stream)
                sal, pr, mask, cut = g.ctx.push_frame(g.inbuf, *g.outs)
                e1.record(g.stream)
                if self.keep:
                    kept = [(b, mask[b].clone(), pr[b].clone(), cut[b].clone()) for b in range(g.B)
                            if g.sid[b] is not None]
                else:
                    kept = []
            launched.append((g, e0, e1, kept))
        for g, e0, e1, kept in launched:
            g.stream.synchronize()
            code, _ = g.ctx.sync()
            if code != 0:
                raise seg.SegError(code, "serve step")
            ms = e0.elapsed_time(e1)
            kept_by_slot = {b: (m, p, c) for b, m, p, c in kept}
            for b in range(g.B):
                sid = g.sid[b]
                if sid is None:
                    continue
                r = self.results[sid]
                r.frame_ms.append(ms)
                if b in kept_by_slot:
                    m, p, c = kept_by_slot[b]
                    r.masks.append(m)
                    r.priors.append(p)
                    r.cuts.append(int(c.item()))
                g.pos[b] += 1
                if g.pos[b] >= self.requests[sid].n_frames:
                    g.sid[b] = None
                    r.done = now
        self.steps += 1
        return len(launched)

    def run(self, requests, clock: str = "wall", max_steps: int = 1_000_000):
        """Serve every request to completion.  clock="wall": arrivals in seconds of
        wall time since the start; clock="steps": arrivals in steps."""
        for r in requests:
            self.submit(r)
        t0 = time.perf_counter()
        while self.steps < max_steps:
            now = time.perf_counter() - t0 if clock == "wall" else float(self.steps)
            pending = self.queue or any(g.active() for g in self.groups)
            if not pending:
                break
            if self.step(now) == 0 and self.queue:
                # nothing on the GPU yet: wait for the next arrival
                nxt = min(r.arrival for r in self.queue)
                if clock == "wall" and nxt > now:
                    time.sleep(min(nxt - now, 0.01))
        wall = time.perf_counter() - t0
        frames = sum(len(r.frame_ms) for r in self.results.values())
        lat = np.array([x for r in self.results.values() for x in r.frame_ms]) if frames else np.zeros(1)
        return {"wall_s": wall, "frames": frames, "frames_per_s": frames / wall if wall > 0 else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "streams": len(self.results), "groups": len(self.groups), "hbm_bytes": self.used,
                "steps": self.steps, "refused": sum(1 for r in self.results.values() if r.refused),
                "evicted_groups": self.evicted_groups}

    def close(self):
        for g in self.groups:
            g.close()
        self.groups = []
        self.used = 0
