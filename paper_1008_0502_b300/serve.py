"""Continuous-batching server for many video streams on one GPU.

Streams of the same resolution share a batch context (``seg_create_batch``):
its B slots are B independent streams advanced together by one
``seg_push_frame`` (one CUDA-graph replay) per step.  Each resolution group runs
on a CUDA stream of its own, so the groups' work overlaps on the device.  B
follows the resolution (``slots_for``): the stacked min cut of a batch lasts as
long as its slowest frame, so small frames, each of which leaves most of the GPU
idle, are batched, and a frame that fills the GPU alone runs alone.

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
  (``seg_reset_stream``: previous mask, Kalman variance, warm-start flows and
  colour mixtures of that slot only).  An empty slot is marked as such
  (``seg_set_stream_active``), and the kernels skip its frame.
* Steps overlap: the host does not wait for a step before launching the next
  one; each group keeps up to ``depth`` steps in flight and collects a step's
  results (latencies, kept outputs) once its completion event has passed.  With
  ``busy_groups`` or more groups active the device is full and more steps in
  flight would only queue, so each group then keeps one.  The
  device status (sticky until read) is read every ``STATUS_EVERY`` steps and
  whenever a group drains, since reading it waits for all of the group's work.
* Pipelined groups (``pipeline=True``): each group's context runs a step's
  saliency beside the previous step's prior, terms and cut (seg_pipeline_enable),
  with the frames copied into a ring of three input buffers on a stream of the
  group's own, so nothing of a step waits for the step before except what the
  method orders (the prior needs the previous mask).
* Per-frame latency is client-side: from the frame's submission (the host
  taking it for a step) to its mask and cut being ready on the device (the
  step's completion event, read on the host clock through a reference event).
* Per-stream state (previous mask, Kalman variance, the last cut's flows for the
  warm start, colour mixtures) stays on the device in the slot.

A stream's results do not depend on which slot or group it runs in or on the
other streams of the batch: every per-frame kernel treats the frames of a batch
independently, so a served stream equals the same stream run alone.  With
``slots=1`` every stream gets a context of its own: the plain per-stream launch
the batched server is compared with; ``slots="auto"`` sizes each group by its
resolution (``slots_for``).
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
    def __init__(self, H, W, slots, params, pipeline=False):
        self.H, self.W, self.B = H, W, slots
        self.bytes = 0  # its workspace, charged to the server's budget
        self.stream = torch.cuda.Stream()
        self.pipeline = bool(pipeline)
        self.ctx = seg.Segmenter(H, W, params, stream=self.stream, batch=slots, pipeline=self.pipeline)
        # a pipelined group's next frames are copied on a stream of their own into a
        # ring of input buffers (a buffer is reused once the step that read it is done),
        # so the copy does not wait for the step before, and a step's saliency can
        # overlap the previous step's prior, terms and cut
        nbuf = 3 if self.pipeline else 1
        self.inbufs = [torch.zeros(slots, H, W, 3, dtype=torch.uint8, device="cuda") for _ in range(nbuf)]
        self.buf_done = [None] * nbuf  # completion event of the last step that read each buffer
        self.copy_stream = torch.cuda.Stream() if self.pipeline else self.stream
        self.nstep = 0
        self.outs = self.ctx.empty_outputs()
        self.sid = [None] * slots
        self.pos = [0] * slots
        self.fresh = [False] * slots
        self.on = [True] * slots  # the slots' flags on the device (all on at creation)
        self.inflight = []        # launched steps not yet collected, oldest first
        self.collected = 0        # steps collected (the device status is read every STATUS_EVERY)

    def free_slot(self):
        for b in range(self.B):
            if self.sid[b] is None:
                return b
        return None

    def active(self):
        return any(s is not None for s in self.sid)

    def close(self):
        self.ctx.close()


STATUS_EVERY = 16  # steps of a group between reads of its device status (each read waits for the group)


class Server:
    def __init__(self, params: seg.seg_params, hbm_budget_bytes: int, slots: int | str = "auto",
                 keep_outputs: bool = False, depth: int = 2, group_pixels: int = 1_300_000,
                 pipeline: bool = False, busy_groups: int = 6):
        self.params = params
        self.pipeline = bool(pipeline)  # groups run pipelined contexts (seg_pipeline_enable)
        self.depth = max(1, int(depth))  # steps in flight per group
        self.busy_groups = int(busy_groups)  # with at least this many active groups, one step in flight (0: off)
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.slots = slots  # slots per group, or "auto": group_pixels // (H * W), 1 to 8
        self.group_pixels = int(group_pixels)
        self.keep = keep_outputs
        self.groups: list[_Group] = []
        self.queue: list[Request] = []
        self.requests: dict[int, Request] = {}
        self.results: dict[int, StreamResult] = {}
        self.steps = 0
        self.rejected_groups = 0  # times a new group could not be created (the request waited)
        self.evicted_groups = 0

    def slots_for(self, H: int, W: int) -> int:
        """Slots of a new H x W group.  "auto": as many frames as fit a pixel budget
        (at least 1, at most 8).  A batch's min cut lasts as long as its slowest
        frame, so batching pays where one frame leaves most of the GPU idle (small
        frames) and not where one frame already fills it."""
        if self.slots == "auto":
            return max(1, min(8, self.group_pixels // (H * W)))
        return int(self.slots)

    def group_bytes(self, H: int, W: int) -> int:
        """Device bytes of a new H x W group: the context's workspace plus, when
        pipelined, the library's second saliency buffers and frame ring and this
        server's input ring (about 19 bytes per pixel of the batch, rounded up)."""
        B = self.slots_for(H, W)
        need = seg.workspace_bytes(B, H, W, self.params)
        if self.pipeline:
            need += 2 * 3 * 3 * B * H * W + 4 * B * H * W + (1 << 20)
        return need

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
                need = self.group_bytes(H, W)
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
        while g.inflight:  # its last steps' results first
            self._collect(g)
        g.close()
        self.groups.remove(g)
        self.used -= g.bytes
        self.evicted_groups += 1

    def _new_group(self, H: int, W: int, need: int):
        """A new group, or None when its device allocation fails (after one retry
        with the idle groups freed)."""
        for attempt in range(2):
            try:
                g = _Group(H, W, self.slots_for(H, W), self.params, pipeline=self.pipeline)
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
    def _collect(self, g: _Group):
        """Waits for g's oldest step in flight and records its results.  The device
        status (sticky until read) is read every STATUS_EVERY steps and when the
        group has nothing else in flight: reading it waits for all of the group's
        work, which would otherwise keep only one step in flight."""
        done, stamp, frames, kept = g.inflight.pop(0)
        done.synchronize()
        g.collected += 1
        if not g.inflight or g.collected % STATUS_EVERY == 0:
            code, _ = g.ctx.sync()
            if code != 0:
                raise seg.SegError(code, "serve step")
        t_done = self._t_ref + self._ev_ref.elapsed_time(done) / 1e3  # the host clock
        for b, sid, t_sub in frames:
            r = self.results[sid]
            r.frame_ms.append((t_done - t_sub) * 1e3)
            if b in kept:
                m, p, c = kept[b]
                r.masks.append(m)
                r.priors.append(p)
                r.cuts.append(int(c.item()))
            if len(r.frame_ms) >= self.requests[sid].n_frames:
                r.done = t_done - self._t0

    def step(self, now: float):
        self._admit(now)
        outer = torch.cuda.current_stream()
        launched = 0
        depth = self.depth
        if self.busy_groups and sum(1 for g in self.groups if g.active()) >= self.busy_groups:
            depth = 1  # the device is full: more steps in flight would only queue
        for g in self.groups:
            if not g.active():
                continue
            while len(g.inflight) >= depth:
                self._collect(g)
            j = g.nstep % len(g.inbufs)
            inbuf = g.inbufs[j]
            cs = g.copy_stream  # (the group's own stream unless pipelined)
            cs.wait_stream(outer)  # frames produced on the caller's stream are ready
            if g.buf_done[j] is not None:  # the step that last read this buffer is done
                cs.wait_event(g.buf_done[j])
            with torch.cuda.stream(cs):
                frames = []
                for b in range(g.B):
                    sid = g.sid[b]
                    if g.B > 1 and g.on[b] != (sid is not None):  # empty slots are skipped
                        g.ctx.set_stream_active(b, sid is not None)
                        g.on[b] = sid is not None
                    if sid is None:
                        continue
                    if g.fresh[b]:
                        g.ctx.reset(stream_index=b)
                        g.fresh[b] = False
                    inbuf[b].copy_(self.requests[sid].frame(g.pos[b]), non_blocking=True)
                    frames.append((b, sid, time.perf_counter()))
                # (pipelined: the saliency starts once the copies are done; the prior,
                # terms and cut, and the group's stream, come after the previous step)
                if g.B > 1:
                    sal, pr, mask, cut = g.ctx.push_frame(inbuf, *g.outs)
                else:  # a single-stream context takes one (H, W, 3) frame
                    sal, pr, mask, cut = g.ctx.push_frame(inbuf[0], *g.outs)
                    pr, mask = pr.unsqueeze(0), mask.unsqueeze(0)
            with torch.cuda.stream(g.stream):  # the step's outputs are ready on the group's stream
                if cs is not g.stream:
                    g.stream.wait_stream(cs)
                done = torch.cuda.Event(enable_timing=True)
                done.record(g.stream)
                kept = {}
                if self.keep:
                    kept = {b: (mask[b].clone(), pr[b].clone(), cut[b].clone()) for b, _, _ in frames}
            g.buf_done[j] = done
            g.nstep += 1
            g.inflight.append((done, now, frames, kept))
            for b, sid, _ in frames:  # frame count decides when a slot frees (no wait for the device)
                g.pos[b] += 1
                if g.pos[b] >= self.requests[sid].n_frames:
                    g.sid[b] = None
            launched += 1
        self.steps += 1
        return launched

    def run(self, requests, clock: str = "wall", max_steps: int = 1_000_000):
        """Serve every request to completion.  clock="wall": arrivals in seconds of
        wall time since the start; clock="steps": arrivals in steps."""
        for r in requests:
            self.submit(r)
        # reference event: device timestamps onto the host clock
        self._ev_ref = torch.cuda.Event(enable_timing=True)
        self._ev_ref.record()
        self._ev_ref.synchronize()
        self._t_ref = time.perf_counter()
        t0 = self._t0 = time.perf_counter()
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
        for g in self.groups:
            while g.inflight:
                self._collect(g)
        wall = time.perf_counter() - t0
        for g in self.groups:  # (every group drained above, so this only reads the status)
            code, _ = g.ctx.sync()
            if code != 0:
                raise seg.SegError(code, "serve step")
        frames = sum(len(r.frame_ms) for r in self.results.values())
        lat = np.array([x for r in self.results.values() for x in r.frame_ms]) if frames else np.zeros(1)
        return {"wall_s": wall, "frames": frames, "frames_per_s": frames / wall if wall > 0 else 0.0,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "of": "frame submission on the host to its mask and cut ready on the device"},
                "streams": len(self.results), "groups": len(self.groups), "hbm_bytes": self.used,
                "steps": self.steps, "refused": sum(1 for r in self.results.values() if r.refused),
                "evicted_groups": self.evicted_groups}

    def close(self):
        for g in self.groups:
            g.close()
        self.groups = []
        self.used = 0
