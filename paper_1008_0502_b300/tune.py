"""Autotuner for the min cut's schedule on a given resolution and frame mix.

The cut is exact for every schedule, so the tuner only measures: it pushes the
same sample frames through a context per candidate (local push/relabel sweeps
per tile visit, global relabel interval), times them with CUDA events, checks
that every candidate produced the same masks and cut values, and returns the
parameters of the fastest one.  Typical use: once per resolution before serving
(`serve.Server` takes the tuned params), or `python -m paper_1008_0502_b300.tune`.
"""
from __future__ import annotations

import dataclasses

import torch

from . import seg

CANDIDATES = ((16, 2), (12, 1), (10, 1), (8, 1), (8, 2), (6, 2), (4, 2))


@dataclasses.dataclass
class TuneResult:
    params: seg.seg_params
    local_iters: int
    global_relabel_every: int
    ms_per_frame: dict  # (local_iters, global_relabel_every) -> ms


def autotune_mincut(frames: torch.Tensor, params: seg.seg_params | None = None, candidates=CANDIDATES,
                    batch: int = 1, pipeline: bool = False) -> TuneResult:
    """frames: (T, H, W, 3) uint8 CUDA tensor (or (T, B, H, W, 3) for a batch context)."""
    base = params if params is not None else seg.default_params()
    T = int(frames.shape[0])
    H, W = int(frames.shape[-3]), int(frames.shape[-2])
    timings, ref = {}, None
    for li, gr in candidates:
        p = seg.params_from({f: getattr(base, f) for f, _ in seg.seg_params._fields_ if f != "w"},
                            w=tuple(base.w), local_iters=li, global_relabel_every=gr)
        sg = seg.Segmenter(H, W, p, batch=batch, pipeline=pipeline)
        outs = [sg.empty_outputs() for _ in range(T)]
        for t in range(min(T, 3)):  # warm-up (graph capture), then a fresh video
            sg.push_frame(frames[t], *outs[t])
        sg.outputs_ready()
        sg.sync()
        sg.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(sg.stream)
        for t in range(T):
            sg.push_frame(frames[t], *outs[t])
        e1.record(sg.stream)
        sg.outputs_ready()
        code, _ = sg.sync()
        if code != 0:
            raise seg.SegError(code, f"autotune candidate {(li, gr)}")
        timings[(li, gr)] = e0.elapsed_time(e1) / T
        res = [(o[2].cpu(), o[3].cpu()) for o in outs]
        if ref is None:
            ref = res
        elif any(not (torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])) for a, b in zip(ref, res)):
            raise AssertionError(f"schedule {(li, gr)} changed the cut")
        sg.close()
    li, gr = min(timings, key=timings.get)
    best = seg.params_from({f: getattr(base, f) for f, _ in seg.seg_params._fields_ if f != "w"},
                           w=tuple(base.w), local_iters=li, global_relabel_every=gr)
    return TuneResult(best, li, gr, timings)


if __name__ == "__main__":
    import json
    import sys

    import numpy as np

    from . import synth

    H, W = (int(sys.argv[1]), int(sys.argv[2])) if len(sys.argv) > 2 else (480, 640)
    fr = torch.from_numpy(np.stack([f for f, _ in synth.clip_vga_frames(40, H, W)])).cuda()
    r = autotune_mincut(fr)
    print(json.dumps({"H": H, "W": W, "local_iters": r.local_iters, "global_relabel_every": r.global_relabel_every,
                      "ms_per_frame": {f"{k[0]},{k[1]}": v for k, v in r.ms_per_frame.items()}}))
