#!/usr/bin/env python
"""Throughput of the per-frame path on seeded synthetic 640x480 video.

A step is one pass over the whole 300-frame clip (the temporal state reset,
then frames 0..299 in order, every frame through the whole path: saliency map,
Kalman-updated prior, MRF terms, exact min cut via seg_push_frame).  The clip
is resident in HBM (276 MB, larger than L2).  --steps K times K passes, so
every timed region holds the clip's easy frames and its ambiguous ones
(frames 200-249, where the fading disk's labelling flips and the cut needs
several push-relabel cycles).  Reported:

  value      frames/s over all ranks, device-resident input (CUDA events),
             frames pipelined (a frame's saliency overlaps the previous
             frame's prior, terms and cut)
  e2e        frames/s from pinned host frames (seg_push_frame_host_async,
             mask and cut value back, one synchronisation at the end), and
             frame by frame (one synchronisation per frame)
  latency    p50/p99 of per-frame device time over every frame of the timed
             passes (events around each frame)
  roofline   the dominant stage's kernel against the measured HBM peak
  cpu_baseline  the FP64 C oracle on a bounded sample of the same clip, one
             core; cpu_baseline_all_cores: one oracle stream per host core
  mincut_profile  the cut's in-kernel time by push-relabel cycles per frame
             and per phase (device timer, one profiled pass over the clip)
  accuracy   Sec. 8.1's error rate, recall, precision and F-value of the
             masks against the clip's synthetic ground truth (sanity only,
             computed on the host after the timed regions)

--impl reference runs that oracle as the reference arm (rank 0 only): a step
is one frame, the K frames spread evenly over the same clip.
Multi-GPU: independent replicas (each rank segments its own copy of the clip;
no collective on the data path), launched by torchrun.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "640x480 frames/s (saliency+Kalman+min-cut, 1 B300) vs plain; p99 frame latency"
H, W = 480, 640
# one push-relabel cycle reads and writes each node's state once: excess 4 B + height 4 B + 4 undirected
# n-link flows x 4 B (8-neighbour)
BYTES_MINCUT_CYCLE_PX = 24
# DRAM bytes (ncu dram__bytes_read + dram__bytes_write) of one k_maxflow<8> launch on a 640x480
# frame graph, from a capture of this workload; None once the kernel changes
TRAFFIC_MAXFLOW = 18524416
VGA = dict(levels=9, c_min=2, c_max=4, d_min=3, d_max=4, n_orient=4, gabor_lambda=4.0, gabor_sigma=2.0,
           gabor_radius=6, norm_tile=8, norm_flat=1e-5, w=(1 / 3, 1 / 6, 1 / 6, 1 / 3), cs_opponent_sum=1,
           border_px=1, sigma1=0.03, sigma2=0.035, f_sigma=2.0, f_radius=6, eps=1e-4, lambda_u=1.0,
           lambda_p=0.0, lambda_s=1.5, sigma_I=0.05, cap_scale=1000.0, neighbourhood=8)
WORKLOAD = ("640x480 RGB8 synthetic clip, 300 frames: low-passed grey texture panned 1 px/frame, "
            "moving yellow ellipse, static 45-degree grating, fading grey disk; 9-level pyramid, "
            "c in 2..4, s = c+3..4, 4 orientations, 8-neighbour grid, int32 capacities")
CLIP_FRAMES = 300


def bench_config():
    """The config of both arms' JSON lines (the same dict)."""
    return {"workload": WORKLOAD, "H": H, "W": W, "frames": CLIP_FRAMES, "parallelism": "replicas",
            "step": "one pass over the whole clip (reset, frames 0..299)",
            "l2": "inputs larger than L2 (276 MB resident clip)"}


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10, help="timed passes over the clip")
    ap.add_argument("--warmup", type=int, default=3, help="untimed passes before them")
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the batched-context measurements")
    ap.add_argument("--only", choices=["saliency_b32", "diff_b32"], default=None,
                    help="run one sub-measurement alone and print its JSON (for profiling)")
    return ap.parse_args()


def make_clip(n, with_gt=False):
    from paper_1008_0502_b300 import synth
    if with_gt:
        return synth.clip_vga(n)  # (frames, ground-truth masks), the same frames
    return np.stack([f for f, _ in synth.clip_vga_frames(n)])


def mincut_profile(stats):
    """Summary of per-frame min-cut statistics (seg_profile_read_ex: cycles, global
    relabels, fixpoint rounds, then device-timer time in initialisation, global
    relabels, discharge cycles and the final reach, in units of 0.1 us): the cut's
    in-kernel time by the number of push-relabel cycles a frame needed, and the
    mean time per phase."""
    a = np.asarray(stats, np.float64).reshape(-1, 7)
    out = {"frames": int(a.shape[0]), "by_cycles": {}, "phase_us_mean": {},
           "of": "device-timer spans inside the cut kernel, profiled frames"}
    if not a.shape[0]:
        return out
    span = a[:, 3:7].sum(1) / 10.0
    for name, sel in (("<=1", a[:, 0] <= 1), ("2", a[:, 0] == 2), (">=3", a[:, 0] >= 3)):
        if sel.any():
            out["by_cycles"][name] = {"frames": int(sel.sum()), "mean_us": float(span[sel].mean()),
                                      "share_of_time": float(span[sel].sum() / span.sum()) if span.sum() else 0.0}
    out["phase_us_mean"] = dict(zip(["init", "global_relabel", "discharge", "final_reach"],
                                    (a[:, 3:7].mean(0) / 10.0).tolist()))
    return out


def confusion(mask, gt):
    """(TP, TN, FP, FN) pixel counts of a 0/1 mask against a 0/1 ground truth."""
    m = np.asarray(mask).astype(bool)
    g = np.asarray(gt).astype(bool)
    if m.shape != g.shape:
        raise ValueError(f"mask {m.shape} vs ground truth {g.shape}")
    tp = int(np.count_nonzero(m & g))
    fp = int(np.count_nonzero(m & ~g))
    fn = int(np.count_nonzero(~m & g))
    return np.array([tp, m.size - tp - fp - fn, fp, fn], np.int64)


def seg_accuracy(counts):
    """Sec. 8.1's accuracy measures from summed (TP, TN, FP, FN): the error rate is
    the fraction of mislabelled pixels, recall the share of object pixels labelled
    object, precision the share of object labels that are right, and the F-value
    their harmonic mean.  A ratio whose denominator is zero is None."""
    tp, tn, fp, fn = (int(c) for c in counts)
    tot = tp + tn + fp + fn
    err = (fp + fn) / tot if tot else None
    rec = tp / (tp + fn) if tp + fn else None
    prec = tp / (tp + fp) if tp + fp else None
    f = 2 * rec * prec / (rec + prec) if rec is not None and prec is not None and rec + prec > 0 else None
    return {"error": err, "recall": rec, "precision": prec, "f_value": f}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0}, "fallback"


def kernels_per_frame(p, H=480, W=640, graph=True, pipeline=False, B=1):
    """Kernels one seg_push_frame launches (memsets excluded), as the library sequences them."""
    dims = [(H, W)]
    for _ in range(p["levels"] - 1):
        h, w = dims[-1]
        dims.append(((h + 1) // 2, (w + 1) // 2))
    tiled = 0
    for l in range(1, p["levels"] - 1):
        if dims[l + 1][0] * dims[l + 1][1] <= 2048:
            break
        tiled += 1
    tail = 1 if 1 + tiled < p["levels"] - 1 else 0
    # rgb max, features + first REDUCE, tiled REDUCEs, tail, Gabor, cs stats, the
    # across-scale accumulation (one fused launch for up to two REDUCE steps and
    # batches of up to 4 frames, else one per center scale), conspicuity
    span = p["c_max"] - p["c_min"]
    accum = 1 if span <= 2 and B <= 4 else span + 1
    sal = 2 + tiled + tail + 1 + 1 + accum + 1
    # prior, moments, terms; min cut; frame-pointer record(s): one per captured half
    return sal + 3 + 1 + (1 if graph else 0) + (1 if graph and pipeline else 0)


def spread_frames(n, n_clip=CLIP_FRAMES):
    """n frame indices spread evenly over the clip (0, n_clip/n, 2 n_clip/n, ..)."""
    return [int(i * n_clip // n) % n_clip for i in range(n)]


def cpu_baseline(clip, seconds):
    """The oracle on one core over frames spread evenly across the clip (so the sample
    holds easy and ambiguous frames alike), each frame from the oracle's state after
    the previous sampled frame.  The number of frames is set from the first frame's
    time so the sample takes about `seconds`."""
    import oracle as O
    sg = O.Segmenter(H, W, O.CONFIG_VGA)
    t0 = time.perf_counter()
    sg.push(clip[0])
    t1 = time.perf_counter() - t0
    n = int(min(len(clip), max(3, seconds / max(t1, 1e-3))))
    idx = spread_frames(n, len(clip))
    sg = O.Segmenter(H, W, O.CONFIG_VGA)
    t0 = time.perf_counter()
    for f in idx:
        sg.push(clip[f])
    return idx, time.perf_counter() - t0


def _oracle_stream(args):
    """One independent oracle stream (a spawned worker): consecutive frames of the clip from `start`."""
    start, seconds = args
    sys.path.insert(0, ROOT)
    import itertools

    import oracle as O
    from paper_1008_0502_b300 import synth
    # frames start.. of the 300-frame clip (a clip's frames depend on its length)
    frames = [f for f, _ in itertools.islice(synth.clip_vga_frames(CLIP_FRAMES), start, start + 40)]
    sg = O.Segmenter(H, W, O.CONFIG_VGA)
    t0 = time.perf_counter()
    n = 0
    while (time.perf_counter() - t0 < seconds or n < 2) and n < len(frames):
        sg.push(frames[n])
        n += 1
    return n, time.perf_counter() - t0


def cpu_baseline_ncores(seconds, max_workers=64):
    """The oracle on every host core: one independent stream per core (streams are
    independent; a stream's frames are sequential), each in a spawned process."""
    import multiprocessing as mp
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ncpu = max(1, min(ncpu, max_workers))
    with mp.get_context("spawn").Pool(ncpu) as pool:
        res = pool.map(_oracle_stream, [((k * CLIP_FRAMES // ncpu) % (CLIP_FRAMES - 40), seconds)
                                        for k in range(ncpu)])
    return sum(n / t for n, t in res), ncpu, sum(n for n, _ in res)


def aggregate(t_local: float, frames_local: int, ws: int, device="cpu"):
    """Whole-job throughput of independent replicas: frames summed over ranks
    divided by the slowest rank's time (max over ranks)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_local], dtype=torch.float64, device=device)
        ff = torch.tensor([frames_local], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(ff, op=dist.ReduceOp.SUM)
        return float(ff.item()) / float(tt.item()), float(tt.item())
    return frames_local / t_local, t_local


def batched_suite(seg, torch, clip_dev, plain_fps, hbm):
    """Batch contexts against plain per-stream contexts (extra keys of the bench line)."""
    from paper_1008_0502_b300 import synth
    out = {}
    p = seg.params_from(VGA)

    def timed(fn, steps, warm=3, streams=()):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # 8 streams of 640x480 in one batch context
    B = 8
    sgb = seg.Segmenter(H, W, p, batch=B)
    outs = sgb.empty_outputs()
    idx = [(37 * k) % clip_dev.shape[0] for k in range(B)]
    frames = torch.stack([clip_dev[i] for i in idx])
    steps = 40
    t = timed(lambda: sgb.push_frame(frames, *outs), steps)
    code, _ = sgb.sync()
    out["vga_b8"] = {"streams": "8 x 640x480", "frames_per_s": B * steps / t, "vs_plain": B * steps / t / plain_fps,
                     "status": code}
    sgb.close()

    # frame-batched saliency, 32 x 640x480 in one call: HBM roofline of the stage
    B = 32
    sgs = seg.Segmenter(H, W, p, batch=B)
    fr32 = torch.stack([clip_dev[(9 * k) % clip_dev.shape[0]] for k in range(B)])
    sal32 = torch.empty(B, H, W, dtype=torch.float32, device="cuda")
    reps = 20
    t = timed(lambda: sgs.saliency(fr32, sal32), reps)
    byts = 7 * B * H * W  # RGB8 in + FP32 saliency out
    ach = byts * reps / t / 1e9
    out["saliency_b32"] = {"frames": "32 x 640x480", "ms_per_call": t / reps * 1e3, "algorithmic_bytes": byts,
                           "achieved_GBps": ach, "frac_of_hbm": ach / hbm}
    sgs.close()

    # the paper's M = 3 EM colour mixtures (Sec. 4 / Sec. 7.3), single 640x480 stream
    sg3 = seg.Segmenter(H, W, seg.params_from(VGA, gmm_components=3, em_iters=5))
    o3 = sg3.empty_outputs()
    pos = [0]

    def step3():
        sg3.push_frame(clip_dev[pos[0] % clip_dev.shape[0]], *o3)
        pos[0] += 1

    t = timed(step3, 100)
    out["gmm3"] = {"streams": "1 x 640x480, M = 3 EM (5 iterations)", "frames_per_s": 100 / t,
                   "status": sg3.sync()[0]}
    sg3.close()

    # the backward form (differentiation of saliency and Kalman prior): a 32-frame 640x480
    # clip, forward + hand-written reverse pass
    d, fwd, bwd, byts = diff_setup(seg, torch, clip_dev)
    reps = 10
    tf = timed(fwd, reps)
    tfb = timed(lambda: (fwd(), bwd()), reps)
    tb = tfb - tf
    out["diff_b32"] = {"frames": "32 x 640x480 float, forward + backward (frames, w, Q, R)",
                       "frames_per_s": 32 * reps / tfb, "ms_forward": tf / reps * 1e3,
                       "ms_backward": tb / reps * 1e3,
                       "backward_achieved_GBps": byts["bwd"] * reps / tb / 1e9,
                       "backward_frac_of_hbm": byts["bwd"] * reps / tb / 1e9 / hbm}
    d.close()

    # the mixed 64-stream workload: one batch context per resolution, the three advanced
    # by one CUDA graph launch per step (seg_group); each context's tile shape and
    # schedule chosen by the autotuner on the group's own step frames (every candidate
    # checked to give the same masks and cuts); against the same streams, each in a
    # plain context of its own with the default (single-stream tuned) parameters
    from paper_1008_0502_b300 import tune
    groups = [(24, 240, 320), (24, 480, 640), (16, 720, 1280)]
    nfr = 4
    data, tuned, plain = [], [], []
    for gi, (nb, h, w) in enumerate(groups):
        clip = np.stack([f for f, _ in synth.clip_vga_frames(nfr + nb, h, w, seed=synth.SEED_BASE + 4 + gi)])
        # stream k of the group sees frames k .. k+nfr-1 of the group's clip
        fr = torch.from_numpy(np.stack([clip[t:t + nb] for t in range(nfr)])).cuda()  # (nfr, nb, h, w, 3)
        data.append(fr)
        tuned.append(tune.autotune_mincut(torch.cat([fr, fr]), p, batch=nb))
        plain.append([seg.Segmenter(h, w, p) for _ in range(nb)])

    def group_of(params):
        ctxs = [seg.Segmenter(h, w, q, batch=nb, stream=torch.cuda.Stream())
                for (nb, h, w), q in zip(groups, params)]
        return ctxs, seg.Group(ctxs), [c.empty_outputs() for c in ctxs]

    def run_group(params, steps):
        ctxs, grp, outs = group_of(params)
        step = [0]

        def batched_step():
            grp.push([fr[step[0] % nfr] for fr in data], outs)
            step[0] += 1

        t = timed(batched_step, steps)
        codes = [c for c, _ in grp.sync()]
        grp.close()
        for c in ctxs:
            c.close()
        return t, max(codes, key=abs)

    steps = 12
    tb, code = run_group([r.params for r in tuned], steps)
    tu, code_u = run_group([p] * len(groups), steps)
    pouts = [[sgp.empty_outputs() for sgp in grp] for grp in plain]
    pstep = [0]

    def plain_step():
        t_ = pstep[0] % nfr
        for grp, fr, po in zip(plain, data, pouts):
            for k, sgp in enumerate(grp):
                sgp.push_frame(fr[t_][k], *po[k])
        pstep[0] += 1

    tp = timed(plain_step, steps)
    n = sum(g[0] for g in groups)
    out["mixed64"] = {"streams": "24 x 320x240 + 24 x 640x480 + 16 x 1280x720", "frames_per_s": n * steps / tb,
                      "launch": "one CUDA graph per step for the three batch contexts (seg_group)",
                      "tuned": {f"{nb}x{w}x{h}": r.best for (nb, h, w), r in zip(groups, tuned)},
                      "untuned_frames_per_s": n * steps / tu, "plain_frames_per_s": n * steps / tp,
                      "vs_plain": tp / tb, "steps": steps, "status": max([code, code_u], key=abs)}
    for grp in plain:
        for sgp in grp:
            sgp.close()
    return out


def serving_suite(seg, torch, horizon_s=1.0, budget_gb=32.0):
    """The serving workload: Poisson arrivals (20 streams/s) of streams lasting
    60-600 frames at 640x480, 1280x720 or 1920x1080, served by the
    continuous-batching server with admission by HBM footprint (slots per group
    by resolution, pipelined groups; also unpipelined, and with 8 slots at every
    resolution), and the same requests through plain per-stream contexts (one slot
    per context, unpipelined, each stream on a CUDA stream of its own, the same
    admission)."""
    from paper_1008_0502_b300 import serve, synth
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 5))
    sizes = [(480, 640), (720, 1280), (1080, 1920)]
    pools = {}
    for k, (h, w) in enumerate(sizes):
        pools[(h, w)] = torch.from_numpy(
            np.stack([f for f, _ in synth.clip_vga_frames(8, h, w, seed=synth.SEED_BASE + 6 + k)])).cuda()
    specs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / 20.0)
        if t >= horizon_s:
            break
        h, w = sizes[int(rng.integers(0, 3))]
        n = int(rng.integers(60, 601))
        off = int(rng.integers(0, 8))
        specs.append((len(specs), (h, w), n, off, t))

    def requests():
        return [serve.Request(sid, (lambda tt, pool=pools[hw], off=off: pool[(off + tt) % 8]), n, arr)
                for sid, hw, n, off, arr in specs]

    # untimed warm-up of every kernel and graph the runs use (first launches load modules)
    warm = serve.Server(seg.params_from(VGA), int(budget_gb * 2**30), slots=2)
    warm.run([serve.Request(k, (lambda tt, pool=pools[hw]: pool[tt % 8]), 6, 0.0)
              for k, hw in enumerate(sizes * 2)], clock="steps")
    warm.close()
    torch.cuda.synchronize()
    out = {}
    for name, slots, pipe in (("served", "auto", True), ("served_unpipelined", "auto", False),
                              ("served_8", 8, False), ("plain", 1, False)):
        srv = serve.Server(seg.params_from(VGA), int(budget_gb * 2**30), slots=slots, pipeline=pipe)
        stats = srv.run(requests(), clock="wall")
        waits = [r.admitted - r.arrival for r in srv.results.values() if r.admitted >= 0] or [0.0]
        srv.close()
        torch.cuda.synchronize()
        stats["admission_wait_ms"] = {"p50": float(np.percentile(waits, 50)) * 1e3, "max": float(np.max(waits)) * 1e3}
        out[name] = stats
    res = dict(out["served"])
    keys = ("frames_per_s", "latency_ms", "wall_s", "groups", "admission_wait_ms")
    res.update({"vs_plain": res["frames_per_s"] / out["plain"]["frames_per_s"],
                "plain": {k: out["plain"][k] for k in keys},
                "served_unpipelined": {k: out["served_unpipelined"][k] for k in keys},
                "served_8_slots": {k: out["served_8"][k] for k in keys},
                "arrivals_per_s": 20, "horizon_s": horizon_s, "hbm_budget_gb": budget_gb,
                "mix": "Poisson arrivals, 60-600 frames, 640x480 / 1280x720 / 1920x1080; served: slots per "
                       "group by resolution (1.3 Mpx per group: 4 / 1 / 1), empty slots skipped, steps "
                       "overlapping (2 in flight per group, 1 while 6 or more groups are active), pipelined groups (a step's saliency beside the "
                       "previous step's prior, terms and cut); served_unpipelined: the same without "
                       "pipelining; served_8_slots: 8 slots at every resolution, unpipelined; plain: one "
                       "unpipelined context per stream"})
    return res


def dist_setup(backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import datetime

        import torch.distributed as dist
        # a rank that dies makes the others' next collective fail within this bound
        # instead of waiting out the library default
        timeout = datetime.timedelta(seconds=float(os.environ.get("SEG_DIST_TIMEOUT_S", "600")))
        dist.init_process_group(backend=backend, timeout=timeout)
    return ws, rank, local


def run_reference(a):
    """The reference arm: the FP64 oracle as it stands, one core, rank 0 only.  A step
    is one frame; the K timed frames are spread evenly over the 300-frame clip (a
    full pass per step would take minutes per step), each segmented from the
    oracle's state after the previous sampled frame."""
    ws, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    clip = make_clip(CLIP_FRAMES)
    import oracle as O
    sg = O.Segmenter(H, W, O.CONFIG_VGA)
    for i in range(a.warmup):
        sg.push(clip[i % len(clip)])
    idx = spread_frames(a.steps, len(clip))
    sg = O.Segmenter(H, W, O.CONFIG_VGA)
    t0 = time.perf_counter()
    for f in idx:
        sg.push(clip[f])
    dt = time.perf_counter() - t0
    v = a.steps / dt
    shown = ", ".join(str(f) for f in idx[:4]) + (", .., " + str(idx[-1]) if len(idx) > 4 else "")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(),
        "cpu_baseline": {"value": v, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": f"{a.steps} frames spread evenly over the 300-frame clip (frames {shown}), "
                         "each from the oracle's state after the previous sampled frame; single-threaded "
                         "FP64 C oracle; a step is one frame here, one pass over the clip in the CUDA arm"},
        "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def diff_setup(seg, torch, clip_dev, B=32):
    """The backward form on a clip batch: B float frames of 640x480 (clip times 0..B-1),
    smoothed previous masks, cotangents on both outputs."""
    p = seg.params_from(VGA)
    d = seg.DiffContext(B, H, W, p)
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.stack([clip_dev[k % clip_dev.shape[0]] for k in range(B)]).float()
    x += torch.rand(x.shape, generator=g, device="cuda") - 0.5
    fmap = torch.rand(B, H, W, generator=g, device="cuda")
    gp = torch.randn(B, H, W, generator=g, device="cuda")
    gs = torch.randn(B, H, W, generator=g, device="cuda")
    theta = seg.theta_from(p)
    outs = [torch.empty(B, H, W, device="cuda") for _ in range(2)]
    g_rgb = torch.empty(B, H, W, 3, device="cuda")
    g_th = torch.empty(6, dtype=torch.float64, device="cuda")

    def fwd():
        d.forward(x, theta, fmap, 0, *outs)

    def bwd():
        d.backward(x, theta, gp, gs, fmap, g_rgb, g_th)

    # minimal traffic per pixel: forward rgb 12 B + fmap 4 B in, saliency and prior 8 B
    # out; backward rgb 12 B + fmap 4 B + two cotangents 8 B in, dL/drgb 12 B out
    return d, fwd, bwd, {"fwd": 24 * B * H * W, "bwd": 36 * B * H * W}


def run_only(a):
    import torch
    from paper_1008_0502_b300 import seg
    pk, _ = peaks()
    clip_dev = torch.from_numpy(make_clip(CLIP_FRAMES)[:40]).cuda()
    if a.only == "diff_b32":
        d, fwd, bwd, byts = diff_setup(seg, torch, clip_dev)
        for _ in range(a.warmup):
            fwd()
            bwd()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            fwd()
            bwd()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        print(json.dumps({"only": a.only, "ms_per_fwd_bwd": t / a.steps * 1e3, "frames_per_s": 32 * a.steps / t}))
        d.close()
        return
    B = 32
    sgs = seg.Segmenter(H, W, seg.params_from(VGA), batch=B)
    fr32 = torch.stack([clip_dev[k] for k in range(B)])
    sal32 = torch.empty(B, H, W, dtype=torch.float32, device="cuda")
    for _ in range(a.warmup):
        sgs.saliency(fr32, sal32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        sgs.saliency(fr32, sal32)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    byts = 7 * B * H * W
    print(json.dumps({"only": a.only, "ms_per_call": t / a.steps * 1e3,
                      "achieved_GBps": byts * a.steps / t / 1e9, "frac": byts * a.steps / t / 1e9 / pk["hbm_gbs"]}))


def run_b300(a):
    import torch
    ws, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_1008_0502_b300 import seg
    clip, gt = make_clip(CLIP_FRAMES, with_gt=True)
    n_clip = len(clip)
    clip_dev = torch.from_numpy(clip).cuda()
    p = seg.params_from(VGA)
    if ws > 1:
        import torch.distributed as dist

    def one_pass(sg, outs, evs=None, k0=0):
        """One step: reset the stream's temporal state, then every frame of the clip."""
        sg.reset()
        st = sg.stream
        for f in range(n_clip):
            if evs is not None:
                evs[k0 + f][0].record(st)
            sg.push_frame(clip_dev[f], *outs)
            if evs is not None:
                evs[k0 + f][1].record(st)

    def timed_pass(pipeline, clocks=False):
        """W warm-up passes, then K timed passes over the clip (CUDA graph replays,
        pipelined or not) on the context's stream; one event pair per frame."""
        sg = seg.Segmenter(H, W, p, pipeline=pipeline)
        outs = sg.empty_outputs()
        st = sg.stream
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(a.steps * n_clip)]
        # the clock sampler starts first; the warm-up passes keep the GPU busy while it
        # comes up (an idle gap before the timed frames lets the clocks drop)
        clk = Clocks(local) if clocks else None
        t_w = time.perf_counter()
        w = 0
        while w < a.warmup or (clocks and time.perf_counter() - t_w < 0.3):
            one_pass(sg, outs)
            sg.outputs_ready()
            torch.cuda.current_stream().synchronize()
            w += 1
        sg.sync()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        for k in range(a.steps):
            one_pass(sg, outs, evs, k * n_clip)
        ev1.record(st)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ck = clk.stop() if clk else None
        code, _ = sg.sync()
        if code != 0:
            raise RuntimeError(f"device status {seg.strerror(code)}")
        v, tt = aggregate(ev0.elapsed_time(ev1) / 1e3, a.steps * n_clip, ws, device="cuda")
        lt = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
        sg.close()
        return v, tt, lt, ck

    # headline: pipelined frames (frame t's saliency overlaps frame t-1's prior, terms
    # and cut; same results bit for bit); then the same passes unpipelined, whose
    # per-frame event pairs give the full per-frame latency
    value, t, period, clocks = timed_pass(True, clocks=True)
    value_plain, _, lat, _ = timed_pass(False)

    def other_contexts(n=4, passes=2):
        """Pipelined frames/s of n more fresh contexts (outside every timed region):
        a context's pipelined rate settles at one of a few levels depending on
        where its buffers land, so one context's figure varies between runs."""
        rates = []
        for _ in range(n):
            sgc = seg.Segmenter(H, W, p, pipeline=True)
            outs = sgc.empty_outputs()
            for _ in range(2):
                one_pass(sgc, outs)
            sgc.outputs_ready()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(sgc.stream)
            for _ in range(passes):
                one_pass(sgc, outs)
            e1.record(sgc.stream)
            torch.cuda.synchronize()
            code_c, _ = sgc.sync()
            if code_c != 0:
                raise RuntimeError(f"device status {seg.strerror(code_c)}")
            rates.append(passes * n_clip / (e0.elapsed_time(e1) / 1e3))
            sgc.close()
        return rates

    rates_ctx = other_contexts()
    sg = seg.Segmenter(H, W, p)
    sal, pr, mask, cut = sg.empty_outputs()

    # per-stage split and min-cut statistics: one more pass over the whole clip with
    # events between the stages (eager launches)
    sg.profile_enable(True)
    one_pass(sg, (sal, pr, mask, cut))
    prof = sg.profile_read()
    sg.profile_enable(False)
    nfr = prof["frames"]
    stage = [x / nfr for x in prof["stage_ms"]]
    cycles = prof["cycles"] / nfr

    # end to end through the host-buffer entry points: pinned RGB8 frames in, mask and
    # cut out, every copy inside the timed region.  Streamed (pipelined context, no host
    # wait per frame, one sync at the end; K passes over the clip) and frame by frame
    # (seg_push_frame_host: one sync per frame; one pass)
    rgb_h = torch.from_numpy(clip).pin_memory()
    masks_h = torch.empty(8, H, W, dtype=torch.uint8).pin_memory()
    cuts_h = torch.empty(8, 1, dtype=torch.int64).pin_memory()
    sgp = seg.Segmenter(H, W, p, pipeline=True)
    for i in range(3):
        sgp.push_frame_host_async(rgb_h[i], masks_h[i], cuts_h[i])
    sgp.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(a.steps):
        sgp.reset()
        for f in range(n_clip):
            sgp.push_frame_host_async(rgb_h[f], masks_h[f % 8], cuts_h[f % 8])
    code_e2e, _ = sgp.sync()
    e2e_value, t_e2e = aggregate(time.perf_counter() - t0, a.steps * n_clip, ws, device="cuda")
    sgp.close()
    if code_e2e != 0:
        raise RuntimeError(f"device status {seg.strerror(code_e2e)}")
    mask_h = torch.empty(H, W, dtype=torch.uint8).pin_memory()
    cut_h = torch.empty(1, dtype=torch.int64).pin_memory()
    sg.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in range(n_clip):
        sg.push_frame_host(rgb_h[f], mask_h, cut_h)
    e2e_sync, _ = aggregate(time.perf_counter() - t0, n_clip, ws, device="cuda")
    # accuracy of the masks against the clip's synthetic ground truth (Sec. 8.1's
    # measures; a sanity figure, outside every timed region): the whole clip again
    sg.reset()
    conf = np.zeros(4, np.int64)
    for f in range(n_clip):
        sg.push_frame_host(rgb_h[f], mask_h, cut_h)
        conf += confusion(mask_h.numpy(), gt[f])
    sg.close()
    if rank != 0:
        return
    pk, pk_kind = peaks()
    hbm = float(pk["hbm_gbs"])
    names = ["saliency", "prior", "terms", "mincut"]
    # the dominant kernel (largest share of the ncu launch list) is k_maxflow: the
    # min-cut stage is that one kernel plus three small memsets
    mincut_bytes = BYTES_MINCUT_CYCLE_PX * H * W * cycles
    ach = mincut_bytes / (stage[3] * 1e-3) / 1e9
    roof = {"kernel": "k_maxflow<8>", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": TRAFFIC_MAXFLOW,
            "algorithmic_bytes": f"{BYTES_MINCUT_CYCLE_PX} B/px per push-relabel cycle x {H * W} px x "
                                 f"{cycles:.2f} cycles (mean over the clip)",
            "peak_kind": pk_kind, "note": "latency-bound (grid barriers, a few busy tiles), not HBM-bound"}
    batched = batched_suite(seg, torch, clip_dev, value / ws, hbm) if a.batched else None
    serving = serving_suite(seg, torch) if a.batched else None
    idx_cpu, dt_cpu = cpu_baseline(clip, a.cpu_seconds)
    n_cpu = len(idx_cpu)
    v_all, cores_all, n_all = cpu_baseline_ncores(0.6 * a.cpu_seconds)
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t * 1e3 / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/i32", "data": "synthetic",
        "config": bench_config(),
        "frames_timed": {"per_step": n_clip, "total": a.steps * n_clip,
                         "which": "every frame of the clip, 0..299, once per step"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max()),
                       "of": f"unpipelined frames (full per-frame device time), all {lat.size} frames of "
                             f"{a.steps} passes"},
        "pipelined": {"frames_per_s": value, "frame_period_ms": {"p50": float(np.percentile(period, 50)),
                      "p99": float(np.percentile(period, 99))},
                      "unpipelined_frames_per_s": value_plain,
                      "other_contexts_frames_per_s": rates_ctx,
                      "other_contexts_note": "4 more fresh pipelined contexts, 2 passes each after 2 warm-up "
                                             "passes, outside the timed region: the spread of the headline "
                                             "between runs"},
        "stages_ms": dict(zip(names, stage)), "mincut_cycles_mean": cycles,
        "mincut_profile": mincut_profile(prof["mincut_stats"]),
        "roofline": roof,
        "cpu_baseline": {"value": n_cpu / dt_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_cpu} frames spread evenly over the same clip (every "
                                   f"{CLIP_FRAMES / n_cpu:.1f}th), each from the oracle's state after the previous "
                                   "sampled frame, single-threaded FP64 C oracle"},
        "cpu_baseline_all_cores": {"value": v_all, "unit": "frames/s", "cores": cores_all, "kind": "oracle",
                                   "sample": f"{cores_all} independent streams, one per core (spawned "
                                   f"processes), {n_all} frames of the same clip in all"},
        "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": H * W * 3,
                "d2h_bytes_per_step": H * W + 8, "path": "seg_push_frame_host_async, pinned host frames, "
                "one sync at the end", "frame_by_frame": e2e_sync},
        "accuracy": dict(seg_accuracy(conf), frames=n_clip,
                         of="masks against the clip's synthetic ground truth (ellipse, grating, and the disk "
                         "while its contrast is at least half), pixel counts summed over the frames; "
                         "a sanity figure"),
        "batched": batched,
        "serving": serving,
        "gpu_launches": a.steps * n_clip * kernels_per_frame(VGA, pipeline=True),
        "clocks": clocks,
    }
    print(json.dumps(out))


def main():
    a = args()
    if a.only:
        run_only(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_b300(a)


if __name__ == "__main__":
    main()
