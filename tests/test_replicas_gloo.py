"""The multi-process path of bench.py on CPU: two gloo ranks, each segmenting
its own copy of a small clip with the oracle (the replicas share nothing), and
the aggregation that turns per-rank times into one whole-job throughput."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_1008_0502_b300 import synth
    ws2, r2, _ = bench.dist_setup("gloo")
    frames, _ = synth.clip_small(3, seed=synth.SEED_BASE + 1 + 100 * rank)
    sg = O.Segmenter(120, 160, O.CONFIG_SMALL)
    cuts = [sg.push(f)[3] for f in frames]
    t_local = 1.0 + rank  # rank 1 is the slow one
    value, t = bench.aggregate(t_local, len(frames), ws2)
    q.put((r2, ws2, value, t, cuts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_max_time_and_total_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, value, t, cuts) in enumerate(res):
        assert rank == r and ws == 2
        assert t == 2.0 and value == 6 / 2.0  # 3 frames per rank over the slowest rank's 2 s
    assert res[0][4] != res[1][4]  # each replica segmented its own video
    assert all(c >= 0 for c in res[0][4] + res[1][4])


def _rank_failing(rank, ws, port, q):
    import sys
    import time
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), SEG_DIST_TIMEOUT_S="10")
    import bench
    bench.dist_setup("gloo")
    if rank == 1:
        raise SystemExit(3)  # this replica fails between steps, before the aggregation
    t0 = time.perf_counter()
    try:
        bench.aggregate(1.0, 3, ws)
        q.put(("no error", time.perf_counter() - t0))
    except Exception as e:  # the surviving rank learns of it from its collective
        q.put((type(e).__name__, time.perf_counter() - t0))


def test_a_failed_replica_ends_the_others_collective_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_failing, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    what, waited = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
    assert ps[1].exitcode == 3
    assert what != "no error" and waited < 60, (what, waited)
    assert ps[0].exitcode == 0


def test_single_process_aggregate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.0, 10, 1) == (5.0, 2.0)
    # as an ncu launch list of 640x480 frames shows: 13 kernels of the frame, the frame-pointer record of
    # a captured frame, and the saliency half's own record when pipelined
    assert bench.kernels_per_frame(bench.VGA) == 14
    assert bench.kernels_per_frame(bench.VGA, pipeline=True) == 15
    assert bench.kernels_per_frame(bench.VGA, B=8) == 16  # batches: one accumulation per center scale
