"""The multi-rank path of the benchmark on two CPU ranks (gloo): each rank
renders its own cameras (rank 0 the workload's), the job's throughput is the
pixels of all ranks over the slowest rank's time, the same on every rank, and
the scene's vertex gradients are summed over the ranks (each rank's views
give part of them).  No GPU is involved: the per-rank gradients come from
the oracle."""

import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_2406_01579_b300.multirank import (allreduce_grads, job_mpix_s, max_over_ranks,
                                             rank_cameras)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        base = synth.scene_sphere16().cams * 2
        cams = rank_cameras(base, rank, 64, 48)
        sig = np.concatenate([np.asarray(c.R, np.float64).ravel() for c in cams])
        sigs = [None] * world
        dist.all_gather_object(sigs, sig)
        pixels = sum(c.width * c.height for c in cams)
        elapsed = 0.010 * (rank + 1)                       # rank 1 is the slowest
        v = job_mpix_s(pixels, 7, elapsed, dist, torch.device("cpu"))
        m = max_over_ranks(elapsed, dist, torch.device("cpu"))
        q.put((rank, [s.tolist() for s in sigs], pixels, v, m, len(cams)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    base = synth.scene_sphere16().cams * 2
    # rank 0 renders the workload's cameras, rank 1 others, as many
    assert out[0][5] == out[1][5] == len(base)
    sig0, sig1 = np.array(out[0][1][0]), np.array(out[0][1][1])
    np.testing.assert_allclose(sig0, np.concatenate([np.asarray(c.R, np.float64).ravel() for c in base]))
    assert np.abs(sig0 - sig1).max() > 1e-3
    # the same job throughput and slowest time on both ranks
    total_pixels = out[0][2] + out[1][2]
    expect = total_pixels * 7 / 0.020 / 1e6
    for r in range(world):
        assert abs(out[r][3] - expect) < 1e-9 * expect
        assert abs(out[r][4] - 0.020) < 1e-15


def _grad_worker(rank, world, port, q):
    from paper_2406_01579_b300 import Params
    sys_path_tests()
    from parity import oracle_run
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = synth.scene_sphere16()
        cam = synth.random_camera(np.random.default_rng(40 + rank), 32, 24)
        up = synth.upstream_grads(50 + rank, [cam])[0]
        o = oracle_run(sc, cam, Params(s=60.0, tile=8), upstream=up)
        g = [tuple(torch.from_numpy(np.ascontiguousarray(o[k], np.float64)) for k in ("dV", "df", "drgb"))]
        allreduce_grads(g, dist)
        q.put((rank, [t.numpy() for t in g[0]]))
    finally:
        dist.destroy_process_group()


def sys_path_tests():
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)


def test_two_gloo_ranks_sum_the_scene_gradient():
    """After the all-reduce both ranks hold the gradient of both ranks' views:
    the sum of the oracle's per-view gradients."""
    from paper_2406_01579_b300 import Params
    sys_path_tests()
    from parity import oracle_run
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = synth.scene_sphere16()
    expect = [0.0, 0.0, 0.0]
    for r in range(world):
        cam = synth.random_camera(np.random.default_rng(40 + r), 32, 24)
        up = synth.upstream_grads(50 + r, [cam])[0]
        o = oracle_run(sc, cam, Params(s=60.0, tile=8), upstream=up)
        for i, k in enumerate(("dV", "df", "drgb")):
            expect[i] = expect[i] + o[k]
    assert np.abs(expect[0]).max() > 0
    for r in range(world):
        for got, exp in zip(out[r], expect):
            np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-12)
