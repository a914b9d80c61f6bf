"""bench.py's multi-rank harness on CPU: gloo, world size 2 (replicas; max-over-ranks time, summed units)."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import time

    import bench

    d = bench.Dist(use_cuda=False)
    calls = {"n": 0}

    def step():
        calls["n"] += 1
        time.sleep(0.01 * (rank + 1))
        return 100.0 * (rank + 1)

    t = [0.0]
    sec, units = bench.timed_steps(step, 3, 2, d, lambda: None, lambda: t.__setitem__(0, time.perf_counter()),
                                   lambda: time.perf_counter() - t[0])
    out[rank] = (sec, units, d.reduce(sec, "max"), d.reduce(units, "sum"), calls["n"])
    d.close()


def test_two_rank_replica_timing_on_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (s0, u0, m0, t0, c0), (s1, u1, m1, t1, c1) = out[0], out[1]
    assert c0 == c1 == 5  # 2 warm-up + 3 timed steps on every rank
    assert u0 == 300.0 and u1 == 600.0
    assert m0 == m1 == max(s0, s1)  # max over ranks
    assert t0 == t1 == 900.0  # whole-job units
    assert s1 >= 0.03


def test_element_counts_match_the_node_ranges():
    sys.path.insert(0, ROOT)
    import bench
    import synthetic as syn
    from oracle.bc import Grid

    wl = syn.sphere_inclusion_32(n=8, radius=2)
    wl.bc[1] = [["N", "D", "N"], ["D", "D", "N"]]
    nodes, per_axis = bench.element_counts(wl)
    g = Grid(wl.n, wl.bc)
    assert nodes == g.N[0] * g.N[1] * g.N[2]
    for a in range(3):
        ref = sum(g.spectral_shape(q)[a] * (nodes // g.N[a]) for q in range(3))
        assert per_axis[a] == ref
