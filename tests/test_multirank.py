"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Every rank advances its own independent batch (weak scaling, no collective
on the data path); the only collectives are the barrier and the reductions
of the timing (max) and of the cell count (sum)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    seed = bench.rank_seed(4, r)
    cases = bench.workload(3, seed)
    cells = sum(c.cells for c in cases)
    mx = bench.reduce_max(float(10 * (r + 1)), w)
    sm = bench.reduce_sum(float(cells), w)
    bench.barrier(w)
    sig = [(c.nx, round(c.props.L, 12), c.bc.ylo.theta_deg) for c in cases]
    q.put((r, w, seed, sig, cells, mx, sm))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, sig0, c0, mx0, sm0), (r1, w1, s1, sig1, c1, mx1, sm1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert s0 != s1 and sig0 != sig1          # independent problems per rank
    assert mx0 == mx1 == 20.0                 # slowest rank's time
    assert sm0 == sm1 == float(c0 + c1)       # whole-job cell count


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        domains, seed, warmup, steps, gpus, tile, graph, geometry = 2, 4, 0, 1, 2, 64, 0, "rz"

    assert bench.run_reference(Args) == 0
    assert capsys.readouterr().out == ""
