"""The halo exchange of a split domain across ranks, on CPU (gloo, world size 2).

Each rank holds some of the k slabs of a synthetic 7-plane domain, with its
halo rows poisoned by NaN.  After slabs.exchange every halo row must equal
the domain's row it stands for -- the row below or above the slab, wrapped
on a periodic axis -- bit for bit, whichever rank owns the neighbour.  The
single-process path (all slabs on one rank, plain copies) is checked the
same way, and the schedule's row split is the library's.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_03366_gb300 import slabs  # noqa: E402

NP, NY, NX = 7, 40, 6


def _domain():
    return np.random.default_rng(3).standard_normal((NP, NY, NX))


def _slab_arrays(D, k, periodic, mine):
    sides = slabs.halo_sides(k, periodic)
    out = {}
    for i, (y0, y1) in enumerate(slabs.split_rows(NY, k)):
        if i not in mine:
            continue
        lo, hi = sides[i]
        a = np.full((NP, lo + (y1 - y0) + hi, NX), np.nan)
        a[:, lo: lo + (y1 - y0)] = D[:, y0:y1]
        out[i] = a
    return out


def _check(D, arrays, k, periodic):
    sides = slabs.halo_sides(k, periodic)
    rows = slabs.split_rows(NY, k)
    for i, a in arrays.items():
        lo, hi = sides[i]
        y0, y1 = rows[i]
        if lo:
            want = D[:, [(y0 - HALO_K) % NY for HALO_K in range(slabs.HALO, 0, -1)]]
            assert np.array_equal(a[:, :lo], want), (i, "below")
        if hi:
            want = D[:, [(y1 + j) % NY for j in range(slabs.HALO)]]
            assert np.array_equal(a[:, lo + (y1 - y0):], want), (i, "above")
        assert not np.isnan(a).any()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, k, periodic, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2507_03366_gb300 import slabs as sl
    D = _domain()
    mine = [i for i, r in enumerate(sl.owners(k, world)) if r == rank]
    arrays = _slab_arrays(D, k, periodic, mine)
    sent = sl.exchange(arrays, k, periodic, rank, world)
    try:
        _check(D, arrays, k, periodic)
        q.put((rank, sent, "ok"))
    except AssertionError as e:
        q.put((rank, sent, f"failed: {e}"))
    dist.destroy_process_group()


@pytest.mark.parametrize("k,periodic", [(2, False), (4, False), (4, True), (5, True)])
def test_exchange_on_two_cpu_ranks(k, periodic):
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, k, periodic, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[2] for r in res] == ["ok", "ok"], res
    # slabs split over both ranks: every rank sends its boundary slab's rows
    assert all(r[1] >= 1 for r in res)


@pytest.mark.parametrize("k,periodic", [(1, False), (3, False), (3, True)])
def test_exchange_in_one_process(k, periodic):
    D = _domain()
    arrays = _slab_arrays(D, k, periodic, range(k))
    assert slabs.exchange(arrays, k, periodic) == 0
    _check(D, arrays, k, periodic)
    assert np.array_equal(slabs.assemble([arrays[i] for i in range(k)], k, periodic), D)


def test_schedule_matches_the_library_rule():
    # eulbfs_add_split_domain: slab i holds rows [i ny / k, (i + 1) ny / k), halos of 3 rows
    assert slabs.split_rows(128, 3) == [(0, 42), (42, 85), (85, 128)]
    assert slabs.halo_sides(3, False) == [(0, 3), (3, 3), (3, 0)]
    assert slabs.halo_sides(2, True) == [(3, 3), (3, 3)]
    assert slabs.halo_links(3, True) == [(0, 1), (1, 2), (2, 0)]
    assert slabs.owners(4, 2) == [0, 0, 1, 1]
