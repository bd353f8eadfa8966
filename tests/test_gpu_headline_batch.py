"""The benchmark's headline configuration against the oracle at its own sizes.

The 64-domain axisymmetric (r, z) static-droplet batch (seed 4, sides drawn
from {128, 192, 256, 384, 512}) runs in its launch configuration: FP32C, all
64 domains in one solver, 64-row work items.  Its first 256^2, 384^2 and
512^2 domains are compared with the FP64 oracle run on each alone for 300
steps, at the stated FP32 tolerances (relative L2 of T, u, C within 1e-3,
front and interface within 0.5 %, total-mass drift within 1e-6 of the
oracle's), and near the axis, where 1/r is largest, on the first four
columns by themselves.  The general streaming steps (0.3, 0.4, 0.3) of the
benchmark's second leg are checked the same way on the batch's first 256^2
domain.  The oracle uses every host core (its results do not depend on the
thread count).
"""
import copy
import os

import numpy as np
import pytest

import oracle
from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

from test_gpu_parity import check_fp32c, rel_l2

pytestmark = pytest.mark.gpu

STEPS = 300
SIDES = (256, 384, 512)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _batch():
    return wl.static_droplet_batch(64, seed=4, axisymmetric=True)


def _check_against_oracle(gpu, slot, case, d0g):
    ref = oracle.OracleSolver(case)
    d0r = ref.diag()
    ref.step(STEPS)
    g, r = gpu.fields(slot), ref.fields()
    check_fp32c(g, r, gpu.diag(slot), ref.diag(), d0g, d0r)
    for k in ("T", "C"):                      # the columns next to the axis
        assert rel_l2(g[k][:, :4], r[k][:, :4]) <= 1e-3, (case.name, k)


@pytest.fixture(scope="module")
def headline_run():
    cases = _batch()
    picks = {s: [c.nx for c in cases].index(s) for s in SIDES}
    gpu = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    gpu.set_tile(64)
    d0 = {s: gpu.diag(k) for s, k in picks.items()}
    gpu.step(STEPS)
    gpu.sync()
    return cases, picks, gpu, d0


@pytest.mark.parametrize("side", SIDES)
def test_headline_batch_domain_matches_oracle(side, headline_run):
    cases, picks, gpu, d0 = headline_run
    k = picks[side]
    assert cases[k].axisymmetric and cases[k].nx == side
    _check_against_oracle(gpu, k, cases[k], d0[side])


def test_general_streaming_steps_in_the_batch_match_oracle():
    cases = []
    for c in _batch():
        g = copy.copy(c)
        g.dt_h, g.dt_f, g.dt_g = 0.3, 0.4, 0.3
        cases.append(g)
    k = [c.nx for c in cases].index(256)
    gpu = eulbfs.Solver(cases, precision=eulbfs.FP32C)
    gpu.set_tile(64)
    d0 = gpu.diag(k)
    gpu.step(STEPS)
    _check_against_oracle(gpu, k, cases[k], d0)
