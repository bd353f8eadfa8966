"""eulbfs_diagnostics_noalloc: diagnostics without any device allocation.

Callers whose device memory belongs to another framework's allocator, or
that cannot afford cudaMalloc/cudaFree inside a step, use this entry point;
its block partials live in a fixed device array inside the library.  The
test calls it through the C ABI on a device copy of a solver's state and
checks it against eulbfs_diagnostics on two calls in a row (the shared
scratch array is reused by the second call).  This file is collected last.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2507_03366_gb300 import eulbfs
from paper_2507_03366_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KEYS = ("mass", "enthalpy", "phase_vol", "solid_vol", "max_speed")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2507_03366_gb300 import build
    build.build()


def _device_state(solver, case, precision):
    """The domain's state planes (working precision) copied to a device tensor."""
    import torch
    blob, _ = solver.save()
    n = case.nx * case.ny
    if precision == eulbfs.FP64:
        planes = np.frombuffer(blob, dtype=np.float64)[: 5 * n]
    else:
        planes = np.frombuffer(blob, dtype=np.float32)[: 7 * n]
    return torch.from_numpy(planes.copy()).cuda()


def _call(precision, state, nx, ny, props, out, stream):
    P = eulbfs._props(props)
    return eulbfs.lib().eulbfs_diagnostics_noalloc(precision, ct.c_void_p(state.data_ptr()), nx, ny, ct.byref(P),
                                                   ct.c_void_p(out.data_ptr()), ct.c_void_p(stream))


@pytest.mark.parametrize("precision", [eulbfs.FP64, eulbfs.FP32C])
def test_noalloc_diagnostics_match_existing_entry_point(precision):
    import torch
    case = wl.droplet(96, theta_deg=100.0, St=0.3)
    s = eulbfs.Solver([case], precision=precision)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        s.step(7)
        ref = s.diag()
        state = _device_state(s, case, precision)
        out.fill_(-1.0)
        eulbfs._check(_call(precision, state, case.nx, case.ny, case.props, out, stream))
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, key in enumerate(KEYS):
            assert abs(got[k] - ref[key]) <= 1e-12 * max(abs(ref[key]), 1.0), (key, got[k], ref[key])
        assert got[5] == 0.0


def test_noalloc_rejects_domains_beyond_its_limit():
    import torch
    lib = eulbfs.lib()
    state = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    big = 2048   # 2048 x 2048 cells > EULBFS_NOALLOC_MAX_CELLS
    rc = _call(eulbfs.FP64, state, big, big, wl.droplet(32).props, out, 0)
    assert rc == eulbfs.EINVAL
    assert b"2097152" in lib.eulbfs_last_error()
