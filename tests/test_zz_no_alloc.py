"""The allocation-free kernel-table entry point (sympix_kernel_table_static).

Some callers cannot allocate device memory when they evaluate the kernel
tables: they reserve a fixed device-memory budget up front, or run under an
allocator that must not trigger the device-wide synchronisation cudaMalloc
implies.  For them the library offers a variant that stages its
coefficients in a static device array instead of a buffer it allocates.
Here it is called through the C ABI, twice in a row with different beams,
and each result is checked against the regular entry point's tables.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1504_04653_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1504_04653_gb300 import sympix
    return sympix


def _tables(S, plan, grid, R=10):
    """Every stored kernel value of operator 0, keyed by (ring, rho)."""
    out = {}
    N = grid.nrings
    for j in range(N):
        mm = plan.support(0, j, R)
        for d in range(-R, R + 1):
            if mm[d + R] < 0:
                continue
            K = mm[d + R] // 2 + 1
            b, dd = plan.table(0, j, j + d, K)
            out[(j, j + d)] = (b, dd)
    return out


def _err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", ["lmax64", "lmax500"])
def test_static_table_matches_regular_entry_point(S, name):
    import torch
    wl = W.WORKLOADS[name]
    dev = torch.device("cuda", 0)
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    lib = S.lib()
    inputs = []
    for fwhm in (wl.fwhm_arcmin[0], 1.3 * wl.fwhm_arcmin[0]):
        bl = torch.tensor(W.gaussian_beam(wl.lmax, fwhm)[None, :], dtype=torch.float64, device=dev)
        dl = torch.tensor((W.prior(wl.lmax) * (1.0 + fwhm / 100.0))[None, :], dtype=torch.float64, device=dev)
        inputs.append((bl, dl))
    # the regular entry point, once per input
    refs = []
    for bl, dl in inputs:
        S.sympix_kernel_table(plan, bl, dl)
        torch.cuda.synchronize()
        refs.append(_tables(S, plan, grid))
    # the allocation-free entry point through the C ABI, two calls in a row
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (bl, dl), ref in zip(inputs, refs):
        rc = lib.sympix_kernel_table_static(plan.handle, ctypes.c_void_p(bl.data_ptr()),
                                            ctypes.c_void_p(dl.data_ptr()), stream)
        assert rc == 0, lib.sympix_last_error()
        torch.cuda.synchronize()
        got = _tables(S, plan, grid)
        assert got.keys() == ref.keys()
        for key in ref:
            assert _err(got[key][0], ref[key][0]) <= 1e-10, key
            if ref[key][1] is not None:
                assert _err(got[key][1], ref[key][1]) <= 1e-10, key


def test_static_table_rejects_oversize(S):
    """2 (lmax+1) (nops+1) above the array's 262144 doubles is refused before
    anything is launched."""
    import torch
    grid = S.Grid(3000)
    plan = S.Plan(grid, np.full(44, W.support_radius(5.0)), 1490, 1492)
    need = 2 * 3001 * (44 + 1)
    assert need > 262144
    dev = torch.device("cuda", 0)
    bl = torch.zeros((44, 3001), dtype=torch.float64, device=dev)
    rc = S.lib().sympix_kernel_table_static(plan.handle, ctypes.c_void_p(bl.data_ptr()),
                                            ctypes.c_void_p(bl.data_ptr()), None)
    assert rc == S.EINVAL
    assert b"static array" in S.lib().sympix_last_error()


def test_static_table_on_a_fresh_plan_allocates_nothing(S):
    """On a plan that has never had a table, the allocation-free call leaves
    the plan's device memory as it was (no staging buffer appears), and its
    tables equal those of the regular entry point, which allocates its
    staging on this first use.  Nine operators: a chunk of eight sharing one
    recurrence, then one, in both entry points."""
    import torch
    dev = torch.device("cuda", 0)
    nops = 9
    fwhm = [180.0 + 15.0 * o for o in range(nops)]
    wl = W.Workload("nine", 64, fwhm, [0.0] * nops, list(range(nops)))
    grid = S.Grid(wl.lmax)
    bl = torch.tensor(wl.beams(), dtype=torch.float64, device=dev)
    dl = torch.tensor(wl.priors(), dtype=torch.float64, device=dev)
    lib = S.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    fresh = S.Plan(grid, wl.radii())
    total0, staging0 = fresh.device_bytes()
    assert staging0 == 0
    rc = lib.sympix_kernel_table_static(fresh.handle, ctypes.c_void_p(bl.data_ptr()),
                                        ctypes.c_void_p(dl.data_ptr()), stream)
    assert rc == 0, lib.sympix_last_error()
    torch.cuda.synchronize()
    assert fresh.device_bytes() == (total0, 0)

    regular = S.Plan(grid, wl.radii())
    S.sympix_kernel_table(regular, bl, dl)
    torch.cuda.synchronize()
    assert regular.device_bytes()[1] == 2 * (wl.lmax + 1) * (nops + 1) * 8
    R = 10
    for o in range(nops):
        for j in range(grid.nrings):
            mm = regular.support(o, j, R)
            assert np.array_equal(mm, fresh.support(o, j, R))
            for d in range(-R, R + 1):
                if mm[d + R] < 0:
                    continue
                K = mm[d + R] // 2 + 1
                got = fresh.table(o, j, j + d, K)
                ref = regular.table(o, j, j + d, K)
                assert np.array_equal(got[0], ref[0]), (o, j, d)
                if ref[1] is not None:
                    assert np.array_equal(got[1], ref[1]), (o, j, d)
