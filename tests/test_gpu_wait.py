"""The bounded device wait of the FP32 factor reports when it runs out.

The fused FP32 kernel's border warps wait, a bounded number of polls, for
rows the band warp of the same CTA publishes.  With a limit of one poll the
first wait runs out before anything is published: the kernel must stop that
sweep, mark the slice's blocks info = -1, set the plan's status so that
sympix_plan_status returns SYMPIX_ETIMEOUT, and return, leaving the context
usable.  Nothing here hangs or faults the GPU: the wait ends by its count.
"""
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


@pytest.mark.parametrize("kernel", [1, 3])
def test_wait_that_runs_out_reports_timeout(S, kernel):
    """kernel 1: the border warps wait on the band warp of their CTA; 3: the
    border CTA waits on the band CTA of the same cooperative launch (global
    progress words, zeroed before every launch, so a run that gave up leaves
    nothing behind for the next)."""
    import torch
    dev = torch.device("cuda", 0)
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = torch.tensor(wl.ninv(colat), dtype=torch.float64, device=dev)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    sampled = S.sympix_sample_blocks(plan, ninv, precision="fp32")
    keep = sampled.clone()
    plan.status()  # nothing pending
    plan.set_narrow_factor(kernel)

    plan.set_wait_limit(1)
    info = S.sympix_factor_blocks(plan, sampled, precision="fp32").cpu().numpy()
    assert np.all((info == -1) | (info >= 0))
    if kernel == 1:  # the border warps catch up with the band warp of their CTA at once
        with pytest.raises(S.SympixError) as e:
            plan.status()
        assert e.value.code == S.ETIMEOUT
        assert np.any(info == -1)
    else:  # the border CTA trails its band CTA and may never wait: a run-out is reported exactly when it happened
        try:
            plan.status()
            assert not np.any(info == -1)
        except S.SympixError as e:
            assert e.code == S.ETIMEOUT and np.any(info == -1)
    plan.status()  # the status was cleared by the read

    # the context is usable and the default limit factors every block
    plan.set_wait_limit(1 << 22)
    again = keep.clone()
    info2 = S.sympix_factor_blocks(plan, again, precision="fp32").cpu().numpy()
    plan.status()
    assert np.all(info2 == 0)
    other = S.Plan(grid, wl.radii())
    other.set_narrow_factor(kernel)
    S.sympix_kernel_table(other, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    ref = keep.clone()
    info3 = S.sympix_factor_blocks(other, ref, precision="fp32").cpu().numpy()
    assert np.array_equal(info2, info3)
    assert torch.equal(again, ref)
