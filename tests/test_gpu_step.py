"""Captured step (sympix_step_create / sympix_step_launch) against direct calls.

The graphs replay the same kernels on the same inputs, so the blocks, the
factors and the info codes must agree bit for bit with the direct calls.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1504_04653_gb300 import sympix as S  # noqa: E402
from paper_1504_04653_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(name, seeds=None):
    wl = W.WORKLOADS[name]
    if seeds is not None:
        wl = W.Workload(wl.name, wl.lmax, wl.fwhm_arcmin, wl.band_deg, seeds, wl.desc)
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    dev = torch.device("cuda", 0)
    bl = torch.tensor(wl.beams(), dtype=torch.float64, device=dev)
    dl = torch.tensor(wl.priors(), dtype=torch.float64, device=dev)
    ninv = torch.tensor(wl.ninv(colat), dtype=torch.float64, device=dev)
    return wl, grid, plan, colat, bl, dl, ninv


def _direct(plan, bl, dl, ninv, storage, sprec, fprec):
    # sampling leaves the border rows of a periodic-band block unwritten (the
    # factor fills them): start from zeros on both sides
    nbytes, _ = plan.blocks_size(storage)
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    S.sympix_kernel_table(plan, bl, dl)
    S.sympix_sample_blocks(plan, ninv, precision=sprec, storage=storage, out=blocks)
    sampled = blocks.clone()
    info = S.sympix_factor_blocks(plan, blocks, storage=storage, precision=fprec)
    torch.cuda.synchronize()
    return sampled.cpu().numpy(), blocks.cpu().numpy(), info.cpu().numpy()


@pytest.mark.parametrize("storage,fprec", [("pband", "fp32"), ("pband", "fp64"), ("dense", "fp64")])
def test_step_wide_bands_match_direct_calls(storage, fprec):
    """Band widths 17..64 (the wide factor, one launch per CTA size and, for
    FP32, an FP64 rescue launch per size): the captured step has as many
    kernels as the plan says and replays the direct calls bit for bit."""
    wl = W.Workload("wide120", 120, [262.0, 450.0, 640.0, 830.0, 1014.0], [0.0, 5.0, 10.0, 15.0, 20.0],
                    [71, 72, 73, 74, 75])
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    dev = torch.device("cuda", 0)
    bl = torch.tensor(wl.beams(), dtype=torch.float64, device=dev)
    dl = torch.tensor(wl.priors(), dtype=torch.float64, device=dev)
    ninv = torch.tensor(wl.ninv(colat), dtype=torch.float64, device=dev)
    widths = {plan.block_layout("pband", o, j)[2] for o in range(wl.nops) for j in range(grid.nrings)
              if plan.block_layout("pband", o, j)[3] == S.BLOCK_PBAND}
    assert any(16 < w <= 32 for w in widths) and any(48 < w <= 64 for w in widths), sorted(widths)
    s_ref, f_ref, i_ref = _direct(plan, bl, dl, ninv, storage, "fp64", fprec)
    nbytes, _ = plan.blocks_size(storage)
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.full((plan.nblocks,), -7, dtype=torch.int32, device="cuda")
    step = S.Step(plan, bl, dl, ninv, blocks, info, storage, "fp64", fprec)
    assert step.kernels() == sum(plan.launches(storage, "fp64", fprec))
    step.launch(S.STAGE_ALL)
    torch.cuda.synchronize()
    assert np.array_equal(blocks.cpu().numpy(), f_ref)
    assert np.array_equal(info.cpu().numpy(), i_ref)


@pytest.mark.parametrize("name,storage,sprec,fprec,narrow", [
    ("lmax500", "pband", "fp32", "fp32", -1),
    ("lmax500", "pband", "fp32", "fp32", 2),
    ("lmax500", "pband", "fp32", "fp32", 3),
    ("lmax500", "pband", "fp64", "fp64", -1),
    ("lmax500", "pband", "fp64", "fp64", 2),
    ("lmax64", "pband", "fp64", "fp64", 2),
    ("lmax500", "pband", "fp32x2", "fp32x2", 2),
    ("lmax64", "dense", "fp32x2", "fp32x2", -1),
])
def test_step_matches_direct_calls(name, storage, sprec, fprec, narrow):
    wl, grid, plan, colat, bl, dl, ninv = _setup(name)
    plan.set_narrow_factor(narrow)
    s_ref, f_ref, i_ref = _direct(plan, bl, dl, ninv, storage, sprec, fprec)
    nbytes, _ = plan.blocks_size(storage)
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.full((plan.nblocks,), -7, dtype=torch.int32, device="cuda")
    step = S.Step(plan, bl, dl, ninv, blocks, info, storage, sprec, fprec)
    assert step.kernels() == sum(plan.launches(storage, sprec, fprec))
    assert step.kernels(S.STAGE_TABLE) == plan.launches(storage, sprec, fprec)[0]
    step.launch(S.STAGE_TABLE | S.STAGE_SAMPLE)
    torch.cuda.synchronize()
    assert np.array_equal(blocks.cpu().numpy(), s_ref)
    step.launch(S.STAGE_FACTOR)
    torch.cuda.synchronize()
    assert np.array_equal(blocks.cpu().numpy(), f_ref)
    assert np.array_equal(info.cpu().numpy(), i_ref)
    # a second replay of the whole step on another stream gives the same
    st = torch.cuda.Stream()
    blocks.zero_()
    step.launch(S.STAGE_ALL, stream=st)
    torch.cuda.synchronize()
    assert np.array_equal(blocks.cpu().numpy(), f_ref)


def test_step_reads_inputs_at_replay():
    """Updating N^-1 in place and replaying sampling + factor gives what
    direct calls on the new N^-1 give."""
    wl, grid, plan, colat, bl, dl, ninv = _setup("lmax500")
    nbytes, _ = plan.blocks_size("pband")
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.empty(plan.nblocks, dtype=torch.int32, device="cuda")
    step = S.Step(plan, bl, dl, ninv, blocks, info, "pband", "fp32", "fp32")
    step.launch()
    wl2 = W.Workload(wl.name, wl.lmax, wl.fwhm_arcmin, wl.band_deg, [s + 17 for s in wl.seeds], wl.desc)
    ninv.copy_(torch.tensor(wl2.ninv(colat), dtype=torch.float64, device="cuda"))
    blocks.zero_()
    step.launch(S.STAGE_SAMPLE | S.STAGE_FACTOR)
    torch.cuda.synchronize()
    got_b, got_i = blocks.cpu().numpy(), info.cpu().numpy()
    _, f_ref, i_ref = _direct(plan, bl, dl, ninv, "pband", "fp32", "fp32")
    assert np.array_equal(got_b, f_ref)
    assert np.array_equal(got_i, i_ref)


def test_step_rejects_bad_arguments():
    wl, grid, plan, colat, bl, dl, ninv = _setup("lmax64")
    nbytes, _ = plan.blocks_size("pband")
    blocks = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.empty(plan.nblocks, dtype=torch.int32, device="cuda")
    step = S.Step(plan, bl, dl, ninv, blocks, info)
    for bad in (0, 8, -1):
        with pytest.raises(S.SympixError):
            step.launch(bad)
    with pytest.raises(S.SympixError):
        S.Step(plan, bl, dl, ninv, blocks[:10], info)


def test_trace_names_every_kernel():
    """SYMPIX_OPT_TRACE: one span per kernel launch group, positive times,
    nothing recorded once tracing is off."""
    wl, grid, plan, colat, bl, dl, ninv = _setup("lmax500")
    plan.set_trace(True)
    plan.set_narrow_factor(0)  # the G-lane kernel for every arithmetic
    S.sympix_kernel_table(plan, bl, dl)
    blocks = S.sympix_sample_blocks(plan, ninv, precision="fp32", storage="pband")
    S.sympix_factor_blocks(plan, blocks, storage="pband", precision="fp32")
    spans = plan.trace_read()
    names = [n for n, _ in spans]
    for k in ("k_table", "k_split_ninv", "k_sample_pband", "k_pband_chol", "k_chol_commit", "k_pband_chol_rescue"):
        assert k in names, names
    assert all(ms >= 0.0 for _, ms in spans)
    # the earlier FP32 kernels: shadow transposes and the fused band / border kernel
    plan.set_narrow_factor(1)
    S.sympix_factor_blocks(plan, S.sympix_sample_blocks(plan, ninv, precision="fp32"), precision="fp32")
    names = [n for n, _ in plan.trace_read()]
    for k in ("k_f32_shadow_in", "k_f32_fused", "k_f32_out", "k_factor_rescue"):
        assert k in names, names
    # the band pass and the border rows by column chunks
    plan.set_narrow_factor(2)
    S.sympix_factor_blocks(plan, S.sympix_sample_blocks(plan, ninv, precision="fp32"), precision="fp32")
    names = [n for n, _ in plan.trace_read()]
    for k in ("k_f32_band_pass", "k_l21_transfer", "k_l21_carry", "k_l21_solve", "k_l21_corner", "k_f32_out"):
        assert k in names, names
    # band and border passes in two CTAs of one launch
    plan.set_narrow_factor(3)
    S.sympix_factor_blocks(plan, S.sympix_sample_blocks(plan, ninv, precision="fp32"), precision="fp32")
    names = [n for n, _ in plan.trace_read()]
    for k in ("k_f32_shadow_in", "k_f32_split", "k_f32_out"):
        assert k in names, names
    # FP64: the one-lane band pass on the FP64 shadow, then the chunked border rows
    S.sympix_factor_blocks(plan, S.sympix_sample_blocks(plan, ninv, precision="fp64"), precision="fp64")
    names = [n for n, _ in plan.trace_read()]
    for k in ("k_f32_shadow_in", "k_f64_band_pass", "k_l21_transfer", "k_l21_corner", "k_f32_out"):
        assert k in names, names
    # split FP32: the same on a split-FP32 shadow
    S.sympix_factor_blocks(plan, S.sympix_sample_blocks(plan, ninv, precision="fp64"), precision="fp32x2")
    names = [n for n, _ in plan.trace_read()]
    for k in ("k_f32_shadow_in", "k_df_band_pass", "k_l21_transfer", "k_l21_corner", "k_f32_out"):
        assert k in names, names
    plan.set_narrow_factor(-1)
    assert plan.trace_read() == []
    plan.set_trace(False)
    S.sympix_kernel_table(plan, bl, dl)
    assert plan.trace_read() == []


def test_launch_shapes_agree_and_autotune():
    """Every launch shape gives the same blocks and factors, bit for bit; the
    autotuner keeps one of the candidates."""
    wl, grid, plan, colat, bl, dl, ninv = _setup("lmax500")
    nbytes, _ = plan.blocks_size("pband")
    ref = None
    for cta, nt in ((32, 512), (64, 256), (128, 512)):
        plan.set_launch_shape(table_cta=cta, border_threads=nt)
        assert plan.tuning() == (cta, nt)
        got = _direct(plan, bl, dl, ninv, "pband", "fp32", "fp32")
        if ref is None:
            ref = got
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b)
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.empty(plan.nblocks, dtype=torch.int32, device="cuda")
    cta, nt = plan.autotune(bl, dl, ninv, blocks, info)
    assert cta in (32, 64, 128) and nt in (256, 512)
    with pytest.raises(S.SympixError):
        plan.set_launch_shape(table_cta=48)
    with pytest.raises(S.SympixError):
        plan.set_launch_shape(border_threads=384)
