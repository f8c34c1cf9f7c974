"""Blocks on the paper's DP grid with k x k tiles (Sec. 2.3 tiling, Sec. 2.5
layout, Sec. 4.2 locality approximation): one dense block per band of k
rings, D^ + B^T diag(N^-1) B^ with both operators cut to pixel pairs in the
same or neighbouring tiles.  Every band block against the oracle's band
block element by element, in the three contraction arithmetics; the FP64
factor through L L^T; a band range, a second operator, the step graph, and
the calls that take ring blocks only.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_04653_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# FP32: an entry sums up to 9 k^2 = 576 products (k = 8) in single
# precision, whose rounding is bounded by 576 x 2^-24 = 3.4e-5 of the sum of
# their magnitudes; against the block's largest entry that is the bound used.
TOL = {"fp64": 1e-10, "fp32x2": 1e-10, "fp32": 3.4e-5}


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1504_04653_gb300 import sympix
    return sympix


def _err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _workload(lmax, k, nops=1):
    # a beam a little narrower than a tile (k pixel spacings of ~pi/lmax)
    fwhm = 60.0 * 180.0 / lmax * k / 4.0
    return W.Workload(f"dp{lmax}k{k}", lmax, [fwhm * (1.0 + 0.3 * i) for i in range(nops)],
                      [20.0] * nops, [31 + i for i in range(nops)])


def _run(S, lmax, k, precision="fp64", nops=1, ring0=0, ring1=None, factor=False, flat_prior=False):
    import torch
    grid = S.Grid(lmax, k=k, layout="dp", polar_thr=0.0)
    wl = _workload(lmax, k, nops)
    plan = S.Plan(grid, wl.radii(), ring0, ring1)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = wl.ninv(colat)
    dl = np.ones_like(wl.priors()) if flat_prior else wl.priors()
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device="cuda"), torch.tensor(dl, device="cuda"))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(ninv, device="cuda"), precision=precision)
    out = dict(grid=grid, plan=plan, wl=wl, ninv=ninv, dl=dl, sampled=blocks.cpu().numpy())
    if factor:
        out["info"] = S.sympix_factor_blocks(plan, blocks, precision="fp64").cpu().numpy()
        out["factored"] = blocks.cpu().numpy()
    return out


def _oracle_grid(lmax, k):
    return O.grid(lmax, k=k, layout="dp", thr=0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32x2"])
@pytest.mark.parametrize("lmax,k", [(31, 2), (63, 4), (47, 8)])
def test_band_blocks_match_oracle(S, lmax, k, precision):
    """Every band block of the grid (polar bands, where every tile pair
    couples; the equatorial pair of bands; tile counts that change between
    bands) against the oracle's band block."""
    r = _run(S, lmax, k, precision)
    og = _oracle_grid(lmax, k)
    plan, wl = r["plan"], r["wl"]
    nb = og["nrings"] // k
    assert plan.nblocks == nb
    tcounts = set()
    for g in range(nb):
        _, n, _, fmt = plan.block_layout("pband", 0, g)
        assert fmt == S.BLOCK_DENSE and n == k * og["nring"][g * k]
        tcounts.add(int(og["nring"][g * k]) // k)
        M = S.unpack_block(r["sampled"], plan, "pband", 0, g)
        ref, _ = O.band_block(og, wl.beams()[0], wl.priors()[0], r["ninv"][0], g)
        assert _err(M, ref) <= TOL[precision], (g, _err(M, ref))
    assert len(tcounts) >= 2


def test_band_blocks_lmax127_k8(S):
    """l_max = 127, k = 8 (bands of up to 2304 pixels): sampled bands from
    the pole to the equator against the oracle."""
    lmax, k = 127, 8
    og = _oracle_grid(lmax, k)
    nb = og["nrings"] // k
    r = _run(S, lmax, k, "fp64")
    plan, wl = r["plan"], r["wl"]
    for g in (0, 1, 4, nb // 2 - 1, nb // 2, nb - 1):
        M = S.unpack_block(r["sampled"], plan, "pband", 0, g)
        ref, _ = O.band_block(og, wl.beams()[0], r["dl"][0], r["ninv"][0], g)
        assert _err(M, ref) <= TOL["fp64"], g


def test_band_blocks_lmax500_k8(S):
    """l_max = 500, k = 8 (64 bands, the equatorial ones of 8640 pixels):
    the polar band, a mid-latitude band and the band next to the equator
    against the oracle; only those blocks leave the device."""
    import torch
    lmax, k = 500, 8
    og = _oracle_grid(lmax, k)
    nb = og["nrings"] // k
    grid = S.Grid(lmax, k=k, layout="dp", polar_thr=0.0)
    wl = _workload(lmax, k)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = wl.ninv(colat)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device="cuda"), torch.tensor(wl.priors(), device="cuda"))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(ninv, device="cuda"), precision="fp64")
    for g in (0, 20, nb // 2 - 1):
        off, n, _, fmt = plan.block_layout("pband", 0, g)
        assert fmt == S.BLOCK_DENSE and n == k * og["nring"][g * k]
        M = blocks[off:off + n * n].reshape(n, n).cpu().numpy()
        ref, _ = O.band_block(og, wl.beams()[0], wl.priors()[0], ninv[0], g)
        assert _err(M, ref) <= TOL["fp64"], (g, _err(M, ref))
    assert n == 8640


def test_band_factor_matches_oracle(S):
    """The FP64 factor of every band block at l_max = 31, k = 2.  A band
    whose rings hold more than 2 l_max + 1 pixels carries a band-limited D^
    that is singular before the tile cut and indefinite after it: there the
    verdict is the oracle's first non-positive pivot.  The other bands are
    positive definite: L matches the oracle's Cholesky factor and L L^T its
    block."""
    lmax, k = 31, 2
    og = _oracle_grid(lmax, k)
    r = _run(S, lmax, k, "fp64", factor=True)
    plan, wl = r["plan"], r["wl"]
    good = bad = 0
    for g in range(og["nrings"] // k):
        ref, _ = O.band_block(og, wl.beams()[0], r["dl"][0], r["ninv"][0], g)
        Lref, info = O.cholesky(ref)
        assert r["info"][g] == info, (g, int(r["info"][g]), info)
        if info:
            bad += 1
            continue
        good += 1
        L = S.unpack_block(r["factored"], plan, "pband", 0, g, factored=True)
        assert _err(L @ L.T, ref) <= 10 * TOL["fp64"], g
        assert _err(L, Lref) <= 1e-8, (g, _err(L, Lref))
    assert good >= 8 and bad >= 2, (good, bad)


def test_band_range_and_two_operators(S):
    """A band-aligned ring range and two operators of different beams: the
    blocks are the oracle's for each operator's beam and N^-1."""
    lmax, k = 63, 4
    og = _oracle_grid(lmax, k)
    r = _run(S, lmax, k, "fp64", nops=2, ring0=2 * k, ring1=og["nrings"] - 3 * k)
    plan, wl = r["plan"], r["wl"]
    assert plan.nblocks == 2 * (og["nrings"] // k - 5)
    for o in range(2):
        for g in (2, 5, og["nrings"] // k - 4):
            M = S.unpack_block(r["sampled"], plan, "pband", o, g)
            ref, _ = O.band_block(og, wl.beams()[o], wl.priors()[o], r["ninv"][o], g)
            assert _err(M, ref) <= TOL["fp64"], (o, g)


def test_step_graph_matches_direct_calls(S):
    """The captured step (table, sampling, factor) on a DP plan equals the
    direct calls bit for bit."""
    import torch
    lmax, k = 63, 4
    grid = S.Grid(lmax, k=k, layout="dp", polar_thr=0.0)
    wl = _workload(lmax, k)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    bl = torch.tensor(wl.beams(), device="cuda")
    dl = torch.tensor(wl.priors(), device="cuda")
    ninv = torch.tensor(wl.ninv(colat), device="cuda")
    S.sympix_kernel_table(plan, bl, dl)
    ref = S.sympix_sample_blocks(plan, ninv, precision="fp64")
    iref = S.sympix_factor_blocks(plan, ref, precision="fp64")
    nbytes, _ = plan.blocks_size("pband")
    blocks = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    info = torch.full((plan.nblocks,), -7, dtype=torch.int32, device="cuda")
    step = S.Step(plan, bl, dl, ninv, blocks, info, "pband", "fp64", "fp64")
    assert step.kernels() == sum(plan.launches("pband", "fp64", "fp64"))
    step.launch(S.STAGE_ALL)
    torch.cuda.synchronize()
    assert np.array_equal(blocks.cpu().numpy(), ref.cpu().numpy())
    assert np.array_equal(info.cpu().numpy(), iref.cpu().numpy())


def test_ring_block_calls_refuse_dp_plans(S):
    """Convolution and the blocks between rings are planned for ring blocks
    (k = 1); on a DP plan they return SYMPIX_EUNSUPPORTED, and a ring range
    that cuts a band is refused."""
    import torch
    grid = S.Grid(31, k=2, layout="dp", polar_thr=0.0)
    wl = _workload(31, 2)
    with pytest.raises(S.SympixError):
        S.Plan(grid, wl.radii(), 1, grid.nrings)
    plan = S.Plan(grid, wl.radii())
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device="cuda"), torch.tensor(wl.priors(), device="cuda"))
    f = torch.zeros((1, grid.npix), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SympixError):
        S.sympix_convolve(plan, f)
