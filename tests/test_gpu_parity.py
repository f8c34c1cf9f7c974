"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer outputs (ring counts, pixel numbering, coupled pixel sets, band
widths) must match bit for bit; floating-point outputs within the stated
tolerances, normwise per block: max|x - x_ref| / max|x_ref| <= 1e-10 for the
FP64 and split-FP32 contractions, <= 1e-6 for the FP32 contraction.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1504_04653_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32x2": 1e-10, "fp32": 1e-6}


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1504_04653_gb300 import sympix
    return sympix


@pytest.fixture(scope="module")
def dev(S):
    import torch
    return torch.device("cuda", 0)


def _err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run(S, dev, wl, grid=None, ring0=0, ring1=None, precision="fp64", storage="pband", factor=False,
         ninv_h=None, radii=None, factor_precision=None, narrow=None):
    import torch
    grid = grid or S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii() if radii is None else radii, ring0, ring1)
    if narrow is not None:
        plan.set_narrow_factor(narrow)
    bl = torch.tensor(wl.beams(), dtype=torch.float64, device=dev)
    dl = torch.tensor(wl.priors(), dtype=torch.float64, device=dev)
    if ninv_h is None:
        colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
        ninv_h = wl.ninv(colat)
    ninv = torch.tensor(ninv_h, dtype=torch.float64, device=dev)
    S.sympix_kernel_table(plan, bl, dl)
    blocks = S.sympix_sample_blocks(plan, ninv, precision=precision, storage=storage)
    sampled = blocks.cpu().numpy()
    out = dict(grid=grid, plan=plan, sampled=sampled, ninv=ninv_h)
    if factor:
        info = S.sympix_factor_blocks(plan, blocks, storage=storage, precision=factor_precision or precision)
        out["info"] = info.cpu().numpy()
        out["factored"] = blocks.cpu().numpy()
    return out


# -- grid --------------------------------------------------------------------------

@pytest.mark.parametrize("lmax", [1, 2, 7, 64, 65, 500, 1000, 3000])
def test_greedy_grid_matches_oracle(S, lmax):
    g = S.Grid(lmax)
    og = O.grid(lmax)
    assert np.array_equal(g.nring, og["nring"])
    assert np.array_equal(g.ring_offset, og["ring_offset"])
    assert np.array_equal(g.ring_stride, og["ring_stride"])
    assert g.npix == og["npix"]
    assert np.max(np.abs(g.theta - og["theta"]) / og["theta"]) <= 4e-15


@pytest.mark.parametrize("lmax,k,thr", [(767, 8, 0.0), (511, 8, 0.0), (2000, 4, 0.0), (511, 8, -1.0),
                                        (63, 2, 0.0), (100, 1, 5.0)])
def test_dp_grid_matches_oracle(S, lmax, k, thr):
    g = S.Grid(lmax, k=k, layout="dp", polar_thr=thr)
    og = O.grid(lmax, k=k, layout="dp", thr=thr)
    assert np.array_equal(g.nring, og["nring"])
    assert np.array_equal(g.ring_offset, og["ring_offset"])
    assert np.array_equal(g.ring_stride, og["ring_stride"])
    if (lmax, k, thr) == (767, 8, 0.0):
        assert g.npix == 838656  # Table comparison


# -- support and kernel table ---------------------------------------------------------

def _coupled_from_mmax(n_j, n_rho, c, m):
    """Columns p of ring rho coupled to column c of ring j by the rule
    |z| <= m, z = (2c+1) Q - (2p+1) P reduced to the nearest longitude."""
    g = math.gcd(n_j, n_rho)
    P, Q = n_j // g, n_rho // g
    half = P * n_rho
    p = np.arange(n_rho, dtype=np.int64)
    z = ((2 * c + 1) * Q - (2 * p + 1) * P) % (2 * half)
    z = np.where(z > half, z - 2 * half, z)
    return p[np.abs(z) <= m].astype(np.int32)


@pytest.mark.parametrize("name,rings", [("lmax64", None), ("lmax500", [0, 1, 2, 3, 60, 249, 250, 251, 498, 500])])
def test_support_matches_oracle_bruteforce(S, name, rings):
    wl = W.WORKLOADS[name]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    og = O.grid(wl.lmax)
    r_s = wl.radii()[0]
    N = grid.nrings
    R = 12
    for j in (rings if rings is not None else range(N)):
        mm = plan.support(0, j, R)
        for d in range(-R, R + 1):
            rho = j + d
            if rho < 0 or rho >= N:
                continue
            n_j, n_r = int(grid.nring[j]), int(grid.nring[rho])
            for c in sorted({0, 1, n_j // 3, n_j - 1}):
                ref = O.coupled(og, j, c, rho, r_s)
                got = _coupled_from_mmax(n_j, n_r, c, mm[d + R]) if mm[d + R] >= 0 else np.zeros(0, np.int32)
                assert np.array_equal(got, ref), (j, rho, c)


def test_support_every_ring_lmax3000(S):
    """l_max = 3000, FWHM 5': the coupled pixel sets of every ring and every
    neighbour ring, at three columns each, bit for bit against the oracle's
    direct test of every pixel pair."""
    wl = W.WORKLOADS["lmax3000"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    og = O.grid(wl.lmax)
    r_s = plan.radius(0)[0]
    N, R = grid.nrings, 6  # r_s is about 4 ring spacings
    checked = 0
    for j in range(N):
        mm = plan.support(0, j, R)
        n_j = int(grid.nring[j])
        for d in range(-R, R + 1):
            rho = j + d
            if rho < 0 or rho >= N:
                continue
            n_r = int(grid.nring[rho])
            for c in sorted({0, n_j // 3, n_j - 1}):
                ref = O.coupled(og, j, c, rho, r_s)
                got = _coupled_from_mmax(n_j, n_r, c, mm[d + R]) if mm[d + R] >= 0 else np.zeros(0, np.int32)
                assert np.array_equal(got, ref), (j, rho, c)
                checked += len(ref)
    assert checked > 10 * N


def _golden_margins():
    from pathlib import Path
    rows = []
    path = Path(__file__).resolve().parent / "golden" / "support_margins.txt"
    for line in path.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, op, lmax, r_s, r_used, margin = line.split()
            rows.append((name, int(op), int(lmax), float.fromhex(r_s), float.fromhex(r_used), float(margin)))
    return rows


@pytest.mark.parametrize("name", ["lmax64", "lmax500", "lmax1500", "lmax3000", "batched32"])
def test_support_radius_and_margin_match_oracle(S, name):
    """The plan's threshold guard takes the oracle's decision at every
    measured workload: the same radius (bit for bit) and the same smallest
    distance of any class from the threshold."""
    wl = W.WORKLOADS[name]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    rows = [r for r in _golden_margins() if r[0] == name]
    assert len(rows) == wl.nops
    for _, op, _, r_s, r_used, margin in rows:
        assert wl.radii()[op] == r_s
        r, m = plan.radius(op)
        assert r == r_used, (name, op)
        assert abs(m - margin) <= 1e-6 * margin, (name, op, m, margin)


def test_support_guard_moves_a_radius_off_a_class(S):
    """A radius placed exactly on one pixel pair's separation: the plan
    scales it as the oracle does, and the coupled sets follow the scaled
    radius on both sides."""
    grid = S.Grid(32)
    og = O.grid(32)
    j, rho = 10, 12
    u = O.pair_u(og["theta"][j], og["nring"][j], 0, og["theta"][rho], og["nring"][rho], 1)
    r_on = 2.0 * math.asin(math.sqrt(u / 2.0))
    r_ref, m_ref = O.guarded_radius(og, r_on)
    assert r_ref != r_on
    plan = S.Plan(grid, np.array([r_on]))
    r, m = plan.radius(0)
    assert r == r_ref and m > 1e-12
    R = 6
    for jj in (j, rho):
        mm = plan.support(0, jj, R)
        for d in range(-R, R + 1):
            rr = jj + d
            if mm[d + R] < 0:
                continue
            for c in range(int(grid.nring[jj])):
                ref = O.coupled(og, jj, c, rr, r_ref)
                got = _coupled_from_mmax(int(grid.nring[jj]), int(grid.nring[rr]), c, mm[d + R])
                assert np.array_equal(got, ref), (jj, rr, c)


@pytest.mark.parametrize("name", ["lmax64", "lmax500", "lmax3000"])
def test_kernel_table_matches_oracle(S, dev, name):
    import torch
    wl = W.WORKLOADS[name]
    grid = S.Grid(wl.lmax)
    N = grid.nrings
    rings = [0, 1, N // 4, N // 2, N - 1]
    plan = S.Plan(grid, wl.radii())
    og = O.grid(wl.lmax)
    bl, dl = wl.beams()[0], wl.priors()[0]
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    torch.cuda.synchronize()
    peak_b = O.kernel_u(wl.lmax, bl, 0.0)[0]
    peak_d = O.kernel_u(wl.lmax, dl, 0.0)[0]
    R = 8
    for j in rings:
        mm = plan.support(0, j, R)
        for d in range(-R, R + 1):
            m = mm[d + R]
            if m < 0:
                continue
            rho = j + d
            n_j, n_r = int(grid.nring[j]), int(grid.nring[rho])
            g = math.gcd(n_j, n_r)
            P, Q = n_j // g, n_r // g
            K = m // 2 + 1
            b, dd = plan.table(0, j, rho, K)
            # one representative pixel pair per class: c = 0, p with |z| = level
            for k in range(0, K, max(1, K // 4)):
                lev = (m % 2) + 2 * k
                found = None
                for c in range(P):
                    for p in range(-n_r, 2 * n_r):
                        if abs((2 * c + 1) * Q - (2 * p + 1) * P) == lev:
                            found = (c, p % n_r)
                            break
                    if found:
                        break
                assert found is not None
                u = O.pair_u(og["theta"][j], n_j, found[0], og["theta"][rho], n_r, found[1])
                ref = O.kernel_u(wl.lmax, bl, u)[0]
                assert abs(b[k] - ref) <= 1e-10 * peak_b, (j, rho, k)
                if rho == j:
                    refd = O.kernel_u(wl.lmax, dl, u)[0]
                    assert abs(dd[k] - refd) <= 1e-10 * peak_d


# -- blocks ----------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32x2"])
@pytest.mark.parametrize("storage", ["pband", "dense"])
def test_blocks_lmax64_all(S, dev, precision, storage):
    wl = W.WORKLOADS["lmax64"]
    r = _run(S, dev, wl, precision=precision, storage=storage, factor=True)
    og = O.grid(wl.lmax)
    plan = r["plan"]
    assert np.all(r["info"] == 0)
    for j in range(og["nrings"]):
        M = S.unpack_block(r["sampled"], plan, storage, 0, j)
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], r["ninv"][0], j)
        assert _err(M, ref) <= TOL[precision], (j, _err(M, ref))
        L = S.unpack_block(r["factored"], plan, storage, 0, j, factored=True)
        Lref, info = O.cholesky(ref)
        assert info == 0
        assert _err(L, Lref) <= 50 * TOL[precision], (j, _err(L, Lref))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32x2"])
def test_blocks_lmax500_sampled(S, dev, precision):
    wl = W.WORKLOADS["lmax500"]
    r = _run(S, dev, wl, precision=precision, factor=True)
    og = O.grid(wl.lmax)
    plan = r["plan"]
    assert np.all(r["info"] == 0)
    for j in (0, 1, 2, 77, 249, 250, 251, 423, 500):
        M = S.unpack_block(r["sampled"], plan, "pband", 0, j)
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], r["ninv"][0], j)
        assert _err(M, ref) <= TOL[precision], (j, _err(M, ref))
        L = S.unpack_block(r["factored"], plan, "pband", 0, j, factored=True)
        # the factor reproduces the oracle's block
        assert _err(L @ L.T, ref) <= 10 * TOL[precision], j
        if M.shape[0] <= 300:
            Lref, _ = O.cholesky(ref)
            assert _err(L, Lref) <= 100 * TOL[precision], j


def test_block_widths_match_oracle_structure(S, dev):
    """The stored band covers exactly the oracle's structural nonzeros."""
    wl = W.WORKLOADS["lmax64"]
    r = _run(S, dev, wl)
    og = O.grid(wl.lmax)
    rng = np.random.default_rng(9)
    ninv = rng.uniform(0.5, 2.0, og["npix"])  # no masked zeros: structure = support
    for j in (10, 20, 32, 50):
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv, j)
        _, n, w, fmt = r["plan"].block_layout("pband", 0, j)
        if fmt != 0:
            continue
        q = np.arange(n)
        dist = np.minimum((q[:, None] - q[None, :]) % n, (q[None, :] - q[:, None]) % n)
        assert np.all(ref[dist > w] == 0.0)
        assert np.any(ref[dist == w] != 0.0)


def test_ring_range_and_batched_operators(S, dev):
    """A ring sub-range, and several operators in one plan, reproduce the
    single-operator full plan block by block."""
    import torch
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(wl.lmax)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    multi = W.Workload("multi", 64, [180.0, 120.0, 240.0], [20.0, 0.0, 30.0], [1, 7, 8])
    full = _run(S, dev, multi, grid=grid, precision="fp64", factor=True)
    sub = _run(S, dev, multi, grid=grid, ring0=20, ring1=33, precision="fp64", factor=True)
    og = O.grid(64)
    ninv_h = multi.ninv(colat)
    for o in range(3):
        for j in (20, 26, 32):
            A = S.unpack_block(full["sampled"], full["plan"], "pband", o, j)
            B = S.unpack_block(sub["sampled"], sub["plan"], "pband", o, j)
            assert np.array_equal(A, B)
            ref, _ = O.block(og, multi.beams()[o], multi.priors()[o], multi.radii()[o], ninv_h[o], j)
            assert _err(A, ref) <= 1e-10
            # a truncated prior over a masked ring need not be definite: the
            # pivot report must agree with the oracle's Cholesky
            _, info = O.cholesky(ref)
            assert full["info"][o * 65 + j] == info
            assert sub["info"][o * 13 + (j - 20)] == info


def test_no_truncation_and_tiny_grids(S, dev):
    """r_s >= pi couples every pixel pair (dense blocks), l_max = 1 and 6."""
    for lmax in (1, 6):
        wl = W.Workload("tiny", lmax, [600.0], [0.0], [3])
        r = _run(S, dev, wl, radii=np.array([math.pi]), precision="fp64", factor=True)
        og = O.grid(lmax)
        for j in range(og["nrings"]):
            M = S.unpack_block(r["sampled"], r["plan"], "pband", 0, j)
            ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], math.pi, r["ninv"][0], j)
            assert _err(M, ref) <= 1e-10


def test_masked_everywhere_gives_prior_only(S, dev):
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(64)
    r = _run(S, dev, wl, grid=grid, ninv_h=np.zeros((1, grid.npix)), precision="fp32")
    og = O.grid(64)
    for j in (0, 32):
        M = S.unpack_block(r["sampled"], r["plan"], "pband", 0, j)
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], np.zeros(grid.npix), j)
        assert _err(M, ref) <= TOL["fp32"]


@pytest.mark.parametrize("narrow", [0, 1, 2])
def test_indefinite_block_reports_pivot(S, dev, narrow):
    """A negative inverse-noise value makes blocks indefinite: info names the
    first bad pivot exactly as the oracle's Cholesky does, in the band part
    and in the corner, for each FP64 narrow-band kernel (the G-lane kernel,
    the band and border passes, and the one-lane shadow path with the border
    rows solved by column chunks)."""
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(64)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = wl.ninv(colat)
    ninv[0, : grid.npix // 3] *= -40.0
    r = _run(S, dev, wl, grid=grid, ninv_h=ninv, precision="fp64", factor=True, narrow=narrow)
    og = O.grid(64)
    bad = 0
    for j in range(og["nrings"]):
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv[0], j)
        _, info = O.cholesky(ref)
        assert r["info"][j] == info, j
        bad += info > 0
    assert bad > 0


@pytest.mark.parametrize("fprec,narrow", [("fp64", 0), ("fp64", 1), ("fp64", 2), ("fp32", 2), ("fp32", 3),
                                          ("fp32x2", 1), ("fp32x2", 2)])
def test_indefinite_corner_reports_pivot(S, dev, fprec, narrow):
    """A single negative inverse-noise pixel near the end of a ring leaves
    every leading minor of the band rows positive and breaks the block in its
    last w rows (the corner, after the border rows) or in the last band rows:
    info is the oracle's pivot index there, for each FP64 narrow-band kernel,
    the split-FP32 kernels, and the FP32 shadow paths (whose rescue
    refactors such blocks in FP64)."""
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(64)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = wl.ninv(colat)
    for j, back in ((40, 3), (20, 9), (55, 1)):
        n = int(grid.nring[j])
        ninv[0, int(grid.ring_offset[j]) + (n - back) * int(grid.ring_stride[j])] *= -3.0
    r = _run(S, dev, wl, grid=grid, ninv_h=ninv, precision="fp64", factor=True, factor_precision=fprec,
             narrow=narrow)
    og = O.grid(64)
    corner = band = 0
    for j in range(og["nrings"]):
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv[0], j)
        _, info = O.cholesky(ref)
        assert r["info"][j] == info, (j, int(r["info"][j]), info)
        _, n, w, fmt = r["plan"].block_layout("pband", 0, j)
        if info > 0 and fmt == S.BLOCK_PBAND:
            corner += info > n - w
            band += info <= n - w
    assert corner >= 2 and band >= 1, (corner, band)


# -- full size, in the bench's configuration ----------------------------------------------

_ORACLE_3000 = {}


def _oracle_block_3000(j, ninv0):
    """The oracle's block of ring j at l_max = 3000 (kept for the module:
    the equatorial ring takes the oracle tens of seconds)."""
    if j not in _ORACLE_3000:
        wl = W.WORKLOADS["lmax3000"]
        og = _ORACLE_3000.setdefault("grid", O.grid(wl.lmax))
        _ORACLE_3000[j] = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv0, j)[0]
    return _ORACLE_3000[j]


@pytest.mark.parametrize("precision,narrow", [("fp32", None), ("fp32x2", 1), ("fp32x2", 2), ("fp64", 0),
                                              ("fp64", 2)])
def test_full_size_lmax3000_sampled(S, dev, precision, narrow):
    """l_max = 3000, FWHM 5': every block factors; sampled blocks match the
    oracle and their factors reproduce them, from the pole to the equator
    (ring 1500, 6075 pixels, the longest elimination chain); FP64 and split
    FP32 with their earlier kernels and with the shadow path of chunked
    border rows."""
    wl = W.WORKLOADS["lmax3000"]
    r = _run(S, dev, wl, precision=precision, factor=True, narrow=narrow)
    assert np.all(r["info"] == 0)
    plan = r["plan"]
    for j in (0, 2, 37, 250, 1500):
        M = S.unpack_block(r["sampled"], plan, "pband", 0, j)
        ref = _oracle_block_3000(j, r["ninv"][0])
        assert _err(M, ref) <= TOL[precision], (j, _err(M, ref))
        L = S.unpack_block(r["factored"], plan, "pband", 0, j, factored=True)
        assert _err(L @ L.T, ref) <= 10 * TOL[precision], j


@pytest.mark.parametrize("fprec", ["fp64", "fp32x2", "fp32"])
@pytest.mark.parametrize("storage", ["pband", "dense"])
def test_factor_precisions_lmax500(S, dev, fprec, storage):
    """Every factor arithmetic reproduces the oracle's block through L L^T, and
    agrees with the oracle's L on rings small enough for its dense Cholesky."""
    wl = W.WORKLOADS["lmax500"]
    r = _run(S, dev, wl, precision="fp64", storage=storage, factor=True, factor_precision=fprec)
    og = O.grid(wl.lmax)
    assert np.all(r["info"] == 0)
    tol = {"fp64": 1e-12, "fp32x2": 1e-12, "fp32": 1e-6}[fprec]
    for j in (0, 3, 40, 250, 377):
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], r["ninv"][0], j)
        L = S.unpack_block(r["factored"], r["plan"], storage, 0, j, factored=True)
        assert _err(L @ L.T, ref) <= 10 * tol, (j, _err(L @ L.T, ref))
        if ref.shape[0] <= 400:
            Lref, _ = O.cholesky(ref)
            assert _err(L, Lref) <= 1000 * tol, (j, _err(L, Lref))


@pytest.mark.parametrize("floor", [0.0, 2.0])
def test_fp32_factor_fp64_rescue(S, dev, floor):
    """floor 2 sends every block through the FP64 rescue (FP64 accuracy),
    floor 0 none (FP32 accuracy)."""
    import torch
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    plan.set_pivot_floor(floor)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv_h = wl.ninv(colat)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(ninv_h, device=dev), precision="fp64")
    info = S.sympix_factor_blocks(plan, blocks, precision="fp32")
    fac = blocks.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    og = O.grid(wl.lmax)
    tol = 1e-12 if floor > 1 else 1e-6
    for j in (0, 5, 250, 499):
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv_h[0], j)
        L = S.unpack_block(fac, plan, "pband", 0, j, factored=True)
        assert _err(L @ L.T, ref) <= 10 * tol, (j, _err(L @ L.T, ref))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_wide_operators(S, dev, precision):
    """Several operators in one plan with beams wide enough for band widths
    above 16 (the wide-band factor and the wide-beam contraction)."""
    wl = W.Workload("wide", 200, [90.0, 150.0, 240.0, 360.0], [10.0, 0.0, 25.0, 5.0], [11, 12, 13, 14])
    r = _run(S, dev, wl, precision=precision, factor=True)
    plan = r["plan"]
    og = O.grid(wl.lmax)
    widths = [plan.block_layout("pband", o, 100)[2] for o in range(4)]
    assert max(widths) > 16, widths
    tol = TOL[precision]
    for o in range(4):
        for j in (0, 3, 47, 100, 200):
            ref, _ = O.block(og, wl.beams()[o], wl.priors()[o], wl.radii()[o], r["ninv"][o], j)
            M = S.unpack_block(r["sampled"], plan, "pband", o, j)
            assert _err(M, ref) <= tol, (o, j, _err(M, ref))
            _, info = O.cholesky(ref)
            assert r["info"][o * 201 + j] == info, (o, j)
            if info == 0:
                L = S.unpack_block(r["factored"], plan, "pband", o, j, factored=True)
                assert _err(L @ L.T, ref) <= 10 * tol, (o, j, _err(L @ L.T, ref))


@pytest.mark.parametrize("precision,storage", [("fp64", "pband"), ("fp32", "pband"), ("fp64", "dense")])
def test_wide_factor_every_block(S, dev, precision, storage):
    """Every block of band width 16 < w <= 64 (the wide-band factor, one CTA
    per block): L L^T against the sampled block, and info against numpy's
    Cholesky of the same block."""
    radii = np.linspace(0.22, 0.85, 6)  # block band widths from 17 to 64 and beyond at l_max = 120
    wl = W.Workload("wide120", 120, [600.0] * 6, [0.0, 5.0, 10.0, 15.0, 20.0, 25.0], list(range(61, 67)))
    r = _run(S, dev, wl, precision="fp64", storage=storage, factor=True, factor_precision=precision,
             radii=radii)
    plan, nr = r["plan"], int(r["grid"].nrings)
    info64 = None
    if precision != "fp64":  # the verdicts must be FP64's, row for row
        import torch
        again = torch.tensor(r["sampled"], dtype=torch.float64, device=dev)
        info64 = S.sympix_factor_blocks(plan, again, storage=storage, precision="fp64").cpu().numpy()
    seen = set()
    for o in range(6):
        for j in range(nr):
            _, n, w, fmt = plan.block_layout("pband", o, j)
            if fmt != S.BLOCK_PBAND or not 16 < w <= 64:
                continue
            seen.add(int(w))
            M = S.unpack_block(r["sampled"], plan, storage, o, j)
            try:
                np.linalg.cholesky(M)
                ok = True
            except np.linalg.LinAlgError:
                ok = False
            info = int(r["info"][o * nr + j])
            assert (info == 0) == ok, (o, j, n, w, info)
            if info64 is not None:
                assert info == int(info64[o * nr + j]), (o, j, n, w, info, int(info64[o * nr + j]))
            if ok:
                L = S.unpack_block(r["factored"], plan, storage, o, j, factored=True)
                assert _err(L @ L.T, M) <= 10 * TOL[precision], (o, j, n, w, _err(L @ L.T, M))
    assert len(seen) >= 20 and max(seen) >= 60, sorted(seen)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wide_band_sampling_matches_oracle(S, dev, precision):
    """Wide bands (w up to 64) next to rings of three times the pixel count:
    the cached-arc walk and, for arcs longer than the cache, the direct walk
    of the contraction, against the oracle's blocks."""
    radii = np.linspace(0.22, 0.85, 6)
    wl = W.Workload("wide120", 120, [600.0] * 6, [0.0, 5.0, 10.0, 15.0, 20.0, 25.0], list(range(61, 67)))
    r = _run(S, dev, wl, precision=precision, radii=radii)
    plan = r["plan"]
    og = O.grid(wl.lmax)
    widths = []
    for o, j in ((0, 11), (1, 12), (1, 13), (2, 14), (3, 25), (5, 60)):
        widths.append(plan.block_layout("pband", o, j)[2])
        ref, _ = O.block(og, wl.beams()[o], wl.priors()[o], radii[o], r["ninv"][o], j)
        M = S.unpack_block(r["sampled"], plan, "pband", o, j)
        assert _err(M, ref) <= TOL[precision], (o, j, _err(M, ref))
    assert max(widths) > 40, widths


# -- pixel-domain convolution g = B^ f (Eq. convolution-pixel) --------------------

def _pixel_ring_col(grid):
    npix = int(grid.npix)
    ring = np.zeros(npix, np.int32)
    col = np.zeros(npix, np.int32)
    for r in range(grid.nrings):
        c = np.arange(int(grid.nring[r]))
        idx = grid.ring_offset[r] + c * grid.ring_stride[r]
        ring[idx] = r
        col[idx] = c
    return ring, col


def _convolve(S, dev, lmax, bl_h, radii, f_h, precision, ring0=0, ring1=None):
    import torch
    grid = S.Grid(lmax)
    plan = S.Plan(grid, radii, ring0, ring1)
    bl = torch.tensor(bl_h, dtype=torch.float64, device=dev)
    S.sympix_kernel_table(plan, bl, torch.zeros_like(bl))
    f = torch.tensor(f_h, dtype=torch.float64, device=dev)
    g = S.sympix_convolve(plan, f, precision=precision)
    return grid, g.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32"])
def test_convolve_lmax64_every_pixel(S, dev, precision):
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(wl.lmax)
    f = np.random.default_rng(21).standard_normal((1, int(grid.npix)))
    _, g = _convolve(S, dev, wl.lmax, wl.beams(), wl.radii(), f, precision)
    ring, col = _pixel_ring_col(grid)
    ref, pairs = O.convolve(O.grid(wl.lmax), wl.beams()[0], wl.radii()[0], f[0], ring, col)
    assert pairs > 0
    assert _err(g[0], ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_convolve_lmax500_sampled(S, dev, precision):
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    f = np.random.default_rng(22).standard_normal((1, int(grid.npix)))
    _, g = _convolve(S, dev, wl.lmax, wl.beams(), wl.radii(), f, precision)
    ring, col = _pixel_ring_col(grid)
    pick = np.random.default_rng(23).choice(int(grid.npix), 300, replace=False)
    pick = np.concatenate([pick, grid.ring_offset[[0, 1, 250, 500]]])  # poles, equator
    ref, _ = O.convolve(O.grid(wl.lmax), wl.beams()[0], wl.radii()[0], f[0], ring[pick], col[pick])
    assert _err(g[0][pick], ref) <= TOL[precision]


def test_convolve_full_sky_support_and_two_operators(S, dev):
    """r_s >= pi couples every pixel pair: each ring is visited whole, once;
    two operators with different kernels and maps in one call."""
    lmax = 16
    grid = S.Grid(lmax)
    npix = int(grid.npix)
    l = np.arange(lmax + 1)
    bl = np.stack([np.exp(-0.01 * l * (l + 1)), 1.0 / (1.0 + l)])
    f = np.random.default_rng(24).standard_normal((2, npix))
    _, g = _convolve(S, dev, lmax, bl, [math.pi, 0.9], f, "fp64")
    ring, col = _pixel_ring_col(grid)
    og = O.grid(lmax)
    for o, r_s in enumerate([math.pi, 0.9]):
        ref, pairs = O.convolve(og, bl[o], r_s, f[o], ring, col)
        if o == 0:
            assert pairs == npix * npix
        assert _err(g[o], ref) <= 1e-10


def test_convolve_ring_range(S, dev):
    """A plan over rings [ring0, ring1) writes exactly those rings' pixels,
    with the values of the whole-sphere plan."""
    wl = W.WORKLOADS["lmax64"]
    grid = S.Grid(wl.lmax)
    f = np.random.default_rng(25).standard_normal((1, int(grid.npix)))
    _, full = _convolve(S, dev, wl.lmax, wl.beams(), wl.radii(), f, "fp64")
    _, part = _convolve(S, dev, wl.lmax, wl.beams(), wl.radii(), f, "fp64", ring0=20, ring1=40)
    ring, _ = _pixel_ring_col(grid)
    inside = (ring >= 20) & (ring < 40)
    assert np.array_equal(part[0][inside], full[0][inside])
    assert np.all(part[0][~inside] == 0.0)


# -- large dense-format blocks (a CTA per block, blocked Cholesky) ----------------

def _dense_block(sampled, plan, storage, ring):
    off, n, w, fmt = plan.block_layout(storage, 0, ring)
    return np.array(sampled[off:off + n * n]).reshape(n, n), fmt, n


def test_dense_storage_large_blocks_lmax1500(S, dev):
    """Dense storage at l_max = 1500 (rings of ~3000 pixels): the sampled
    blocks match the oracle's and L L^T reproduces them to FP64 accuracy."""
    wl = W.WORKLOADS["lmax1500"]
    grid = S.Grid(wl.lmax)
    j0 = grid.nrings // 2 - 1
    r = _run(S, dev, wl, grid=grid, ring0=j0, ring1=j0 + 2, precision="fp64", storage="dense", factor=True)
    assert np.all(r["info"] == 0)
    og = O.grid(wl.lmax)
    for j in (j0, j0 + 1):
        M, _, n = _dense_block(r["sampled"], r["plan"], "dense", j)
        L = np.tril(_dense_block(r["factored"], r["plan"], "dense", j)[0])
        assert n > 1024
        ref, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], r["ninv"][0], j)
        assert _err(M, ref) <= TOL["fp64"], (j, _err(M, ref))
        assert _err(L @ L.T, ref) <= 1e-11


def test_pband_storage_dense_format_large_blocks(S, dev):
    """A beam wide enough that the equatorial blocks are stored dense in
    periodic-band storage (w > 64) with n > 1024; FP64 factor."""
    wl = W.Workload("wide600", 600, [240.0], [0.0], [31])
    grid = S.Grid(wl.lmax)
    j0 = grid.nrings // 2 - 1
    r = _run(S, dev, wl, grid=grid, ring0=j0, ring1=j0 + 2, precision="fp64", storage="pband", factor=True,
             factor_precision="fp64")
    for j in (j0, j0 + 1):
        M, fmt, n = _dense_block(r["sampled"], r["plan"], "pband", j)
        assert fmt == S.BLOCK_DENSE and n > 1024
    if np.all(r["info"] == 0):
        for j in (j0, j0 + 1):
            M, _, _ = _dense_block(r["sampled"], r["plan"], "pband", j)
            L = np.tril(_dense_block(r["factored"], r["plan"], "pband", j)[0])
            assert _err(L @ L.T, M) <= 1e-11
    else:  # an indefinite block: the same verdict as numpy's dense Cholesky
        for k, j in enumerate((j0, j0 + 1)):
            M, _, _ = _dense_block(r["sampled"], r["plan"], "pband", j)
            try:
                np.linalg.cholesky(M)
                ok = True
            except np.linalg.LinAlgError:
                ok = False
            assert ok == (r["info"][k] == 0)


@pytest.mark.parametrize("nops", [9, 17])
def test_chunked_tables(S, dev, nops):
    """Operators share the recurrence in chunks (9 = 8 + 1, 17 = 8 + 8 + 1):
    every operator's blocks match the oracle with its own beam and prior."""
    fwhm = [180.0 + 20.0 * o for o in range(nops)]
    wl = W.Workload("chunked", 64, fwhm, [0.0] * nops, list(range(40, 40 + nops)))
    r = _run(S, dev, wl, precision="fp64")
    og = O.grid(wl.lmax)
    for o in range(nops):
        for j in (0, 20, 32):
            ref, _ = O.block(og, wl.beams()[o], wl.priors()[o], wl.radii()[o], r["ninv"][o], j)
            M = S.unpack_block(r["sampled"], r["plan"], "pband", o, j)
            assert _err(M, ref) <= TOL["fp64"], (o, j, _err(M, ref))


# -- the narrow-band factor (w <= 12): every width, every arithmetic ------------

@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("fprec", ["fp64", "fp32", "fp32x2"])
def test_narrow_factor_every_width(S, dev, fprec, kernel):
    """Operators whose radii give periodic-band widths from 0 to 12 at
    l_max = 120: every such block's factor reproduces the sampled block
    (L L^T), equals numpy's Cholesky of it, and its pivot verdict is numpy's;
    blocks of every width, in both the 8-lane (FP32) and the 4 / 16-lane
    (FP64, split FP32) slicings, including ragged slices."""
    radii = np.array([0.004, 0.012, 0.021, 0.033, 0.047, 0.063, 0.081, 0.1, 0.125, 0.155])
    nops = len(radii)
    wl = W.Workload("narrow120", 120, [300.0] * nops, [0.0, 5, 10, 15, 20, 0, 5, 10, 15, 20][:nops],
                    list(range(80, 80 + nops)))
    import torch
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, radii)
    plan.set_narrow_factor(kernel)
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(wl.ninv(colat), device=dev), precision="fp64")
    r = {"sampled": blocks.cpu().numpy()}
    r["info"] = S.sympix_factor_blocks(plan, blocks, precision=fprec).cpu().numpy()
    r["factored"] = blocks.cpu().numpy()
    nr = int(grid.nrings)
    tol = {"fp64": 1e-12, "fp32x2": 1e-12, "fp32": 1e-6}[fprec]
    seen = set()
    for o in range(nops):
        for j in range(nr):
            _, n, w, fmt = plan.block_layout("pband", o, j)
            if fmt != S.BLOCK_PBAND or w > 12:
                continue
            seen.add(int(w))
            M = S.unpack_block(r["sampled"], plan, "pband", o, j)
            try:
                Lref = np.linalg.cholesky(M)
                ok = True
            except np.linalg.LinAlgError:
                ok = False
            info = int(r["info"][o * nr + j])
            assert (info == 0) == ok, (o, j, n, w, info)
            if ok:
                L = S.unpack_block(r["factored"], plan, "pband", o, j, factored=True)
                assert _err(L @ L.T, M) <= 10 * tol, (o, j, n, w, _err(L @ L.T, M))
                assert _err(L, Lref) <= 1000 * tol, (o, j, n, w, _err(L, Lref))
    assert len(seen) >= 6 and min(seen) <= 2 and max(seen) >= 10, sorted(seen)


@pytest.mark.parametrize("fprec", ["fp64", "fp32", "fp32x2"])
def test_narrow_factor_matches_earlier_kernels(S, dev, fprec):
    """The G-lane narrow-band kernel and the earlier kernels (plan option 1)
    factor the l_max = 500 blocks to the same result within the arithmetic's
    rounding, with the same pivot verdicts."""
    import torch
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(wl.ninv(colat), device=dev), precision="fp64")
    a, b = blocks.clone(), blocks.clone()
    plan.set_narrow_factor(0)
    ia = S.sympix_factor_blocks(plan, a, precision=fprec).cpu().numpy()
    plan.set_narrow_factor(1)
    ib = S.sympix_factor_blocks(plan, b, precision=fprec).cpu().numpy()
    plan.set_narrow_factor(-1)
    assert plan.narrow_kernels() == {"fp64": 2, "fp32": 3, "fp32x2": 2}
    assert np.array_equal(ia, ib) and np.all(ia == 0)
    A, B = a.cpu().numpy(), b.cpu().numpy()
    tol = {"fp64": 1e-13, "fp32x2": 1e-11, "fp32": 1e-5}[fprec]
    for j in range(0, grid.nrings, 7):
        La = S.unpack_block(A, plan, "pband", 0, j, factored=True)
        Lb = S.unpack_block(B, plan, "pband", 0, j, factored=True)
        assert _err(La, Lb) <= tol, (j, _err(La, Lb))


def _fp32_factors(S, dev, wl, kernels, rings):
    import torch
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(wl.ninv(colat), device=dev), precision="fp32")
    out = {}
    for k in kernels:
        b = blocks.clone()
        plan.set_narrow_factor(k)
        info = S.sympix_factor_blocks(plan, b, precision="fp32").cpu().numpy()
        h = b.cpu().numpy()
        out[k] = (info, {j: S.unpack_block(h, plan, "pband", 0, j, factored=True) for j in rings})
        del b
    return plan, blocks, out


def test_chunked_border_matches_column_sweep_lmax500(S, dev):
    """FP32 option 2 (the band pass, then the border rows solved by column
    chunks with exact carries) and option 3 (band and border passes in two
    CTAs of one cooperative launch) against option 1 (the border swept column
    by column behind the band in the same CTA): the same factor within FP32
    rounding, the same pivot verdicts, on rings long enough for several
    chunks (and so the carry between them)."""
    wl = W.WORKLOADS["lmax500"]
    rings = list(range(0, 501, 25)) + [249, 250, 251]
    plan, _, out = _fp32_factors(S, dev, wl, (1, 2, 3), rings)
    assert np.array_equal(out[1][0], out[2][0]) and np.all(out[1][0] == 0)
    assert np.array_equal(out[1][0], out[3][0])
    for j in rings:
        assert _err(out[3][1][j], out[1][1][j]) <= 1e-5, j
    nchunks = 0
    for j in rings:
        _, n, w, fmt = plan.block_layout("pband", 0, j)
        if fmt == S.BLOCK_PBAND:
            nchunks = max(nchunks, -(-(n - w) // ((288 // (w + 1)) * (w + 1))))
        assert _err(out[2][1][j], out[1][1][j]) <= 1e-5, (j, n, w, _err(out[2][1][j], out[1][1][j]))
    assert nchunks >= 3


def test_chunked_border_matches_column_sweep_lmax3000(S, dev):
    """The same at full size: the equatorial rings (n = 6075, 22 chunks of
    288 columns), the w = 10 rings where the ring count changes, and polar
    and mid-latitude rings."""
    wl = W.WORKLOADS["lmax3000"]
    rings = [0, 5, 300, 901, 902, 1500, 2098, 2293, 2700, 3000]
    plan, _, out = _fp32_factors(S, dev, wl, (1, 2, 3), rings)
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][0], out[3][0])
    for j in rings:
        assert _err(out[3][1][j], out[1][1][j]) <= 1e-5, j
    widths = set()
    for j in rings:
        _, n, w, fmt = plan.block_layout("pband", 0, j)
        widths.add(int(w))
        assert _err(out[2][1][j], out[1][1][j]) <= 1e-5, (j, n, w, _err(out[2][1][j], out[1][1][j]))
    assert {8, 9, 10} <= widths


def test_chunked_border_rescue_restores_fp64(S, dev):
    """Option 2 with the pivot floor at 2: every block is sent to the FP64
    rescue, and the result is the FP64 factor (FP64 accuracy)."""
    import torch
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(wl.ninv(colat), device=dev), precision="fp64")
    a, b = blocks.clone(), blocks.clone()
    plan.set_narrow_factor(2)
    plan.set_pivot_floor(2.0)
    ia = S.sympix_factor_blocks(plan, a, precision="fp32").cpu().numpy()
    plan.set_pivot_floor(0.05)
    ib = S.sympix_factor_blocks(plan, b, precision="fp64").cpu().numpy()
    assert np.all(ia == 0) and np.all(ib == 0)
    A, B = a.cpu().numpy(), b.cpu().numpy()
    for j in range(0, grid.nrings, 5):
        La = S.unpack_block(A, plan, "pband", 0, j, factored=True)
        Lb = S.unpack_block(B, plan, "pband", 0, j, factored=True)
        assert _err(La, Lb) <= 1e-12, j


def test_narrow_factor_fp32_rescue_restores_fp64(S, dev):
    """With the pivot floor at 2 every FP32 narrow-band block is marked and
    refactored in FP64 from its untouched input: FP64 accuracy, and the same
    factor as the FP64 narrow kernel bit for bit."""
    import torch
    wl = W.WORKLOADS["lmax500"]
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    S.sympix_kernel_table(plan, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev))
    blocks = S.sympix_sample_blocks(plan, torch.tensor(wl.ninv(colat), device=dev), precision="fp64")
    a, b = blocks.clone(), blocks.clone()
    plan.set_narrow_factor(0)
    plan.set_pivot_floor(2.0)
    ia = S.sympix_factor_blocks(plan, a, precision="fp32").cpu().numpy()
    plan.set_pivot_floor(0.05)
    ib = S.sympix_factor_blocks(plan, b, precision="fp64").cpu().numpy()
    assert np.all(ia == 0) and np.all(ib == 0)
    # the FP64 rescue runs the FP64 G-lane kernel on the FP64 slicing, as the FP64
    # factor does for w <= 8 (wider bands go to the lane groups there): bit for bit
    A, B = a.cpu().numpy(), b.cpu().numpy()
    for j in range(0, grid.nrings, 5):
        _, n, w, fmt = plan.block_layout("pband", 0, j)
        La = S.unpack_block(A, plan, "pband", 0, j, factored=True)
        Lb = S.unpack_block(B, plan, "pband", 0, j, factored=True)
        if fmt == S.BLOCK_PBAND and w <= 8:
            assert np.array_equal(La, Lb), j
        else:
            assert _err(La, Lb) <= 1e-12, j
