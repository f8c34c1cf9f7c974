"""Blocks between rings and the block preconditioner applied to a vector.

The blocks M_jk between ring j and ring j + delta (Eq. system-rewritten and
Eq. Dhat with rows and columns on different rings) against the oracle's
block between two rings, element by element; the block-Jacobi apply
y_j = M_jj^-1 x_j against the oracle's Cholesky and triangular solves; and
a preconditioned conjugate-gradient solve on the operator assembled from the
sampled diagonal and off-diagonal blocks, which must converge faster than
the unpreconditioned one.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


def _err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _setup(S, wl, ninv_h=None, ring0=0, ring1=None):
    import torch
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii(), ring0, ring1)
    if ninv_h is None:
        colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
        ninv_h = wl.ninv(colat)
    dev = torch.device("cuda", 0)
    return grid, plan, ninv_h, torch.tensor(wl.beams(), device=dev), torch.tensor(wl.priors(), device=dev), \
        torch.tensor(ninv_h, device=dev)


@pytest.mark.parametrize("delta", [1, 2, 5])
def test_coupling_lmax64_matches_oracle(S, delta):
    """Every block between ring j and ring j + delta at l_max = 64 (masked
    band, 20 deg), FP64, within 1e-10 of the oracle's block."""
    wl = W.WORKLOADS["lmax64"]
    grid, plan, ninv_h, bl, dl, ninv = _setup(S, wl)
    nbytes, el = plan.coupling_size(delta)
    assert el > 0
    S.sympix_kernel_table(plan, bl, dl)  # d at every class after the layout exists
    buf = S.sympix_sample_coupling(plan, ninv, delta).cpu().numpy()
    og = O.grid(wl.lmax)
    nonzero = 0
    for j in range(grid.nrings - delta):
        M = S.unpack_coupling(buf, plan, delta, 0, j)
        ref, _ = O.block_pair(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv_h[0], j, j + delta)
        if not np.any(ref):
            assert not np.any(M), j
            continue
        nonzero += 1
        assert _err(M, ref) <= 1e-10, (j, _err(M, ref))
    assert nonzero > 0


def test_coupling_prior_only_and_ring_range(S):
    """N^-1 = 0 leaves D^ between the rings alone; a ring sub-range plans
    only the pairs inside it, with the values of the whole plan."""
    import torch
    wl = W.WORKLOADS["lmax64"]
    grid, plan, _, bl, dl, _ = _setup(S, wl)
    zero = torch.zeros((1, int(grid.npix)), dtype=torch.float64, device="cuda")
    plan.coupling_size(1)
    S.sympix_kernel_table(plan, bl, dl)
    buf = S.sympix_sample_coupling(plan, zero, 1).cpu().numpy()
    og = O.grid(wl.lmax)
    for j in (3, 20, 32, 50):
        M = S.unpack_coupling(buf, plan, 1, 0, j)
        ref, _ = O.block_pair(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], np.zeros(grid.npix), j, j + 1)
        assert np.any(ref) and _err(M, ref) <= 1e-10, j
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = torch.tensor(wl.ninv(colat), device="cuda")
    full = S.sympix_sample_coupling(plan, ninv, 1).cpu().numpy()
    sub = S.Plan(grid, wl.radii(), 20, 30)
    sub.coupling_size(1)
    S.sympix_kernel_table(sub, bl, dl)
    part = S.sympix_sample_coupling(sub, ninv, 1).cpu().numpy()
    for j in range(20, 29):
        assert np.array_equal(S.unpack_coupling(part, sub, 1, 0, j), S.unpack_coupling(full, plan, 1, 0, j))
    with pytest.raises(S.SympixError):
        sub.coupling_layout(1, 0, 29)  # ring 30 is outside the plan


def test_coupling_lmax500_sampled(S):
    wl = W.WORKLOADS["lmax500"]
    grid, plan, ninv_h, bl, dl, ninv = _setup(S, wl)
    plan.coupling_size(1)
    S.sympix_kernel_table(plan, bl, dl)
    buf = S.sympix_sample_coupling(plan, ninv, 1).cpu().numpy()
    og = O.grid(wl.lmax)
    for j in (0, 1, 60, 249, 250, 499):
        M = S.unpack_coupling(buf, plan, 1, 0, j)
        ref, _ = O.block_pair(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv_h[0], j, j + 1)
        assert _err(M, ref) <= 1e-10, (j, _err(M, ref))


@pytest.mark.parametrize("storage", ["pband", "dense"])
def test_apply_matches_oracle_solves(S, storage):
    """y_j = L^-T L^-1 x_j with the GPU factors against the oracle's Cholesky
    of its own block and its forward and back substitution, every ring at
    l_max = 64."""
    import torch
    wl = W.WORKLOADS["lmax64"]
    grid, plan, ninv_h, bl, dl, ninv = _setup(S, wl)
    S.sympix_kernel_table(plan, bl, dl)
    blocks = S.sympix_sample_blocks(plan, ninv, precision="fp64", storage=storage)
    info = S.sympix_factor_blocks(plan, blocks, storage=storage, precision="fp64")
    x_h = np.random.default_rng(41).standard_normal((1, int(grid.npix)))
    y = S.sympix_apply(plan, blocks, info, torch.tensor(x_h, device="cuda"), storage=storage).cpu().numpy()
    og = O.grid(wl.lmax)
    assert np.all(info.cpu().numpy() == 0)
    for j in range(grid.nrings):
        idx = grid.ring_offset[j] + grid.ring_stride[j] * np.arange(grid.nring[j])
        ref_M, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv_h[0], j)
        Lr, inf = O.cholesky(ref_M)
        assert inf == 0
        ref = O.trisolve(Lr, O.trisolve(Lr, x_h[0, idx]), trans=True)
        assert _err(y[0, idx], ref) <= 1e-9, (j, _err(y[0, idx], ref))


def test_apply_lmax500_and_failed_blocks_pass_through(S):
    """l_max = 500 rings (bands with borders, polar dense blocks): apply
    against the oracle; blocks made indefinite by negative N^-1 pass x
    through unchanged."""
    import torch
    wl = W.WORKLOADS["lmax500"]
    grid, plan, ninv_h, bl, dl, ninv = _setup(S, wl)
    S.sympix_kernel_table(plan, bl, dl)
    blocks = S.sympix_sample_blocks(plan, ninv, precision="fp64")
    info = S.sympix_factor_blocks(plan, blocks, precision="fp64")
    x_h = np.random.default_rng(42).standard_normal((1, int(grid.npix)))
    y = S.sympix_apply(plan, blocks, info, torch.tensor(x_h, device="cuda")).cpu().numpy()
    og = O.grid(wl.lmax)
    for j in (0, 2, 100, 250, 498):
        idx = grid.ring_offset[j] + grid.ring_stride[j] * np.arange(grid.nring[j])
        ref_M, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv_h[0], j)
        Lr, _ = O.cholesky(ref_M)
        ref = O.trisolve(Lr, O.trisolve(Lr, x_h[0, idx]), trans=True)
        assert _err(y[0, idx], ref) <= 1e-9, j
    bad = ninv_h.copy()
    bad[0, : grid.npix // 4] *= -40.0
    blocks = S.sympix_sample_blocks(plan, torch.tensor(bad, device="cuda"), precision="fp64")
    info = S.sympix_factor_blocks(plan, blocks, precision="fp64")
    inf_h = info.cpu().numpy()
    assert np.any(inf_h != 0)
    y = S.sympix_apply(plan, blocks, info, torch.tensor(x_h, device="cuda")).cpu().numpy()
    for j in np.nonzero(inf_h)[0][:5]:
        idx = grid.ring_offset[j] + grid.ring_stride[j] * np.arange(grid.nring[j])
        assert np.array_equal(y[0, idx], x_h[0, idx])


def test_block_jacobi_preconditions_the_assembled_operator(S):
    """The operator assembled from the sampled ring blocks (diagonal and
    every offset with a nonzero block) is the truncated D^ + B^T N^-1 B^.
    Truncating the prior's kernel can make it indefinite, so the prior is
    scaled down until it is positive definite (checked); conjugate gradients
    with the block preconditioner (sympix_apply) then reach a relative
    residual of 1e-6 in well under half the iterations that plain CG needs."""
    import torch
    wl = W.Workload("cg32", 32, [180.0], [0.0], [17])
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv = torch.tensor(wl.ninv(colat), device="cuda")
    bl = torch.tensor(wl.beams(), device="cuda")
    dl = torch.tensor(wl.priors() * 0.01, device="cuda")
    N, npix = grid.nrings, int(grid.npix)
    deltas = list(range(1, 12))
    for delta in deltas:
        plan.coupling_size(delta)
    S.sympix_kernel_table(plan, bl, dl)
    blocks = S.sympix_sample_blocks(plan, ninv, precision="fp64")
    sampled = blocks.cpu().numpy()
    info = S.sympix_factor_blocks(plan, blocks, precision="fp64")
    assert np.all(info.cpu().numpy() == 0)
    idx = [grid.ring_offset[j] + grid.ring_stride[j] * np.arange(grid.nring[j]) for j in range(N)]
    A = np.zeros((npix, npix))
    for j in range(N):
        A[np.ix_(idx[j], idx[j])] = S.unpack_block(sampled, plan, "pband", 0, j)
    widest = 0
    for delta in deltas:
        buf = S.sympix_sample_coupling(plan, ninv, delta).cpu().numpy()
        for j in range(N - delta):
            M = S.unpack_coupling(buf, plan, delta, 0, j)
            if np.any(M):
                widest = max(widest, delta)
            A[np.ix_(idx[j], idx[j + delta])] = M
            A[np.ix_(idx[j + delta], idx[j])] = M.T
    assert widest < deltas[-1], "the offsets planned must reach past the last nonzero block"
    np.linalg.cholesky(A)  # positive definite
    rhs = np.random.default_rng(5).standard_normal(npix)

    def cg(prec, cap=6000):
        x = np.zeros(npix)
        r = rhs.copy()
        z = prec(r)
        p = z.copy()
        rz = r @ z
        for it in range(1, cap):
            Ap = A @ p
            a = rz / (p @ Ap)
            x += a * p
            r -= a * Ap
            if np.linalg.norm(r) <= 1e-6 * np.linalg.norm(rhs):
                return it, x
            z = prec(r)
            rz2 = r @ z
            p = z + (rz2 / rz) * p
            rz = rz2
        return cap, x

    def jacobi(r):
        t = torch.tensor(r[None, :], device="cuda")
        return S.sympix_apply(plan, blocks, info, t).cpu().numpy()[0]

    it_plain, _ = cg(lambda r: r)
    it_prec, x1 = cg(jacobi)
    assert np.linalg.norm(A @ x1 - rhs) <= 2e-6 * np.linalg.norm(rhs)
    assert 2 * it_prec < it_plain, (it_prec, it_plain)
