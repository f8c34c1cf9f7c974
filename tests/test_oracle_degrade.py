"""Pins of the oracle's Y2 != Y1 functions (Sec. 4.2, Eq. substitution and Eq.
degrade): the noise of an external observation grid carried onto an auxiliary
grid, and the preconditioner block whose B^ = Y2 B Y1^T sums over that grid.

Everything the oracle computes here goes through its own kernel evaluation
(the addition theorem summed over m); the pins compare it with dense spherical
harmonics from scipy (`sph_harm_y`) and with direct sums over 3-vectors and
numpy's Legendre series, which share nothing with it."""
import math

import numpy as np
import scipy.special as sp
from numpy.polynomial import legendre as npleg

from oracle import oracle as O


def _ymat(th, ph, L):
    """Dense complex spherical harmonics, columns (l, m) for l <= L."""
    return np.stack([sp.sph_harm_y(l, m, th, ph) for l in range(L + 1) for m in range(-l, l + 1)], axis=1)


def _pixels(g):
    """Colatitude and longitude of every pixel of a grid, in its numbering."""
    T = np.zeros(int(g["npix"]))
    P = np.zeros(int(g["npix"]))
    for r in range(int(g["nrings"])):
        n = int(g["nring"][r])
        c = np.arange(n)
        k = int(g["ring_offset"][r]) + c * int(g["ring_stride"][r])
        T[k] = g["theta"][r]
        P[k] = 2.0 * math.pi * (c + 0.5) / n
    return T, P


def _observation(seed=7, nobs=600):
    rng = np.random.default_rng(seed)
    th = np.arccos(rng.uniform(-1.0, 1.0, nobs))
    ph = rng.uniform(0.0, 2.0 * math.pi, nobs)
    return th, ph, np.exp(0.3 * rng.standard_normal(nobs))


def _substitution_error(L1, L2, g2, obs):
    """max |Y_obs^H N^-1 Y_obs - Y_2^H N_2^-1 Y_2| / max |Y_obs^H N^-1 Y_obs| over l, l' <= L1."""
    th, ph, val = obs
    Yo = _ymat(th, ph, L1)
    lhs = Yo.conj().T @ (val[:, None] * Yo)
    t2 = O.degrade(L2, th, ph, val, g2)
    T, P = _pixels(g2)
    Y2 = _ymat(T, P, L1)
    rhs = Y2.conj().T @ (t2[:, None] * Y2)
    return np.abs(lhs - rhs).max() / np.abs(lhs).max()


def test_substitution_exact_on_an_exact_grid():
    """Eq. substitution holds to rounding for harmonics up to L1 when Y2 keeps
    l <= 2 L1 and the auxiliary grid integrates band limit 2 L1 + L2 exactly
    (Gauss-Legendre rings, enough pixels per ring), at arbitrary observation
    points with white noise; with Y2 cut below 2 L1 it does not hold."""
    obs = _observation()
    L1 = 5
    exact = O.gl_grid(2 * L1 + 1, 4 * L1 + 1)
    assert _substitution_error(L1, 2 * L1, exact, obs) < 1e-13
    assert _substitution_error(L1, 3 * L1, O.gl_grid(3 * L1, 5 * L1 + 1), obs) < 1e-13
    assert _substitution_error(L1, 2 * L1 - 2, exact, obs) > 1e-3
    assert _substitution_error(L1, L1, exact, obs) > 1e-3


def test_substitution_on_the_papers_dp_grids():
    """The paper's accuracy statement for the auxiliary SymPix grid: with the
    band limit of Y2 one times that of Y1 the substitution is only approximate
    (the paper quotes O(1e-2)), with two or four times it holds to rounding
    on the DP grid with the paper's polar threshold (quoted O(1e-10) and
    O(1e-14) with HEALPix observations)."""
    obs = _observation(seed=11)
    L1 = 6
    err = {f: _substitution_error(L1, f * L1, O.grid(f * L1, k=2, layout="dp"), obs) for f in (1, 2, 4)}
    assert err[1] > 1e-3, err
    assert err[2] < 1e-12 and err[4] < 1e-12, err


def test_block_y2_equals_direct_sum_over_observations():
    """Without truncation (r_s = pi) the block of a grid-1 ring with the noise
    carried to an exact auxiliary grid equals the direct sum over the
    observation points, D^_qr + sum_i b(n_q.n_i) theta_i b(n_i.n_r), with b
    and d as numpy Legendre series of 3-vector dot products."""
    L1 = 5
    g1 = O.grid(L1)
    th, ph, val = _observation(seed=3, nobs=400)
    g2 = O.gl_grid(2 * L1 + 1, 4 * L1 + 1)
    t2 = O.degrade(2 * L1, th, ph, val, g2)
    ell = np.arange(L1 + 1)
    bl = np.exp(-0.5 * ell * (ell + 1) * (0.4) ** 2)
    dl = (ell * (ell + 1.0)) ** 2 / (L1 * (L1 + 1.0)) ** 2 + 0.1
    cb, cd = (2 * ell + 1) / (4 * math.pi) * bl, (2 * ell + 1) / (4 * math.pi) * dl

    def vec(t, p):
        return np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], axis=-1)

    obs_v = vec(th, ph)
    for j in (0, int(g1["nrings"]) // 2):
        n = int(g1["nring"][j])
        q = vec(np.full(n, g1["theta"][j]), 2 * math.pi * (np.arange(n) + 0.5) / n)
        Bq = npleg.legval(np.clip(q @ obs_v.T, -1.0, 1.0), cb)  # [q, i]
        ref = npleg.legval(np.clip(q @ q.T, -1.0, 1.0), cd) + (Bq * val[None, :]) @ Bq.T
        M, triples = O.block_y2(g1, j, g2, bl, dl, math.pi, t2)
        assert triples == n * n * int(g2["npix"])
        assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(M - ref).max() / np.abs(ref).max()


def test_block_y2_with_the_same_grid_is_the_block():
    """With the auxiliary grid equal to grid 1 the Y2 != Y1 block is the
    Y2 = Y1 block, truncated support included, bit for bit."""
    L1 = 24
    g = O.grid(L1)
    rng = np.random.default_rng(5)
    ninv = np.exp(0.3 * rng.standard_normal(int(g["npix"])))
    ell = np.arange(L1 + 1)
    bl = np.exp(-0.5 * ell * (ell + 1) * (0.12) ** 2)
    dl = (ell * (ell + 1.0)) ** 2 / (L1 * (L1 + 1.0)) ** 2
    r_s = 0.5
    for j in (1, int(g["nrings"]) // 2):
        M1, t1 = O.block(g, bl, dl, r_s, ninv, j)
        M2, t2 = O.block_y2(g, j, g, bl, dl, r_s, ninv)
        assert t1 == t2 and np.array_equal(M1, M2)
