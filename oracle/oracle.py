"""ctypes front end of the SymPix oracle (plain FP64 C, ``sympix_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU baseline / reference arm of ``bench.py``.  The library package
never imports this module; the CUDA path and the oracle share no code.

Every function is a thin marshalling layer over one C function; the C file
states which passage of the paper each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sympix_oracle.c"
_LIB = _HERE / "liboracle.so"

_dptr = ctypes.POINTER(ctypes.c_double)
_i32ptr = ctypes.POINTER(ctypes.c_int32)
_i64ptr = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        subprocess.run(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-o", str(tmp), str(_SRC), "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        L.sympix_oracle_kernel_u.restype = ctypes.c_double
        L.sympix_oracle_kernel_u.argtypes = [ctypes.c_int, _dptr, ctypes.c_double]
        L.sympix_oracle_gl_theta.argtypes = [ctypes.c_int, _dptr]
        L.sympix_oracle_gl_weights.argtypes = [ctypes.c_int, _dptr, _dptr]
        L.sympix_oracle_layout_greedy.argtypes = [ctypes.c_int, _dptr, _i32ptr]
        L.sympix_oracle_layout_dp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              _dptr, _i32ptr, _i32ptr]
        L.sympix_oracle_u.restype = ctypes.c_double
        L.sympix_oracle_u.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_long,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_long]
        L.sympix_oracle_coupled.argtypes = [_dptr, _i32ptr, ctypes.c_int, ctypes.c_long,
                                            ctypes.c_int, ctypes.c_double, _i32ptr]
        L.sympix_oracle_block.restype = ctypes.c_long
        L.sympix_oracle_block.argtypes = [ctypes.c_int, _dptr, _i32ptr, _i64ptr, _i32ptr,
                                          ctypes.c_int, _dptr, _dptr, ctypes.c_double,
                                          _dptr, ctypes.c_int, _dptr]
        L.sympix_oracle_cholesky.argtypes = [ctypes.c_int, _dptr, _dptr]
        L.sympix_oracle_convolve.restype = ctypes.c_long
        L.sympix_oracle_convolve.argtypes = [ctypes.c_int, _dptr, _i32ptr, _i64ptr, _i32ptr, ctypes.c_int, _dptr,
                                             ctypes.c_double, _dptr, ctypes.c_int, _i32ptr, _i32ptr, _dptr]
        L.sympix_oracle_ordering.restype = ctypes.c_long
        L.sympix_oracle_ordering.argtypes = [ctypes.c_int, ctypes.c_int, _i32ptr, _i64ptr, _i32ptr]
        L.sympix_oracle_block_pair.restype = ctypes.c_long
        L.sympix_oracle_block_pair.argtypes = [ctypes.c_int, _dptr, _i32ptr, _i64ptr, _i32ptr,
                                               ctypes.c_int, _dptr, _dptr, ctypes.c_double,
                                               _dptr, ctypes.c_int, ctypes.c_int, _dptr]
        L.sympix_oracle_tiles_coupled.argtypes = [ctypes.c_int, ctypes.c_int, _i32ptr, ctypes.c_int, ctypes.c_long,
                                                  ctypes.c_int, ctypes.c_long]
        L.sympix_oracle_band_block.restype = ctypes.c_long
        L.sympix_oracle_band_block.argtypes = [ctypes.c_int, _dptr, _i32ptr, _i64ptr, _i32ptr, ctypes.c_int,
                                               ctypes.c_int, _dptr, _dptr, _dptr, ctypes.c_int, _dptr]
        L.sympix_oracle_trisolve.argtypes = [ctypes.c_int, _dptr, _dptr, ctypes.c_int, _dptr]
        L.sympix_oracle_support_margin.restype = ctypes.c_double
        L.sympix_oracle_support_margin.argtypes = [ctypes.c_int, _dptr, _i32ptr, ctypes.c_double,
                                                   ctypes.c_int, ctypes.c_int]
        L.sympix_oracle_guarded_radius.restype = ctypes.c_double
        L.sympix_oracle_guarded_radius.argtypes = [ctypes.c_int, _dptr, _i32ptr, ctypes.c_double,
                                                   ctypes.c_int, ctypes.c_int, _dptr]
        L.sympix_oracle_degrade.restype = ctypes.c_long
        L.sympix_oracle_degrade.argtypes = [ctypes.c_int, ctypes.c_long, _dptr, _dptr, _dptr, ctypes.c_int, _dptr,
                                            _i32ptr, _dptr, _i64ptr, _i32ptr, _dptr]
        L.sympix_oracle_block_y2.restype = ctypes.c_long
        L.sympix_oracle_block_y2.argtypes = [_dptr, _i32ptr, ctypes.c_int, ctypes.c_int, _dptr, _i32ptr, _i64ptr,
                                             _i32ptr, ctypes.c_int, _dptr, _dptr, ctypes.c_double, _dptr, _dptr]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# -- grid ---------------------------------------------------------------------

def gl_theta(N: int) -> np.ndarray:
    """Ring colatitudes theta_j (north to south), roots of P_N(cos theta)."""
    th = np.empty(N, dtype=np.float64)
    if lib().sympix_oracle_gl_theta(N, _p(th, _dptr)) != 0:
        raise ValueError("bad ring count")
    return th


def gl_weights(theta: np.ndarray) -> np.ndarray:
    th = _f64(theta)
    w = np.empty_like(th)
    lib().sympix_oracle_gl_weights(len(th), _p(th, _dptr), _p(w, _dptr))
    return w


def layout_greedy(lmax: int, theta: np.ndarray) -> np.ndarray:
    th = _f64(theta)
    n = np.zeros(lmax + 1, dtype=np.int32)
    lib().sympix_oracle_layout_greedy(lmax, _p(th, _dptr), _p(n, _i32ptr))
    return n


def dp_nrings(lmax: int, k: int) -> int:
    N = lmax + 1
    if N % (2 * k):
        N += 2 * k - N % (2 * k)
    return N


def layout_dp(lmax: int, k: int, thr: float, theta: np.ndarray):
    """Tiles per northern band T_i and the bound alpha_i (Fig. Optimal-SymPix-Grid)."""
    th = _f64(theta)
    nb = len(th) // (2 * k)
    T = np.zeros(nb, dtype=np.int32)
    alpha = np.zeros(nb, dtype=np.int32)
    rc = lib().sympix_oracle_layout_dp(lmax, k, float(thr), _p(th, _dptr), _p(T, _i32ptr),
                                       _p(alpha, _i32ptr))
    if rc != 0:
        raise ValueError("no DP layout satisfies the constraints")
    return T, alpha


def ordering(N: int, k: int, nring: np.ndarray):
    nr = np.ascontiguousarray(nring, dtype=np.int32)
    off = np.zeros(N, dtype=np.int64)
    stride = np.zeros(N, dtype=np.int32)
    npix = lib().sympix_oracle_ordering(N, k, _p(nr, _i32ptr), _p(off, _i64ptr), _p(stride, _i32ptr))
    if npix < 0:
        raise ValueError("ring counts do not form bands of k rings")
    return off, stride, int(npix)


def grid(lmax: int, k: int = 1, layout: str = "greedy", thr: float = -1.0) -> dict:
    """The whole grid: theta, per-ring counts, pixel numbering."""
    if layout == "greedy":
        if k != 1:
            raise ValueError("the greedy layout has k = 1")
        N = lmax + 1
        theta = gl_theta(N)
        nring = layout_greedy(lmax, theta)
    elif layout == "dp":
        N = dp_nrings(lmax, k)
        theta = gl_theta(N)
        T, _ = layout_dp(lmax, k, thr, theta)
        nb = N // (2 * k)
        nring = np.zeros(N, dtype=np.int32)
        for i in range(nb):
            for r in range(k):
                nring[i * k + r] = k * T[i]
                nring[N - 1 - i * k - r] = k * T[i]
    else:
        raise ValueError(layout)
    off, stride, npix = ordering(N, k, nring)
    return dict(lmax=lmax, k=k, nrings=N, theta=theta, nring=nring,
                ring_offset=off, ring_stride=stride, npix=npix)


# -- kernel values and support -----------------------------------------------

def kernel_u(lmax: int, cl: np.ndarray, u) -> np.ndarray:
    """Eq. addition-theorem at x = 1 - u (vectorised over u by a Python loop)."""
    c = _f64(cl)
    assert len(c) >= lmax + 1
    f = lib().sympix_oracle_kernel_u
    uu = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([f(lmax, _p(c, _dptr), float(x)) for x in uu])


def pair_u(theta1: float, n1: int, c1: int, theta2: float, n2: int, c2: int) -> float:
    return lib().sympix_oracle_u(float(theta1), int(n1), int(c1), float(theta2), int(n2), int(c2))


def support_margin(g: dict, r_s: float, ring0: int = 0, ring1: int | None = None) -> float:
    """Smallest |u - u_s| / u_s over the pixel pairs of rings [ring0, ring1)."""
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    r1 = g["nrings"] if ring1 is None else int(ring1)
    return lib().sympix_oracle_support_margin(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr), float(r_s),
                                              int(ring0), r1)


def guarded_radius(g: dict, r_s: float, ring0: int = 0, ring1: int | None = None):
    """(radius, margin): r_s, or r_s scaled by (1 - 1e-9) until no pixel pair
    lies within 1e-12 (relative) of the support threshold."""
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    r1 = g["nrings"] if ring1 is None else int(ring1)
    m = ctypes.c_double()
    r = lib().sympix_oracle_guarded_radius(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr), float(r_s),
                                           int(ring0), r1, ctypes.byref(m))
    return float(r), float(m.value)


def coupled(g: dict, j: int, c: int, rho: int, r_s: float) -> np.ndarray:
    out = np.zeros(int(g["nring"][rho]), dtype=np.int32)
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    cnt = lib().sympix_oracle_coupled(_p(th, _dptr), _p(nr, _i32ptr), int(j), int(c), int(rho),
                                      float(r_s), _p(out, _i32ptr))
    return out[:cnt].copy()


# -- blocks -------------------------------------------------------------------

def block(g: dict, bl: np.ndarray, dl: np.ndarray, r_s: float, ninv: np.ndarray, j: int):
    """Dense preconditioner block of ring j and the number of triples summed."""
    n = int(g["nring"][j])
    M = np.zeros((n, n), dtype=np.float64)
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    off = np.ascontiguousarray(g["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g["ring_stride"], dtype=np.int32)
    b = _f64(bl)
    d = _f64(dl)
    nv = _f64(ninv)
    assert len(nv) == g["npix"]
    triples = lib().sympix_oracle_block(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr),
                                        _p(off, _i64ptr), _p(st, _i32ptr), g["lmax"],
                                        _p(b, _dptr), _p(d, _dptr), float(r_s),
                                        _p(nv, _dptr), int(j), _p(M, _dptr))
    return M, int(triples)


def block_pair(g: dict, bl: np.ndarray, dl: np.ndarray, r_s: float, ninv: np.ndarray, j: int, k: int):
    """Dense block between ring j (rows) and ring k (columns), and the triples summed."""
    nj, nk = int(g["nring"][j]), int(g["nring"][k])
    M = np.zeros((nj, nk), dtype=np.float64)
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    off = np.ascontiguousarray(g["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g["ring_stride"], dtype=np.int32)
    b = _f64(bl)
    d = _f64(dl)
    nv = _f64(ninv)
    assert len(nv) == g["npix"]
    triples = lib().sympix_oracle_block_pair(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr), _p(off, _i64ptr),
                                             _p(st, _i32ptr), g["lmax"], _p(b, _dptr), _p(d, _dptr), float(r_s),
                                             _p(nv, _dptr), int(j), int(k), _p(M, _dptr))
    return M, int(triples)


def tiles_coupled(g: dict, ra: int, ca: int, rb: int, cb: int) -> bool:
    """Tile adjacency of two pixels of a DP grid (Sec. 2.3 tiling, Sec. 4.2)."""
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    return bool(lib().sympix_oracle_tiles_coupled(g["nrings"], g["k"], _p(nr, _i32ptr), int(ra), int(ca),
                                                  int(rb), int(cb)))


def band_block(g: dict, bl: np.ndarray, dl: np.ndarray, ninv: np.ndarray, band: int):
    """Dense block of band `band` (k rings) of a DP grid under tile adjacency,
    in the band's pixel order, and the triples summed."""
    k = g["k"]
    K = k * int(g["nring"][band * k])
    M = np.zeros((K, K), dtype=np.float64)
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    off = np.ascontiguousarray(g["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g["ring_stride"], dtype=np.int32)
    b = _f64(bl)
    d = _f64(dl)
    nv = _f64(ninv)
    assert len(nv) == g["npix"]
    triples = lib().sympix_oracle_band_block(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr), _p(off, _i64ptr),
                                             _p(st, _i32ptr), k, g["lmax"], _p(b, _dptr), _p(d, _dptr),
                                             _p(nv, _dptr), int(band), _p(M, _dptr))
    if triples < 0:
        raise ValueError("not a band of the grid")
    return M, int(triples)


def trisolve(L: np.ndarray, b: np.ndarray, trans: bool = False) -> np.ndarray:
    """Solve L y = b (or L^T y = b) by substitution."""
    L = _f64(L)
    bb = _f64(b)
    y = np.zeros_like(bb)
    rc = lib().sympix_oracle_trisolve(L.shape[0], _p(L, _dptr), _p(bb, _dptr), 1 if trans else 0, _p(y, _dptr))
    if rc != 0:
        raise ValueError(f"zero diagonal at row {rc - 1}")
    return y


def convolve(g: dict, bl: np.ndarray, r_s: float, f: np.ndarray, q_ring, q_col):
    """Pixel-domain convolution g_q = sum_p b(n_q . n_p) f_p over the pixels
    within r_s (Eq. convolution-pixel), at the pixels (q_ring[i], q_col[i]);
    returns (g, number of coupled pairs summed)."""
    qr = np.ascontiguousarray(q_ring, dtype=np.int32)
    qc = np.ascontiguousarray(q_col, dtype=np.int32)
    out = np.zeros(len(qr))
    th = _f64(g["theta"])
    nr = np.ascontiguousarray(g["nring"], dtype=np.int32)
    off = np.ascontiguousarray(g["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g["ring_stride"], dtype=np.int32)
    b = _f64(bl)
    fv = _f64(f)
    assert len(fv) == g["npix"]
    pairs = lib().sympix_oracle_convolve(g["nrings"], _p(th, _dptr), _p(nr, _i32ptr), _p(off, _i64ptr),
                                         _p(st, _i32ptr), g["lmax"], _p(b, _dptr), float(r_s), _p(fv, _dptr),
                                         len(qr), _p(qr, _i32ptr), _p(qc, _i32ptr), _p(out, _dptr))
    return out, int(pairs)


def cholesky(A: np.ndarray):
    """Lower Cholesky factor and LAPACK-style info (0, or first bad row + 1)."""
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros_like(A)
    info = lib().sympix_oracle_cholesky(n, _p(A, _dptr), _p(L, _dptr))
    return L, int(info)


# -- Y2 != Y1 (Sec. 4.2, Eq. substitution, Eq. degrade) --------------------------

def degrade(lmax2: int, obs_theta, obs_phi, obs_val, g2: dict) -> np.ndarray:
    """Eq. degrade: theta_2 = W_2 Y_2 Y_obs^T theta on grid g2 (its pixel numbering),
    Y_obs^T the unweighted adjoint synthesis at the observation points, lmax2 the
    band limit of Y_2, W_2 the quadrature weights of g2 (ring weight x 2 pi / n)."""
    th, ph, v = _f64(obs_theta), _f64(obs_phi), _f64(obs_val)
    assert th.shape == ph.shape == v.shape
    t2 = _f64(g2["theta"])
    nr = np.ascontiguousarray(g2["nring"], dtype=np.int32)
    w = _f64(g2["weight"]) if "weight" in g2 else gl_weights(t2)
    off = np.ascontiguousarray(g2["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g2["ring_stride"], dtype=np.int32)
    out = np.zeros(int(g2["npix"]), dtype=np.float64)
    n = lib().sympix_oracle_degrade(int(lmax2), len(v), _p(th, _dptr), _p(ph, _dptr), _p(v, _dptr), int(g2["nrings"]),
                                    _p(t2, _dptr), _p(nr, _i32ptr), _p(w, _dptr), _p(off, _i64ptr), _p(st, _i32ptr),
                                    _p(out, _dptr))
    assert n == int(nr.sum())
    return out


def block_y2(g1: dict, j: int, g2: dict, bl, dl, r_s: float, ninv2):
    """Block of ring j of grid g1 with B^ = Y_2 B Y_1^T: the noise ninv2 lives on the
    pixels of grid g2.  Returns (dense block, triples summed)."""
    n = int(g1["nring"][j])
    M = np.zeros((n, n), dtype=np.float64)
    t1 = _f64(g1["theta"])
    n1 = np.ascontiguousarray(g1["nring"], dtype=np.int32)
    t2 = _f64(g2["theta"])
    n2 = np.ascontiguousarray(g2["nring"], dtype=np.int32)
    off = np.ascontiguousarray(g2["ring_offset"], dtype=np.int64)
    st = np.ascontiguousarray(g2["ring_stride"], dtype=np.int32)
    b, d, nv = _f64(bl), _f64(dl), _f64(ninv2)
    assert len(nv) == int(g2["npix"]) and len(b) == len(d)
    tr = lib().sympix_oracle_block_y2(_p(t1, _dptr), _p(n1, _i32ptr), int(j), int(g2["nrings"]), _p(t2, _dptr),
                                      _p(n2, _i32ptr), _p(off, _i64ptr), _p(st, _i32ptr), len(b) - 1, _p(b, _dptr),
                                      _p(d, _dptr), float(r_s), _p(nv, _dptr), _p(M, _dptr))
    return M, int(tr)


def gl_grid(nrings: int, n: int) -> dict:
    """A Gauss-Legendre grid with the same count n on every ring, numbered ring by
    ring (a quadrature that is exact for band limit 2 nrings - 1 in cos theta and
    n - 1 in longitude): the exact auxiliary grid for Eq. degrade."""
    theta = gl_theta(nrings)
    nring = np.full(nrings, n, dtype=np.int32)
    return dict(lmax=None, k=1, nrings=nrings, theta=theta, nring=nring, weight=gl_weights(theta),
                ring_offset=np.arange(nrings, dtype=np.int64) * n, ring_stride=np.ones(nrings, dtype=np.int32),
                npix=nrings * n)
