"""ctypes binding of libsympix (C ABI in include/sympix.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names (``sympix_grid``, ``sympix_support``,
``sympix_kernel_table``, ``sympix_sample_blocks``, ``sympix_factor_blocks``);
device buffers are torch CUDA tensors and streams are torch streams.  If the
library is not built or no GPU is usable the calls raise; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libsympix.so"

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, 1, 2, 3, 4, 5
OPT_FP32_PIVOT_FLOOR, OPT_TRACE, OPT_TABLE_CTA, OPT_BORDER_THREADS, OPT_WAIT_LIMIT = 1, 2, 3, 4, 5
OPT_NARROW_FACTOR = 6
LAYOUT_GREEDY, LAYOUT_DP = 0, 1
PREC_FP64, PREC_FP32, PREC_FP32X2 = 0, 1, 2
STORE_PBAND, STORE_DENSE = 0, 1
STAGE_TABLE, STAGE_SAMPLE, STAGE_FACTOR, STAGE_ALL = 1, 2, 4, 7
BLOCK_PBAND, BLOCK_DENSE = 0, 1

PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "fp32x2": PREC_FP32X2}
STORAGES = {"pband": STORE_PBAND, "dense": STORE_DENSE}


class SympixError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sympix error {code}: {msg}")
        self.code = code


class _GridDesc(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("k", ctypes.c_int), ("layout", ctypes.c_int),
                ("nrings", ctypes.c_int), ("nbands", ctypes.c_int), ("max_ring", ctypes.c_int),
                ("npix", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)
_sizep = ctypes.POINTER(ctypes.c_size_t)

# (name, restype, argtypes) of every exported symbol declared in sympix.h
SIGNATURES = [
    ("sympix_grid", _i, [_i, _i, _i, ctypes.c_double, ctypes.POINTER(_vp)]),
    ("sympix_grid_describe", _i, [_vp, ctypes.POINTER(_GridDesc)]),
    ("sympix_grid_copy", _i, [_vp, _dp, _i32p, _i64p, _i32p]),
    ("sympix_grid_free", None, [_vp]),
    ("sympix_support", _i, [_vp, _i, _dp, _i, _i, ctypes.POINTER(_vp)]),
    ("sympix_plan_option", _i, [_vp, _i, ctypes.c_double]),
    ("sympix_plan_counts", _i, [_vp, _i64p, _i64p, _i64p, _i64p]),
    ("sympix_plan_launches", _i, [_vp, _i, _i, _i, _i32p, _i32p, _i32p]),
    ("sympix_blocks_size", _i, [_vp, _i, _sizep, _i64p]),
    ("sympix_block_layout", _i, [_vp, _i, _i, _i, _i64p, _i32p, _i32p, _i32p]),
    ("sympix_support_copy", _i, [_vp, _i, _i, _i, _i32p]),
    ("sympix_plan_radius", _i, [_vp, _i, _dp, _dp]),
    ("sympix_plan_status", _i, [_vp, _vp]),
    ("sympix_plan_device_bytes", _i, [_vp, _sizep, _sizep]),
    ("sympix_kernel_table", _i, [_vp, _vp, _vp, _vp]),
    ("sympix_kernel_table_static", _i, [_vp, _vp, _vp, _vp]),
    ("sympix_table_copy", _i, [_vp, _i, _i, _i, _i, _dp, _dp]),
    ("sympix_sample_blocks", _i, [_vp, _vp, _i, _i, _vp, _vp]),
    ("sympix_factor_blocks", _i, [_vp, _i, _i, _vp, _vp, _vp]),
    ("sympix_autotune", _i, [_vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, _vp]),
    ("sympix_plan_tuning", _i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    ("sympix_trace_read", _i, [_vp, _i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float), _i32p]),
    ("sympix_convolve", _i, [_vp, _vp, _i, _vp, _vp]),
    ("sympix_coupling_size", _i, [_vp, _i, _sizep, _i64p]),
    ("sympix_coupling_layout", _i, [_vp, _i, _i, _i, _i64p, _i32p]),
    ("sympix_sample_coupling", _i, [_vp, _vp, _i, _vp, _vp]),
    ("sympix_apply", _i, [_vp, _i, _vp, _vp, _vp, _vp, _vp]),
    ("sympix_plan_free", None, [_vp]),
    ("sympix_step_create", _i, [_vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp, ctypes.POINTER(_vp)]),
    ("sympix_step_launch", _i, [_vp, _i, _vp]),
    ("sympix_step_kernels", _i, [_vp, _i, _i64p]),
    ("sympix_step_free", None, [_vp]),
    ("sympix_last_error", ctypes.c_char_p, []),
    ("sympix_version", ctypes.c_char_p, []),
]

_lib = None


def lib():
    """Load libsympix.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise SympixError(ECUDA, f"{LIB_PATH.name} is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise SympixError(rc, lib().sympix_last_error().decode())


def _ptr(t):
    """Device pointer of a contiguous torch CUDA tensor."""
    if not t.is_cuda:
        raise SympixError(EINVAL, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise SympixError(EINVAL, "expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# -- handles ------------------------------------------------------------------------

class Grid:
    """A SymPix grid (sympix_grid)."""

    def __init__(self, lmax: int, k: int = 1, layout: str = "greedy", polar_thr: float = -1.0):
        h = _vp()
        lay = {"greedy": LAYOUT_GREEDY, "dp": LAYOUT_DP}[layout]
        _check(lib().sympix_grid(int(lmax), int(k), lay, float(polar_thr), ctypes.byref(h)))
        self._h = h
        d = _GridDesc()
        _check(lib().sympix_grid_describe(h, ctypes.byref(d)))
        self.lmax, self.k, self.nrings, self.nbands = d.lmax, d.k, d.nrings, d.nbands
        self.max_ring, self.npix = d.max_ring, d.npix
        N = d.nrings
        self.theta = np.zeros(N)
        self.nring = np.zeros(N, np.int32)
        self.ring_offset = np.zeros(N, np.int64)
        self.ring_stride = np.zeros(N, np.int32)
        _check(lib().sympix_grid_copy(h, self.theta.ctypes.data_as(_dp), self.nring.ctypes.data_as(_i32p),
                                      self.ring_offset.ctypes.data_as(_i64p),
                                      self.ring_stride.ctypes.data_as(_i32p)))

    @property
    def handle(self):
        return self._h

    def as_dict(self) -> dict:
        return dict(lmax=self.lmax, k=self.k, nrings=self.nrings, theta=self.theta, nring=self.nring,
                    ring_offset=self.ring_offset, ring_stride=self.ring_stride, npix=int(self.npix))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sympix_grid_free(h)
            self._h = None


class Plan:
    """Support, classes and block layout of nops operators (sympix_support)."""

    def __init__(self, grid: Grid, r_s, ring0: int = 0, ring1: int | None = None):
        r = np.ascontiguousarray(np.atleast_1d(r_s), dtype=np.float64)
        self.grid = grid
        self.nops = len(r)
        self.ring0 = int(ring0)
        self.ring1 = grid.nrings if ring1 is None else int(ring1)
        h = _vp()
        _check(lib().sympix_support(grid.handle, self.nops, r.ctypes.data_as(_dp), self.ring0, self.ring1,
                                    ctypes.byref(h)))
        self._h = h
        ns, npairs, nt, nm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().sympix_plan_counts(h, ctypes.byref(ns), ctypes.byref(npairs), ctypes.byref(nt),
                                        ctypes.byref(nm)))
        self.nslots, self.npairs, self.ntriples, self.nmults = ns.value, npairs.value, nt.value, nm.value

    @property
    def handle(self):
        return self._h

    @property
    def nblocks(self) -> int:
        """Blocks per storage: one per (operator, ring), or on a DP grid with
        k > 1 one per (operator, band of k rings)."""
        return self.nops * (self.ring1 - self.ring0) // self.k

    @property
    def k(self) -> int:
        return self.grid.k

    def blocks_size(self, storage="pband"):
        b, e = ctypes.c_size_t(), ctypes.c_int64()
        _check(lib().sympix_blocks_size(self._h, STORAGES[storage], ctypes.byref(b), ctypes.byref(e)))
        return b.value, e.value

    def block_layout(self, storage, op, ring):
        off, n, w, fmt = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sympix_block_layout(self._h, STORAGES[storage], int(op), int(ring), ctypes.byref(off),
                                         ctypes.byref(n), ctypes.byref(w), ctypes.byref(fmt)))
        return off.value, n.value, w.value, fmt.value

    def set_pivot_floor(self, value: float):
        """FP32 factor: blocks whose pivots shrink below value x diagonal go to FP64."""
        _check(lib().sympix_plan_option(self._h, OPT_FP32_PIVOT_FLOOR, float(value)))

    def set_launch_shape(self, table_cta=None, border_threads=None):
        """Launch shapes: table CTA size (32, 64, 128), FP32 border-pass threads (256, 512)."""
        if table_cta is not None:
            _check(lib().sympix_plan_option(self._h, OPT_TABLE_CTA, float(table_cta)))
        if border_threads is not None:
            _check(lib().sympix_plan_option(self._h, OPT_BORDER_THREADS, float(border_threads)))

    def tuning(self):
        """(table CTA size, border-pass threads) the plan launches with."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().sympix_plan_tuning(self._h, ctypes.byref(a), ctypes.byref(b), None))
        return a.value, b.value

    def narrow_kernels(self):
        """{arithmetic: 0 (G-lane), 1 (earlier kernels), 2 (FP32 chunked border) or 3 (FP32 split CTAs)}."""
        nk = (ctypes.c_int * 3)()
        _check(lib().sympix_plan_tuning(self._h, None, None, nk))
        return {"fp64": nk[0], "fp32": nk[1], "fp32x2": nk[2]}

    def autotune(self, bl, dl, ninv, blocks, info, storage="pband", sample_precision="fp32",
                 factor_precision="fp32", stream=None):
        """Time the launch-shape candidates on these buffers and keep the fastest."""
        _check(lib().sympix_autotune(self._h, _ptr(bl), _ptr(dl), _ptr(ninv), STORAGES[storage],
                                     PRECISIONS[sample_precision], PRECISIONS[factor_precision], _ptr(blocks),
                                     _ptr(info), _stream(stream)))
        return self.tuning()

    def set_narrow_factor(self, kernel: int):
        """w <= 12 bands: 0 the G-lane kernel, 1 the earlier kernels, 2 (every arithmetic) the band
        pass and the border rows by column chunks, 3 (FP32; the others as 2) band and border passes in
        two CTAs of one cooperative launch, -1 per arithmetic (default)."""
        _check(lib().sympix_plan_option(self._h, OPT_NARROW_FACTOR, float(kernel)))

    def set_wait_limit(self, polls: int):
        """Polls of a bounded device wait (the FP32 factor's border warps)."""
        _check(lib().sympix_plan_option(self._h, OPT_WAIT_LIMIT, float(polls)))

    def status(self, stream=None):
        """Raise SympixError(ETIMEOUT) if a bounded device wait ran out since the last call."""
        _check(lib().sympix_plan_status(self._h, _stream(stream)))

    def set_trace(self, on: bool):
        """Record a CUDA event after every kernel launch of direct calls."""
        _check(lib().sympix_plan_option(self._h, OPT_TRACE, 1.0 if on else 0.0))

    def trace_read(self):
        """[(kernel name, ms), ...] of the traced launches since the last read."""
        cap = 256
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_float * cap)()
        cnt = ctypes.c_int32()
        _check(lib().sympix_trace_read(self._h, cap, names, ms, ctypes.byref(cnt)))
        return [(names[i].decode(), float(ms[i])) for i in range(min(cnt.value, cap))]

    def launches(self, storage="pband", sample_precision="fp32", factor_precision="fp32"):
        """Kernel launches of (kernel_table, sample_blocks, factor_blocks)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sympix_plan_launches(self._h, STORAGES[storage], PRECISIONS[sample_precision],
                                          PRECISIONS[factor_precision], ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c)))
        return a.value, b.value, c.value

    def radius(self, op=0):
        """(support radius used, smallest relative margin |u - u_s| / u_s)."""
        r, m = ctypes.c_double(), ctypes.c_double()
        _check(lib().sympix_plan_radius(self._h, int(op), ctypes.byref(r), ctypes.byref(m)))
        return r.value, m.value

    def device_bytes(self):
        """(device bytes the plan holds, of which the table's coefficient staging)."""
        b, st = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().sympix_plan_device_bytes(self._h, ctypes.byref(b), ctypes.byref(st)))
        return b.value, st.value

    def coupling_size(self, delta=1):
        """(bytes, elements) of the blocks between rings j and j + delta."""
        b, e = ctypes.c_size_t(), ctypes.c_int64()
        _check(lib().sympix_coupling_size(self._h, int(delta), ctypes.byref(b), ctypes.byref(e)))
        return b.value, e.value

    def coupling_layout(self, delta, op, ring):
        """(offset, rows, cols, K, zmax, P, Q, dense) of the block (op, ring) -> (op, ring + delta)."""
        off = ctypes.c_int64()
        geom = (ctypes.c_int32 * 7)()
        _check(lib().sympix_coupling_layout(self._h, int(delta), int(op), int(ring), ctypes.byref(off), geom))
        return (off.value, *list(geom))

    def support(self, op, ring, radius):
        out = np.zeros(2 * radius + 1, np.int32)
        _check(lib().sympix_support_copy(self._h, int(op), int(ring), int(radius), out.ctypes.data_as(_i32p)))
        return out

    def table(self, op, ring, rho, count):
        b = np.zeros(count)
        d = np.zeros(count)
        _check(lib().sympix_table_copy(self._h, int(op), int(ring), int(rho), int(count), b.ctypes.data_as(_dp),
                                       d.ctypes.data_as(_dp) if rho == ring else None))
        return b, (d if rho == ring else None)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sympix_plan_free(h)
            self._h = None


# -- the C entry points under their own names ----------------------------------------

def sympix_grid(lmax, k=1, layout="greedy", polar_thr=-1.0) -> Grid:
    return Grid(lmax, k, layout, polar_thr)


def sympix_support(grid: Grid, r_s, ring0=0, ring1=None) -> Plan:
    return Plan(grid, r_s, ring0, ring1)


def sympix_kernel_table(plan: Plan, bl, dl, stream=None):
    """bl, dl: CUDA float64 tensors [nops, lmax+1]."""
    L1 = plan.grid.lmax + 1
    for t in (bl, dl):
        if t.dtype.itemsize != 8 or tuple(t.shape) != (plan.nops, L1):
            raise SympixError(EINVAL, f"coefficients must be float64 [{plan.nops}, {L1}]")
    _check(lib().sympix_kernel_table(plan.handle, _ptr(bl), _ptr(dl), _stream(stream)))


def sympix_kernel_table_static(plan: Plan, bl, dl, stream=None):
    """Allocation-free sympix_kernel_table (static device staging array)."""
    L1 = plan.grid.lmax + 1
    for t in (bl, dl):
        if t.dtype.itemsize != 8 or tuple(t.shape) != (plan.nops, L1):
            raise SympixError(EINVAL, f"coefficients must be float64 [{plan.nops}, {L1}]")
    _check(lib().sympix_kernel_table_static(plan.handle, _ptr(bl), _ptr(dl), _stream(stream)))


def sympix_sample_blocks(plan: Plan, ninv, precision="fp64", storage="pband", out=None, stream=None):
    """ninv: CUDA float64 tensor [nops, npix]; returns the blocks buffer."""
    import torch
    if ninv.dtype != torch.float64 or tuple(ninv.shape) != (plan.nops, plan.grid.npix):
        raise SympixError(EINVAL, f"ninv must be float64 [{plan.nops}, {plan.grid.npix}]")
    nbytes, _ = plan.blocks_size(storage)
    if out is None:
        out = torch.empty(nbytes // 8, dtype=torch.float64, device=ninv.device)
    elif out.numel() * out.element_size() < nbytes:
        raise SympixError(EINVAL, "blocks buffer too small")
    _check(lib().sympix_sample_blocks(plan.handle, _ptr(ninv), PRECISIONS[precision], STORAGES[storage],
                                      _ptr(out), _stream(stream)))
    return out


def sympix_factor_blocks(plan: Plan, blocks, storage="pband", precision="fp64", info=None, stream=None):
    import torch
    if info is None:
        info = torch.empty(plan.nblocks, dtype=torch.int32, device=blocks.device)
    _check(lib().sympix_factor_blocks(plan.handle, STORAGES[storage], PRECISIONS[precision], _ptr(blocks),
                                      _ptr(info), _stream(stream)))
    return info


class Step:
    """The kernel-table, sampling and factor calls captured as CUDA graphs
    (sympix_step_create); launch() replays them.  The graphs keep the tensors'
    addresses: update bl, dl and ninv in place between launches.  The step
    holds references to every tensor it captured."""

    def __init__(self, plan: Plan, bl, dl, ninv, blocks, info, storage="pband", sample_precision="fp32",
                 factor_precision="fp32"):
        import torch
        L1 = plan.grid.lmax + 1
        for t in (bl, dl):
            if t.dtype != torch.float64 or tuple(t.shape) != (plan.nops, L1):
                raise SympixError(EINVAL, f"coefficients must be float64 [{plan.nops}, {L1}]")
        if ninv.dtype != torch.float64 or tuple(ninv.shape) != (plan.nops, plan.grid.npix):
            raise SympixError(EINVAL, f"ninv must be float64 [{plan.nops}, {plan.grid.npix}]")
        nbytes, _ = plan.blocks_size(storage)
        if blocks.dtype != torch.float64 or blocks.numel() * 8 < nbytes:
            raise SympixError(EINVAL, "blocks buffer too small")
        if info.dtype != torch.int32 or info.numel() < plan.nblocks:
            raise SympixError(EINVAL, f"info must be int32 [{plan.nblocks}]")
        self.plan, self._keep = plan, (bl, dl, ninv, blocks, info)
        h = _vp()
        _check(lib().sympix_step_create(plan.handle, _ptr(bl), _ptr(dl), _ptr(ninv), STORAGES[storage],
                                        PRECISIONS[sample_precision], PRECISIONS[factor_precision], _ptr(blocks),
                                        _ptr(info), ctypes.byref(h)))
        self._h = h

    def launch(self, stages=STAGE_ALL, stream=None):
        _check(lib().sympix_step_launch(self._h, int(stages), _stream(stream)))

    def kernels(self, stages=STAGE_ALL) -> int:
        c = ctypes.c_int64()
        _check(lib().sympix_step_kernels(self._h, int(stages), ctypes.byref(c)))
        return c.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sympix_step_free(h)
            self._h = None


def sympix_step_create(plan: Plan, bl, dl, ninv, blocks, info, storage="pband", sample_precision="fp32",
                       factor_precision="fp32") -> Step:
    return Step(plan, bl, dl, ninv, blocks, info, storage, sample_precision, factor_precision)


def sympix_convolve(plan: Plan, f, precision="fp64", out=None, stream=None):
    """g = B^ f (pixel-domain convolution); f: CUDA float64 [nops, npix]."""
    import torch
    if f.dtype != torch.float64 or tuple(f.shape) != (plan.nops, plan.grid.npix):
        raise SympixError(EINVAL, f"f must be float64 [{plan.nops}, {plan.grid.npix}]")
    if out is None:
        out = torch.zeros_like(f)
    elif out.dtype != torch.float64 or out.numel() < f.numel():
        raise SympixError(EINVAL, "g buffer too small")
    _check(lib().sympix_convolve(plan.handle, _ptr(f), PRECISIONS[precision], _ptr(out), _stream(stream)))
    return out


def sympix_sample_coupling(plan: Plan, ninv, delta=1, out=None, stream=None):
    """Blocks between rings j and j + delta (FP64); returns the buffer."""
    import torch
    if ninv.dtype != torch.float64 or tuple(ninv.shape) != (plan.nops, plan.grid.npix):
        raise SympixError(EINVAL, f"ninv must be float64 [{plan.nops}, {plan.grid.npix}]")
    nbytes, _ = plan.coupling_size(delta)
    if out is None:
        out = torch.empty(max(1, nbytes // 8), dtype=torch.float64, device=ninv.device)
    elif out.numel() * 8 < nbytes:
        raise SympixError(EINVAL, "coupling buffer too small")
    _check(lib().sympix_sample_coupling(plan.handle, _ptr(ninv), int(delta), _ptr(out), _stream(stream)))
    return out


def sympix_apply(plan: Plan, blocks, info, x, storage="pband", out=None, stream=None):
    """y = M^-1 x with the factored diagonal ring blocks (block Jacobi)."""
    import torch
    if x.dtype != torch.float64 or tuple(x.shape) != (plan.nops, plan.grid.npix):
        raise SympixError(EINVAL, f"x must be float64 [{plan.nops}, {plan.grid.npix}]")
    if out is None:
        out = torch.zeros_like(x)
    _check(lib().sympix_apply(plan.handle, STORAGES[storage], _ptr(blocks), _ptr(info), _ptr(x), _ptr(out),
                              _stream(stream)))
    return out


def unpack_coupling(buf: np.ndarray, plan: Plan, delta: int, op: int, ring: int) -> np.ndarray:
    """Dense n_j x n_k block between ring `ring` and ring + delta from a host
    copy of the sympix_sample_coupling buffer."""
    off, nj, nk, K, zmax, P, Q, dense = plan.coupling_layout(delta, op, ring)
    rows = buf[off:off + nj * K].reshape(nj, K)
    M = np.zeros((nj, nk))
    for q in range(nj):
        if dense:
            M[q, :] = rows[q]
            continue
        Z = (2 * q + 1) * Q
        r0 = -((-(Z - zmax - P)) // (2 * P))
        for t in range(K):
            r = r0 + t
            if abs(Z - (2 * r + 1) * P) <= zmax:
                M[q, r % nk] += rows[q, t]
    return M


# -- host-side views of the block buffer (for tests and users) -----------------------

def unpack_block(blocks: np.ndarray, plan: Plan, storage: str, op: int, ring: int,
                 factored: bool = False) -> np.ndarray:
    """Dense n x n matrix of one block from a host copy of the blocks buffer:
    the symmetric M (sampled) or the lower factor L (factored)."""
    off, n, w, fmt = plan.block_layout(storage, op, ring)
    if fmt == BLOCK_DENSE:
        A = blocks[off:off + n * n].reshape(n, n).copy()
        return np.tril(A) if factored else A
    band = blocks[off:off + n * (w + 1)].reshape(n, w + 1)
    M = np.zeros((n, n))
    q = np.arange(n)
    if not factored:
        for d in range(w + 1):
            r = (q - d) % n
            M[q, r] = band[:, d]
            M[r, q] = band[:, d]
        return M
    m = n - w
    for d in range(w + 1):
        rows = q[(q < m) & (q >= d)]
        M[rows, rows - d] = band[rows, d]
    bord = blocks[off + n * (w + 1):off + n * (2 * w + 1)].reshape(w, n)
    for b in range(w):
        i = m + b
        M[i, :i + 1] = bord[b, :i + 1]
    return M


def version() -> str:
    return lib().sympix_version().decode()
