"""Why the B^T N^-1 B^ contraction stays on the FP32 SIMT pipes: the multiply-adds
a dense tile product would do, against the sparse triples the sum needs (Eq.
`Dhat`, Sec. 4.2), from the oracle's own support geometry (CPU only).

A tensor-core form of one block tile would gather every pixel p coupled to one
of 64 consecutive columns q of ring j (the K dimension), and multiply the
gathered B^ rows of those columns by the B^ rows of the band columns
r = q - w .. q (N = 64 + w outputs per row).  The sum itself needs one
multiply-add per (q, r, p) with p coupled to both q and r."""
import numpy as np

from oracle import oracle as O
from paper_1504_04653_gb300 import workloads as W

def _tile_work(g, j, r_s, q0=0, T=64):
    th, nr = g["theta"], g["nring"]
    rings = [rho for rho in range(g["nrings"]) if abs(th[rho] - th[j]) <= r_s]
    cache = {}

    def sup(x):
        x %= int(nr[j])
        if x not in cache:
            cache[x] = {(rho, int(p)) for rho in rings for p in O.coupled(g, j, x, rho, r_s)}
        return cache[x]

    w = 0  # the block's band half-width: the largest offset whose supports meet
    while w < nr[j] // 2 and sup(q0) & sup(q0 - w - 1):
        w += 1
    cols = range(q0, q0 + T)
    P = set().union(*[sup(q) for q in cols])
    triples = sum(len(sup(q) & sup(r)) for q in cols for r in range(q - w, q + 1))
    dense = len(P) * T * (T + w)
    return w, triples, dense


def test_dense_tile_product_waste_on_wide_beams():
    """For the widest beam of the 32-operator workload (FWHM 60', band
    half-width ~32) a 64-row dense tile does 20x or more the multiply-adds of
    the sparse sum, at the equator and at mid latitude; narrower beams waste
    more.  A split product (bf16x3 or 3xTF32) multiplies that by three."""
    wl = W.WORKLOADS["batched32"]
    radii = wl.radii()
    g = O.grid(wl.lmax)
    o_wide, o_mid = int(np.argmax(radii)), int(np.argsort(radii)[len(radii) // 2])
    ratios = {}
    for o in (o_wide, o_mid):
        for j in (g["nrings"] // 2, g["nrings"] // 4):
            w, triples, dense = _tile_work(g, j, float(radii[o]))
            assert triples > 0 and w >= 8
            ratios[(o, j)] = dense / triples
    for j in (g["nrings"] // 2, g["nrings"] // 4):
        assert ratios[(o_wide, j)] >= 18.0, ratios
        assert ratios[(o_mid, j)] > ratios[(o_wide, j)], ratios
