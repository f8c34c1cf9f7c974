"""Seeded synthetic inputs for the SymPix preconditioner-block workloads.

This module holds input generation only: beam and prior transfer functions,
the support radius of the truncated kernels and the inverse-noise map.  It
contains none of the method's arithmetic (no grid, kernel, block or factor
computation), so both the CUDA path and the oracle can be fed from it.

The paper measured on Planck-like noise maps and a HEALPix N_side = 2048 mask
(Sec. 4.2), which are not available here; the maps below stand in for them
with the same structure: a smooth Gaussian beam b_l, a steep prior d_l, and a
lognormal inverse-variance map with a masked band around the galactic plane.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)


def fwhm_to_sigma(fwhm_arcmin: float) -> float:
    """Gaussian beam width in radians from its full width at half maximum."""
    return fwhm_arcmin * ARCMIN / math.sqrt(8.0 * math.log(2.0))


def gaussian_beam(lmax: int, fwhm_arcmin: float) -> np.ndarray:
    """b_l = exp(-l (l+1) sigma^2 / 2), l = 0..lmax."""
    s = fwhm_to_sigma(fwhm_arcmin)
    ell = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * ell * (ell + 1.0) * s * s)


def prior(lmax: int) -> np.ndarray:
    """d_l = (l (l+1))^2 / (lmax (lmax+1))^2, l = 0..lmax."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    return (ell * (ell + 1.0)) ** 2 / (float(lmax) * (lmax + 1.0)) ** 2


def support_radius(fwhm_arcmin: float, floor: float = 1e-10) -> float:
    """Radius where the Gaussian envelope exp(-g^2 / 2 sigma^2) falls to `floor`."""
    return fwhm_to_sigma(fwhm_arcmin) * math.sqrt(2.0 * math.log(1.0 / floor))


def pixel_colatitude(theta: np.ndarray, nring: np.ndarray, ring_offset: np.ndarray,
                     ring_stride: np.ndarray, npix: int) -> np.ndarray:
    """Colatitude of every pixel, indexed by the grid's pixel numbering."""
    out = np.empty(npix, dtype=np.float64)
    for j in range(len(theta)):
        idx = int(ring_offset[j]) + int(ring_stride[j]) * np.arange(int(nring[j]))
        out[idx] = theta[j]
    return out


def ninv_map(seed: int, colat: np.ndarray, band_deg: float = 20.0,
             sigma: float = 0.3) -> np.ndarray:
    """N^-1_p = exp(sigma z_p), z_p ~ N(0, 1) white, zero where |latitude| < band_deg."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(colat.shape[0])
    m = np.exp(sigma * z)
    lat = np.abs(0.5 * math.pi - colat)
    m[lat < band_deg * math.pi / 180.0] = 0.0
    return m


@dataclass
class Workload:
    """One named workload: grid size, beam, prior and map recipe."""
    name: str
    lmax: int
    fwhm_arcmin: list
    band_deg: list
    seeds: list
    desc: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nops(self) -> int:
        return len(self.fwhm_arcmin)

    def beams(self) -> np.ndarray:
        return np.stack([gaussian_beam(self.lmax, f) for f in self.fwhm_arcmin])

    def priors(self) -> np.ndarray:
        return np.stack([prior(self.lmax) for _ in self.fwhm_arcmin])

    def radii(self) -> np.ndarray:
        return np.array([support_radius(f) for f in self.fwhm_arcmin], dtype=np.float64)

    def ninv(self, colat: np.ndarray) -> np.ndarray:
        return np.stack([ninv_map(s, colat, b) for s, b in zip(self.seeds, self.band_deg)])


def _batched(lmax: int = 1000, nops: int = 32, seed: int = 5) -> Workload:
    rng = np.random.default_rng(seed)
    fwhm = rng.uniform(10.0, 60.0, nops).tolist()
    band = rng.uniform(0.0, 30.0, nops).tolist()
    return Workload(f"batched_{nops}ops_lmax{lmax}", lmax, fwhm, band,
                    list(range(100, 100 + nops)),
                    f"{nops} operators, l_max={lmax}, FWHM U[10',60'], mask band U[0,30] deg")


WORKLOADS = {
    "lmax64": Workload("lmax64_fwhm180", 64, [180.0], [20.0], [1],
                       "l_max=64, FWHM 180', 20 deg masked band"),
    "lmax500": Workload("lmax500_fwhm30", 500, [30.0], [20.0], [2],
                        "l_max=500, FWHM 30', 20 deg masked band"),
    "lmax1500": Workload("lmax1500_fwhm10", 1500, [10.0], [20.0], [3],
                         "l_max=1500, FWHM 10', 20 deg masked band"),
    "lmax3000": Workload("lmax3000_fwhm5", 3000, [5.0], [20.0], [4],
                         "l_max=3000, FWHM 5', 20 deg masked band"),
    "batched32": _batched(),
}
