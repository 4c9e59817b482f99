"""Seeded synthetic galaxy catalogs shaped like the survey mocks of the multipole 3PCF estimator.

This module only draws inputs. It holds none of the estimator's arithmetic, so both the CUDA
library's tests/bench and the FP64 oracle's tests take their catalogs from here.

Catalog model (stand-in for the N-body mocks of Sec. 4 and Sec. 6 of the paper, which are not
available here):

* positions uniform on a flat square patch [0, L)^2 in arcmin, optionally with circular holes;
* shear either pure shape noise, or a lognormal convergence field converted to shear by the
  Kaiser--Squires relation plus shape noise sigma_e per component;
* weights either 1 or U(0.5, 1.5);
* positions are stored as int32 fixed point with a quantum of 2^-13 arcmin, so that pair
  separations are exact integers on every device.

Draw order from one ``numpy.random.default_rng(seed)``: positions, field, noise, weights.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

QUANTUM = 2.0 ** -13  # arcmin per fixed-point unit


@dataclass
class Catalog:
    """A flat-sky shear catalog in the library's input format (structure of arrays)."""

    xq: np.ndarray  # int32 fixed-point x (units of ``quantum`` arcmin)
    yq: np.ndarray  # int32 fixed-point y
    g1: np.ndarray  # float32 shear/ellipticity component 1
    g2: np.ndarray  # float32 component 2
    w: np.ndarray  # float32 weight
    zbin: Optional[np.ndarray] = None  # uint8 tomographic bin index, or None
    side: float = 0.0  # patch side in arcmin
    quantum: float = QUANTUM
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xq.shape[0])

    def subset(self, idx: np.ndarray) -> "Catalog":
        idx = np.asarray(idx)
        return Catalog(self.xq[idx].copy(), self.yq[idx].copy(), self.g1[idx].copy(),
                       self.g2[idx].copy(), self.w[idx].copy(),
                       None if self.zbin is None else self.zbin[idx].copy(),
                       self.side, self.quantum, dict(self.meta))


def quantise(x_arcmin: np.ndarray, quantum: float = QUANTUM) -> np.ndarray:
    q = np.floor(np.asarray(x_arcmin, dtype=np.float64) / quantum)
    if q.size and (q.min() < 0 or q.max() >= 2 ** 31 - 1):
        raise ValueError("position outside the int32 fixed-point range")
    return q.astype(np.int32)


def _fft_freqs(ngrid: int):
    k = np.fft.fftfreq(ngrid)
    return k[:, None], k[None, :]


def lognormal_shear_grid(ngrid: int, rng: np.random.Generator, slope: float = -1.5,
                         sigma_g2: float = 1.0, shift: float = 0.02):
    """Periodic lognormal convergence grid and its Kaiser--Squires shear.

    A Gaussian field g with power spectrum P(k) ~ k^slope (k=0 zeroed) is scaled to variance
    ``sigma_g2``; kappa = shift * (exp(g - sigma_g2/2) - 1); the shear follows from
    gamma_hat = [(k1^2 - k2^2) + 2 i k1 k2] / k^2 * kappa_hat.
    Returns (kappa, gamma1, gamma2) as float32 arrays indexed [iy, ix].
    """
    ky, kx = _fft_freqs(ngrid)
    k2 = kx * kx + ky * ky
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P) with P ~ k^slope
    white = rng.standard_normal((ngrid, ngrid))
    g = np.fft.ifft2(np.fft.fft2(white) * amp).real
    g *= np.sqrt(sigma_g2) / g.std()
    kappa = shift * (np.exp(g - 0.5 * sigma_g2) - 1.0)
    del g, white
    khat = np.fft.fft2(kappa)
    ks = np.zeros(k2.shape, dtype=np.complex128)
    ks[nz] = ((kx * kx - ky * ky) + 2j * kx * ky)[nz] / k2[nz]
    gam = np.fft.ifft2(khat * ks)
    return kappa.astype(np.float32), gam.real.astype(np.float32), gam.imag.astype(np.float32)


def _sample_grid(grid: np.ndarray, x: np.ndarray, y: np.ndarray, side: float) -> np.ndarray:
    n = grid.shape[0]
    ix = np.clip(np.floor(x / side * n).astype(np.int64), 0, n - 1)
    iy = np.clip(np.floor(y / side * n).astype(np.int64), 0, n - 1)
    return grid[iy, ix]


def hole_mask(side: float, rng: np.random.Generator, rmin: float = 2.0, rmax: float = 10.0,
              frac: float = 0.15, raster: float = 0.1):
    """Circular holes with uniform centres and radii U(rmin, rmax), added until the masked area
    measured on a ``raster``-arcmin grid reaches ``frac``. Returns (cx, cy, r) arrays."""
    n = int(round(side / raster))
    masked = np.zeros((n, n), dtype=bool)
    cs = (np.arange(n) + 0.5) * raster
    cx, cy, rr = [], [], []
    while masked.mean() < frac:
        x0, y0 = rng.uniform(0, side, 2)
        r = rng.uniform(rmin, rmax)
        i0, i1 = max(0, int((y0 - r) / raster)), min(n, int((y0 + r) / raster) + 2)
        j0, j1 = max(0, int((x0 - r) / raster)), min(n, int((x0 + r) / raster) + 2)
        yy = cs[i0:i1, None] - y0
        xx = cs[None, j0:j1] - x0
        masked[i0:i1, j0:j1] |= (xx * xx + yy * yy) < r * r
        cx.append(x0), cy.append(y0), rr.append(r)
    return np.array(cx), np.array(cy), np.array(rr), float(masked.mean())


def _in_holes(x, y, holes):
    cx, cy, rr = holes[:3]
    bad = np.zeros(x.shape, dtype=bool)
    for a, b, r in zip(cx, cy, rr):
        sel = (np.abs(x - a) < r) & (np.abs(y - b) < r)
        if sel.any():
            bad[sel] |= (x[sel] - a) ** 2 + (y[sel] - b) ** 2 < r * r
    return bad


def uniform_positions(n: int, side: float, rng: np.random.Generator, holes=None):
    if holes is None:
        return rng.uniform(0, side, n), rng.uniform(0, side, n)
    xs, ys, have = [], [], 0
    while have < n:
        m = int((n - have) * 1.3) + 16
        x = rng.uniform(0, side, m)
        y = rng.uniform(0, side, m)
        keep = ~_in_holes(x, y, holes)
        xs.append(x[keep]), ys.append(y[keep])
        have += int(keep.sum())
    return np.concatenate(xs)[:n], np.concatenate(ys)[:n]


def make_catalog(n: int, side: float, seed: int, *, field: str = "noise", sigma_e: float = 0.26,
                 weights: str = "unit", ngrid: int = 4096, holes: bool = False,
                 amplitude: float = 1.0, quantum: float = QUANTUM, slope: float = -1.5) -> Catalog:
    """One catalog. ``field`` is "noise" (pure shape noise) or "lognormal" (lognormal
    Kaiser--Squires shear + noise, the Gaussian field's P(k) ~ k^slope); ``weights`` is "unit" or
    "uniform" (U(0.5, 1.5))."""
    rng = np.random.default_rng(seed)
    hl = hole_mask(side, rng) if holes else None
    x, y = uniform_positions(n, side, rng, hl)
    g1 = np.zeros(n)
    g2 = np.zeros(n)
    meta = {"field": field, "seed": seed}
    if field == "lognormal":
        _, s1, s2 = lognormal_shear_grid(ngrid, rng, slope=slope)
        g1 += amplitude * _sample_grid(s1, x, y, side)
        g2 += amplitude * _sample_grid(s2, x, y, side)
        meta["ngrid"] = ngrid
    elif field != "noise":
        raise ValueError(field)
    if sigma_e > 0:
        g1 += rng.normal(0.0, sigma_e, n)
        g2 += rng.normal(0.0, sigma_e, n)
    if weights == "unit":
        w = np.ones(n)
    elif weights == "uniform":
        w = rng.uniform(0.5, 1.5, n)
    else:
        raise ValueError(weights)
    if hl is not None:
        meta["masked_fraction"] = hl[3]
    return Catalog(quantise(x, quantum), quantise(y, quantum), g1.astype(np.float32),
                   g2.astype(np.float32), w.astype(np.float32), None, side, quantum, meta)


def make_tomographic_catalog(seed: int, side: float = 300.0, n_z: int = 5,
                             n_range: Sequence[int] = (50_000, 400_000), ngrid: int = 4096,
                             sigma_e: float = 0.26, amp_step: float = 0.2,
                             quantum: float = QUANTUM) -> Catalog:
    """One tomographic realisation: one lognormal field; bin Z (1-based) carries amplitude
    ``amp_step * Z`` times that field; positions and noise are drawn independently per bin."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(n_range[0], n_range[1] + 1, n_z)
    pos = [uniform_positions(int(c), side, rng) for c in counts]
    _, s1, s2 = lognormal_shear_grid(ngrid, rng)
    xs, ys, g1s, g2s, ws, zs = [], [], [], [], [], []
    for z, (x, y) in enumerate(pos):
        a = amp_step * (z + 1)
        c = x.shape[0]
        g1 = a * _sample_grid(s1, x, y, side) + rng.normal(0.0, sigma_e, c)
        g2 = a * _sample_grid(s2, x, y, side) + rng.normal(0.0, sigma_e, c)
        xs.append(x), ys.append(y), g1s.append(g1), g2s.append(g2)
        zs.append(np.full(c, z, dtype=np.uint8))
    for z in range(n_z):
        ws.append(rng.uniform(0.5, 1.5, counts[z]))
    return Catalog(quantise(np.concatenate(xs), quantum), quantise(np.concatenate(ys), quantum),
                   np.concatenate(g1s).astype(np.float32), np.concatenate(g2s).astype(np.float32),
                   np.concatenate(ws).astype(np.float32), np.concatenate(zs), side, quantum,
                   {"field": "lognormal", "seed": seed, "counts": counts.tolist()})


# The measurement setups of the paper's workloads, as parameters (bins in arcmin).
WORKLOADS = {
    "uniform_noise_2k": dict(n=2000, side=60.0, field="noise", weights="unit", seed=0,
                             n_bins=10, theta_min=0.5, theta_max=30.0, n_max=10,
                             theta_ap=[2.0, 4.0, 8.0]),
    "lognormal_200k": dict(n=200_000, side=300.0, field="lognormal", weights="uniform", seed=1,
                           n_bins=20, theta_min=0.5, theta_max=120.0, n_max=30,
                           theta_ap=[2.0, 4.0, 8.0, 16.0]),
    "masked_lognormal_1m": dict(n=1_000_000, side=600.0, field="lognormal", weights="uniform",
                                seed=2, holes=True, n_bins=30, theta_min=0.5, theta_max=240.0,
                                n_max=40, theta_ap=[2.0, 4.0, 8.0, 16.0]),
    "tomo_64x5_lognormal": dict(side=300.0, n_z=5, realisations=64, n_bins=20, theta_min=0.5,
                                theta_max=120.0, n_max=30, theta_ap=[2.0, 4.0, 8.0, 16.0]),
    "grad_lognormal_500k": dict(n=500_000, side=420.0, field="lognormal", weights="uniform",
                                seed=4, n_bins=20, theta_min=0.5, theta_max=120.0, n_max=30,
                                theta_ap=[4.0, 8.0, 16.0]),
    # the density and binning of the combined estimator's accuracy test (3.1e6 galaxies on
    # 100 deg^2, 33 logarithmic bins 0.25'-80', noise-free) on a tenth of the area
    "multiscale_310k": dict(n=310_000, side=190.0, field="lognormal", weights="uniform", seed=5,
                            sigma_e=0.0, n_bins=33, theta_min=0.25, theta_max=80.0, n_max=30,
                            grid_base_arcmin=0.25, grid_max_arcmin=1.0),
    # the same at the paper's full area (3.1e6 galaxies on 100 deg^2)
    "multiscale_3m": dict(n=3_100_000, side=600.0, field="lognormal", weights="uniform", seed=6,
                          sigma_e=0.0, n_bins=33, theta_min=0.25, theta_max=80.0, n_max=30,
                          grid_base_arcmin=0.25, grid_max_arcmin=1.0),
    # the same with a redder Gaussian field (P(k) ~ k^-3: less power at the pixel scales)
    "multiscale_3m_smooth": dict(n=3_100_000, side=600.0, field="lognormal", weights="uniform", seed=6,
                                 sigma_e=0.0, n_bins=33, theta_min=0.25, theta_max=80.0, n_max=30,
                                 grid_base_arcmin=0.25, grid_max_arcmin=1.0, slope=-3.0),
}


def grid_levels(edges, base_q: int, quantum: float, ratio: float = 20.0, max_q: Optional[int] = None):
    """The combined estimator's levels (b_start, pixel_q) for bin edges (arcmin), as in the
    paper's accuracy test of it (ratio 20): pixels of side Delta (base_q quanta first) for the
    bins with ratio Delta <= lower edge < 2 ratio Delta, then 2 Delta, and so on, up to pixels of
    max_q quanta (that test stops at 1'; None: no limit); the bins below ratio base_q stay
    discrete."""
    levels = []
    d = int(base_q)
    for b in range(len(edges) - 1):
        lo = float(edges[b]) / quantum
        if lo < ratio * base_q:
            continue
        while lo >= 2 * ratio * d and (max_q is None or 2 * d <= max_q):
            d *= 2
        if not levels or levels[-1][1] != d:
            levels.append((b, d))
    return levels


def workload_catalog(name: str, ngrid: int = 4096, n: Optional[int] = None) -> Catalog:
    p = WORKLOADS[name]
    return make_catalog(n if n is not None else p["n"], p["side"], p["seed"], field=p["field"],
                        weights=p["weights"], ngrid=ngrid, holes=p.get("holes", False),
                        sigma_e=p.get("sigma_e", 0.26), slope=p.get("slope", -1.5))
