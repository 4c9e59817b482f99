"""ctypes marshalling for the FP64 C oracle (``mp3pcf_oracle.c``). Test infrastructure only.

Most functions here convert numpy arrays to pointers and back, the arithmetic being in the C file;
grid_catalog (per-pixel sums) and combined_moments (a copy of the pixel moments into the grid
bins) are plain numpy steps around the C routines.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp3pcf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, OpenMP over centres)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcCfg(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("theta_min", C.c_double), ("theta_max", C.c_double),
                ("n_max", C.c_int32), ("n_phi", C.c_int32), ("n_z", C.c_int32),
                ("quantum", C.c_double), ("norm_truncate", C.c_int32),
                ("radial_nodes", C.c_int32), ("exclude_degenerate", C.c_int32)]


@dataclass
class Setup:
    """Measurement setup (bins in arcmin)."""
    n_bins: int
    theta_min: float
    theta_max: float
    n_max: int
    n_phi: int = 100
    n_z: int = 1
    quantum: float = 2.0 ** -13
    norm_truncate: int = 0
    radial_nodes: int = 0
    exclude_degenerate: int = 0

    def c(self) -> OrcCfg:
        return OrcCfg(self.n_bins, self.theta_min, self.theta_max, self.n_max, self.n_phi,
                      self.n_z, self.quantum, self.norm_truncate, self.radial_nodes,
                      self.exclude_degenerate)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        P = C.c_void_p
        I64 = C.c_int64
        for name, args in {
            "orc_edges": [P, P, P],
            "orc_moments": [P, I64, P, P, P, P, P, P, I64, P, P, P],
            "orc_count_pairs": [P, I64, P, P, I64, P, P],
            "orc_contract": [P, P, P, P, P, I64, P, P, P, P, P],
            "orc_degenerate_correction": [P, I64, P, P, P, P, P, P, I64, P, P, P],
            "orc_edge_correct": [P, P, P, P, P],
            "orc_to_gamma": [P, P, C.c_int32, P],
            "orc_to_map3": [P, P, I64, P, P, P],
            "orc_filter": [C.c_int32, C.c_double, C.c_double, C.c_double, P, P],
            "orc_cen_factor": [C.c_int32, C.c_double, C.c_double, C.c_double, P],
            "orc_combine8": [P, P],
            "orc_to_map3_four": [P, P, I64, P, P],
            "orc_combine4": [P, P, P, P, P],
            "orc_brute": [P, I64, P, P, P, P, P, P, C.c_int32, P, P, P, P, P, P],
            "orc_num_threads": [],
            "orc_map3_direct_brute": [I64, P, P, P, P, P, C.c_double, C.c_double, C.c_double, P, C.c_double,
                                      P, P],
            "orc_map3_direct": [I64, P, P, P, P, P, C.c_double, I64, P, P, C.c_double, P],
            "orc_set_num_threads": [C.c_int32],
        }.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = C.c_int
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc: int, ok=(0,)):
    if rc not in ok:
        raise RuntimeError("oracle call failed with status %d" % rc)
    return rc


def map3_direct(cat, centres, theta, rcut_factor: float = 4.0, brute: bool = False) -> np.ndarray:
    """Numerator and denominator of the direct <M_ap^3> estimator (Sec. 5.3, Eq.
    MapDirectEstimator) at every aperture centre [n][2] (arcmin) for the radii theta (3,):
    [n][2]. Galaxies beyond rcut_factor * max(theta) from a centre are left out. brute: the
    literal triple loop over distinct galaxies (tiny catalogs only)."""
    xq, yq, g1, g2, w, _ = _cat(cat)
    th = _c(np.asarray(theta, dtype=np.float64).reshape(3), np.float64)
    cen = _c(np.atleast_2d(np.asarray(centres, dtype=np.float64)), np.float64)
    rcut = float(rcut_factor) * float(th.max())
    out = np.zeros((cen.shape[0], 2), dtype=np.float64)
    if brute:
        for t in range(cen.shape[0]):
            nu, de = C.c_double(), C.c_double()
            _check(lib().orc_map3_direct_brute(cat.n, _p(xq), _p(yq), _p(g1), _p(g2), _p(w), float(cat.quantum),
                                               float(cen[t, 0]), float(cen[t, 1]), _p(th), rcut,
                                               C.byref(nu), C.byref(de)))
            out[t] = (nu.value, de.value)
    else:
        _check(lib().orc_map3_direct(cat.n, _p(xq), _p(yq), _p(g1), _p(g2), _p(w), float(cat.quantum),
                                     cen.shape[0], _p(cen), _p(th), rcut, _p(out)))
    return out


def grid_catalog(cat, origin, pixel_q: int, npx: int, npy: int, n_z: int = 1):
    """The pixel catalog of the grid-based approximation (Sec. 3.2): the weights w and the
    products w gamma of the galaxies summed per pixel of side pixel_q quanta (pixel (ix, iy) of
    z-bin z covers [origin + i pixel_q, origin + (i + 1) pixel_q) on each axis); each pixel becomes
    a galaxy at its centre with weight W = sum w and shear (sum w gamma) / W; the non-empty pixels
    in (z, iy, ix) order. The sums are taken in FP64, where the products of two float32 numbers
    and their sums over a pixel are exact."""
    x0, y0 = int(origin[0]), int(origin[1])
    ix = np.clip((np.asarray(cat.xq, np.int64) - x0) // pixel_q, 0, npx - 1)
    iy = np.clip((np.asarray(cat.yq, np.int64) - y0) // pixel_q, 0, npy - 1)
    z = np.zeros(cat.n, np.int64) if cat.zbin is None else np.asarray(cat.zbin, np.int64)
    p = (z * npy + iy) * npx + ix
    npix = n_z * npy * npx
    w = np.asarray(cat.w, np.float64)
    W = np.zeros(npix)
    A = np.zeros(npix)
    B = np.zeros(npix)
    np.add.at(W, p, w)
    np.add.at(A, p, w * np.asarray(cat.g1, np.float64))
    np.add.at(B, p, w * np.asarray(cat.g2, np.float64))
    k = np.nonzero(W > 0)[0]
    pix_x = x0 + (k % npx) * pixel_q + pixel_q // 2
    pix_y = y0 + ((k // npx) % npy) * pixel_q + pixel_q // 2
    from paper_2309_08601_gb300.synth import Catalog
    return Catalog(pix_x.astype(np.int32), pix_y.astype(np.int32), (A[k] / W[k]).astype(np.float32),
                   (B[k] / W[k]).astype(np.float32), W[k].astype(np.float32),
                   None if n_z == 1 else (k // (npx * npy)).astype(np.uint8), 0.0, cat.quantum)


def combined_moments(s: Setup, cat, levels, centres: Optional[np.ndarray] = None, extent=None):
    """The moments of the combined estimator (Sec. 3.3): level l = (b_start, pixel_q) of levels
    covers the radial bins [b_start_l, b_start_{l+1}) (the last up to n_bins) with the pixel
    catalog of side pixel_q quanta on the grid whose origin is the catalog's lower corner
    (min xq, min yq); there a centre galaxy takes the moments of the pixel it lies in, evaluated
    about the pixel centre (G_n^Delta at its pixel, with no division by the galaxies per pixel:
    the reading under which Eq. CombinedEstimatorRegridding's two lines agree). The bins below the
    first level keep the galaxies' discrete moments (Eq. Gn_disc). A galaxy whose pixel has no
    weight gets zeros. extent = (x0, y0, x1, y1) in quanta (a fixed patch extent, x1 and y1 the
    largest positions) replaces the catalog's bounding box when given. Plain steps: all moments
    of the galaxies and of every pixel catalog, then a copy of the levels' bins."""
    if centres is None:
        centres = np.arange(cat.n, dtype=np.int64)
    centres = np.asarray(centres, dtype=np.int64)
    G, W = moments(s, cat, centres)
    xq = np.asarray(cat.xq, np.int64)
    yq = np.asarray(cat.yq, np.int64)
    z = np.zeros(cat.n, np.int64) if cat.zbin is None else np.asarray(cat.zbin, np.int64)
    if extent is None:
        x0, y0, x1, y1 = int(xq.min()), int(yq.min()), int(xq.max()), int(yq.max())
    else:
        x0, y0, x1, y1 = (int(v) for v in extent)
    for l, (b0, q) in enumerate(levels):
        b1 = int(levels[l + 1][0]) if l + 1 < len(levels) else s.n_bins
        q = int(q)
        npx = (x1 - x0) // q + 1
        npy = (y1 - y0) // q + 1
        pix = grid_catalog(cat, (x0, y0), q, npx, npy, s.n_z)
        Gp, Wp = moments(s, pix)
        # the catalog index of each centre's pixel among the non-empty pixels ((z, iy, ix) order)
        pid = ((z * npy + np.clip((yq - y0) // q, 0, npy - 1)) * npx + np.clip((xq - x0) // q, 0, npx - 1))[centres]
        pz = np.zeros(pix.n, np.int64) if pix.zbin is None else np.asarray(pix.zbin, np.int64)
        kid = (pz * npy + (np.asarray(pix.yq, np.int64) - y0) // q) * npx + (np.asarray(pix.xq, np.int64) - x0) // q
        j = np.searchsorted(kid, pid)
        ok = (j < pix.n) & (kid[np.minimum(j, max(pix.n - 1, 0))] == pid) if pix.n else np.zeros(len(pid), bool)
        G[:, :, b0:b1, :] = 0
        W[:, :, b0:b1, :] = 0
        G[ok, :, b0:b1, :] = Gp[j[ok], :, b0:b1, :]
        W[ok, :, b0:b1, :] = Wp[j[ok], :, b0:b1, :]
    return G, W


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> int:
    """Threads of the oracle's parallel loops from now on (for timing on n host cores)."""
    return lib().orc_set_num_threads(int(n))


def edges(s: Setup):
    e = np.zeros(s.n_bins + 1)
    e2 = np.zeros(s.n_bins + 1, dtype=np.int64)
    cfg = s.c()
    _check(lib().orc_edges(C.byref(cfg), _p(e), _p(e2)))
    return e, e2


def _cat(cat):
    zb = None if cat.zbin is None else _c(cat.zbin, np.uint8)
    return (_c(cat.xq, np.int32), _c(cat.yq, np.int32), _c(cat.g1, np.float32),
            _c(cat.g2, np.float32), _c(cat.w, np.float32), zb)


def moments(s: Setup, cat, centres: Optional[np.ndarray] = None):
    """G [nc][n_z][n_bins][2n_max+3] and W [nc][n_z][n_bins][2n_max+1], complex128."""
    xq, yq, g1, g2, w, zb = _cat(cat)
    if centres is None:
        centres = np.arange(cat.n, dtype=np.int64)
    centres = _c(centres, np.int64)
    nc = centres.shape[0]
    G = np.zeros((nc, s.n_z, s.n_bins, 2 * s.n_max + 3), dtype=np.complex128)
    W = np.zeros((nc, s.n_z, s.n_bins, 2 * s.n_max + 1), dtype=np.complex128)
    cfg = s.c()
    _check(lib().orc_moments(C.byref(cfg), cat.n, _p(xq), _p(yq), _p(g1), _p(g2), _p(w), _p(zb),
                             nc, _p(centres), _p(G), _p(W)))
    return G, W


def count_pairs(s: Setup, cat, centres: Optional[np.ndarray] = None) -> int:
    xq, yq = _c(cat.xq, np.int32), _c(cat.yq, np.int32)
    if centres is None:
        centres = np.arange(cat.n, dtype=np.int64)
    centres = _c(centres, np.int64)
    out = np.zeros(1, dtype=np.int64)
    cfg = s.c()
    _check(lib().orc_count_pairs(C.byref(cfg), cat.n, _p(xq), _p(yq), centres.shape[0],
                                 _p(centres), _p(out)))
    return int(out[0])


def contract(s: Setup, cat, G, W, centres: Optional[np.ndarray] = None, ups=None, norm=None):
    """Adds into ups [n_z^3][4][n_max+1][nb][nb] and norm [n_z^3][2n_max+1][nb][nb]."""
    _, _, g1, g2, w, zb = _cat(cat)
    if centres is None:
        centres = np.arange(cat.n, dtype=np.int64)
    centres = _c(centres, np.int64)
    z3 = s.n_z ** 3
    if ups is None:
        ups = np.zeros((z3, 4, s.n_max + 1, s.n_bins, s.n_bins), dtype=np.complex128)
    if norm is None:
        norm = np.zeros((z3, 2 * s.n_max + 1, s.n_bins, s.n_bins), dtype=np.complex128)
    G = _c(G, np.complex128)
    W = _c(W, np.complex128)
    cfg = s.c()
    _check(lib().orc_contract(C.byref(cfg), _p(g1), _p(g2), _p(w), _p(zb), centres.shape[0],
                              _p(centres), _p(G), _p(W), _p(ups), _p(norm)))
    return ups, norm


def degenerate_correction(s: Setup, cat, ups, norm, centres: Optional[np.ndarray] = None):
    """With s.exclude_degenerate, removes the j = k triplets from (ups, norm) in place."""
    xq, yq, g1, g2, w, zb = _cat(cat)
    if centres is None:
        centres = np.arange(cat.n, dtype=np.int64)
    centres = _c(centres, np.int64)
    cfg = s.c()
    _check(lib().orc_degenerate_correction(C.byref(cfg), cat.n, _p(xq), _p(yq), _p(g1), _p(g2), _p(w),
                                           _p(zb), centres.shape[0], _p(centres), _p(ups), _p(norm)))
    return ups, norm


def edge_correct(s: Setup, ups, norm):
    """Returns (gamma_n [n_z^3][4][2n_max+1][nb][nb], number of singular systems)."""
    z3 = s.n_z ** 3
    gam = np.zeros((z3, 4, 2 * s.n_max + 1, s.n_bins, s.n_bins), dtype=np.complex128)
    ns = np.zeros(1, dtype=np.int64)
    ups = _c(ups, np.complex128)
    norm = _c(norm, np.complex128)
    cfg = s.c()
    _check(lib().orc_edge_correct(C.byref(cfg), _p(ups), _p(norm), _p(gam), _p(ns)), ok=(0, 5))
    return gam, int(ns[0])


def to_gamma(s: Setup, gam_n, projection: int):
    z3 = s.n_z ** 3
    out = np.zeros((z3, 4, s.n_bins, s.n_bins, s.n_phi), dtype=np.complex128)
    gam_n = _c(gam_n, np.complex128)
    cfg = s.c()
    _check(lib().orc_to_gamma(C.byref(cfg), _p(gam_n), projection, _p(out)))
    return out


def to_map3(s: Setup, gamma_cen, theta_ap):
    """theta_ap: [n_ap][3] arcmin. Returns (corr [n_z^3][n_ap][4] complex, m8 [..][8])."""
    th = _c(np.atleast_2d(theta_ap), np.float64)
    n_ap = th.shape[0]
    z3 = s.n_z ** 3
    corr = np.zeros((z3, n_ap, 4), dtype=np.complex128)
    m8 = np.zeros((z3, n_ap, 8))
    gc = _c(gamma_cen, np.complex128)
    cfg = s.c()
    _check(lib().orc_to_map3(C.byref(cfg), _p(gc), n_ap, _p(th), _p(corr), _p(m8)))
    return corr, m8


def to_map3_four(s: Setup, gamma_cen, theta_ap):
    """The four-equation form (App. C): m4 [n_z^3][n_ap][4] = (Map^3, <Map^2 Mx>, <Map Mx^2>,
    <Mx^3>) from <M^3> and the Gamma_1 correlator at three orderings of the radii."""
    th = _c(np.atleast_2d(theta_ap), np.float64)
    n_ap = th.shape[0]
    m4 = np.zeros((s.n_z ** 3, n_ap, 4))
    gc = _c(gamma_cen, np.complex128)
    cfg = s.c()
    _check(lib().orc_to_map3_four(C.byref(cfg), _p(gc), n_ap, _p(th), _p(m4)))
    return m4


def combine4(m3, a123, a132, a231) -> np.ndarray:
    """Eqs. MapTrafo4_1-4 from <M^3>(t1, t2, t3) and the one-conjugate correlators A123, A132,
    A231 (conjugate on the last radius of each ordering), each a complex number."""
    vals = [_c(np.array([complex(v)]), np.complex128) for v in (m3, a123, a132, a231)]
    out = np.zeros(4)
    _check(lib().orc_combine4(*[_p(v) for v in vals], _p(out)))
    return out


def filter_F(mu: int, t1: float, t2: float, phi: float, theta) -> complex:
    th = _c(theta, np.float64)
    out = np.zeros(2)
    _check(lib().orc_filter(mu, t1, t2, phi, _p(th), _p(out)))
    return complex(out[0], out[1])


def cen_factor(mu: int, t1: float, t2: float, phi: float) -> complex:
    out = np.zeros(2)
    _check(lib().orc_cen_factor(mu, t1, t2, phi, _p(out)))
    return complex(out[0], out[1])


def combine8(corr) -> np.ndarray:
    c = _c(corr, np.complex128)
    out = np.zeros(8)
    _check(lib().orc_combine8(_p(c), _p(out)))
    return out


@dataclass
class Brute:
    ups_n: np.ndarray
    norm_n: np.ndarray
    ups_b: np.ndarray
    norm_b: np.ndarray
    upsc_b: np.ndarray
    p5_dev: float


def brute(s: Setup, cat, n_phib: int = 16) -> Brute:
    xq, yq, g1, g2, w, zb = _cat(cat)
    z3 = s.n_z ** 3
    nb = s.n_bins
    ups_n = np.zeros((z3, 4, s.n_max + 1, nb, nb), dtype=np.complex128)
    norm_n = np.zeros((z3, 2 * s.n_max + 1, nb, nb), dtype=np.complex128)
    ups_b = np.zeros((z3, 4, nb, nb, n_phib), dtype=np.complex128)
    norm_b = np.zeros((z3, nb, nb, n_phib), dtype=np.complex128)
    upsc_b = np.zeros((z3, 4, nb, nb, n_phib), dtype=np.complex128)
    dev = np.zeros(1)
    cfg = s.c()
    _check(lib().orc_brute(C.byref(cfg), cat.n, _p(xq), _p(yq), _p(g1), _p(g2), _p(w), _p(zb),
                           n_phib, _p(ups_n), _p(norm_n), _p(ups_b), _p(norm_b), _p(upsc_b),
                           _p(dev)))
    return Brute(ups_n, norm_n, ups_b, norm_b, upsc_b, float(dev[0]))


@dataclass
class Result:
    G: np.ndarray
    W: np.ndarray
    ups: np.ndarray
    norm: np.ndarray
    gamma_n: np.ndarray
    n_singular: int
    gamma_x: np.ndarray
    gamma_cen: np.ndarray
    corr: np.ndarray
    m8: np.ndarray


def pipeline(s: Setup, cat, theta_ap, centres: Optional[np.ndarray] = None) -> Result:
    """The whole path on the oracle: moments, multipoles, edge correction, Gamma, Map^3."""
    G, W = moments(s, cat, centres)
    ups, norm = contract(s, cat, G, W, centres)
    if s.exclude_degenerate:
        degenerate_correction(s, cat, ups, norm, centres)
    gam, ns = edge_correct(s, ups, norm)
    gx = to_gamma(s, gam, 0)
    gc = to_gamma(s, gam, 1)
    corr, m8 = to_map3(s, gc, theta_ap)
    return Result(G, W, ups, norm, gam, ns, gx, gc, corr, m8)


__all__ = ["Setup", "build_oracle", "edges", "moments", "count_pairs", "contract",
           "edge_correct", "degenerate_correction", "to_gamma", "to_map3", "to_map3_four", "combine4", "filter_F", "cen_factor", "combine8", "brute",
           "pipeline", "num_threads", "set_num_threads", "map3_direct", "grid_catalog", "combined_moments", "Result",
           "Brute"]
