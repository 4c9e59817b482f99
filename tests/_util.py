"""Small helpers shared by the tests (no estimator arithmetic)."""
import numpy as np

from paper_2309_08601_gb300.synth import Catalog, QUANTUM


def rel_err(a, b):
    """max|a - b| / max|b| over the whole array (normwise relative error)."""
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.abs(b).max() if b.size else 0.0
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0)) if a.size else 0.0


def hand_catalog(xy_arcmin, g, w=None, zbin=None, quantum=QUANTUM, offset=1000.0):
    """A catalog from explicit positions (arcmin, shifted by ``offset``), complex shears g."""
    xy = np.asarray(xy_arcmin, dtype=np.float64) + offset
    g = np.asarray(g, dtype=np.complex128)
    n = xy.shape[0]
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    return Catalog(np.round(xy[:, 0] / quantum).astype(np.int32),
                   np.round(xy[:, 1] / quantum).astype(np.int32),
                   g.real.astype(np.float32), g.imag.astype(np.float32), w.astype(np.float32),
                   None if zbin is None else np.asarray(zbin, dtype=np.uint8), 0.0, quantum)
