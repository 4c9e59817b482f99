"""Pins of the oracle's pixel catalog for the grid-based approximation (Sec. 3.2): the gridding
conserves the total weight and the total w gamma; a catalog with at most one galaxy per pixel,
each at its pixel centre, is reproduced exactly; and then the multipoles of the pixel catalog
equal those of the catalog itself."""
import numpy as np

from paper_2309_08601_gb300 import synth

SETUP = dict(n_bins=5, theta_min=1.0, theta_max=8.0, n_max=4)


def test_gridding_conserves_weight_and_shear(orc):
    cat = synth.make_catalog(5000, 40.0, 2, field="noise", weights="uniform")
    pq = 1 << 13  # 1 arcmin
    x0, y0 = int(cat.xq.min()), int(cat.yq.min())
    npx = (int(cat.xq.max()) - x0) // pq + 1
    npy = (int(cat.yq.max()) - y0) // pq + 1
    pix = orc.grid_catalog(cat, (x0, y0), pq, npx, npy)
    w = cat.w.astype(np.float64)
    assert abs(pix.w.astype(np.float64).sum() - w.sum()) <= 1e-6 * w.sum()
    for a, b in ((pix.g1, cat.g1), (pix.g2, cat.g2)):
        tot = (w * b).sum()
        assert abs((pix.w.astype(np.float64) * a).sum() - tot) <= 1e-6 * np.abs(w * b).sum()


def _lattice_catalog(rng, pq, n_side, fill, n_z=1):
    ix, iy = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    keep = rng.uniform(size=ix.shape) < fill
    x = (ix[keep] * pq + pq // 2 + 10_000_000).astype(np.int32)
    y = (iy[keep] * pq + pq // 2 + 10_000_000).astype(np.int32)
    n = x.size
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    z = None if n_z == 1 else rng.integers(0, n_z, n).astype(np.uint8)
    return synth.Catalog(x, y, g.real.astype(np.float32), g.imag.astype(np.float32),
                         rng.uniform(0.5, 1.5, n).astype(np.float32), z, 0.0, synth.QUANTUM)


def test_one_galaxy_per_pixel_centre_is_reproduced(orc):
    rng = np.random.default_rng(3)
    pq = 4096  # 0.5 arcmin
    cat = _lattice_catalog(rng, pq, 40, 0.6)
    pix = orc.grid_catalog(cat, (10_000_000, 10_000_000), pq, 40, 40)
    assert pix.n == cat.n
    order = np.lexsort((cat.xq, cat.yq))  # (iy, ix) order, as the pixel catalog
    for f in ("xq", "yq", "g1", "g2", "w"):
        assert np.array_equal(getattr(pix, f), getattr(cat, f)[order])


def test_pixel_catalog_multipoles_equal_the_catalogs(orc):
    rng = np.random.default_rng(4)
    pq = 4096
    for n_z in (1, 2):
        cat = _lattice_catalog(rng, pq, 36, 0.5, n_z)
        pix = orc.grid_catalog(cat, (10_000_000, 10_000_000), pq, 36, 36, n_z)
        s = orc.Setup(**SETUP, n_z=n_z)
        G, W = orc.moments(s, cat)
        u0, n0 = orc.contract(s, cat, G, W)
        G, W = orc.moments(s, pix)
        u1, n1 = orc.contract(s, pix, G, W)
        assert np.abs(u1 - u0).max() <= 1e-12 * np.abs(u0).max()
        assert np.abs(n1 - n0).max() <= 1e-12 * np.abs(n0).max()
