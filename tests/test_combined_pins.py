"""Pins of the oracle's combined estimator (Sec. 3.3): with pixels of one quantum and one galaxy
per position every pixel is its galaxy, so the combined moments are the discrete ones whatever
the levels; with every bin on one grid level the galaxies' contraction of their pixels' moments
is the pixel catalog's own contraction (Eq. UpsilonmuGrid, the gg block), which holds only if a
galaxy takes its pixel's moments undivided by the galaxies per pixel (the reading of
Eq. CombinedEstimatorRegridding)."""
import numpy as np
import pytest

from paper_2309_08601_gb300 import synth

from ._util import rel_err


def _unique_positions_catalog(rng, n, side_q, quantum, n_z=1):
    """n galaxies at distinct integer positions of a side_q x side_q square (fixed-point quanta)."""
    cells = rng.choice(side_q * side_q, size=n, replace=False)
    x = (cells % side_q + 5000).astype(np.int32)
    y = (cells // side_q + 7000).astype(np.int32)
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    z = None if n_z == 1 else rng.integers(0, n_z, n).astype(np.uint8)
    return synth.Catalog(x, y, g.real.astype(np.float32), g.imag.astype(np.float32),
                         rng.uniform(0.5, 1.5, n).astype(np.float32), z, 0.0, quantum)


@pytest.mark.parametrize("n_z", [1, 2])
def test_unit_pixels_give_the_discrete_moments(orc, n_z):
    rng = np.random.default_rng(11 + n_z)
    quantum = 1.0 / 16  # 240 quanta = 15 arcmin per side: 57 600 one-quantum pixels per z-bin
    cat = _unique_positions_catalog(rng, 1500, 240, quantum, n_z)
    s = orc.Setup(n_bins=6, theta_min=0.5, theta_max=5.0, n_max=4, n_z=n_z, quantum=quantum)
    centres = np.sort(rng.choice(cat.n, size=400, replace=False))
    G0, W0 = orc.moments(s, cat, centres)
    for levels in ([(2, 1)], [(0, 1)], [(1, 1), (4, 1)]):
        G1, W1 = orc.combined_moments(s, cat, levels, centres)
        assert rel_err(G1, G0) < 1e-12, levels
        assert rel_err(W1, W0) < 1e-12, levels


def test_discrete_bins_are_left_as_they_are(orc):
    rng = np.random.default_rng(5)
    cat = synth.make_catalog(2500, 30.0, 9, field="noise", weights="uniform")
    s = orc.Setup(n_bins=6, theta_min=0.5, theta_max=6.0, n_max=3)
    G0, W0 = orc.moments(s, cat)
    G1, W1 = orc.combined_moments(s, cat, [(3, 1 << 12)])
    assert np.array_equal(G1[:, :, :3], G0[:, :, :3]) and np.array_equal(W1[:, :, :3], W0[:, :, :3])
    # the grid bins differ from the discrete ones (the pixels are 0.5', the bins from 1.5')
    assert rel_err(G1[:, :, 3:], G0[:, :, 3:]) > 1e-3
    del rng


@pytest.mark.parametrize("n_z", [1, 2])
def test_one_grid_level_is_the_pixel_catalogs_contraction(orc, n_z):
    """Sum over galaxies of w_i gamma_i G^Delta(p_i) G^Delta(p_i) = sum over pixels of
    (w gamma)_p G^Delta(p) G^Delta(p): equal up to the float32 rounding of the pixel catalog's
    weights and shears (the pixel sums are exact in FP64, the emitted W and (sum w gamma) / W are
    rounded once to float32, a relative 6e-8). A division of the pixel moments by the galaxies per
    pixel (about 5 here) would miss by a factor of that order."""
    if n_z == 1:
        cat = synth.make_catalog(3000, 24.0, 3, field="noise", weights="uniform")
    else:
        cat = synth.make_tomographic_catalog(4, side=24.0, n_z=2, n_range=(1200, 1800), ngrid=128)
    q = 1 << 13  # 1 arcmin
    s = orc.Setup(n_bins=5, theta_min=1.0, theta_max=6.0, n_max=4, n_z=n_z)
    G, W = orc.combined_moments(s, cat, [(0, q)])
    u0, n0 = orc.contract(s, cat, G, W)
    x0, y0 = int(cat.xq.min()), int(cat.yq.min())
    npx = (int(cat.xq.max()) - x0) // q + 1
    npy = (int(cat.yq.max()) - y0) // q + 1
    pix = orc.grid_catalog(cat, (x0, y0), q, npx, npy, n_z)
    assert cat.n > 2 * pix.n  # several galaxies per pixel
    Gp, Wp = orc.moments(s, pix)
    u1, n1 = orc.contract(s, pix, Gp, Wp)
    assert rel_err(u0, u1) < 1e-6
    assert rel_err(n0, n1) < 1e-6


def test_grid_levels_follow_the_octave_rule():
    """20 Delta <= lower edge < 40 Delta per level, Delta doubling: for 24 logarithmic bins
    0.25'-60' and 0.25' base pixels the levels start at the first edges above 5', 10', 20', 40'."""
    edges = 0.25 * 240.0 ** (np.arange(25) / 24)
    q = 2.0 ** -13
    lv = synth.grid_levels(edges, 1 << 11, q)
    assert lv == [(14, 1 << 11), (17, 1 << 12), (20, 1 << 13), (23, 1 << 14)]
    for k, (b, d) in enumerate(lv):
        last = lv[k + 1][0] if k + 1 < len(lv) else 24
        for bb in range(b, last):
            assert 20 * d <= edges[bb] / q < 40 * d
    assert edges[lv[0][0] - 1] / q < 20 * (1 << 11)
    # twice the pixels per bin: the same discrete range on pixels half the size
    assert synth.grid_levels(edges, 1 << 10, q, ratio=40) == [(b, d // 2) for b, d in lv]
