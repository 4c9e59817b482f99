"""Pins of the oracle's direct estimator of <M_ap^3> (Sec. 5.3, Eq. MapDirectEstimator):
the O(n) inclusion-exclusion form against the literal triple loop over distinct galaxies, and
closed forms: a purely tangential shear pattern of amplitude g0 about the aperture centre gives
exactly g0^3, a purely cross pattern gives 0, a quarter turn of the catalog about the centre
(with the shears rotated by the spin-2 phase) changes nothing, and galaxies beyond the cut-off
contribute nothing."""
import numpy as np
import pytest

from paper_2309_08601_gb300.synth import QUANTUM
from tests._util import hand_catalog

OFF = 1000.0  # hand_catalog's position offset (arcmin)


def _rand_cat(rng, n, half=6.0, z=None):
    xy = rng.uniform(-half, half, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    return hand_catalog(xy, g, rng.uniform(0.5, 1.5, n), z)


@pytest.mark.parametrize("n,seed", [(5, 0), (7, 1), (9, 2)])
def test_inclusion_exclusion_equals_the_triple_loop(orc, n, seed):
    rng = np.random.default_rng(seed)
    cat = _rand_cat(rng, n)
    cen = OFF + rng.uniform(-2, 2, (4, 2))
    for th in ([1.5, 1.5, 1.5], [1.0, 2.0, 3.0]):
        a = orc.map3_direct(cat, cen, th, rcut_factor=100.0)
        b = orc.map3_direct(cat, cen, th, rcut_factor=100.0, brute=True)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        # with the paper's cut-off at 4 max(theta) some galaxies drop out; still equal
        a = orc.map3_direct(cat, cen, th)
        b = orc.map3_direct(cat, cen, th, brute=True)
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)


def _pattern(rng, n, g0, cross):
    xy = rng.uniform(-6, 6, (n, 2))
    zeta = np.arctan2(xy[:, 1], xy[:, 0])
    # gamma(x; zeta) = -gamma e^{-2 i zeta}: tangential part g0 for gamma = -g0 e^{2 i zeta}
    g = (-1j if cross else -1.0) * g0 * np.exp(2j * zeta)
    return hand_catalog(xy, g, rng.uniform(0.5, 1.5, n))


def test_tangential_pattern_gives_the_cube_of_its_amplitude(orc):
    rng = np.random.default_rng(5)
    g0 = 0.07
    cat = _pattern(rng, 400, g0, cross=False)
    r = orc.map3_direct(cat, [[OFF, OFF]], [2.0, 2.0, 2.0])[0]
    assert abs(r[0] / r[1] - g0 ** 3) <= 1e-6 * g0 ** 3
    r = orc.map3_direct(cat, [[OFF, OFF]], [1.0, 1.5, 2.5])[0]
    assert abs(r[0] / r[1] - g0 ** 3) <= 1e-6 * g0 ** 3


def test_cross_pattern_gives_zero(orc):
    rng = np.random.default_rng(6)
    cat = _pattern(rng, 400, 0.07, cross=True)
    r = orc.map3_direct(cat, [[OFF, OFF]], [2.0, 2.0, 2.0])[0]
    assert abs(r[0] / r[1]) <= 1e-12


def test_quarter_turn_about_the_centre(orc):
    rng = np.random.default_rng(7)
    cat = _rand_cat(rng, 300)
    c = np.array([np.round(OFF / QUANTUM), np.round(OFF / QUANTUM)], dtype=np.int64)
    rot = hand_catalog(np.zeros((cat.n, 2)), np.zeros(cat.n), cat.w)
    rot.xq = (c[0] - (cat.yq.astype(np.int64) - c[1])).astype(np.int32)
    rot.yq = (c[1] + (cat.xq.astype(np.int64) - c[0])).astype(np.int32)
    rot.g1, rot.g2 = -cat.g1, -cat.g2  # gamma e^{2 i pi/2}
    cen = [[c[0] * QUANTUM, c[1] * QUANTUM]]
    for th in ([2.0, 2.0, 2.0], [1.0, 2.0, 3.0]):
        a = orc.map3_direct(cat, cen, th)[0]
        b = orc.map3_direct(rot, cen, th)[0]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_galaxies_beyond_the_cut_off_do_not_count(orc):
    rng = np.random.default_rng(8)
    cat = _rand_cat(rng, 200, half=3.0)
    far = _rand_cat(rng, 50, half=3.0)
    far.xq = far.xq + np.int32(round(40.0 / QUANTUM))  # 40' away: beyond 4 x 3'
    both = hand_catalog(np.zeros((250, 2)), np.zeros(250), np.ones(250))
    for f in ("xq", "yq", "g1", "g2", "w"):
        setattr(both, f, np.concatenate([getattr(cat, f), getattr(far, f)]))
    a = orc.map3_direct(cat, [[OFF, OFF]], [1.0, 2.0, 3.0])
    b = orc.map3_direct(both, [[OFF, OFF]], [1.0, 2.0, 3.0])
    assert np.array_equal(a, b)


def test_aperture_grid_and_the_mean_over_apertures():
    """api.aperture_centres keeps every aperture rcut_factor * max(theta) inside the bounding box
    on a grid of the smallest radius; api.map3_from_direct averages numerator / denominator over
    the apertures with a non-zero denominator."""
    from paper_2309_08601_gb300 import api
    q = 2.0 ** -13
    xq = np.array([0, 800_000, 0, 800_000], dtype=np.int32)  # a 97.66' square
    yq = np.array([0, 0, 800_000, 800_000], dtype=np.int32)
    th = [[2.0, 2.0, 2.0], [4.0, 4.0, 8.0]]
    c = api.aperture_centres(xq, yq, q, th)
    side = 800_000 * q
    assert c.shape[1] == 2 and len(c) > 0
    assert (c >= 32.0 - 1e-9).all() and (c <= side - 32.0 + 1e-9).all()
    steps = np.diff(np.unique(c[:, 0]))
    assert np.allclose(steps, 2.0)
    assert api.aperture_centres(xq[:2], yq[:2], q, th).shape == (0, 2)  # no room inside the margins
    out = np.zeros((3, 2, 2))  # [aperture][radii triple][numerator, denominator]
    out[..., 0] = [[1.0, 2.0], [2.0, 0.0], [3.0, 4.0]]
    out[..., 1] = [[1.0, 2.0], [2.0, 0.0], [0.0, 4.0]]  # zero denominators are left out
    np.testing.assert_allclose(api.map3_from_direct(out), [1.0, 1.0])
