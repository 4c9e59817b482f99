"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: the triplet-sum definitions
(brute force), exact symmetries, closed forms, a library linear solver, the defining integrals
of the aperture filters, or Fourier convergence.
"""
import numpy as np
import pytest

from paper_2309_08601_gb300.synth import Catalog, QUANTUM, make_catalog
from tests._util import hand_catalog, rel_err

S0 = dict(n_bins=10, theta_min=0.5, theta_max=30.0, n_max=10)
THETA_EQ = [[2.0, 2.0, 2.0], [4.0, 4.0, 4.0], [8.0, 8.0, 8.0]]


def _cat_from_int(xq, yq, g, w):
    g = np.asarray(g, dtype=np.complex128)
    return Catalog(np.asarray(xq, np.int32), np.asarray(yq, np.int32), g.real.astype(np.float32),
                   g.imag.astype(np.float32), np.asarray(w, np.float32), None, 0.0, QUANTUM)


# ---------------------------------------------------------------- bins (Sec. 2.4, half-open reading)

def test_bin_edges_are_log_spaced_and_half_open(orc):
    s = orc.Setup(n_bins=5, theta_min=1.0, theta_max=10.0, n_max=2)
    e, e2 = orc.edges(s)
    assert e[0] == 1.0 and abs(e[-1] - 10.0) < 1e-12
    np.testing.assert_allclose(e[1:] / e[:-1], 10 ** 0.2, rtol=1e-13)
    np.testing.assert_array_equal(e2, np.ceil((e / QUANTUM) ** 2).astype(np.int64))
    x0 = 10_000_000
    for b in range(1, 5):
        d = int(np.ceil(np.sqrt(float(e2[b]))))
        while d * d < e2[b]:
            d += 1
        while (d - 1) * (d - 1) >= e2[b]:
            d -= 1
        for sep, expect in ((d, b), (d - 1, b - 1)):
            cat = _cat_from_int([x0, x0 + sep], [x0, x0], [0.1, 0.2], [1.0, 1.0])
            G, W = orc.moments(s, cat, centres=np.array([0]))
            occupied = np.nonzero(np.abs(W[0, 0, :, 0]))[0]
            assert occupied.tolist() == [expect], (b, sep)
            assert W[0, 0, expect, 0] == 1.0


# ------------------------------------------- P1: moment route == triplet sums (Sec. 3.1)

@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_moments_equal_triplet_sums_hand_placed(orc, n):
    rng = np.random.default_rng(100 + n)
    xy = rng.uniform(0, 8, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    w = rng.uniform(0.5, 1.5, n)
    s = orc.Setup(n_bins=4, theta_min=0.5, theta_max=12.0, n_max=6)
    cat = hand_catalog(xy, g, w)
    b = orc.brute(s, cat)
    G, W = orc.moments(s, cat)
    ups, norm = orc.contract(s, cat, G, W)
    assert np.abs(b.norm_n).max() > 0
    assert rel_err(ups, b.ups_n) < 1e-12
    assert rel_err(norm, b.norm_n) < 1e-12


def test_moments_equal_triplet_sums_equilateral(orc):
    # equilateral triangle plus a fourth point: every triplet lands in the same radial bin
    xy = [[0, 0], [3, 0], [1.5, 1.5 * np.sqrt(3)], [1.5, 0.5]]
    g = [0.1 + 0.05j, -0.2 + 0.1j, 0.05 - 0.3j, 0.2 + 0.2j]
    s = orc.Setup(n_bins=3, theta_min=1.0, theta_max=4.0, n_max=8)
    cat = hand_catalog(xy, g)
    b = orc.brute(s, cat)
    G, W = orc.moments(s, cat)
    ups, norm = orc.contract(s, cat, G, W)
    assert rel_err(ups, b.ups_n) < 1e-12 and rel_err(norm, b.norm_n) < 1e-12


def test_moments_equal_triplet_sums_noise_subset(orc, noise2k):
    sub = noise2k.subset(np.arange(300))
    s = orc.Setup(**S0)
    b = orc.brute(s, sub)
    G, W = orc.moments(s, sub)
    ups, norm = orc.contract(s, sub, G, W)
    for mu in range(4):
        assert rel_err(ups[:, mu], b.ups_n[:, mu]) < 1e-12
    assert rel_err(norm, b.norm_n) < 1e-12
    assert b.p5_dev < 1e-12  # P5: per-triplet x -> centroid identity (Eqs. X2Centroid0-3)


def test_tomographic_moments_equal_triplet_sums(orc):
    rng = np.random.default_rng(7)
    n = 120
    xy = rng.uniform(0, 20, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    z = rng.integers(0, 2, n)
    s = orc.Setup(n_bins=3, theta_min=1.0, theta_max=8.0, n_max=4, n_z=2)
    cat = hand_catalog(xy, g, rng.uniform(0.5, 1.5, n), z)
    b = orc.brute(s, cat)
    G, W = orc.moments(s, cat)
    ups, norm = orc.contract(s, cat, G, W)
    assert rel_err(ups, b.ups_n) < 1e-12 and rel_err(norm, b.norm_n) < 1e-12
    # summing the tomographic components over all (Z1, Z2, Z3) gives the plain estimator
    s1 = orc.Setup(n_bins=3, theta_min=1.0, theta_max=8.0, n_max=4, n_z=1)
    cat1 = hand_catalog(xy, g, cat.w)
    G1, W1 = orc.moments(s1, cat1)
    u1, n1 = orc.contract(s1, cat1, G1, W1)
    assert rel_err(ups.sum(axis=0), u1[0]) < 1e-12 and rel_err(norm.sum(axis=0), n1[0]) < 1e-12


@pytest.mark.parametrize("n_z", [1, 2])
def test_excluding_degenerate_triplets_equals_triplet_sums_without_j_eq_k(orc, n_z):
    """exclude_degenerate (j = k left out): the moment route with the degenerate correction
    equals the brute-force triplet sums that skip j = k; the removed part sits only on b1 = b2
    and Z2 = Z3."""
    rng = np.random.default_rng(17 + n_z)
    n = 90
    xy = rng.uniform(0, 16, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    z = rng.integers(0, n_z, n) if n_z > 1 else None
    cat = hand_catalog(xy, g, rng.uniform(0.5, 1.5, n), z)
    kw = dict(n_bins=4, theta_min=0.8, theta_max=8.0, n_max=5, n_z=n_z)
    s_in, s_ex = orc.Setup(**kw), orc.Setup(**kw, exclude_degenerate=1)
    b = orc.brute(s_ex, cat)
    G, W = orc.moments(s_ex, cat)
    ups, norm = orc.contract(s_ex, cat, G, W)
    u_in, n_in = ups.copy(), norm.copy()
    orc.degenerate_correction(s_ex, cat, ups, norm)
    assert rel_err(ups, b.ups_n) < 1e-12 and rel_err(norm, b.norm_n) < 1e-12
    d_u, d_n = u_in - ups, n_in - norm
    mask = np.zeros((n_z ** 3, 4, 4), bool)  # (zt, b1, b2) where j = k can occur
    for zt in range(n_z ** 3):
        if (zt // n_z) % n_z == zt % n_z:
            mask[zt, np.arange(4), np.arange(4)] = True
    assert np.abs(d_u[~mask[:, None, None].repeat(4, 1).repeat(6, 2)]).max() == 0
    assert np.abs(d_n[~mask[:, None].repeat(11, 1)]).max() == 0
    assert np.abs(d_n).max() > 0
    # the default (include) equals the plain brute force
    bi = orc.brute(s_in, cat)
    assert rel_err(u_in, bi.ups_n) < 1e-12


# ------------------------------------------------------ P2: exact invariants of the estimator

@pytest.fixture(scope="module")
def base_run(orc, noise2k):
    s = orc.Setup(**S0)
    return s, orc.pipeline(s, noise2k, THETA_EQ)


def _with(cat, xq=None, yq=None, g=None, w=None):
    g = (cat.g1.astype(np.float64) + 1j * cat.g2) if g is None else g
    return Catalog(cat.xq if xq is None else xq.astype(np.int32),
                   cat.yq if yq is None else yq.astype(np.int32),
                   np.real(g).astype(np.float32), np.imag(g).astype(np.float32),
                   cat.w if w is None else w.astype(np.float32), None, cat.side, cat.quantum)


def test_translation_is_bitwise_invariant(orc, noise2k, base_run):
    s, r = base_run
    r2 = orc.pipeline(s, _with(noise2k, xq=noise2k.xq + 123457, yq=noise2k.yq + 7), THETA_EQ)
    np.testing.assert_array_equal(r2.ups, r.ups)
    np.testing.assert_array_equal(r2.norm, r.norm)


def test_quarter_turn_rotation_invariance(orc, noise2k, base_run):
    s, r = base_run
    # positions rotated by +90 degrees, shear spin-2: gamma -> gamma e^{2 i pi/2} = -gamma
    g = noise2k.g1.astype(np.float64) + 1j * noise2k.g2.astype(np.float64)
    xr = int(noise2k.yq.max()) + 1 - noise2k.yq.astype(np.int64)
    r2 = orc.pipeline(s, _with(noise2k, xq=xr, yq=noise2k.xq.astype(np.int64), g=-g), THETA_EQ)
    assert rel_err(r2.ups, r.ups) < 1e-12 and rel_err(r2.norm, r.norm) < 1e-12
    assert rel_err(r2.gamma_n, r.gamma_n) < 1e-10
    assert rel_err(r2.m8, r.m8) < 1e-9


def test_reflection_parity(orc, noise2k, base_run):
    s, r = base_run
    g = noise2k.g1.astype(np.float64) - 1j * noise2k.g2.astype(np.float64)  # gamma_2 -> -gamma_2
    xr = int(noise2k.xq.max()) + 1 - noise2k.xq.astype(np.int64)  # x -> -x
    r2 = orc.pipeline(s, _with(noise2k, xq=xr, g=g), THETA_EQ)
    assert rel_err(r2.ups, np.conj(r.ups)) < 1e-12 and rel_err(r2.norm, np.conj(r.norm)) < 1e-12
    # parity-even measures unchanged, parity-odd ones flip sign (Sec. 5.2)
    sign = np.array([1, -1, -1, -1, 1, 1, 1, -1])
    assert rel_err(r2.m8, r.m8 * sign) < 1e-9


def test_e_to_b_rotation(orc, noise2k, base_run):
    s, r = base_run
    g = 1j * (noise2k.g1.astype(np.float64) + 1j * noise2k.g2.astype(np.float64))
    r2 = orc.pipeline(s, _with(noise2k, g=g), THETA_EQ)
    # M -> i M: Map -> -Mx, Mx -> Map, so Map^3 -> -Mx^3 and Mx^3 -> Map^3
    assert rel_err(r2.m8[..., 0], -r.m8[..., 7]) < 1e-9
    assert rel_err(r2.m8[..., 7], r.m8[..., 0]) < 1e-9


def test_scaling(orc, noise2k, base_run):
    s, r = base_run
    g = noise2k.g1.astype(np.float64) + 1j * noise2k.g2.astype(np.float64)
    r2 = orc.pipeline(s, _with(noise2k, g=0.5 * g), THETA_EQ)
    assert rel_err(r2.ups, 0.125 * r.ups) < 1e-12
    r3 = orc.pipeline(s, _with(noise2k, w=2.0 * noise2k.w.astype(np.float64)), THETA_EQ)
    assert rel_err(r3.gamma_n, r.gamma_n) < 1e-10 and rel_err(r3.m8, r.m8) < 1e-9


# ----------------------------------- P3: the mode-coupling solve (Eqs. ModeCoupling, App. A)

def _extended(s, ups, norm, zt, b1, b2):
    """Upsilon_l (l in [-n_max, n_max]) and N_m (m in [-2n_max, 2n_max]) via App. A symmetries."""
    nmax, nz = s.n_max, s.n_z
    z1, z2, z3 = zt // (nz * nz), (zt // nz) % nz, zt % nz
    zs = (z1 * nz + z3) * nz + z2
    swap = {0: 0, 1: 1, 2: 3, 3: 2}
    U = np.zeros((4, 2 * nmax + 1), complex)
    for mu in range(4):
        for l in range(-nmax, nmax + 1):
            U[mu, l + nmax] = ups[zt, mu, l, b1, b2] if l >= 0 else ups[zs, swap[mu], -l, b2, b1]
    N = {m: (norm[zt, m, b1, b2] if m >= 0 else norm[zs, -m, b2, b1])
         for m in range(-2 * nmax, 2 * nmax + 1)}
    A = np.array([[N[l - n] for n in range(-nmax, nmax + 1)] for l in range(-nmax, nmax + 1)])
    return U, A


def test_edge_correction_matches_library_solve(orc, noise2k, base_run):
    s, r = base_run
    for (b1, b2) in [(0, 0), (3, 7), (9, 2), (9, 9)]:
        U, A = _extended(s, r.ups, r.norm, 0, b1, b2)
        # N_{-m}(i,j) = N_m(j,i) = N_m(i,j)^*: the coupling matrix is Hermitian
        np.testing.assert_allclose(A, A.conj().T, rtol=0, atol=1e-12 * np.abs(A).max())
        x = np.linalg.solve(A, U.T)
        assert rel_err(r.gamma_n[0, :, :, b1, b2], x.T) < 1e-9
        assert rel_err(A @ r.gamma_n[0, :, :, b1, b2].T, U.T) < 1e-11


def test_constant_gamma_is_recovered_exactly(orc, noise2k, base_run):
    # Upsilon = c N  =>  Gamma_n = c delta_n0  =>  Gamma^x(phi) = c (the 2 pi reading)
    s, r = base_run
    c = 0.3 - 0.2j
    ups = np.zeros_like(r.ups)
    for mu in range(4):
        ups[:, mu] = c * r.norm[:, : s.n_max + 1]
    gam, ns = orc.edge_correct(s, ups, r.norm)
    assert ns == 0
    expect = np.zeros_like(gam)
    expect[:, :, s.n_max] = c
    assert rel_err(gam, expect) < 1e-10
    gx = orc.to_gamma(s, gam, 0)
    np.testing.assert_allclose(gx, c, rtol=0, atol=1e-10)


def test_singular_systems_are_reported(orc):
    s = orc.Setup(n_bins=2, theta_min=1.0, theta_max=4.0, n_max=2)
    ups = np.zeros((1, 4, 3, 2, 2), complex)
    norm = np.zeros((1, 5, 2, 2), complex)
    norm[0, 0, 0, 0] = 1.0  # only (b1, b2) = (0, 0) has triplets
    gam, ns = orc.edge_correct(s, ups, norm)
    assert ns == 3
    assert np.isnan(gam[0, :, :, 1, 1]).all() and np.isfinite(gam[0, :, :, 0, 0]).all()


# ------------------------------------------ P4: Fourier convergence to the binned triplet sums

def _merge0(a):
    out = a[..., :-1].copy()
    out[..., 0] += a[..., -1]
    return out


def test_multipoles_converge_to_binned_triplet_sums(orc):
    rng = np.random.default_rng(3)
    n = 40
    xy = rng.uniform(0, 6, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    cat = hand_catalog(xy, g, rng.uniform(0.5, 1.5, n))
    nphib = 6
    edges = np.linspace(0, 2 * np.pi, nphib + 1)
    errs_u, errs_n = [], []
    ref = None
    for nmax in (10, 40, 160, 640):
        s = orc.Setup(n_bins=3, theta_min=0.5, theta_max=6.0, n_max=nmax)
        if ref is None:
            ref = orc.brute(s, cat, n_phib=nphib)
        G, W = orc.moments(s, cat)
        ups, norm = orc.contract(s, cat, G, W)
        ns = np.arange(-nmax, nmax + 1)
        # integral of e^{i n phi} over each angular bin
        I = np.empty((ns.size, nphib), complex)
        for k in range(nphib):
            a, b = edges[k], edges[k + 1]
            with np.errstate(divide="ignore", invalid="ignore"):
                I[:, k] = np.where(ns == 0, b - a, (np.exp(1j * ns * b) - np.exp(1j * ns * a)) / (1j * ns))
        rec_u = np.zeros_like(ref.ups_b)
        rec_n = np.zeros_like(ref.norm_b)
        for b1 in range(3):
            for b2 in range(3):
                U, A = _extended(s, ups, norm, 0, b1, b2)
                Nn = np.array([A[l + nmax, nmax] for l in range(-nmax, nmax + 1)])  # N_l
                rec_u[0, :, b1, b2] = U @ I / (2 * np.pi)
                rec_n[0, b1, b2] = Nn @ I / (2 * np.pi)
        # degenerate triplets (j = k) sit exactly at phi = 0, an angular bin edge, where a
        # Fourier partial sum splits their weight evenly; merge the two bins around phi = 0
        errs_u.append(rel_err(_merge0(rec_u), _merge0(ref.ups_b)))
        errs_n.append(rel_err(_merge0(rec_n), _merge0(ref.norm_b)))
    assert all(a > b for a, b in zip(errs_u, errs_u[1:])), errs_u
    assert all(a > b for a, b in zip(errs_n, errs_n[1:])), errs_n
    # a Fourier partial sum integrated over a bin converges like 1/n_max away from its edges
    assert errs_u[-1] < 0.12 * errs_u[0] and errs_n[-1] < 0.12 * errs_n[0]


def test_to_gamma_converges_to_binned_triplet_sums(orc):
    """orc_to_gamma against the brute-force angular bins, in both projections (Sec. 3.4, the
    multipole series of Gamma; Sec. 2.3, Eqs. X2Centroid0-3; the binned sums of Sec. 2.4).

    Fed the multipoles Upsilon_n themselves (extended to n < 0 by the edge correction with a unit
    mode-coupling matrix, i.e. N_0 = 1 and N_m = 0 otherwise), to_gamma returns
    sum_n Upsilon_n e^{i n phi}, which tends to 2 pi times the triplet density in phi; its average
    over an angular bin of width 2 pi / K then tends to K times the brute-force sum of that bin.
    The averages are taken over 512 points of to_gamma's own phi grid per bin. In the centroid
    projection the brute force applies each triplet's own factor at its exact radii, to_gamma
    the factor at the radial nodes, so narrow radial bins are used and only b1 != b2 blocks are
    compared (for b1 = b2 the exact factor of a nearly isosceles triplet flips sign near
    phi = pi). Projection 2, the bin average in closed form (Sec. 2.4, the binned 3PCF), on the
    brute force's own bins converges the same way and matches the sampled averages. A flipped
    exponent (Gamma(-phi) returned for Gamma(phi)) does not converge."""
    rng = np.random.default_rng(7)
    n = 400
    xy = rng.uniform(0, 10, (n, 2))
    g = rng.normal(0, 0.3, n) + 1j * rng.normal(0, 0.3, n)
    cat = hand_catalog(xy, g, rng.uniform(0.5, 1.5, n))
    K, S = 6, 512
    setup = dict(n_bins=3, theta_min=2.0, theta_max=2.1)
    ref = orc.brute(orc.Setup(**setup, n_max=2), cat, n_phib=K)
    off = ~np.eye(setup["n_bins"], dtype=bool)

    def bin_avg(out):
        return out.reshape(out.shape[:-1] + (K, S)).mean(-1) / K

    ex, ec, eflip, eb = [], [], [], []
    for nmax in (10, 40, 160, 640):
        s = orc.Setup(**setup, n_max=nmax)
        G, W = orc.moments(s, cat)
        ups, norm = orc.contract(s, cat, G, W)
        unit = np.zeros_like(norm)
        unit[:, 0] = 1.0
        ext, ns = orc.edge_correct(s, ups, unit)
        assert ns == 0
        sp = orc.Setup(**setup, n_max=nmax, n_phi=K * S)
        out0, out1 = orc.to_gamma(sp, ext, 0), orc.to_gamma(sp, ext, 1)
        # degenerate triplets (j = k) sit at phi = 0, a bin edge: merge the bins around it
        ex.append(rel_err(_merge0(bin_avg(out0)), _merge0(ref.ups_b)))
        eflip.append(rel_err(_merge0(bin_avg(out0[..., ::-1])), _merge0(ref.ups_b)))
        ec.append(rel_err(bin_avg(out1)[:, :, off], ref.upsc_b[:, :, off]))
        # projection 2 (the bin average in closed form) on the brute force's own K bins
        out2 = orc.to_gamma(orc.Setup(**setup, n_max=nmax, n_phi=K), ext, 2) / K
        eb.append(rel_err(_merge0(out2), _merge0(ref.ups_b)))
        assert rel_err(out2, bin_avg(out0)) < 2e-3  # 512 point samples per bin vs the closed form
    assert all(a > b for a, b in zip(eb, eb[1:])), eb
    assert all(a > b for a, b in zip(ex, ex[1:])), ex
    assert all(a > b for a, b in zip(ec, ec[1:])), ec
    assert ex[-1] < 0.25 * ex[0] and ec[-1] < 0.35 * ec[0], (ex, ec)
    assert min(eflip) > 10 * ex[-1], eflip


# ------------------------------------- P6: aperture filters against their defining integrals

def _F_by_integration(mu, t1, t2, phi, th, n=801):
    """2 pi t1 t2 * integral over the aperture position of prod_a Q_a(|y_a|) times the spin
    phases of Eq. MapGamma and the centroid projection; the conjugate sits at vertex mu."""
    th = np.asarray(th, float)
    v1, v2 = t1 + 0j, t2 * np.exp(1j * phi)
    q = [-(v1 + v2) / 3, (2 * v1 - v2) / 3, (2 * v2 - v1) / 3]
    L = 9 * th.max() + max(t1, t2)
    xs = np.linspace(-L, L, n)
    h = xs[1] - xs[0]
    X, Y = np.meshgrid(xs, xs)
    y1 = X + 1j * Y - (v1 + v2) / 3
    tot = np.ones_like(y1)
    for a, ya in enumerate((y1, y1 + v1, y1 + v2)):
        Qe = np.exp(-np.abs(ya) ** 2 / (2 * th[a] ** 2)) / (4 * np.pi * th[a] ** 4)
        if mu == a + 1:
            tot *= ya ** 2 * Qe * (np.conj(q[a]) / q[a])
        else:
            tot *= np.conj(ya) ** 2 * Qe * (q[a] / np.conj(q[a]))
    return 2 * np.pi * t1 * t2 * tot.sum() * h * h


def test_Q_filter_is_normalised():
    th = 1.7
    r = np.linspace(0, 20 * th, 200001)
    Q = r ** 2 / (4 * np.pi * th ** 4) * np.exp(-r ** 2 / (2 * th ** 2))
    assert abs(np.trapezoid(2 * np.pi * r * Q, r) - 1.0) < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_filters_match_their_defining_integrals(orc, seed):
    rng = np.random.default_rng(seed)
    th = rng.uniform(1.0, 3.0, 3)
    t1, t2 = rng.uniform(0.5, 4.0, 2)
    phi = rng.uniform(0, 2 * np.pi)
    for mu in range(4):
        a = orc.filter_F(mu, t1, t2, phi, th)
        b = _F_by_integration(mu, t1, t2, phi, th)
        assert abs(a - b) < 1e-10 * abs(b), (mu, a, b)


def test_centroid_factors_are_pure_phases(orc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        t1, t2, phi = rng.uniform(0.5, 5), rng.uniform(0.5, 5), rng.uniform(0, 2 * np.pi)
        for mu in range(4):
            assert abs(abs(orc.cen_factor(mu, t1, t2, phi)) - 1) < 1e-14


def test_eight_measure_combination_inverts_the_products(orc):
    # c_mu = <M1^(*) M2^(*) M3^(*)> with M = Map + i Mx; Eqs. MapTrafo8_1-8 recover the 8 products
    rng = np.random.default_rng(11)
    Mp = rng.normal(size=(3, 50000))
    Mx = rng.normal(size=(3, 50000)) * 0.7 + 0.3 * Mp
    M = Mp + 1j * Mx
    c = np.array([np.mean(M[0] * M[1] * M[2]), np.mean(np.conj(M[0]) * M[1] * M[2]),
                  np.mean(M[0] * np.conj(M[1]) * M[2]), np.mean(M[0] * M[1] * np.conj(M[2]))])
    P, X = Mp, Mx
    want = [np.mean(P[0] * P[1] * P[2]), np.mean(X[0] * P[1] * P[2]), np.mean(P[0] * X[1] * P[2]),
            np.mean(P[0] * P[1] * X[2]), np.mean(P[0] * X[1] * X[2]), np.mean(X[0] * P[1] * X[2]),
            np.mean(X[0] * X[1] * P[2]), np.mean(X[0] * X[1] * X[2])]
    np.testing.assert_allclose(orc.combine8(c), want, rtol=1e-12, atol=1e-14)


def test_four_measure_combination_recovers_the_products(orc):
    """Eqs. MapTrafo4_1-4, with the conjugate of each one-conjugate correlator on the last radius of
    its ordering: from <M^3>(t1,t2,t3) and A123 = <M1 M2 M3^*>, A132 = <M1 M3 M2^*>,
    A231 = <M2 M3 M1^*> they return Map^3, <Map^2 Mx>, <Map Mx^2>, <Mx^3> at (t1,t2,t3) exactly,
    whatever the joint distribution of the fields (sample moments of one set of fields obey the
    relabelling symmetries as identities). With the conjugate on the first radius the printed
    orderings (t1,t2,t3) and (t1,t3,t2) coincide and no term conjugates t3, which fails here."""
    rng = np.random.default_rng(12)
    P = rng.normal(size=(3, 40000))
    X = rng.normal(size=(3, 40000)) * 0.6 + 0.4 * P[[1, 2, 0]]
    P = P + 0.3 * P[[2, 0, 1]] ** 2  # skewed, correlated, distinct per radius
    M = P + 1j * X

    def last_conj(a, b, c):
        return np.mean(M[a] * M[b] * np.conj(M[c]))

    m3 = np.mean(M[0] * M[1] * M[2])
    got = orc.combine4(m3, last_conj(0, 1, 2), last_conj(0, 2, 1), last_conj(1, 2, 0))
    want = [np.mean(P[0] * P[1] * P[2]), np.mean(P[0] * P[1] * X[2]), np.mean(P[0] * X[1] * X[2]),
            np.mean(X[0] * X[1] * X[2])]
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-13)

    def first_conj(a, b, c):
        return np.mean(np.conj(M[a]) * M[b] * M[c])

    wrong = orc.combine4(m3, first_conj(0, 1, 2), first_conj(0, 2, 1), first_conj(1, 2, 0))
    assert np.abs(wrong - want).max() > 1e-3


@pytest.mark.slow
def test_four_and_eight_equation_forms_agree_within_quadrature(orc):
    """App. C: on a noise-free lognormal field the four-equation Map^3 (built from Gamma_0 and
    Gamma_1 alone) and the eight-equation one (all four Gamma_mu) agree to the accuracy of the
    estimated 3PCF's binning, truncation to [theta_min, theta_max] and quadrature (a few per cent
    at these coarse bins), and both give small parity-odd <Mx^3>."""
    cat = make_catalog(12000, 80.0, 3, field="lognormal", sigma_e=0.0, weights="unit", ngrid=1024)
    s = orc.Setup(n_bins=20, theta_min=0.25, theta_max=25.0, n_max=16)
    th = [[3.0, 3.0, 3.0], [2.0, 3.0, 4.0]]
    r = orc.pipeline(s, cat, th)
    m4 = orc.to_map3_four(s, r.gamma_cen, th)[0]
    m8 = r.m8[0]
    assert np.all(m8[:, 0] > 0) and np.all(m4[:, 0] > 0)
    np.testing.assert_allclose(m4[:, 0], m8[:, 0], rtol=0.05)
    assert np.all(np.abs(m4[:, 3]) < 0.05 * m4[:, 0]) and np.all(np.abs(m8[:, 7]) < 0.05 * m8[:, 0])


# --------------------------------------------- P7: physics check on a parity-even lognormal field

@pytest.mark.slow
def test_lognormal_field_has_E_modes_only(orc):
    cat = make_catalog(12000, 100.0, 21, field="lognormal", sigma_e=0.0, weights="unit", ngrid=1024)
    s = orc.Setup(n_bins=14, theta_min=0.5, theta_max=30.0, n_max=10)
    r = orc.pipeline(s, cat, [[2.0, 2.0, 2.0], [3.0, 3.0, 3.0]])
    m8 = r.m8[0]
    assert np.all(m8[:, 0] > 0)  # skewed convergence field: positive Map^3
    for k in (1, 2, 3, 7):  # parity-odd measures vanish
        assert np.all(np.abs(m8[:, k]) < 0.1 * m8[:, 0]), m8
