"""The combined estimator on the GPU (Sec. 3.3): the moments of mp3pcf_accumulate_moments_combined
and the multipoles contracted from them against the oracle's combined moments (FP64 1e-10, FP32
1e-4), tomographic and with centre subsets; the argument checks; and, on a denser noise-free
field, agreement with the discrete estimator and the time it saves."""
import time

import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import synth
from tests._util import rel_err

pytestmark = pytest.mark.gpu

SETUP = dict(n_bins=6, theta_min=0.5, theta_max=8.0, n_max=5)
Q = 1 << 12  # 0.5 arcmin in quanta of 2^-13 arcmin
LEVELS = [(2, Q), (4, 2 * Q)]  # bins from 1.26' on 0.5' pixels, from 3.17' on 1' pixels


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


def _catalog(n_z):
    if n_z == 1:
        cat = synth.make_catalog(3500, 30.0, 21, field="lognormal", weights="uniform", ngrid=512)
    else:
        cat = synth.make_tomographic_catalog(22, side=30.0, n_z=2, n_range=(1500, 2200), ngrid=256)
    cat.w[::97] = 0.0  # zero-weight galaxies: some alone in a pixel without weight
    return cat


@pytest.mark.parametrize("grid_fft", [False, True])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("n_z", [1, 2])
@pytest.mark.parametrize("subset", [False, True])
def test_combined_moments_and_multipoles_match_the_oracle(gpu, orc, precision, tol, n_z, subset, grid_fft):
    """Direct pixel-pair sums and the FFT form (grid_fft) of the grid levels, each against the
    oracle's combined moments (its pixel sums by direct loops) and their contraction."""
    cat = _catalog(n_z)
    rng = np.random.default_rng(7)
    mask = (rng.uniform(size=cat.n) < 0.4).astype(np.uint8) if subset else None
    centres = np.nonzero(mask)[0] if subset else np.arange(cat.n)
    s = orc.Setup(**SETUP, n_z=n_z)
    G0, W0 = orc.combined_moments(s, cat, LEVELS, centres)
    u0, n0 = orc.contract(s, cat, G0, W0, centres)
    dev = gpu.catalog_to_device(cat)
    m = None if mask is None else torch.as_tensor(mask, device=dev[0].device)
    with gpu.Estimator(**SETUP, n_z=n_z, precision=precision, grid_fft=grid_fft) as est:
        est.accumulate_moments_combined(*dev[:5], dev[5], m, levels=LEVELS)
        nc, npairs = est.counts()
        assert nc == len(centres) and npairs > 0
        G, W = est.moments()
        ups, norm = est.contract()
    G, W = G.cpu().numpy(), W.cpu().numpy()
    errs = (rel_err(G, G0), rel_err(W, W0), rel_err(ups.cpu().numpy(), u0), rel_err(norm.cpu().numpy(), n0))
    assert max(errs) < tol, errs
    # the grid bins of a galaxy alone in a weightless pixel are zero on both sides
    assert np.array_equal(G[:, :, 2:] == 0, G0[:, :, 2:] == 0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_fft_grid_moments_equal_the_pixel_pair_sums(gpu, precision, tol):
    """The FFT form of the grid levels against the direct pixel-pair sums on a denser field with
    three levels and many pixels per bin: the same pixel fields, bin tests and angles, so they
    differ by the FFT's rounding only (FP64 ~1e-13, FP32 ~1e-6 normwise)."""
    cat = synth.make_catalog(40000, 60.0, 9, field="lognormal", weights="uniform", ngrid=1024)
    setup = dict(n_bins=12, theta_min=0.5, theta_max=20.0, n_max=8)
    edges = 0.5 * 40.0 ** (np.arange(13) / 12)
    levels = synth.grid_levels(edges, 1 << 10, 2.0 ** -13, ratio=10.0)
    assert len(levels) >= 3
    dev = gpu.catalog_to_device(cat)
    out = {}
    for fft in (False, True):
        with gpu.Estimator(**setup, precision=precision, grid_fft=fft) as est:
            est.accumulate_moments_combined(*dev[:5], levels=levels)
            G, W = est.moments()
            ups, norm = est.contract()
            out[fft] = (G.cpu().numpy(), W.cpu().numpy(), ups.cpu().numpy(), norm.cpu().numpy())
    errs = [rel_err(a, b) for a, b in zip(out[True], out[False])]
    print(precision, "FFT vs pixel pairs (G, W, Upsilon, N):", errs)
    assert max(errs) < tol, errs


def test_all_bins_on_the_grid_and_empty_catalogs(gpu, orc):
    cat = _catalog(1)
    s = orc.Setup(**SETUP)
    G0, W0 = orc.combined_moments(s, cat, [(0, Q)])
    dev = gpu.catalog_to_device(cat)
    with gpu.Estimator(**SETUP, precision="fp64") as est:
        est.accumulate_moments_combined(*dev[:5], levels=[(0, Q)])
        G, W = est.moments()
        assert rel_err(G.cpu().numpy(), G0) < 1e-10 and rel_err(W.cpu().numpy(), W0) < 1e-10
        e = [t[:0] for t in dev[:5]]
        est.accumulate_moments_combined(*e, levels=LEVELS)
        assert est.counts() == (0, 0)
        ups, norm = est.contract()
        assert not ups.abs().any() and not norm.abs().any()


def test_fixed_extent_and_context_reuse(gpu, orc):
    """With a fixed extent the grids start at its lower corner (the oracle given the same extent);
    and one context running catalogs and levels of different sizes in turn gives, bit for bit,
    what a fresh context gives for each (FP64, whose sums run in a fixed order)."""
    cat = _catalog(1)
    s = orc.Setup(**SETUP)
    ext = (int(cat.xq.min()) - 3001, int(cat.yq.min()) - 1777, int(cat.xq.max()) + 999, int(cat.yq.max()) + 5)
    G0, W0 = orc.combined_moments(s, cat, LEVELS, extent=ext)
    G1, _ = orc.combined_moments(s, cat, LEVELS)
    assert rel_err(G1[:, :, 2:], G0[:, :, 2:]) > 1e-3  # the shifted grids change the grid bins
    dev = gpu.catalog_to_device(cat)
    with gpu.Estimator(**SETUP, precision="fp64") as est:
        est.set_extent(ext)
        est.accumulate_moments_combined(*dev[:5], levels=LEVELS)
        G, W = est.moments()
    assert rel_err(G.cpu().numpy(), G0) < 1e-10 and rel_err(W.cpu().numpy(), W0) < 1e-10

    small = synth.make_catalog(800, 20.0, 5, field="noise", weights="uniform")
    big = synth.make_catalog(6000, 40.0, 6, field="lognormal", weights="uniform", ngrid=512)
    seq = [(big, LEVELS), (small, [(1, Q)]), (big, [(3, 2 * Q)]), (small, LEVELS), (big, LEVELS)]

    def run(est, c, lv):
        d = gpu.catalog_to_device(c)
        est.accumulate_moments_combined(*d[:5], levels=lv)
        G, _ = est.moments()
        ups, norm = est.contract()
        return G.cpu().numpy(), ups.cpu().numpy(), norm.cpu().numpy()

    with gpu.Estimator(**SETUP, precision="fp64") as est:
        reused = [run(est, c, lv) for c, lv in seq]
    for (c, lv), got in zip(seq, reused):
        with gpu.Estimator(**SETUP, precision="fp64") as fresh:
            want = run(fresh, c, lv)
        assert all(np.array_equal(a, b) for a, b in zip(got, want)), lv


def test_combined_arguments_are_checked(gpu):
    from paper_2309_08601_gb300 import native
    cat = _catalog(1)
    dev = gpu.catalog_to_device(cat)
    with gpu.Estimator(**SETUP) as est:
        for levels in ([], [(2, Q), (2, 2 * Q)], [(4, Q), (3, Q)], [(6, Q)], [(-1, Q)], [(2, 0)]):
            with pytest.raises(native.Mp3pcfError) as ei:
                est.accumulate_moments_combined(*dev[:5], levels=levels)
            assert ei.value.status == native.EINVAL, levels
        # no adjoint of the grid bins; a plain accumulate call makes the adjoint available again
        est.accumulate_moments_combined(*dev[:5], levels=LEVELS)
        gu, gn = est.new_multipoles()
        with pytest.raises(native.Mp3pcfError) as ei:
            est.moments_adjoint(gu, gn, *dev[2:5])
        assert ei.value.status == native.EUNSUPPORTED
        est.accumulate_moments(*dev[:5])
        est.moments_adjoint(gu, gn, *dev[2:5])
    with gpu.Estimator(**SETUP, exclude_degenerate=True) as est:
        with pytest.raises(native.Mp3pcfError) as ei:
            est.accumulate_moments_combined(*dev[:5], levels=LEVELS)
        assert ei.value.status == native.EUNSUPPORTED


def test_combined_converges_to_the_discrete_estimator_and_is_faster(gpu):
    """500 000 galaxies on 150' (22 per arcmin^2, noise-free lognormal shear), 24 bins 0.25'-60',
    n_max 20. Levels of the paper's accuracy test: 0.25' pixels from 5', 0.5' from 10', 1' from
    20', 2' from 40' (every grid bin 20-40 pixels wide); and the same discrete range on pixels
    half that size (40-80 pixels). Compared with the discrete estimator over every block with a
    grid bin: the multipoles norm-wise (Upsilon n <= 3 and n <= 10, N n <= 20) and the
    centroid-projected Gamma_0 on the equilateral bins, per bin the largest difference over phi
    relative to the largest |Gamma_0| (the paper's measure in Fig. MultiScaleValidation). On this
    field (a sixteenth of the paper's area, so larger sampling fluctuations between neighbouring
    bins) the paper's levels agree to a few per cent; halving the pixels at least halves the
    differences; the blocks of two discrete bins are the discrete estimator's; both combined
    accumulate calls are several times faster than the discrete one."""
    cat = synth.make_catalog(500_000, 150.0, 31, field="lognormal", sigma_e=0.0, weights="uniform")
    dev = gpu.catalog_to_device(cat)
    setup = dict(n_bins=24, theta_min=0.25, theta_max=60.0, n_max=20)
    edges = 0.25 * 240.0 ** (np.arange(25) / 24)
    runs = {"disc": None,
            "paper": synth.grid_levels(edges, 1 << 11, 2.0 ** -13),
            "fine": synth.grid_levels(edges, 1 << 10, 2.0 ** -13, ratio=40)}
    b0 = runs["paper"][0][0]
    assert runs["fine"][0][0] == b0

    def nerr(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def timed(f):
        f()
        torch.cuda.synchronize()
        t = time.perf_counter()
        f()
        torch.cuda.synchronize()
        return time.perf_counter() - t

    out = {}
    with gpu.Estimator(**setup, precision="bf16x3") as est:
        for name, lv in runs.items():
            if lv is None:
                t = timed(lambda: est.accumulate_moments(*dev[:5]))
            else:
                t = timed(lambda: est.accumulate_moments_combined(*dev[:5], levels=lv))
            ups, norm = est.contract()
            gam, _ = est.edge_correct(ups, norm, report_singular=False)
            gc = est.to_gamma(gam, 1)
            out[name] = (t, ups.cpu().numpy(), norm.cpu().numpy(), gc[0, 0].cpu().numpy())
    td, ud, nd, gd = out["disc"]
    grid = np.zeros((24, 24), bool)
    grid[b0:, :] = grid[:, b0:] = True
    res = {}
    for name in ("paper", "fine"):
        tc, uc, nc, gcm = out[name]
        eq = np.array([np.abs(gcm[b, b] - gd[b, b]).max() / np.abs(gd[b, b]).max() for b in range(b0, 24)])
        res[name] = dict(t=tc, e3=nerr(uc[:, :, :4][..., grid], ud[:, :, :4][..., grid]),
                         eu=nerr(uc[:, :, :11][..., grid], ud[:, :, :11][..., grid]),
                         en=nerr(nc[:, :21][..., grid], nd[:, :21][..., grid]),
                         ed=rel_err(uc[..., ~grid], ud[..., ~grid]), eq=eq)
        print("%s levels %s: discrete %.1f ms, combined %.1f ms (x%.1f); grid blocks: Upsilon n<=3 %.4f "
              "n<=10 %.4f N %.5f; discrete block %.2e; equilateral Gamma_0 per bin %s" % (
                  name, runs[name], td * 1e3, tc * 1e3, td / tc, res[name]["e3"], res[name]["eu"],
                  res[name]["en"], res[name]["ed"], np.array2string(eq, precision=4)))
    p, f = res["paper"], res["fine"]
    for r in (p, f):
        assert r["ed"] < 1e-5  # the discrete block is the discrete estimator's (up to the order of the sums)
        assert r["t"] < td / 4
    assert p["eu"] < 0.06 and p["en"] < 0.03 and p["eq"].max() < 0.1
    assert f["e3"] < 0.5 * p["e3"] and f["eu"] < 0.5 * p["eu"] and f["en"] < 0.5 * p["en"]
    assert np.median(f["eq"]) < 0.5 * np.median(p["eq"])
