"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (normwise, max|gpu - oracle| / max|oracle| per output array): 1e-10 for the FP64
path; 1e-4 for the FP32 path on every multipole output, and on Map^3 for a signal-bearing
catalog. On a pure-noise catalog Map^3 is a cancellation residual and the FP32 path is only
reported there.
"""
import numpy as np
import pytest

from paper_2309_08601_gb300 import synth
from tests._util import hand_catalog, rel_err

pytestmark = pytest.mark.gpu

S0 = dict(n_bins=10, theta_min=0.5, theta_max=30.0, n_max=10)
TH0 = [[2.0, 2.0, 2.0], [4.0, 4.0, 4.0], [8.0, 8.0, 8.0]]


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


def run(api, cat, setup, precision, theta=TH0, centres=None, stages="all"):
    import torch
    dev = api.catalog_to_device(cat)
    mask = None
    if centres is not None:
        m = np.zeros(cat.n, np.uint8)
        m[np.asarray(centres)] = 1
        mask = torch.as_tensor(m, device="cuda")
    out = {}
    with api.Estimator(**setup, precision=precision) as est:
        est.accumulate_moments(*dev, centre_mask=mask)
        out["n_centres"], out["n_pairs"] = est.counts()
        G, W = est.moments()
        out["G"], out["W"] = G.cpu().numpy(), W.cpu().numpy()
        if stages == "moments":
            return out
        ups, norm = est.contract()
        out["ups"], out["norm"] = ups.cpu().numpy(), norm.cpu().numpy()
        gam, ns = est.edge_correct(ups, norm)
        out["gamma_n"], out["n_singular"] = gam.cpu().numpy(), ns
        gx = est.to_gamma(gam, 0)
        gc = est.to_gamma(gam, 1)
        corr, m8 = est.to_map3(gc, theta)
        out["gamma_x"], out["gamma_cen"] = gx.cpu().numpy(), gc.cpu().numpy()
        out["corr"], out["m8"] = corr.cpu().numpy(), m8.cpu().numpy()
    return out


def oracle_run(orc, cat, setup, theta=TH0, centres=None):
    s = orc.Setup(**setup)
    r = orc.pipeline(s, cat, theta, None if centres is None else np.sort(np.asarray(centres)))
    return s, r


def compare(g, r, tol, keys=("G", "W", "ups", "norm", "gamma_n", "gamma_x", "gamma_cen", "corr", "m8")):
    ref = {"G": r.G, "W": r.W, "ups": r.ups, "norm": r.norm, "gamma_n": r.gamma_n,
           "gamma_x": r.gamma_x, "gamma_cen": r.gamma_cen, "corr": r.corr, "m8": r.m8}
    errs = {k: rel_err(g[k], ref[k]) for k in keys}
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (errs, tol)
    return errs


# ------------------------------------------------------------- 2000-galaxy noise catalog

@pytest.fixture(scope="module")
def noise_ref(orc, noise2k):
    return oracle_run(orc, noise2k, S0)


def test_fp64_path_matches_oracle_on_every_output(gpu, orc, noise2k, noise_ref):
    s, r = noise_ref
    g = run(gpu, noise2k, S0, "fp64")
    assert g["n_pairs"] == orc.count_pairs(s, noise2k)
    assert g["n_singular"] == r.n_singular
    compare(g, r, 1e-10)


def test_fp32_path_matches_oracle(gpu, orc, noise2k, noise_ref):
    s, r = noise_ref
    g = run(gpu, noise2k, S0, "fp32")
    assert g["n_pairs"] == orc.count_pairs(s, noise2k)  # identical binning decisions
    errs = compare(g, r, 1e-4, keys=("G", "W", "ups", "norm", "gamma_n", "gamma_x", "gamma_cen"))
    print("fp32 errors", errs, "Map3 (pure noise, not gated):", rel_err(g["m8"], r.m8))


def test_four_equation_form_matches_oracle(gpu, orc, noise2k, noise_ref):
    """mp3pcf_to_map3_four (App. C, Eqs. MapTrafo4_1-4) against the oracle's four-equation form,
    with equal and unequal radii (the orderings of the one-conjugate correlator differ only for
    unequal ones)."""
    import torch
    s, r = noise_ref
    th = [[2.0, 2.0, 2.0], [1.5, 2.5, 4.0], [4.0, 1.5, 2.5]]
    want = orc.to_map3_four(s, r.gamma_cen, th)
    with gpu.Estimator(**S0, precision="fp64") as est:
        gc = torch.as_tensor(r.gamma_cen, device="cuda")
        got = est.to_map3_four(gc, th).cpu().numpy()
    assert rel_err(got, want) < 1e-10, rel_err(got, want)


def test_bin_averaged_projection_matches_oracle(gpu, orc, noise2k, noise_ref):
    """to_gamma projection 2 (the x-projection averaged over each angular bin) against the oracle."""
    import torch
    s, r = noise_ref
    want = orc.to_gamma(s, r.gamma_n, 2)
    with gpu.Estimator(**S0, precision="fp64") as est:
        got = est.to_gamma(torch.as_tensor(r.gamma_n, device="cuda"), 2).cpu().numpy()
    assert rel_err(got, want) < 1e-10, rel_err(got, want)


def test_fp64_is_deterministic(gpu, noise2k):
    a = run(gpu, noise2k, S0, "fp64", stages="all")
    b = run(gpu, noise2k, S0, "fp64", stages="all")
    for k in ("G", "W", "ups", "norm", "gamma_n", "m8"):
        np.testing.assert_array_equal(a[k], b[k])


def test_centre_subsets_add_up(gpu, noise2k):
    idx = np.arange(noise2k.n)
    a = run(gpu, noise2k, S0, "fp64", centres=idx[::2])
    b = run(gpu, noise2k, S0, "fp64", centres=idx[1::2])
    full = run(gpu, noise2k, S0, "fp64")
    assert rel_err(a["ups"] + b["ups"], full["ups"]) < 1e-12
    assert rel_err(a["norm"] + b["norm"], full["norm"]) < 1e-12
    assert a["n_pairs"] + b["n_pairs"] == full["n_pairs"]


# ------------------------------------------------------------- signal-bearing lognormal field

@pytest.fixture(scope="module")
def lognormal_small():
    return synth.make_catalog(12000, 100.0, 21, field="lognormal", sigma_e=0.0, weights="uniform",
                              ngrid=1024)


def test_fp32_map3_on_a_lognormal_field(gpu, orc, lognormal_small):
    setup = dict(n_bins=14, theta_min=0.5, theta_max=30.0, n_max=10)
    th = [[2.0, 2.0, 2.0], [3.0, 3.0, 3.0], [2.0, 3.0, 4.0]]
    s, r = oracle_run(orc, lognormal_small, setup, th)
    g64 = run(gpu, lognormal_small, setup, "fp64", th)
    compare(g64, r, 1e-10)
    g32 = run(gpu, lognormal_small, setup, "fp32", th)
    compare(g32, r, 1e-4)
    assert r.m8[0, :2, 0].min() > 0


# ------------------------------------------------------------- the full-size workload, sampled

@pytest.fixture(scope="module")
def lognormal_200k():
    return synth.workload_catalog("lognormal_200k")


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-10)])
def test_full_size_catalog_sampled_centres(gpu, orc, lognormal_200k, precision, tol):
    """All 200k galaxies are neighbours; 40 sampled centres are compared row by row."""
    p = synth.WORKLOADS["lognormal_200k"]
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                 n_max=p["n_max"])
    rng = np.random.default_rng(9)
    centres = np.sort(rng.choice(lognormal_200k.n, 40, replace=False))
    s = orc.Setup(**setup)
    G, W = orc.moments(s, lognormal_200k, centres)
    g = run(gpu, lognormal_200k, setup, precision, centres=centres, stages="moments")
    assert g["n_pairs"] == orc.count_pairs(s, lognormal_200k, centres)
    assert rel_err(g["G"], G) < tol and rel_err(g["W"], W) < tol
    ups, norm = orc.contract(s, lognormal_200k, G, W, centres)
    g2 = run(gpu, lognormal_200k, setup, precision, centres=centres, stages="all")
    assert rel_err(g2["ups"], ups) < tol and rel_err(g2["norm"], norm) < tol


def test_full_size_run_sampled_rows(gpu, orc, lognormal_200k):
    """The bench configuration (every galaxy a centre, FP32): sampled rows of G, W."""
    import torch
    from paper_2309_08601_gb300 import api
    p = synth.WORKLOADS["lognormal_200k"]
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                 n_max=p["n_max"])
    dev = api.catalog_to_device(lognormal_200k)
    with api.Estimator(**setup, precision="fp32") as est:
        est.accumulate_moments(*dev)
        nc, npairs = est.counts()
        G, W = est.moments()
        rng = np.random.default_rng(10)
        rows = np.sort(rng.choice(lognormal_200k.n, 24, replace=False))
        Gs, Ws = G[torch.as_tensor(rows, device="cuda")].cpu().numpy(), W[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        del G, W
    s = orc.Setup(**setup)
    Go, Wo = orc.moments(s, lognormal_200k, rows)
    assert nc == lognormal_200k.n
    assert rel_err(Gs, Go) < 1e-4 and rel_err(Ws, Wo) < 1e-4
    assert npairs > 1e10


# ------------------------------------------------------------- edge cases

def test_empty_catalog(gpu):
    cat = hand_catalog(np.zeros((0, 2)), np.zeros(0))
    g = run(gpu, cat, S0, "fp32")
    assert g["n_centres"] == 0 and g["n_pairs"] == 0
    assert not np.abs(g["ups"]).any() and not np.abs(g["norm"]).any()
    assert g["n_singular"] == S0["n_bins"] ** 2 and np.isnan(g["gamma_n"]).all()


def test_single_and_coincident_galaxies(gpu, orc):
    cat = hand_catalog([[0, 0], [0, 0], [5, 0]], [0.1, 0.2j, -0.1])
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        g = run(gpu, cat, S0, prec, stages="moments")
        G, W = orc.moments(orc.Setup(**S0), cat)
        assert rel_err(g["G"], G) < tol and rel_err(g["W"], W) < tol
    one = hand_catalog([[3, 3]], [0.1])
    g = run(gpu, one, S0, "fp64")
    assert g["n_pairs"] == 0 and g["n_singular"] == S0["n_bins"] ** 2


def test_pairs_exactly_on_bin_edges(gpu, orc):
    s = orc.Setup(**S0)
    _, e2 = orc.edges(s)
    x0 = 5_000_000
    xs, ys = [x0], [x0]
    for b in range(1, S0["n_bins"]):
        d = int(np.ceil(np.sqrt(float(e2[b]))))
        while d * d < e2[b]:
            d += 1
        while (d - 1) * (d - 1) >= e2[b]:
            d -= 1
        xs += [x0 + d, x0 - (d - 1)]  # on the edge (upper bin) and just inside (lower bin)
        ys += [x0, x0]
    from paper_2309_08601_gb300.synth import Catalog
    n = len(xs)
    rng = np.random.default_rng(1)
    cat = Catalog(np.array(xs, np.int32), np.array(ys, np.int32), rng.normal(0, .3, n).astype(np.float32),
                  rng.normal(0, .3, n).astype(np.float32), np.ones(n, np.float32), None, 0.0, synth.QUANTUM)
    G, W = orc.moments(s, cat)
    for prec in ("fp64", "fp32"):
        g = run(gpu, cat, S0, prec, stages="moments")
        np.testing.assert_array_equal(g["W"][..., 0].real, W[..., 0].real)  # pair counts per bin
        assert g["n_pairs"] == orc.count_pairs(s, cat)


@pytest.mark.parametrize("n", [1, 31, 33, 1025])
def test_ragged_sizes_dense_field(gpu, orc, n):
    rng = np.random.default_rng(n)
    cat = hand_catalog(rng.uniform(0, 12, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n))
    setup = dict(n_bins=5, theta_min=0.2, theta_max=6.0, n_max=7)
    s, r = oracle_run(orc, cat, setup, [[1.0, 1.0, 1.0]])
    g = run(gpu, cat, setup, "fp64", [[1.0, 1.0, 1.0]])
    compare(g, r, 1e-10, keys=("G", "W", "ups", "norm"))


def test_tomographic_fp64(gpu, orc):
    rng = np.random.default_rng(4)
    n = 900
    cat = hand_catalog(rng.uniform(0, 30, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n), rng.integers(0, 3, n))
    setup = dict(n_bins=6, theta_min=0.5, theta_max=10.0, n_max=5, n_z=3)
    th = [[2.0, 2.0, 2.0]]
    s, r = oracle_run(orc, cat, setup, th)
    g = run(gpu, cat, setup, "fp64", th)
    compare(g, r, 1e-10, keys=("G", "W", "ups", "norm", "gamma_n", "gamma_cen", "m8"))


@pytest.mark.parametrize("n_max", [0, 3, 17, 50])
def test_other_orders(gpu, orc, n_max):
    rng = np.random.default_rng(n_max)
    n = 400
    cat = hand_catalog(rng.uniform(0, 20, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n))
    setup = dict(n_bins=4, theta_min=0.5, theta_max=8.0, n_max=n_max)
    s, r = oracle_run(orc, cat, setup, [[2.0, 2.0, 2.0]])
    compare(run(gpu, cat, setup, "fp64", [[2.0, 2.0, 2.0]]), r, 1e-10,
            keys=("G", "W", "ups", "norm", "gamma_n", "gamma_cen", "m8"))
    compare(run(gpu, cat, setup, "fp32", [[2.0, 2.0, 2.0]]), r, 1e-4, keys=("G", "W", "ups", "norm"))


def test_invalid_inputs_are_rejected(gpu):
    from paper_2309_08601_gb300 import native
    cat = hand_catalog([[0, 0], [1, 0]], [0.1, 0.1], zbin=[0, 5])
    dev = gpu.catalog_to_device(cat)
    with gpu.Estimator(**S0, n_z=2) as est:
        with pytest.raises(native.Mp3pcfError) as ei:  # zbin value >= n_z
            est.accumulate_moments(*dev)
        assert ei.value.status == native.EINVAL
        with pytest.raises(native.Mp3pcfError) as ei:  # n_z > 1 needs zbin
            est.accumulate_moments(*dev[:5])
        assert ei.value.status == native.EINVAL
