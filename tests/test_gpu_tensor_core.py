"""Tensor-core (tcgen05) contraction, BF16x3 and TF32x3 split forms, against the FP64 oracle.

The moments are the FP32 ones in every FP32 mode; only stage (b) differs. Two comparisons:
the whole path against the oracle (normwise tolerance 1e-4, as for the FP32 path), and the
contraction alone against the oracle's FP64 contraction of the SAME FP32 moments the GPU made,
which isolates the split-product error (bounded by about 2^-17 per product for BF16x3 and
2^-21 for TF32x3, plus FP32 accumulation: gated at 2e-5 and 2e-6).
"""
import numpy as np
import pytest

from paper_2309_08601_gb300 import synth
from tests._util import hand_catalog, rel_err
from tests.test_gpu_parity import S0, TH0, compare, oracle_run, run

pytestmark = pytest.mark.gpu

TC = ["bf16x3", "tf32x3"]
ISOLATED_TOL = {"bf16x3": 2e-5, "tf32x3": 2e-6}


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.fixture(scope="module")
def noise_ref(orc, noise2k):
    return oracle_run(orc, noise2k, S0)


@pytest.mark.parametrize("precision", TC)
def test_tensor_core_path_matches_oracle(gpu, orc, noise2k, noise_ref, precision):
    s, r = noise_ref
    g = run(gpu, noise2k, S0, precision)
    assert g["n_pairs"] == orc.count_pairs(s, noise2k)
    errs = compare(g, r, 1e-4, keys=("G", "W", "ups", "norm", "gamma_n", "gamma_x", "gamma_cen"))
    print(precision, errs)


@pytest.mark.parametrize("precision", TC)
def test_contraction_alone_of_the_same_moments(gpu, orc, noise2k, precision):
    """Oracle contraction of the GPU's own FP32 moments: only the split products differ."""
    s = orc.Setup(**S0)
    g = run(gpu, noise2k, S0, precision, stages="all")
    ups, norm = orc.contract(s, noise2k, g["G"].astype(np.complex128), g["W"].astype(np.complex128))
    e_u, e_n = rel_err(g["ups"], ups), rel_err(g["norm"], norm)
    print(precision, "isolated contraction error", e_u, e_n)
    assert e_u < ISOLATED_TOL[precision] and e_n < ISOLATED_TOL[precision]


def test_tensor_core_is_deterministic(gpu, noise2k):
    for p in TC:
        a = run(gpu, noise2k, S0, p)
        b = run(gpu, noise2k, S0, p)
        for k in ("ups", "norm", "gamma_n", "m8"):
            np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("n_bins,n_max", [(1, 0), (7, 5), (31, 4), (32, 3), (33, 3), (64, 2), (4, 50)])
def test_tile_shapes(gpu, orc, n_bins, n_max):
    """Tiles of two sides (n_bins <= 32: Upsilon_0..3 of one order from four moment rows, N tiles
    of two orders; 1 bin: 4 of 128 rows; 31 bins: padded bin rows; 32 bins: all 128 rows and
    N = 128), tiles of one side (33 bins: 66 rows, N = 96; 64 bins: all 128 rows); largest
    order."""
    rng = np.random.default_rng(100 + n_bins)
    n = 500
    cat = hand_catalog(rng.uniform(0, 20, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n))
    setup = dict(n_bins=n_bins, theta_min=0.3, theta_max=9.0, n_max=n_max)
    s = orc.Setup(**setup)
    for p in TC:
        g = run(gpu, cat, setup, p, stages="all")
        ups, norm = orc.contract(s, cat, g["G"].astype(np.complex128), g["W"].astype(np.complex128))
        assert rel_err(g["ups"], ups) < ISOLATED_TOL[p], p
        assert rel_err(g["norm"], norm) < ISOLATED_TOL[p], p


@pytest.mark.parametrize("n_bins", [6, 34])
def test_tomographic_tensor_core(gpu, orc, n_bins):
    """n_z = 3: every Z-triplet's centre range; with two sides per tile (6 bins) Upsilon_1 of a
    triplet comes from the tile of the triplet with Z2 and Z3 exchanged, with one side (34 bins)
    from its own tile."""
    rng = np.random.default_rng(4)
    n = 900
    cat = hand_catalog(rng.uniform(0, 30, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n), rng.integers(0, 3, n))
    setup = dict(n_bins=n_bins, theta_min=0.5, theta_max=10.0, n_max=5, n_z=3)
    th = [[2.0, 2.0, 2.0]]
    s, r = oracle_run(orc, cat, setup, th)
    # with 34 bins this catalog leaves bin pairs without triplets: their edge-correction systems
    # are singular, so the comparison stops at the multipoles
    keys = ("G", "W", "ups", "norm") + (("gamma_n", "gamma_cen") if n_bins <= 8 else ())
    for p in TC:
        g = run(gpu, cat, setup, p, th)
        compare(g, r, 1e-4, keys=keys)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1025])
def test_ragged_centre_counts(gpu, orc, n):
    """Centre counts below, at and across one 32-centre stage, slices of unequal length."""
    rng = np.random.default_rng(n)
    cat = hand_catalog(rng.uniform(0, 12, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n))
    setup = dict(n_bins=5, theta_min=0.2, theta_max=6.0, n_max=7)
    s = orc.Setup(**setup)
    for p in TC:
        g = run(gpu, cat, setup, p, [[1.0, 1.0, 1.0]])
        ups, norm = orc.contract(s, cat, g["G"].astype(np.complex128), g["W"].astype(np.complex128))
        assert rel_err(g["ups"], ups) < ISOLATED_TOL[p] or np.abs(ups).max() == 0
        assert rel_err(g["norm"], norm) < ISOLATED_TOL[p] or np.abs(norm).max() == 0


def test_empty_catalog_tensor_core(gpu):
    cat = hand_catalog(np.zeros((0, 2)), np.zeros(0))
    for p in TC:
        g = run(gpu, cat, S0, p)
        assert g["n_centres"] == 0
        assert not np.abs(g["ups"]).any() and not np.abs(g["norm"]).any()


@pytest.fixture(scope="module")
def lognormal_200k():
    return synth.workload_catalog("lognormal_200k")


@pytest.mark.parametrize("precision", TC)
def test_full_size_sampled_centres(gpu, orc, lognormal_200k, precision):
    """All 200k galaxies as neighbours, 40 sampled centres through the whole contraction."""
    p = synth.WORKLOADS["lognormal_200k"]
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                 n_max=p["n_max"])
    rng = np.random.default_rng(9)
    centres = np.sort(rng.choice(lognormal_200k.n, 40, replace=False))
    s = orc.Setup(**setup)
    G, W = orc.moments(s, lognormal_200k, centres)
    ups, norm = orc.contract(s, lognormal_200k, G, W, centres)
    g = run(gpu, lognormal_200k, setup, precision, centres=centres, stages="all")
    assert rel_err(g["ups"], ups) < 1e-4 and rel_err(g["norm"], norm) < 1e-4


def test_full_size_every_centre_against_fp32_cuda_core_sum(gpu, lognormal_200k):
    """The bench configuration (all 200k centres): the tensor-core sums agree with the FP32
    CUDA-core form (FP64 tile sums) of the same moments to the split-product error."""
    import torch
    from paper_2309_08601_gb300 import api
    p = synth.WORKLOADS["lognormal_200k"]
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                 n_max=p["n_max"])
    dev = api.catalog_to_device(lognormal_200k)
    out = {}
    for prec in ["fp32"] + TC:
        with api.Estimator(**setup, precision=prec) as est:
            est.accumulate_moments(*dev)
            ups, norm = est.contract()
            est.counts()  # raises if a bounded device wait gave up
            out[prec] = (ups.cpu().numpy(), norm.cpu().numpy())
        torch.cuda.empty_cache()
    for prec in TC:
        eu = rel_err(out[prec][0], out["fp32"][0])
        en = rel_err(out[prec][1], out["fp32"][1])
        print(prec, "vs fp32 CUDA-core contraction", eu, en)
        assert eu < 1e-4 and en < 1e-4
