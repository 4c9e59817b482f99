"""The precision-form workload at full size: 10^6 galaxies on a 10 deg x 10 deg patch with
circular holes (15 % masked), 30 bins 0.5'-240', n_max = 40; moments in FP32, contraction in BF16
and in TF32 with hi+lo split products and FP32 accumulation.

Compared with the FP64 oracle on what it can compute one by one: 40 sampled centres (all 10^6
galaxies as neighbours) through moments and contraction, and sampled rows of the moments of the
full all-centre run; at the full size, the two split precisions and the FP32 CUDA-core sum of the
same moments agree with each other, and the Map^3 measures of the three forms agree.
"""
import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import synth
from tests._util import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.fixture(scope="module")
def c2():
    p = synth.WORKLOADS["masked_lognormal_1m"]
    cat = synth.workload_catalog("masked_lognormal_1m")
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"], n_max=p["n_max"])
    return p, cat, setup


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_sampled_centres_against_the_oracle(gpu, orc, c2, precision):
    p, cat, setup = c2
    rng = np.random.default_rng(2)
    centres = np.sort(rng.choice(cat.n, 40, replace=False))
    s = orc.Setup(**setup)
    G, W = orc.moments(s, cat, centres)
    ups, norm = orc.contract(s, cat, G, W, centres)
    dev = gpu.catalog_to_device(cat)
    m = np.zeros(cat.n, np.uint8)
    m[centres] = 1
    with gpu.Estimator(**setup, precision=precision) as est:
        est.accumulate_moments(*dev[:5], centre_mask=torch.as_tensor(m, device="cuda"))
        nc, npairs = est.counts()
        Gg, Wg = est.moments()
        u, n = est.contract()
    assert nc == 40 and npairs == orc.count_pairs(s, cat, centres)
    assert rel_err(Gg.cpu().numpy(), G) < 1e-4 and rel_err(Wg.cpu().numpy(), W) < 1e-4
    eu, en = rel_err(u.cpu().numpy(), ups), rel_err(n.cpu().numpy(), norm)
    print(precision, "40 sampled centres: Upsilon", eu, "N", en)
    assert eu < 1e-4 and en < 1e-4


def test_full_size_all_centres(gpu, orc, c2):
    p, cat, setup = c2
    th = [[t, t, t] for t in (2.0, 4.0, 8.0, 16.0)]
    dev = gpu.catalog_to_device(cat)
    out = {}
    rows = np.sort(np.random.default_rng(3).choice(cat.n, 16, replace=False))
    for prec in ("bf16x3", "tf32x3", "fp32"):
        with gpu.Estimator(**setup, precision=prec) as est:
            m = est.measure(*dev[:5], theta_ap=th, report_singular=False)
            est.counts()
            out[prec] = (m.upsilon.cpu().numpy(), m.norm.cpu().numpy(), m.m8.cpu().numpy())
            if prec == "bf16x3":
                G, W = est.moments()
                idx = torch.as_tensor(rows, device="cuda")
                Gs, Ws = G[idx].cpu().numpy(), W[idx].cpu().numpy()
                del G, W
        torch.cuda.empty_cache()
    s = orc.Setup(**setup)
    Go, Wo = orc.moments(s, cat, rows)
    assert rel_err(Gs, Go) < 1e-4 and rel_err(Ws, Wo) < 1e-4
    for prec in ("bf16x3", "tf32x3"):
        eu = rel_err(out[prec][0], out["fp32"][0])
        en = rel_err(out[prec][1], out["fp32"][1])
        e8 = rel_err(out[prec][2][..., 0], out["fp32"][2][..., 0])
        print(prec, "vs FP32 CUDA-core sum at 10^6: Upsilon", eu, "N", en, "Map^3", e8)
        assert eu < 1e-4 and en < 1e-4 and e8 < 1e-4
