"""Batching form: many (tomographic) catalogs of uneven sizes through mp3pcf_run_batch with
captured CUDA graphs, and the tile-shape autotuner.

The batch path must give bit-identical aperture measures to running each catalog on its own with
the same fixed extent (the kernels are deterministic and a CUDA graph replays the same launches),
both with and without graphs; and it must agree with the FP64 oracle (tomographic, all Z-triplets).
"""
import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import synth
from tests._util import rel_err

pytestmark = pytest.mark.gpu

SET = dict(n_bins=8, theta_min=0.5, theta_max=15.0, n_max=8, n_z=3)
TH = [[2.0, 2.0, 2.0], [4.0, 4.0, 4.0]]
SIDE = 60.0


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.fixture(scope="module")
def mocks():
    # tomographic realisations with uneven counts per bin (the C3 recipe, smaller)
    return [synth.make_tomographic_catalog(100 + r, side=SIDE, n_z=3, n_range=(1500, 6000), ngrid=512)
            for r in range(5)]


def _extent(side, quantum=synth.QUANTUM):
    return (0, 0, int(np.ceil(side / quantum)), int(np.ceil(side / quantum)))


def _dev(api, cat):
    t = api.catalog_to_device(cat)
    return t[:5] + (t[5],)


@pytest.mark.parametrize("precision", ["bf16x3", "fp64"])
def test_batch_equals_individual_runs(gpu, mocks, precision):
    cats = [_dev(gpu, c) for c in mocks]
    ext = _extent(SIDE)
    with gpu.Estimator(**SET, precision=precision) as est:
        m_graph = est.run_batch(cats, ext, TH, use_graphs=True).cpu().numpy()
        launches, inst = est.graph_stats()
        print("run_batch note:", est.last_error())
        m_direct = est.run_batch(cats, ext, TH, use_graphs=False).cpu().numpy()
        est.set_extent(ext)
        single = []
        for c in cats:
            m = est.measure(*c[:5], theta_ap=TH, zbin=c[5], report_singular=False)
            single.append(m.m8.cpu().numpy())
        est.set_extent(None)
    assert launches == len(cats) - 1 and inst >= 1  # every catalog but the first was a graph replay
    print(precision, "graph launches", launches, "instantiations", inst)
    np.testing.assert_array_equal(m_graph, m_direct)
    np.testing.assert_array_equal(m_graph, np.stack(single))


def test_batch_against_oracle(gpu, orc, mocks):
    cat = mocks[2]
    s = orc.Setup(**SET)
    r = orc.pipeline(s, cat, TH)
    with gpu.Estimator(**SET, precision="fp64") as est:
        m64 = est.run_batch([_dev(gpu, c) for c in mocks], _extent(SIDE), TH)[2].cpu().numpy()
    with gpu.Estimator(**SET, precision="bf16x3") as est:
        m32 = est.run_batch([_dev(gpu, c) for c in mocks], _extent(SIDE), TH)[2].cpu().numpy()
    assert rel_err(m64, r.m8) < 1e-10
    # the precision form against the oracle, Map^3 of the auto-correlation triplets (signal-bearing)
    auto = [(z * 3 + z) * 3 + z for z in range(3)]
    print("bf16x3 Map^3 error (auto triplets)", rel_err(m32[auto, :, 0], r.m8[auto, :, 0]))
    assert rel_err(m32[auto, :, 0], r.m8[auto, :, 0]) < 1e-4


def test_positions_outside_the_extent_are_rejected(gpu, mocks):
    from paper_2309_08601_gb300 import native
    cats = [_dev(gpu, c) for c in mocks[:2]]
    small = _extent(SIDE / 2)
    with gpu.Estimator(**SET, precision="bf16x3") as est:
        with pytest.raises(native.Mp3pcfError) as ei:
            est.run_batch(cats, small, TH)
        assert ei.value.status == native.EINVAL


def test_autotuner_picks_a_measured_candidate(gpu, mocks):
    from paper_2309_08601_gb300 import autotune
    cat = _dev(gpu, mocks[0])
    res = autotune.tune(SET, cat, "bf16x3", occupancies=(2, 4, 8), slices=(0, 4, 16), repeats=1)
    assert res["cell_occupancy"] in (2, 4, 8) and res["contract_slices"] in (0, 4, 16)
    assert res["moments_ms"] == min(res["trials"]["moments"].values())
    # the tuned shapes change the launch, not the result (up to FP32 summation order)
    with gpu.Estimator(**SET, precision="bf16x3") as e0, \
            gpu.Estimator(**SET, precision="bf16x3", cell_occupancy=res["cell_occupancy"],
                          contract_slices=res["contract_slices"]) as e1:
        a = e0.measure(*cat[:5], theta_ap=TH, zbin=cat[5], report_singular=False).upsilon.cpu().numpy()
        b = e1.measure(*cat[:5], theta_ap=TH, zbin=cat[5], report_singular=False).upsilon.cpu().numpy()
    assert rel_err(a, b) < 1e-5
