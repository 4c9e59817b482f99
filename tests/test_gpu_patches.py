"""The patch decomposition on the GPU: the catalog measured as 3 x 2 patches (centres of each
patch, members with the theta_max halo, multipoles summed) equals the whole-catalog measurement
(paper App. B, Eq. PatchGamma: additivity over centres), one- and two-z-bin catalogs."""
import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import patches, synth
from tests._util import rel_err
from tests.test_gpu_parity import S0, TH0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_patched_measurement_equals_the_whole_catalog(gpu, noise2k, precision, tol):
    dev = gpu.catalog_to_device(noise2k)
    with gpu.Estimator(**S0, precision=precision) as est:
        whole = est.measure(*dev[:5], theta_ap=TH0, report_singular=False)
        parts = patches.measure_patched(est, noise2k, TH0, 3, 2)
    for a, b in ((parts.upsilon, whole.upsilon), (parts.norm, whole.norm), (parts.m8, whole.m8)):
        assert rel_err(a.cpu().numpy(), b.cpu().numpy()) < tol


def test_patched_tomographic_fp64(gpu):
    cat = synth.make_tomographic_catalog(9, side=50.0, n_z=2, n_range=(1500, 2500), ngrid=512)
    setup = dict(n_bins=6, theta_min=0.5, theta_max=8.0, n_max=6, n_z=2)
    th = [[2.0, 2.0, 2.0]]
    dev = gpu.catalog_to_device(cat)
    with gpu.Estimator(**setup, precision="fp64") as est:
        whole = est.measure(*dev[:5], theta_ap=th, zbin=dev[5], report_singular=False)
        parts = patches.measure_patched(est, cat, th, 2, 2)
    assert rel_err(parts.upsilon.cpu().numpy(), whole.upsilon.cpu().numpy()) < 1e-10
    assert rel_err(parts.m8.cpu().numpy(), whole.m8.cpu().numpy()) < 1e-10
