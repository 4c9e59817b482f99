"""Checkpoint / resume over centre chunks (additivity of Upsilon and N over centres, App. B):
an interrupted run resumed from its checkpoint ends bit-identical to an uninterrupted chunked run,
and both agree with the single-pass measurement."""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_resume_after_interruption(gpu, noise2k, tmp_path, precision):
    from paper_2309_08601_gb300 import checkpoint
    dev = gpu.catalog_to_device(noise2k)
    with gpu.Estimator(**S0, precision=precision) as est:
        whole = checkpoint.measure_resumable(est, *dev[:5], TH0, str(tmp_path / "a.npz"), n_chunks=5)
        assert checkpoint.measure_resumable(est, *dev[:5], TH0, str(tmp_path / "b.npz"), n_chunks=5,
                                            stop_after=2) is None  # interrupted after 2 chunks
        resumed = checkpoint.measure_resumable(est, *dev[:5], TH0, str(tmp_path / "b.npz"), n_chunks=5)
        single = est.measure(*dev[:5], theta_ap=TH0)
    assert torch.equal(whole.upsilon, resumed.upsilon) and torch.equal(whole.norm, resumed.norm)
    assert torch.equal(whole.m8, resumed.m8)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rel_err(whole.upsilon.cpu().numpy(), single.upsilon.cpu().numpy()) < tol
    assert rel_err(whole.m8.cpu().numpy(), single.m8.cpu().numpy()) < (1e-10 if precision == "fp64" else 1e-4)
