"""Failure detection, tested without any GPU fault: injections made on the host.

* A bounded wait that runs out: with MP3PCF_INJECT_WAIT_TIMEOUT the tensor-core contraction
  issues no TMA copies, so the converter warps' waits on the copies (about a second) give up,
  every warp role aborts and returns, and mp3pcf_counts reports ETIMEOUT. The context stays
  usable: the next contraction gives the same result as before the injection.
* An allocation failure: MP3PCF_INJECT_ALLOC_FAILURE makes accumulate_moments fail with ENOMEM;
  switched off, the same context works again.
"""
import time

import numpy as np
import pytest
import torch

from tests._util import hand_catalog

pytestmark = pytest.mark.gpu

S = dict(n_bins=6, theta_min=0.5, theta_max=8.0, n_max=5)


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.fixture(scope="module")
def cat600():
    rng = np.random.default_rng(8)
    n = 600
    return hand_catalog(rng.uniform(0, 20, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                        rng.uniform(0.5, 1.5, n))


def test_bounded_wait_gives_up_and_the_context_recovers(gpu, cat600):
    from paper_2309_08601_gb300 import native
    dev = gpu.catalog_to_device(cat600)
    with gpu.Estimator(**S, precision="bf16x3") as est:
        est.accumulate_moments(*dev[:5])
        ref_u, ref_n = est.contract()
        est.counts()
        native.check(native.lib().mp3pcf_inject(est._ctx, native.INJECT_WAIT_TIMEOUT, 1), "inject")
        t0 = time.perf_counter()
        u, n = est.contract()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        with pytest.raises(native.Mp3pcfError) as ei:
            est.counts()
        assert ei.value.status == native.ETIMEOUT
        assert not u.abs().any() and not n.abs().any()
        assert dt < 60.0
        print("contraction with its waits run out returned after %.2f s" % dt)
        native.check(native.lib().mp3pcf_inject(est._ctx, native.INJECT_WAIT_TIMEOUT, 0), "inject")
        est.accumulate_moments(*dev[:5])
        u2, n2 = est.contract()
        est.counts()
        assert torch.equal(u2, ref_u) and torch.equal(n2, ref_n)


def test_injected_allocation_failure(gpu, cat600):
    from paper_2309_08601_gb300 import native
    dev = gpu.catalog_to_device(cat600)
    with gpu.Estimator(**S, precision="fp32") as est:
        native.check(native.lib().mp3pcf_inject(est._ctx, native.INJECT_ALLOC_FAILURE, 1), "inject")
        with pytest.raises(native.Mp3pcfError) as ei:
            est.accumulate_moments(*dev[:5])
        assert ei.value.status == native.ENOMEM
        native.check(native.lib().mp3pcf_inject(est._ctx, native.INJECT_ALLOC_FAILURE, 0), "inject")
        est.accumulate_moments(*dev[:5])
        nc, npairs = est.counts()
        assert nc == cat600.n and npairs > 0
