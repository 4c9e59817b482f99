"""The allocation-free Map^3 entry point (mp3pcf_to_map3_noalloc) against mp3pcf_to_map3.

It exists for callers that may not allocate device memory themselves (a plugin inside a host
application that owns all device memory, a service with a fixed memory budget). It keeps its
scratch in a static device array of the library, so two calls in a row must both agree with the
context-based entry point, which allocates its own scratch. This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from tests._util import hand_catalog, rel_err

pytestmark = pytest.mark.gpu

SETUP = dict(n_bins=8, theta_min=0.5, theta_max=12.0, n_max=8)


def _gamma_cen(api, n_z=1):
    rng = np.random.default_rng(42)
    n = 1500
    zb = rng.integers(0, n_z, n) if n_z > 1 else None
    cat = hand_catalog(rng.uniform(0, 40, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n), zb)
    est = api.Estimator(**SETUP, n_z=n_z, precision="fp64")
    dev = api.catalog_to_device(cat)
    est.accumulate_moments(*dev)
    ups, norm = est.contract()
    gam, _ = est.edge_correct(ups, norm)
    return est, est.to_gamma(gam, 1)


def _noalloc(native, est, gc, theta):
    import torch
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64), device="cuda").contiguous()
    n_ap = th.shape[0]
    corr = torch.full((est.z3, n_ap, 4), np.nan, dtype=torch.complex128, device="cuda")
    m8 = torch.full((est.z3, n_ap, 8), np.nan, dtype=torch.float64, device="cuda")
    st = native.lib().mp3pcf_to_map3_noalloc(C.byref(est.cfg), C.c_void_p(est.stream.cuda_stream),
                                             gc.data_ptr(), n_ap, th.data_ptr(), corr.data_ptr(),
                                             m8.data_ptr())
    return st, corr, m8


@pytest.mark.parametrize("n_z", [1, 2])
def test_noalloc_matches_context_entry_point_twice(n_z):
    import torch
    from paper_2309_08601_gb300 import api, native
    from paper_2309_08601_gb300.build import build_native
    build_native()
    est, gc = _gamma_cen(api, n_z)
    thetas = ([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0], [1.0, 2.0, 3.0]], [[3.0, 3.0, 3.0], [1.5, 2.5, 2.0]])
    for theta in thetas:  # two calls in a row reuse the same static scratch
        corr_ref, m8_ref = est.to_map3(gc, theta)
        st, corr, m8 = _noalloc(native, est, gc, theta)
        assert st == native.OK
        torch.cuda.synchronize()
        assert rel_err(corr.cpu().numpy(), corr_ref.cpu().numpy()) < 1e-10
        assert rel_err(m8.cpu().numpy(), m8_ref.cpu().numpy()) < 1e-10
    est.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_2309_08601_gb300 import api, native
    from paper_2309_08601_gb300.build import build_native
    build_native()
    est, gc = _gamma_cen(api, 1)
    st, _, _ = _noalloc(native, est, gc, [[1.0, 1.0, 1.0]] * 256)  # 256 > 255 jobs
    assert st == native.EINVAL
    cfg = native.make_config(**SETUP)
    cfg.n_bins = 0
    assert native.lib().mp3pcf_to_map3_noalloc(C.byref(cfg), None, gc.data_ptr(), 1, gc.data_ptr(),
                                               None, None) == native.EINVAL
    est.close()
