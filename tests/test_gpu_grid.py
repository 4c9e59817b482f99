"""The grid-based approximation on the GPU (Sec. 3.2): the pixel catalog against the oracle's
(bit-identical: the per-pixel FP64 sums are exact), and the grid estimator against the discrete
one for bins far above the pixel size."""
import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.mark.parametrize("n_z", [1, 3])
def test_pixel_catalog_is_the_oracles(gpu, orc, n_z):
    if n_z == 1:
        cat = synth.make_catalog(20_000, 100.0, 5, field="lognormal", weights="uniform", ngrid=1024)
    else:
        cat = synth.make_tomographic_catalog(6, side=80.0, n_z=3, n_range=(4000, 9000), ngrid=512)
    dev = gpu.catalog_to_device(cat)
    pq = 1 << 13
    with gpu.Estimator(n_bins=4, theta_min=1.0, theta_max=8.0, n_max=2, n_z=n_z) as est:
        pix = est.grid_catalog(*dev[:5], dev[5], pixel_arcmin=1.0)
    x0, y0 = int(cat.xq.min()), int(cat.yq.min())
    npx = (int(cat.xq.max()) - x0) // pq + 1
    npy = (int(cat.yq.max()) - y0) // pq + 1
    ref = orc.grid_catalog(cat, (x0, y0), pq, npx, npy, n_z)
    for k, f in enumerate(("xq", "yq", "g1", "g2", "w")):
        assert np.array_equal(pix[k].cpu().numpy(), getattr(ref, f)), f
    if n_z > 1:
        assert np.array_equal(pix[5].cpu().numpy(), ref.zbin)


def test_grid_estimator_converges_to_the_discrete_one(gpu):
    """200 000 galaxies on 300' with noise-free lognormal shear (with shape noise the multipoles at
    these scales are noise sums that any regridding reshuffles), 20 bins 0.5'-120', n_max 30.
    For the bins whose lower edge is at least 20 pixels of 0.5' (the regime of Sec. 3.2) the grid
    multipoles of the low orders (Upsilon n <= 10, N n <= 20) agree with the discrete ones to 2 %
    and 1 % norm-wise, and closer with 0.25' pixels; Map^3 at 8' and 16' (all bins, the small ones
    included) agrees to 2 % with 0.25' pixels."""
    cat = synth.make_catalog(200_000, 300.0, 1, field="lognormal", sigma_e=0.0, weights="uniform")
    dev = gpu.catalog_to_device(cat)
    setup = dict(n_bins=20, theta_min=0.5, theta_max=120.0, n_max=30)
    th = [[8.0, 8.0, 8.0], [16.0, 16.0, 16.0]]
    edges = 0.5 * 240.0 ** (np.arange(21) / 20)
    b0 = int(np.argmax(edges[:-1] >= 20 * 0.5))

    def nerr(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    with gpu.Estimator(**setup, precision="fp32") as est:
        d = est.measure(*dev[:5], theta_ap=th, report_singular=False)
        u_d, n_d, m_d = d.upsilon.cpu().numpy(), d.norm.cpu().numpy(), d.m8[0, :, 0].cpu().numpy()
        res = {}
        for delta in (0.5, 0.25):
            pix = est.grid_catalog(*dev[:5], pixel_arcmin=delta)
            g = est.measure(*pix[:5], theta_ap=th, report_singular=False)
            u_g, n_g, m_g = g.upsilon.cpu().numpy(), g.norm.cpu().numpy(), g.m8[0, :, 0].cpu().numpy()
            res[delta] = (nerr(u_g[:, :, :11, b0:, b0:], u_d[:, :, :11, b0:, b0:]),
                          nerr(n_g[:, :21, b0:, b0:], n_d[:, :21, b0:, b0:]), np.abs(m_g / m_d - 1))
            print("pixel %.2f' (%d pixels): Upsilon %.4f N %.5f (bins from %.1f'), Map^3 rel. diff %s" % (
                delta, int(pix[0].numel()), res[delta][0], res[delta][1], edges[b0], res[delta][2]))
    assert res[0.5][0] < 0.02 and res[0.5][1] < 0.01
    assert res[0.25][0] < res[0.5][0] and res[0.25][1] < res[0.5][1]
    assert (res[0.25][2] < 0.02).all()
