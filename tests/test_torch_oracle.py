"""The differentiable FP64 restatement of the oracle (oracle/torch_oracle.py), pinned on CPU.

Its forward must equal the C oracle's pipeline; its gradient (torch autograd, chunked VJP of the
moments) must satisfy the exact homogeneity identities of the method and central finite
differences. Map^3 is cubic in the shears (every Upsilon is a product of three shears, the
normalisation N has none) and of degree zero in the weights (Upsilon and N are both cubic in
w, and Gamma = N^-1 Upsilon), so for L = sum c . m8:
    sum_k (g1_k dL/dg1_k + g2_k dL/dg2_k) = 3 L      and      sum_k w_k dL/dw_k = 0.
"""
import numpy as np
import pytest
import torch

from tests._util import hand_catalog, rel_err

S_SMALL = dict(n_bins=6, theta_min=0.5, theta_max=8.0, n_max=5, n_phi=40)
TH = [[2.0, 2.0, 2.0], [1.5, 2.5, 3.0]]


@pytest.fixture(scope="module")
def small_case(orc):
    from oracle import torch_oracle as to
    rng = np.random.default_rng(42)
    n = 350
    cat = hand_catalog(rng.uniform(0, 14, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n))
    s = orc.Setup(**S_SMALL)
    return s, cat, to.Map3Oracle(s, cat, TH, chunk_pairs=20_000)


def _t(a):
    return torch.as_tensor(np.asarray(a, np.float64))


def test_forward_equals_c_oracle(orc, small_case):
    s, cat, mo = small_case
    r = orc.pipeline(s, cat, TH)
    ups, norm, gam, gc, corr, m8 = [x.detach().numpy() for x in mo.forward(_t(cat.g1), _t(cat.g2), _t(cat.w))]
    for a, b in ((ups, r.ups), (norm, r.norm), (gam, r.gamma_n), (gc, r.gamma_cen), (m8, r.m8)):
        assert rel_err(a, b) < 1e-11


def test_homogeneity_identities(small_case):
    s, cat, mo = small_case
    c = np.random.default_rng(0).normal(size=(1, len(TH), 8))
    g1, g2, w = _t(cat.g1), _t(cat.g2), _t(cat.w)
    d1, d2, dw, m8 = mo.grad(g1, g2, w, c)
    L = float((torch.as_tensor(c) * m8).sum())
    euler_g = float((g1 * d1 + g2 * d2).sum())
    euler_w = float((w * dw).sum())
    assert abs(euler_g - 3 * L) < 1e-10 * max(abs(L), 1e-300) * 1e3
    assert abs(euler_w) < 1e-9 * float((w * dw).abs().sum())


def test_gradient_against_central_differences(small_case):
    s, cat, mo = small_case
    c = np.random.default_rng(1).normal(size=(1, len(TH), 8))
    g1, g2, w = _t(cat.g1), _t(cat.g2), _t(cat.w)
    d1, d2, dw, _ = mo.grad(g1, g2, w, c)
    ct = torch.as_tensor(c)
    L = lambda a, b, u: float((ct * mo.forward(a, b, u)[-1]).sum())
    h = 1e-5
    for k in (3, 77, 210):
        for which, grad in ((0, d1), (1, d2), (2, dw)):
            args_p = [g1.clone(), g2.clone(), w.clone()]
            args_m = [g1.clone(), g2.clone(), w.clone()]
            args_p[which][k] += h
            args_m[which][k] -= h
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert abs(fd - float(grad[k])) <= 1e-6 * max(abs(fd), float(grad.abs().max())), (k, which)


@pytest.mark.parametrize("n_z", [1, 2])
def test_forward_excluding_degenerate_triplets_equals_c_oracle(orc, n_z):
    """exclude_degenerate (j = k left out) in the differentiable restatement against the C oracle,
    whose correction is pinned against the brute force without j = k."""
    from oracle import torch_oracle as to
    rng = np.random.default_rng(8 + n_z)
    n = 250
    cat = hand_catalog(rng.uniform(0, 14, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n), rng.integers(0, n_z, n) if n_z > 1 else None)
    s = orc.Setup(**S_SMALL, n_z=n_z, exclude_degenerate=1)
    r = orc.pipeline(s, cat, TH)
    mo = to.Map3Oracle(s, cat, TH, chunk_pairs=20_000)
    ups, norm, gam, gc, corr, m8 = [x.detach().numpy() for x in mo.forward(_t(cat.g1), _t(cat.g2), _t(cat.w))]
    for a, b in ((ups, r.ups), (norm, r.norm), (gam, r.gamma_n), (m8, r.m8)):
        assert rel_err(a, b) < 1e-11
