"""The hand-written adjoint (differentiation form) against the FP64 autograd of the oracle.

Stage by stage: the adjoints of to_map3, to_gamma and edge_correct are compared with torch
autograd through the oracle's own stage functions (oracle/torch_oracle.py) at the same inputs;
the whole chain (api.map3 backward: to_map3 -> to_gamma -> edge_correct -> contraction ->
moments) with the oracle's full FP64 autograd. At any size the exact homogeneity identities
hold: Map^3 is cubic in the shears and of degree zero in the weights, so
    sum_k (g1 dL/dg1 + g2 dL/dg2) = 3 L   and   sum_k w dL/dw = 0.
Tolerances (normwise relative, per gradient array): 1e-9 for the FP64 stages, 2e-6 for the whole
FP64 chain (the gradients are returned in float32), 1e-4 for the FP32 chains (FP32 moments and
adjoint; measured ~1e-6); central differences 1e-5 (FP64) and 1e-4 (FP32); the identities to
1e-6 (FP64) and 1e-4 (FP32) of sum |terms|.
"""
import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import synth
from tests._util import hand_catalog, rel_err

pytestmark = pytest.mark.gpu

S1 = dict(n_bins=6, theta_min=0.5, theta_max=8.0, n_max=5, n_phi=40)
TH1 = [[2.0, 2.0, 2.0], [1.5, 2.5, 3.0]]


@pytest.fixture(scope="module")
def gpu():
    from paper_2309_08601_gb300.build import build_native
    build_native()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2309_08601_gb300 import api
    return api


@pytest.fixture(scope="module")
def case1(orc):
    from oracle import torch_oracle as to
    rng = np.random.default_rng(42)
    n = 350
    cat = hand_catalog(rng.uniform(0, 14, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n))
    s = orc.Setup(**S1)
    return s, cat, to.Map3Oracle(s, cat, TH1, chunk_pairs=20_000)


def _cpu64(cat):
    return (torch.as_tensor(np.asarray(cat.g1, np.float64)), torch.as_tensor(np.asarray(cat.g2, np.float64)),
            torch.as_tensor(np.asarray(cat.w, np.float64)))


def _est(api, setup, precision):
    kw = dict(setup)
    return api.Estimator(**kw, precision=precision)


def test_stage_adjoints_fp64(gpu, orc, case1):
    """to_map3, to_gamma and edge_correct adjoints against torch autograd of the same stages."""
    from oracle import torch_oracle as to
    s, cat, mo = case1
    dev = gpu.catalog_to_device(cat)
    rng = np.random.default_rng(3)
    c = torch.as_tensor(rng.normal(size=(1, len(TH1), 8)))
    with _est(gpu, S1, "fp64") as est:
        m = est.measure(*dev[:5], theta_ap=TH1)
        ups = m.upsilon.cpu().clone().requires_grad_(True)
        norm = m.norm.cpu().clone().requires_grad_(True)
        gam = to.edge_correct(s, ups, norm)
        gam.retain_grad()
        gx = torch.einsum("zmnbc,nk->zmbck", gam, mo.ephi)
        gc = gx * mo.cen[None]
        gc.retain_grad()
        corr = torch.einsum("zmbck,ambck->zam", gc, mo.filt)
        (c * to.combine8(corr)).sum().backward()
        g_gc = est.to_map3_adjoint(TH1, grad_m8=c.cuda())
        assert rel_err(g_gc.cpu().numpy(), gc.grad.numpy()) < 1e-9
        g_gam = est.to_gamma_adjoint(gc.grad.cuda(), 1)
        assert rel_err(g_gam.cpu().numpy(), gam.grad.numpy()) < 1e-9
        g_u, g_n = est.edge_correct_adjoint(m.norm, m.gamma_n, gam.grad.cuda())
        assert rel_err(g_u.cpu().numpy(), ups.grad.numpy()) < 1e-9
        assert rel_err(g_n.cpu().numpy(), norm.grad.numpy()) < 1e-9


@pytest.mark.parametrize("precision,tol", [("fp64", 2e-6), ("fp32", 1e-4), ("bf16x3", 1e-4)])
def test_whole_chain_against_oracle_autograd(gpu, case1, precision, tol):
    s, cat, mo = case1
    c = np.random.default_rng(5).normal(size=(1, len(TH1), 8))
    o1, o2, ow, m8o = mo.grad(*_cpu64(cat), c)
    dev = gpu.catalog_to_device(cat)
    g1 = dev[2].clone().requires_grad_(True)
    g2 = dev[3].clone().requires_grad_(True)
    w = dev[4].clone().requires_grad_(True)
    with _est(gpu, S1, precision) as est:
        m8 = gpu.map3(est, dev[0], dev[1], g1, g2, w, TH1)
        (torch.as_tensor(c, device="cuda") * m8).sum().backward()
    errs = [rel_err(g1.grad.cpu().numpy(), o1.numpy()), rel_err(g2.grad.cpu().numpy(), o2.numpy()),
            rel_err(w.grad.cpu().numpy(), ow.numpy())]
    print(precision, "gradient errors vs FP64 autograd oracle", errs)
    assert max(errs) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 2e-6), ("bf16x3", 1e-4)])
def test_tomographic_chain_against_oracle_autograd(gpu, orc, precision, tol):
    """Two z-bins (all 8 Z-triplets, each centre contracted only in its own Z1): the whole chain's
    gradient against the oracle's FP64 autograd."""
    from oracle import torch_oracle as to
    rng = np.random.default_rng(44)
    n = 300
    cat = hand_catalog(rng.uniform(0, 14, (n, 2)), rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n),
                       rng.uniform(0.5, 1.5, n), rng.integers(0, 2, n))
    setup = dict(S1, n_z=2)
    mo = to.Map3Oracle(orc.Setup(**setup), cat, TH1, chunk_pairs=20_000)
    c = np.random.default_rng(6).normal(size=(8, len(TH1), 8))
    o1, o2, ow, _ = mo.grad(*_cpu64(cat), c)
    dev = gpu.catalog_to_device(cat)
    g1 = dev[2].clone().requires_grad_(True)
    g2 = dev[3].clone().requires_grad_(True)
    w = dev[4].clone().requires_grad_(True)
    with gpu.Estimator(**setup, precision=precision) as est:
        m8 = gpu.map3(est, dev[0], dev[1], g1, g2, w, TH1, zbin=dev[5])
        (torch.as_tensor(c, device="cuda") * m8).sum().backward()
    errs = [rel_err(g1.grad.cpu().numpy(), o1.numpy()), rel_err(g2.grad.cpu().numpy(), o2.numpy()),
            rel_err(w.grad.cpu().numpy(), ow.numpy())]
    print(precision, "tomographic gradient errors vs FP64 autograd oracle", errs)
    assert max(errs) < tol


def _euler(api, cat, setup, theta, precision, c):
    dev = api.catalog_to_device(cat)
    g1 = dev[2].clone().requires_grad_(True)
    g2 = dev[3].clone().requires_grad_(True)
    w = dev[4].clone().requires_grad_(True)
    with api.Estimator(**setup, precision=precision) as est:
        m8 = api.map3(est, dev[0], dev[1], g1, g2, w, theta)
        L = (torch.as_tensor(c, device="cuda") * m8).sum()
        L.backward()
    eg = (g1.detach().double() * g1.grad.double() + g2.detach().double() * g2.grad.double())
    ew = w.detach().double() * w.grad.double()
    return float(L.detach()), float(eg.sum()), float(eg.abs().sum()), float(ew.sum()), float(ew.abs().sum())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_homogeneity_identities_lognormal(gpu, precision, tol):
    cat = synth.make_catalog(12000, 100.0, 21, field="lognormal", sigma_e=0.26, weights="uniform", ngrid=1024)
    setup = dict(n_bins=14, theta_min=0.5, theta_max=30.0, n_max=10)
    th = [[2.0, 2.0, 2.0], [4.0, 4.0, 4.0]]
    c = np.random.default_rng(7).normal(size=(1, 2, 8))
    L, eg, eg_abs, ew, ew_abs = _euler(gpu, cat, setup, th, precision, c)
    print(precision, "3L", 3 * L, "sum g dL/dg", eg, "sum w dL/dw", ew, "(of", ew_abs, ")")
    assert abs(eg - 3 * L) <= tol * eg_abs
    assert abs(ew) <= tol * ew_abs


def _c4_density_case():
    """The differentiation workload's density (5e5 galaxies on 420') on a 42' patch of 5000
    galaxies, with the first 12 of its 20 log bins (0.5'-13.4', the same edges), so that its
    small-scale systems are filled as at full size (~1.6 pairs per galaxy in the 0.5' bin)."""
    p = synth.WORKLOADS["grad_lognormal_500k"]
    ratio = (p["theta_max"] / p["theta_min"]) ** (1.0 / p["n_bins"])
    side = p["side"] * np.sqrt(5000 / p["n"])
    cat = synth.make_catalog(5000, side, p["seed"], field=p["field"], weights=p["weights"])
    setup = dict(n_bins=12, theta_min=p["theta_min"], theta_max=p["theta_min"] * ratio ** 12, n_max=p["n_max"])
    return cat, setup, [[2.0, 2.0, 2.0], [4.0, 4.0, 4.0]]


def _c4_patch_case():
    """The differentiation workload's patch and model at 100x lower density (5000 galaxies on
    420'): the 0.5' bins would hold ~0.02 pairs per galaxy and their edge-correction systems be
    nearly singular, so the 20 log bins start at 10' (every (b1, b2) system well filled)."""
    p = synth.WORKLOADS["grad_lognormal_500k"]
    cat = synth.make_catalog(5000, p["side"], p["seed"], field=p["field"], weights=p["weights"])
    setup = dict(n_bins=p["n_bins"], theta_min=10.0, theta_max=p["theta_max"], n_max=p["n_max"])
    return cat, setup, [[t, t, t] for t in p["theta_ap"]]


@pytest.mark.parametrize("case", ["c4_density_small_bins", "c4_patch_large_bins"])
def test_finite_differences_5000(gpu, orc, case):
    """5000 galaxies of the differentiation workload's model, n_max 30: FP64 forward central
    differences (h = 1e-4) on 100 random galaxies against the FP32 and FP64 adjoints, and the whole
    FP64 gradient against the oracle's FP64 autograd; once at the workload's density with its own
    small-scale bins, once on its whole patch with bins from 10'."""
    from oracle import torch_oracle as to
    cat, setup, th = _c4_density_case() if case == "c4_density_small_bins" else _c4_patch_case()
    c = np.zeros((1, len(th), 8))
    c[0, :, 0] = 1.0  # L = sum of Map^3 over the apertures
    dev = gpu.catalog_to_device(cat)
    grads = {}
    for prec in ("fp64", "fp32"):
        g1 = dev[2].clone().requires_grad_(True)
        g2 = dev[3].clone().requires_grad_(True)
        w = dev[4].clone().requires_grad_(True)
        with gpu.Estimator(**setup, precision=prec) as est:
            m8 = gpu.map3(est, dev[0], dev[1], g1, g2, w, th)
            (torch.as_tensor(c, device="cuda") * m8).sum().backward()
        grads[prec] = [g1.grad.cpu().double().numpy(), g2.grad.cpu().double().numpy(),
                       w.grad.cpu().double().numpy()]
    # oracle FP64 autograd
    s = orc.Setup(**setup)
    mo = to.Map3Oracle(s, cat, th, chunk_pairs=100_000)
    o = mo.grad(*_cpu64(cat), c)
    for k in range(3):
        print("param", k, "FP64 adjoint vs oracle autograd", rel_err(grads["fp64"][k], o[k].numpy()))
    for k in range(3):
        assert rel_err(grads["fp64"][k], o[k].numpy()) < 2e-6
    # central differences with the FP64 GPU forward
    rng = np.random.default_rng(11)
    idx = rng.choice(cat.n, 100, replace=False)
    h = 1e-4
    with gpu.Estimator(**setup, precision="fp64") as est:
        def L(a1, a2, aw):
            m = est.measure(dev[0], dev[1], a1, a2, aw, theta_ap=th, report_singular=False)
            return float((torch.as_tensor(c, device="cuda") * m.m8).sum())
        fd = np.zeros((3, len(idx)))
        base = [dev[2].clone(), dev[3].clone(), dev[4].clone()]
        for j, k in enumerate(idx):
            for which in range(3):
                ap = [t.clone() for t in base]
                am = [t.clone() for t in base]
                # the perturbation actually applied in float32
                xp = float(torch.tensor(float(base[which][k]) + h, dtype=torch.float32))
                xm = float(torch.tensor(float(base[which][k]) - h, dtype=torch.float32))
                ap[which][k] = xp
                am[which][k] = xm
                fd[which, j] = (L(*ap) - L(*am)) / (xp - xm)
    for prec, tol in (("fp64", 1e-5), ("fp32", 1e-4)):
        for which in range(3):
            e = rel_err(grads[prec][which][idx], fd[which])
            print(prec, "param", which, "adjoint vs central differences", e)
            assert e < tol


def test_full_size_c4_identities(gpu):
    """The differentiation workload (500 000 galaxies, 7 deg x 7 deg, apertures 4', 8', 16') in
    FP32: forward + backward through the adjoint kernels; gradients finite and the homogeneity
    identities hold."""
    p = synth.WORKLOADS["grad_lognormal_500k"]
    cat = synth.workload_catalog("grad_lognormal_500k")
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"], n_max=p["n_max"])
    th = [[t, t, t] for t in p["theta_ap"]]
    c = np.zeros((1, len(th), 8))
    c[0, :, 0] = 1.0
    L, eg, eg_abs, ew, ew_abs = _euler(gpu, cat, setup, th, "bf16x3", c)
    print("C4 FP32/BF16x3: 3L", 3 * L, "sum g dL/dg", eg, "sum w dL/dw", ew, "(of", ew_abs, ")")
    assert np.isfinite([L, eg, ew]).all()
    assert abs(eg - 3 * L) <= 1e-4 * eg_abs
    assert abs(ew) <= 1e-4 * ew_abs
