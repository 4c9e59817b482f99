"""Checkpoint / resume (checkpoint.measure_resumable) on the CPU: an estimator stand-in whose
moments and contraction are the oracle's runs the chunked measurement uninterrupted and with
interruptions; the resumed sums equal the uninterrupted ones bit for bit and the whole catalog's
to rounding, and a checkpoint of another measurement is refused."""
import os

import numpy as np
import pytest
import torch

from paper_2309_08601_gb300 import checkpoint, synth

from ._util import rel_err


class OracleEstimator:
    """The parts of api.Estimator that measure_resumable calls, computed by the oracle."""

    def __init__(self, orc, setup, cat):
        self.orc, self.s, self.cat = orc, setup, cat
        self.centres = None
        self.contract_calls = 0

    def new_multipoles(self):
        s = self.s
        z3 = s.n_z ** 3
        return (torch.zeros((z3, 4, s.n_max + 1, s.n_bins, s.n_bins), dtype=torch.complex128),
                torch.zeros((z3, 2 * s.n_max + 1, s.n_bins, s.n_bins), dtype=torch.complex128))

    def accumulate_moments(self, xq, yq, g1, g2, w, zbin=None, centre_mask=None):
        self.centres = np.nonzero(centre_mask.numpy())[0]

    def contract(self, ups, norm):
        G, W = self.orc.moments(self.s, self.cat, self.centres)
        u, n = self.orc.contract(self.s, self.cat, G, W, self.centres)
        ups += torch.as_tensor(u)
        norm += torch.as_tensor(n)
        self.contract_calls += 1
        return ups, norm

    def edge_correct(self, ups, norm, report_singular=True):
        return ups, 0

    def to_gamma(self, gam, projection):
        return gam

    def to_map3(self, gamma_cen, theta_ap):
        return None, None


@pytest.fixture(scope="module")
def case(orc):
    cat = synth.make_catalog(700, 20.0, 12, field="noise", weights="uniform")
    s = orc.Setup(n_bins=5, theta_min=0.5, theta_max=5.0, n_max=4)
    t = [torch.as_tensor(np.ascontiguousarray(a)) for a in (cat.xq, cat.yq, cat.g1, cat.g2, cat.w)]
    return cat, s, t


def test_resume_is_bit_identical_and_sums_to_the_whole_catalog(orc, case, tmp_path):
    cat, s, t = case
    full = checkpoint.measure_resumable(OracleEstimator(orc, s, cat), *t, None, str(tmp_path / "a.npz"),
                                        n_chunks=6)
    path = str(tmp_path / "b.npz")
    est = OracleEstimator(orc, s, cat)
    assert checkpoint.measure_resumable(est, *t, None, path, n_chunks=6, stop_after=2) is None
    assert est.contract_calls == 2 and int(np.load(path)["next"]) == 2
    est = OracleEstimator(orc, s, cat)
    assert checkpoint.measure_resumable(est, *t, None, path, n_chunks=6, stop_after=3) is None
    assert est.contract_calls == 3 and int(np.load(path)["next"]) == 5
    est = OracleEstimator(orc, s, cat)
    resumed = checkpoint.measure_resumable(est, *t, None, path, n_chunks=6)
    assert est.contract_calls == 1
    assert torch.equal(resumed.upsilon, full.upsilon) and torch.equal(resumed.norm, full.norm)
    G, W = orc.moments(s, cat)
    u, n = orc.contract(s, cat, G, W)
    assert rel_err(full.upsilon.numpy(), u) < 1e-12 and rel_err(full.norm.numpy(), n) < 1e-12
    assert not os.path.exists(path + ".tmp.npz")


def test_a_checkpoint_of_another_measurement_is_refused(orc, case, tmp_path):
    cat, s, t = case
    path = str(tmp_path / "c.npz")
    assert checkpoint.measure_resumable(OracleEstimator(orc, s, cat), *t, None, path, n_chunks=4,
                                        stop_after=1) is None
    with pytest.raises(ValueError):
        checkpoint.measure_resumable(OracleEstimator(orc, s, cat), *t, None, path, n_chunks=5)
