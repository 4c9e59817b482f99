"""The autotuner's host logic on the CPU: with an estimator stand-in whose stage timers report a
known cost per launch shape, tune() picks the fastest cell occupancy and contraction slice count,
times the slices at the chosen occupancy only for the tensor-core precisions, and serves a
repeated request from its cache."""
import types

import pytest

from paper_2309_08601_gb300 import api, autotune


class FakeEstimator:
    made = []

    def __init__(self, n_bins, theta_min, theta_max, n_max, *, precision="fp32", cell_occupancy=0,
                 contract_slices=0, **kw):
        self.occ, self.sl, self.precision = cell_occupancy, contract_slices, precision
        self._t = {}
        FakeEstimator.made.append((precision, cell_occupancy, contract_slices))

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def set_timing(self, on):
        pass

    def accumulate_moments(self, *a):
        self._t["moments"] = (10.0 + (self.occ - 3) ** 2, 1)

    def contract(self, *a):
        self._t["contract"] = (1.0 + abs(self.sl - 16), 1)

    def stage_times(self, reset=False):
        t, self._t = self._t, ({} if reset else self._t)
        return t


@pytest.fixture
def fake(monkeypatch):
    FakeEstimator.made = []
    monkeypatch.setattr(api, "Estimator", FakeEstimator)
    monkeypatch.setattr(autotune, "_key", lambda setup, precision, n: (tuple(sorted(setup.items())), precision, n))
    autotune._CACHE.clear()
    yield FakeEstimator
    autotune._CACHE.clear()


def _catalog(n):
    return (types.SimpleNamespace(numel=lambda: n),) + (None,) * 4


SETUP = dict(n_bins=20, theta_min=0.5, theta_max=120.0, n_max=30)


def test_picks_the_fastest_shapes(fake):
    r = autotune.tune(SETUP, _catalog(1000), precision="bf16x3")
    assert r["cell_occupancy"] == 3 and r["contract_slices"] == 16
    assert r["moments_ms"] == 10.0 and r["contract_ms"] == 1.0
    assert set(r["trials"]["moments"]) == set(autotune.OCCUPANCIES)
    assert set(r["trials"]["contract"]) == set(autotune.SLICES)
    # the slices are timed at the chosen occupancy
    assert all(occ == 3 for p, occ, sl in fake.made if sl != 0)


def test_cuda_core_precisions_keep_the_default_slices(fake):
    r = autotune.tune(SETUP, _catalog(1000), precision="fp64")
    assert r["contract_slices"] == 0 and r["trials"]["contract"] == {}


def test_a_repeated_request_is_served_from_the_cache(fake):
    r1 = autotune.tune(SETUP, _catalog(1000), precision="bf16x3")
    n = len(fake.made)
    assert autotune.tune(SETUP, _catalog(1000), precision="bf16x3") is r1 and len(fake.made) == n
    autotune.tune(SETUP, _catalog(2000), precision="bf16x3")  # another catalog size: tuned again
    assert len(fake.made) > n
    autotune.tune(SETUP, _catalog(1000), precision="bf16x3", use_cache=False)
    assert len(fake.made) > 2 * n
