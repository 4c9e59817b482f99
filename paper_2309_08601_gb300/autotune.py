"""Tile-shape autotuner for the two hot kernels.

Two launch shapes matter and depend on the catalog's density, the radial range and the GPU:

* the moment kernel's tile is a cell of the sorting grid: ``cell_occupancy`` galaxies per cell
  and redshift bin sets how many candidates an annulus row holds against how many of them fall
  outside the bin (candidates per accepted pair);
* the tensor-core contraction splits the centre axis into ``contract_slices`` slices: more slices
  fill the resident CTA slots in whole waves, fewer keep the FP64 partial sums small.

``tune`` times every candidate on a sample catalog with device events (the library's own stage
timers), picks the fastest and caches the choice per (setup, precision, catalog size, GPU).
"""
from __future__ import annotations

import statistics
from typing import Dict, Sequence, Tuple

_CACHE: Dict[Tuple, dict] = {}

OCCUPANCIES = (2, 3, 4, 6, 8, 12)
SLICES = (0, 4, 8, 16, 24, 32, 48, 64)


def _key(setup: dict, precision: str, n: int):
    import torch
    return (tuple(sorted(setup.items())), precision, int(n), torch.cuda.get_device_name())


def _time_stage(est, run, stage: str, repeats: int) -> float:
    est.set_timing(True)
    ts = []
    for _ in range(repeats):
        est.stage_times(reset=True)
        run()
        ts.append(est.stage_times(reset=True)[stage][0])
    est.set_timing(False)
    return statistics.median(ts)


def tune(setup: dict, catalog, precision: str = "bf16x3", occupancies: Sequence[int] = OCCUPANCIES,
         slices: Sequence[int] = SLICES, repeats: int = 2, use_cache: bool = True) -> dict:
    """Returns {"cell_occupancy", "contract_slices", "moments_ms", "contract_ms", "trials"} for a
    device catalog (xq, yq, g1, g2, w[, zbin]) and an Estimator setup (n_bins, theta_min, ...)."""
    from . import api
    xq, yq, g1, g2, w = catalog[:5]
    zb = catalog[5] if len(catalog) > 5 else None
    key = _key(setup, precision, xq.numel())
    if use_cache and key in _CACHE:
        return _CACHE[key]
    trials = {"moments": {}, "contract": {}}
    for occ in occupancies:
        with api.Estimator(**setup, precision=precision, cell_occupancy=occ) as est:
            est.accumulate_moments(xq, yq, g1, g2, w, zb)  # warm-up
            trials["moments"][occ] = _time_stage(
                est, lambda: est.accumulate_moments(xq, yq, g1, g2, w, zb), "moments", repeats)
    best_occ = min(trials["moments"], key=trials["moments"].get)
    best_sl = 0
    if precision in ("bf16x3", "tf32x3"):
        for sl in slices:
            with api.Estimator(**setup, precision=precision, cell_occupancy=best_occ, contract_slices=sl) as est:
                est.accumulate_moments(xq, yq, g1, g2, w, zb)
                est.contract()  # warm-up
                trials["contract"][sl] = _time_stage(est, lambda: est.contract(), "contract", repeats)
        best_sl = min(trials["contract"], key=trials["contract"].get)
    res = {"cell_occupancy": int(best_occ), "contract_slices": int(best_sl),
           "moments_ms": trials["moments"][best_occ],
           "contract_ms": trials["contract"].get(best_sl), "trials": trials}
    _CACHE[key] = res
    return res
