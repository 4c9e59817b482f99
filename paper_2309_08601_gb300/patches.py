"""Patch decomposition of one flat catalog, for sharding a measurement over several processes
(one per GPU) or over time (catalogs whose moments exceed one device's memory).

The multipole components are sums over centre galaxies (paper App. B, Eq. PatchGamma), and a
centre's moments involve only neighbours closer than theta_max. So the catalog's bounding box is
cut into n_px x n_py rectangles; patch p takes as centres the galaxies of rectangle p and as
members the galaxies of rectangle p grown by a halo of theta_max on every side (every neighbour
of every centre of the patch). The patches' Upsilon and N add up to the whole catalog's (up to
the order of the floating-point sums). Patches are spread over the ranks by a greedy balance of
their work estimate (members x centres, the pair count scale); each rank sums its patches'
multipoles and one all-reduce of Upsilon and N (about 1 MB at 20 bins, n_max 30) adds the ranks'.
The FP64 edge correction, Gamma and the aperture measures then run on every rank.

Host logic only (numpy); the per-patch work goes through the estimator's C-ABI calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np


@dataclass
class Patch:
    centres: np.ndarray   # global indices of the patch's centre galaxies (sorted)
    members: np.ndarray   # global indices of the galaxies it needs: centres and halo (sorted)
    centre_mask: np.ndarray  # uint8 over members: 1 for the centres

    @property
    def cost(self) -> float:
        return float(len(self.members)) * float(len(self.centres))


def plan(xq: np.ndarray, yq: np.ndarray, quantum: float, theta_max: float, n_px: int,
         n_py: int) -> List[Patch]:
    """The n_px x n_py patches of a catalog with fixed-point positions (xq, yq) in units of
    quantum arcmin; rectangles are half-open in the integer positions, so every galaxy is the
    centre of exactly one patch. Empty patches are dropped."""
    if n_px < 1 or n_py < 1:
        raise ValueError("n_px and n_py must be >= 1")
    xq = np.asarray(xq, dtype=np.int64)
    yq = np.asarray(yq, dtype=np.int64)
    if xq.size == 0:
        return []
    x0, x1 = int(xq.min()), int(xq.max()) + 1
    y0, y1 = int(yq.min()), int(yq.max()) + 1
    ex = x0 + ((x1 - x0) * np.arange(n_px + 1, dtype=np.int64)) // n_px
    ey = y0 + ((y1 - y0) * np.arange(n_py + 1, dtype=np.int64)) // n_py
    ix = np.clip(np.searchsorted(ex, xq, side="right") - 1, 0, n_px - 1)
    iy = np.clip(np.searchsorted(ey, yq, side="right") - 1, 0, n_py - 1)
    # a neighbour in range is closer than theta_max, so within this many quanta along each axis
    halo = int(math.ceil(theta_max / quantum)) + 1
    out = []
    for py in range(n_py):
        for px in range(n_px):
            centres = np.nonzero((ix == px) & (iy == py))[0]
            if centres.size == 0:
                continue
            inside = ((xq >= ex[px] - halo) & (xq < ex[px + 1] + halo) &
                      (yq >= ey[py] - halo) & (yq < ey[py + 1] + halo))
            members = np.nonzero(inside)[0]
            mask = np.isin(members, centres, assume_unique=True).astype(np.uint8)
            out.append(Patch(centres, members, mask))
    return out


def assign(patches: Sequence[Patch], world: int) -> List[List[int]]:
    """Patch indices per rank: the patches in decreasing cost, each to the rank with the least
    total so far (the lowest rank on ties), so the result is the same on every rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    owned: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(patches)), key=lambda j: (-patches[j].cost, j)):
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        load[r] += patches[i].cost
    for o in owned:
        o.sort()
    return owned


def all_reduce_sum(tensors, dist=None):
    """Sums torch tensors (complex ones as their real views) over the ranks of dist, in place."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return tensors
    import torch
    for t in tensors:
        dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, op=dist.ReduceOp.SUM)
    return tensors


def measure_patched(est, cat, theta_ap, n_px: int, n_py: int, dist=None, device=None,
                    report_singular: bool = False):
    """The whole path for a host catalog (synth.Catalog) in patches: this rank's patches are
    accumulated and contracted into one pair of multipole buffers, which are summed over the ranks
    of dist (torch.distributed, optional); then edge correction, Gamma and Map^3 on the total.
    Returns the estimator's Measurement (identical on every rank)."""
    import torch
    from .api import Measurement, catalog_to_device
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    theta_max = float(est.cfg.theta_max)
    patches = plan(cat.xq, cat.yq, cat.quantum, theta_max, n_px, n_py)
    mine = assign(patches, world)[rank]
    ups, norm = est.new_multipoles()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    for i in mine:
        p = patches[i]
        d = catalog_to_device(cat.subset(p.members), dev)
        mask = torch.as_tensor(p.centre_mask, device=dev)
        est.accumulate_moments(*d[:5], d[5], mask)
        est.contract(ups, norm)
    all_reduce_sum([ups, norm], dist)
    gam, ns = est.edge_correct(ups, norm, report_singular=report_singular)
    gx = est.to_gamma(gam, 0)
    gc = est.to_gamma(gam, 1)
    corr, m8 = est.to_map3(gc, theta_ap)
    return Measurement(ups, norm, gam, ns, gx, gc, corr, m8)
