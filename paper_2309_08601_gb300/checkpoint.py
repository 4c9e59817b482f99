"""Checkpoint / resume of a long measurement by the additivity of the multipole components over
centre galaxies (App. B, Eq. PatchGamma: Upsilon and N are sums over centres).

The centres are processed in fixed chunks; after every chunk the running FP64 sums of Upsilon and
N and the index of the next chunk are written to a checkpoint file (atomically, by rename). A run
that is interrupted resumes from the last completed chunk and ends with the same sums, bit for
bit, as an uninterrupted chunked run, since the chunks and their order are the same. The FP64
edge correction, Gamma and the aperture measures then run once on the total.
"""
from __future__ import annotations

import os
from typing import Optional

import numpy as np


def _chunks(n: int, n_chunks: int):
    edges = np.linspace(0, n, n_chunks + 1).round().astype(np.int64)
    return [(int(edges[i]), int(edges[i + 1])) for i in range(n_chunks)]


def measure_resumable(est, xq, yq, g1, g2, w, theta_ap, path: str, n_chunks: int = 8, zbin=None,
                      stop_after: Optional[int] = None):
    """Runs est's whole path with centres in n_chunks contiguous index ranges, checkpointing
    (ups, norm, next chunk) to `path` after each. Returns the Measurement, or None when it
    stopped early because `stop_after` chunks were done in this call (an interruption)."""
    import torch
    n = int(xq.numel())
    chunks = _chunks(n, n_chunks)
    ups, norm = est.new_multipoles()
    start = 0
    if os.path.exists(path):
        ck = np.load(path)
        if int(ck["n"]) != n or int(ck["n_chunks"]) != n_chunks or tuple(ck["ups"].shape) != tuple(ups.shape):
            raise ValueError("checkpoint %s belongs to another measurement" % path)
        ups.copy_(torch.as_tensor(ck["ups"]))
        norm.copy_(torch.as_tensor(ck["norm"]))
        start = int(ck["next"])
    done = 0
    for i in range(start, len(chunks)):
        if stop_after is not None and done == stop_after:
            return None
        lo, hi = chunks[i]
        mask = torch.zeros(n, dtype=torch.uint8, device=xq.device)
        mask[lo:hi] = 1
        est.accumulate_moments(xq, yq, g1, g2, w, zbin, mask)
        est.contract(ups, norm)
        tmp = path + ".tmp.npz"
        np.savez(tmp, ups=ups.cpu().numpy(), norm=norm.cpu().numpy(), next=i + 1, n=n, n_chunks=n_chunks)
        os.replace(tmp, path)
        done += 1
    from .api import Measurement
    gam, ns = est.edge_correct(ups, norm, report_singular=False)
    gx = est.to_gamma(gam, 0)
    gc = est.to_gamma(gam, 1)
    corr, m8 = est.to_map3(gc, theta_ap)
    return Measurement(ups, norm, gam, ns, gx, gc, corr, m8)
