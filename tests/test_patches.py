"""Patch decomposition (paper App. B, Eq. PatchGamma, flat part) as the sharding rule for one
catalog over several processes: host logic on CPU, the additivity of the oracle's multipoles
over the patches, and two gloo ranks that each contract their patches and all-reduce."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2309_08601_gb300 import patches, synth  # noqa: E402

SETUP = dict(n_bins=6, theta_min=0.5, theta_max=6.0, n_max=4)


def _cat(n=700, seed=3, n_z=None):
    rng = np.random.default_rng(seed)
    cat = synth.make_catalog(n, 40.0, seed, field="noise", weights="uniform")
    if n_z:
        cat.zbin = rng.integers(0, n_z, n).astype(np.uint8)
    return cat


@pytest.mark.parametrize("n_px,n_py", [(1, 1), (2, 3), (4, 4), (7, 2)])
def test_every_galaxy_is_the_centre_of_exactly_one_patch(n_px, n_py):
    cat = _cat()
    ps = patches.plan(cat.xq, cat.yq, cat.quantum, SETUP["theta_max"], n_px, n_py)
    allc = np.concatenate([p.centres for p in ps])
    assert np.array_equal(np.sort(allc), np.arange(cat.n))
    for p in ps:
        assert np.all(np.isin(p.centres, p.members))
        assert np.array_equal(p.members[p.centre_mask.astype(bool)], p.centres)


def test_halo_holds_every_neighbour_in_range():
    cat = _cat(500)
    tmax_q2 = (SETUP["theta_max"] / cat.quantum) ** 2
    x = cat.xq.astype(np.int64)
    y = cat.yq.astype(np.int64)
    for p in patches.plan(cat.xq, cat.yq, cat.quantum, SETUP["theta_max"], 3, 3):
        dx = x[None, :] - x[p.centres][:, None]
        dy = y[None, :] - y[p.centres][:, None]
        near = np.nonzero(((dx * dx + dy * dy) <= tmax_q2).any(axis=0))[0]
        assert np.all(np.isin(near, p.members))


def test_assignment_covers_each_patch_once_and_balances():
    cat = _cat(3000)
    ps = patches.plan(cat.xq, cat.yq, cat.quantum, SETUP["theta_max"], 5, 5)
    for world in (1, 2, 3, 8):
        own = patches.assign(ps, world)
        assert sorted(i for o in own for i in o) == list(range(len(ps)))
        assert own == patches.assign(ps, world)  # the same on every rank
        loads = [sum(ps[i].cost for i in o) for o in own]
        assert max(loads) <= sum(loads) / world + max(p.cost for p in ps)


def _patch_multipoles(orc, s, cat, ps, idx):
    ups = norm = None
    for i in idx:
        p = ps[i]
        sub = cat.subset(p.members)
        local = np.nonzero(p.centre_mask)[0]
        G, W = orc.moments(s, sub, local)
        ups, norm = orc.contract(s, sub, G, W, local, ups, norm)
    return ups, norm


@pytest.mark.parametrize("n_z", [None, 2])
def test_patch_multipoles_add_up_to_the_whole_catalog(orc, n_z):
    cat = _cat(600, n_z=n_z)
    s = orc.Setup(**SETUP, n_z=n_z or 1)
    G, W = orc.moments(s, cat)
    ups0, norm0 = orc.contract(s, cat, G, W)
    ps = patches.plan(cat.xq, cat.yq, cat.quantum, SETUP["theta_max"], 3, 2)
    ups, norm = _patch_multipoles(orc, s, cat, ps, range(len(ps)))
    assert np.abs(ups - ups0).max() <= 1e-12 * np.abs(ups0).max()
    assert np.abs(norm - norm0).max() <= 1e-12 * np.abs(norm0).max()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cat = _cat(600)
        s = oracle.Setup(**SETUP)
        ps = patches.plan(cat.xq, cat.yq, cat.quantum, SETUP["theta_max"], 3, 3)
        mine = patches.assign(ps, world)[rank]
        ups, norm = _patch_multipoles(oracle, s, cat, ps, mine)
        tu, tn = torch.as_tensor(ups), torch.as_tensor(norm)
        patches.all_reduce_sum([tu, tn], dist)
        q.put((rank, len(mine), tu.numpy(), tn.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_all_reduce_their_patches(orc):
    import torch.multiprocessing as mp
    cat = _cat(600)
    s = orc.Setup(**SETUP)
    G, W = orc.moments(s, cat)
    ups0, norm0 = orc.contract(s, cat, G, W)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] > 0 and out[1][1] > 0  # both ranks had work
    for _, _, ups, norm in out:
        assert np.abs(ups - ups0).max() <= 1e-12 * np.abs(ups0).max()
        assert np.abs(norm - norm0).max() <= 1e-12 * np.abs(norm0).max()
