#!/usr/bin/env python3
"""Benchmark of the multipole shear-3PCF hot path on GB300.

One step = the whole path on one catalog: cell sort, moments (stage a), multipole contraction
(stage b), edge correction, Gamma^x and Gamma^cen, and the aperture measures. The workload is the
200k-galaxy lognormal catalog on a 300'x300' patch (20 log bins 0.5'-120', n_max = 30, Map^3 at
2', 4', 8', 16'). With N GPUs (torchrun) every rank measures its own catalog realisation
(independent problems, weak scaling, no data-path collective).

Prints one JSON line on rank 0. ``--impl reference`` times the FP64 CPU oracle on a bounded
centre sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "neighbour-pair harmonic accumulations/s; catalogs/s vs FP64 GPU path at ≤1e-4 Map³ err"
UNIT = "pair-accumulations/s"
PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (derived; FP32 FMA pipe)"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12


def _measured_hbm_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback: one earlier copy measurement on a GB300


HBM_PEAK_GBS = _measured_hbm_gbs()
# DRAM bytes (read + write) per launch of the current moments kernel at the lognormal_200k
# workload: ncu capture at 50 000 galaxies (profiles/moments_kernel_lognormal_50k.md) scaled to
# 200 000 centres (the traffic is the G/W write, proportional to the number of centres).
# Set to None whenever the kernel changes until it is captured again.
MOMENTS_TRAFFIC_BYTES = 4 * (125.665792e6 + 1052.680e6)
# DRAM bytes per launch of the tensor-core contraction (BF16x3) at lognormal_200k, from an ncu
# capture scaled by the centres, or None. None now: the kernel has since been changed to read only
# each Z1's centre range (the same work at one z-bin); its last capture, 4 x (1.066084e9 +
# 9.231360e6) bytes, is kept in profiles/contract_tc_bf16x3_lognormal_50k.md.
CONTRACT_TRAFFIC_BYTES = None


def flops_per_pair(n_max: int) -> int:
    """Algorithmic FP32 flops of stage (a) per neighbour pair, counted for the plain form of
    Eq. Gn_disc and the W_n of Eq. 3PCF_Normalization: geometry (15), the powers z^1..z^{2 n_max}
    (2 n_max complex products, 6 flops each), 2 n_max + 3 complex multiply-adds into G (8 each)
    and 2 n_max + 1 real x complex multiply-adds into W (4 each): 36 n_max + 43."""
    return 15 + 6 * 2 * n_max + 8 * (2 * n_max + 3) + 4 * (2 * n_max + 1)


def kernel_flops_per_pair(n_max: int) -> int:
    """The flops the moment kernel's own formulation needs per pair (fewer than the plain form:
    with real weights, G_m and G_-m come from the same two real sums A_m = sum w g1 z^m and
    B_m = sum w g2 z^m): unit vector (6), powers z^2..z^{2 n_max} (6 each), A_m and B_m for
    m <= n_max + 3 (4 each), W_m for m <= 2 n_max (4 each)."""
    return 6 + 6 * (2 * n_max - 1) + 8 * (n_max + 4) + 4 * (2 * n_max + 1)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_setup(name: str, n: int = 0):
    """Parameters of a named workload; n > 0 rescales it to n galaxies at the same density."""
    from paper_2309_08601_gb300 import synth
    p = dict(synth.WORKLOADS[name])
    if n:
        p["side"] = p["side"] * float(np.sqrt(n / p["n"]))
        p["n"] = int(n)
    setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                 n_max=p["n_max"])
    theta = [[t, t, t] for t in p["theta_ap"]]
    return p, setup, theta


def workload_config(name, p, precision):
    return {"workload": name, "n_galaxies": p["n"], "patch_arcmin": p["side"], "field": p["field"],
            "n_bins": p["n_bins"], "theta_min_arcmin": p["theta_min"], "theta_max_arcmin": p["theta_max"],
            "n_max": p["n_max"], "n_phi": 100, "theta_ap_arcmin": p["theta_ap"], "precision": precision,
            "l2": "inputs (catalog 4 MB) are L2-resident by design; a 256 MiB buffer is written "
                  "between steps to flush L2", "parallelism": "one catalog per GPU"}


# ------------------------------------------------------------------ oracle (CPU) timing

def oracle_sample(cat, setup, theta, target_s: float, seed: int = 0):
    """Runs the FP64 oracle's whole path on a centre subset sized for about target_s seconds.
    Returns (pairs, seconds, n_centres, threads)."""
    import oracle
    s = oracle.Setup(**setup)
    rng = np.random.default_rng(seed)
    order = rng.permutation(cat.n)
    # calibrate on a few centres, then size the sample
    nprobe = 4 * oracle.num_threads()
    probe = np.sort(order[:nprobe])
    t0 = time.perf_counter()
    pp = oracle.count_pairs(s, cat, probe)
    G, W = oracle.moments(s, cat, probe)
    oracle.contract(s, cat, G, W, probe)
    dt = max(time.perf_counter() - t0, 1e-3)
    per_centre = dt / nprobe
    k = int(np.clip(target_s / per_centre, 8, cat.n))
    cen = np.sort(order[:k])
    pairs = oracle.count_pairs(s, cat, cen)
    t0 = time.perf_counter()
    r = oracle.pipeline(s, cat, theta, cen)
    sec = time.perf_counter() - t0
    del r, pp
    return pairs, sec, k, oracle.num_threads()


def measure_adjoint(api, est, dev, theta, stream):
    """One forward and one backward of the differentiable Map^3 (api.map3) on the bench catalog,
    each timed with CUDA events (after one untimed pair); L = sum of the Map^3 measures."""
    import torch
    xq, yq, g1, g2, w = dev[:5]

    def once():
        a1, a2, aw = (t.clone().requires_grad_(True) for t in (g1, g2, w))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        m8 = api.map3(est, xq, yq, a1, a2, aw, theta)
        L = m8[..., 0].sum()
        ev[1].record(stream)
        L.backward()
        ev[2].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), a1.grad, float(L.detach())

    once()
    fwd, bwd, gr, L = once()
    return {"loss": "sum of Map^3 over the apertures", "forward_ms": fwd, "backward_ms": bwd,
            "backward_over_forward": bwd / fwd, "grad_finite": bool(torch.isfinite(gr).all()),
            "kernels": "map3/to_gamma/edge_correct adjoints, contraction adjoint, moments adjoint"}


def measure_batch(api, n_real: int, precision: str, stream):
    """n_real realisations of the tomographic batching workload through one mp3pcf_run_batch call
    (the largest catalog sizes the workspace, the others replay a captured CUDA graph)."""
    import torch
    from paper_2309_08601_gb300 import synth
    tp = synth.WORKLOADS["tomo_64x5_lognormal"]
    bset = dict(n_bins=tp["n_bins"], theta_min=tp["theta_min"], theta_max=tp["theta_max"],
                n_max=tp["n_max"], n_z=tp["n_z"])
    bth = [[t, t, t] for t in tp["theta_ap"]]
    cats = [synth.make_tomographic_catalog(1000 + r, side=tp["side"], n_z=tp["n_z"]) for r in range(n_real)]
    devs = [api.catalog_to_device(c) for c in cats]
    ext = (0, 0, int(np.ceil(tp["side"] / synth.QUANTUM)), int(np.ceil(tp["side"] / synth.QUANTUM)))
    with api.Estimator(**bset, precision=precision, stream=stream) as eb:
        pairs = 0
        for d in devs:  # untimed: the pair counter holds the last accumulation
            eb.accumulate_moments(*d[:5], zbin=d[5])
            pairs += eb.counts()[1]
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        m8 = eb.run_batch([d[:5] + (d[5],) for d in devs], ext, bth, use_graphs=True)
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        launches, inst = eb.graph_stats()
        finite = bool(torch.isfinite(m8).all())
    return {"workload": "tomo_64x5_lognormal: %d of the 64 realisations, 5 z-bins of U{50k..400k} "
                        "galaxies on 300', all 125 Z-triplets" % n_real,
            "galaxies": [int(c.n) for c in cats], "pairs": int(pairs), "seconds": sec,
            "catalogs_per_s": n_real / sec, "pairs_per_s": pairs / sec,
            "graph_launches": launches, "graph_instantiations": inst, "m8_finite": finite}


def measure_combined(api, precision: str, stream):
    """The combined estimator (Sec. 3.3) against the discrete one on the multiscale_310k workload
    (the density and binning of the paper's accuracy test of it, a tenth of its area): moments and
    contraction of each, timed with CUDA events after one untimed run; the levels start at 20
    pixels of 0.25' and double the pixel every octave, as in that test."""
    import torch
    from paper_2309_08601_gb300 import synth
    p = synth.WORKLOADS["multiscale_310k"]
    cat = synth.workload_catalog("multiscale_310k")
    dev = api.catalog_to_device(cat)
    cset = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"], n_max=p["n_max"])
    with api.Estimator(**cset, precision=precision, stream=stream) as ec:
        edges = ec.bin_edges()[0]
        levels = synth.grid_levels(edges, int(round(p["grid_base_arcmin"] / synth.QUANTUM)), synth.QUANTUM)

        def run(combined):
            if combined:
                ec.accumulate_moments_combined(*dev[:5], levels=levels)
            else:
                ec.accumulate_moments(*dev[:5])
            return ec.contract()

        out = {}
        for combined in (False, True):
            run(combined)
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            ups, norm = run(combined)
            t1.record(stream)
            torch.cuda.synchronize()
            out[combined] = (t0.elapsed_time(t1), ec.counts()[1], ups.cpu().numpy(), norm.cpu().numpy())
    b0 = levels[0][0]
    nb = p["n_bins"]
    grid = np.zeros((nb, nb), bool)
    grid[b0:, :] = grid[:, b0:] = True
    ud, nd, uc, nc = out[False][2], out[False][3], out[True][2], out[True][3]

    def nerr(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    return {"workload": "multiscale_310k: %d galaxies on %g' (noise-free lognormal), %d bins %g'-%g', n_max %d"
                        % (cat.n, p["side"], nb, p["theta_min"], p["theta_max"], p["n_max"]),
            "levels": [[int(b), float(q * synth.QUANTUM)] for b, q in levels],
            "discrete_ms": out[False][0], "combined_ms": out[True][0], "speedup": out[False][0] / out[True][0],
            "discrete_pairs": int(out[False][1]), "combined_pairs": int(out[True][1]),
            "grid_blocks_rel_err_upsilon_n_le_10": nerr(uc[:, :, :11][..., grid], ud[:, :, :11][..., grid]),
            "grid_blocks_rel_err_norm_n_le_20": nerr(nc[:, :21][..., grid], nd[:, :21][..., grid]),
            "discrete_block_rel_err": float(np.abs(uc[..., ~grid] - ud[..., ~grid]).max() /
                                            np.abs(ud[..., ~grid]).max())}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2309_08601_gb300 import synth
    oracle.build_oracle()
    p, setup, theta = workload_setup(args.workload, args.n)
    cat = synth.make_catalog(p["n"], p["side"], p["seed"], field=p["field"], weights=p["weights"],
                             holes=p.get("holes", False))
    for _ in range(args.warmup):
        oracle_sample(cat, setup, theta, target_s=2.0, seed=99)
    tot_pairs, tot_s, cents = 0, 0.0, 0
    for k in range(args.steps):
        pairs, sec, nc, threads = oracle_sample(cat, setup, theta, target_s=args.ref_step_s, seed=k)
        tot_pairs += pairs
        tot_s += sec
        cents += nc
    value = tot_pairs / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.workload, p, "fp64-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d random centres per step (all %d galaxies as neighbours), "
                                       "whole path" % (cents // max(args.steps, 1), cat.n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ multi-rank host logic

def rank_seed(seed: int, rank: int) -> int:
    """Catalog seed of a rank: every rank measures its own independent realisation (weak scaling)."""
    return seed + 1000 * rank


def reduce_over_ranks(values, op: str, dist=None):
    """Reduces a list of floats over the process group ('max' or 'sum'); identity on one rank.
    NCCL groups reduce on the current CUDA device, gloo groups on the host."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    dev = torch.device("cpu")
    if dist.get_backend() == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return [float(v) for v in t.cpu()]


def whole_job(units_per_step_all_ranks: float, steps: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_step_all_ranks * steps / seconds_max


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2309_08601_gb300 import api, native, synth
    if rank == 0:
        from paper_2309_08601_gb300.build import build_native
        build_native()
    if dist is not None:
        dist.barrier()
    native.lib()

    p, setup, theta = workload_setup(args.workload, args.n)
    cat = synth.make_catalog(p["n"], p["side"], rank_seed(p["seed"], rank), field=p["field"],
                             weights=p["weights"], holes=p.get("holes", False))
    dev = api.catalog_to_device(cat)
    stream = torch.cuda.current_stream()
    est = api.Estimator(**setup, precision=args.precision, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        return est.measure(*dev[:5], theta_ap=theta, report_singular=False)

    for _ in range(max(args.warmup, 0)):
        m = step()
    torch.cuda.synchronize()
    n_centres, pairs = est.counts()
    est.set_timing(True)
    est.stage_times(reset=True)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        m = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks.stop()
    ms = ev0.elapsed_time(ev1)
    stages = est.stage_times(reset=True)
    est.set_timing(False)
    ms_max = reduce_over_ranks([ms], "max", dist)[0]
    pairs_all = reduce_over_ranks([pairs], "sum", dist)[0]  # each rank has its own catalog
    sec = ms_max / 1e3
    value = whole_job(pairs_all, args.steps, sec)
    cat_per_s = whole_job(world, args.steps, sec)

    # ---- roofline of the dominant kernel (stage a, FP32 FMA pipe)
    k1_ms = stages["moments"][0] / args.steps
    fpp = flops_per_pair(p["n_max"])
    achieved = fpp * pairs / (k1_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "moments_kernel<float,30>", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": (args.k1_traffic if args.k1_traffic is not None else
                            (MOMENTS_TRAFFIC_BYTES if (args.workload == "lognormal_200k" and not args.n
                                                       and args.precision != "fp64") else None)),
                "traffic_note": "ncu DRAM read+write, capture at 50 000 galaxies scaled by centres",
                "flops_per_pair": fpp, "pairs_per_launch": pairs,
                "kernel_flops_per_pair": kernel_flops_per_pair(p["n_max"]),
                "frac_kernel_flops": kernel_flops_per_pair(p["n_max"]) * pairs / (k1_ms / 1e3) / 1e12
                / FP32_PEAK_TFLOPS,
                "launch_ms": k1_ms, "peak_source": PEAK_NOTE}
    launches = sum(v[1] for v in stages.values())
    # ---- stage (b): HBM-bound; algorithmic bytes = every moment row read once (complex, moment
    # precision) + the FP64 partial sums written and read once by the slice reduction
    k2_ms = stages["contract"][0] / args.steps
    esz = 16 if args.precision == "fp64" else 8
    nbins, nmax = p["n_bins"], p["n_max"]
    k2_bytes = n_centres * nbins * ((2 * nmax + 3) + (2 * nmax + 1)) * esz
    roofline_contract = {"bound": "hbm", "kernel": "contract (%s)" % args.precision,
                         "achieved": k2_bytes / (k2_ms / 1e3) / 1e9, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                         "frac": k2_bytes / (k2_ms / 1e3) / 1e9 / HBM_PEAK_GBS, "bytes_per_launch": k2_bytes,
                         "launch_ms": k2_ms, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "traffic": (CONTRACT_TRAFFIC_BYTES if (args.workload == "lognormal_200k" and not args.n
                                                                and args.precision == "bf16x3") else None),
                         "traffic_note": "ncu DRAM read+write, capture at 50 000 galaxies scaled by centres"}

    # ---- end to end through the public API with host buffers
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
            (cat.xq, cat.yq, cat.g1, cat.g2, cat.w)]
    h2d = sum(h.numel() * h.element_size() for h in host)
    out_host = torch.empty((1, len(theta), 8), dtype=torch.float64).pin_memory()
    d2h = out_host.numel() * out_host.element_size()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        for d, h in zip(dev[:5], host):
            d.copy_(h, non_blocking=True)
        m = step()
        out_host.copy_(m.m8, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_over_ranks([e2e_s], "max", dist)[0]
    e2e = {"value": whole_job(pairs_all, args.steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    m8_fp32 = m.m8.cpu().numpy()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded lognormal Kaiser-Squires shear + shape noise)",
            "config": workload_config(args.workload, p, args.precision),
            "catalogs_per_s": cat_per_s, "pairs_per_catalog": pairs,
            "pairs_per_s_moments_kernel": pairs / (k1_ms / 1e3),
            "moment_terms_per_s": pairs * ((2 * nmax + 3) + (2 * nmax + 1)) / (k1_ms / 1e3),
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "roofline": roofline, "roofline_contract": roofline_contract, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks.summary()}

    # ---- the plain FP64 GPU path on the same catalog (rank 0, one untimed-warmup + one run)
    if rank == 0 and args.fp64_compare:
        with api.Estimator(**setup, precision="fp64", stream=stream) as e64:
            sub = torch.zeros(cat.n, dtype=torch.uint8, device="cuda")
            sub[:64] = 1
            e64.measure(*dev[:5], theta_ap=theta, centre_mask=sub, report_singular=False)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            m64 = e64.measure(*dev[:5], theta_ap=theta, report_singular=False)
            a1.record(stream)
            torch.cuda.synchronize()
            s64 = a0.elapsed_time(a1) / 1e3
            m8_64 = m64.m8.cpu().numpy()
        err = float(np.abs(m8_fp32[..., 0] - m8_64[..., 0]).max() / np.abs(m8_64[..., 0]).max())
        err_all = float(np.abs(m8_fp32 - m8_64).max() / np.abs(m8_64).max())
        line["fp64_path"] = {"catalogs_per_s": 1.0 / s64, "pairs_per_s": pairs / s64,
                             "speedup_of_measured_path": (cat_per_s / world) * s64,
                             "map3_rel_err_vs_fp64": err, "m8_rel_err_vs_fp64": err_all}

    # ---- the differentiation form on the same catalog: forward + backward through api.map3
    if rank == 0 and args.adjoint:
        line["adjoint"] = measure_adjoint(api, est, dev, theta, stream)

    # ---- the batching form: whole tomographic realisations (5 z-bins of 50k-400k galaxies)
    # through mp3pcf_run_batch with CUDA graphs, rank 0; pairs counted by an untimed pass
    if rank == 0 and args.batch_realisations > 0:
        line["batch"] = measure_batch(api, args.batch_realisations, args.precision, stream)

    # ---- the combined estimator against the discrete one (rank 0)
    if rank == 0 and args.combined:
        line["combined"] = measure_combined(api, args.precision, stream)

    if rank == 0 and args.cpu_baseline:
        import oracle
        pr, sec, k, threads = oracle_sample(cat, setup, theta, target_s=args.cpu_s)
        line["cpu_baseline"] = {"value": pr / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d random centres (all %d galaxies as neighbours), whole "
                                          "path, %.1f s" % (k, cat.n, sec),
                                "cpu_model": cpu_model()}
        if threads > 1:
            oracle.set_num_threads(1)
            pr1, sec1, k1, _ = oracle_sample(cat, setup, theta, target_s=args.cpu_s / 2, seed=1)
            oracle.set_num_threads(threads)
            line["cpu_baseline"]["one_core"] = {
                "value": pr1 / sec1, "unit": UNIT, "cores": 1,
                "sample": "%d random centres, whole path, %.1f s" % (k1, sec1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    est.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lognormal_200k")
    ap.add_argument("--n", type=int, default=0,
                    help="rescale the workload to n galaxies at the same density (profiling runs)")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp32", "fp64"],
                    help="bf16x3 (default): FP32 moments, BF16 hi+lo tensor-core contraction, FP64 "
                         "edge correction and sums")
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-s", type=float, default=12.0, help="seconds of oracle work sampled")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the forward + backward timing of the differentiable Map^3")
    ap.add_argument("--batch-realisations", type=int, default=2,
                    help="tomographic realisations timed through mp3pcf_run_batch (0: skip)")
    ap.add_argument("--no-combined", dest="combined", action="store_false",
                    help="skip the combined-versus-discrete estimator timing")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--k1-traffic", type=float, default=None,
                    help="DRAM bytes per moments launch (default: the committed ncu figure, at "
                         "the lognormal_200k workload only)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
