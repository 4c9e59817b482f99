#!/usr/bin/env python3
"""Benchmark of the multipole shear-3PCF hot path on GB300.

One step = the whole path on one catalog: cell sort, moments (stage a), multipole contraction
(stage b), edge correction, Gamma^x and Gamma^cen, and the aperture measures. The headline
workload is the largest single-GPU configuration, the masked precision-form catalog: 10^6
galaxies on a 600'x600' patch with circular holes covering 15 % of it, lognormal
Kaiser-Squires shear plus shape noise, 30 log bins 0.5'-240', n_max = 40, Map^3 at 2', 4', 8',
16', FP32 moments with the BF16x3 tensor-core contraction. Beside it: the plain FP64 GPU path on
an exact centre subset of the same catalog (extrapolated by pairs), the precision form against
the oracle on sampled centres, the 200k-galaxy lognormal catalog, the differentiation and
batching forms, the combined estimator and the oracle on the host cores. With N GPUs (torchrun)
every rank measures its own catalog realisation (independent problems, weak scaling, no
data-path collective).

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
# FP32 FMA pipe of a GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2070 MHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (derived from unit counts and clock)"
DEFAULT_WORKLOAD = "masked_lognormal_1m"
MOMENT_KERNEL_NMAX = (4, 10, 20, 30, 40, 50)  # compiled order sets of moments_kernel<T, NMAX>


def _measured_hbm_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (one earlier copy measurement on a GB300; of fallback)"


HBM_PEAK_GBS, HBM_PEAK_NOTE = _measured_hbm_gbs()
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it stands, per
# (kernel, workload), scaled to the workload's centres where the capture was a smaller catalog of
# the same density (the traffic of both kernels is proportional to the centres); None until the
# kernel has been captured since its last change.
TRAFFIC_BYTES = {
    # moments_kernel<float,40>: capture at 100 000 galaxies of the same density, x10
    # (profiles/moments_kernel_masked_lognormal_100k.md)
    ("moments", "masked_lognormal_1m"): 10 * (630.813440e6 + 4.473916e9),
    # moments_kernel<float,30>: capture at 50 000 galaxies of the same density, x4
    # (profiles/moments_kernel_lognormal_50k.md)
    ("moments", "lognormal_200k"): 4 * (147.244544e6 + 1.073786e9),
    # contract_tc_kernel<Bf16Split>: captures at 50 000 galaxies of each density, x20 and x4
    # (profiles/contract_tc_bf16x3_traffic_50k.md)
    ("contract", "masked_lognormal_1m"): 20 * (1.981240576e9 + 35.888640e6),
    ("contract", "lognormal_200k"): 4 * (993.852928e6 + 19.601408e6),
}
TRAFFIC_NOTE = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (profiles/)"


def compiled_nmax(n_max: int) -> int:
    """n_max of the moment kernel instantiation that serves n_max (the smallest compiled set)."""
    for k in MOMENT_KERNEL_NMAX:
        if n_max <= k:
            return k
    raise ValueError("n_max above the compiled range")


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
    """The workload a bench line measures; both arms print the same dict (the reference arm's own
    arithmetic, FP64, is in its dtype)."""
    return {"workload": name, "n_galaxies": p["n"], "patch_arcmin": p["side"], "field": p["field"],
            "masked_holes": bool(p.get("holes", False)), "n_bins": p["n_bins"],
            "theta_min_arcmin": p["theta_min"], "theta_max_arcmin": p["theta_max"], "n_max": p["n_max"],
            "n_phi": 100, "theta_ap_arcmin": ",".join("%g" % t for t in p["theta_ap"]),
            "precision": precision,
            "l2": "inputs (catalog %d MB) are L2-resident by design; a 256 MiB buffer is written "
                  "between steps to flush L2" % max(1, int(round(p["n"] * 24 / 1e6))),
            "parallelism": "one catalog per GPU"}


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


def measure_adjoint(api, precision: str, stream):
    """The differentiation form on its own workload (grad_lognormal_500k: 5e5 galaxies on 420',
    20 bins 0.5'-120', n_max 30, Map^3 at 4', 8', 16'): one forward and one backward of the
    differentiable Map^3 (api.map3, L = sum of Map^3 over the apertures), each timed with CUDA
    events after one untimed pair."""
    import torch
    from paper_2309_08601_gb300 import synth
    p, setup, theta = workload_setup("grad_lognormal_500k")
    cat = synth.workload_catalog("grad_lognormal_500k")
    dev = api.catalog_to_device(cat)
    xq, yq, g1, g2, w = dev[:5]
    with api.Estimator(**setup, precision=precision, stream=stream) as est:
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
            return ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), (a1.grad, a2.grad, aw.grad), L

        once()
        fwd, bwd, grads, L = once()
        # exact identities of the gradient: Map^3 is cubic in the shears and of degree 0 in the
        # weights, so sum g dL/dg = 3 L and sum w dL/dw = 0
        eg = float((g1.double() * grads[0].double() + g2.double() * grads[1].double()).sum())
        ew = w.double() * grads[2].double()
        Lf = float(L.detach())
    return {"workload": "grad_lognormal_500k: %d galaxies on %g', %d bins %g'-%g', n_max %d"
                        % (cat.n, p["side"], p["n_bins"], p["theta_min"], p["theta_max"], p["n_max"]),
            "loss": "sum of Map^3 over the apertures", "forward_ms": fwd, "backward_ms": bwd,
            "backward_over_forward": bwd / fwd,
            "grad_finite": bool(all(torch.isfinite(g).all() for g in grads)),
            "homogeneity_rel_err_gamma": abs(eg - 3 * Lf) / max(abs(3 * Lf), 1e-300),
            "homogeneity_rel_err_w": abs(float(ew.sum())) / max(float(ew.abs().sum()), 1e-300),
            "kernels": "map3/to_gamma/edge_correct adjoints, contraction adjoint, moments adjoint"}


def measure_batch(api, n_real: int, precision: str, stream, fp64_frac: float):
    """n_real realisations of the tomographic batching workload through one mp3pcf_run_batch call
    (the largest catalog sizes the workspace, the others replay a captured CUDA graph), and the
    plain FP64 GPU path on an exact random centre subset of the first realisation, extrapolated to
    the whole realisation by its pairs."""
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
        pairs_each = []
        for d in devs:  # untimed: the pair counter holds the last accumulation
            eb.accumulate_moments(*d[:5], zbin=d[5])
            pairs_each.append(eb.counts()[1])
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        m8 = eb.run_batch([d[:5] + (d[5],) for d in devs], ext, bth, use_graphs=True)
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        launches, inst = eb.graph_stats()
        finite = bool(torch.isfinite(m8).all())
    pairs = int(sum(pairs_each))
    out = {"workload": "tomo_64x5_lognormal: %d of the 64 realisations, 5 z-bins of U{50k..400k} "
                       "galaxies on 300', all 125 Z-triplets" % n_real,
           "galaxies": [int(c.n) for c in cats], "pairs": pairs, "seconds": sec,
           "catalogs_per_s": n_real / sec, "pairs_per_s": pairs / sec,
           "seconds_for_64_extrapolated": 64 * sec / n_real,
           "extrapolation": "64 realisations at the measured seconds per realisation (counts are drawn "
                            "from the same distribution)",
           "graph_launches": launches, "graph_instantiations": inst, "m8_finite": finite}
    if fp64_frac > 0:
        c0 = cats[0]
        rng = np.random.default_rng(13)
        sel = torch.as_tensor((rng.random(c0.n) < fp64_frac).astype(np.uint8), device="cuda")
        d0 = devs[0]
        res = {}
        for prec in ("fp64", precision):
            with api.Estimator(**bset, precision=prec, stream=stream) as e:
                e.measure(*d0[:5], theta_ap=bth, zbin=d0[5], centre_mask=sel, report_singular=False)
                torch.cuda.synchronize()
                e.set_timing(True)
                e.stage_times(reset=True)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                m = e.measure(*d0[:5], theta_ap=bth, zbin=d0[5], centre_mask=sel, report_singular=False)
                a1.record(stream)
                torch.cuda.synchronize()
                st = e.stage_times(reset=True)
                e.set_timing(False)
                res[prec] = (a0.elapsed_time(a1) / 1e3, e.counts()[1], m.m8.cpu().numpy(),
                             {k: v[0] for k, v in st.items()})
        s64, p64, m64, _ = res["fp64"]
        sp, _, mp, stp = res[precision]
        frac = p64 / pairs_each[0]
        fp64_cat_s = frac / s64  # realisations per second, extrapolated by pairs
        auto = np.zeros(m64.shape[0], bool)
        for z in range(tp["n_z"]):
            auto[(z * tp["n_z"] + z) * tp["n_z"] + z] = True
        out["fp64_path"] = {
            "sample": "exact random centre subset (%.1f %% of the pairs) of realisation 0, whole path "
                      "with those centres; catalogs/s extrapolated to the whole realisation by pairs"
                      % (100 * frac),
            "fp64_catalogs_per_s": fp64_cat_s, "fp64_pairs_per_s": p64 / s64,
            "precision_over_fp64_same_subset": s64 / sp,
            "batched_over_fp64_catalogs_per_s": (n_real / sec) / fp64_cat_s,
            "map3_rel_err_vs_fp64_auto_triplets": float(np.abs(mp[auto, :, 0] - m64[auto, :, 0]).max() /
                                                        np.abs(m64[auto, :, 0]).max()),
            "precision_stage_ms_on_subset": stp,
            "contraction_over_moments": stp["contract"] / max(stp["moments"], 1e-9)}
    return out


def measure_combined(api, precision: str, stream, name: str = "multiscale_310k"):
    """The combined estimator (Sec. 3.3) against the discrete one on a noise-free multi-scale
    workload (the density and binning of the paper's accuracy test of it: multiscale_310k on a
    tenth of its area, multiscale_3m on all of it): moments and contraction of each, timed with
    CUDA events after one untimed run, with the grid levels by direct pixel-pair sums and by FFT
    convolution (grid_fft); the levels start at 20 pixels of 0.25' and double the pixel every
    octave up to 1', as in that test. Differences against the discrete estimator: the multipoles
    norm-wise over every block with a grid bin, and the centroid-projected Gamma_0 of the
    equal-side bins (largest difference over phi, and at phi = 60 deg, relative to the largest
    |Gamma_0|: the measure of the paper's figure)."""
    import torch
    from paper_2309_08601_gb300 import synth
    p = synth.WORKLOADS[name]
    cat = synth.workload_catalog(name)
    dev = api.catalog_to_device(cat)
    cset = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"], n_max=p["n_max"])
    out = {}
    levels = None
    for mode in ("discrete", "direct", "fft"):
        with api.Estimator(**cset, precision=precision, stream=stream, grid_fft=(mode == "fft")) as ec:
            if levels is None:
                edges = ec.bin_edges()[0]
                levels = synth.grid_levels(edges, int(round(p["grid_base_arcmin"] / synth.QUANTUM)), synth.QUANTUM,
                                           max_q=int(round(p["grid_max_arcmin"] / synth.QUANTUM)))

            def run():
                if mode == "discrete":
                    ec.accumulate_moments(*dev[:5])
                else:
                    ec.accumulate_moments_combined(*dev[:5], levels=levels)
                return ec.contract()

            run()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            ups, norm = run()
            t1.record(stream)
            torch.cuda.synchronize()
            gam, _ = ec.edge_correct(ups, norm, report_singular=False)
            g0 = ec.to_gamma(gam, 1)[0, 0].cpu().numpy()
            out[mode] = (t0.elapsed_time(t1), ec.counts()[1], ups.cpu().numpy(), norm.cpu().numpy(), g0)
    b0 = levels[0][0]
    nb = p["n_bins"]
    grid = np.zeros((nb, nb), bool)
    grid[b0:, :] = grid[:, b0:] = True
    ud, nd, gd = out["discrete"][2], out["discrete"][3], out["discrete"][4]
    k60 = [int(np.floor(gd.shape[-1] / 6.0 - 0.5)), int(np.ceil(gd.shape[-1] / 6.0 - 0.5))]

    def nerr(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    res = {"workload": "%s: %d galaxies on %g' (noise-free lognormal, P(k) ~ k^%g), %d bins %g'-%g', n_max %d"
                       % (name, cat.n, p["side"], p.get("slope", -1.5), nb, p["theta_min"], p["theta_max"],
                          p["n_max"]),
           "levels": [[int(b), float(q * synth.QUANTUM)] for b, q in levels],
           "discrete_ms": out["discrete"][0], "discrete_pairs": int(out["discrete"][1])}
    for mode in ("direct", "fft"):
        uc, nc, gcm = out[mode][2], out[mode][3], out[mode][4]
        eq = [float(np.abs(gcm[b, b] - gd[b, b]).max() / np.abs(gd[b, b]).max()) for b in range(b0, nb)]
        eq60 = [float(np.abs(gcm[b, b, k60] - gd[b, b, k60]).max() / np.abs(gd[b, b, k60]).max())
                for b in range(b0, nb)]
        res[mode] = {"ms": out[mode][0], "speedup": out["discrete"][0] / out[mode][0],
                     "pairs_counted": int(out[mode][1]),
                     "grid_blocks_rel_err_upsilon_n_le_3": nerr(uc[:, :, :4][..., grid], ud[:, :, :4][..., grid]),
                     "grid_blocks_rel_err_upsilon_n_le_10": nerr(uc[:, :, :11][..., grid], ud[:, :, :11][..., grid]),
                     "grid_blocks_rel_err_norm_n_le_20": nerr(nc[:, :21][..., grid], nd[:, :21][..., grid]),
                     "equal_sides_gamma0_rel_err_over_phi_median": float(np.median(eq)),
                     "equal_sides_gamma0_rel_err_over_phi_max": float(np.max(eq)),
                     "equilateral_gamma0_rel_err_median": float(np.median(eq60)),
                     "equilateral_gamma0_rel_err_max": float(np.max(eq60)),
                     "discrete_block_rel_err": float(np.abs(uc[..., ~grid] - ud[..., ~grid]).max() /
                                                     np.abs(ud[..., ~grid]).max())}
    res["fft_vs_direct_upsilon_rel_err"] = nerr(out["fft"][2], out["direct"][2])
    res["fft_vs_direct_norm_rel_err"] = nerr(out["fft"][3], out["direct"][3])
    return res


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
            "data": "synthetic (seeded lognormal Kaiser-Squires shear + shape noise)",
            "config": workload_config(args.workload, p, args.precision), "oracle_precision": "fp64",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d random centres per step (all %d galaxies as neighbours), "
                                       "whole path" % (cents // max(args.steps, 1), cat.n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_oracle_plan(args):
    """The oracle's timing plan on the host cores (part of the reference arm). Per workload: the
    pair-proportional part of the path (moments and contraction) on a random centre sample (all
    galaxies as neighbours; the whole uniform_noise_2k catalog), with all cores and with one,
    median of three runs, giving pairs/s; and the per-catalog post-processing (edge correction,
    Gamma, aperture measures), timed once with all cores and once with one. A whole catalog's
    seconds = its pairs / that rate + the post-processing, the pairs estimated from the sample
    (a uniform random subset of the centres). Prints one JSON line per workload."""
    import oracle
    from paper_2309_08601_gb300 import synth
    oracle.build_oracle()
    threads = oracle.num_threads()
    plan = [("uniform_noise_2k", None), ("lognormal_200k", 6.0), ("masked_lognormal_1m", 6.0),
            ("grad_lognormal_500k", 6.0), ("tomo_64x5_lognormal", 6.0)]
    for name, target in plan:
        p = synth.WORKLOADS[name]
        if name == "tomo_64x5_lognormal":
            cat = synth.make_tomographic_catalog(1000, side=p["side"], n_z=p["n_z"])
            setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"],
                         n_max=p["n_max"], n_z=p["n_z"])
        else:
            cat = synth.workload_catalog(name)
            setup = dict(n_bins=p["n_bins"], theta_min=p["theta_min"], theta_max=p["theta_max"], n_max=p["n_max"])
        theta = [[t, t, t] for t in p["theta_ap"]]
        s = oracle.Setup(**setup)
        row = {"workload": name, "n_galaxies": int(cat.n), "cpu_model": cpu_model()}

        def pair_part(cen):
            t0 = time.perf_counter()
            G, W = oracle.moments(s, cat, cen)
            ups, norm = oracle.contract(s, cat, G, W, cen)
            return time.perf_counter() - t0, ups, norm

        for nt in (threads, 1):
            oracle.set_num_threads(nt)
            rates = []
            for rep in range(3):
                rng = np.random.default_rng(100 + rep)
                if target is None:
                    cen = np.arange(cat.n)
                else:
                    # size the sample for about target seconds (one core: half of it)
                    order = rng.permutation(cat.n)
                    probe = np.sort(order[:max(2, 2 * nt)])
                    per = max(pair_part(probe)[0], 1e-3) / probe.size
                    k = int(np.clip((target if nt > 1 else target / 2) / per, 2, cat.n))
                    cen = np.sort(order[:k])
                pairs = oracle.count_pairs(s, cat, cen)
                sec, ups, norm = pair_part(cen)
                rates.append((pairs / sec, pairs, cen.size, sec))
            rates.sort()
            rate, pairs, k, sec = rates[1]
            full_pairs = pairs * cat.n / k
            t0 = time.perf_counter()
            gam, _ = oracle.edge_correct(s, ups, norm)
            gc = oracle.to_gamma(s, gam, 1)
            oracle.to_map3(s, gc, theta)
            post = time.perf_counter() - t0
            row["cores_%d" % nt] = {"pairs_per_s": rate, "centres_sampled": int(k), "sample_seconds": sec,
                                    "post_seconds": post, "catalog_seconds": full_pairs / rate + post,
                                    "catalog_seconds_kind": "measured" if k == cat.n else "extrapolated by pairs"}
        row["pairs_per_catalog_estimate"] = float(full_pairs)
        oracle.set_num_threads(threads)
        print(json.dumps(row), flush=True)
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

def measure_peaks(native):
    """FP32 FMA (scalar and packed two-lane), FP64 FMA and tcgen05 BF16 / TF32 MMA throughput of
    this GPU, measured by the library's probe (mp3pcf_measure_peak), in TFLOP/s, with the probe's
    SM clock."""
    import ctypes as C
    out = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32_ffma2"), (2, "fp64_fma"), (3, "bf16_tcgen05"), (4, "tf32_tcgen05")):
        f, mhz = C.c_double(0.0), C.c_double(0.0)
        native.check(native.lib().mp3pcf_measure_peak(kind, None, C.byref(f), C.byref(mhz)), "measure_peak")
        out[name + "_tflops"] = f.value / 1e12
        out[name + "_sm_mhz_estimate"] = mhz.value
    return out


def time_steps(step, steps, stream):
    """CUDA-event time (ms) of `steps` calls of step() on `stream`, L2 flushed before each."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    m = None
    for k in range(steps):
        flush.fill_(k & 0xFF)
        m = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), m


def moment_roofline(name, n_max, pairs, k1_ms, precision, peaks):
    """Roofline of stage (a) on the FP32 FMA pipe: algorithmic flops (the plain form of
    Eq. Gn_disc, flops_per_pair) x pairs per launch / launch time, against the derived peak;
    the kernel's own flop count and the measured probe peaks are reported beside it."""
    fpp = flops_per_pair(n_max)
    achieved = fpp * pairs / (k1_ms / 1e3) / 1e12
    kfl = kernel_flops_per_pair(n_max) * pairs / (k1_ms / 1e3) / 1e12
    r = {"bound": "alu", "kernel": "moments_kernel<float,%d>" % compiled_nmax(n_max), "achieved": achieved,
         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
         "traffic": TRAFFIC_BYTES.get(("moments", name)) if precision != "fp64" else None,
         "traffic_note": TRAFFIC_NOTE, "flops_per_pair": fpp, "pairs_per_launch": pairs,
         "kernel_flops_per_pair": kernel_flops_per_pair(n_max),
         "frac_kernel_flops": kfl / FP32_PEAK_TFLOPS, "launch_ms": k1_ms, "peak_source": PEAK_NOTE}
    if peaks:
        meas = max(peaks["fp32_fma_tflops"], peaks["fp32_ffma2_tflops"])
        r["peak_measured"] = meas
        r["frac_of_measured"] = achieved / meas
        r["peak_measured_source"] = "mp3pcf_measure_peak: best of FP32 FMA and packed FFMA2 probes"
    return r


def contract_roofline(name, n_centres, n_bins, n_max, n_z, k2_ms, precision):
    """Roofline of stage (b) on HBM: every moment row read once (complex, moment precision)."""
    esz = 16 if precision == "fp64" else 8
    k2_bytes = n_centres * n_z * n_bins * ((2 * n_max + 3) + (2 * n_max + 1)) * esz
    achieved = k2_bytes / (k2_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": "contract (%s)" % precision, "achieved": achieved, "peak": HBM_PEAK_GBS,
            "unit": "GB/s", "frac": achieved / HBM_PEAK_GBS, "bytes_per_launch": k2_bytes, "launch_ms": k2_ms,
            "peak_source": HBM_PEAK_NOTE,
            "traffic": TRAFFIC_BYTES.get(("contract", name)) if precision == "bf16x3" else None,
            "traffic_note": TRAFFIC_NOTE}


def measure_fp64_subset(api, dev, n, setup, theta, pairs_full, precision, stream, frac, seed=11):
    """The plain FP64 GPU path (FP64 moments, FP64 CUDA-core contraction, FP64 post-processing)
    on an exact random centre subset of the catalog, and the precision form on the same centres;
    FP64 catalogs/s extrapolated to the whole catalog by its pairs."""
    import torch
    rng = np.random.default_rng(seed)
    sel = torch.as_tensor((rng.random(n) < frac).astype(np.uint8), device="cuda")
    res = {}
    for prec in ("fp64", precision):
        with api.Estimator(**setup, precision=prec, stream=stream) as e:
            e.measure(*dev[:5], theta_ap=theta, centre_mask=sel, report_singular=False)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            m = e.measure(*dev[:5], theta_ap=theta, centre_mask=sel, report_singular=False)
            a1.record(stream)
            torch.cuda.synchronize()
            res[prec] = (a0.elapsed_time(a1) / 1e3, e.counts(), m.m8.cpu().numpy())
    s64, (nc, p64), m64 = res["fp64"]
    sp, _, mp = res[precision]
    share = p64 / pairs_full
    return {"sample": "exact random centre subset: %d centres (%.2f %% of the pairs), whole path with "
                      "those centres; catalogs/s extrapolated to the whole catalog by pairs" % (nc, 100 * share),
            "catalogs_per_s": share / s64, "pairs_per_s": p64 / s64, "seconds_subset": s64,
            "precision_over_fp64_same_subset": s64 / sp,
            "map3_rel_err_vs_fp64": float(np.abs(mp[..., 0] - m64[..., 0]).max() / np.abs(m64[..., 0]).max()),
            "m8_rel_err_vs_fp64": float(np.abs(mp - m64).max() / np.abs(m64).max())}


def oracle_parity(api, dev, cat, setup, theta, precision, stream, n_centres, seed=12):
    """The precision form against the FP64 oracle on a random sample of centres (all galaxies as
    neighbours): normwise relative errors of Upsilon and N. The edge correction and what follows
    are compared on the FP64 GPU path's subset instead (measure_fp64_subset): with a few dozen
    centres most small-scale mode-coupling systems hold a handful of triplets, and their solution
    amplifies any rounding without bound."""
    import torch
    import oracle
    rng = np.random.default_rng(seed)
    cen = np.sort(rng.choice(cat.n, n_centres, replace=False))
    t0 = time.perf_counter()
    r = oracle.pipeline(oracle.Setup(**setup), cat, theta, cen)
    t_orc = time.perf_counter() - t0
    mask = np.zeros(cat.n, np.uint8)
    mask[cen] = 1
    with api.Estimator(**setup, precision=precision, stream=stream) as e:
        m = e.measure(*dev[:5], theta_ap=theta, centre_mask=torch.as_tensor(mask, device="cuda"),
                      report_singular=False)
        torch.cuda.synchronize()
        g = {"ups": m.upsilon.cpu().numpy(), "norm": m.norm.cpu().numpy()}

    def rel(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())

    return {"centres": int(n_centres), "oracle_seconds": t_orc, "upsilon_rel_err": rel(g["ups"], r.ups),
            "norm_rel_err": rel(g["norm"], r.norm)}


def measure_workload(api, name, precision, stream, steps, warmup, seed_offset=0):
    """A few timed steps of the whole path on another workload (same method as the headline)."""
    import torch
    from paper_2309_08601_gb300 import synth
    p, setup, theta = workload_setup(name)
    cat = synth.make_catalog(p["n"], p["side"], p["seed"] + seed_offset, field=p["field"], weights=p["weights"],
                             holes=p.get("holes", False))
    dev = api.catalog_to_device(cat)
    with api.Estimator(**setup, precision=precision, stream=stream) as est:
        def step():
            return est.measure(*dev[:5], theta_ap=theta, report_singular=False)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        n_centres, pairs = est.counts()
        est.set_timing(True)
        est.stage_times(reset=True)
        ms, _ = time_steps(step, steps, stream)
        stages = est.stage_times(reset=True)
        est.set_timing(False)
    k1 = stages["moments"][0] / steps
    k2 = stages["contract"][0] / steps
    return {"workload": name, "n_galaxies": p["n"], "ms_per_step": ms / steps, "catalogs_per_s": 1e3 * steps / ms,
            "pairs_per_catalog": pairs, "pairs_per_s": pairs * steps / (ms / 1e3),
            "stage_ms_per_step": {k: v[0] / steps for k, v in stages.items()},
            "roofline": moment_roofline(name, p["n_max"], pairs, k1, precision, None),
            "roofline_contract": contract_roofline(name, n_centres, p["n_bins"], p["n_max"], 1, k2, precision)}


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
    peaks = measure_peaks(native) if (rank == 0 and args.peaks) else None

    p, setup, theta = workload_setup(args.workload, args.n)
    cat = synth.make_catalog(p["n"], p["side"], rank_seed(p["seed"], rank), field=p["field"],
                             weights=p["weights"], holes=p.get("holes", False))
    dev = api.catalog_to_device(cat)
    stream = torch.cuda.current_stream()
    est = api.Estimator(**setup, precision=args.precision, stream=stream)

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
    ms, m = time_steps(step, args.steps, stream)
    if dist is not None:
        dist.barrier()
    clocks.stop()
    stages = est.stage_times(reset=True)
    est.set_timing(False)
    ms_max = reduce_over_ranks([ms], "max", dist)[0]
    pairs_all = reduce_over_ranks([pairs], "sum", dist)[0]  # each rank has its own catalog
    sec = ms_max / 1e3
    value = whole_job(pairs_all, args.steps, sec)
    cat_per_s = whole_job(world, args.steps, sec)
    k1_ms = stages["moments"][0] / args.steps
    k2_ms = stages["contract"][0] / args.steps
    roofline = moment_roofline(args.workload if not args.n else "", p["n_max"], pairs, k1_ms, args.precision, peaks)
    roofline_contract = contract_roofline(args.workload if not args.n else "", n_centres, p["n_bins"], p["n_max"],
                                          1, k2_ms, args.precision)
    launches = sum(v[1] for v in stages.values())

    # ---- end to end through the public API with host buffers (pinned), copies inside the region
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
            (cat.xq, cat.yq, cat.g1, cat.g2, cat.w)]
    h2d = sum(h.numel() * h.element_size() for h in host)
    out_host = torch.empty((1, len(theta), 8), dtype=torch.float64).pin_memory()
    d2h = out_host.numel() * out_host.element_size()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        for d, h in zip(dev[:5], host):
            d.copy_(h, non_blocking=True)
        m = step()
        out_host.copy_(m.m8, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_over_ranks([e2e_s], "max", dist)[0]
    e2e = {"value": whole_job(pairs_all, e2e_steps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded lognormal Kaiser-Squires shear + shape noise)",
            "config": workload_config(args.workload, p, args.precision),
            "catalogs_per_s": cat_per_s, "pairs_per_catalog": pairs,
            "pairs_per_s_moments_kernel": pairs / (k1_ms / 1e3),
            "moment_terms_per_s": pairs * ((2 * p["n_max"] + 3) + (2 * p["n_max"] + 1)) / (k1_ms / 1e3),
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "roofline": roofline, "roofline_contract": roofline_contract, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks.summary()}
    if peaks:
        line["peaks_measured"] = peaks
    est.close()

    # ---- the plain FP64 GPU path on an exact centre subset of the same catalog (rank 0)
    if rank == 0 and args.fp64_frac > 0:
        line["fp64_path"] = measure_fp64_subset(api, dev, cat.n, setup, theta, pairs, args.precision, stream,
                                                args.fp64_frac)
        line["fp64_path"]["speedup_of_measured_path"] = (cat_per_s / world) / line["fp64_path"]["catalogs_per_s"]

    # ---- the precision form against the oracle on sampled centres (rank 0)
    if rank == 0 and args.oracle_centres > 0:
        line["oracle_parity"] = oracle_parity(api, dev, cat, setup, theta, args.precision, stream,
                                              args.oracle_centres)

    # ---- the 200k-galaxy lognormal workload, a few steps (rank 0)
    if rank == 0 and args.extra_workload and args.extra_workload != args.workload:
        line["extra_workload"] = measure_workload(api, args.extra_workload, args.precision, stream, 3, 1)

    # ---- the differentiation form on its own workload (rank 0)
    if rank == 0 and args.adjoint:
        line["adjoint"] = measure_adjoint(api, args.precision, stream)

    # ---- the batching form: whole tomographic realisations through mp3pcf_run_batch (rank 0)
    if rank == 0 and args.batch_realisations > 0:
        line["batch"] = measure_batch(api, args.batch_realisations, args.precision, stream, args.fp64_frac)

    # ---- the combined estimator against the discrete one (rank 0)
    if rank == 0 and args.combined:
        line["combined"] = measure_combined(api, args.precision, stream, args.combined_workload)
    if rank == 0 and args.combined_full_area:
        line["combined_full_area"] = measure_combined(api, args.precision, stream, "multiscale_3m")
        line["combined_full_area_smooth"] = measure_combined(api, args.precision, stream, "multiscale_3m_smooth")

    if rank == 0 and args.cpu_baseline:
        import oracle
        pr, sec_o, k, threads = oracle_sample(cat, setup, theta, target_s=args.cpu_s)
        line["cpu_baseline"] = {"value": pr / sec_o, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d random centres (all %d galaxies as neighbours), whole "
                                          "path, %.1f s" % (k, cat.n, sec_o),
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
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=0,
                    help="rescale the workload to n galaxies at the same density (profiling runs)")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp32", "fp64"],
                    help="bf16x3 (default): FP32 moments, BF16 hi+lo tensor-core contraction, FP64 "
                         "edge correction and sums")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end (host buffer) timing")
    ap.add_argument("--fp64-frac", type=float, default=0.005,
                    help="fraction of centres for the FP64 GPU path subset (0: skip)")
    ap.add_argument("--oracle-centres", type=int, default=48,
                    help="centres of the precision form checked against the oracle (0: skip)")
    ap.add_argument("--extra-workload", default="lognormal_200k",
                    help="a second workload timed for a few steps ('' to skip)")
    ap.add_argument("--no-peaks", dest="peaks", action="store_false", help="skip the FP32/FP64 pipe probes")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-s", type=float, default=12.0, help="seconds of oracle work sampled")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the forward + backward timing of the differentiable Map^3")
    ap.add_argument("--batch-realisations", type=int, default=8,
                    help="tomographic realisations timed through mp3pcf_run_batch (0: skip)")
    ap.add_argument("--no-combined", dest="combined", action="store_false",
                    help="skip the combined-versus-discrete estimator timing")
    ap.add_argument("--combined-full-area", action="store_true",
                    help="also the combined-versus-discrete comparison at the paper's full area (3.1e6 galaxies)")
    ap.add_argument("--combined-workload", default="multiscale_310k",
                    help="workload of the default combined-estimator leg")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--oracle-plan", action="store_true",
                    help="with --impl reference: the oracle's timing plan over every workload")
    args = ap.parse_args(argv)
    if args.impl == "reference" and args.oracle_plan:
        return run_oracle_plan(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
