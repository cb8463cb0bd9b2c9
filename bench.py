#!/usr/bin/env python
"""Benchmark of the batched MBHB log-likelihood on GB300 (arXiv:2602.12011 likelihood hot path).

Workload (default): one LISA-like detector, modes (2,2) (2,1) (3,3) (3,2) (4,4), TDI 2.0 A/E/T,
T_obs = 2^22 s (209,296 bins), data = injection + seeded Gaussian noise, a batch of 1024 prior
samples per GPU. A step is one pe_loglike_batch call over the batch (all rows of the path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank evaluates its own batch (independent
samples, no data-path collective: weak scaling); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_12011_gb300 import workloads as W  # noqa: E402

METRIC = "log-likelihood evals/s (HM, 3 TDI ch, batched) vs plain path; grad evals/s"
UNIT = "evals/s"
MSUN_S = 4.925490947641267e-6
# Work per active (sample, mode, bin) unit of the fused forward kernel, from the ncu SASS counters
# of one launch on the 64-sample case of this workload:
#   fp64_flops  DFMA x 2 + DMUL + DADD
#   fp64_inst   every FP64-pipe instruction (DFMA, DMUL, DADD, DSETP, F2F, FRND)
#   fp32_inst   FFMA + FMUL + FADD (the double-word arithmetic of the mixed path)
UNIT_COUNTS = {
    "fp64": {"fp64_flops": 386.2, "fp64_inst": 243.4, "fp32_inst": 0.2},
    # mixed: the MINB 4 (128-register) variant, the autotuner's usual pick for the mixed path
    "mixed": {"fp64_flops": 41.2, "fp64_inst": 31.1, "fp32_inst": 2054.6},
    # FP32 path: fp64_inst counts the FRND and F2F of CUDA's FP32 sincospif/sinf and conversions
    "fp32": {"fp64_flops": 0.3, "fp64_inst": 8.9, "fp32_inst": 354.4},
}
# SHA-256 (first 16 hex digits) of the per-bin unit's sources the counts were taken on; the bench
# marks the counts stale (and warns) when the sources have changed since.
UNIT_SOURCES = {
    "fp64": ("pe_device.cuh", "pe_kernels.cu", "pe_internal.h"),
    "mixed": ("pe_device.cuh", "pe_device_mixed.cuh", "pe_df.cuh", "pe_kernels.cu", "pe_internal.h"),
    "fp32": ("pe_device.cuh", "pe_device_f32.cuh", "pe_kernels.cu", "pe_internal.h"),
}
UNIT_COUNTS_SOURCE_SHA = {"fp64": "292696e716174956", "mixed": "7c7bef97e00bebcd", "fp32": "5ceb52c2077064e4"}
# DRAM bytes (read + write) of one full-size launch (B = 1024), ncu dram__bytes_{read,write}.sum:
# the per-bin tables, read once per launch
TRAFFIC = {"fp64": 36.62e6 + 0.01e6, "mixed": 40.42e6 + 1.06e6, "fp32": None}
# Algorithmic work of the method (oracle/flop_model.py: the oracle's own operations, counted on
# 16 samples of this workload): add/sub/mul/div per active (sample, mode, bin) unit and per active
# (sample, bin) for the A/E/T and likelihood terms, and math-library calls per unit.
ALG_MODEL = {"flops_per_unit": 1755.0, "flops_per_bin": 63.0, "math_calls_per_unit": 81.0,
             "source": "oracle/flop_model.py (plain per-bin formulation, counted with an operation-counting scalar)"}


def unit_sources_sha(prec: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in UNIT_SOURCES[prec]:
        with open(os.path.join(ROOT, "paper_2602_12011_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-network", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="headline forward path: all FP64, or FP64 phase/t_f/sums with double-word geometry")
    ap.add_argument("--no-precision-study", action="store_true")
    ap.add_argument("--no-hetero", action="store_true")
    return ap.parse_args()


def active_units(theta: np.ndarray, T: float, k0: int, nb: int, mode_mask: int) -> int:
    """Active (sample, mode, bin) units: bins of each mode below its taper end m F_isco
    (odd-m modes vanish for q = 1). Work accounting only."""
    tot = 0
    f_lo = k0 / T
    f_hi = (k0 + nb - 1) / T
    for th in theta:
        M = th[0] * MSUN_S
        fisco = 6 ** -1.5 / (2 * math.pi * M)
        for bit, (l, m) in enumerate(W.MODES):
            if not (mode_mask >> bit) & 1:
                continue
            if m % 2 == 1 and th[1] == 1.0:
                continue
            fe = min(m * fisco, f_hi + 1.0 / T)
            if fe <= f_lo:
                continue
            tot += min(nb, int(math.ceil(fe * T - 1e-9)) - k0)
    return tot


def active_bins(theta: np.ndarray, T: float, k0: int, nb: int, mode_mask: int) -> int:
    """Active (sample, bin) pairs: bins below the largest active mode's taper end."""
    tot = 0
    f_hi = (k0 + nb - 1) / T
    for th in theta:
        M = th[0] * MSUN_S
        fisco = 6 ** -1.5 / (2 * math.pi * M)
        fe = 0.0
        for bit, (l, m) in enumerate(W.MODES):
            if (mode_mask >> bit) & 1 and not (m % 2 == 1 and th[1] == 1.0):
                fe = max(fe, m * fisco)
        fe = min(fe, f_hi + 1.0 / T)
        tot += max(0, min(nb, int(math.ceil(fe * T - 1e-9)) - k0))
    return tot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self, gpu_index: int):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != gpu_index:
                    continue
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_dets(O, dets_spec, inj, inj_mask, noise_seed):
    ods = []
    for det, T, k0, nb in dets_spec:
        data = O.make_data(det, inj, inj_mask, T, k0, nb, W.normals(nb, noise_seed))
        psd = O.psd(det, (k0 + np.arange(nb)) / T)
        ods.append(O.Detector(det, T, k0, nb, data, psd))
    return ods


def _timed_oracle(O, ods, theta, mask, nthreads):
    t0 = time.perf_counter()
    O.loglike_batch(ods, theta, mask, nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_baseline(dets_spec, theta, mode_mask, n_samples, noise_seed, inj, inj_mask):
    """The oracle, as it stands, on the host cores: bounded samples of the benchmark workload (all
    cores, and one core as in the paper's CPU comparison), of the single-source plain workload
    (whole) and of the three-detector network (one core and all cores)."""
    from oracle import oracle as O
    O.build()
    ods = _oracle_dets(O, dets_spec, inj, inj_mask, noise_seed)
    th = theta[:n_samples]
    cores = O.max_threads()
    dt = _timed_oracle(O, ods, th, mode_mask, cores)
    n1 = 16
    dt1 = _timed_oracle(O, ods, theta[:n1], mode_mask, 1)
    ws = W.single_22()
    o1 = _oracle_dets(O, ws["dets"], ws["inj"], ws["inj_mask"], ws["noise_seed"])
    ds1 = _timed_oracle(O, o1, ws["theta"], ws["mode_mask"], 1)
    wn = W.network_hm(4096)
    on = _oracle_dets(O, wn["dets"], wn["inj"], wn["inj_mask"], wn["noise_seed"])
    dn1 = _timed_oracle(O, on, wn["theta"][:16], wn["mode_mask"], 1)
    dn = _timed_oracle(O, on, wn["theta"][:64], wn["mode_mask"], cores)
    return {"value": th.shape[0] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d of the %d-sample batch, all modes, full grid, OpenMP over samples (%.1f s wall)"
                      % (th.shape[0], theta.shape[0], dt),
            "single_core": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": "first %d samples of the same batch, one thread (%.1f s)" % (n1, dt1)},
            "single_source": {"value": 1.0 / ds1, "unit": UNIT, "cores": 1, "workload": ws["name"],
                              "sample": "the whole workload: one sample, (2,2), 52,324 bins (%.2f s)" % ds1},
            "network": {"value": 64 / dn, "unit": UNIT, "cores": cores, "workload": wn["name"],
                        "sample": "first 64 of the 4096 samples, OpenMP over samples (%.1f s)" % dn,
                        "single_core": {"value": 16 / dn1, "unit": UNIT, "cores": 1,
                                        "sample": "first 16 samples, one thread (%.1f s)" % dn1}}}


def run_reference(args, wl):
    """--impl reference: the FP64 CPU oracle on the host cores, each step a bounded sample."""
    from oracle import oracle as O
    O.build()
    dets_spec = wl["dets"]
    ods = []
    for det, T, k0, nb in dets_spec:
        data = O.make_data(det, wl["inj"], wl["inj_mask"], T, k0, nb, W.normals(nb, wl["noise_seed"]))
        psd = O.psd(det, (k0 + np.arange(nb)) / T)
        ods.append(O.Detector(det, T, k0, nb, data, psd))
    n = 32
    th = wl["theta"][:n]
    cores = O.max_threads()
    for _ in range(args.warmup):
        O.loglike_batch(ods, th[:4], wl["mode_mask"], nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.loglike_batch(ods, th, wl["mode_mask"], nthreads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["name"], "detectors": "+".join(d[0]["name"] for d in dets_spec),
                       "modes": "22,21,33,32,44", "batch_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first %d samples of the %d-sample batch per step" % (n, wl["theta"].shape[0])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Issue rate of each pipe per SM and clock: FP64 2 DFMA (the nominal 1.25 TFLOP/s FP64 of a
# 152-SM part at 2070 MHz), FP32 128 FFMA. Nominal peak = rate x SMs x maximum SM clock.
PIPE_PER_CLK = {"fp64": 2.0, "fp32": 128.0}


def roofline(prec: str, units: int, launch_s: float, peaks: dict, n_sm: int = 152, sm_max_mhz: float = 2070.0,
             sm_mhz_run: float = None, bins: int = 0) -> dict:
    """ALU roofline of the fused forward kernel: per pipe, the instructions one launch issues
    (per-unit count x active units) per second against the pipe's measured FMA-loop rate, against
    the nominal rate at the maximum clock, and against the nominal rate at the median SM clock
    sampled while the kernel ran; the binding pipe is the busier one. Beside it, the algorithmic
    view: the oracle-counted work of the method (ALG_MODEL) per second against the FP64 peak."""
    if prec not in UNIT_COUNTS:
        return None
    c = UNIT_COUNTS[prec]
    ups = units / launch_s
    pipes = {}
    for name, inst in (("fp64", c["fp64_inst"]), ("fp32", c["fp32_inst"])):
        loop = peaks[name]
        peak = loop["tflops"] * 1e3 / 2.0   # G FMA instructions/s of the measured loop
        nominal = PIPE_PER_CLK[name] * n_sm * sm_max_mhz / 1e3
        ach = inst * ups / 1e9
        pipes[name] = {"inst_per_unit": inst, "achieved_ginst_s": ach, "peak_ginst_s": peak, "frac": ach / peak,
                       "peak_loop_sm_mhz": loop.get("sm_mhz"),
                       "peak_loop_at_its_clock_frac_nominal": (peak / (PIPE_PER_CLK[name] * n_sm * loop["sm_mhz"] / 1e3)
                                                               if loop.get("sm_mhz") else None),
                       "peak_nominal_ginst_s": nominal, "frac_nominal": ach / nominal}
        if sm_mhz_run:
            pipes[name]["frac_nominal_at_run_clock"] = ach / (PIPE_PER_CLK[name] * n_sm * sm_mhz_run / 1e3)
    bind = max(pipes, key=lambda k: pipes[k]["frac"])
    sha = unit_sources_sha(prec)
    alg_tflops = (ALG_MODEL["flops_per_unit"] * units + ALG_MODEL["flops_per_bin"] * bins) / launch_s / 1e12
    fp64_nominal_tflops = 2 * PIPE_PER_CLK["fp64"] * n_sm * sm_max_mhz / 1e6
    return {"bound": "alu", "pipe": bind, "unit": "Ginst/s", "achieved": pipes[bind]["achieved_ginst_s"],
            "peak": pipes[bind]["peak_ginst_s"], "frac": pipes[bind]["frac"],
            "peak_kind": "measured FMA loops (FP64 and FP32, 1 s each; clocks sampled during them)",
            "peak_nominal": pipes[bind]["peak_nominal_ginst_s"], "frac_nominal": pipes[bind]["frac_nominal"],
            "peak_nominal_kind": "%g inst/clk/SM x %d SMs x %g MHz" % (PIPE_PER_CLK[bind], n_sm, sm_max_mhz),
            "frac_nominal_at_run_clock": pipes[bind].get("frac_nominal_at_run_clock"), "run_sm_mhz": sm_mhz_run,
            "kernel": "k_loglike_fwd",
            "launch_ms": launch_s * 1e3, "units_per_launch": units, "bins_per_launch": bins, "units_per_s": ups,
            "fp64_tflops": c["fp64_flops"] * ups / 1e12, "fp64_tflops_peak": peaks["fp64"]["tflops"],
            "fp64_flops_frac": c["fp64_flops"] * ups / 1e12 / peaks["fp64"]["tflops"],
            "alg_flops_per_unit": ALG_MODEL["flops_per_unit"], "alg_flops_per_bin": ALG_MODEL["flops_per_bin"],
            "alg_tflops": alg_tflops, "alg_frac_nominal": alg_tflops / fp64_nominal_tflops,
            "alg_note": ("the oracle's plain formulation counted per active unit (%s); a fraction above 1 is work "
                         "the kernel's factored algebra and tables avoid" % ALG_MODEL["source"]),
            "unit_counts_source_sha": UNIT_COUNTS_SOURCE_SHA[prec], "unit_sources_sha": sha,
            "unit_counts_current": UNIT_COUNTS_SOURCE_SHA[prec] == sha,
            "pipes": pipes,
            "traffic": TRAFFIC[prec] if UNIT_COUNTS_SOURCE_SHA[prec] == sha else None,
            "traffic_gbs": (TRAFFIC[prec] / launch_s / 1e9
                            if TRAFFIC[prec] and UNIT_COUNTS_SOURCE_SHA[prec] == sha else None)}


def measure_peaks(L, local_rank: int) -> dict:
    """The FP64 and FP32 FMA-loop rates (1 s each) with the SM clock sampled during each."""
    out = {}
    for name, fn in (("fp64", L.pe_measure_fp64_peak), ("fp32", L.pe_measure_fp32_peak)):
        cs = ClockSampler()
        time.sleep(0.2)
        tf = fn(1.0)
        clk = cs.stop(local_rank)
        out[name] = {"tflops": tf, "sm_mhz": clk.get("sm_mhz"), "clock_reasons": clk.get("reasons")}
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = W.batch_hm(args.batch)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, wl)
        return

    import torch
    import torch.distributed as dist
    from paper_2602_12011_gb300 import build as Bld
    from paper_2602_12011_gb300 import _lib as L
    from paper_2602_12011_gb300 import shard

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    Bld.build()
    L.lib()

    det, T, k0, nb = wl["dets"][0]
    mask64 = wl["mode_mask"]                       # FP64 likelihood, gradient and Fisher
    mask = mask64 | (L.PE_PREC_MIXED if args.precision == "mixed" else 0)
    B = args.batch
    theta = wl["theta"] if rank == 0 else W.draw_prior(B, W.SEED_BATCH_HM + 1000 * rank, T)
    gd = L.Detector(det, T, k0, nb)
    gd.inject(wl["inj"], wl["inj_mask"], W.normals(nb, wl["noise_seed"]))
    hs = [gd.handle]

    stream = torch.cuda.current_stream()
    th_dev = torch.tensor(theta, device="cuda")
    out_dev = torch.empty(B, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # 256 MiB > 129 MB L2

    def step():
        L.pe_loglike_batch(hs, th_dev, B, mask, out_dev, None, None, stream)

    # project autotuner (set-up, untimed): register-budget variant and persistent grid size of the
    # fused kernel for this workload; pe_loglike_batch then uses the cached choice
    tuned = L.pe_autotune(hs, th_dev, B, mask)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K batched steps, L2 flushed before each, device-timed on the stream
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler()
    time.sleep(0.3)
    L.pe_profile_read()
    L.pe_profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    L.pe_profile_enable(False)
    fwd_ms, fwd_launches = L.pe_profile_read()
    clk = clocks.stop(local_rank)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = shard.max_over_ranks(sum(step_ms) / 1e3, device="cuda")
    value = world * B * K / t_total
    result_ok = bool(torch.isfinite(out_dev).all().item())

    units = active_units(theta, T, k0, nb, mask)
    bins = active_bins(theta, T, k0, nb, mask)
    fwd_avg_s = (fwd_ms / max(fwd_launches, 1)) / 1e3
    peaks = measure_peaks(L, local_rank)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_max = clk.get("sm_max_mhz") or 2070.0
    roof = roofline(args.precision, units, fwd_avg_s, peaks, n_sm, sm_max, clk.get("sm_mhz"), bins)
    if roof and not roof["unit_counts_current"]:
        sys.stderr.write("bench: the per-unit instruction counts were taken on other unit sources (%s, now %s); "
                         "re-take them with ncu\n" % (roof["unit_counts_source_sha"], roof["unit_sources_sha"]))
    # every rank's per-sample results in one place (what a sampler's driver needs), outside the
    # timed region
    gathered = shard.gather_results(out_dev, world * B, world) if world > 1 else out_dev
    result_ok = result_ok and bool(torch.isfinite(gathered).all().item())

    # ---- precision study (the paper's low-precision option against FP64): the same batch through
    # the other forward path, device-timed the same way; accuracy of its log L against the FP64
    # result on the likelihood's scale 1/2 <d|d> + |<d|h>| + 1/2 <h|h>
    study = None
    if not args.no_precision_study:
        dh64 = torch.empty((B, 1, 3, 2), dtype=torch.float64, device="cuda")
        ll64 = torch.empty(B, dtype=torch.float64, device="cuda")
        L.pe_loglike_batch(hs, th_dev, B, mask64, ll64, dh64, None, stream)
        torch.cuda.synchronize()
        dd = float(gd.data_norm().sum())
        scale = 0.5 * dd + dh64[:, :, :, 0].sum(dim=(1, 2)).abs() + 0.5 * dh64[:, :, :, 1].sum(dim=(1, 2))
        study = {args.precision: {"value": value, "ms_per_step": 1e3 * t_total / K,
                                  "roofline_frac": roof["frac"] if roof else None}}
        for other in ("fp64", "mixed", "fp32"):
            if other == args.precision:
                continue
            m = mask64 | {"fp64": 0, "mixed": L.PE_PREC_MIXED, "fp32": L.PE_PREC_FP32}[other]
            tuned_o = L.pe_autotune(hs, th_dev, B, m)
            llo = torch.empty(B, dtype=torch.float64, device="cuda")
            for _ in range(3):
                L.pe_loglike_batch(hs, th_dev, B, m, llo, None, None, stream)
            torch.cuda.synchronize()
            L.pe_profile_read()
            L.pe_profile_enable(True)
            for k in range(K):
                flush.zero_()
                ev[k][0].record(stream)
                L.pe_loglike_batch(hs, th_dev, B, m, llo, None, None, stream)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            L.pe_profile_enable(False)
            o_ms, o_n = L.pe_profile_read()
            ems = [a.elapsed_time(b) for a, b in ev]
            rel = ((llo - ll64).abs() / scale).max().item()
            absmax = (llo - ll64).abs().max().item()
            study[other] = {"value": B * K / (sum(ems) / 1e3), "ms_per_step": sum(ems) / K, "tuning": tuned_o,
                            "max_rel_dlogl_vs_fp64": rel, "max_abs_dlogl_vs_fp64": absmax, "parity_bar": 1e-10,
                            "roofline": roofline(other, units, (o_ms / max(o_n, 1)) / 1e3, peaks, n_sm, sm_max,
                                                 clk.get("sm_mhz"), bins)}
        study["note"] = ("mixed: FP64 TaylorF2 phase, t_f, turn reductions and tile sums; response "
                         "geometry, TDI, A/E/T and per-bin products in double-word FP32 arithmetic. "
                         "fp32: every step in FP32 (the paper's float32 option); misses the 1e-10 bar")

    # ---- plain path: one call per sample (B = 1), same samples, device-timed
    n_plain = 64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out1 = torch.empty(1, dtype=torch.float64, device="cuda")
    for i in range(4):
        L.pe_loglike_batch(hs, th_dev[i:i + 1], 1, mask, out1, None, None, stream)
    flush.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(n_plain):
        L.pe_loglike_batch(hs, th_dev[i:i + 1], 1, mask, out1, None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_value = n_plain / (e0.elapsed_time(e1) / 1e3)
    # the same samples batched, for the like-for-like ratio
    e0.record(stream)
    L.pe_loglike_batch(hs, th_dev[:n_plain], n_plain, mask, out_dev[:n_plain], None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    batched_same = n_plain / (e0.elapsed_time(e1) / 1e3)

    # the plain path again through a B = 1 CUDA-graph plan (no per-call host work)
    plan1 = L.Plan([gd], 1, mask, theta=th_dev[:1].clone(), autotune=False)
    for i in range(4):
        plan1.launch(stream)
    flush.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(n_plain):
        plan1.theta.copy_(th_dev[i:i + 1])
        plan1.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_graph_value = n_plain / (e0.elapsed_time(e1) / 1e3)
    plan1.close()

    # ---- the single-source plain workload (LISA, (2,2), T = 2^20 s, 52,324 bins, one parameter
    # point): one call per evaluation, device-timed over 200 calls
    ws = W.single_22()
    det1, T1, k01, nb1 = ws["dets"][0]
    g1 = L.Detector(det1, T1, k01, nb1)
    g1.inject(ws["inj"], ws["inj_mask"], W.normals(nb1, ws["noise_seed"]))
    th1 = torch.tensor(ws["theta"], device="cuda")
    for _ in range(5):
        L.pe_loglike_batch([g1.handle], th1, 1, ws["mode_mask"], out1, None, None, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(200):
        L.pe_loglike_batch([g1.handle], th1, 1, ws["mode_mask"], out1, None, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    single = {"value": 200 / (e0.elapsed_time(e1) / 1e3), "unit": UNIT, "workload": ws["name"],
              "calls": 200, "note": "one pe_loglike_batch call (B = 1) per evaluation, device-timed"}
    g1.close()

    # ---- gradient evals/s: hand-written adjoint over the same batch, device-timed
    grad_dev = torch.empty((B, 11), dtype=torch.float64, device="cuda")
    ll_dev = torch.empty(B, dtype=torch.float64, device="cuda")
    L.pe_loglike_grad_batch(hs, th_dev, B, mask64, ll_dev, grad_dev, None, stream)
    Kg = max(2, K // 2)
    gms = []
    for k in range(Kg):
        flush.zero_()
        e0.record(stream)
        L.pe_loglike_grad_batch(hs, th_dev, B, mask64, ll_dev, grad_dev, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        gms.append(e0.elapsed_time(e1))
    grad_value = world * B * Kg / (sum(gms) / 1e3)
    grad_ok = bool(torch.isfinite(grad_dev).all().item())
    # the same gradient in mixed precision (PE_PREC_MIXED): the forward mode sum and the reverse
    # sweeps with double-word geometry. Its deviation from the FP64 gradient: per component, the
    # largest |g_mixed - g_fp64| over the batch divided by the largest |g_fp64|
    grad_mx = torch.empty_like(grad_dev)
    ll_mx = torch.empty_like(ll_dev)
    L.pe_loglike_grad_batch(hs, th_dev, B, mask64 | L.PE_PREC_MIXED, ll_mx, grad_mx, None, stream)
    gms_mx = []
    for k in range(Kg):
        flush.zero_()
        e0.record(stream)
        L.pe_loglike_grad_batch(hs, th_dev, B, mask64 | L.PE_PREC_MIXED, ll_mx, grad_mx, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        gms_mx.append(e0.elapsed_time(e1))
    grad_mixed = {"value": world * B * Kg / (sum(gms_mx) / 1e3), "unit": "grad evals/s",
                  "ms_per_step": sum(gms_mx) / Kg, "steps": Kg,
                  "max_rel_dgrad_vs_fp64": float(((grad_mx - grad_dev).abs().amax(dim=0)
                                                  / grad_dev.abs().amax(dim=0).clamp_min(1e-300)).max().item()),
                  "note": ("FP64 TaylorF2 phase, t_f, turn reductions, PN chain rule and sums; "
                           "double-word geometry, link factors and their cotangents")}

    # ---- Fisher matrix at the injected source (5 modes, all 11 parameters), device-timed
    thf = torch.tensor(wl["inj"][None, :], device="cuda")
    Fd = torch.empty((1, 11, 11), dtype=torch.float64, device="cuda")
    L.pe_fisher(hs, thf, 1, mask64, Fd, stream)
    e0.record(stream)
    L.pe_fisher(hs, thf, 1, mask64, Fd, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    fisher = {"ms": e0.elapsed_time(e1), "theta": "injection", "finite": bool(torch.isfinite(Fd).all().item())}

    # ---- detector network (LISA 2^22 s + Taiji 2^21 s + TianQin 2^20 s), B = 4096, one CUDA-graph
    # plan with autotuned launch parameters
    net = None
    if not args.no_network:
        wn = W.network_hm(4096)
        nds = []
        for det_n, T_n, k0_n, nb_n in wn["dets"]:
            dn = L.Detector(det_n, T_n, k0_n, nb_n)
            dn.inject(wn["inj"], wn["inj_mask"], W.normals(nb_n, wn["noise_seed"]))
            nds.append(dn)
        thn = torch.tensor(wn["theta"] if rank == 0 else W.draw_prior(4096, W.SEED_BATCH_NET + 1000 * rank, 2.0 ** 20),
                           device="cuda")
        pn = L.Plan(nds, 4096, wn["mode_mask"] | (mask & L.PE_PREC_MIXED), theta=thn, autotune=True)
        for _ in range(3):
            pn.launch(stream)
        nms = []
        for k in range(max(2, K // 2)):
            flush.zero_()
            e0.record(stream)
            pn.launch(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            nms.append(e0.elapsed_time(e1))
        net = {"value": world * 4096 * len(nms) / (sum(nms) / 1e3), "unit": UNIT, "ms_per_step": sum(nms) / len(nms),
               "workload": wn["name"], "detectors": "LISA(2^22 s)+Taiji(2^21 s)+TianQin(2^20 s)",
               "launch": "one CUDA graph per step", "tuned": pn.info(),
               "finite": bool(torch.isfinite(pn.logl).all().item())}
        pn.close()
        for dn in nds:
            dn.close()

    # ---- learned surrogate: trained on the GPU (set-up, untimed) on 2^20 prior samples, then the
    # surrogate path against the plain path on one 16384-sample inference batch
    sur = None
    if not args.no_surrogate:
        srg = L.Surrogate(seed=2605)
        t_tr = time.perf_counter()
        sl, _ = srg.train(torch.tensor(W.draw_prior(1 << 20, 2605, T), device="cuda"), 60, batch=1024, lr=2e-3)
        torch.cuda.synchronize()
        t_tr = time.perf_counter() - t_tr
        Bs = 16384
        ths = W.draw_prior(Bs, 2609 + rank, T)
        tts = torch.tensor(ths, device="cuda")
        outs = torch.empty(Bs, dtype=torch.float64, device="cuda")
        srg.loglike([gd], tts, mask64)
        L.pe_loglike_batch(hs, tts, Bs, mask, outs, None, None, stream)
        torch.cuda.synchronize()
        flush.zero_()
        e0.record(stream)
        _, used = srg.loglike([gd], tts, mask64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1)
        flush.zero_()
        e0.record(stream)
        L.pe_loglike_batch(hs, tts, Bs, mask, outs, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        tho = W.draw_prior(2048, 2606, T)
        mm = srg.mismatch(gd, torch.tensor(tho, device="cuda"), mask64).cpu().numpy()
        inbox = (tho[:, 0] >= 1e5) & (tho[:, 1] <= 10.0)   # the default box of the spline path

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        # the same node-spline path without the network (the plain generator's exact node values),
        # and the plain mixed-precision path, on the same batch
        srg.set_node_source(1)
        ms_n = timed(lambda: srg.loglike([gd], tts, mask64))
        mm_n = srg.mismatch(gd, torch.tensor(tho, device="cuda"), mask64).cpu().numpy()
        ms_nx = timed(lambda: srg.loglike([gd], tts, mask64 | L.PE_PREC_MIXED))
        srg.set_node_source(0)
        ms_mx = timed(lambda: L.pe_loglike_batch(hs, tts, Bs, mask64 | L.PE_PREC_MIXED, outs, None, None, stream))
        # the surrogate path in mixed precision (out-of-box samples on the mixed plain unit, in-box
        # ones with the spline phase's sincos and the transfer functions on the FP32 pipe), and its
        # deviation from the FP64 surrogate path on the likelihood's scale
        ms_sx = timed(lambda: srg.loglike([gd], tts, mask64 | L.PE_PREC_MIXED))
        ll_s64, _ = srg.loglike([gd], tts, mask64)
        ll_smx, _ = srg.loglike([gd], tts, mask64 | L.PE_PREC_MIXED)
        dhs = torch.empty((Bs, 1, 3, 2), dtype=torch.float64, device="cuda")
        L.pe_loglike_batch(hs, tts, Bs, mask64, outs, dhs, None, stream)
        torch.cuda.synchronize()
        scale_s = (0.5 * float(gd.data_norm().sum()) + dhs[:, :, :, 0].sum(dim=(1, 2)).abs()
                   + 0.5 * dhs[:, :, :, 1].sum(dim=(1, 2)))
        dev_sx = ((ll_smx - ll_s64).abs() / scale_s).max().item()
        sur = {"value": world * Bs / (ms_s / 1e3), "unit": UNIT, "plain_same_batch": world * Bs / (ms_p / 1e3),
               "gain": ms_p / ms_s, "batch": Bs, "used_fraction": float(used.float().mean().item()),
               "no_network_same_batch": world * Bs / (ms_n / 1e3), "network_over_no_network": ms_n / ms_s,
               "plain_mixed_same_batch": world * Bs / (ms_mx / 1e3), "network_over_plain_mixed": ms_mx / ms_s,
               "network_mixed_same_batch": world * Bs / (ms_sx / 1e3),
               "no_network_mixed_same_batch": world * Bs / (ms_nx / 1e3),
               "network_mixed_over_plain_mixed": ms_mx / ms_sx,
               "network_mixed_max_rel_dlogl_vs_network_fp64": dev_sx,
               "train_s": t_tr, "train_loss": sl, "heldout_pass_1e-3": float(np.mean(mm[inbox] <= 1e-3)),
               "heldout_max_mismatch_no_network": float(np.max(mm_n[inbox])),
               "heldout_in_box": int(inbox.sum()),
               "note": ("network: MLP node values (3PN/3.5PN phase terms, |H_lm|) + node splines; no_network: "
                        "the same splines from the plain generator's exact node values; plain: per-bin FP64; "
                        "plain_mixed: per-bin FP64 phase with double-word geometry (1e-10 parity); *_mixed: "
                        "the surrogate path with PE_PREC_MIXED (fallbacks on the mixed plain unit, in-box spline "
                        "sincos and transfer functions in FP32, double-word A/E/T and products)")}
        srg.close()

    # ---- heterodyned (relative-binning) likelihood, the second workload: 1024 draws in the posterior's
    # bulk around the injection (the all-parameter Fisher-Gaussian at 0.1 of its width), evaluated
    # through 256 coarse bins against the exact path on the same draws
    het = None
    if not args.no_hetero:
        idx = np.arange(11, dtype=np.int32)
        nrm = 0.1 * np.random.Generator(np.random.PCG64(2607 + rank)).standard_normal((1400, 11))
        _, draws = L.fisher_gaussian([gd], wl["inj"], mask64, idx, nrm)
        ok = (draws[:, 1] >= 1.0) & (np.abs(draws[:, 2]) < 1) & (np.abs(draws[:, 3]) < 1) & (draws[:, 4] > 0)
        thh = torch.tensor(draws[ok][:1024], device="cuda")
        Bh = thh.shape[0]
        t_c = time.perf_counter()
        hobj = L.Hetero(gd, wl["inj"], mask64, nbins_coarse=256)
        t_c = time.perf_counter() - t_c
        llh = torch.empty(Bh, dtype=torch.float64, device="cuda")
        lle = torch.empty(Bh, dtype=torch.float64, device="cuda")
        for _ in range(3):
            L.pe_hetero_loglike_batch([hobj.handle], thh, Bh, llh, None, None, stream)
        L.pe_loglike_batch(hs, thh, Bh, mask64, lle, None, None, stream)
        torch.cuda.synchronize()
        hms, ems = [], []
        for k in range(max(3, K // 2)):
            flush.zero_()
            e0.record(stream)
            L.pe_hetero_loglike_batch([hobj.handle], thh, Bh, llh, None, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            hms.append(e0.elapsed_time(e1))
            flush.zero_()
            e0.record(stream)
            L.pe_loglike_batch(hs, thh, Bh, mask64, lle, None, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ems.append(e0.elapsed_time(e1))
        dl = (llh - lle).abs()
        het = {"value": world * Bh / (sum(hms) / len(hms) / 1e3), "unit": UNIT, "ms_per_step": sum(hms) / len(hms),
               "exact_same_samples": world * Bh / (sum(ems) / len(ems) / 1e3), "gain": sum(ems) / sum(hms),
               "batch": Bh, "coarse_edges": int(hobj.edges.size), "create_s": t_c,
               "max_abs_dlogl_vs_exact": dl.max().item(), "median_abs_dlogl_vs_exact": dl.median().item(),
               "samples": "Fisher-Gaussian draws at 0.1 of its width around the injection (posterior bulk)",
               "dtype": "f64"}
        # the same summary data with the signal at the edges from the mixed-precision unit
        hmix = L.Hetero(gd, wl["inj"], mask64 | L.PE_PREC_MIXED, edges=hobj.edges)
        llm = torch.empty_like(llh)
        for _ in range(3):
            L.pe_hetero_loglike_batch([hmix.handle], thh, Bh, llm, None, None, stream)
        torch.cuda.synchronize()
        mms = []
        for k in range(max(3, K // 2)):
            flush.zero_()
            e0.record(stream)
            L.pe_hetero_loglike_batch([hmix.handle], thh, Bh, llm, None, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            mms.append(e0.elapsed_time(e1))
        het["mixed"] = {"value": world * Bh / (sum(mms) / len(mms) / 1e3), "unit": UNIT,
                        "ms_per_step": sum(mms) / len(mms),
                        "max_abs_dlogl_vs_fp64_heterodyned": (llm - llh).abs().max().item(),
                        "note": "signal at the edges from the mixed-precision unit; ratios and sums FP64"}
        hmix.close()
        hobj.close()

    # ---- end to end through the C ABI with host buffers (pinned): H2D of theta, D2H of logL
    th_host = torch.tensor(theta).pin_memory()
    out_host = torch.empty(B, dtype=torch.float64).pin_memory()
    e2e_t = []
    for k in range(K + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.pe_loglike_batch(hs, th_host, B, mask, out_host, None, None, stream)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_t.append(dt)
    e2e_tot = shard.max_over_ranks(sum(e2e_t), device="cuda")
    e2e_value = world * B * K / e2e_tot

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * t_total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f64+f32x2 (double-word)", "data": "synthetic",
            "config": {"workload": wl["name"], "detectors": "LISA", "modes": "22,21,33,32,44", "T_obs_s": T,
                       "nbins": nb, "batch_per_gpu": B, "parallelism": "replicas (independent samples per GPU)",
                       "l2": "flushed before every timed step (256 MiB write)"},
            "roofline": roof,
            "precision_study": study,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(B * 11 * 8),
                    "d2h_bytes_per_step": int(B * 8)},
            "plain_path": {"value": plain_value, "unit": UNIT, "samples": n_plain,
                           "graph_plan_value": plain_graph_value, "batched_same_samples": batched_same},
            "single_source": single,
            "fisher": fisher,
            "network": net,
            "surrogate": sur,
            "heterodyne": het,
            "tuning": tuned,
            "grad": {"value": grad_value, "unit": "grad evals/s", "ms_per_step": sum(gms) / Kg, "steps": Kg,
                     "finite": grad_ok, "mixed": grad_mixed},
            # per step: prep, sub-tile scan (plus the work-item scan when items hold R > 1
            # sub-tiles), forward, reduce
            "gpu_launches": (5 if int(tuned.get("subtiles", 1)) > 1 else 4) * K,
            "clocks": clk,
            "results_finite": result_ok}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl["dets"], theta, mask, 128, wl["noise_seed"], wl["inj"], wl["inj_mask"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    gd.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
