"""Throughput of the boiling time step on GB300 (MLUPS and HBM roofline).

Workload: 2048 x 2048 fluid sites over a 64-row heater, fluctuating bottom
temperature (+-1 % per column and step), FP32 shifted populations; one step =
flow kernel (collision + force + streaming), heat kernel (RK4 of the energy
equation) and diagnostics kernel.  The FP64 path is measured on the same
workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: independent replicas, one per GPU (the method has
no exchange between runs), value = all ranks' site updates / max time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "boiling step, 2048x2048 fluid + 64 heater rows, noisy bottom, FP32 shifted populations"
METRIC = "MLUPS (fluid-site updates per second), one GB300"
# algorithmic bytes per fluid site per step (9 populations read + written,
# temperature read + written) and per launch of the flow kernel (populations
# read + written, temperature read)
ALG_STEP_BYTES = {"fp32": 80, "fp64": 160, "fp16": 44}
ALG_FLOW_BYTES = {"fp32": 76, "fp64": 152, "fp16": 40}
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops x clock
FP32_LANES = 152 * 128
PROFILES = {"flow": os.path.join(ROOT, "profiles", "flow_kernel_2048x2048_fp32.md"),
            "heat": os.path.join(ROOT, "profiles", "heat_kernel_2048x2048_fp32.md"),
            "fp64": os.path.join(ROOT, "profiles", "fp64_kernels_1024x1024.md")}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("lbm_device.cuh", "lbm_dfloat.cuh", "lbm_fast.cuh", "lbm_tma.cuh", "lbm_flowwave.cuh")
FP64_SOURCES = ("lbm_device.cuh", "lbm_fp64.cu")  # the FP64 kernels and their launch shapes


def max_sm_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


def kernel_source_hash(names=KERNEL_SOURCES) -> str:
    """Hash of the kernel sources' code (comments and white space removed):
    an ncu summary taken on other code is stale, one taken before a comment
    edit is not."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1911_10747_gb300", "csrc", name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_figure(kind: str, key: str, variant: str):
    """A per-variant figure (`key[variant]: value`) from the committed ncu
    summary of the flow or heat kernel, or None when absent, taken on a
    different kernel source, or not taken on that launch-shape variant."""
    try:
        text = open(PROFILES[kind]).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(re.escape(key) + r"\[" + re.escape(variant) + r"\]:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def ncu_traffic(kind: str, variant: str):
    """DRAM bytes (read + written) per launch of the timed variant."""
    return ncu_figure(kind, "dram_bytes_per_full_launch", variant)


def ncu_instructions(kind: str, variant: str):
    """Executed instructions per site (warp instructions x 32 / sites)."""
    return ncu_figure(kind, "instructions_per_site", variant)


# the heat variant whose FP32 operations were counted when the timed one was not
HEAT_COUNTED_VARIANT = "heatpair16_64x12x4_down"


def heat_flops(variant: str):
    """FP32 flops per temperature site the heat kernel executes (ncu thread
    instruction counts: FADD + FMUL + 2 FFMA, twice that for the packed
    FADD2 / FMUL2 / FFMA2; the recomputed tile halo included) and the variant
    they were counted on: the timed variant's own count, else the paired
    64 x 12 x 4 kernel's (every variant does the same per-site arithmetic,
    with its own halo share), else (None, None)."""
    for v in (variant, HEAT_COUNTED_VARIANT):
        f = ncu_figure("heat", "flops_per_site", v)
        if f is not None:
            return f, v
    return None, None


def issue_roofline(inst_per_site, sites, ms):
    """Warp-instruction issue rate against the issue peak (152 SMs x 4
    schedulers x 1 instruction per clock at the maximum SM clock)."""
    if inst_per_site is None:
        return None
    peak = 152 * 4 * max_sm_mhz() * 1e6 / 1e12
    achieved = inst_per_site / 32.0 * sites / (ms / 1e3) / 1e12
    return {"achieved": achieved, "peak": peak, "unit": "T warp-instructions/s", "frac": achieved / peak,
            "instructions_per_site": inst_per_site}


def ncu_fp64_instructions(kind: str):
    """FP64 pipe instructions per site (DADD + DMUL + DFMA executed, from ncu)
    of the FP64 flow or heat kernel in the committed summary, or None."""
    try:
        text = open(PROFILES["fp64"]).read()
    except OSError:
        return None
    m = re.search(r"fp64_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"fp64_instructions_per_site\[" + re.escape(kind) + r"\]:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash(FP64_SOURCES):
        return None
    return float(t.group(1))


def ncu_fp64_flops(kind: str):
    """FP64 flops per site (DADD + DMUL + 2 DFMA executed, from ncu) of the
    FP64 flow or heat kernel in the committed summary, or None when absent
    or taken on a different kernel source."""
    try:
        text = open(PROFILES["fp64"]).read()
    except OSError:
        return None
    m = re.search(r"fp64_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"fp64_flops_per_site\[" + re.escape(kind) + r"\]:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash(FP64_SOURCES):
        return None
    return float(t.group(1))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(cfg, steps: int, budget_s: float = None, threads: int = 1):
    """Time the FP64 oracle as it stands on up to `steps` steps of the
    workload, stopping after the step that passes `budget_s` seconds, with
    its per-site loops on `threads` threads (results are bit-identical for
    every count); returns (MLUPS, seconds, steps timed)."""
    from oracle import oracle as O
    O.build()
    O.set_threads(threads)
    try:
        r = O.OracleRun(cfg.replace(precision="fp64"))
        done = 0
        t0 = time.perf_counter()
        while done < steps:
            r.step(1)
            done += 1
            if budget_s is not None and time.perf_counter() - t0 >= budget_s:
                break
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(1)
    return cfg.fluid_sites * done / dt / 1e6, dt, done


def aggregate_over_ranks(ms: float, sites: int, steps: int, device=None):
    """Replicas: every rank ran `steps` steps of its own run of `sites` fluid
    sites in `ms` milliseconds.  Returns (slowest rank's ms, whole-job MLUPS
    = all ranks' site updates / slowest time)."""
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, ws * sites * steps / (ms_max / 1e3) / 1e6


def workload_config(nx: int, nf: int, ns: int, ws: int, precision: str = "fp32") -> dict:
    """The `config` object of both arms' JSON lines: the workload they time."""
    return {"workload": WORKLOAD if precision == "fp32" else WORKLOAD.replace("FP32 shifted", precision.upper()),
            "nx": nx, "ny_fluid": nf, "ny_solid": ns,
            "l2": "inputs larger than L2 (populations alone 2 x 151 MB in FP32)",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single run"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1911_10747_gb300 import workloads as W
    cfg = W.large(precision="fp64")
    cores = host_cores()
    for _ in range(args.warmup and 1):
        oracle_sample(cfg, 1, threads=cores)  # warm caches / page in once
    # the oracle takes ~1.5 s per step of this workload on one core: the
    # timed sample is the requested steps or 90 s of them, whichever ends first
    mlups, dt, done = oracle_sample(cfg, max(1, args.steps), budget_s=90.0, threads=cores)
    sample = (f"{done} of the {max(1, args.steps)} requested step(s) of the full 2048x2048+64 workload by the "
              f"FP64 CPU oracle ({dt:.1f} s, time-boxed at 90 s), per-site loops on {cores} threads (OpenMP over "
              "rows; the same workload the GPU arm times in FP32)")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000 / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded initial density noise and bottom-temperature noise)",
            "config": workload_config(cfg.nx, cfg.nf, cfg.ns, 1),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_sweep(lbm, W, torch, dev, steps, seq_precision="fp64_fma"):
    """Runs/hour of the 48-run boiling-curve sweep (widths 128-512, 20,000
    steps per run): batched FP32 through one concurrent graph vs the same 48
    runs stepped one after another in FP64 (the FMA-contracted FP64 path,
    held to 1e-12 of the oracle by the tests; plain FP64 timed beside it).
    The batched leg runs the whole sweep (20,000 steps of every run, timed
    end to end); the sequential legs time `steps` steps of every run and
    scale that time to 20,000 steps (a step costs the same throughout a
    run)."""
    full = 20000
    cfgs = W.sweep(48)
    sites = sum(c.fluid_sites for c in cfgs)
    runs = [lbm.Run(c) for c in cfgs]
    batch = lbm.Batch(runs)
    batch.step(4)
    batch.sync()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    batch.step(full)
    batch.sync()
    dt_b = time.perf_counter() - t0
    vap = [r.vapour_fraction() for r in runs]
    batch.close()
    for r in runs:
        r.close()

    def sequential(cfg_list, prec):
        t = 0.0
        for c in cfg_list:
            r = lbm.Run(c.replace(precision=prec))
            r.step(2)
            r.sync()
            t0 = time.perf_counter()
            r.step(steps)
            r.sync()
            t += time.perf_counter() - t0
            r.close()
        return t

    t_seq = sequential(cfgs, seq_precision)
    t_plain = sequential(cfgs, "fp64")
    hours_b = dt_b / 3600.0
    hours_s = t_seq * full / steps / 3600.0
    return {"runs": len(cfgs), "fluid_sites": sites, "steps_per_run": full, "timed_steps": steps,
            "batched_fp32_runs_per_hour": len(cfgs) / hours_b, "batched_fp32_seconds": dt_b,
            "sequential_fp64_runs_per_hour": len(cfgs) / hours_s, "sequential_precision": seq_precision,
            "sequential_plain_fp64_runs_per_hour": len(cfgs) / (t_plain * full / steps / 3600.0),
            "batched_fp32_mlups": sites * full / dt_b / 1e6,
            "vapour_fraction_after": [min(vap), max(vap)],
            "note": f"batched leg: all 48 runs for the full {full} steps, timed end to end; "
                    f"sequential legs: {steps} steps of every run, scaled to {full}"}


def measure_serving(lbm, W, n_requests, step_scale, load=0.8):
    """Served requests (Poisson arrivals at `load` x the measured capacity,
    150 GB device-memory budget): p50 / p99 time-to-result and aggregate
    MLUPS.  Step counts are the workload's times step_scale."""
    import random
    reqs = W.serving_requests(n_requests, step_scale=step_scale)
    # capacity: measured site-update rate of each precision on a mid-size run
    rate = {}
    for prec in ("fp32", "fp64"):
        c = W.serving_requests(1)[0][0].replace(nx=512, nf=768, ns=32, liquid_rows=256, precision=prec)
        r = lbm.Run(c)
        r.step(4)
        r.sync()
        t0 = time.perf_counter()
        r.step(100)
        r.sync()
        rate[prec] = c.fluid_sites * 100 / (time.perf_counter() - t0)
        r.close()
    mean_service = sum(c.fluid_sites * n / rate[c.precision] for c, n in reqs) / len(reqs)
    lam = load / mean_service
    rng = random.Random(55)
    arrivals, t = [], 0.0
    for _ in reqs:
        t += rng.expovariate(lam)
        arrivals.append(t)
    srv = lbm.Server(hbm_budget_bytes=150 * 10**9, max_active=64, chunk_steps=100)
    ids = [None] * len(reqs)
    nxt = 0
    t0 = time.perf_counter()
    done = 0
    while done < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            ids[nxt] = srv.submit(reqs[nxt][0], reqs[nxt][1])
            nxt += 1
        q, a, _ = srv.counts()
        if a == 0 and q == 0:
            if nxt < len(reqs):
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            continue
        # non-blocking: arrivals are admitted while a chunk runs and join at
        # the next chunk boundary
        fin = srv.poll()
        done += fin
        if fin == 0:
            time.sleep(0.0002)
    makespan = time.perf_counter() - t0
    ttr, work = [], 0.0
    for i, (c, n) in zip(ids, reqs):
        st, (ts, t1, t2) = srv.status(i)
        if st == 2:
            ttr.append(t2 - ts)
            work += c.fluid_sites * n
    srv.close()
    ttr.sort()

    def pct(p):
        return ttr[min(len(ttr) - 1, int(round(p / 100.0 * (len(ttr) - 1))))] if ttr else None

    return {"requests": len(reqs), "completed": len(ttr), "step_scale": step_scale, "offered_load": load,
            "arrival_rate_per_s": lam, "p50_s": pct(50), "p99_s": pct(99), "makespan_s": makespan,
            "aggregate_mlups": work / makespan / 1e6, "budget_bytes": 150 * 10**9,
            "capacity_mlups": {k: v / 1e6 for k, v in rate.items()}}


def measure_wetting(steps):
    """Contact angles of sessile drops at the library's wettability
    coefficients (the three nucleate-spot values and the base), stepped
    together in one batch: the calibration check of Eq. 14's c_w."""
    from paper_1911_10747_gb300 import calibration as K
    from paper_1911_10747_gb300 import workloads as W
    cws = list(W.DEFAULT_CW_SPOTS) + [W.DEFAULT_CW_BASE]
    t0 = time.perf_counter()
    table = K.measure(cws, steps=steps)
    dt = time.perf_counter() - t0
    return {"c_w": cws, "target_deg": [105.0, 115.0, 125.0, 55.0],
            "theta_deg": [None if r["theta_deg"] is None else round(r["theta_deg"], 2) for r in table],
            "mass_drift": [r.get("mass_drift") for r in table],
            "setting": f"200x100 fluid, drop radius 30, isothermal at T_sat, g = 0, FP32, {steps} steps, "
                       "4 runs in one batch; 55 deg is outside the stable range (base c_w = -1.6)",
            "seconds": dt}


def measure_validation(wetting_steps: int = 30000):
    """The paper's validation cases on the GPU path, under both readings of
    the attraction parameter (a = 2/49 as stated; a = 3/49, which gives the
    printed Tc = 0.1094): the Laplace test (surface tension), film boiling
    against Berenson (Eq. 34 vs Eq. 35) for three wall wettabilities, the
    contact angle over a sweep of wall coefficients (is the paper's 55 deg
    base reachable?), and the storage-precision report (stated reading)."""
    import numpy as np
    from paper_1911_10747_gb300 import calibration as K
    from paper_1911_10747_gb300 import validation as V
    from paper_1911_10747_gb300 import workloads as W
    t0 = time.perf_counter()
    out = {"readings": {}}
    prec = None
    for reading in ("stated", "paper_tc"):
        lap = V.laplace([16, 20, 25, 30, 36], precision="fp64", reading=reading)
        dp_max = max(d["dp"] for d in lap["drops"])
        vap_wall = -W.psi_of(0.38, V.with_reading(W.small_parity(), reading))
        film = {}
        fb = None
        for cw in (-1.6, -1.2, round(vap_wall, 4)):
            fb = V.film_boiling(lap["sigma"], precision="fp32", c_w=cw, reading=reading)
            film[f"c_w={cw}"] = {k: fb[k] for k in ("nu_lbm_surface", "nu_lbm_bottom", "nu_berenson",
                                                     "rel_dev_surface", "T_w_over_Tc", "rho_first_fluid_row")}
        grid = [round(v, 2) for v in np.arange(-1.9, -0.95, 0.1)]
        table = K.measure(grid, steps=wetting_steps, reading=reading)
        angles = {str(r["c_w"]): (None if r.get("theta_deg") is None else
                                  ("detached" if r.get("detached") else round(r["theta_deg"], 2))) for r in table}
        attached = [r["theta_deg"] for r in table if r.get("theta_deg") is not None and not r.get("detached")]
        out["readings"][reading] = {
            "a": lap["setting"].split("a = ")[-1],
            "laplace": {"sigma": lap["sigma"], "r2": lap["r2"], "intercept_over_max_dp": lap["intercept"] / dp_max,
                        "setting": lap["setting"]},
            "film_boiling": {"setting": f"model B {fb['domain']}, T_b = 1.27 Tc, sine 5 < t* < 24.98, "
                                        f"averages over 41.63 < t* < 60 ({fb['steps']} steps), FP32",
                             "lambda_d": fb["lambda_d"], "t0": fb["t0"], "by_wall": film,
                             "paper_nu_ratio": 54.01 / 51.28},
            "contact_angle": {"theta_by_c_w": angles, "smallest_stable_deg": min(attached) if attached else None,
                              "55_deg_reachable": bool(attached) and min(attached) <= 55.0,
                              "setting": f"200x100 fluid, drop radius 30, isothermal at T_sat, g = 0, FP32, "
                                         f"{wetting_steps} steps; None: the run faulted (negative psi radicand)"}}
        if reading == "stated":
            prec = V.precision_report(lap["sigma"])
    out["precision"] = prec
    out["seconds"] = time.perf_counter() - t0
    return out


def measure_paper_scale(lbm, W, steps):
    """The paper-scale runs: 400 x 600 fluid over 30 heater rows, superheats
    0.05 / 0.10 / 0.15 / 0.20 Tc, nucleate spots and the noisy bottom, each
    in FP64 and FP32 (the 8 runs of a precision stepped together).  Reports
    per run the time averages of the heater-bottom flux and the vapour
    fraction over the second half and FP32's deviation from FP64."""
    cases = [(d, m) for m in ("spots", "noise") for d in (0.05, 0.10, 0.15, 0.20)]
    out = {"setting": f"400x600 fluid + 30 heater rows, {steps} steps, averages over the second half", "runs": []}
    res = {}
    for prec in ("fp64", "fp32"):
        runs = [lbm.Run(W.paper_scale(d, m, precision=prec), series_capacity=steps + 8) for d, m in cases]
        t0 = time.perf_counter()
        b = lbm.Batch(runs)
        b.step(steps)
        try:
            b.sync()
        except lbm.LbmError:
            pass
        b.close()
        dt = time.perf_counter() - t0
        out[f"{prec}_seconds"] = dt
        out[f"{prec}_mlups"] = len(runs) * 400 * 600 * steps / dt / 1e6
        for (d, m), r in zip(cases, runs):
            try:
                r.sync()
                ser = r.series(0, steps)
                res[(d, m, prec)] = (float(ser[steps // 2:, 0].mean()), float(ser[steps // 2:, 2].mean()))
            except lbm.LbmError as e:
                res[(d, m, prec)] = str(e)
            r.close()
    worst = 0.0
    for d, m in cases:
        a, c = res[(d, m, "fp64")], res[(d, m, "fp32")]
        row = {"superheat_over_Tc": d, "bc": m}
        if isinstance(a, tuple) and isinstance(c, tuple):
            row.update(q_fp64=a[0], q_fp32=c[0], vf_fp64=a[1], vf_fp32=c[1],
                       q_rel_dev=c[0] / a[0] - 1.0, vf_rel_dev=c[1] / a[1] - 1.0)
            worst = max(worst, abs(row["q_rel_dev"]), abs(row["vf_rel_dev"]))
        else:
            row.update(fault_fp64=None if isinstance(a, tuple) else a, fault_fp32=None if isinstance(c, tuple) else c)
        out["runs"].append(row)
    out["max_rel_dev"] = worst
    return out


def measure_chf(lbm, W, steps):
    """Boiling curve on a 256 x 384 domain over 16 heater rows (constant
    bottom with nucleate spots): time-averaged heater-bottom flux Q'' over
    the second half of `steps` steps at 7 superheats, in FP32, FP64 and FP16
    storage (all 21 runs in one batch).  CHF = max Q'' over the superheats."""
    base = W.sweep(1)[0].replace(nx=256, nf=384, ns=16, liquid_rows=128, bc_mode="spots",
                                 spot_x=W.scaled_spots(256), spot_half_width=3,
                                 c_w_spot=W.DEFAULT_CW_SPOTS, g=W.stable_gravity(384, 128), seed=21)
    dts = [0.04, 0.08, 0.12, 0.16, 0.20, 0.24, 0.28]
    precs = ("fp32", "fp64", "fp16", "fp32_dfsrc")
    cfgs = [base.replace(T_b_over_Tc=0.86 + d, precision=p) for p in precs for d in dts]
    runs = [lbm.Run(c, series_capacity=steps + 8) for c in cfgs]
    alive = list(range(len(runs)))
    fault = [None] * len(runs)
    t0 = time.perf_counter()
    chunk = 1000
    done = 0
    while done < steps and alive:
        k = min(chunk, steps - done)
        b = lbm.Batch([runs[i] for i in alive])
        try:
            b.step(k)
            b.sync()
        except lbm.LbmError:
            pass
        b.close()
        still = []
        for i in alive:
            try:
                runs[i].sync()
                still.append(i)
            except lbm.LbmError:
                fault[i] = done + k  # faulted within this chunk
        alive = still
        done += k
    dt = time.perf_counter() - t0
    q = [None] * len(runs)
    for i in alive:
        ser = runs[i].series(0, steps)
        q[i] = float(ser[steps // 2:, 0].mean())
    for r in runs:
        r.close()
    n = len(dts)
    q32, q64, q16, qdf = q[:n], q[n:2 * n], q[2 * n:3 * n], q[3 * n:]
    both = [j for j in range(n) if q32[j] is not None and q64[j] is not None]
    c32 = max(q32[j] for j in both) if both else None
    c64 = max(q64[j] for j in both) if both else None
    all3 = [j for j in both if q16[j] is not None]
    c16 = max(q16[j] for j in all3) if all3 else None
    c64b = max(q64[j] for j in all3) if all3 else None
    bdf = [j for j in both if qdf[j] is not None]
    cdf = max(qdf[j] for j in bdf) if bdf else None
    c64d = max(q64[j] for j in bdf) if bdf else None
    return {"domain": "256x384 fluid + 16 heater rows, spots", "steps": steps, "superheats_over_Tc": dts,
            "q_fp32": q32, "q_fp64": q64, "q_fp16": q16, "q_fp32_dfsrc": qdf, "fault_step_fp32": fault[:n],
            "fault_step_fp64": fault[n:2 * n], "fault_step_fp16": fault[2 * n:3 * n],
            "fault_step_fp32_dfsrc": fault[3 * n:],
            "chf_rel_error_fp32_dfsrc": abs(cdf - c64d) / abs(c64d) if bdf else None,
            "max_rel_error_curve_fp32_dfsrc": max(abs(qdf[j] - q64[j]) / abs(q64[j]) for j in bdf) if bdf else None,
            "max_rel_diff_curve_fp32_vs_dfsrc": max(abs(q32[j] - qdf[j]) / abs(qdf[j]) for j in bdf) if bdf else None,
            "chf_fp32": c32, "chf_fp64": c64, "chf_fp16": c16,
            "chf_superheat_fp32": dts[q32.index(c32)] if both else None,
            "chf_superheat_fp64": dts[q64.index(c64)] if both else None,
            "chf_rel_error": abs(c32 - c64) / abs(c64) if both else None,
            "max_rel_error_curve": max(abs(q32[j] - q64[j]) / abs(q64[j]) for j in both) if both else None,
            "chf_rel_error_fp16": abs(c16 - c64b) / abs(c64b) if all3 else None,
            "max_rel_error_curve_fp16": max(abs(q16[j] - q64[j]) / abs(q64[j]) for j in all3) if all3 else None,
            "seconds": dt}


def measure_dfsrc(lbm, W, torch, stream, steps, err_steps=20):
    """FP32 with the Eq. 24 source in double-float arithmetic on the
    benchmarked workload: step time (autotuned among its heat shapes), and
    the errors of it and of the all-FP32 path on the same heat-kernel shape
    after `err_steps` steps against the FP64 GPU path (which matches the FP64
    oracle bit for bit in the parity tests), so the source term's share of
    the FP32 error shows."""
    import numpy as np
    cfg = W.large(precision="fp32_dfsrc", seed=3)
    r = lbm.Run(cfg, stream=stream.cuda_stream)
    r.autotune(10)
    v = r.variants()
    r.step(3)
    r.sync()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    r.step(steps)
    a1.record(stream)
    a1.synchronize()
    ms = a0.elapsed_time(a1) / steps
    r.set_timing(True)
    r.step(min(steps, 100))
    kms, _ = r.kernel_times()
    r.close()
    torch.cuda.empty_cache()
    ref = lbm.Run(W.large(precision="fp64", seed=3), stream=stream.cuda_stream)
    ref.step(err_steps)
    want = ref.fields(("rho", "T"))
    ref.close()
    torch.cuda.empty_cache()
    errs = {}
    for prec, heat in (("fp32", "heatrows_64x8x4"), ("fp32_dfsrc", "heatrows_64x8x4_dfsrc")):
        g = lbm.Run(W.large(precision=prec, seed=3), stream=stream.cuda_stream)
        gv = g.variants()
        g.select_variants(0, gv["heat"].index(heat))
        g.step(err_steps)
        got = g.fields(("rho", "T"))
        g.close()
        torch.cuda.empty_cache()
        errs[prec] = {k: float(np.max(np.abs(got[k] - want[k]) / np.abs(want[k]))) for k in ("rho", "T")}
    return {"value": cfg.fluid_sites / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
            "kernel_ms": {"flow": kms[0], "heat": kms[1], "diag": kms[2]},
            "variants": {"flow": v["flow"][v["selected"][0]], "heat": v["heat"][v["selected"][1]]},
            "max_rel_error_vs_fp64": errs, "error_steps": err_steps,
            "note": "source term of Eq. 24 in double-float (FP32 pairs, ~45-48-bit significand); errors after "
                    f"{err_steps} steps against the FP64 GPU path, both FP32 runs on the same heat shape "
                    "(heatrows_64x8x4) and flow variant"}


def run_ours(args):
    import numpy as np
    import torch

    from paper_1911_10747_gb300 import build as B
    from paper_1911_10747_gb300 import lbm
    from paper_1911_10747_gb300 import workloads as W

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    lbm.load()

    cfg = W.large(precision=args.precision, seed=3 + rank)
    stream = torch.cuda.Stream(device=dev)
    run = lbm.Run(cfg, stream=stream.cuda_stream, device=local)
    kps = run.kernels_per_step()
    sites = cfg.fluid_sites

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # launch-shape autotuning (does not advance the run), then warm-up (also
    # builds the two-step graph)
    variants = run.variants()
    if args.flow_variant or args.heat_variant:
        fv = variants["flow"].index(args.flow_variant) if args.flow_variant else variants["selected"][0]
        hv = variants["heat"].index(args.heat_variant) if args.heat_variant else variants["selected"][1]
        run.select_variants(fv, hv)
    else:
        run.autotune(20)
    variants = run.variants()
    run.step(max(args.warmup, 3))
    run.sync()
    # ---- timed region: K steps, CUDA events on the run's stream ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        e0.record(stream)
        run.step(args.steps)
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    run.sync()
    ms_max, value = aggregate_over_ranks(ms, sites, args.steps, dev)

    # ---- per-kernel durations over K more steps (events around each launch) ----
    run.set_timing(True)
    run.step(min(args.steps, 200))
    kms, nl = run.kernel_times()
    run.set_timing(False)
    hbm, peak_kind = peaks()
    vnames = (variants["flow"][variants["selected"][0]], variants["heat"][variants["selected"][1]])
    flow_bytes = ALG_FLOW_BYTES[args.precision] * sites
    flow_achieved = flow_bytes / (kms[0] / 1e3) / 1e9
    flow_roof = {"bound": "hbm", "achieved": flow_achieved, "peak": hbm, "unit": "GB/s",
                 "frac": flow_achieved / hbm, "kernel": "k_flow", "bytes_per_site": ALG_FLOW_BYTES[args.precision],
                 "traffic": ncu_traffic("flow", vnames[0]) if args.precision == "fp32" else None,
                 "peak_source": peak_kind}
    fp32_peak = FP32_LANES * 2 * max_sm_mhz() * 1e6 / 1e12
    hflops, hcounted = heat_flops(vnames[1]) if args.precision == "fp32" else (None, None)
    heat_achieved = hflops * cfg.temperature_sites / (kms[1] / 1e3) / 1e12 if hflops else None
    heat_roof = {"bound": "alu", "achieved": heat_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                 "frac": heat_achieved / fp32_peak if hflops else None, "kernel": "k_heat",
                 "flops_per_site": hflops, "flops_counted_on": hcounted,
                 "flops_kind": "executed FP32 operations (ncu SASS counts, tile halo included)",
                 "traffic": ncu_traffic("heat", vnames[1]) if args.precision == "fp32" else None,
                 "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    # the same fraction against the FMA throughput measured on this GPU (context)
    fma32 = lbm.peak_fma(32, device=local)
    heat_roof.update(measured_fma_peak=fma32, frac_of_measured_fma=heat_achieved / fma32 if hflops else None)
    # instruction issue (context: both kernels spend their time issuing or
    # waiting, not moving bytes or doing flops at the pipes' rates)
    if args.precision == "fp32":
        flow_roof["issue"] = issue_roofline(ncu_instructions("flow", vnames[0]), sites, kms[0])
        heat_roof["issue"] = issue_roofline(ncu_instructions("heat", vnames[1]), cfg.temperature_sites, kms[1])
    step_ms = ms_max / args.steps
    step_achieved = ALG_STEP_BYTES[args.precision] * sites / (step_ms / 1e3) / 1e9
    dominant = flow_roof if kms[0] >= kms[1] else heat_roof

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        nfl, ntl = cfg.fluid_sites, cfg.temperature_sites
        st = run.fields(("f", "T"))
        e2e_steps = max(2, min(args.steps, 10))

        def end_to_end(dtype, setter):
            hf = torch.from_numpy(st["f"].reshape(-1).astype(dtype)).pin_memory()
            hT = torch.from_numpy(st["T"].reshape(-1).astype(dtype)).pin_memory()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for k in range(e2e_steps):
                setter(hf.data_ptr(), hT.data_ptr(), step=1000 + k, src_is_device=False)
                run.step(1)
                run.wall_heat_flux()
                run.vapour_fraction()
            return ws * sites * e2e_steps / (time.perf_counter() - t0) / 1e6

        # the run's storage is float32 (or narrower) unless it is the FP64
        # path: its state crosses the host link as float32
        if args.precision == "fp64":
            e2e = {"value": end_to_end(np.float64, run.set_state), "unit": "MLUPS",
                   "h2d_bytes_per_step": (9 * nfl + ntl) * 8, "d2h_bytes_per_step": 16,
                   "note": "per step: lbm_set_state from pinned float64 host arrays (read by the import kernel "
                           "over the host link), lbm_step(1), lbm_wall_heat_flux + lbm_vapour_fraction read-back"}
        else:
            v32 = end_to_end(np.float32, run.set_state_f32)
            v64 = end_to_end(np.float64, run.set_state)
            e2e = {"value": v32, "unit": "MLUPS",
                   "h2d_bytes_per_step": (9 * nfl + ntl) * 4, "d2h_bytes_per_step": 16,
                   "note": "per step: lbm_set_state_f32 from pinned float32 host arrays (read by the import kernel "
                           "over the host link), lbm_step(1), lbm_wall_heat_flux + lbm_vapour_fraction read-back",
                   "float64_state": {"value": v64, "unit": "MLUPS", "h2d_bytes_per_step": (9 * nfl + ntl) * 8,
                                     "note": "the same with lbm_set_state and float64 arrays"}}

    # ---- FP64 path on the same workload ----
    fp64 = None
    if not args.no_fp64 and args.precision != "fp64":
        run.close()
        torch.cuda.empty_cache()
        r64 = lbm.Run(W.large(precision="fp64", seed=3 + rank), stream=stream.cuda_stream, device=local)
        r64.step(3)
        r64.sync()
        k64 = max(4, min(100, args.steps // 10))
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r64.step(k64)
        a1.record(stream)
        a1.synchronize()
        ms64 = a0.elapsed_time(a1) / k64
        r64.set_timing(True)
        r64.step(k64)
        k64ms, _ = r64.kernel_times()
        r64.close()
        # the FMA-contracted FP64 path (held to 1e-12 of the oracle) on the same workload
        rf = lbm.Run(W.large(precision="fp64_fma", seed=3 + rank), stream=stream.cuda_stream, device=local)
        rf.step(3)
        rf.sync()
        a0.record(stream)
        rf.step(k64)
        a1.record(stream)
        a1.synchronize()
        msf = a0.elapsed_time(a1) / k64
        rf.set_timing(True)
        rf.step(k64)
        kfms, _ = rf.kernel_times()
        rf.close()
        fp64 = {"value": sites / (ms64 / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms64,
                "kernel_ms": {"flow": k64ms[0], "heat": k64ms[1], "diag": k64ms[2]},
                "fma": {"value": sites / (msf / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": msf,
                        "kernel_ms": {"flow": kfms[0], "heat": kfms[1], "diag": kfms[2]},
                        "note": "FP64 kernels compiled with FMA contraction; within 1e-12 of the oracle, "
                                "not bit-identical"},
                "flow_hbm_frac": ALG_FLOW_BYTES["fp64"] * sites / (k64ms[0] / 1e3) / 1e9 / hbm}
        # FP64 is arithmetic-bound: flops counted by ncu against the measured
        # FP64 FMA throughput of this GPU
        fma64 = lbm.peak_fma(64, iters=1024, device=local)
        fl, fh = ncu_fp64_flops("flow"), ncu_fp64_flops("heat")
        fp64["fma_peak_tflops"] = fma64
        if fl is not None and fh is not None:
            ach = (fl * sites / (k64ms[0] / 1e3) / 1e12, fh * cfg.temperature_sites / (k64ms[1] / 1e3) / 1e12)
            fp64["alu_roofline"] = {
                "flow": {"bound": "fp64_alu", "achieved": ach[0], "peak": fma64, "unit": "TFLOP/s",
                         "frac": ach[0] / fma64, "flops_per_site": fl},
                "heat": {"bound": "fp64_alu", "achieved": ach[1], "peak": fma64, "unit": "TFLOP/s",
                         "frac": ach[1] / fma64, "flops_per_site": fh},
                "peak_source": "lbm_peak_fma(64): FMA chains on every SM, measured in this run"}
            # the same kernels against the FP64 pipe's instruction rate: a
            # DADD or DMUL takes the pipe like a DFMA, so with -fmad=false the
            # flop fraction understates how busy the pipe is
            il, ih = ncu_fp64_instructions("flow"), ncu_fp64_instructions("heat")
            if il is not None and ih is not None:
                ipk = fma64 / 2.0  # T FP64 instructions/s
                ia = (il * sites / (k64ms[0] / 1e3) / 1e12, ih * cfg.temperature_sites / (k64ms[1] / 1e3) / 1e12)
                fp64["pipe_roofline"] = {
                    "flow": {"achieved": ia[0], "peak": ipk, "unit": "T FP64 instructions/s", "frac": ia[0] / ipk,
                             "instructions_per_site": il},
                    "heat": {"achieved": ia[1], "peak": ipk, "unit": "T FP64 instructions/s", "frac": ia[1] / ipk,
                             "instructions_per_site": ih},
                    "peak_source": "half the measured FP64 FMA flop rate (one DFMA = 2 flops per instruction)"}
    else:
        run.close()

    # ---- FP16-storage probe on the same workload (populations stored as
    # half, arithmetic in FP32) ----
    fp16 = None
    if not args.no_fp16 and args.precision == "fp32":
        torch.cuda.empty_cache()
        r16 = lbm.Run(W.large(precision="fp16", seed=3 + rank), stream=stream.cuda_stream, device=local)
        r16.autotune(20)
        r16.step(max(args.warmup, 3))
        r16.sync()
        k16 = max(20, min(1000, args.steps // 2))
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        r16.step(k16)
        a1.record(stream)
        a1.synchronize()
        ms16 = a0.elapsed_time(a1) / k16
        r16.set_timing(True)
        r16.step(min(k16, 200))
        k16ms, _ = r16.kernel_times()
        v16 = r16.variants()
        r16.close()
        fl16 = ALG_FLOW_BYTES["fp16"] * sites / (k16ms[0] / 1e3) / 1e9
        fp16 = {"value": sites / (ms16 / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms16, "steps": k16,
                "kernel_ms": {"flow": k16ms[0], "heat": k16ms[1], "diag": k16ms[2]},
                "variants": {"flow": v16["flow"][v16["selected"][0]], "heat": v16["heat"][v16["selected"][1]]},
                "flow_roofline": {"bound": "hbm", "achieved": fl16, "peak": hbm, "unit": "GB/s", "frac": fl16 / hbm,
                                  "bytes_per_site": ALG_FLOW_BYTES["fp16"]}}

    # ---- FP32 with the Eq. 24 source in double-float arithmetic ----
    dfsrc = None
    if not args.no_dfsrc and args.precision == "fp32":
        dfsrc = measure_dfsrc(lbm, W, torch, stream, max(20, min(500, args.steps // 4)))

    # ---- boiling-curve sweep: 48 runs batched (FP32, one concurrent graph)
    # versus the same runs one after another in FP64 ----
    sweep = None
    if not args.no_sweep:
        sweep = measure_sweep(lbm, W, torch, dev, args.sweep_steps)

    wetting = None
    if rank == 0 and not args.no_wetting:
        wetting = measure_wetting(args.wetting_steps)
    validation = None
    if rank == 0 and not args.no_validation:
        validation = measure_validation(args.wetting_steps)

    paper = None
    if args.paper_scale and rank == 0:
        paper = measure_paper_scale(lbm, W, args.paper_scale_steps)

    chf = None
    if not args.no_chf and ws == 1:
        chf = measure_chf(lbm, W, args.chf_steps)
    serve = None
    if not args.no_serve and ws == 1:
        serve = measure_serving(lbm, W, args.serve_requests, args.serve_step_scale)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ----
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cores = host_cores()
        cm, cdt, csteps = oracle_sample(W.large(precision="fp64"), 200, budget_s=12.0, threads=cores)
        sm, sdt, ssteps = oracle_sample(W.large(precision="fp64"), 10, budget_s=6.0, threads=1)
        cpu = {"value": cm, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{csteps} steps of the full 2048x2048+64 workload in FP64 ({cdt:.1f} s, per-site loops "
                         f"on {cores} threads, OpenMP over rows)",
               "single_thread": {"value": sm, "unit": "MLUPS", "cores": 1,
                                 "sample": f"{ssteps} steps of the same workload ({sdt:.1f} s, 1 thread)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "fp16": "f16-storage/f32"}[args.precision],
            "data": "synthetic (seeded initial density noise and bottom-temperature noise)",
            "config": workload_config(cfg.nx, cfg.nf, cfg.ns, ws, args.precision),
            "roofline": dict(dominant, step={"bound": "hbm", "achieved": step_achieved, "peak": hbm,
                                             "frac": step_achieved / hbm,
                                             "bytes_per_site": ALG_STEP_BYTES[args.precision]}),
            "kernel_rooflines": {"flow": flow_roof, "heat": heat_roof},
            "kernel_ms": {"flow": kms[0], "heat": kms[1], "diag": kms[2], "launches_timed": nl},
            "variants": {"flow": variants["flow"][variants["selected"][0]],
                         "heat": variants["heat"][variants["selected"][1]]},
            "gpu_launches": kps * args.steps,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64": fp64,
            "fp16": fp16,
            "fp32_dfsrc": dfsrc,
            "sweep": sweep,
            "serve": serve,
            "chf": chf,
            "wetting": wetting,
            "paper_scale": paper,
            "validation": validation,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-storage throughput block")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-dfsrc", action="store_true", help="skip the double-float source-term block")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=500)
    ap.add_argument("--flow-variant", default="", help="pin the flow kernel variant (no autotuning)")
    ap.add_argument("--heat-variant", default="", help="pin the heat kernel variant (no autotuning)")
    ap.add_argument("--no-wetting", action="store_true", help="skip the contact-angle check of the c_w values")
    ap.add_argument("--no-validation", action="store_true", help="skip the Laplace / film-boiling / precision cases")
    ap.add_argument("--wetting-steps", type=int, default=30000)
    ap.add_argument("--paper-scale", action="store_true", help="also run the 400x600 FP64 vs FP32 comparison")
    ap.add_argument("--paper-scale-steps", type=int, default=100000)
    ap.add_argument("--no-chf", action="store_true", help="skip the FP32 / FP16 / FP64 boiling-curve comparison")
    ap.add_argument("--chf-steps", type=int, default=6000)
    ap.add_argument("--no-serve", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--serve-requests", type=int, default=80)
    ap.add_argument("--serve-step-scale", type=float, default=0.01)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
