#!/usr/bin/env python
"""Throughput benchmark of the 1D Maxwell-Bloch hot path on GB300.

Workload (one bench step = one whole simulation): the two-level SIT medium at
scale -- 1,048,576 cells, 200,000 time steps, +-1 % seeded per-cell jitter of
density and transition frequency -- solved through the C ABI.  Metric:
Gcell-steps/s (cells x time steps / device time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (the path does
not need any exchange between GPUs); value = all ranks' cell-steps / the
slowest rank's time.  --impl reference times the CPU FP64 oracle on bounded
samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "Gcell-steps/s"
HBM_FALLBACK = 6800.0


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def compute_peaks():
    """Arithmetic peaks measured on this GPU model by the library's own
    microbenchmarks (mbs_peak_rates; profiles/compute_peaks.json, written by
    `python -m paper_2005_05412_gb300.peaks`), per SM and clock cycle."""
    try:
        return json.load(open(os.path.join(ROOT, "profiles", "compute_peaks.json")))
    except Exception:
        return {}


def issue_peak(cp, sm_mhz, n_sm=152):
    """Warp instructions per second the SMs can issue at the sampled clock:
    the measured FP32-FMA warp-instruction rate per SM cycle (the FMA lanes
    issue one warp instruction per scheduler and cycle), else the nominal 4
    schedulers x 1 instruction per cycle."""
    per = cp.get("issue_warp_inst_per_cycle_per_sm")
    src = "measured (FP32 FMA microbenchmark, profiles/compute_peaks.json) x sampled clock"
    if not per:
        per, src = 4.0, "nominal 4 schedulers x 1 warp instruction per cycle x sampled clock"
    return per * n_sm * sm_mhz / 1e3, src


def issue_roof(prof, per_launch_s, clocks, cp, hbm_obj):
    """The binding roof of the tiled kernels: warp instructions issued per
    second (ncu smsp__inst_executed.sum per launch of the same kernel and
    tile shape / the CUDA-event launch time) against the issue peak; the HBM
    figure by algorithmic bytes (which temporal tiling lets exceed 1) kept as
    a secondary field."""
    if not (prof and prof.get("warp_inst") and clocks.get("sm_mhz")):
        return dict(hbm_obj, note="no current ncu instruction count for this kernel: HBM figure only")
    ach = prof["warp_inst"] / per_launch_s / 1e9
    pk, src = issue_peak(cp, clocks["sm_mhz"])
    return {"bound": "alu", "resource": "instruction issue", "achieved": round(ach, 1), "peak": round(pk, 1),
            "unit": "Gwarp-inst/s", "frac": round(ach / pk, 4), "traffic": hbm_obj.get("traffic"),
            "peak_source": src, "warp_inst_per_launch": prof["warp_inst"],
            "inst_source": "ncu smsp__inst_executed.sum of the same kernel and tile shape (profiles/traffic.json)",
            "kernel": hbm_obj.get("kernel"), "launch_ms": hbm_obj.get("launch_ms"), "hbm": hbm_obj}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_label(p):
    """The workload named by what it is, identical in both arms' `config`."""
    return (f"{p.name}: {p.n_cells} cells x {p.n_steps} steps, N={p.qms[0].n_levels}"
            + (", per-cell jitter" if p.jitter is not None else ""))


def workload(name):
    if name == "sit_2lvl_jitter":
        return W.sit_2lvl_jitter()
    if name == "sit_2lvl_jitter_small":
        return W.sit_2lvl_jitter(n_cells=65_536, n_steps=20_000)
    return W.WORKLOADS[name]()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- ranks
def max_over_ranks(t_local, world, device):
    """The slowest rank's time (an all-reduce MAX over the process group)."""
    if world == 1:
        return t_local
    import torch
    t = torch.tensor([t_local], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(cell_steps, steps, world, t_max):
    """Whole-job throughput [Gcell-steps/s]: every rank solves its own replica
    of the workload `steps` times; all ranks' cell-steps over the slowest
    rank's time."""
    return cell_steps * steps * world / t_max / 1e9


# ---------------------------------------------------------------- CPU oracle
def cpu_sample(p, cells, steps):
    """A slab of the workload for timing the oracle: `cells` consecutive
    medium cells (with their jitter) driven by the same source; probes (E and
    rho_11) 500 and 2,000 cells in, which the pulse has passed within the
    sampled steps."""
    m0 = int(math.ceil(0.05 * p.n_cells))
    jit = None if p.jitter is None else p.jitter[m0:m0 + cells].copy()
    length = cells * p.dz
    probes = [W.Probe(c, q) for c in (500, 2000) for q in (W.Q_E, W.Q_RHO_RE)]
    return p.replace(n_cells=cells, length=length, regions=[W.Region(1, 0.0, length)], jitter=jit,
                     n_steps=steps, t_end=0.0, probes=probes,
                     sources=[W.Source(W.SRC_TFSF_RIGHT, 2, *[getattr(p.sources[0], k) for k in
                                                               ("e0", "tau", "t0", "omega", "phase")])])


def time_oracle(p, target_s=12.0, cells=65_536):
    import oracle
    probe = oracle.run(cpu_sample(p, cells, 20))
    rate = cells * 20 / probe["seconds"]
    steps = max(20, int(target_s * rate / cells))
    smp = cpu_sample(p, cells, steps)
    r = oracle.run(smp)
    return dict(value=cells * steps / r["seconds"] / 1e9, cores=r["threads"], seconds=r["seconds"],
                sample=f"{cells} medium cells x {steps} steps of the workload (jitter slab, one source)",
                problem=smp, records=r["records"])


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local):
    import torch
    import paper_2005_05412_gb300 as mbs
    from paper_2005_05412_gb300 import build as mbs_build
    if rank == 0 or not os.path.exists(mbs.LIB_PATH):
        mbs_build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    p = workload(args.workload)
    if args.nsteps > 0:
        p = p.replace(n_steps=args.nsteps)
    cell_steps = p.n_cells * p.n_steps
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    T = args.tile
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def solve():
        mbs.mbs_solve([sc], args.precision, "tiled", tile_steps=T, stream=stream.cuda_stream,
                      wide_tiles=args.wide_tiles)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev_index) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            stream.wait_stream(torch.cuda.current_stream())
            ev[k][0].record(stream)
            solve()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    if world > 1:
        torch.distributed.barrier()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_local = dev_ms / 1e3
    t_max = max_over_ranks(t_local, world, "cuda")
    ctr = mbs.mbs_scenario_counters(sc)
    launches = ctr["kernel_launches"]
    value = job_value(cell_steps, args.steps, world, t_max)
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    # roofline of the dominant kernel (the tiled step): algorithmic bytes per
    # cell-step = (2 + K) state values read + written, plus the 2 read-only
    # per-cell parameters of a jittered medium
    n_lv = p.qms[0].n_levels
    K = n_lv * n_lv - 1
    jit = p.jitter is not None
    rb = 4 if args.precision == "fp32" else 8
    alg_bytes = (2 * (2 + K) + (2 if jit else 0)) * rb
    tiled_launches = math.ceil(p.n_steps / T)
    per_launch_s = t_local / args.steps / max(1, launches)
    units_per_launch = p.n_cells * T
    achieved = alg_bytes * units_per_launch / per_launch_s / 1e9
    prof = load_profile(f"{args.workload}_{args.precision}_T{args.tile}" + ("_C256" if args.wide_tiles else ""))
    traffic = prof.get("dram_bytes") if prof else None
    hbm_obj = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm or HBM_FALLBACK, "unit": "GB/s",
               "frac": round(achieved / (hbm or HBM_FALLBACK), 4), "traffic": traffic,
               "peak_source": "measured" if hbm else "fallback",
               "kernel": (f"k_tiled_tc<{n_lv}> (tcgen05 3xTF32)" if n_lv >= 4 else
                          f"k_tiled<{args.precision},N={n_lv}{',percell' if jit else ''}>") + f" T={T}",
               "alg_bytes_per_cell_step": alg_bytes, "launch_ms": round(per_launch_s * 1e3, 5),
               "launches_per_solve": launches, "tiled_launches_per_solve": tiled_launches}
    clocks = clk.summary()
    cp = compute_peaks()
    roof = issue_roof(prof, per_launch_s, clocks, cp, hbm_obj)
    out = {"metric": METRIC, "value": round(value, 3), "unit": METRIC, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max * 1e3 / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
           "data": "synthetic (seeded)",
           "config": {"workload": workload_label(p),
                      "precision": args.precision, "algo": "tiled", "tile_steps": T,
                      "parallelism": f"replicas x{world}", "l2": "flushed between steps (256 MB write)",
                      "fp64_baseline_samples": "the FP64 legs time rates on samples: main workload plain and tiled "
                                               "on its first 4,000 steps, the three- and six-level plain paths on "
                                               "their first 1,000, the FP64 batch on its first 64 simulations; "
                                               "the FP32-vs-FP64 parity runs them in full, untimed"},
           "roofline": roof, "clocks": clocks, "gpu_launches": launches * args.steps,
           "wall_s": round(wall, 3)}
    if rank == 0 and not args.quick:
        # per-result error against the FP64 path (all outside the timed region)
        par = {}
        if args.precision == "fp32" and args.nsteps == 0:
            par[p.name] = fp32_vs_fp64(mbs, stream, torch, p, sc, "tiled", T)
        out["fp64_plain"] = fp64_plain(p, mbs, stream, torch)
        out["six_level"] = level_leg(mbs, stream, torch, "ladder_6lvl", 0, pk, clocks)
        out["three_level"] = level_leg(mbs, stream, torch, "lambda_3lvl", 0, pk, clocks)
        for leg in ("three_level", "six_level"):
            par[out[leg]["workload"].split(":")[0]] = out[leg].pop("parity")
        out["cells"] = cells_leg(mbs, stream, torch, clocks)
        out["n_scaling"] = n_scaling_leg(mbs, stream, torch)
        if not args.no_batch:
            out["batch"] = batch_leg(mbs, stream, torch, "fp32")
            par["batch_mixed"] = out["batch"].pop("parity")
        out["e2e"] = e2e(p, mbs, args, torch, stream)
        if world == 1 and not args.no_cpu:
            cb = time_oracle(p)
            out["cpu_baseline"] = {"value": round(cb["value"], 5), "unit": METRIC, "cores": cb["cores"],
                                   "kind": "oracle", "sample": cb["sample"]}
            # the GPU paths on the oracle's own timed sample
            smp = {}
            for prec, algo in (("fp32", "tiled"), ("fp64", "plain")):
                g = mbs.run(cb["problem"], precision=prec, algo=algo, stream=stream.cuda_stream)["records"]
                smp[f"{prec}_{algo}_vs_oracle"] = float(f"{trace_errors(g, cb['records'], cb['problem'].probes)[0]:.3e}")
            smp["sample"] = cb["sample"]
            par["cpu_baseline_sample"] = smp
        par["oracle_windows"] = stored_oracle_parity()
        out["parity"] = par
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- parity
def trace_errors(a, b, probes):
    """Worst relative L2 of the traces a against b over the probes, and the
    worst for the populations' deviation from their initial value."""
    worst = dev = 0.0
    for k, q in enumerate(probes):
        nb = np.linalg.norm(b[k])
        if nb == 0.0:
            continue
        worst = max(worst, float(np.linalg.norm(a[k] - b[k]) / nb))
        if q.quantity == W.Q_RHO_RE and np.any(b[k] != b[k][0]):
            d = b[k] - b[k][0]
            dev = max(dev, float(np.linalg.norm(a[k] - b[k][0] - d) / np.linalg.norm(d)))
    return worst, dev


def fetch_all(mbs, sc, n):
    return np.stack([mbs.mbs_fetch_records(sc, k) for k in range(n)])


def fp32_vs_fp64(mbs, stream, torch, p, sc32, algo64, tile64=0):
    """Per-result error of a full-length FP32 solve (the scenario sc32 after
    its last solve) against the FP64 path on the GPU, every probe trace over
    the whole run, plus the state checks of both; outside any timed region."""
    r32 = fetch_all(mbs, sc32, len(p.probes))
    st32 = mbs.mbs_scenario_stats(sc32)
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)
    mbs.mbs_solve([sc], "fp64", algo64, tile_steps=tile64, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    r64 = fetch_all(mbs, sc, len(p.probes))
    st64 = mbs.mbs_scenario_stats(sc)
    worst, pdev = trace_errors(r32, r64, p.probes)
    return {"fp32_vs_fp64_worst_trace": float(f"{worst:.3e}"), "fp32_vs_fp64_worst_population_deviation":
            float(f"{pdev:.3e}"), "probes": len(p.probes), "steps": p.n_steps, "fp64_path": algo64,
            "max_trace_dev": float(f"{max(st32['max_trace_dev'], st64['max_trace_dev']):.3e}"),
            "min_eig": float(f"{min(st32['min_eig'], st64['min_eig']):.3e}")}


def stored_oracle_parity():
    """The oracle comparisons of the GPU test suite (light-cone windows of the
    full-size workloads, the 2,048-cell SIT case in full, the batch truncated
    to 5,000 steps), as written by `MBS_PARITY_OUT=profiles/parity_gb300.json
    python -m pytest tests -m gpu` and committed; summarised by worst case."""
    f = os.path.join(ROOT, "profiles", "parity_gb300.json")
    try:
        d = json.load(open(f))
    except Exception:
        return None
    out = {}
    for k, v in d.items():
        if isinstance(v, dict) and "worst" in v:
            w = v["worst"]
            out[k] = {"worst_trace": w.get("err"), "worst_population_deviation": max(r.get("dev", 0.0) for r in v["rows"]),
                      "items": v.get("simulations", len(v["rows"]))}
        else:
            out[k] = v
    out["source"] = "profiles/parity_gb300.json (pytest -m gpu with MBS_PARITY_OUT)"
    return out


# bytes of algorithmic state per cell-step (2 + K values read and written)
def state_bytes(n_levels, rb=4):
    return 2 * (2 + n_levels * n_levels - 1) * rb


def level_leg(mbs, stream, torch, name, T, pk, clocks, reps=2, fp64_steps=1000, parity=True):
    """One whole simulation of the multi-level workloads at full size (the
    six-level ladder, 131,072 cells x 50,000 steps, on the tensor-core tiles;
    the three-level Lambda medium, 262,144 cells x 100,000 steps), FP32, with
    the FP32 and FP64 plain paths timed on their first steps."""
    p = W.WORKLOADS[name]()
    n = p.qms[0].n_levels
    K = n * n - 1
    dev = mbs.device_from_problem(p)
    sc = mbs.scenario_from_problem(dev, p)

    def timed(scn, prec, algo, tile, tune=False):
        # warm-up (with tune: measures the tile depth, cached for the timed calls)
        mbs.mbs_solve([scn], prec, algo, tile_steps=tile, stream=stream.cuda_stream, autotune=tune)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mbs.mbs_solve([scn], prec, algo, tile_steps=tile, stream=stream.cuda_stream, autotune=tune)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            best = t if best is None else min(best, t)
        return best

    t = timed(sc, "fp32", "tiled", T, tune=T == 0)
    launches = mbs.mbs_scenario_counters(sc)["kernel_launches"]
    Teff = mbs.mbs_scenario_tile(sc)
    cells = mbs.mbs_scenario_tile_cells(sc)
    value = p.n_cells * p.n_steps / t / 1e9
    hbm = pk.get("hbm_gbs") or HBM_FALLBACK
    per_launch = t / max(1, launches)
    out = {"value": round(value, 3), "unit": METRIC,
           "workload": f"{p.name}: {p.n_cells} cells x {p.n_steps} steps, N={n}", "precision": "fp32",
           "tile_steps": Teff, "tile_cells": cells,
           "tile_choice": "autotuned (MBS_SOLVE_AUTOTUNE)" if T == 0 else "fixed"}
    hb = {"bound": "hbm", "achieved": round(state_bytes(n) * value, 1), "peak": hbm, "unit": "GB/s",
          "frac": round(state_bytes(n) * value / hbm, 4), "alg_bytes_per_cell_step": state_bytes(n),
          "peak_source": "measured" if pk.get("hbm_gbs") else "fallback", "launch_ms": round(per_launch * 1e3, 5),
          "kernel": (f"k_tiled_tc<{n},{cells // 128}>" if n >= 4 else f"k_tiled<fp32,N={n}>") + f" T={Teff}"}
    prof = load_profile(f"{name}_fp32_T{Teff}" + ("" if n < 4 or cells == 128 else f"_C{cells}"))
    hb["traffic"] = prof.get("dram_bytes") if prof else None
    cp = compute_peaks()
    out["roofline"] = issue_roof(prof, per_launch, clocks, cp, hb)
    if n >= 4:
        # the propagator apply on the tensor cores: 2 K^2 useful flops per
        # cell-step; the 3xTF32 MMAs execute 3 x 2 x NO x KA per computed cell
        sh = (n - 1) & 1
        ka = (K + 1 + 7) // 8 * 8
        no = (K + sh + 1 + 15) // 16 * 16
        own = cells - 2 * Teff
        mhz = clocks.get("sm_mhz") or 2070.0
        tfm = cp.get("tf32_mma", {}).get("flops_per_cycle_per_sm")
        if tfm:
            tf32 = tfm * 152 * mhz * 1e6 / 1e12
            src = "measured (tcgen05 kind::tf32 microbenchmark, profiles/compute_peaks.json) x sampled clock"
        else:
            bf16 = pk.get("bf16_tflops")
            tf32 = (bf16 or 1900.0) * 1.1 / 2.25
            src = "bf16 x nominal tf32/bf16 (1.1/2.25)"
        exec_tf = 3 * 2 * no * ka * value * 1e9 * cells / own / 1e12
        out["tensor"] = {"bound": "tensor", "achieved": round(exec_tf, 1), "peak": round(tf32, 1),
                         "unit": "TFLOP/s", "frac": round(exec_tf / tf32, 4),
                         "useful_tflops": round(2 * K * K * value * 1e9 / 1e12, 2), "peak_source": src,
                         "kernel": f"k_tiled_tc<{n},{cells // 128}> (tcgen05 kind::tf32, 3xTF32, M=128 N={no} K={ka})"}
    if parity:
        out["parity"] = fp32_vs_fp64(mbs, stream, torch, p, sc, "plain")
    q = p.replace(n_steps=fp64_steps)
    dq = mbs.device_from_problem(q)
    sq = mbs.scenario_from_problem(dq, q)
    for prec in ("fp32", "fp64"):
        tq = timed(sq, prec, "plain", 0)
        out[f"{prec}_plain"] = round(q.n_cells * q.n_steps / tq / 1e9, 3)
    out["plain_sample"] = f"first {fp64_steps} steps"
    out["speedup_vs_fp64_plain"] = round(value / out["fp64_plain"], 1)
    return out


def n_scaling_leg(mbs, stream, torch, n_cells=524_288, n_steps=10_000, fp64_steps=500):
    """Throughput against the number of levels: the anharmonic ladder of the
    paper's six-level example (Gaussian source) for N = 2..6 on 524,288 cells
    x 10,000 steps; FP32 with autotuned tiles (CUDA-core tiles for N = 2, 3,
    tensor-core tiles for N >= 4) and the FP64 plain path on its first 500
    steps."""
    out = {}
    for n in range(2, 7):
        p = W.ladder_anharmonic(n, n_cells=n_cells, n_steps=n_steps)
        dev = mbs.device_from_problem(p)
        sc = mbs.scenario_from_problem(dev, p)
        mbs.mbs_solve([sc], "fp32", "tiled", stream=stream.cuda_stream, autotune=True)   # tunes
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mbs.mbs_solve([sc], "fp32", "tiled", stream=stream.cuda_stream, autotune=True)
        b.record(stream)
        torch.cuda.synchronize()
        v32 = n_cells * n_steps / (a.elapsed_time(b) / 1e3) / 1e9
        q = p.replace(n_steps=fp64_steps)
        dq = mbs.device_from_problem(q)
        sq = mbs.scenario_from_problem(dq, q)
        mbs.mbs_solve([sq], "fp64", "plain", stream=stream.cuda_stream)
        torch.cuda.synchronize()
        a.record(stream)
        mbs.mbs_solve([sq], "fp64", "plain", stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        v64 = n_cells * fp64_steps / (a.elapsed_time(b) / 1e3) / 1e9
        out[f"N={n}"] = {"fp32": round(v32, 2), "fp64_plain": round(v64, 3), "tile_steps": mbs.mbs_scenario_tile(sc),
                         "kernel": "tensor-core tiles" if n >= 4 else "CUDA-core tiles"}
    return {"unit": METRIC, "workload": f"ladder_anharmonic: {n_cells} cells x {n_steps} steps, N = 2..6, "
                                        "Gaussian source", "by_levels": out}


def cells_leg(mbs, stream, torch, clocks, n_sys=131_072, n_steps=10_000, every=100, reps=2):
    """Driven single cells (Nx = 1, the master equation alone): the V-type
    three-level example as a batch of 131,072 systems (parameters +-10 %,
    drive amplitude swept over 0.25..2 e0) x 10,000 steps over 80 fs, one
    thread per system, populations recorded every 100 steps; FP32 and FP64;
    the oracle's driven-cell solver timed on 32 of the systems."""
    b = W.song_vtype(n_sys=n_sys, n_steps=n_steps, record_every=every)
    c = mbs.cells_from_batch(b)
    out = {}
    for prec in ("fp32", "fp64"):
        mbs.mbs_cells_solve(c, prec, stream=stream.cuda_stream)    # warm-up (allocates)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mbs.mbs_cells_solve(c, prec, stream=stream.cuda_stream)
            e.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(e) / 1e3
            best = t if best is None else min(best, t)
        out[prec] = n_sys * n_steps / best / 1e9
    K = 8
    flops = 2 * K * K + 6 * 3 + 4 * K           # propagator apply, rotations, compensated adds
    mhz = clocks.get("sm_mhz") or 2070.0
    fma = compute_peaks().get("fp32_fma", {}).get("flops_per_cycle_per_sm")
    if fma:
        peak = fma * 152 * mhz / 1e6
        psrc = "measured (FP32 FMA microbenchmark, profiles/compute_peaks.json) x sampled clock"
    else:
        peak = 2 * 128 * 152 * mhz / 1e6         # FP32 FMA lanes x 2 flops x SMs x clock [TFLOP/s]
        psrc = "nominal FP32 FMA rate of 152 SMs x 128 lanes at the sampled SM clock"
    ach = flops * out["fp32"] * 1e9 / 1e12
    res = {"value": round(out["fp32"], 2), "unit": METRIC, "fp64": round(out["fp64"], 2),
           "workload": f"song_vtype: {n_sys} driven three-level systems x {n_steps} steps (Nx = 1)",
           "roofline": {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                        "frac": round(ach / peak, 4), "alg_flops_per_cell_step": flops,
                        "peak_source": psrc}}
    try:
        import oracle
        import time as _t
        t0 = _t.perf_counter()
        m = 32
        for s in range(m):
            oracle.cell_evolve(b.qms[s], b.dt, W.cell_field(b.drives[s], b.dt, n_steps))
        res["cpu_oracle"] = {"value": round(m * n_steps / (_t.perf_counter() - t0) / 1e9, 5), "cores": 1,
                             "sample": f"{m} systems x {n_steps} steps, one at a time on one core"}
    except Exception as ex:   # the oracle is optional here
        res["cpu_oracle"] = {"unavailable": str(ex)[:80]}
    return res


def batch_leg(mbs, stream, torch, precision):
    """The 512-simulation mixed batch (two- and three-level media, 1,024 to
    65,536 cells, 20,000 to 100,000 steps).  FP32: one batched solve with
    autotuned tile depths, recorded as a CUDA graph on the warm-up call and
    replayed on the timed call, against the same scenarios solved one after
    another (library default depths).  FP64: one batched solve (default
    depths, a single timed call)."""
    ps = W.batch_mixed()
    devs = [mbs.device_from_problem(p) for p in ps]
    scs = [mbs.scenario_from_problem(d, p) for d, p in zip(devs, ps)]
    cell_steps = sum(p.n_cells * p.n_steps for p in ps)

    def timed(**kw):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mbs.mbs_solve(scs, stream=stream.cuda_stream, **kw)
        b.record(stream)
        torch.cuda.synchronize()
        return cell_steps / (a.elapsed_time(b) / 1e3) / 1e9

    kw32 = dict(precision="fp32", algo="tiled", autotune=True, graph=True)
    timed(**kw32)                                                       # tunes, records the graph
    batched = timed(**kw32)                                             # replays it
    tiles = sorted({(p.qms[0].n_levels, mbs.mbs_scenario_tile(sc)) for p, sc in zip(ps, scs)})
    one = timed(precision="fp32", algo="tiled", one_at_a_time=True)
    # FP64 and FP32 batched on the first 64 simulations (a bounded sample)
    sub, sub_ps = scs[:64], ps[:64]
    sub_cs = sum(p.n_cells * p.n_steps for p in sub_ps)
    rate, recs = {}, {}
    for prec in ("fp64", "fp32"):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mbs.mbs_solve(sub, prec, "tiled", stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        rate[prec] = sub_cs / (a.elapsed_time(b) / 1e3) / 1e9
        recs[prec] = [fetch_all(mbs, sc, len(q.probes)) for sc, q in zip(sub, sub_ps)]
    errs = [trace_errors(x, y, q.probes) for x, y, q in zip(recs["fp32"], recs["fp64"], sub_ps)]
    worst = max(range(len(errs)), key=lambda i: errs[i][0])
    parity = {"fp32_vs_fp64_worst_trace": float(f"{errs[worst][0]:.3e}"), "worst_simulation": worst,
              "fp32_vs_fp64_worst_population_deviation": float(f"{max(e[1] for e in errs):.3e}"),
              "simulations": len(sub_ps), "sample": "first 64 simulations, full length, batched FP32 vs batched FP64"}
    n2 = sum(1 for p in ps if p.qms[0].n_levels == 2)
    return {"value": round(batched, 2), "one_at_a_time": round(one, 2), "speedup": round(batched / one, 2),
            "fp64_batched": {"value": round(rate["fp64"], 2), "fp32_same_sample": round(rate["fp32"], 2),
                             "sample": f"first 64 simulations, {sub_cs:.3e} cell-steps, default tile depths"},
            "unit": METRIC,
            "workload": f"{len(ps)} simulations ({n2} two-level, {len(ps) - n2} three-level), "
                        f"{cell_steps:.3e} cell-steps", "precision": precision,
            "tile_steps": {f"N={n}": t for n, t in tiles}, "launch": "CUDA graph replay (MBS_SOLVE_GRAPH)",
            "parity": parity}


def fp64_plain(p, mbs, stream, torch, steps=4000):
    """The plain FP64 form (one thread per cell, two launches per step) on
    the first `steps` steps of the same workload."""
    q = p.replace(n_steps=steps)
    dev = mbs.device_from_problem(q)
    sc = mbs.scenario_from_problem(dev, q)
    res = {}
    for algo in ("plain", "tiled"):
        mbs.mbs_solve([sc], "fp64", algo, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mbs.mbs_solve([sc], "fp64", algo, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        res[algo] = round(q.n_cells * steps / (a.elapsed_time(b) / 1e3) / 1e9, 3)
    return {"value": res["plain"], "fp64_tiled": res["tiled"], "unit": METRIC,
            "sample": f"first {steps} steps of the workload"}


def e2e(p, mbs, args, torch, stream, reps=2):
    """End to end through the public API with host buffers: device and
    scenario creation (host FP64 setup + host->device copies), the solve, and
    the device->host read of every probe trace, per step."""
    times, h2d, d2h = [], 0, 0
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dev = mbs.device_from_problem(p)
        sc = mbs.scenario_from_problem(dev, p)
        mbs.mbs_solve([sc], args.precision, "tiled", tile_steps=args.tile, stream=stream.cuda_stream)
        recs = [mbs.mbs_fetch_records(sc, k) for k in range(len(p.probes))]
        times.append(time.perf_counter() - t0)
        c = mbs.mbs_scenario_counters(sc)
        h2d, d2h = c["h2d_bytes"], c["d2h_bytes"]
        assert all(np.all(np.isfinite(r)) for r in recs)
        sc.close()
        dev.close()
    t = min(times)
    return {"value": round(p.n_cells * p.n_steps / t / 1e9, 3), "unit": METRIC,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "seconds_per_step": round(t, 3)}


def load_profile(key):
    """ncu figures per launch of a kernel (DRAM bytes, warp instructions)
    from the committed summary profiles/traffic.json, or None when no
    capture exists for `key` or its kernel sources changed after the capture
    (each entry records a hash of the sources it measured)."""
    import hashlib
    f = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(f))
        e = d[key]
        h = hashlib.sha256()
        for name in e["sources"]:
            h.update(open(os.path.join(ROOT, name), "rb").read())
        if h.hexdigest()[:16] != e["kernel_source_sha256_16"]:
            return None
        return e
    except Exception:
        return None


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    p = workload(args.workload)
    import oracle
    oracle.build()
    vals = []
    for k in range(args.warmup + args.steps):
        r = time_oracle(p, target_s=6.0, cells=32_768)
        if k >= args.warmup:
            vals.append(r)
    value = float(np.mean([v["value"] for v in vals]))
    secs = sum(v["seconds"] for v in vals)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": METRIC, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded)",
           "config": {"workload": workload_label(p), "precision": "fp64", "algo": "oracle (CPU, OpenMP over cells)"},
           "cpu_baseline": {"value": round(value, 5), "unit": METRIC, "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": round(value, 5), "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sit_2lvl_jitter")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tile", type=int, default=32)
    ap.add_argument("--quick", action="store_true", help="skip the FP64, e2e and CPU legs")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-simulation batch leg")
    ap.add_argument("--nsteps", type=int, default=0, help="override the workload's step count (profiling)")
    ap.add_argument("--wide-tiles", action="store_true",
                    help="256-cell tensor-core tiles for the main workload (N >= 4; profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
