"""Measure the GPU's arithmetic peaks (FP32 FMA, FP64 FMA, TF32 tensor-core
MMA) with the library's microbenchmarks (mbs_peak_rates) and write them, per
SM clock cycle and at the sampled clock, to a JSON file:

    python -m paper_2005_05412_gb300.peaks --out profiles/compute_peaks.json

The per-cycle figures let a roofline scale the peak to the clock sampled
while the measured kernel ran.  nvidia-smi is only queried (clocks and
throttle reasons), never used to change a setting.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading

import numpy as np

NAMES = {0: "fp32_fma", 1: "fp64_fma", 2: "tf32_mma"}


class _Clocks:
    Q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"

    def __init__(self, gpu):
        self.gpu, self.lines, self.proc = gpu, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=lambda: [self.lines.append(x) for x in self.proc.stdout], daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def median_mhz(self):
        v = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            try:
                v.append(float(f[0]))
            except (ValueError, IndexError):
                pass
        return float(np.median(v)) if v else None


def measure(reps: int = 5):
    import torch

    import paper_2005_05412_gb300 as mbs
    torch.cuda.init()
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    out = {"device": props.name, "sms": props.multi_processor_count, "kernels": "csrc/mbs_peaks.cu"}
    for which, name in NAMES.items():
        rates, mhz = [], []
        for _ in range(reps):
            with _Clocks(dev) as clk:
                r, _t = mbs.mbs_peak_rates(which)
            rates.append(r)
            mhz.append(clk.median_mhz())
        best = max(rates)
        m = [x for x in mhz if x] or [None]
        clock = float(np.median(m)) if m[0] else None
        e = {"tflops": round(best / 1e12, 3), "sm_mhz": clock}
        if clock:
            e["flops_per_cycle_per_sm"] = round(best / (clock * 1e6) / props.multi_processor_count, 2)
        out[name] = e
    f32 = out["fp32_fma"]
    if f32.get("flops_per_cycle_per_sm"):
        # one FP32 FMA warp instruction = 64 flops; the FMA lanes issue one
        # warp instruction per scheduler and clock
        out["issue_warp_inst_per_cycle_per_sm"] = round(f32["flops_per_cycle_per_sm"] / 64.0, 3)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = measure()
    text = json.dumps(res, indent=1)
    print(text)
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as f:
            f.write(text + "\n")


if __name__ == "__main__":
    sys.exit(main())
