#!/usr/bin/env python
"""Throughput of the multi-scale blob-detection filter bank on GB300.

Workload: one 4096 x 4096 FP32 synthetic frame (1/f background, 500 bright and
dark elliptical blobs), 6 scales (blob radii 2, 4, 8, 16, 32, 48 px).  One
step = the fourth-order repeated-pole IIR bank (Filter D) and the colored
Savitzky-Golay FIR bank (Filter C, <= 193 taps), each followed by the
3 x 3 x 6 scale-space extremum detector and the read-back of its blob list.
Metric: Mpixel-scales/s = banks x pixels x scales / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel-scales/s blob detection (IIR & FIR), gated vs plain on 1 GB300; % HBM peak"
UNIT = "Mpixel-scales/s"
SCALES = [2.0, 4.0, 8.0, 16.0, 32.0, 48.0]
H = W = 4096
THRESHOLD = 0.05
BANKS = (("iir_repeated_pole_order4", 0, 4), ("fir_colored_sg", 2, 1))
WORKLOAD = ("4096x4096 FP32 frame, 6 scales (lambda 2-48 px): 4th-order repeated-pole IIR bank "
            "+ colored Savitzky-Golay FIR bank (K<=96), Laplacian response, 3x3x6 extremum, "
            "blob lists read back")
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ---------------------------------------------------------------------------
# algorithmic work per kernel launch (one frame, all scales)
# ---------------------------------------------------------------------------
def fir_taps(scales, kmax=96):
    import math
    return [min(math.ceil(5 * s / 2), kmax) for s in scales]


def algorithmic(name, S, HW, taps):
    """(bytes, flops) a kernel must move / compute per launch."""
    fb = 4.0
    if name in ("iir_row", "fir_row"):
        byts = fb * HW + fb * S * HW                 # read frame, write S planes
    elif name in ("iir_colseg", "iir_coldet", "fir_coldet"):
        byts = fb * S * HW                           # read S planes
    else:
        byts = 0.0
    flops = 0.0
    if name in ("fir_row", "fir_coldet"):           # 2K+1 multiply-adds per output
        flops = sum(2.0 * (2 * k + 1) for k in taps) * HW
    return byts, flops


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1912_07133_gb300 import kf, synthetic

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build() if rank == 0 or world == 1 else None
    if world > 1:
        dist.barrier()
    kf.load()
    dev = torch.device("cuda", local)
    img = synthetic.iir_fir_frame(seed=1, H=H, W=W)
    X = torch.from_numpy(img).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    bank = kf.Bank(local, stream.cuda_stream)

    # one-time designs (FP64 kernel), timed separately: the bank reuses them
    t0 = time.perf_counter()
    for _, ft, order in BANKS:
        for s in SCALES:
            kf.kf_design(ft, order, s)
    design_ms = (time.perf_counter() - t0) * 1e3

    def step(profile):
        n, times = 0, {}
        for _, ft, order in BANKS:
            bank.run([X], SCALES, ft, order, threshold=THRESHOLD, profile=profile)
            n += len(bank.blobs())
            if profile:
                for k, (nl, ms) in bank.kernel_times().items():
                    a, b = times.get(k, (0, 0.0))
                    times[k] = (a + nl, b + ms)
        return n, times

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(False)

    def timed(profile):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        kt, nb = {}, 0
        barrier()
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()
                ev[i][0].record(stream)
                nb, times = step(profile)
                ev[i][1].record(stream)
                for k, (nl, ms) in times.items():
                    a, b = kt.get(k, (0, 0.0))
                    kt[k] = (a + nl, b + ms)
            barrier()
        return sum(a.elapsed_time(b) for a, b in ev), kt, nb, clk.summary()

    # --- device-resident timed region (no profiling events) ------------------
    total_ms, _, nblobs, clocks = timed(False)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    pix_scales = len(BANKS) * H * W * len(SCALES)
    value = world * pix_scales / (ms_per_step * 1e-3) / 1e6
    # --- the same steps again with CUDA events around every kernel ------------
    _, ktimes, _, _ = timed(True)

    # --- end to end: host frame in pinned memory, copies inside the timed region
    host = torch.from_numpy(img).pin_memory()
    Xe = torch.empty_like(X)
    e2e_ms, bo = [], 0
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Xe.copy_(host, non_blocking=True)
        nb = 0
        for _, ft, order in BANKS:
            bank.run([Xe], SCALES, ft, order, threshold=THRESHOLD)
            nb += len(bank.blobs())
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
            bo = nb * np.dtype(kf.BLOB_DTYPE).itemsize
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_step = float(t.item())
    e2e = {"value": world * pix_scales / (e2e_step * 1e-3) / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(img.nbytes), "d2h_bytes_per_step": int(bo),
           "ms_per_step": e2e_step}

    # --- roofline of the dominant kernel -------------------------------------
    hbm, hbm_src = peaks()
    alu_peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12  # TFLOP/s
    taps = fir_taps(SCALES)
    kern = {}
    for k, (nl, ms) in ktimes.items():
        per = ms / max(nl, 1)
        byts, flops = algorithmic(k, len(SCALES), H * W, taps)
        kern[k] = {"launches": nl, "ms_per_launch": round(per, 4),
                   "share": round(ms / max(sum(v[1] for v in ktimes.values()), 1e-9), 4)}
        if byts:
            kern[k]["GB_s"] = round(byts / (per * 1e-3) / 1e9, 1)
        if flops:
            kern[k]["TFLOP_s"] = round(flops / (per * 1e-3) / 1e12, 2)
    dom = max(ktimes, key=lambda k: ktimes[k][1])
    nl, ms = ktimes[dom]
    per = ms / nl
    byts, flops = algorithmic(dom, len(SCALES), H * W, taps)
    if flops:
        ach = flops / (per * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 1),
                "unit": "TFLOP/s", "frac": round(ach / alu_peak, 4), "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    else:
        ach = byts / (per * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": None, "peak_source": hbm_src}
    launches = sum(v[0] for v in ktimes.values())
    bank.close()

    cpu = cpu_baseline(img) if (rank == 0 and not args.no_cpu) else None
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frame": f"{H}x{W} f32", "scales_px": SCALES,
                   "banks": [b[0] for b in BANKS], "threshold": THRESHOLD,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}", "designs": "FP64 design kernel run once "
                   "per bank configuration, timed separately (design_ms)"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "kernels": kern, "blobs_per_step": nblobs,
        "design_ms": round(design_ms, 2),
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(img, rows=None):
    """The FP64 oracle as it stands, on the host cores, on `rows` rows of the
    frame (all 6 scales, both banks); designs are made before timing."""
    import numpy as np

    from oracle import oracle as O

    sub = img if rows is None else img[:rows]
    x = sub.astype(np.float64)
    for l in SCALES:  # designs (cached), excluded like the GPU designs
        O.design_colored_sg_mp(1, O.sg_half_length(1, l / 2, 96), 6.0 / l)
    t0 = time.perf_counter()
    for _, ft, order in BANKS:
        R = O.bank(x, SCALES, {0: O.IIR_REPEATED_POLE, 2: O.FIR_COLORED_SG}[ft], order)
        O.detect(R, THRESHOLD)
    dt = time.perf_counter() - t0
    ps = len(BANKS) * sub.shape[0] * sub.shape[1] * len(SCALES)
    return {"value": round(ps / dt / 1e6, 3), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{sub.shape[0]}x{sub.shape[1]} rows of the frame, 6 scales, both banks "
                      f"({dt:.2f} s)"}


# ---------------------------------------------------------------------------
# reference arm: the oracle timed as a program
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as O
    from paper_1912_07133_gb300 import synthetic

    O.build()
    img = synthetic.iir_fir_frame(seed=1, H=H, W=W)
    rows = 256  # bounded sample per step: 256 x 4096 x 6 scales x 2 banks
    x = img[:rows].astype(np.float64)
    for l in SCALES:
        O.design_colored_sg_mp(1, O.sg_half_length(1, l / 2, 96), 6.0 / l)

    def step():
        for _, ft, order in BANKS:
            R = O.bank(x, SCALES, {0: O.IIR_REPEATED_POLE, 2: O.FIR_COLORED_SG}[ft], order)
            O.detect(R, THRESHOLD)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    ps = len(BANKS) * rows * W * len(SCALES)
    v = ps / dt / 1e6
    sample = f"{rows}x{W} rows of the 4096x4096 frame per step, 6 scales, both banks"
    line = {"metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "kind": "oracle", "cores": O.threads(),
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
