#!/usr/bin/env python
"""Throughput of the multi-scale blob-detection filter bank on GB300.

Default workload (iir_fir): one 4096 x 4096 FP32 synthetic frame (1/f
background, 500 bright and dark elliptical blobs), 6 scales (blob radii 2, 4,
8, 16, 32, 48 px).  One step = the fourth-order repeated-pole IIR bank
(Filter D) and the colored Savitzky-Golay FIR bank (Filter C, <= 193 taps),
each followed by the 3 x 3 x 6 scale-space extremum detector and the
read-back of its blob list.

--workload batch: 64 FP32 frames of uneven sizes (about 574 Mpx), 8 scales,
Filter D order 4 and the Butterworth bank, all frames in one call; the line
adds the same steps launched frame by frame (per_frame_schedule).

--workload gated: 120 clustered 6144^2 FP16 frames (blob clusters in ~5% of
the 64x64 tiles), 8 scales, both banks at threshold 0.3, gated by the trained
proposal network against the plain bank (recall judged in the same run).

--workload quartic: the D = 5 derivative bank (all 15 D_{dx,dy}, dx + dy <= 4)
of one 2048 x 2048 FP32 frame at 4 scales, Filter D with L_D = 2.

--workload counts: 16 uint16 frames of 8192 x 8192 (12-bit Poisson counts on a
1/f background, 2000 blobs of radii 2-64 px; one generated frame in 16 device
buffers), value scale 1/4095, 8 scales (radii 2-64 px), Filter D order 4 and
Filter C with K <= 160, one-sided planes stored as --storage (default f16).

Metric: Mpixel-scales/s = banks x frames x pixels x scales / step time.

The default run (--workload iir_fir) prints one line for the 4096^2 workload
and adds, measured after its own timed region with --sub-steps steps each,
the sub-objects "gated" (gated vs plain on the clustered workload, recall),
"batch" and "counts" (the workloads above); --only leaves them out.  Every
line reports the HBM fraction of the algorithmic bytes per bank and per step
("hbm") and the roofline of the dominant kernel ("roofline").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload iir_fir|counts|batch|gated|table5|quartic]
                  [--storage f32|f16|bf16] [--no-graph] [--no-tune] [--only]
                  [--sub-steps K2] [--gate-mode tiles|dilated]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel-scales/s blob detection (IIR & FIR), gated vs plain on 1 GB300; % HBM peak"
UNIT = "Mpixel-scales/s"
THRESHOLD = 0.05
IIR_FIR = (("iir_repeated_pole_order4", 0, 4), ("fir_colored_sg", 2, 1))
IIR_BW = (("iir_repeated_pole_order4", 0, 4), ("iir_butterworth_order2", 1, 2))
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
SB = {"f32": 4, "f16": 2, "bf16": 2}
EIGHT = [2.0 * 32.0 ** (s / 7.0) for s in range(8)]
WORKLOADS = {
    "iir_fir": dict(
        frames=1, dtype="f32", s_in=4, value_scale=1.0, fir_kmax=96, storage="f32", banks=IIR_FIR,
        scales=[2.0, 4.0, 8.0, 16.0, 32.0, 48.0], ref_rows=256,
        text=("4096x4096 FP32 frame, 6 scales (lambda 2-48 px): 4th-order repeated-pole IIR bank "
              "+ colored Savitzky-Golay FIR bank (K<=96), Laplacian response, 3x3x6 extremum, "
              "blob lists read back")),
    "counts": dict(
        frames=16, dtype="u16", s_in=2, value_scale=1.0 / 4095.0, fir_kmax=160, storage="f16", banks=IIR_FIR,
        scales=EIGHT, ref_rows=32,
        text=("16 x 8192x8192 uint16 12-bit Poisson-count frames (one generated frame in 16 device "
              "buffers), value scale 1/4095, 8 scales (lambda 2-64 px): 4th-order repeated-pole IIR "
              "bank + colored Savitzky-Golay FIR bank (K<=160), Laplacian response, 3x3x8 extremum, "
              "blob lists read back")),
    "batch": dict(
        frames=64, dtype="f32", s_in=4, value_scale=1.0, fir_kmax=96, storage="f32", banks=IIR_BW,
        scales=EIGHT, ref_rows=64,
        text=("64 FP32 frames of uneven sizes drawn from {1024x768, 1920x1080, 2048x2048, 4096x3072, "
              "6144x4096} (uniform background, 20 blobs per 512^2), 8 scales (lambda 2-64 px): 4th-order "
              "repeated-pole IIR bank + Butterworth bank (L_B = 4), Laplacian response, 3x3x8 extremum, "
              "blob lists read back; all frames in one call")),
}
FP32_LANES = 128  # FP32 lanes per SM (Blackwell)
GATED_THRESHOLD = 0.3  # clustered frames: the 1/f background alone stays below it
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel, from one
# ncu capture (summaries in profiles/), keyed by (workload, kernel, storage):
# (bytes, digest of the kernel sources the capture ran).  A figure is reported
# only while the sources still have that digest; otherwise traffic is null.
MEASURED_TRAFFIC = {
    ("iir_fir", "fir_row", "f32"): (410.3e6, "bc30a23c87b096b4"),     # k_rowfir: 67.29 read + 342.98 written
    ("iir_fir", "fir_coldet", "f32"): (431.4e6, "bc30a23c87b096b4"),  # k_colfir_tc: 423.76 + 7.65
    ("iir_fir", "iir_row", "f32"): (406.0e6, "bc30a23c87b096b4"),     # k_row: 67.28 + 338.72
}
CSRC = os.path.join(ROOT, "paper_1912_07133_gb300", "csrc")


_COMMENT_OR_LITERAL = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'', re.S)


def code_only(text):
    """C++/CUDA source without its comments (string and character literals
    kept), whitespace runs collapsed: what the compiler sees of it."""
    text = _COMMENT_OR_LITERAL.sub(lambda m: " " if m.group(0).startswith("/") else m.group(0), text)
    return " ".join(text.split())


def csrc_digest():
    """sha256 (first 16 hex digits) over the CUDA sources of the library
    without their comments, in name order: changes whenever any kernel's code
    changes, not when only a comment does."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            with open(os.path.join(CSRC, name), encoding="utf-8") as f:
                h.update(code_only(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_of(workload, kernel, storage):
    """Measured DRAM bytes per launch of `kernel`, or None when there is no
    capture of the current sources."""
    t = MEASURED_TRAFFIC.get((workload, kernel, storage))
    if t is None or t[1] != csrc_digest():
        return None
    return t[0]


def make_frames(wl):
    """Host frames of the workload (the counts workload: one frame, used by
    every device buffer)."""
    from paper_1912_07133_gb300 import synthetic
    if wl["dtype"] == "u16":
        return [synthetic.counts_frame(seed=3, H=8192, W=8192)]
    if wl["frames"] == 1:
        return [synthetic.iir_fir_frame(seed=1, H=4096, W=4096)]
    return synthetic.batch_frames(seed=2, nframes=wl["frames"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# nominal dense tensor rates (PFLOP/s): TF32 1.1, bf16 2.25
TF32_PER_BF16 = 1.1 / 2.25
# kernels whose contraction runs on the tensor cores as three TF32 products
# per FP32-accurate product (hi x hi, hi x lo, lo x hi)
TENSOR_3XTF32 = ("fir_coldet",)


def tf32_peak():
    """TF32 dense peak (TFLOP/s): the measured sustained bf16 GEMM rate (the
    kernel is timed inside a long step) times the nominal TF32/bf16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["bf16_tflops_sustained"]) * TF32_PER_BF16, "measured bf16 sustained x nominal TF32/bf16"
    except Exception:
        return 1700.0 * TF32_PER_BF16, "fallback bf16 sustained x nominal TF32/bf16"


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device):
    """x of the slowest rank (every rank gets it): the step time of a job of
    independent replicas is the time of the last one to finish."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput in millions of units per second: the units all
    ranks processed (each replica the same workload) over the slowest rank's
    step time."""
    return world * units_per_rank / (ms_per_step * 1e-3) / 1e6


# ---------------------------------------------------------------------------
# algorithmic work per kernel launch (one frame, all scales)
# ---------------------------------------------------------------------------
def fir_taps(scales, kmax=96):
    import math
    return [min(math.ceil(5 * s / 2), kmax) for s in scales]


def algorithmic(name, S, HW, taps, s_in=4.0, s_b=4.0):
    """(bytes, flops) a kernel must move / compute per launch (one frame):
    s_in bytes per input pixel, s_b per stored plane element."""
    if name in ("iir_row", "fir_row"):
        byts = s_in * HW + s_b * S * HW              # read frame, write S planes
    elif name in ("iir_colseg", "iir_coldet", "iir_colscan", "fir_coldet"):
        byts = s_b * S * HW                          # read S planes
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
# device facts and peaks
# ---------------------------------------------------------------------------
def sm_max_mhz(clocks=None):
    """Maximum SM clock: the measured-peaks file's record, else the sampled
    clocks.max.sm, else the GB300 nominal 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        pass
    if clocks and clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"])
    return 2070.0


def alu_peak(nsm, mhz):
    """FP32 ALU peak (TFLOP/s): SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return nsm * FP32_LANES * 2 * mhz * 1e6 / 1e12


def bank_bytes(S, pixels, s_in, s_b):
    """Algorithmic bytes of one bank over `pixels` frame pixels at S scales:
    the two-pass design reads the frame once, writes and reads back S planes
    (2 s_b + s_in / S per pixel-scale)."""
    return pixels * (s_in + 2.0 * s_b * S)


def roofline_of(kernel, ms_total, launches, byts, flops, hbm, hbm_src, nsm, mhz, traffic):
    """Roofline record of one kernel: its algorithmic work per launch over its
    average event-timed launch duration against the bound that applies.  A
    FIR pass's work is the method's 2(2K + 1) flop per output and scale,
    counted once (the tensor-core pass spends three TF32 products on each to
    keep FP32 accuracy; that factor is reported, not counted as work)."""
    per = ms_total / max(launches, 1) * 1e-3  # s per launch
    rec = {"kernel": kernel, "launches": launches, "ms_per_launch": round(per * 1e3, 4)}
    if flops:
        ach = flops / launches / per / 1e12
        if kernel in TENSOR_3XTF32:
            tp, tsrc = tf32_peak()
            rec.update(bound="tensor", achieved=round(ach, 3), peak=round(tp, 1), unit="TFLOP/s",
                       frac=round(ach / tp, 4), peak_source=tsrc, tf32_products_per_tap=3,
                       work="2(2K+1) flop per output and scale (method work, counted once)")
        else:
            pk = alu_peak(nsm, mhz)
            rec.update(bound="alu", achieved=round(ach, 3), peak=round(pk, 1), unit="TFLOP/s",
                       frac=round(ach / pk, 4),
                       peak_source=f"derived: {nsm} SMs x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz",
                       work="2(2K+1) flop per output and scale")
        if byts:
            rec["hbm_frac"] = round(byts / launches / per / 1e9 / hbm, 4)
    else:
        ach = byts / launches / per / 1e9
        rec.update(bound="hbm", achieved=round(ach, 1), peak=hbm, unit="GB/s", frac=round(ach / hbm, 4),
                   peak_source=hbm_src)
    rec["traffic"] = traffic
    rec["algorithmic_bytes_per_launch"] = round(byts / max(launches, 1))
    return rec


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def setup_device(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1912_07133_gb300 import kf

    rank, world, local = dist_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build() if rank == 0 or world == 1 else None
    if world > 1:
        dist.barrier()
    kf.load()
    return rank, world, local


PASS_NAMES = ("row", "seg", "fold", "det")


def shape_overrides(spec, bank_name):
    """(pass, grid_mult) pairs of `spec` ("iir.row=-2,fir.row=-3": bank name
    prefix before the first '_', pass name, kf_set_launch_shape value) that
    apply to the bank `bank_name`."""
    out = []
    for part in filter(None, (spec or "").split(",")):
        key, val = part.split("=")
        bank, pname = key.strip().split(".")
        if pname not in PASS_NAMES:
            raise ValueError(f"--shape: unknown pass {pname!r} (one of {PASS_NAMES})")
        if bank_name.split("_")[0] == bank:
            out.append((pname, int(val)))
    return out


def measure_workload(args, name, steps, warmup, full=True):
    """Steps of one workload of WORKLOADS on this rank's GPU.  full: also the
    serial and frame-by-frame schedules, end to end and the profiled pass's
    per-kernel roofline (the sub-workloads of the default run take the device
    timing, the per-bank HBM fractions and the kernel list only)."""
    import numpy as np
    import torch

    from paper_1912_07133_gb300 import kf

    rank, world, local = dist_info()
    wl = WORKLOADS[name]
    storage = (args.storage if name == args.workload else None) or wl["storage"]
    NF, SCALES, BANKS = wl["frames"], wl["scales"], wl["banks"]
    graph = not args.no_graph
    dev = torch.device("cuda", local)
    host = make_frames(wl)
    u16 = host[0].dtype == np.uint16
    as_t = (lambda a: torch.from_numpy(a.view(np.int16))) if u16 else torch.from_numpy
    dview = (lambda t: t.view(torch.uint16)) if u16 else (lambda t: t)
    # device frames (inputs resident in HBM for the device-timed value)
    if len(host) == NF:
        X = [as_t(h).to(dev) for h in host]
        src = list(range(NF))
    else:  # one generated frame in NF device buffers
        X = [as_t(host[0]).to(dev) for _ in range(NF)]
        src = [0] * NF
    Xs = [dview(x) for x in X]
    pixels = sum(host[i].size for i in src)
    vscales = [wl["value_scale"]] * NF
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    # one library context per bank, each on its own stream: the banks of a
    # step are independent passes over the same frames and run at once
    bstreams = {bn: torch.cuda.Stream(dev) for bn, _, _ in BANKS}
    banks = {bn: kf.Bank(local, bstreams[bn].cuda_stream) for bn, _, _ in BANKS}
    if args.column_pass:  # a fixed column pass for the recursive banks (the autotuner may change it)
        mode = {"segments": kf.KF_COLUMN_SEGMENTS, "single-read": kf.KF_COLUMN_SINGLE_READ}[args.column_pass]
        for bn, ft, _ in BANKS:
            if ft in (kf.KF_IIR_REPEATED_POLE, kf.KF_IIR_BUTTERWORTH):
                kf.kf_set_column_pass(banks[bn].ctx, ft, mode)
    concurrent = len(BANKS) > 1 and not args.serial

    # one-time designs (FP64 kernel), timed separately: the bank reuses them
    t0 = time.perf_counter()
    for _, ft, order in BANKS:
        for s in SCALES:
            kf.kf_design(ft, order, s)
    design_ms = (time.perf_counter() - t0) * 1e3

    # launch shapes and segment lengths tuned once per bank on this workload
    tuned = {}
    if not args.no_tune:
        for bn, ft, order in BANKS:
            o = kf.kf_bank_opts_default()
            o.threshold = THRESHOLD
            o.fir_kmax = wl["fir_kmax"]
            o.storage = STORAGE[storage]
            shapes, lc, _ = kf.kf_autotune(banks[bn].ctx, Xs, SCALES, ft, order, o, vscales)
            tuned[bn] = {"grid_mult": {p: m for p, m in zip(("row", "seg", "fold", "det"), shapes) if m >= 0}}
            if lc > 0:
                tuned[bn]["column_pass"] = f"segments of {lc} rows"
            elif lc == 0:
                tuned[bn]["column_pass"] = "single read"
    # fixed launch shapes over the tuned ones (e.g. per-SM shares, so that the
    # banks' kernels share every SM)
    for bn, ft, _ in BANKS:
        for pname, m in shape_overrides(args.shape, bn):
            kf.kf_set_launch_shape(banks[bn].ctx, ft, PASS_NAMES.index(pname), m)
            tuned.setdefault(bn, {}).setdefault("grid_mult", {})[pname] = m

    def run_bank(bn, frames, ft, order, profile=False, schedule=kf.KF_SCHED_BATCHED, use_graph=graph):
        banks[bn].run(frames, SCALES, ft, order, threshold=THRESHOLD, profile=profile, fir_kmax=wl["fir_kmax"],
                      storage=STORAGE[storage], value_scales=vscales, schedule=schedule, graph=use_graph)

    def step(profile, schedule=kf.KF_SCHED_BATCHED, frames=None, serial=None):
        """One pass of every bank over the frames, blob lists read back.  The
        banks' streams start after the work already on `stream` and `stream`
        waits for them at the end.  Concurrent: all banks launched, then the
        lists read; serial (profiling, frame-by-frame launches): one bank after
        the other.  Returns (blobs, {bank: {kernel: (launches, ms)}})."""
        n, times = 0, {}
        frames = Xs if frames is None else frames
        use_graph = graph and not profile and schedule == kf.KF_SCHED_BATCHED
        serial = (profile or not concurrent or schedule != kf.KF_SCHED_BATCHED) if serial is None else serial
        for bn, _, _ in BANKS:
            bstreams[bn].wait_stream(stream)
        if serial:
            for bn, ft, order in BANKS:
                run_bank(bn, frames, ft, order, profile, schedule, use_graph)
                n += len(banks[bn].blobs())
                if profile:
                    times[bn] = banks[bn].kernel_times()
        else:
            for bn, ft, order in BANKS:
                run_bank(bn, frames, ft, order, profile, schedule, use_graph)
            for bn, _, _ in BANKS:
                n += len(banks[bn].blobs())
        for bn, _, _ in BANKS:
            stream.wait_stream(bstreams[bn])
        return n, times

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(warmup):
        step(False)

    def timed(profile, schedule=kf.KF_SCHED_BATCHED, serial=None, nsteps=steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(nsteps)]
        kt, nb = {}, 0
        barrier()
        with ClockSampler(local) as clk:
            for i in range(nsteps):
                flush.zero_()
                ev[i][0].record(stream)
                nb, times = step(profile, schedule, serial=serial)
                ev[i][1].record(stream)
                for bn, tk in times.items():
                    for k, (nl, ms) in tk.items():
                        a, b = kt.setdefault(bn, {}).get(k, (0, 0.0))
                        kt[bn][k] = (a + nl, b + ms)
            barrier()
        return sum(a.elapsed_time(b) for a, b in ev), kt, nb, clk.summary()

    def slowest(x):
        return max_over_ranks(x, world, dev)

    # --- device-resident timed region (no profiling events) ------------------
    total_ms, _, nblobs, clocks = timed(False)
    ms_per_step = slowest(total_ms) / steps
    pix_scales = len(BANKS) * pixels * len(SCALES)
    value = job_value(pix_scales, world, ms_per_step)
    out = {"value": round(value, 1), "unit": UNIT, "ms_per_step": round(ms_per_step, 4), "steps": steps,
           "warmup": warmup, "clocks": clocks, "blobs_per_step": nblobs, "design_ms": round(design_ms, 2)}
    # --- the same steps with the banks one after the other ------------------
    if concurrent and full:
        s_ms, _, _, _ = timed(False, serial=True)
        s_step = slowest(s_ms) / steps
        out["serial"] = {"value": round(world * pix_scales / (s_step * 1e-3) / 1e6, 1),
                         "ms_per_step": round(s_step, 4),
                         "launches": "the banks one after the other on their streams"}
    # --- the same steps again with CUDA events around every kernel ------------
    _, ktimes, _, _ = timed(True)
    # --- the same steps launched frame by frame (batch workloads) ------------
    if NF > 1 and full:
        for _ in range(2):
            step(False, kf.KF_SCHED_PER_FRAME)
        pf_ms, _, _, _ = timed(False, kf.KF_SCHED_PER_FRAME)
        pf_step = slowest(pf_ms) / steps
        out["per_frame_schedule"] = {"value": round(world * pix_scales / (pf_step * 1e-3) / 1e6, 1),
                                     "ms_per_step": round(pf_step, 4),
                                     "launches": "every pass once per frame, eager (no graph)"}

    # --- end to end: host frames in pinned memory, copies inside the timed region
    if full:
        pinned = [as_t(h).pin_memory() for h in host]
        Xe = [torch.empty_like(x) for x in X]
        Xev = [dview(x) for x in Xe]
        e2e_ms, bo = [], 0
        for i in range(warmup + steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for x, j in zip(Xe, src):
                x.copy_(pinned[j], non_blocking=True)
            nb, _ = step(False, frames=Xev)
            b.record(stream)
            b.synchronize()
            if i >= warmup:
                e2e_ms.append(a.elapsed_time(b))
                bo = nb * np.dtype(kf.BLOB_DTYPE).itemsize
        e2e_step = slowest(sum(e2e_ms) / len(e2e_ms))
        out["e2e"] = {"value": world * pix_scales / (e2e_step * 1e-3) / 1e6, "unit": UNIT,
                      "h2d_bytes_per_step": int(sum(host[j].nbytes for j in src)), "d2h_bytes_per_step": int(bo),
                      "ms_per_step": e2e_step}
        del pinned, Xe, Xev

    # --- HBM fractions and the roofline of the dominant kernel ---------------
    hbm, hbm_src = peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_max_mhz(clocks)
    taps = fir_taps(SCALES, wl["fir_kmax"])
    sizes = dict(s_in=wl["s_in"], s_b=SB[storage])
    per_bank_bytes = bank_bytes(len(SCALES), pixels, wl["s_in"], SB[storage])
    banks_rec, step_bytes = {}, 0.0
    for bn, ft, _o in BANKS:
        kms = sum(ms for _, ms in ktimes.get(bn, {}).values()) / steps
        step_bytes += per_bank_bytes
        banks_rec[bn] = {"kernel_ms": round(kms, 4), "algorithmic_bytes": round(per_bank_bytes),
                         "hbm_frac": round(per_bank_bytes / (kms * 1e-3) / 1e9 / hbm, 4) if kms else None}
    out["hbm"] = {"peak_gbs": hbm, "peak_source": hbm_src,
                  "bytes_per_pixel_scale": round(2.0 * SB[storage] + wl["s_in"] / len(SCALES), 3),
                  "step_frac": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm, 4),
                  "banks": banks_rec,
                  "note": "algorithmic bytes (2 s_b + s_in / S per pixel-scale) over the device-timed step "
                          "(step_frac) or over the sum of the bank's kernel event times (banks)",
                  "target_frac": 0.70}
    # per-kernel totals over the banks (the kernels of two banks of one kind share names)
    kall = {}
    for bn, tk in ktimes.items():
        for k, (nl, ms) in tk.items():
            a, b = kall.get(k, (0, 0.0))
            kall[k] = (a + nl, b + ms)

    def work(k):
        byts = flops = 0.0
        for _, ft, _o in BANKS:
            if k.startswith("fir_") == (ft in (2, 3)):
                b_, f_ = algorithmic(k, len(SCALES), pixels, taps, **sizes)
                byts, flops = byts + b_, flops + f_
        return byts * steps, flops * steps

    kern = {}
    total_kms = max(sum(v[1] for v in kall.values()), 1e-9)
    for k, (nl, ms) in kall.items():
        byts, flops = work(k)
        kern[k] = {"launches": nl, "ms_per_launch": round(ms / max(nl, 1), 4), "share": round(ms / total_kms, 4)}
        if byts:
            kern[k]["GB_s"] = round(byts / (ms * 1e-3) / 1e9, 1)
            kern[k]["hbm_frac"] = round(byts / (ms * 1e-3) / 1e9 / hbm, 4)
        if flops:
            kern[k]["TFLOP_s"] = round(flops / (ms * 1e-3) / 1e12, 2)
    dom = max(kall, key=lambda k: kall[k][1])
    byts, flops = work(dom)
    out["roofline"] = roofline_of(dom, kall[dom][1], kall[dom][0], byts, flops, hbm, hbm_src, nsm, mhz,
                                  traffic_of(name, dom, storage))
    out["kernels"] = kern
    # filter-bank kernels launched in the timed region (the profiled pass runs the same steps)
    out["gpu_launches"] = sum(v[0] for v in kall.values())
    for b in banks.values():
        b.close()
    shapes = sorted({f"{host[j].shape[1]}x{host[j].shape[0]}" for j in src})
    out["config"] = {"workload": wl["text"], "frames": NF, "frame_sizes": shapes, "input": wl["dtype"],
                     "storage": storage, "scales_px": [round(x, 3) for x in SCALES],
                     "banks": [b[0] for b in BANKS], "threshold": THRESHOLD, "fir_kmax": wl["fir_kmax"],
                     "launch": ("batched schedule, replayed from a CUDA graph" if graph else "batched schedule, eager")
                     + ("; one context and stream per bank, the banks of a step launched at once" if concurrent
                        else "; the banks one after the other"),
                     "tuned": tuned or "library defaults (one block per work item, 64-row segments)",
                     "l2": "flushed between steps (256 MiB write outside the timed events)",
                     "parallelism": f"replicas x{world}"}
    out["_host0"] = host[0]
    del X, Xs, flush
    torch.cuda.empty_cache()
    return out


def measure_gated(args, steps, warmup, full=True, mode_name="tiles"):
    """Gated vs plain on the clustered 6144^2 f16 workload: 120 frames in
    calls of 16, both banks at T = 0.3; recall = share of the plain bank's
    blobs (both banks) that the gated run reports, judged in the same run."""
    import numpy as np
    import torch

    from paper_1912_07133_gb300 import kf, synthetic, train_proposal

    rank, world, local = dist_info()
    NF, CHUNK, SIZE, T = 120, 16, 6144, GATED_THRESHOLD
    BANKS = IIR_FIR
    dev = torch.device("cuda", local)
    weights, p_gate, train_stats = train_proposal.load_weights()
    mode = {"dilated": kf.KF_GATE_DILATED, "tiles": kf.KF_GATE_TILES}[mode_name]
    frames = [synthetic.clustered_frame_device(4000 + i, SIZE, SIZE, device=f"cuda:{local}") for i in range(NF)]
    chunks = [frames[i:i + CHUNK] for i in range(0, NF, CHUNK)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    bank = kf.Bank(local, stream.cuda_stream)
    kf.kf_proposal_set_weights(bank.ctx, weights)

    def step(gate, graph=True, profile=False, collect=None, src=None):
        n, times = 0, {}
        for ci, ch in enumerate(src if src is not None else chunks):
            for bi, (_, ft, order) in enumerate(BANKS):
                # the second bank of a chunk reuses the first one's tile marks
                # (the proposal network runs once per frame)
                bank.run(ch, EIGHT, ft, order, threshold=T, fir_kmax=96, gate=mode if gate else kf.KF_GATE_OFF,
                         gate_threshold=p_gate, graph=graph and not profile, profile=profile,
                         gate_reuse=gate and bi > 0)
                b = bank.blobs()
                n += len(b)
                if collect is not None:
                    collect |= {(ci * CHUNK + int(r["frame"]), bi, int(r["scale"]), int(r["y"]), int(r["x"])) for r in b}
                if profile:
                    for k, (nl, ms) in bank.kernel_times().items():
                        a, c = times.get(k, (0, 0.0))
                        times[k] = (a + nl, c + ms)
        return n, times

    def timed(gate, profile=False):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        kt = {}
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clk:
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                _, times = step(gate, profile=profile)
                ev[i][1].record(stream)
                for k, (nl, ms) in times.items():
                    a, c = kt.get(k, (0, 0.0))
                    kt[k] = (a + nl, c + ms)
            torch.cuda.synchronize(dev)
        t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, world, dev)
        return t, kt, clk.summary()

    for _ in range(warmup):
        step(True)
        step(False)
    full_set, gated_set = set(), set()
    step(False, collect=full_set)
    step(True, collect=gated_set)
    recall = len(full_set & gated_set) / max(len(full_set), 1)
    ms_g, _, clocks = timed(True)
    ms_p, _, clocks_p = timed(False)
    _, ktimes, _ = timed(True, profile=True)
    _, ktimes_p, _ = timed(False, profile=True)
    pix_scales = len(BANKS) * NF * SIZE * SIZE * len(EIGHT)
    value = world * pix_scales / (ms_g * 1e-3) / 1e6
    plain = world * pix_scales / (ms_p * 1e-3) / 1e6

    def kernel_list(kt):
        tot = max(sum(v[1] for v in kt.values()), 1e-9)
        return {k: {"launches": nl, "ms_per_step": round(ms / steps, 4), "share": round(ms / tot, 4)}
                for k, (nl, ms) in sorted(kt.items(), key=lambda kv: -kv[1][1])}

    out = {"value": round(value, 1), "unit": UNIT, "ms_per_step": round(ms_g, 4), "steps": steps, "warmup": warmup,
           "plain": {"value": round(plain, 1), "ms_per_step": round(ms_p, 4), "clocks": clocks_p,
                     "kernels": kernel_list(ktimes_p)},
           "recall": round(recall, 5), "blobs_plain": len(full_set), "blobs_gated": len(gated_set),
           "speedup_vs_plain": round(ms_p / ms_g, 3), "clocks": clocks, "kernels": kernel_list(ktimes),
           "gpu_launches": sum(v[0] for v in ktimes.values())}
    if full:
        # end to end: every chunk copied from pinned host memory before its calls
        host = [f.cpu().pin_memory() for f in frames]
        dbuf = [torch.empty_like(frames[0]) for _ in range(CHUNK)]
        e2e_ms, bo = [], 0
        for i in range(warmup + steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nb = 0
            for c0 in range(0, NF, CHUNK):
                for j in range(min(CHUNK, NF - c0)):
                    dbuf[j].copy_(host[c0 + j], non_blocking=True)
                n, _ = step(True, src=[dbuf[:min(CHUNK, NF - c0)]])
                nb += n
            b.record(stream)
            b.synchronize()
            if i >= warmup:
                e2e_ms.append(a.elapsed_time(b))
                bo = nb * np.dtype(kf.BLOB_DTYPE).itemsize
        e2e_step = sum(e2e_ms) / len(e2e_ms)
        out["e2e"] = {"value": world * pix_scales / (e2e_step * 1e-3) / 1e6, "unit": UNIT,
                      "h2d_bytes_per_step": int(sum(h.numel() * 2 for h in host)), "d2h_bytes_per_step": int(bo),
                      "ms_per_step": e2e_step}
        del host, dbuf
    out["config"] = {"workload": ("120 x 6144x6144 FP16 clustered frames (1/f background std 0.1, blob clusters in "
                                  "~5% of the 64x64 tiles, radii 2-32 px; seeds 4000-4119), 8 scales (lambda 2-64 px), "
                                  "colored SG (K<=96) and 4th-order repeated-pole banks, threshold 0.3, calls of 16 "
                                  "frames; gated by the trained proposal network vs the plain bank"),
                     "gate": mode_name, "gate_threshold": p_gate, "frames": NF, "calls_of": CHUNK,
                     "training": {k: train_stats[k] for k in ("frames", "epochs", "seeds", "label_prior")},
                     "l2": "flushed between steps (256 MiB write outside the timed events)",
                     "value_counts": "all pixel-scales of the workload (gated work done on a subset)",
                     "parallelism": f"replicas x{world}"}
    out["_frame0"] = frames[0]
    bank.close()
    del frames, chunks, flush
    torch.cuda.empty_cache()
    return out


SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "clocks", "hbm", "roofline", "kernels",
            "config", "gpu_launches", "per_frame_schedule", "blobs_per_step")


def run_ours(args):
    """The workload's JSON line.  The default workload (the 4096^2 six-scale
    frame, both banks) also carries, as sub-objects measured after its own
    timed region, the gated-vs-plain comparison on the clustered workload and
    the uneven-batch and 12-bit-counts workloads (fewer steps each)."""
    rank, world, local = setup_device(args)
    import torch.distributed as dist
    main = measure_workload(args, args.workload, args.steps, args.warmup, full=True)
    host0 = main.pop("_host0")
    subs = {}
    if args.workload == "iir_fir" and not args.only:
        ss, sw = args.sub_steps, max(3, args.sub_warmup)
        g = measure_gated(args, ss, sw, full=False, mode_name=args.gate_mode)
        g.pop("_frame0")
        subs["gated"] = g
        for sub in ("batch", "counts"):
            r = measure_workload(args, sub, ss, sw, full=False)
            r.pop("_host0")
            subs[sub] = {k: r[k] for k in SUB_KEYS if k in r}
    wl = WORKLOADS[args.workload]
    cpu = cpu_baseline(host0, wl, rows=None if args.workload == "iir_fir" else wl["ref_rows"]) \
        if (rank == 0 and not args.no_cpu) else None
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(main["config"], designs="FP64 design kernel run once per bank configuration, "
                                               "timed separately (design_ms)"),
        "roofline": main["roofline"], "hbm": main["hbm"], "cpu_baseline": cpu, "e2e": main["e2e"],
        "gpu_launches": main["gpu_launches"], "clocks": main["clocks"], "kernels": main["kernels"],
        "blobs_per_step": main["blobs_per_step"], "design_ms": main["design_ms"],
    }
    for k in ("serial", "per_frame_schedule"):
        if k in main:
            line[k] = main[k]
    line.update(subs)
    print(json.dumps(line), flush=True)


def run_gated(args):
    """The gated workload as its own JSON line (value: the gated bank)."""
    rank, world, local = setup_device(args)
    import torch.distributed as dist
    g = measure_gated(args, args.steps, args.warmup, full=True, mode_name=args.gate_mode)
    f0 = g.pop("_frame0")
    cpu = None
    if rank == 0 and not args.no_cpu:
        wl = dict(WORKLOADS["iir_fir"], scales=EIGHT, banks=IIR_FIR, value_scale=1.0)
        cpu = cpu_baseline(f0.float().cpu().numpy(), wl, rows=64)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": g["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": g["config"],
            "plain": g["plain"], "recall": g["recall"], "blobs_plain": g["blobs_plain"],
            "blobs_gated": g["blobs_gated"], "speedup_vs_plain": g["speedup_vs_plain"],
            "roofline": {"kernel": next(iter(g["kernels"])), "bound": None, "achieved": None, "peak": None,
                         "frac": None, "traffic": None,
                         "note": "gated: the kernels run a data-dependent subset of their work items; the "
                                 "default workload's line carries the per-kernel roofline"},
            "cpu_baseline": cpu, "e2e": g["e2e"], "gpu_launches": g["gpu_launches"], "clocks": g["clocks"],
            "kernels": g["kernels"]}
    print(json.dumps(line), flush=True)


def oracle_step(x, wl):
    """Both banks and the detector through the FP64 oracle on the array x."""
    from oracle import oracle as O
    for _, ft, order in wl["banks"]:
        R = O.bank(x, wl["scales"], {0: O.IIR_REPEATED_POLE, 1: O.IIR_BUTTERWORTH, 2: O.FIR_COLORED_SG,
                                     3: O.FIR_GAUSSIAN}[ft],
                   order, fir_kmax=wl["fir_kmax"])
        O.detect(R, THRESHOLD)


def oracle_designs(wl):
    """The oracle's colored-SG designs (cached), made before any timing."""
    from oracle import oracle as O
    if not any(ft == 2 for _, ft, _o in wl["banks"]):
        return
    for l in wl["scales"]:
        O.design_colored_sg_mp(1, O.sg_half_length(1, l / 2, wl["fir_kmax"]), 6.0 / l)


def cpu_baseline(img, wl, rows=None):
    """The FP64 oracle as it stands, on the host cores, on `rows` rows of the
    frame (all scales, both banks); designs are made before timing."""
    import numpy as np

    from oracle import oracle as O

    sub = img if rows is None else img[:rows]
    x = sub.astype(np.float64) * wl["value_scale"]
    oracle_designs(wl)
    t0 = time.perf_counter()
    oracle_step(x, wl)
    dt = time.perf_counter() - t0
    ps = len(wl["banks"]) * sub.shape[0] * sub.shape[1] * len(wl["scales"])
    return {"value": round(ps / dt / 1e6, 3), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"{sub.shape[0]}x{sub.shape[1]} rows of one frame, {len(wl['scales'])} scales, "
                      f"both banks ({dt:.2f} s)"}


# ---------------------------------------------------------------------------
# reference arm: the oracle timed as a program
# ---------------------------------------------------------------------------
# Table V (Sec. 5): one 4096 x 4096 frame, one scale per bank call, the
# Gaussian FIR (Filter A, K = 5 sigma) against the repeated-pole IIR (Filter D,
# K^lpf = 3), sigma = 3, 6, 12, 24.  The paper's GPU times (s) for context
# (another machine; its stage 1 alone).
TABLE5_SIGMAS = (3.0, 6.0, 12.0, 24.0)
TABLE5_PAPER_GPU_S = {"A": (0.30, 0.33, 0.42, 0.56), "D": (0.14, 0.14, 0.14, 0.13)}


def run_table5(args):
    """Single-scale banks, Filter A vs Filter D, on the 4096^2 six-scale frame
    generator; every call with the 3x3 extremum and the ordered read-back."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1912_07133_gb300 import kf, synthetic

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    kf.load()
    dev = torch.device("cuda", local)
    x = torch.from_numpy(synthetic.iir_fir_frame(seed=1, H=4096, W=4096)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    bank = kf.Bank(local, stream.cuda_stream)
    runs = [("A", kf.KF_FIR_GAUSSIAN, 1), ("D", kf.KF_IIR_REPEATED_POLE, 3)]
    table, total_ms = {}, 0.0
    with ClockSampler(local) as clk:
        for name, ft, order in runs:
            table[name] = {}
            for sig in TABLE5_SIGMAS:
                lam = [2.0 * sig]

                def call():
                    bank.run([x], lam, ft, order, threshold=THRESHOLD, fir_kmax=160, graph=True,
                             neighbourhood=kf.KF_NEIGH_ALL_SCALES)
                    return len(bank.blobs())

                for _ in range(args.warmup):
                    call()
                ms = []
                for _ in range(args.steps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    nb = call()
                    b.record(stream)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                med = float(np.median(ms))
                total_ms += med
                table[name][str(sig)] = {"ms": round(med, 4), "blobs": nb,
                                         "K": (min(int(np.ceil(5 * sig)), 160) if ft == kf.KF_FIR_GAUSSIAN else order)}
        clocks = clk.summary()
    bank.close()
    pix_scales = 4096 * 4096 * len(runs) * len(TABLE5_SIGMAS)
    line = {
        "metric": "Mpixel-scales/s, Table V single-scale banks (Filter A FIR vs Filter D IIR) on 1 GB300",
        "value": round(pix_scales / (total_ms * 1e-3) / 1e6, 1), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "4096x4096 FP32 frame (six-scale generator), one scale per call: sigma = 3, 6, "
                               "12, 24 px; Filter A (Gaussian FIR, K = 5 sigma) and Filter D (repeated pole, "
                               "K^lpf = 3); Laplacian response, 3x3 extremum, blob list read back",
                   "statistic": "median of the steps per (filter, sigma); value: their sum",
                   "l2": "flushed between calls (256 MiB write outside the timed events)",
                   "launch": "graph replays"},
        "table_ms": table, "paper_gpu_seconds": {k: dict(zip(map(str, TABLE5_SIGMAS), v))
                                                 for k, v in TABLE5_PAPER_GPU_S.items()},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# The D = 5 derivative bank (Sec. 4, L_D = 2): every D_{dx,dy}, dx + dy <= 4
# (15 channels), of one 2048 x 2048 frame at 4 scales, Filter D with L_D = 2
# and one Nyquist constraint pair (K^lpf = 4).
QUARTIC_SCALES = (4.0, 8.0, 16.0, 32.0)
QUARTIC_HW = 2048


def quartic_bytes(name, S, H, W, nch=15):
    """Algorithmic bytes of one launch of a kernel of the D = 5 bank (all 15
    channels): the differentiator reads the frame and writes the 15 channel
    planes (W x (H + 4): two rows beyond each end); the row pass reads them
    and writes S planes each; the segment-state pass reads those; the column
    pass (either form) reads them and writes the 15 S output planes (H rows)."""
    P = (H + 4) * W
    return {"quartic_hpf": 4 * H * W + 4 * nch * P, "iir_row": nch * (4 * P + 4 * S * P),
            "iir_colseg": nch * 4 * S * P, "iir_coldet": nch * (4 * S * P + 4 * S * H * W),
            "iir_colscan": nch * (4 * S * P + 4 * S * H * W)}.get(name)


def run_quartic(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1912_07133_gb300 import kf, synthetic

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    __graft_entry__.build()
    kf.load()
    dev = torch.device("cuda", local)
    H = W = QUARTIC_HW
    S = len(QUARTIC_SCALES)
    host = synthetic.iir_fir_frame(seed=1, H=H, W=W, nblobs=250)
    x = torch.from_numpy(host).to(dev)
    out = torch.empty((S, kf.KF_QUARTIC_CHANNELS, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = kf.kf_create(local, stream.cuda_stream)
    ft, order = kf.KF_IIR_REPEATED_POLE, 4

    def call(frame=x, profile=False):
        kf.kf_quartic_bank(ctx, frame, QUARTIC_SCALES, ft, order, out=out, profile=profile)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        clocks = clk.summary()
    step_ms = float(np.mean(ms))
    # end to end: the frame from pinned host memory, the bank, all planes back
    # to pinned host memory
    pin_in = torch.from_numpy(host).pin_memory()
    pin_out = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    xe = torch.empty_like(x)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xe.copy_(pin_in, non_blocking=True)
        call(xe)
        pin_out.copy_(out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    # per-kernel times of one profiled call (the step's own launches)
    call(profile=True)
    kt = kf.kf_kernel_times(ctx)
    kf.kf_destroy(ctx)
    ps = H * W * S
    total = sum(v[1] for v in kt.values())
    kernels = {}
    for name, (n, t) in sorted(kt.items(), key=lambda kv: -kv[1][1]):
        k = {"launches": n, "ms_per_launch": round(t / n, 4), "share": round(t / total, 4)}
        b = quartic_bytes(name, S, H, W)
        if b is not None and t > 0:
            k["GB_s"] = round(b / (t / n * 1e-3) / 1e9, 1)
        kernels[name] = k
    top = max(kt, key=lambda k: kt[k][1])
    n_top, t_top = kt[top]
    peak, src = peaks()
    b_top = quartic_bytes(top, S, H, W)
    ach = b_top / (t_top / n_top * 1e-3) / 1e9 if b_top else None
    roof = {"kernel": top, "bound": "hbm", "achieved": round(ach, 1) if ach else None, "peak": peak,
            "unit": "GB/s", "frac": round(ach / peak, 4) if ach else None,
            "traffic": traffic_of("quartic", top, "f32"),
            "peak_source": src, "bytes_per_launch": b_top}
    cpu = None
    if not args.no_cpu:
        cpu = quartic_cpu_baseline(host)
    line = {
        "metric": "Mpixel-scales/s, D = 5 derivative bank (15 channels D_{dx,dy}, dx + dy <= 4) on 1 GB300",
        "value": round(ps / (step_ms * 1e-3) / 1e6, 1), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{H}x{W} FP32 frame (1/f background, 250 blobs), {S} scales (lambda 4-32 px), "
                               "Filter D with L_D = 2, K^lpf = 4; all 15 channels written to HBM",
                   "l2": "flushed between steps (256 MiB write outside the timed events); output 1 GiB",
                   "launch": "eager: the differentiator, then one bank call over the 15 channel planes"},
        "e2e": {"value": round(ps / (float(np.mean(e2e_ms)) * 1e-3) / 1e6, 1), "unit": UNIT,
                "h2d_bytes_per_step": int(pin_in.numel() * 4), "d2h_bytes_per_step": int(pin_out.numel() * 4)},
        "gpu_launches": int(sum(v[0] for v in kt.values())),
        "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def quartic_cpu_baseline(host, rows=64):
    """The D = 5 oracle on `rows` rows of the frame, all scales."""
    import numpy as np

    from oracle import oracle as O
    from oracle import quartic as Q

    sub = host[:rows].astype(np.float64)
    Q.quartic_bank(sub[:8, :64], QUARTIC_SCALES[:1], O.IIR_REPEATED_POLE, 4)  # build, warm
    t0 = time.perf_counter()
    Q.quartic_bank(sub, QUARTIC_SCALES, O.IIR_REPEATED_POLE, 4)
    dt = time.perf_counter() - t0
    return {"value": round(sub.size * len(QUARTIC_SCALES) / dt / 1e6, 4), "unit": UNIT, "cores": 1,
            "kind": "oracle", "sample": f"{sub.shape[0]}x{sub.shape[1]} rows of the frame, "
                                        f"{len(QUARTIC_SCALES)} scales, 15 channels ({dt:.2f} s)"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import numpy as np

    from oracle import oracle as O

    O.build()
    if args.workload == "quartic":
        from paper_1912_07133_gb300 import synthetic
        host = synthetic.iir_fir_frame(seed=1, H=QUARTIC_HW, W=QUARTIC_HW, nblobs=250)
        for _ in range(args.warmup):
            quartic_cpu_baseline(host, rows=8)
        vals = [quartic_cpu_baseline(host, rows=16) for _ in range(args.steps)]
        v = float(sum(c["value"] for c in vals) / len(vals))
        sample = vals[0]["sample"].split(" (")[0] + " per step"
        print(json.dumps({
            "metric": "Mpixel-scales/s, D = 5 derivative bank (15 channels D_{dx,dy}, dx + dy <= 4) on 1 GB300",
            "value": round(v, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(16 * QUARTIC_HW * len(QUARTIC_SCALES) / (v * 1e6) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{QUARTIC_HW}x{QUARTIC_HW} FP32 frame, 4 scales, Filter D L_D = 2",
                       "sample": sample, "parallelism": "host core"},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "kind": "oracle", "cores": 1, "sample": sample},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
            flush=True)
        return
    if args.workload == "gated":
        from paper_1912_07133_gb300 import synthetic
        wl = dict(banks=IIR_FIR, scales=EIGHT, fir_kmax=96, value_scale=1.0, ref_rows=64,
                  text="clustered 6144-wide FP16 frames, 8 scales, both banks (oracle: plain bank, no gating)")
        img = synthetic.clustered_frame(seed=4000, H=256, W=6144).astype(np.float32)
    elif args.workload == "table5":
        from paper_1912_07133_gb300 import synthetic
        wl = dict(banks=(("gaussian_fir", 3, 1), ("iir_repeated_pole_order3", 0, 3)),
                  scales=[2.0 * s for s in TABLE5_SIGMAS], fir_kmax=160, value_scale=1.0, ref_rows=64,
                  text="4096x4096 FP32 frame, sigma = 3, 6, 12, 24 px, Filter A (K = 5 sigma) and Filter D "
                       "(K^lpf = 3), Laplacian response, 3x3 extremum")
        img = synthetic.iir_fir_frame(seed=1, H=256, W=4096)
    else:
        wl = WORKLOADS[args.workload]
        img = make_frames(wl)[0]
    rows = wl["ref_rows"]  # bounded sample per step: rows x W x all scales x 2 banks
    W = img.shape[1]
    x = img[:rows].astype(np.float64) * wl["value_scale"]
    oracle_designs(wl)

    for _ in range(args.warmup):
        oracle_step(x, wl)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(x, wl)
    dt = (time.perf_counter() - t0) / args.steps
    ps = len(wl["banks"]) * rows * W * len(wl["scales"])
    v = ps / dt / 1e6
    sample = (f"{rows}x{W} rows of one {img.shape[0]}x{W} frame per step, {len(wl['scales'])} scales, "
              f"both banks")
    line = {"metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl["text"], "sample": sample, "parallelism": "host cores"},
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
    ap.add_argument("--workload", choices=tuple(WORKLOADS) + ("gated", "table5", "quartic"), default="iir_fir")
    ap.add_argument("--gate-mode", choices=("dilated", "tiles"), default="tiles",
                    help="gated workload: marked tiles with their neighbours, or marked tiles only")
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of replaying a CUDA graph")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library default launch shapes)")
    ap.add_argument("--serial", action="store_true", help="run the banks of a step one after the other")
    ap.add_argument("--only", action="store_true",
                    help="default workload: skip the gated, batch and counts sub-workloads")
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of each sub-workload")
    ap.add_argument("--sub-warmup", type=int, default=3, help="warm-up steps of each sub-workload (>= 3)")
    ap.add_argument("--column-pass", choices=("segments", "single-read"), default=None,
                    help="column pass of the recursive banks (with --no-tune it stays fixed)")
    ap.add_argument("--shape", default=None,
                    help="launch shapes over the tuned ones, e.g. iir.row=-2,fir.row=-3 (negative: blocks per SM)")
    ap.add_argument("--storage", choices=tuple(STORAGE), default=None,
                    help="element type of the one-sided planes (default: the workload's)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "gated":
        run_gated(args)
    elif args.workload == "table5":
        run_table5(args)
    elif args.workload == "quartic":
        run_quartic(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
