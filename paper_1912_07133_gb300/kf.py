"""Thin Python binding of the C ABI in ``include/kf.h`` (ctypes).

Argument marshalling only: every step of the filter bank runs in the CUDA
kernels of ``_lib/libkf.so``.  Device buffers come from PyTorch tensors
(``data_ptr``) and work is issued on PyTorch's current CUDA stream.  Loading
fails loudly if the library is missing (build it with
``python -c "import __graft_entry__ as g; g.build()"``) or no GPU is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libkf.so")

KF_OK = 0
KF_EINVAL = -1
KF_ECOND = -2
KF_ENOMEM = -3
KF_ECUDA = -4
KF_ETIMEOUT = -5
KF_EOVERFLOW = -6
KF_ENODEV = -7
KF_ERERUN = -8
KF_ERANGE = -9

KF_IIR_REPEATED_POLE = 0
KF_IIR_BUTTERWORTH = 1
KF_FIR_COLORED_SG = 2
KF_FIR_GAUSSIAN = 3
FIR_TYPES = (KF_FIR_COLORED_SG, KF_FIR_GAUSSIAN)

KF_DTYPE_F32 = 0
KF_DTYPE_F16 = 1
KF_DTYPE_BF16 = 2
KF_DTYPE_U16 = 3

KF_RESP_LAPLACIAN = 0
KF_RESP_HESSIAN = 1
KF_BOUNDARY_HOLD = 0
KF_BOUNDARY_ZERO = 1
KF_NEIGH_ALL_SCALES = 0
KF_NEIGH_ADJACENT = 1
KF_GATE_OFF, KF_GATE_DILATED, KF_GATE_TILES = 0, 1, 2
KF_SCHED_BATCHED = 0
KF_SCHED_PER_FRAME = 1
KF_COLUMN_SINGLE_READ = 0
KF_COLUMN_SEGMENTS = 1
KF_MAX_SCALES = 16
KF_MAX_ORDER = 8
KF_MAX_FIR_K = 160

ENTRY_POINTS = ("kf_bank_opts_default", "kf_create", "kf_destroy", "kf_last_error", "kf_design",
                "kf_filter_bank", "kf_detect_blobs", "kf_kernel_times", "kf_responses_noalloc",
                "kf_set_launch_shape", "kf_set_segment_length", "kf_set_column_pass", "kf_autotune",
                "kf_proposal_set_weights", "kf_proposal_get_weights", "kf_proposal_pool", "kf_proposal_logits",
                "kf_proposal_grad", "kf_proposal_train_step", "kf_proposal_labels", "kf_blob_shapes",
                "kf_quartic_bank", "kf_quartic_steer", "kf_set_wait_limit")
KF_QUARTIC_CHANNELS = 15
# (dx, dy) of the D = 5 bank's channels: total order n = 0..4, within it dy = 0..n
QUARTIC_CHANNELS = tuple((n - dy, dy) for n in range(5) for dy in range(n + 1))
KF_NET_NPARAM = 3640
KF_NET_CHANNELS = 8
KF_PASS_ROW, KF_PASS_SEG, KF_PASS_FOLD, KF_PASS_DET, KF_NPASS = 0, 1, 2, 3, 4
GRID_CANDIDATES = (1, 2, 4, 0)
KF_NOALLOC_SCRATCH_MB = 32


class kf_coeffs(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("order", ctypes.c_int32), ("K", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("scale", ctypes.c_double), ("sigma", ctypes.c_double),
                ("param", ctypes.c_double), ("b0", ctypes.c_double),
                ("bplus", ctypes.c_double * (KF_MAX_ORDER + 1)),
                ("aplus", ctypes.c_double * (KF_MAX_ORDER + 1)),
                ("h", ctypes.c_double * (KF_MAX_FIR_K + 1)),
                ("dc_gain", ctypes.c_double), ("moment2", ctypes.c_double)]


class kf_frame(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch", ctypes.c_int64), ("dtype", ctypes.c_int32), ("value_scale", ctypes.c_float)]


class kf_bank_opts(ctypes.Structure):
    _fields_ = [("response", ctypes.c_int32), ("boundary", ctypes.c_int32),
                ("neighbourhood", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("threshold", ctypes.c_double), ("fir_kmax", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("responses", ctypes.c_void_p),
                ("schedule", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("gate", ctypes.c_int32), ("gate_threshold", ctypes.c_float),
                ("offset_limit", ctypes.c_float), ("gate_reuse", ctypes.c_int32),
                ("reserved", ctypes.c_int64 * 1)]


class kf_blob(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_int32), ("x", ctypes.c_int32), ("y", ctypes.c_int32),
                ("scale", ctypes.c_int32), ("polarity", ctypes.c_int32), ("response", ctypes.c_float),
                ("dx", ctypes.c_float), ("dy", ctypes.c_float)]


class kf_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int32), ("ms", ctypes.c_float)]


BLOB_DTYPE = np.dtype([("frame", "<i4"), ("x", "<i4"), ("y", "<i4"), ("scale", "<i4"),
                       ("polarity", "<i4"), ("response", "<f4"), ("dx", "<f4"), ("dy", "<f4")])

_lib = None


class KfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kf error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the library and declare its signatures (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.kf_bank_opts_default.restype = i32
    L.kf_bank_opts_default.argtypes = [ctypes.POINTER(kf_bank_opts)]
    L.kf_create.restype = i32
    L.kf_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    L.kf_destroy.restype = None
    L.kf_destroy.argtypes = [vp]
    L.kf_last_error.restype = ctypes.c_char_p
    L.kf_last_error.argtypes = [vp]
    L.kf_design.restype = i32
    L.kf_design.argtypes = [i32, i32, dbl, ctypes.POINTER(kf_coeffs)]
    L.kf_filter_bank.restype = i32
    L.kf_filter_bank.argtypes = [vp, ctypes.POINTER(kf_frame), i32, ctypes.POINTER(dbl), i32, i32, i32,
                                 ctypes.POINTER(kf_bank_opts)]
    L.kf_detect_blobs.restype = i32
    L.kf_detect_blobs.argtypes = [vp, dbl, ctypes.POINTER(kf_blob), i64, ctypes.POINTER(i64)]
    L.kf_blob_shapes.restype = i32
    L.kf_blob_shapes.argtypes = [vp, dbl, ctypes.POINTER(kf_blob_shape), i64, ctypes.POINTER(i64)]
    L.kf_kernel_times.restype = i32
    L.kf_kernel_times.argtypes = [vp, ctypes.POINTER(kf_kernel_time), i32, ctypes.POINTER(i32)]
    L.kf_responses_noalloc.restype = i32
    L.kf_responses_noalloc.argtypes = [ctypes.POINTER(kf_frame), ctypes.POINTER(dbl), i32, i32, i32, vp, vp]
    L.kf_set_launch_shape.restype = i32
    L.kf_set_launch_shape.argtypes = [vp, i32, i32, i32]
    fp = ctypes.POINTER(ctypes.c_float)
    L.kf_proposal_set_weights.restype = i32
    L.kf_proposal_set_weights.argtypes = [vp, fp]
    L.kf_proposal_get_weights.restype = i32
    L.kf_proposal_get_weights.argtypes = [vp, fp]
    L.kf_proposal_pool.restype = i32
    L.kf_proposal_pool.argtypes = [vp, ctypes.POINTER(kf_frame), i32, vp]
    L.kf_proposal_logits.restype = i32
    L.kf_proposal_logits.argtypes = [vp, vp, i32, i32, i32, vp]
    L.kf_proposal_grad.restype = i32
    L.kf_proposal_grad.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, fp, fp]
    L.kf_proposal_train_step.restype = i32
    L.kf_proposal_train_step.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_float, fp]
    L.kf_proposal_labels.restype = i32
    L.kf_proposal_labels.argtypes = [vp, dbl, vp]
    L.kf_set_wait_limit.restype = i32
    L.kf_set_wait_limit.argtypes = [vp, i32]
    L.kf_set_segment_length.restype = i32
    L.kf_set_segment_length.argtypes = [vp, i32, i32]
    L.kf_set_column_pass.restype = i32
    L.kf_set_column_pass.argtypes = [vp, i32, i32]
    L.kf_quartic_bank.restype = i32
    L.kf_quartic_bank.argtypes = [vp, ctypes.POINTER(kf_frame), ctypes.POINTER(dbl), i32, i32, i32, vp, i32]
    L.kf_quartic_steer.restype = i32
    L.kf_quartic_steer.argtypes = [vp, vp, i64, i32, dbl, vp]
    L.kf_autotune.restype = i32
    L.kf_autotune.argtypes = [vp, ctypes.POINTER(kf_frame), i32, ctypes.POINTER(dbl), i32, i32, i32,
                              ctypes.POINTER(kf_bank_opts), ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
    _lib = L
    return L


def _check(rc: int, ctx=None):
    if rc != KF_OK:
        raise KfError(rc, load().kf_last_error(ctx).decode())


# ---- entry points under their C names ---------------------------------------
def kf_bank_opts_default() -> kf_bank_opts:
    o = kf_bank_opts()
    _check(load().kf_bank_opts_default(ctypes.byref(o)))
    return o


def kf_create(device: int = 0, stream=None) -> int:
    """Context on `device` using `stream` (default: torch's current stream)."""
    import torch

    if not torch.cuda.is_available():
        raise KfError(KF_ENODEV, "no CUDA device (the filter bank has no CPU path)")
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    ctx = ctypes.c_void_p()
    _check(load().kf_create(ctypes.byref(ctx), device, ctypes.c_void_p(stream)))
    return ctx.value


def kf_destroy(ctx: int) -> None:
    load().kf_destroy(ctx)
    _count_guess.pop(ctx, None)


def kf_last_error(ctx=None) -> str:
    return load().kf_last_error(ctx).decode()


def kf_design(ftype: int, order: int, scale: float) -> dict:
    c = kf_coeffs()
    _check(load().kf_design(ftype, order, float(scale), ctypes.byref(c)))
    K = c.K
    d = dict(type=c.type, order=c.order, K=K, scale=c.scale, sigma=c.sigma, param=c.param, b0=c.b0,
             dc_gain=c.dc_gain, moment2=c.moment2)
    if ftype in FIR_TYPES:
        d["h"] = np.array(c.h[: K + 1])
    else:
        d["bplus"] = np.array(c.bplus[: K + 1])
        d["aplus"] = np.array(c.aplus[: K + 1])
    return d


def _frame_desc(t, value_scale: float = 0.0) -> kf_frame:
    import torch

    if not t.is_cuda or t.dim() != 2:
        raise ValueError("frames must be 2-D CUDA tensors")
    if t.stride(1) != 1:
        raise ValueError("frames must have unit column stride")
    dt = {torch.float32: KF_DTYPE_F32, torch.float16: KF_DTYPE_F16, torch.bfloat16: KF_DTYPE_BF16,
          torch.uint16: KF_DTYPE_U16}.get(t.dtype)
    if dt is None:
        raise ValueError(f"unsupported frame dtype {t.dtype}")
    return kf_frame(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0), dt, float(value_scale))


def kf_filter_bank(ctx: int, frames, scales, ftype: int, order: int, opts: kf_bank_opts = None,
                   value_scales=None) -> None:
    """Enqueue the bank on the context stream; `frames` are CUDA tensors
    (float32, float16, bfloat16 or uint16), each multiplied by its entry of
    `value_scales` (None: 1)."""
    vs = value_scales if value_scales is not None else [0.0] * len(frames)
    if len(vs) != len(frames):
        raise ValueError("one value scale per frame")
    descs = (kf_frame * len(frames))(*[_frame_desc(f, v) for f, v in zip(frames, vs)])
    sc = (ctypes.c_double * len(scales))(*[float(s) for s in scales])
    if opts is None:
        opts = kf_bank_opts_default()
    _check(load().kf_filter_bank(ctx, descs, len(frames), sc, len(scales), ftype, order,
                                 ctypes.byref(opts)), ctx)


_count_guess: dict = {}  # ctx -> capacity to offer the next kf_detect_blobs call


def _host_records(n: int) -> np.ndarray:
    """n blob records in page-locked host memory (the device copy runs at full
    speed into it); plain memory where no CUDA device is present."""
    if n > 0:
        import torch

        if torch.cuda.is_available():
            t = torch.empty(n * BLOB_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
            return t.numpy().view(BLOB_DTYPE)  # the array keeps the pinned block alive
    return np.empty(n, dtype=BLOB_DTYPE)


def kf_detect_blobs(ctx: int, threshold: float, capacity: int = None) -> np.ndarray:
    """Blob list of the last bank call, sorted by (frame, scale, y, x).

    The library orders the list on the GPU and keeps it.  Without a capacity
    the list is copied into pinned memory sized from the previous call's
    count: one library call (ordering, count and copy under one stream
    synchronisation) unless the list outgrew it, when a second call copies
    the rest of the kept list."""
    L = load()
    n = ctypes.c_int64(0)
    guessed = capacity is None
    if guessed:
        capacity = _count_guess.get(ctx, 1 << 16)
    out = _host_records(capacity)
    rc = L.kf_detect_blobs(ctx, float(threshold), out.ctypes.data_as(ctypes.POINTER(kf_blob)) if capacity else None,
                           capacity, ctypes.byref(n))
    if guessed and rc in (KF_OK, KF_EOVERFLOW):
        _count_guess[ctx] = int(n.value) + int(n.value) // 4 + 1024
    if rc == KF_EOVERFLOW and n.value > capacity:
        return kf_detect_blobs(ctx, threshold, int(n.value))
    _check(rc, ctx)
    return out[: n.value]


class kf_blob_shape(ctypes.Structure):
    _fields_ = [("p1", ctypes.c_float), ("p2", ctypes.c_float), ("theta", ctypes.c_float), ("det", ctypes.c_float)]


def kf_quartic_bank(ctx: int, frame, scales, ftype: int, order: int, out=None, value_scale: float = 0.0,
                    profile: bool = False):
    """D_{dx,dy} for dx + dy <= 4 (the D = 5 bank) of one CUDA frame: a float32
    CUDA tensor (len(scales), 15, H, W) in the QUARTIC_CHANNELS order, written
    on the context stream (`out`: an existing tensor of that shape, or None).
    profile: time each kernel (kf_kernel_times returns the totals)."""
    import torch

    desc = _frame_desc(frame, value_scale)
    H, W = frame.shape
    if out is None:
        out = torch.empty((len(scales), KF_QUARTIC_CHANNELS, H, W), dtype=torch.float32, device=frame.device)
    if out.shape != (len(scales), KF_QUARTIC_CHANNELS, H, W) or out.dtype != torch.float32 or \
            not out.is_contiguous() or out.device != frame.device:
        raise ValueError("out must be a contiguous float32 tensor (S, 15, H, W) on the frame's device")
    sc = (ctypes.c_double * len(scales))(*[float(s) for s in scales])
    _check(load().kf_quartic_bank(ctx, ctypes.byref(desc), sc, len(scales), ftype, order, out.data_ptr(),
                                  1 if profile else 0), ctx)
    return out


def kf_quartic_steer(ctx: int, D, phi: float, out=None):
    """Steered derivatives of a (..., 15, H, W) float32 CUDA tensor of D = 5
    bank outputs (Sec. 2): a tensor of the same shape (`out` may be D)."""
    import torch

    if not D.is_cuda or D.dtype != torch.float32 or not D.is_contiguous() or D.dim() < 3 or \
            D.shape[-3] != KF_QUARTIC_CHANNELS:
        raise ValueError("D must be a contiguous float32 CUDA tensor (..., 15, H, W)")
    if out is None:
        out = torch.empty_like(D)
    if out.shape != D.shape or out.dtype != D.dtype or not out.is_contiguous():
        raise ValueError("out must match D")
    npix = D.shape[-1] * D.shape[-2]
    nsets = D.numel() // (KF_QUARTIC_CHANNELS * npix)
    _check(load().kf_quartic_steer(ctx, D.data_ptr(), npix, nsets, float(phi), out.data_ptr()), ctx)
    return out


SHAPE_DTYPE = np.dtype([("p1", "<f4"), ("p2", "<f4"), ("theta", "<f4"), ("det", "<f4")])


def kf_blob_shapes(ctx: int, threshold: float) -> np.ndarray:
    """Shapes (p1, p2, theta, |H|) of the blobs kf_detect_blobs returns at
    this threshold, in the same order (the last call must have run the
    derivative bank)."""
    L = load()
    n = ctypes.c_int64(0)
    rc = L.kf_blob_shapes(ctx, float(threshold), None, 0, ctypes.byref(n))
    if rc not in (KF_OK, KF_EOVERFLOW):
        _check(rc, ctx)
    out = np.empty(int(n.value), dtype=SHAPE_DTYPE)
    if n.value == 0:
        return out
    _check(L.kf_blob_shapes(ctx, float(threshold), out.ctypes.data_as(ctypes.POINTER(kf_blob_shape)), len(out),
                            ctypes.byref(n)), ctx)
    return out


def kf_kernel_times(ctx: int) -> dict:
    """{kernel name: (launches, ms)} of the last bank call."""
    out = (kf_kernel_time * 64)()
    n = ctypes.c_int(0)
    _check(load().kf_kernel_times(ctx, out, 64, ctypes.byref(n)), ctx)
    return {out[i].name.decode(): (out[i].launches, out[i].ms) for i in range(min(n.value, 64))}


def kf_responses_noalloc(frame, scales, ftype: int, order: int, responses, stream=None,
                         value_scale: float = 0.0) -> None:
    """Response planes of one frame without any device allocation by the
    library (for callers whose device memory is owned by another allocator or
    whose loops may not allocate); see include/kf.h for the size limit."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    if not responses.is_cuda or responses.dtype != torch.float32 or not responses.is_contiguous():
        raise ValueError("responses must be a contiguous float32 CUDA tensor")
    if responses.numel() < len(scales) * frame.shape[0] * frame.shape[1]:
        raise ValueError("responses is too small")
    d = _frame_desc(frame, value_scale)
    sc = (ctypes.c_double * len(scales))(*[float(s) for s in scales])
    _check(load().kf_responses_noalloc(ctypes.byref(d), sc, len(scales), ftype, order, responses.data_ptr(),
                                       ctypes.c_void_p(stream)))


def kf_set_launch_shape(ctx: int, ftype: int, pass_: int, grid_mult: int) -> None:
    """Launch shape of one pass (0: one block per work item; k: k x the
    resident blocks of the GPU, looping over items; -b: b blocks per SM, a
    share that leaves the rest of every SM to other streams' kernels)."""
    _check(load().kf_set_launch_shape(ctx, ftype, pass_, grid_mult), ctx)


def kf_set_wait_limit(ctx, polls: int) -> None:
    """Failure-detection test hook: polls > 0 makes the column pass's bounded
    load wait give up (no copy issued); 0 restores normal waits.  ctx None:
    the hook of kf_responses_noalloc."""
    _check(load().kf_set_wait_limit(ctx, int(polls)), ctx)


def kf_set_segment_length(ctx: int, ftype: int, rows: int) -> None:
    """Column segment length (32 or 64 rows) of a recursive bank."""
    _check(load().kf_set_segment_length(ctx, ftype, rows), ctx)


def kf_set_column_pass(ctx: int, ftype: int, mode: int) -> None:
    """Column pass of a recursive bank: KF_COLUMN_SEGMENTS (default) or
    KF_COLUMN_SINGLE_READ."""
    _check(load().kf_set_column_pass(ctx, ftype, mode), ctx)


def kf_autotune(ctx: int, frames, scales, ftype: int, order: int, opts: kf_bank_opts = None,
                value_scales=None):
    """Time every pass at each candidate launch shape (and, for the recursive
    banks, segment length) on these frames and keep the fastest; returns
    (chosen shapes per pass, segment length, {pass: [ms per shape candidate]})."""
    vs = value_scales if value_scales is not None else [0.0] * len(frames)
    descs = (kf_frame * len(frames))(*[_frame_desc(f, v) for f, v in zip(frames, vs)])
    sc = (ctypes.c_double * len(scales))(*[float(s) for s in scales])
    if opts is None:
        opts = kf_bank_opts_default()
    chosen = (ctypes.c_int32 * (KF_NPASS + 1))()
    ms = (ctypes.c_float * (KF_NPASS * 4))()
    _check(load().kf_autotune(ctx, descs, len(frames), sc, len(scales), ftype, order, ctypes.byref(opts),
                              chosen, ms), ctx)
    times = {p: list(ms[4 * p: 4 * p + 4]) for p in range(KF_NPASS) if chosen[p] >= 0}
    return list(chosen[:KF_NPASS]), chosen[KF_NPASS], times


def _cuda_tensor(t, dtype, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous {dtype} CUDA tensor")
    return t.data_ptr()


def kf_proposal_set_weights(ctx: int, weights) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if w.size != KF_NET_NPARAM:
        raise ValueError(f"need {KF_NET_NPARAM} weights")
    _check(load().kf_proposal_set_weights(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), ctx)


def kf_proposal_get_weights(ctx: int) -> np.ndarray:
    w = np.empty(KF_NET_NPARAM, np.float32)
    _check(load().kf_proposal_get_weights(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), ctx)
    return w


def pooled_shape(H: int, W: int):
    return (H + 7) // 8, (W + 7) // 8


def kf_proposal_pool(ctx: int, frames, out, value_scales=None) -> None:
    """Pooled frames, back to back, into the float32 CUDA tensor `out`."""
    import torch
    need = sum(int(np.prod(pooled_shape(*f.shape))) for f in frames)
    if out.numel() < need:
        raise ValueError(f"out needs {need} elements")
    vs = value_scales if value_scales is not None else [0.0] * len(frames)
    descs = (kf_frame * len(frames))(*[_frame_desc(f, v) for f, v in zip(frames, vs)])
    _check(load().kf_proposal_pool(ctx, descs, len(frames), _cuda_tensor(out, torch.float32, "out")), ctx)


def kf_proposal_logits(ctx: int, pooled, logits) -> None:
    """pooled [n, h, w] float32 -> logits [n, 8, ceil(h/8), ceil(w/8)] float32 (CUDA tensors)."""
    import torch
    n, h, w = pooled.shape
    _check(load().kf_proposal_logits(ctx, _cuda_tensor(pooled, torch.float32, "pooled"), n, h, w,
                                     _cuda_tensor(logits, torch.float32, "logits")), ctx)


def kf_proposal_grad(ctx: int, pooled, labels, pos_weight: float):
    """(loss, gradient[KF_NET_NPARAM]) on a batch (CUDA tensors: pooled float32
    [n, h, w], labels uint8 [n, 8, ceil(h/8), ceil(w/8)])."""
    import torch
    n, h, w = pooled.shape
    g = np.empty(KF_NET_NPARAM, np.float32)
    loss = ctypes.c_float(0)
    _check(load().kf_proposal_grad(ctx, _cuda_tensor(pooled, torch.float32, "pooled"),
                                   _cuda_tensor(labels, torch.uint8, "labels"), n, h, w, float(pos_weight),
                                   g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)), ctx)
    return float(loss.value), g


def kf_proposal_train_step(ctx: int, pooled, labels, pos_weight: float, lr: float, want_loss=True):
    import torch
    n, h, w = pooled.shape
    loss = ctypes.c_float(0)
    _check(load().kf_proposal_train_step(ctx, _cuda_tensor(pooled, torch.float32, "pooled"),
                                         _cuda_tensor(labels, torch.uint8, "labels"), n, h, w, float(pos_weight),
                                         float(lr), ctypes.byref(loss) if want_loss else None), ctx)
    return float(loss.value) if want_loss else None


def kf_proposal_labels(ctx: int, threshold: float, labels) -> None:
    import torch
    _check(load().kf_proposal_labels(ctx, float(threshold), _cuda_tensor(labels, torch.uint8, "labels")), ctx)


class Bank:
    """Convenience wrapper: one context, repeated bank calls."""

    def __init__(self, device: int = 0, stream=None):
        self.ctx = kf_create(device, stream)

    def run(self, frames, scales, ftype=KF_IIR_REPEATED_POLE, order=4, threshold=0.05,
            neighbourhood=KF_NEIGH_ALL_SCALES, responses=None, fir_kmax=96, profile=False,
            storage=KF_DTYPE_F32, value_scales=None, schedule=KF_SCHED_BATCHED, graph=False, gate=False,
            gate_threshold=None, response=KF_RESP_LAPLACIAN, offset_limit=0.0, boundary=KF_BOUNDARY_HOLD,
            gate_reuse=False):
        o = kf_bank_opts_default()
        o.threshold = float(threshold)
        o.profile = 1 if profile else 0
        o.neighbourhood = neighbourhood
        o.fir_kmax = fir_kmax
        o.storage = storage
        o.schedule = schedule
        o.graph = 1 if graph else 0
        o.gate = int(gate) if not isinstance(gate, bool) else (KF_GATE_DILATED if gate else KF_GATE_OFF)
        o.response = response
        o.offset_limit = float(offset_limit)
        o.boundary = int(boundary)
        o.gate_reuse = 1 if gate_reuse else 0
        if gate_threshold is not None:
            o.gate_threshold = float(gate_threshold)
        if responses is not None:
            import torch

            if not responses.is_cuda or responses.dtype != torch.float32 or not responses.is_contiguous():
                raise ValueError("responses must be a contiguous float32 CUDA tensor")
            need = sum(len(scales) * f.shape[0] * f.shape[1] for f in frames)
            if responses.numel() < need:
                raise ValueError(f"responses needs {need} elements")
            o.responses = responses.data_ptr()
        self.threshold = float(threshold)
        self._last = (frames, scales, ftype, order, o, value_scales)
        kf_filter_bank(self.ctx, frames, scales, ftype, order, o, value_scales)

    def kernel_times(self) -> dict:
        return kf_kernel_times(self.ctx)

    def shapes(self, threshold=None) -> np.ndarray:
        """Shapes of the blobs `blobs(threshold)` returns (derivative bank)."""
        return kf_blob_shapes(self.ctx, self.threshold if threshold is None else threshold)

    def blobs(self, threshold=None, capacity=None) -> np.ndarray:
        """Blob list of the last run.  If the context's device candidate list
        overflowed (KF_ERERUN: the library has raised its capacity), the last
        run is repeated once on the same frames and the list read again."""
        thr = self.threshold if threshold is None else threshold
        try:
            return kf_detect_blobs(self.ctx, thr, capacity)
        except KfError as e:
            if e.code != KF_ERERUN or getattr(self, "_last", None) is None:
                raise
        kf_filter_bank(self.ctx, *self._last)
        return kf_detect_blobs(self.ctx, thr, capacity)

    def close(self):
        if self.ctx:
            kf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
