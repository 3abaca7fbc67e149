"""Test-side helpers: run the GPU bank through the C ABI, run the oracle on the
same seeded input, and compare responses and blob lists."""
import numpy as np

from oracle import oracle as O

# filter type ids are the same small integers on both sides of the comparison
OT = {0: O.IIR_REPEATED_POLE, 1: O.IIR_BUTTERWORTH, 2: O.FIR_COLORED_SG, 3: O.FIR_GAUSSIAN}
TOL = 1e-5  # max |err| / per-scale response range (FP32 path)


def to_device(f):
    """A host frame (numpy f32 / f16 / u16 array, or a CPU torch tensor, e.g.
    bfloat16) as a contiguous CUDA tensor of the same element type."""
    import torch

    if isinstance(f, torch.Tensor):
        return f.contiguous().cuda()
    a = np.ascontiguousarray(f)
    if a.dtype == np.uint16:  # through a same-size view: uint16 copies need no arithmetic support
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(a).cuda()


def gpu_bank(frames, scales, ftype, order, threshold=0.05, neigh=0, fir_kmax=96, storage=0,
             value_scales=None):
    import torch

    from paper_1912_07133_gb300 import kf

    ts = [to_device(f) for f in frames]
    n = sum(len(scales) * t.numel() for t in ts)
    R = torch.empty(n, device="cuda", dtype=torch.float32)
    bank = kf.Bank(0)
    bank.run(ts, scales, ftype, order, threshold=threshold, neighbourhood=neigh, responses=R,
             fir_kmax=fir_kmax, storage=storage, value_scales=value_scales)
    blobs = bank.blobs()
    torch.cuda.synchronize()
    Rh = R.cpu().numpy().astype(np.float64)
    out, off = [], 0
    for t in ts:
        k = len(scales) * t.numel()
        out.append(Rh[off:off + k].reshape(len(scales), *t.shape))
        off += k
    bank.close()
    return out, blobs


def oracle_bank(frame, scales, ftype, order, fir_kmax=96):
    return O.bank(frame.astype(np.float64), scales, OT[ftype], order, fir_kmax=fir_kmax)


def scale_errors(Rg, Ro):
    return [float(np.abs(Rg[s] - Ro[s]).max() / max(np.ptp(Ro[s]), 1e-300)) for s in range(len(Ro))]


def margin(R, s, y, x, pol, T, neigh=0):
    """Distance of (s, y, x, pol) from the candidate boundary in the oracle's R
    (positive: a candidate by that much; negative: rejected by that much)."""
    S, H, W = R.shape
    v = pol * R[s, y, x]
    m = v - T
    srange = range(S) if neigh == 0 else range(max(0, s - 1), min(S, s + 2))
    for t in srange:
        for yy in (y - 1, y, y + 1):
            for xx in (x - 1, x, x + 1):
                if (t, yy, xx) == (s, y, x) or not (0 <= yy < H and 0 <= xx < W):
                    continue
                m = min(m, v - pol * R[t, yy, xx])
    return m


def compare_blobs(got, Ro, T, neigh=0, frame=0, tol=TOL):
    """Blob lists must agree on every blob whose margin exceeds the tolerance;
    returns (n_oracle, n_gpu, n_differing_small_margin)."""
    ref = O.detect(Ro, T, O.RESP_LAPLACIAN, neigh)
    g = got[got["frame"] == frame]
    gs = {(int(b["scale"]), int(b["y"]), int(b["x"]), int(b["polarity"])) for b in g}
    rs = {(int(b["scale"]), int(b["y"]), int(b["x"]), int(b["polarity"])) for b in ref}
    ranges = np.array([np.ptp(Ro[s]) for s in range(len(Ro))])
    bound = 2 * tol * ranges.max()
    diff = gs ^ rs
    for key in diff:
        m = margin(Ro, *key, T, neigh)
        assert abs(m) <= bound, f"blob {key} differs with margin {m:.3e} > {bound:.3e}"
    # responses of the common blobs agree within the tolerance
    rmap = {(int(b["scale"]), int(b["y"]), int(b["x"]), int(b["polarity"])): b["response"] for b in ref}
    for b in g:
        key = (int(b["scale"]), int(b["y"]), int(b["x"]), int(b["polarity"]))
        if key in rmap:
            assert abs(float(b["response"]) - rmap[key]) <= tol * ranges[key[0]] * 1.01
    # list order: (frame, scale, y, x)
    keys = [(int(b["frame"]), int(b["scale"]), int(b["y"]), int(b["x"])) for b in got]
    assert keys == sorted(keys)
    return len(rs), len(gs), len(diff)
