"""Python access to the FP64 CPU oracle (``kf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``; never by the product package.  The
oracle shares no code with the CUDA library.  It implements Kennedy,
"Digital filters with vanishing moments for shape analysis"
(arXiv:1912.07133): designs of Sec. 4 (Filters C, D, E), the three-term DE of
the Appendix (A6-A10, A17, A32), the separable bank and the detector of Sec. 5
(eqs 26-27).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libkforacle.so")
_lock = threading.Lock()
_lib = None

IIR_REPEATED_POLE = 0  # Filter D
IIR_BUTTERWORTH = 1  # Filter E
FIR_COLORED_SG = 2  # Filter C
FIR_GAUSSIAN = 3  # Filter A
RESP_LAPLACIAN = 0
RESP_HESSIAN = 1
BOUNDARY_HOLD = 0
BOUNDARY_ZERO = 1
NEIGH_ALL = 0
NEIGH_ADJACENT = 1
MAXK = 8


class Blob(ctypes.Structure):
    _fields_ = [
        ("frame", ctypes.c_int),
        ("x", ctypes.c_int),
        ("y", ctypes.c_int),
        ("scale", ctypes.c_int),
        ("polarity", ctypes.c_int),
        ("response", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("det", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "kf_oracle.h"))
    ):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i, l = ctypes.c_double, ctypes.c_int, ctypes.c_long
            P = ctypes.POINTER(ctypes.c_double)
            L.ko_eulerian.restype = d
            L.ko_eulerian.argtypes = [i, i]
            L.ko_li_neg.restype = d
            L.ko_li_neg.argtypes = [i, d]
            L.ko_solve.restype = i
            L.ko_solve.argtypes = [i, P, P]
            L.ko_poly_roots.restype = i
            L.ko_poly_roots.argtypes = [i, P, P, P]
            L.ko_a17.restype = i
            L.ko_a17.argtypes = [i, P, P, P, P, P, P, P, P]
            L.ko_design_repeated_pole.restype = i
            L.ko_design_repeated_pole.argtypes = [i, i, d, P, P, P, P]
            L.ko_design_butterworth.restype = i
            L.ko_design_butterworth.argtypes = [i, d, P, P, P, P]
            L.ko_design_colored_sg.restype = i
            L.ko_design_colored_sg.argtypes = [i, d, i, P]
            L.ko_design_colored_sg_raw.restype = i
            L.ko_design_colored_sg_raw.argtypes = [i, i, d, P]
            L.ko_design_gaussian.restype = i
            L.ko_design_gaussian.argtypes = [d, i, P]
            L.ko_iir1d.restype = None
            L.ko_iir1d.argtypes = [P, l, l, P, l, i, d, P, P, d, i]
            L.ko_fir1d.restype = None
            L.ko_fir1d.argtypes = [P, l, l, P, l, i, P, i]
            L.ko_bank.restype = i
            L.ko_bank.argtypes = [P, i, i, i, P, i, i, i, i, i, P,
                                  ctypes.POINTER(ctypes.c_int), i, P, P]
            L.ko_threads.restype = i
            L.ko_threads.argtypes = []
            L.ko_eq27.restype = None
            L.ko_eq27.argtypes = [d, d, d, d, d, P, P, P]
            L.ko_detect.restype = l
            L.ko_detect.argtypes = [P, P, i, i, i, d, i, i, d, i, ctypes.POINTER(Blob), l]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def eulerian(n: int, k: int) -> float:
    return lib().ko_eulerian(n, k)


def li_neg(n: int, z: float) -> float:
    return lib().ko_li_neg(n, z)


def solve(A, b) -> np.ndarray:
    A = _f64(A).copy()
    b = _f64(b).copy()
    if lib().ko_solve(len(b), _p(A), _p(b)):
        raise np.linalg.LinAlgError("singular")
    return b


def poly_roots(c) -> np.ndarray:
    c = _f64(c)
    d = len(c) - 1
    re = np.zeros(d)
    im = np.zeros(d)
    if lib().ko_poly_roots(d, _p(c), _p(re), _p(im)):
        raise ValueError("root finding failed")
    return re + 1j * im


def a17(b, a, aplus):
    """Three-part decomposition of eq (A17). Returns dict of arrays."""
    b, a, aplus = _f64(b), _f64(a), _f64(aplus)
    K = len(aplus) - 1
    bt = np.zeros(2 * K + 1)
    a0c = np.zeros(1)
    bp = np.zeros(K + 1)
    bm = np.zeros(K + 1)
    b0 = np.zeros(1)
    if lib().ko_a17(K, _p(b), _p(a), _p(aplus), _p(bt), _p(a0c), _p(bp), _p(bm), _p(b0)):
        raise np.linalg.LinAlgError("A17 solve failed")
    return dict(btilde=bt, a0circ=float(a0c[0]), bplus=bp, bminus=bm, b0=float(b0[0]))


def design_repeated_pole(L_D: int, Lpi: int, sigma: float):
    """Filter D (Sec. 4.3). Returns dict(K, b0, bplus, aplus, c)."""
    b0 = np.zeros(1)
    bp = np.zeros(MAXK + 1)
    ap = np.zeros(MAXK + 1)
    c = np.zeros(MAXK + 2)
    K = lib().ko_design_repeated_pole(L_D, Lpi, sigma, _p(b0), _p(bp), _p(ap), _p(c))
    if K < 0:
        raise ValueError("design failed")
    return dict(K=K, b0=float(b0[0]), bplus=bp[: K + 1].copy(), aplus=ap[: K + 1].copy(),
                c=c[: L_D + 1 + Lpi].copy(), p=float(np.exp(-1.0 / sigma)))


def design_butterworth(L_D: int, sigma: float):
    """Filter E (Sec. 4.4). Returns dict(K, b0, bplus, aplus, omega_c)."""
    b0 = np.zeros(1)
    bp = np.zeros(MAXK + 1)
    ap = np.zeros(MAXK + 1)
    wc = np.zeros(1)
    K = lib().ko_design_butterworth(L_D, sigma, _p(b0), _p(bp), _p(ap), _p(wc))
    if K < 0:
        raise ValueError("design failed")
    return dict(K=K, b0=float(b0[0]), bplus=bp[: K + 1].copy(), aplus=ap[: K + 1].copy(),
                omega_c=float(wc[0]))


def design_colored_sg(L_D: int, sigma: float, kmax: int = 0) -> np.ndarray:
    """Filter C (Sec. 4.2). Returns h[0..K] (h(-m) = h(m))."""
    K0 = int(np.ceil((5.0 if L_D == 1 else 7.0) * sigma)) + 1
    h = np.zeros(K0 + 1)
    K = lib().ko_design_colored_sg(L_D, sigma, kmax, _p(h))
    if K < 0:
        raise ValueError("design failed")
    return h[: K + 1].copy()


_MP_CACHE = {}


def design_colored_sg_mp(L_D: int, K: int, omega_c: float, dps: int = 40) -> np.ndarray:
    """Filter C (Sec. 4.2, eqs 16, 20-22) solved in `dps`-digit arithmetic.

    The KKT matrix of eq (20) is nearly singular when omega_c = 3/sigma
    approaches pi (condition number ~1e17 at sigma = 1), where an FP64 solve
    is not reproducible; 40 digits give the minimiser to full FP64 accuracy.
    Same steps as ko_design_colored_sg_raw: Sbar of eq (22b), S = T Sbar T^T
    (eq 22c), dc constraints of the pure-delay basis (eq 16c-d), eq (20)."""
    import mpmath as mp

    key = (L_D, K, float(omega_c), dps)
    if key in _MP_CACHE:
        return _MP_CACHE[key].copy()
    ctx = mp.MPContext()
    ctx.dps = dps
    wc = ctx.mpf(omega_c)
    NK, Ldc = K + 1, L_D + 1
    N = NK + Ldc

    def sbar(d):  # eq (22b); sin(pi d) = 0 for integer d
        if d == 0:
            return (ctx.pi - wc) / ctx.pi
        return (ctx.sin(ctx.pi * d) - ctx.sin(wc * d)) / (ctx.pi * d)

    sb = {d: sbar(d) for d in range(-2 * K, 2 * K + 1)}
    A = ctx.zeros(N, N)
    rhs = ctx.zeros(N, 1)
    for k1 in range(NK):
        for k2 in range(NK):
            v = 0
            for s1 in ((-1,) if k1 == 0 else (-1, 1)):
                for s2 in ((-1,) if k2 == 0 else (-1, 1)):
                    v += sb[s1 * k1 - s2 * k2]
            A[k1, k2] = v
    for lb in range(Ldc):
        for k in range(NK):
            mu = ctx.mpf(1) / 2 if k == 0 else 1
            v = 2 * mu * (-1) ** lb * (1 if lb == 0 else ctx.mpf(k) ** (2 * lb))
            A[NK + lb, k] = v
            A[k, NK + lb] = v
    rhs[NK] = 1
    x = ctx.lu_solve(A, rhs)
    h = np.array([float(x[k]) for k in range(NK)])
    _MP_CACHE[key] = h
    return h.copy()


def design_gaussian(sigma: float, kmax: int = 96) -> np.ndarray:
    """Filter A taps h[0..K] (Sec. 3.1, eqs 9 and 11, d = 0; K = ceil(5 sigma)
    capped at kmax)."""
    h = np.zeros(int(np.ceil(5.0 * sigma)) + 1)
    K = lib().ko_design_gaussian(float(sigma), int(kmax), _p(h))
    if K < 0:
        raise ValueError("design failed")
    return h[:K + 1].copy()


def sg_half_length(L_D: int, sigma: float, kmax: int = 96) -> int:
    K = int(np.ceil((5.0 if L_D == 1 else 7.0) * sigma))
    return min(K, kmax) if kmax > 0 else K


def design_colored_sg_raw(L_D: int, K: int, omega_c: float) -> np.ndarray:
    h = np.zeros(K + 1)
    if lib().ko_design_colored_sg_raw(L_D, K, omega_c, _p(h)) < 0:
        raise ValueError("design failed")
    return h


def iir1d(x, K, b0, bplus, aplus, sym=1.0, boundary=BOUNDARY_HOLD) -> np.ndarray:
    x = _f64(x)
    y = np.zeros_like(x)
    lib().ko_iir1d(_p(x), len(x), 1, _p(y), 1, K, b0, _p(_f64(bplus)), _p(_f64(aplus)),
                   sym, boundary)
    return y


def fir1d(x, h, boundary=BOUNDARY_HOLD) -> np.ndarray:
    x = _f64(x)
    h = _f64(h)
    y = np.zeros_like(x)
    lib().ko_fir1d(_p(x), len(x), 1, _p(y), 1, len(h) - 1, _p(h), boundary)
    return y


def bank(img, lambdas, ftype=IIR_REPEATED_POLE, order=3, resp=RESP_LAPLACIAN,
         boundary=BOUNDARY_HOLD, fir_kmax=96, want_d=False):
    """Responses R (S,H,W) and optionally derivatives D (S,5,H,W)."""
    img = _f64(img)
    H, W = img.shape
    lam = _f64(lambdas)
    S = len(lam)
    R = np.zeros((S, H, W))
    D = np.zeros((S, 5, H, W)) if want_d else None
    taps = tapK = None
    stride = 0
    if ftype == FIR_COLORED_SG:  # high-precision design (see design_colored_sg_mp)
        hs = []
        for l in lam:
            sigma = l / 2.0
            if not (3.0 / sigma < np.pi):
                raise ValueError("oracle bank: design failed")
            hs.append(design_colored_sg_mp(order, sg_half_length(order, sigma, fir_kmax), 3.0 / sigma))
        stride = max(len(h) for h in hs)
        taps = np.zeros((S, stride))
        for s, h in enumerate(hs):
            taps[s, :len(h)] = h
        tapK = (ctypes.c_int * S)(*[len(h) - 1 for h in hs])
    rc = lib().ko_bank(_p(img), H, W, S, _p(lam), ftype, order, resp, boundary, fir_kmax,
                       _p(taps) if taps is not None else None, tapK, stride,
                       _p(R), _p(D) if want_d else None)
    if rc:
        raise ValueError("oracle bank: design failed")
    return (R, D) if want_d else R


def blob_shape(d20, d02, d11, pol=1):
    """Shape of a detection (Sec. 5, the Hessian passage after eq 26): with
    H = [[D20, D11], [D11, D02]], P = (-pol H)^-1 is the covariance of the blob
    read as a pdf (pol = +1 bright, -1 dark).  Returns (p1, p2, theta, det):
    the eigenvalues of P, p1 >= p2 (pixels^2), the orientation of the p1
    eigenvector (radians from +x towards +y, in (-pi/2, pi/2]) and |H|;
    (nan, nan, nan, det) where -pol H is not positive definite.  A library
    symmetric eigen-solver is the step."""
    Hm = np.array([[d20, d11], [d11, d02]], dtype=np.float64)
    det = float(d20 * d02 - d11 * d11)
    M = -pol * Hm
    w = np.linalg.eigvalsh(M)
    if not (w[0] > 0.0):
        return float("nan"), float("nan"), float("nan"), det
    Pm = np.linalg.inv(M)
    vals, vecs = np.linalg.eigh(Pm)  # ascending
    v = vecs[:, 1]
    theta = math.atan2(v[1], v[0])
    if theta <= -math.pi / 2:
        theta += math.pi
    elif theta > math.pi / 2:
        theta -= math.pi
    return float(vals[1]), float(vals[0]), theta, det


def threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(lib().ko_threads())


def eq27(d10, d01, d20, d02, d11):
    """(dx, dy, det) of eqs (26)-(27)."""
    dx, dy, det = np.zeros(1), np.zeros(1), np.zeros(1)
    lib().ko_eq27(d10, d01, d20, d02, d11, _p(dx), _p(dy), _p(det))
    return float(dx[0]), float(dy[0]), float(det[0])


def detect(R, T, resp=RESP_LAPLACIAN, neigh=NEIGH_ALL, D=None, limit2=0.0, frame=0):
    """Blob list (numpy structured array) in (scale, y, x) order."""
    R = _f64(R)
    S, H, W = R.shape
    Dp = _p(_f64(D)) if D is not None else None
    cap = 1 << 16
    while True:
        out = (Blob * cap)()
        n = lib().ko_detect(_p(R), Dp, S, H, W, T, resp, neigh, limit2, frame, out, cap)
        if n <= cap:
            break
        cap = int(n)
    dt = np.dtype([("frame", "i4"), ("x", "i4"), ("y", "i4"), ("scale", "i4"),
                   ("polarity", "i4"), ("response", "f8"), ("dx", "f8"), ("dy", "f8"),
                   ("det", "f8")])
    arr = np.zeros(n, dtype=dt)
    for i in range(n):
        b = out[i]
        arr[i] = (b.frame, b.x, b.y, b.scale, b.polarity, b.response, b.dx, b.dy, b.det)
    return arr
