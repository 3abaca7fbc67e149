"""The D = 5 derivative bank (L_D = 2) of Kennedy, "Digital filters with
vanishing moments for shape analysis" (arXiv:1912.07133), in FP64 on the CPU.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library.

* ``hpf_taps``: the FIR differentiators of Sec. 4.1 (eqs 12-17, pure-delay
  basis, dc constraints only: the differentiator is cascaded with a blur
  that is flat at dc, so no Nyquist constraint is imposed).
* ``Blur``: the blur of a D = 5 bank, flat at dc up to order 4 (L_D = 2):
  Filter D (Sec. 4.3), Filter E (Sec. 4.4, order L_B / 2 = L_D + 1) or
  Filter C (Sec. 4.2, L_D = 2, K = ceil(7 sigma), omega_c = 3 / sigma).
* ``quartic_bank``: the estimates of D_{dx,dy} (eq 3) for every dx + dy <= 4
  of the frame held at its edges, by separable filtering (Sec. 2): the
  differentiator then the blur along x, then along y.
* ``steer``: the rotated coefficients of eq (1) under the substitution of
  Sec. 2 (x~ = x cos phi + y sin phi, y~ = -x sin phi + y cos phi).

Conventions.  A 1-D filter h(m) acts by convolution, y(n) = sum_m h(m)
x(n - m), and its frequency response is H(w) = sum_m h(m) exp(-i w m), so that
the ideal d-th differentiator has H^(l)(0) = i^d d! delta_{l,d} (the rho of
eq 13).  Eq (16c) gives the response of the basis function f_k: the impulse
weighted mu_k sits at m = +(k + Delta_d) and the one weighted (-1)^Delta_d mu_k
at m = -(k + Delta_d).  (Eq 16a, read literally, places them mirrored, which
would flip the sign of every odd-order filter; eq 16c is taken as the
definition.)  x is the column index (along a row), y the row index.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

# derivative channels of the D = 5 bank: total order n = dx + dy = 0..4, and
# within an order dy = 0..n
CHANNELS = [(n - dy, dy) for n in range(5) for dy in range(n + 1)]


def channel_index(dx: int, dy: int) -> int:
    n = dx + dy
    return n * (n + 1) // 2 + dy


def hpf_taps(d: int, D: int = 5) -> np.ndarray:
    """Differentiator h_d(m), m = -K..K (index m + K), of a bank of D filters
    (D = 2 L_D + 1).  Sec. 4.1: with the pure-delay basis of eq (16), the
    constraints rho = F c of eqs (13)-(15) at dc only, l = 2 lbar + Delta_d
    for lbar < Lbar_dc = L_D - Delta_d + 1 (Sec. 4), so N_K = Lbar_dc and
    K^hpf = N_K + Delta_d - 1 (the text after eq 17)."""
    if D < 1 or D % 2 == 0 or not 0 <= d < D:
        raise ValueError("D must be odd and 0 <= d < D")
    L_D = (D - 1) // 2
    delta = d % 2
    NK = L_D - delta + 1
    F = np.zeros((NK, NK), dtype=complex)
    rho = np.zeros(NK, dtype=complex)
    for lbar in range(NK):
        l = 2 * lbar + delta
        for k in range(NK):
            mu = 0.5 if (k == 0 and delta == 0) else 1.0  # eq (16d)
            n = k + delta
            # l-th derivative at w = 0 of mu (exp(-i n w) + (-1)^Delta exp(i n w)), eq (15a)
            F[lbar, k] = mu * ((-1j * n) ** l + (-1) ** delta * (1j * n) ** l)
        if l == d:
            rho[lbar] = (1j ** d) * math.factorial(d)
    c = np.linalg.solve(F, rho)
    if np.max(np.abs(c.imag)) > 1e-12 * max(1.0, np.max(np.abs(c.real))):
        raise ArithmeticError("differentiator coefficients are not real")
    c = c.real
    K = NK + delta - 1
    h = np.zeros(2 * K + 1)
    for k in range(NK):
        mu = 0.5 if (k == 0 and delta == 0) else 1.0
        n = k + delta
        h[K + n] += mu * c[k]
        h[K - n] += (-1) ** delta * mu * c[k]
    return h


def conv_same(x: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """y(n) = sum_m h(m) x(n - m) along `axis` for the samples whose whole
    window lies inside x (the output is 2K shorter)."""
    K = (len(h) - 1) // 2
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    N = x.shape[-1]
    y = np.zeros(x.shape[:-1] + (N - 2 * K,))
    for m in range(-K, K + 1):
        y += h[K + m] * x[..., K - m:N - K - m]
    return np.moveaxis(y, -1, axis)


class Blur:
    """The blur of a D = 5 bank at one scale lambda (sigma = lambda / 2)."""

    def __init__(self, ftype: int, order: int, lam: float, fir_kmax: int = 96):
        sigma = lam / 2.0
        self.ftype = ftype
        if ftype == O.IIR_REPEATED_POLE:
            # order = K^lpf = L_D + Lbar_pi with L_D = 2 (Sec. 4.3); with no
            # Nyquist constraint (order 2) the dc constraints alone give the
            # unit impulse, so at least one is required
            if order < 3:
                raise ValueError("Filter D of a D = 5 bank needs order >= 3")
            d = O.design_repeated_pole(2, order - 2, sigma)
        elif ftype == O.IIR_BUTTERWORTH:
            # order = L_B / 2 = L_D + 1 >= 3 (Sec. 4.4): flat to order 2 L_B / 2 - 1
            if order < 3:
                raise ValueError("Filter E of a D = 5 bank needs order >= 3")
            d = O.design_butterworth(order - 1, sigma)
        elif ftype == O.FIR_COLORED_SG:
            if order != 2:
                raise ValueError("Filter C of a D = 5 bank needs L_D = 2")
            K = O.sg_half_length(2, sigma, fir_kmax)
            self.h = O.design_colored_sg_mp(2, K, 3.0 / sigma)
            return
        else:
            raise ValueError("the D = 5 bank needs a blur with vanishing moments (Filters C, D, E)")
        self.K, self.b0, self.bplus, self.aplus = d["K"], d["b0"], d["bplus"], d["aplus"]

    def __call__(self, x: np.ndarray) -> np.ndarray:
        """The blur of the sequence x held beyond both ends."""
        if self.ftype == O.FIR_COLORED_SG:
            return O.fir1d(x, self.h, O.BOUNDARY_HOLD)
        return O.iir1d(x, self.K, self.b0, self.bplus, self.aplus, 1.0, O.BOUNDARY_HOLD)

    def impulse_response(self, half: int) -> np.ndarray:
        """IR g(m), m = -half..half, of the blur on an unbounded sequence."""
        if self.ftype == O.FIR_COLORED_SG:
            K = len(self.h) - 1
            g = np.zeros(2 * half + 1)
            for m in range(-min(K, half), min(K, half) + 1):
                g[half + m] = self.h[abs(m)]
            return g
        e = np.zeros(4 * half + 1)
        e[2 * half] = 1.0
        y = O.iir1d(e, self.K, self.b0, self.bplus, self.aplus, 1.0, O.BOUNDARY_ZERO)
        return y[half:3 * half + 1].copy()


def quartic_bank(img, lambdas, ftype=O.IIR_REPEATED_POLE, order=4, fir_kmax=96) -> np.ndarray:
    """D_{dx,dy} estimates, array (S, 15, H, W) in the order of CHANNELS.

    The frame X is held beyond its edges (the hold boundary of the Appendix,
    A32).  For each channel: g_dx along x on the held frame (the differentiator
    reads two columns beyond the edge, so its output is formed on x = -2 ..
    W + 1, and beyond that it is constant), the blur along x over that held
    sequence, then g_dy along y on the rows held beyond the top and bottom
    (formed on y = -2 .. H + 1) and the blur along y."""
    X = np.asarray(img, dtype=np.float64)
    H, W = X.shape
    lam = [float(v) for v in lambdas]
    taps = [hpf_taps(d, 5) for d in range(5)]
    Xp = np.pad(X, ((0, 0), (4, 4)), mode="edge")  # columns -4 .. W + 3
    out = np.zeros((len(lam), len(CHANNELS), H, W))
    for s, l in enumerate(lam):
        blur = Blur(ftype, order, l, fir_kmax)
        # along x: U(y, x) for x = -2 .. W + 1, then the blur, kept on 0 .. W - 1
        ux = {}
        for dx in range(5):
            U = conv_same(Xp, taps[dx], axis=1)  # columns -2 .. W + 1
            ux[dx] = np.stack([blur(U[y])[2:W + 2] for y in range(H)])
        for c, (dx, dy) in enumerate(CHANNELS):
            Vp = np.pad(ux[dx], ((4, 4), (0, 0)), mode="edge")  # rows -4 .. H + 3
            V = conv_same(Vp, taps[dy], axis=0)  # rows -2 .. H + 1
            out[s, c] = np.stack([blur(V[:, x])[2:H + 2] for x in range(W)], axis=1)
    return out


def steer_matrix(n: int, phi: float) -> np.ndarray:
    """M with beta~_{a,n-a} = sum_b M[a', b'] beta_{b,n-b} for the coefficients
    of total order n (Sec. 2, after eq 3): the coefficient of x^a y^(n-a) in
    (x cos phi + y sin phi)^dx (-x sin phi + y cos phi)^dy, with rows indexed
    by the steered dy~ = n - a and columns by the raw dy (the CHANNELS order
    within an order)."""
    cph, sph = math.cos(phi), math.sin(phi)
    M = np.zeros((n + 1, n + 1))
    for dy in range(n + 1):
        dx = n - dy
        # (x c + y s)^dx = sum_i C(dx, i) (x c)^(dx-i) (y s)^i
        # (-x s + y c)^dy = sum_j C(dy, j) (-x s)^(dy-j) (y c)^j
        for i in range(dx + 1):
            for j in range(dy + 1):
                ypow = i + j
                coef = (math.comb(dx, i) * cph ** (dx - i) * sph ** i *
                        math.comb(dy, j) * (-sph) ** (dy - j) * cph ** j)
                M[ypow, dy] += coef
    return M


def steer(D: np.ndarray, phi: float) -> np.ndarray:
    """Steered derivative estimates from raw ones (array (..., 15, H, W) in the
    CHANNELS order): beta = D / (dx! dy!) (eq 2) of each order n is mapped by
    steer_matrix(n, phi), and returned as D~ = beta~ dx~! dy~!."""
    D = np.asarray(D, dtype=np.float64)
    out = np.zeros_like(D)
    for n in range(5):
        M = steer_matrix(n, phi)
        idx = [channel_index(n - dy, dy) for dy in range(n + 1)]
        fac = np.array([math.factorial(n - dy) * math.factorial(dy) for dy in range(n + 1)], dtype=np.float64)
        beta = D[..., idx, :, :] / fac[:, None, None]
        bt = np.einsum("ab,...bhw->...ahw", M, beta)
        out[..., idx, :, :] = bt * fac[:, None, None]
    return out
