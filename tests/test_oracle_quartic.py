"""Pins of the D = 5 oracle (oracle/quartic.py) to the paper and to
mathematics, independent of the oracle's own formulas.

* The differentiators of a D = 3 bank are Table I, with the dc derivatives of
  Table II; those of a D = 5 bank are the textbook five-point central
  differences, and differentiate every polynomial of degree <= 4 exactly.
* Each blur of a D = 5 bank is flat at dc to order 4 (moments 2 and 4 vanish,
  Sec. 4), and is not the unit impulse; Filter D with no Nyquist constraint is
  the unit impulse.
* Each differentiator-blur cascade has moments (-1)^d d! delta_{l,d}, l < 5.
* The bank reproduces the derivatives of a bivariate quartic exactly (FIR
  blur, interior), and equals a brute-force 2-D convolution of the outer
  product of the impulse responses over the held frame (all three blurs).
* Steering maps coefficients so that both polynomials of eq (1) agree at
  every point, reduces to the identity and to the quarter turn, and maps the
  Hessian by its congruence transform.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import quartic as Q

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.json")))

# Textbook central differences on five points (Taylor expansion to fourth
# order), correlation form: y(n) = sum_j g(j) x(n + j), j = -2..2.
FIVE_POINT = {
    0: [0, 0, 1, 0, 0],
    1: [1 / 12, -8 / 12, 0, 8 / 12, -1 / 12],
    2: [-1 / 12, 16 / 12, -30 / 12, 16 / 12, -1 / 12],
    3: [-1 / 2, 1, 0, -1, 1 / 2],
    4: [1, -4, 6, -4, 1],
}

BLURS = [(O.IIR_REPEATED_POLE, 3), (O.IIR_REPEATED_POLE, 4), (O.IIR_BUTTERWORTH, 3), (O.FIR_COLORED_SG, 2)]


def test_d3_differentiators_are_table_I():
    g = GOLD["table_I_hpf"]
    for d in range(3):
        h = Q.hpf_taps(d, 3)
        full = np.zeros(5)
        full[1:4] = h
        assert np.allclose(full, g[f"d{d}"], atol=1e-15), d


def test_d3_differentiators_have_the_table_II_moments():
    """rho_{d,l} = sum_m h(m) (-i m)^l (H^(l)(0) with H(w) = sum h(m) e^{-iwm})."""
    g = GOLD["table_II_rho_hpf"]
    m = np.arange(-1, 2)
    for d in range(3):
        h = Q.hpf_taps(d, 3)
        for l in range(5):
            rho = np.sum(h * (-1j * m) ** l)
            want = complex(*g[f"d{d}"][l])
            assert abs(rho - want) < 1e-12, (d, l, rho, want)


@pytest.mark.parametrize("d", range(5))
def test_d5_differentiators_are_five_point_central_differences(d):
    h = Q.hpf_taps(d, 5)
    assert len(h) == 5
    g = h[::-1]  # correlation form: g(j) = h(-j)
    assert np.allclose(g, FIVE_POINT[d], atol=1e-14)


@pytest.mark.parametrize("d", range(5))
def test_d5_differentiators_are_exact_on_quartics(d):
    rng = np.random.default_rng(d)
    a = rng.normal(size=5)  # p(t) = sum a_k t^k
    n = np.arange(-6, 9, dtype=float)
    x = sum(a[k] * n ** k for k in range(5))
    y = Q.conv_same(x, Q.hpf_taps(d, 5), axis=0)
    nn = n[2:-2]
    want = sum(a[k] * math.perm(k, d) * nn ** (k - d) for k in range(d, 5))
    assert np.allclose(y, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("ftype,order", BLURS)
@pytest.mark.parametrize("lam", [2.0, 6.0])
def test_blur_is_flat_to_order_four(ftype, order, lam):
    g = Q.Blur(ftype, order, lam).impulse_response(int(60 * lam) + 40)
    half = (len(g) - 1) // 2
    m = np.arange(-half, half + 1, dtype=float)
    for l in (0, 2, 4):
        scale = np.sum(np.abs(g) * np.abs(m) ** l)
        want = 1.0 if l == 0 else 0.0
        assert abs(np.sum(g * m ** l) - want) <= 1e-9 * max(scale, 1.0), (l, np.sum(g * m ** l))
    # a real blur: the sixth moment does not vanish and the IR spreads
    assert abs(np.sum(g * m ** 6)) > 1e-3 * np.sum(np.abs(g) * m ** 6)
    assert g[half] < 0.9


def test_filter_d_without_nyquist_constraints_is_the_impulse():
    """With L_D = 2 and no Nyquist constraint the three dc constraints on the
    three basis functions are met by the unit impulse alone (Sec. 4.3)."""
    d = O.design_repeated_pole(2, 0, 3.0)
    e = np.zeros(201)
    e[100] = 1.0
    y = O.iir1d(e, d["K"], d["b0"], d["bplus"], d["aplus"], 1.0, O.BOUNDARY_ZERO)
    assert np.allclose(y, e, atol=1e-12)
    with pytest.raises(ValueError):
        Q.Blur(O.IIR_REPEATED_POLE, 2, 6.0)


@pytest.mark.parametrize("ftype,order", BLURS)
def test_cascade_moments(ftype, order):
    g = Q.Blur(ftype, order, 4.0).impulse_response(300)
    for d in range(5):
        k = np.convolve(Q.hpf_taps(d, 5), g)
        half = (len(k) - 1) // 2
        m = np.arange(-half, half + 1, dtype=float)
        for l in range(5):
            want = (-1) ** d * math.factorial(d) if l == d else 0.0
            scale = np.sum(np.abs(k) * np.abs(m) ** l)
            assert abs(np.sum(k * m ** l) - want) <= 1e-9 * max(scale, 1.0), (d, l)


def quartic_surface(seed, H, W):
    rng = np.random.default_rng(seed)
    cx, cy = W / 2 + 0.3, H / 2 - 0.2
    coef = {(a, b): rng.normal() * 10.0 ** (-(a + b)) for a in range(5) for b in range(5 - a)}

    def P(da=0, db=0):
        yy, xx = np.mgrid[0:H, 0:W].astype(float)
        v = np.zeros((H, W))
        for (a, b), c in coef.items():
            if a >= da and b >= db:
                v += c * math.perm(a, da) * math.perm(b, db) * (xx - cx) ** (a - da) * (yy - cy) ** (b - db)
        return v
    return P


def test_fir_bank_is_exact_on_a_bivariate_quartic():
    H, W = 60, 56
    P = quartic_surface(4, H, W)
    lam = 2.5
    D = Q.quartic_bank(P(), [lam], O.FIR_COLORED_SG, 2)
    m = O.sg_half_length(2, lam / 2) + 3
    sl = (slice(m, H - m), slice(m, W - m))
    for c, (dx, dy) in enumerate(Q.CHANNELS):
        want = P(dx, dy)[sl]
        assert np.allclose(D[0, c][sl], want, rtol=1e-9, atol=1e-9 * np.max(np.abs(want))), (dx, dy)


@pytest.mark.parametrize("ftype,order,lam", [(O.FIR_COLORED_SG, 2, 2.0), (O.IIR_REPEATED_POLE, 3, 2.0),
                                             (O.IIR_REPEATED_POLE, 4, 3.0), (O.IIR_BUTTERWORTH, 3, 2.5)])
def test_bank_equals_brute_force_convolution_of_the_held_frame(ftype, order, lam):
    rng = np.random.default_rng(11)
    H, W = 9, 12
    img = rng.uniform(0, 1, (H, W))
    g = Q.Blur(ftype, order, lam).impulse_response(150)
    D = Q.quartic_bank(img, [lam], ftype, order)
    M = 160
    Xp = np.pad(img, M, mode="edge")  # the held frame, far enough
    for c, (dx, dy) in enumerate(Q.CHANNELS):
        kx, ky = np.convolve(Q.hpf_taps(dx), g), np.convolve(Q.hpf_taps(dy), g)
        K = (len(kx) - 1) // 2
        T = sum(ky[K + m] * Xp[M - m:M - m + H, :] for m in range(-K, K + 1))
        R = sum(kx[K + m] * T[:, M - m:M - m + W] for m in range(-K, K + 1))
        assert np.allclose(D[0, c], R, rtol=1e-12, atol=1e-12 * np.max(np.abs(R))), (dx, dy)


def test_steering_preserves_the_polynomial():
    rng = np.random.default_rng(5)
    beta = {ch: rng.normal() for ch in Q.CHANNELS}
    D = np.array([beta[(a, b)] * math.factorial(a) * math.factorial(b) for a, b in Q.CHANNELS])
    phi = 0.7
    Dt = Q.steer(D[:, None, None], phi)[:, 0, 0]
    bt = {(a, b): Dt[Q.channel_index(a, b)] / (math.factorial(a) * math.factorial(b)) for a, b in Q.CHANNELS}
    for _ in range(5):
        x, y = rng.normal(size=2)
        xt, yt = x * math.cos(phi) + y * math.sin(phi), -x * math.sin(phi) + y * math.cos(phi)
        raw = sum(beta[(a, b)] * xt ** a * yt ** b for a, b in Q.CHANNELS)
        steered = sum(bt[(a, b)] * x ** a * y ** b for a, b in Q.CHANNELS)
        assert abs(raw - steered) < 1e-12 * max(1.0, abs(raw))


def test_steering_special_angles():
    rng = np.random.default_rng(6)
    D = rng.normal(size=(15, 2, 3))
    assert np.allclose(Q.steer(D, 0.0), D, atol=1e-15)
    # quarter turn: x~ = y, y~ = -x, so beta~_{dy,dx} = (-1)^dy beta_{dx,dy}
    Dq = Q.steer(D, math.pi / 2)
    for dx, dy in Q.CHANNELS:
        assert np.allclose(Dq[Q.channel_index(dy, dx)], (-1) ** dy * D[Q.channel_index(dx, dy)], atol=1e-12)
    # order 1: the derivative along (cos phi, -sin phi)
    phi = 0.3
    Ds = Q.steer(D, phi)
    assert np.allclose(Ds[1], math.cos(phi) * D[1] - math.sin(phi) * D[2], atol=1e-14)


def test_steering_of_the_hessian_is_its_congruence_transform():
    """Order 2: with [x~, y~]^T = M [x, y]^T, M = [[cos, sin], [-sin, cos]], the
    Hessian of the polynomial in (x, y) is M^T H M, H = [[D20, D11], [D11, D02]]
    the Hessian in (x~, y~)."""
    rng = np.random.default_rng(12)
    D = rng.normal(size=(15, 1, 1))
    for phi in (0.3, 1.1, -2.4):
        c, s = math.cos(phi), math.sin(phi)
        M = np.array([[c, s], [-s, c]])
        Hm = np.array([[D[3, 0, 0], D[4, 0, 0]], [D[4, 0, 0], D[5, 0, 0]]])  # (2,0), (1,1), (0,2)
        Ht = M.T @ Hm @ M
        Ds = Q.steer(D, phi)[:, 0, 0]
        assert np.allclose([Ds[3], Ds[4], Ds[5]], [Ht[0, 0], Ht[0, 1], Ht[1, 1]], atol=1e-13)
        # the determinant and trace are invariant
        assert abs(Ds[3] * Ds[5] - Ds[4] ** 2 - np.linalg.det(Hm)) < 1e-12
        assert abs(Ds[3] + Ds[5] - np.trace(Hm)) < 1e-13


@pytest.mark.parametrize("order", [3, 4, 6])
def test_butterworth_is_flat_to_order_two_n_minus_one(order):
    """Filter E of order n = L_B / 2 (Sec. 4.4): |H| = (1 + (w/wc)^(2n))^(-1/2)
    before the bilinear map, flat at dc to order 2n - 1, so the moments 2, 4,
    .. 2n - 2 vanish and moment 2n does not."""
    g = Q.Blur(O.IIR_BUTTERWORTH, order, 5.0).impulse_response(600)
    half = (len(g) - 1) // 2
    m = np.arange(-half, half + 1, dtype=float)
    assert abs(np.sum(g) - 1.0) < 1e-9
    # relative to sum |g| |m|^l (dominated by the tails at high l): the
    # vanishing moments sit at rounding level, the first non-vanishing one
    # orders of magnitude above it
    for l in range(2, 2 * order, 2):
        scale = np.sum(np.abs(g) * np.abs(m) ** l)
        assert abs(np.sum(g * m ** l)) <= 1e-10 * scale, l
    l = 2 * order
    assert abs(np.sum(g * m ** l)) > 1e-8 * np.sum(np.abs(g) * np.abs(m) ** l)
