"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Kennedy, "Digital filters with vanishing moments for shape analysis"
(arXiv:1912.07133).  Every test compares the oracle with something other than
itself: printed values (tests/golden/), closed forms printed in the paper,
invariants (vanishing moments, Nyquist zeros), textbook special cases, and
brute force on tiny inputs.  None of these needs a GPU.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import signal

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_printed_values.json")))


# ----------------------------------------------------------------------------
# helpers (test side only)
# ----------------------------------------------------------------------------
def ir_of_de(d, half=None):
    """Impulse response h(m), m = -half..half, of a designed IIR DE."""
    K = d["K"]
    if half is None:
        sigma = -1.0 / math.log(d["p"]) if "p" in d else 20.0
        half = int(80 * sigma) + 200
    x = np.zeros(2 * half + 1)
    x[half] = 1.0
    y = O.iir1d(x, K, d["b0"], d["bplus"], d["aplus"], 1.0, O.BOUNDARY_ZERO)
    return np.arange(-half, half + 1), y


def moment(m, h, l, alternate=False):
    w = (-1.0) ** np.abs(m) if alternate else 1.0
    terms = w * (m.astype(float) ** l) * h
    return terms.sum(), np.abs(terms).sum()


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------
def test_eulerian_numbers_known_rows():
    # <n,k> rows are 1; 1 1; 1 4 1; 1 11 11 1; 1 26 66 26 1 (OEIS A008292)
    assert [O.eulerian(3, k) for k in range(3)] == [1, 4, 1]
    assert [O.eulerian(4, k) for k in range(4)] == [1, 11, 11, 1]
    assert [O.eulerian(5, k) for k in range(5)] == [1, 26, 66, 26, 1]
    for n in range(1, 12):  # row sums are n!
        assert sum(O.eulerian(n, k) for k in range(n)) == math.factorial(n)


@pytest.mark.parametrize("z", [0.3, 0.8825, 0.97])
def test_polylog_negative_order_vs_brute_sum(z):
    m = np.arange(1, 40000, dtype=float)  # positive terms: the float sum is accurate
    for n in range(0, 9):
        brute = np.sum(m ** n * z ** m)
        assert O.li_neg(n, z) == pytest.approx(brute, rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("z", [Fraction(-1, 2), Fraction(-1, 5), Fraction(-7, 8)])
def test_polylog_negative_order_alternating_exact(z):
    for n in range(0, 9):
        exact = sum(Fraction(m) ** n * z ** m for m in range(1, 700))
        assert O.li_neg(n, float(z)) == pytest.approx(float(exact), rel=1e-12, abs=1e-14)


def test_dense_solver_against_numpy():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((9, 9))
    b = rng.standard_normal(9)
    np.testing.assert_allclose(O.solve(A, b), np.linalg.solve(A, b), rtol=1e-11)


def test_poly_roots_of_known_factors():
    roots = np.array([0.5, -0.25, 0.3 + 0.4j, 0.3 - 0.4j, 2.0])
    c = np.real(np.poly(roots)[::-1])
    got = O.poly_roots(c)
    for r in roots:  # every true root found, each exactly once
        dist = np.abs(got - r)
        assert dist.min() < 1e-12 and np.sum(dist < 1e-6) == 1


# ----------------------------------------------------------------------------
# Filter D (Sec. 4.3, Table IV)
# ----------------------------------------------------------------------------
def table_iv(p):
    """Closed form of Table IV (Sec. 5): DE of the (L_D, Lpi) = (1, 2) blur."""
    b0 = p ** 3 / 16 - 9 * p / 16 + 0.5
    b1 = 3 * p ** 4 / 32 - 3 * p ** 2 / 8 + 9 / 32
    b2 = -3 * p ** 5 / 32 + 9 * p ** 3 / 16 - 15 * p / 32
    b3 = p ** 6 / 32 - 9 * p ** 4 / 32 + 9 * p ** 2 / 32 - 1 / 32
    return b0, [0.0, b1, b2, b3], [1.0, -3 * p, 3 * p ** 2, -p ** 3]


@pytest.mark.parametrize("sigma", [1.0, 2.0, 3.0, 8.0, 12.0, 24.0, 32.0])
def test_filter_d_generic_design_matches_table_iv(sigma):
    d = O.design_repeated_pole(1, 2, sigma)
    b0, bp, ap = table_iv(math.exp(-1.0 / sigma))
    assert d["K"] == 3
    np.testing.assert_allclose(d["aplus"], ap, rtol=1e-13, atol=1e-15)
    scale = max(abs(b0), max(abs(v) for v in bp))
    np.testing.assert_allclose(d["bplus"], bp, rtol=0, atol=1e-10 * scale)
    assert d["b0"] == pytest.approx(b0, abs=1e-10 * scale)


def test_filter_d_printed_sigma8():
    g = GOLD["filter_D_sigma8"]
    d = O.design_repeated_pole(1, 2, g["sigma"])
    np.testing.assert_allclose(d["bplus"], g["bplus"], atol=5e-5)
    np.testing.assert_allclose(d["aplus"], g["aplus"], atol=5e-5)
    assert d["b0"] == pytest.approx(g["b0"], abs=5e-5)


@pytest.mark.parametrize("Lpi,sigma", [(2, 1.0), (2, 4.0), (2, 24.0), (3, 1.0), (3, 4.0),
                                       (3, 12.0), (3, 24.0), (3, 32.0)])
def test_filter_d_vanishing_moments_and_nyquist_zeros(Lpi, sigma):
    """eq (7): sum h = 1, sum m^2 h = 0; Nyquist constraints of eq (15b)."""
    d = O.design_repeated_pole(1, Lpi, sigma)
    m, h = ir_of_de(d)
    # the FP64 direct-form DE amplifies rounding by 1/A+(1) = (1-p)^-K: the
    # measured IR carries ~1e-12..3e-9 relative noise at K = 4, sigma = 24..32
    s, _ = moment(m, h, 0)
    assert s == pytest.approx(1.0, abs=1e-9)
    s, a = moment(m, h, 2)
    assert abs(s) <= 1e-8 * a
    for j in range(Lpi):
        s, a = moment(m, h, 2 * j, alternate=True)
        assert abs(s) <= 1e-9 * max(a, 1.0), (j, s, a)


@pytest.mark.parametrize("Lpi,sigma", [(2, 2.0), (2, 8.0), (3, 3.0), (3, 16.0)])
def test_filter_d_impulse_response_equals_basis_expansion(Lpi, sigma):
    """The realised three-term DE (A10, A17) reproduces eq (12a)/(23)."""
    d = O.design_repeated_pole(1, Lpi, sigma)
    m, h = ir_of_de(d)
    p, c = d["p"], d["c"]
    expect = np.zeros_like(h)
    am = np.abs(m).astype(float)
    for k in range(len(c) - 1):
        expect += c[k] * am ** k * p ** am
    expect[m == 0] += c[-1]
    np.testing.assert_allclose(h, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


# ----------------------------------------------------------------------------
# Appendix Example 1 (A20-A25) pins the three-part decomposition
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("p", [0.3, 0.7, 0.9])
def test_a17_blunt_exponential_closed_form(p):
    K = 3
    c0 = p ** 6 / 64 - 3 * p ** 5 / 32 + 15 * p ** 4 / 64 - 5 * p ** 3 / 16 \
        + 15 * p ** 2 / 64 - 3 * p / 32 + 1 / 64                         # (A22)
    b = c0 * np.array([1, 6, 15, 20, 15, 6, 1], float)                  # (A22)
    t1 = -(3 * p ** 5 + 9 * p ** 3 + 3 * p)
    a = np.array([-p ** 3, 3 * (p ** 4 + p ** 2), t1, p ** 6 + 9 * p ** 4 + 9 * p ** 2 + 1,
                  t1, 3 * (p ** 4 + p ** 2), -p ** 3])                  # (A22)
    aplus = np.array([1, -3 * p, 3 * p ** 2, -p ** 3])                  # (A23)
    r = O.a17(b, a, aplus)
    e_b0 = -p ** 3 / 32 + 3 * p ** 2 / 16 - 15 * p / 32 + 5 / 16         # (A25)
    e_b1 = -3 * p ** 4 / 64 + 3 * p ** 3 / 16 - 3 * p ** 2 / 16 - 3 * p / 16 + 15 / 64
    e_b2 = 3 * p ** 5 / 64 - 9 * p ** 4 / 32 + 15 * p ** 3 / 32 + 3 * p ** 2 / 16 \
        - 33 * p / 64 + 3 / 32
    e_b3 = -p ** 6 / 64 + 3 * p ** 5 / 32 - 15 * p ** 4 / 64 + 15 * p ** 2 / 64 \
        - 3 * p / 32 + 1 / 64
    # eq (A17) is ill conditioned for p -> 1; agreement to 1e-8 still pins its structure
    assert r["a0circ"] == pytest.approx(1.0, rel=1e-14)
    assert r["b0"] == pytest.approx(e_b0, rel=1e-8)
    np.testing.assert_allclose(r["bplus"][1:], [e_b1, e_b2, e_b3], rtol=1e-8)
    np.testing.assert_allclose(r["bminus"][1:], [e_b1, e_b2, e_b3], rtol=1e-8)


# ----------------------------------------------------------------------------
# Appendix Example 2 (A26-A31) and Filter E (Sec. 4.4)
# ----------------------------------------------------------------------------
def butterworth_k3_closed_form(w):
    d3 = w ** 3 + 4 * w ** 2 + 8 * w + 8
    a1 = (3 * w ** 3 + 4 * w ** 2 - 8 * w - 24) / d3                     # (A29)
    a2 = (3 * w ** 2 - 10 * w + 12) / (w ** 2 + 2 * w + 4)
    a3 = (w ** 3 - 4 * w ** 2 + 8 * w - 8) / d3
    a0c = d3 ** 2                                                        # (A30)
    bt_c = (3 * w ** 6 + 20 * w ** 5 + 64 * w ** 4 + 120 * w ** 3 + 128 * w ** 2 + 64 * w) / 3
    b1 = (4 * w ** 5 + 32 * w ** 4 + 104 * w ** 3 + 128 * w ** 2 + 64 * w) / (3 * a0c)  # (A31)
    b2 = (8 * w ** 5 + 32 * w ** 4 - 128 * w ** 2 - 128 * w) / (3 * a0c)
    b3 = (4 * w ** 5 - 8 * w ** 3 + 64 * w) / (3 * a0c)
    return [1.0, a1, a2, a3], a0c, bt_c, [0.0, b1, b2, b3]


@pytest.mark.parametrize("lam,tol", [(4.0, 1e-9), (8.0, 1e-8), (16.0, 1e-6)])
def test_a17_butterworth_example_closed_form(lam, tol):
    """A27 expansion -> oracle root finder (A19) + A17 solve vs A29-A31."""
    w = 1.0 / lam
    w6 = w ** 6
    b = w6 * np.array([1, 6, 15, 20, 15, 6, 1], float)                    # (A27)
    a = np.array([w6 - 64, 6 * w6 + 384, 15 * w6 - 960, 20 * w6 + 1280,
                  15 * w6 - 960, 6 * w6 + 384, w6 - 64])                  # (A27)
    roots = O.poly_roots(a)
    inside = roots[np.abs(roots) < 1]
    assert len(inside) == 3
    aplus = np.real(np.poly(inside))
    ap, a0c, bt_c, bp = butterworth_k3_closed_form(w)
    # roots of the A27 polynomial cluster near z = 1 as lam grows, and eq (A17)
    # is ill conditioned there: the tolerance widens with lam
    np.testing.assert_allclose(aplus, ap, atol=tol)
    r = O.a17(b, a, aplus)
    assert r["a0circ"] == pytest.approx(a0c, rel=tol)
    assert r["btilde"][3] == pytest.approx(bt_c, rel=tol)
    np.testing.assert_allclose(r["bplus"], bp, rtol=tol, atol=1e-14)
    # the centre coefficient of the DE is btilde_centre / a0circ (unity dc gain)
    assert r["b0"] == pytest.approx(bt_c / a0c, rel=tol)
    dc = r["b0"] + 2 * sum(bp) / sum(ap)
    assert dc == pytest.approx(1.0, abs=10 * tol)


@pytest.mark.parametrize("lam", [4.0, 8.0])
def test_filter_e_design_k3_matches_appendix_example(lam):
    """Sec. 4.4 route with L_D = 2 (L_B = 6) at omega_c = 1/lam equals A29-A31."""
    sigma = lam * math.sqrt(2 * math.log(2))  # omega_c = sqrt(2 ln 2)/sigma = 1/lam
    d = O.design_butterworth(2, sigma)
    ap, a0c, bt_c, bp = butterworth_k3_closed_form(1.0 / lam)
    assert d["K"] == 3
    np.testing.assert_allclose(d["aplus"], ap, atol=1e-12)
    np.testing.assert_allclose(d["bplus"], bp, atol=1e-13)
    assert d["b0"] == pytest.approx(bt_c / a0c, rel=1e-12)


def test_filter_e_printed_sigma8():
    g = GOLD["filter_E_sigma8"]
    d = O.design_butterworth(1, g["sigma"])
    assert d["omega_c"] == pytest.approx(g["omega_c"], abs=5e-5)
    assert d["omega_c"] / (2 * math.pi) == pytest.approx(g["f_c"], abs=5e-5)
    np.testing.assert_allclose(d["bplus"], g["bplus"], atol=5e-5)
    np.testing.assert_allclose(d["aplus"], g["aplus"], atol=5e-5)
    assert d["b0"] == pytest.approx(g["b0"], abs=5e-5)


@pytest.mark.parametrize("L_D,sigma", [(1, 1.0), (1, 8.0), (1, 24.0), (2, 6.0)])
def test_filter_e_frequency_response_is_bilinear_butterworth(L_D, sigma):
    """DTFT of the realised IR equals eq (25) under s = 2(z-1)/(z+1):
    H(e^iw) = 1 / (1 + (2 tan(w/2) / omega_c)^{L_B})."""
    d = O.design_butterworth(L_D, sigma)
    m, h = ir_of_de(dict(d, p=math.exp(-1.0 / (3 * sigma))), half=int(200 * sigma) + 400)
    LB = 2 * (L_D + 1)
    for w in [0.0, 0.05, 0.1, 0.3, 0.7, 1.5, 2.5, 3.0, math.pi]:
        H = np.sum(h * np.cos(m * w))
        expect = 1.0 / (1.0 + (2 * math.tan(w / 2) / d["omega_c"]) ** LB) if w < math.pi else 0.0
        assert H == pytest.approx(expect, abs=1e-11), w


@pytest.mark.parametrize("sigma", [1.0, 8.0, 24.0])
def test_filter_e_flatness_at_dc_and_nyquist(sigma):
    """Sec. 4.4: rho^dc_{0,l} = delta_{0,l} and rho^pi_{0,l} = 0 for l < L_B."""
    d = O.design_butterworth(1, sigma)
    m, h = ir_of_de(dict(d, p=math.exp(-1.0 / (3 * sigma))), half=int(200 * sigma) + 400)
    s, _ = moment(m, h, 0)
    assert s == pytest.approx(1.0, abs=1e-11)
    s, a = moment(m, h, 2)
    assert abs(s) <= 1e-10 * a
    for l in (0, 2):
        s, a = moment(m, h, l, alternate=True)
        assert abs(s) <= 1e-10 * max(a, 1.0)


# ----------------------------------------------------------------------------
# Filter C (Sec. 4.2)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("sigma,kmax", [(1.0, 0), (2.0, 0), (4.0, 0), (8.0, 0), (16.0, 96),
                                        (24.0, 96)])
def test_colored_sg_constraints(sigma, kmax):
    h = O.design_colored_sg(1, sigma, kmax)
    K = len(h) - 1
    expectK = min(math.ceil(5 * sigma), kmax) if kmax else math.ceil(5 * sigma)
    assert K == expectK
    m = np.arange(-K, K + 1)
    hh = h[np.abs(m)]
    s, _ = moment(m, hh, 0)
    assert s == pytest.approx(1.0, abs=1e-12)
    s, a = moment(m, hh, 2)
    assert abs(s) <= 1e-11 * a


@pytest.mark.parametrize("K", [2, 5, 12, 30])
def test_colored_sg_white_noise_limit_is_textbook_savitzky_golay(K):
    """omega_c -> 0 turns the CNG into the WNG (eq 18-19): classic quadratic SG."""
    h = O.design_colored_sg_raw(1, K, 0.0)
    m = np.arange(0, K + 1)
    textbook = (3 * (3 * K ** 2 + 3 * K - 1) - 15 * m ** 2) / ((2 * K - 1) * (2 * K + 1) * (2 * K + 3))
    np.testing.assert_allclose(h, textbook, atol=1e-13)
    # brute force: least-squares quadratic through 2K+1 points, evaluated at 0
    mm = np.arange(-K, K + 1, dtype=float)
    V = np.stack([np.ones_like(mm), mm, mm ** 2], axis=1)
    row = np.linalg.pinv(V)[0]
    np.testing.assert_allclose(h[np.abs(np.arange(-K, K + 1))], row, atol=1e-13)


def cng(hfull, m, wc, n=40001):
    w = np.linspace(wc, math.pi, n)
    H = (hfull[None, :] * np.cos(np.outer(w, m))).sum(axis=1)
    return np.trapezoid(H ** 2, w) / math.pi


@pytest.mark.parametrize("sigma", [2.0, 4.0])
def test_colored_sg_minimises_colored_noise_gain(sigma):
    """eq (21): the design is a constrained minimum of (1/pi) int_wc^pi |H|^2."""
    h = O.design_colored_sg(1, sigma)
    K = len(h) - 1
    m = np.arange(-K, K + 1)
    hfull = h[np.abs(m)]
    wc = 3.0 / sigma
    base = cng(hfull, m, wc)
    rng = np.random.default_rng(3)
    C = np.stack([np.ones(2 * K + 1), m.astype(float) ** 2])
    for _ in range(6):
        v = rng.standard_normal(K + 1)
        v = v[np.abs(m)]                       # symmetric perturbation
        v -= C.T @ np.linalg.lstsq(C.T, v, rcond=None)[0]  # keep the constraints
        v *= 1e-3 / np.abs(v).max()
        for sgn in (1, -1):
            assert cng(hfull + sgn * v, m, wc) > base * (1 - 1e-9)


# ----------------------------------------------------------------------------
# 1-D realisation: edge initialisation (Appendix, eq A32)
# ----------------------------------------------------------------------------
def test_iir_edge_hold_init_equals_paper_a32_tdf2_state():
    """Causal part with the oracle's edge-hold start equals a transposed
    direct-form II filter whose states are w0 = T v0 of eq (A32)."""
    d = O.design_repeated_pole(1, 2, 8.0)
    b1, b2, b3 = d["bplus"][1:]
    _, a1, a2, a3 = d["aplus"]
    rng = np.random.default_rng(11)
    x = rng.uniform(0, 1, 300)
    v0 = np.ones(3) * x[0] / (1 + a1 + a2 + a3)                     # (A32a)
    T = np.array([[b1, b2, b3],
                  [b2, b3 + a1 * b2 - a2 * b1, a1 * b3 - a3 * b1],
                  [b3, a1 * b3 - a3 * b1, a2 * b3 - a3 * b2]])      # (A32b)
    y_tdf, _ = signal.lfilter([0, b1, b2, b3], [1, a1, a2, a3], x, zi=T @ v0)
    y_or = O.iir1d(x, 3, 0.0, d["bplus"], d["aplus"], 0.0, O.BOUNDARY_HOLD)  # causal only
    np.testing.assert_allclose(y_or, y_tdf, rtol=0, atol=1e-13)


def test_iir_edge_hold_equals_long_constant_extension():
    d = O.design_repeated_pole(1, 3, 6.0)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200)
    n_ext = 6000
    xl = np.concatenate([np.full(n_ext, x[0]), x, np.full(n_ext, x[-1])])
    yl = O.iir1d(xl, d["K"], d["b0"], d["bplus"], d["aplus"], 1.0, O.BOUNDARY_ZERO)
    y = O.iir1d(x, d["K"], d["b0"], d["bplus"], d["aplus"], 1.0, O.BOUNDARY_HOLD)
    np.testing.assert_allclose(y, yl[n_ext:n_ext + len(x)], atol=1e-12)


def test_fir_boundaries_against_padding():
    h = O.design_colored_sg(1, 2.0)
    K = len(h) - 1
    hf = h[np.abs(np.arange(-K, K + 1))]
    x = np.random.default_rng(2).standard_normal(31)
    for bnd, mode in ((O.BOUNDARY_HOLD, "edge"), (O.BOUNDARY_ZERO, "constant")):
        xp = np.pad(x, K, mode=mode)
        expect = np.convolve(xp, hf, mode="valid")
        np.testing.assert_allclose(O.fir1d(x, h, bnd), expect, atol=1e-14)


# ----------------------------------------------------------------------------
# 2-D bank against brute-force direct 2-D convolution (Sec. 2, Fig. 5)
# ----------------------------------------------------------------------------
def one_d_ir(ftype, order, sigma):
    if ftype == O.FIR_GAUSSIAN:
        h = O.design_gaussian(sigma, 96)
        K = len(h) - 1
        return h[np.abs(np.arange(-K, K + 1))]
    if ftype == O.FIR_COLORED_SG:
        h = O.design_colored_sg_mp(order, O.sg_half_length(order, sigma, 96), 3.0 / sigma)
        K = len(h) - 1
        return h[np.abs(np.arange(-K, K + 1))]
    if ftype == O.IIR_REPEATED_POLE:
        d = O.design_repeated_pole(1, order - 1, sigma)
    else:
        d = O.design_butterworth(order - 1, sigma)
        d["p"] = math.exp(-1.0 / (3 * sigma))
    m, h = ir_of_de(d)
    keep = np.abs(h) >= 1e-17 * np.abs(h).max()
    lim = np.abs(m[keep]).max()
    return h[np.abs(m) <= lim]


def brute_response(img, ftype, order, lam, resp, boundary):
    sigma = lam / 2
    h1 = one_d_ir(ftype, order, sigma)
    M = (len(h1) - 1) // 2
    k2 = np.outer(h1, h1)
    mode = "edge" if boundary == O.BOUNDARY_HOLD else "constant"
    xp = np.pad(img, M + 1, mode=mode)
    B = signal.convolve2d(xp, k2, mode="valid")  # blur on [-1, H] x [-1, W]
    c = B[1:-1, 1:-1]
    d10 = 0.5 * (B[1:-1, 2:] - B[1:-1, :-2])
    d01 = 0.5 * (B[2:, 1:-1] - B[:-2, 1:-1])
    d20 = B[1:-1, 2:] - 2 * c + B[1:-1, :-2]
    d02 = B[2:, 1:-1] - 2 * c + B[:-2, 1:-1]
    d11 = 0.25 * (B[2:, 2:] - B[2:, :-2] - B[:-2, 2:] + B[:-2, :-2])
    if resp == O.RESP_HESSIAN:
        return sigma ** 4 * (d20 * d02 - d11 ** 2), (d10, d01, d20, d02, d11)
    return -sigma ** 2 * (d20 + d02), (d10, d01, d20, d02, d11)


@pytest.mark.parametrize("ftype,order,lam", [
    (O.IIR_REPEATED_POLE, 3, 4.0), (O.IIR_REPEATED_POLE, 4, 7.0),
    (O.IIR_BUTTERWORTH, 2, 4.0), (O.FIR_COLORED_SG, 1, 4.0), (O.FIR_COLORED_SG, 1, 6.0),
    (O.FIR_GAUSSIAN, 1, 4.0), (O.FIR_GAUSSIAN, 1, 5.0)])
@pytest.mark.parametrize("resp", [O.RESP_LAPLACIAN, O.RESP_HESSIAN])
def test_bank_equals_brute_force_2d_convolution(ftype, order, lam, resp):
    rng = np.random.default_rng(int(lam * 10) + ftype)
    img = rng.uniform(0, 1, (17, 23))
    R, D = O.bank(img, [lam], ftype, order, resp, O.BOUNDARY_HOLD, want_d=True)
    Rb, Db = brute_response(img, ftype, order, lam, resp, O.BOUNDARY_HOLD)
    # inputs are O(1): FP64 rounding of the DE and of the brute sum is ~1e-14
    np.testing.assert_allclose(R[0], Rb, rtol=0, atol=1e-9 * max(np.ptp(Rb), 1.0))
    for i in range(5):
        np.testing.assert_allclose(D[0, i], Db[i], rtol=0, atol=1e-11)


def test_bank_zero_boundary_equals_brute_force():
    img = np.random.default_rng(9).uniform(0, 1, (15, 19))
    for ftype, order in ((O.FIR_COLORED_SG, 1), (O.IIR_REPEATED_POLE, 3)):
        R = O.bank(img, [4.0], ftype, order, O.RESP_LAPLACIAN, O.BOUNDARY_ZERO)
        Rb, _ = brute_response(img, ftype, order, 4.0, O.RESP_LAPLACIAN, O.BOUNDARY_ZERO)
        np.testing.assert_allclose(R[0], Rb, rtol=0, atol=1e-9 * max(np.ptp(Rb), 1.0))


# ----------------------------------------------------------------------------
# derivative stage: polynomial inputs (eq 1-3, 7, Table II) and eq (27)
# ----------------------------------------------------------------------------
def test_hpf_taps_follow_table_i_convention():
    """D10 = sum_m h1(m) B(x-m) with Table I taps gives +d/dx on a ramp."""
    g = GOLD["table_I_hpf"]
    x = np.arange(-10, 11, dtype=float)
    B = 3.0 * x + 1.0
    m = np.array(g["m"])
    d1 = sum(hm * np.roll(B, mm) for hm, mm in zip(g["d1"], m))[5:-5]
    d2 = sum(hm * np.roll(B ** 2, mm) for hm, mm in zip(g["d2"], m))[5:-5]
    np.testing.assert_allclose(d1, 3.0)
    np.testing.assert_allclose(d2, 2 * 9.0)
    img = np.tile(3.0 * np.arange(40.0), (40, 1))
    _, D = O.bank(img, [2.0], O.FIR_COLORED_SG, 1, want_d=True)
    np.testing.assert_allclose(D[0, 0, 10:30, 10:30], 3.0, atol=1e-12)  # D10
    np.testing.assert_allclose(D[0, 1, 10:30, 10:30], 0.0, atol=1e-12)  # D01


@pytest.mark.parametrize("ftype,order,lam", [(O.FIR_COLORED_SG, 1, 2.0),
                                             (O.IIR_REPEATED_POLE, 3, 2.0),
                                             (O.IIR_REPEATED_POLE, 4, 2.0),
                                             (O.IIR_BUTTERWORTH, 2, 2.0)])
def test_quadratic_surface_exact_derivatives_and_eq27_offsets(ftype, order, lam):
    """Vanishing moments (eq 7) make the bank exact on a bivariate quadratic;
    eq (27) then points at the true stationary point."""
    H = W = 96
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    x0, y0 = 47.3, 48.6
    a, b, c = -0.02, 0.006, -0.015  # concave: a bright "blob"
    img = a * (xx - x0) ** 2 + b * (xx - x0) * (yy - y0) + c * (yy - y0) ** 2 + 1.0
    R, D = O.bank(img, [lam], ftype, order, O.RESP_HESSIAN, want_d=True)
    sl = (slice(40, 56), slice(40, 56))
    tol = 1e-9
    np.testing.assert_allclose(D[0, 2][sl], 2 * a, atol=tol)
    np.testing.assert_allclose(D[0, 3][sl], 2 * c, atol=tol)
    np.testing.assert_allclose(D[0, 4][sl], b, atol=tol)
    np.testing.assert_allclose(D[0, 0][sl], (2 * a * (xx - x0) + b * (yy - y0))[sl], atol=tol)
    np.testing.assert_allclose(D[0, 1][sl], (b * (xx - x0) + 2 * c * (yy - y0))[sl], atol=tol)
    for y in range(40, 56, 3):
        for x in range(40, 56, 3):
            dx, dy, det = O.eq27(*(D[0, i, y, x] for i in range(5)))
            assert det == pytest.approx(4 * a * c - b * b, rel=1e-8)
            assert x + dx == pytest.approx(x0, abs=1e-6)
            assert y + dy == pytest.approx(y0, abs=1e-6)


def test_detector_threshold2_uses_eq27_offsets():
    """Threshold #2 keeps the plateau pixel whose eq (27) offset is short."""
    R = np.full((1, 5, 5), 1.0)
    D = np.zeros((1, 5, 5, 5))
    D[0, 2], D[0, 3], D[0, 4] = -2.0, -2.0, 0.0       # D20, D02, D11: bright bowl
    yy, xx = np.mgrid[0:5, 0:5]
    x0, y0 = 3.2, 1.9
    D[0, 0] = -2.0 * (xx - x0)                        # D10 = D20 (x - x0)
    D[0, 1] = -2.0 * (yy - y0)
    R[0] = 1.0 + 1e-3 * np.exp(-((xx - 2) ** 2 + (yy - 2) ** 2))  # peak at (2, 2)
    assert _coords(O.detect(R, 0.5, O.RESP_HESSIAN, D=D, limit2=0.0)) == [(0, 2, 2, 1)]
    assert len(O.detect(R, 0.5, O.RESP_HESSIAN, D=D, limit2=1.0)) == 0   # |offset| = 1.4
    bl = O.detect(R, 0.5, O.RESP_HESSIAN, D=D, limit2=1.5)
    assert len(bl) == 1
    assert (bl[0]["dx"], bl[0]["dy"]) == pytest.approx((1.2, -0.1), abs=1e-12)


def test_cubic_is_not_exact_for_first_derivative():
    """Negative control (Table II: rho_{1,3} != 0): on x^3 the d = 1 filter
    returns 3x^2 + 1, not 3x^2; the d = 2 filter stays exact (6x)."""
    H, W = 30, 60
    x = np.arange(W, dtype=float) - 30.0
    img = np.tile(x ** 3, (H, 1)) * 1e-3
    _, D = O.bank(img, [2.0], O.FIR_COLORED_SG, 1, want_d=True)
    xs = x[10:50]
    np.testing.assert_allclose(D[0, 0, 15, 10:50], 1e-3 * (3 * xs ** 2 + 1), atol=1e-10)
    np.testing.assert_allclose(D[0, 2, 15, 10:50], 1e-3 * 6 * xs, atol=1e-10)


# ----------------------------------------------------------------------------
# detector rules (Sec. 5 Threshold #1; tie and border rules)
# ----------------------------------------------------------------------------
def _coords(bl):
    return [(int(b["scale"]), int(b["y"]), int(b["x"]), int(b["polarity"])) for b in bl]


def test_detector_plateau_keeps_first_in_scale_y_x_order():
    R = np.zeros((2, 5, 5))
    R[0, 2, 2] = R[0, 2, 3] = 1.0          # same-scale tie: earlier x wins
    R[1, 2, 2] = 1.0                        # cross-scale tie: scale 0 wins
    assert _coords(O.detect(R, 0.5)) == [(0, 2, 2, 1)]


def test_detector_border_pixels_and_threshold():
    R = np.zeros((1, 4, 6))
    R[0, 0, 0] = 0.9                        # corner: out-of-frame neighbours ignored
    R[0, 3, 5] = 0.5                        # exactly T: not above threshold
    R[0, 1, 3] = -0.8                       # dark blob (Laplacian response)
    assert _coords(O.detect(R, 0.5)) == [(0, 0, 0, 1), (0, 1, 3, -1)]
    assert _coords(O.detect(R, 0.5, resp=O.RESP_HESSIAN)) == [(0, 0, 0, 1)]


def test_detector_all_scales_versus_adjacent_scales():
    R = np.zeros((4, 5, 5))
    R[0, 2, 2] = 1.0
    R[3, 2, 2] = 2.0                        # two scales away
    assert _coords(O.detect(R, 0.1, neigh=O.NEIGH_ALL)) == [(3, 2, 2, 1)]
    assert _coords(O.detect(R, 0.1, neigh=O.NEIGH_ADJACENT)) == [(0, 2, 2, 1), (3, 2, 2, 1)]


def test_detector_diagonal_neighbour_suppresses():
    R = np.zeros((1, 5, 5))
    R[0, 1, 1] = 1.0
    R[0, 2, 2] = 1.5
    assert _coords(O.detect(R, 0.1)) == [(0, 2, 2, 1)]


@pytest.mark.parametrize("Lpi,sigma", [(2, 2.0), (3, 2.0), (3, 3.0)])
def test_filter_d_a17_route_matches_ir_route(Lpi, sigma):
    """Sec. 4.3 as printed: rearrange eq (12b)/(24) to B(z)/A(z) and solve eq
    (A17).  Built here independently (numpy polynomials) and compared with the
    oracle's DE, which takes the causal IR instead; equal where A17 is well
    conditioned."""
    d = O.design_repeated_pole(1, Lpi, sigma)
    K, p, c = d["K"], d["p"], d["c"]
    P = np.polynomial.polynomial
    one_minus_w_K = P.polypow([1.0, -1.0], K)
    aplus = P.polypow([1.0, -p], K)                      # coefficients of z^-m
    # Laurent polynomials as dicts power -> coefficient
    def lau(coeffs, sign):                               # sum c_j z^{sign*j}
        return {sign * j: v for j, v in enumerate(coeffs)}
    def mul(a, b):
        out = {}
        for i, x in a.items():
            for j, y in b.items():
                out[i + j] = out.get(i + j, 0.0) + x * y
        return out
    Ap, Am = lau(aplus, -1), lau(aplus, +1)
    A = mul(Ap, Am)
    B = {k: c[-1] * v for k, v in A.items()}
    for k in range(len(c) - 1):
        if k == 0:
            Nw = P.polypow([1.0, -1.0], K - 1)
        else:
            Ak = [O.eulerian(k, j) for j in range(k)]
            Nw = P.polymul(P.polymul([0.0, 1.0], Ak), P.polypow([1.0, -1.0], K - k - 1))
        Nw = np.asarray(Nw) * p ** np.arange(len(Nw))
        term = mul(lau(Nw, -1), Am)
        for kk, v in mul(lau(Nw, +1), Ap).items():
            term[kk] = term.get(kk, 0.0) + v
        if k == 0:
            for kk, v in A.items():
                term[kk] = term.get(kk, 0.0) - v
        for kk, v in term.items():
            B[kk] = B.get(kk, 0.0) + c[k] * v
    assert one_minus_w_K is not None
    b = np.array([B.get(i, 0.0) for i in range(-K, K + 1)])
    a = np.array([A.get(i, 0.0) for i in range(-K, K + 1)])
    r = O.a17(b, a, aplus)
    np.testing.assert_allclose(r["bplus"], d["bplus"], rtol=1e-9, atol=1e-15)
    assert r["b0"] == pytest.approx(d["b0"], rel=1e-9)


# ----------------------------------------------------------------------------
# Filter C in high precision (the design used by the oracle bank)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("sigma", [2.0, 4.0, 8.0])
def test_colored_sg_high_precision_matches_fp64_where_well_conditioned(sigma):
    K = math.ceil(5 * sigma)
    hmp = O.design_colored_sg_mp(1, K, 3.0 / sigma)
    h64 = O.design_colored_sg(1, sigma)
    np.testing.assert_allclose(hmp, h64, rtol=0, atol=1e-9 * np.abs(hmp).max())


@pytest.mark.parametrize("sigma", [1.0, 1.25, 1.5])
def test_colored_sg_high_precision_constraints_near_nyquist_cutoff(sigma):
    """omega_c = 3/sigma close to pi: the constraints of eq (20) still hold."""
    K = math.ceil(5 * sigma)
    h = O.design_colored_sg_mp(1, K, 3.0 / sigma)
    m = np.arange(-K, K + 1)
    hh = h[np.abs(m)]
    assert hh.sum() == pytest.approx(1.0, abs=1e-14)
    assert abs((m.astype(float) ** 2 * hh).sum()) <= 1e-13


def test_colored_sg_high_precision_white_noise_limit():
    K = 7
    h = O.design_colored_sg_mp(1, K, 0.0)
    m = np.arange(0, K + 1)
    textbook = (3 * (3 * K ** 2 + 3 * K - 1) - 15 * m ** 2) / ((2 * K - 1) * (2 * K + 1) * (2 * K + 3))
    np.testing.assert_allclose(h, textbook, atol=1e-15)


def test_colored_sg_high_precision_is_the_cng_minimum_at_sigma_1():
    """eq (21) evaluated by adaptive quadrature in 40 digits (independent of the
    Sbar closed form): perturbations that keep the constraints raise the CNG."""
    import mpmath as mp
    ctx = mp.MPContext()
    ctx.dps = 40
    sigma, K = 1.0, 5
    wc = 3.0 / sigma
    h = O.design_colored_sg_mp(1, K, wc)
    c = [ctx.mpf(float(v)) for v in h]  # FP64-rounded minimiser

    def cng(cc):
        f = lambda w: (cc[0] + 2 * sum(cc[k] * ctx.cos(k * w) for k in range(1, K + 1))) ** 2
        return ctx.quad(f, [wc, ctx.pi]) / ctx.pi

    base = cng(c)
    rng = np.random.default_rng(1)
    m = np.arange(K + 1, dtype=float)
    Cm = np.stack([np.r_[1.0, 2 * np.ones(K)], np.r_[0.0, 2 * m[1:] ** 2]])  # sum h, sum m^2 h
    for _ in range(3):
        v = rng.standard_normal(K + 1)
        v -= Cm.T @ np.linalg.lstsq(Cm.T, v, rcond=None)[0]
        v *= 1e-2 / np.abs(v).max()
        for sg in (1, -1):
            assert cng([c[k] + sg * ctx.mpf(float(v[k])) for k in range(K + 1)]) > base


# ----------------------------------------------------------------------------
# Filter A: the Gaussian FIR blur (Sec. 3.1, eqs 9-11, Table III)
# ----------------------------------------------------------------------------
def rho_dc(h_full, lmax=4):
    """rho_l = d^l/d omega^l of H(omega) = sum_m h(m) e^{-i omega m} at dc
    (the convention of Table III), l = 0..lmax; h_full on m = -K..K."""
    K = (len(h_full) - 1) // 2
    m = np.arange(-K, K + 1, dtype=float)
    return np.array([np.sum(h_full * (-1j * m) ** l) for l in range(lmax + 1)])


def full(h):
    K = len(h) - 1
    return h[np.abs(np.arange(-K, K + 1))]


def test_filter_a_one_stage_moments_match_table_iii():
    """sigma = 1, K = 5: rho_{0,l} printed to 4 decimals."""
    g = GOLD["table_III_gaussian_sigma1"]
    h = O.design_gaussian(g["sigma"], 96)
    assert len(h) - 1 == g["K"]
    rho = rho_dc(full(h))
    want = np.array(g["one_stage_d0"]["re"]) + 1j * np.array(g["one_stage_d0"]["im"])
    np.testing.assert_allclose(rho, want, rtol=0, atol=0.5e-4)


def test_filter_a_two_stage_moments_match_table_iii():
    """The Gaussian blur cascaded with the Table I taps (d = 1, 2): the italic
    rows of Table III."""
    g = GOLD["table_III_gaussian_sigma1"]
    t = GOLD["table_I_hpf"]
    h = full(O.design_gaussian(g["sigma"], 96))
    for d, key in ((1, "two_stage_d1"), (2, "two_stage_d2")):
        hpf = np.array(t["d%d" % d], dtype=float)  # m = -2..2
        bpf = np.convolve(h, hpf)  # m = -(K+2)..(K+2)
        rho = rho_dc(bpf)
        want = np.array(g[key]["re"]) + 1j * np.array(g[key]["im"])
        np.testing.assert_allclose(rho, want, rtol=0, atol=0.5e-4, err_msg="d = %d" % d)


@pytest.mark.parametrize("sigma,kmax", [(0.7, 96), (1.0, 96), (3.3, 96), (8.0, 96), (24.0, 96), (24.0, 40)])
def test_filter_a_taps_are_the_normalised_sampled_gaussian(sigma, kmax):
    """h(m) / h(0) = exp(-m^2 / 2 sigma^2) (eq 9c), unit dc gain (eq 11),
    K = ceil(5 sigma) capped at kmax."""
    h = O.design_gaussian(sigma, kmax)
    K = len(h) - 1
    assert K == min(math.ceil(5 * sigma), kmax)
    m = np.arange(K + 1, dtype=float)
    np.testing.assert_allclose(h / h[0], np.exp(-m * m / (2 * sigma * sigma)), rtol=1e-14, atol=0)
    assert h[0] + 2 * h[1:].sum() == pytest.approx(1.0, abs=1e-15)


def test_filter_a_moments_approach_the_continuous_gaussian():
    """Table III, analog column: rho_{0,2} = -sigma^2, rho_{0,4} = 3 sigma^4;
    sampling a wide Gaussian at 5 sigma leaves only the truncated tails."""
    for sigma in (4.0, 8.0):
        rho = rho_dc(full(O.design_gaussian(sigma, 200)))
        assert rho[2].real == pytest.approx(-sigma ** 2, rel=2e-5)
        assert rho[4].real == pytest.approx(3 * sigma ** 4, rel=2e-4)
        assert abs(rho[1]) < 1e-15 and abs(rho[3]) < 1e-12


# ----------------------------------------------------------------------------
# shape descriptors (Sec. 5: -H as the Fisher information of a blob read as a
# pdf, P = (-H)^-1 its covariance, principal axes from P's eigen-decomposition)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("a,b,theta", [(3.0, 1.0, 0.0), (5.0, 2.0, 0.3), (4.0, 4.0 / 3, -1.1), (2.0, 1.5, 1.2)])
def test_blob_shape_of_a_rotated_quadratic(a, b, theta):
    """I = -(u^2 / 2a^2 + v^2 / 2b^2), (u, v) the axes rotated by theta: its
    Hessian is -R diag(1/a^2, 1/b^2) R^T, so P = R diag(a^2, b^2) R^T."""
    c, s_ = math.cos(theta), math.sin(theta)
    R = np.array([[c, -s_], [s_, c]])
    Hm = -R @ np.diag([1 / a ** 2, 1 / b ** 2]) @ R.T
    p1, p2, th, det = O.blob_shape(Hm[0, 0], Hm[1, 1], Hm[0, 1], 1)
    assert p1 == pytest.approx(a * a, rel=1e-12) and p2 == pytest.approx(b * b, rel=1e-12)
    assert math.remainder(th - theta, math.pi) == pytest.approx(0.0, abs=1e-12)
    assert det == pytest.approx(1 / (a * a * b * b), rel=1e-12)
    # a dark blob (minimum) is the same surface negated
    q1, q2, tq, _ = O.blob_shape(-Hm[0, 0], -Hm[1, 1], -Hm[0, 1], -1)
    assert (q1, q2) == pytest.approx((p1, p2), rel=1e-12) and tq == pytest.approx(th, abs=1e-12)


def test_blob_shape_of_a_saddle_or_wrong_polarity_is_undefined():
    for args in [(-1.0, 1.0, 0.0, 1), (-1.0, -1.0, 0.0, -1), (1.0, 2.0, 3.0, 1)]:
        p1, p2, th, det = O.blob_shape(*args)
        assert math.isnan(p1) and math.isnan(p2) and math.isnan(th)


def test_blob_shape_of_a_blurred_gaussian_blob():
    """A Gaussian blob of covariance C blurred by the Gaussian of Filter A is a
    Gaussian of covariance C + sigma^2 I: at its centre the Hessian of the
    blur is -A (C + sigma^2 I)^-1, so P = (C + sigma^2 I) / A: the orientation
    and the axis ratio of C + sigma^2 I, up to sampling and truncation.  The
    Table I differences see a Gaussian of variance v as the continuous
    derivative times about 1 - 1/(4v) (v = 25 and 65 here): a bias of up to 1%
    per axis, a few milliradians on the angle."""
    H = W = 129
    y, x = np.mgrid[0:H, 0:W].astype(float)
    th, s1, s2 = 0.5, 7.0, 3.0
    c, s_ = math.cos(th), math.sin(th)
    R = np.array([[c, -s_], [s_, c]])
    C = R @ np.diag([s1 ** 2, s2 ** 2]) @ R.T
    Ci = np.linalg.inv(C)
    dx, dy = x - 64, y - 64
    img = np.exp(-0.5 * (Ci[0, 0] * dx * dx + 2 * Ci[0, 1] * dx * dy + Ci[1, 1] * dy * dy))
    lam = 8.0  # sigma = 4
    _, D = O.bank(img, [lam], O.FIR_GAUSSIAN, 1, want_d=True)
    d = D[0, :, 64, 64]
    p1, p2, theta, _ = O.blob_shape(d[2], d[3], d[4], 1)
    want = C + (lam / 2) ** 2 * np.eye(2)
    w, V = np.linalg.eigh(want)
    assert math.remainder(theta - math.atan2(V[1, 1], V[0, 1]), math.pi) == pytest.approx(0.0, abs=1e-2)
    assert p1 / p2 == pytest.approx(w[1] / w[0], rel=2e-2)


# ----------------------------------------------------------------------------
# Figs. 6 and 7 (Sec. 5): scale selectivity of the normalised Hessian with one
# scale-invariant Threshold #1, and Threshold #2 against detections on the
# tips of elongated blobs
# ----------------------------------------------------------------------------
def nearest(b, centres):
    return min((math.hypot(b["y"] - cy, b["x"] - cx), a, r) for cy, cx, a, r in centres)


# Threshold #1 per blur: the figures print none.  Each blur's normalised
# determinant at a matched ellipse's centre has its own level (D 0.037-0.055,
# C 0.134-0.226, E 0.071-0.102 on this pattern), and one value per blur
# separates it from every other maximum at all five scales.
FIG6 = {"D": (O.IIR_REPEATED_POLE, 3, 0.035), "C": (O.FIR_COLORED_SG, 1, 0.132),
        "E": (O.IIR_BUTTERWORTH, 2, 0.066)}


@pytest.mark.parametrize("blur", ["D", "C", "E"])
def test_fig6_each_scale_detects_the_centres_of_its_matched_ellipses(blur):
    """Axis ratio 2, axes 4..64 px, rotations 0..45 deg; Filter D (Table IV),
    C (colored SG, L_D = 1, K = ceil(5 sigma) up to 160) or E (Butterworth,
    L_B = 4), lambda = 4..64 one at a time: every detection lies at the
    centre of an ellipse whose semi-major axis equals lambda, and all four
    rotations are found, with one threshold for all scales."""
    from paper_1912_07133_gb300 import synthetic as SYN
    ft, order, T = FIG6[blur]
    img, centres = SYN.ellipse_pattern(2.0)
    for lam in (4, 8, 16, 32, 64):
        R = O.bank(img.astype(np.float64), [float(lam)], ft, order, O.RESP_HESSIAN, fir_kmax=160)
        b = O.detect(R, T, O.RESP_HESSIAN, O.NEIGH_ALL)
        near = [nearest(r, centres) for r in b]
        assert all(a == lam and d <= 0.05 * lam + 1.0 for d, a, _ in near), (lam, near)
        assert sorted(r for _, _, r in near) == [0, 15, 30, 45], lam


def test_fig7_threshold_2_keeps_only_the_centres_of_matched_ellipses():
    """Axis ratio 4, lambda = 16: Threshold #1 alone also fires on the tips of
    the longer ellipses; with Threshold #2 (offset limit 2 px) only the
    centres of the 16-px ellipses remain."""
    from paper_1912_07133_gb300 import synthetic as SYN
    img, centres = SYN.ellipse_pattern(4.0)
    R, D = O.bank(img.astype(np.float64), [16.0], O.IIR_REPEATED_POLE, 3, O.RESP_HESSIAN, want_d=True)
    t1 = [nearest(r, centres) for r in O.detect(R, 0.02, O.RESP_HESSIAN, O.NEIGH_ALL, D=D)]
    tips = [x for x in t1 if x[1] > 16 and x[0] > 0.3 * x[1]]
    assert len(tips) >= 8
    t12 = [nearest(r, centres) for r in O.detect(R, 0.02, O.RESP_HESSIAN, O.NEIGH_ALL, D=D, limit2=2.0)]
    assert t12 and all(a == 16 and d <= 1.0 for d, a, _ in t12)
