"""Pins of the proposal-network oracle (oracle/proposal.py) against what does not
come from it: a library convolution, finite differences of its own loss, the
closed form of Adam's first step, torch's bfloat16 conversion, brute-force
pooling and labels.  CPU only."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import proposal as P


def rand_params(rng, scale=0.3):
    return [(rng.normal(0, scale, w), rng.normal(0, 0.1, b)) for w, b in P.param_shapes()]


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 11, 14))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    got = P.conv3x3(x, W, b)
    for o in range(4):
        ref = b[o] + sum(correlate2d(x[i], W[o, i], mode="same", boundary="fill") for i in range(3))
        np.testing.assert_allclose(got[o], ref, rtol=0, atol=1e-12)


def test_pool8_is_the_block_mean_with_partial_edges():
    rng = np.random.default_rng(1)
    f = rng.uniform(size=(19, 30))
    p = P.pool8(f, 0.5)
    assert p.shape == (3, 4)
    assert p[0, 0] == pytest.approx(0.5 * f[:8, :8].mean(), abs=1e-15)
    assert p[2, 3] == pytest.approx(0.5 * f[16:19, 24:30].mean(), abs=1e-15)  # a 3 x 6 corner block


def test_maxpool8_takes_the_first_maximum():
    o = np.zeros((1, 16, 12))
    o[0, 3, 5] = 2.0
    o[0, 6, 1] = 2.0          # the same value later in row-major order
    o[0, 9, 10] = -1.0
    o[0, 8:16, 8:12] -= 5.0   # a partial 8 x 4 block, all negative
    o[0, 12, 9] = -0.5
    z, arg = P.maxpool8(o)
    assert z.shape == (1, 2, 2)
    assert z[0, 0, 0] == 2.0 and arg[0, 0, 0] == 3 * 12 + 5
    assert z[0, 1, 1] == -0.5 and arg[0, 1, 1] == 12 * 12 + 9


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.5e-3]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.bf16_round(x), ref)


def test_bce_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    z = rng.normal(size=(8, 2, 3))
    t = (rng.uniform(size=z.shape) < 0.3).astype(float)
    _, dz = P.bce(z, t, 7.0)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 1, 2), (7, 0, 1)]:
        zp, zm = z.copy(), z.copy()
        zp[idx] += h
        zm[idx] -= h
        fd = (P.bce(zp, t, 7.0)[0] - P.bce(zm, t, 7.0)[0]) / (2 * h)
        assert dz[idx] == pytest.approx(fd, rel=1e-7, abs=1e-12)


def test_network_gradient_matches_finite_differences():
    """Every parameter of a small network on two 16 x 24 pooled frames."""
    rng = np.random.default_rng(4)
    params = rand_params(rng)
    frames = [rng.normal(size=(16, 24)) for _ in range(2)]
    labels = [(rng.uniform(size=(8, 2, 3)) < 0.4).astype(float) for _ in range(2)]

    def loss(pr):
        tot = 0.0
        for p, t in zip(frames, labels):
            z, _ = P.forward(p, pr)
            tot += P.bce(z, t, 3.0)[0] / 2
        return tot

    grad = np.zeros(P.n_params())
    for p, t in zip(frames, labels):
        z, cache = P.forward(p, params)
        _, dz = P.bce(z, t, 3.0)
        grad += P.pack(P.backward(params, cache, dz / 2))
    flat = P.pack(params)
    h = 1e-6
    picks = rng.choice(flat.size, 120, replace=False)
    picks = np.concatenate([picks, [0, 159, 160, 2479, 2480, flat.size - 1]])  # layer boundaries and biases
    for k in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        fd = (loss(P.unpack(fp)) - loss(P.unpack(fm))) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=2e-5, abs=1e-9), k


def test_loss_and_grad_uses_bf16_weights():
    rng = np.random.default_rng(5)
    master = (rng.normal(0, 0.3, P.n_params())).astype(np.float32)
    frames = [rng.normal(size=(16, 16))]
    labels = [(rng.uniform(size=(8, 2, 2)) < 0.5).astype(float)]
    l, g = P.loss_and_grad(frames, labels, master, 2.0)
    params = P.unpack(P.bf16_round(master))
    z, cache = P.forward(frames[0], params)
    l2, dz = P.bce(z, labels[0], 2.0)
    assert l == pytest.approx(l2, rel=1e-15)
    np.testing.assert_allclose(g, P.pack(P.backward(params, cache, dz)), rtol=1e-14, atol=0)


def test_adam_first_step_closed_form():
    """m^ = g and v^ = g^2 on the first step: theta moves by lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    th1, m, v = P.adam(th, np.zeros(50), np.zeros(50), g, 1, 0.01)
    np.testing.assert_allclose(th1, th - 0.01 * g / (np.abs(g) + P.EPS), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_labels_mark_the_tile_and_scale_of_each_blob():
    rec = np.zeros(3, dtype=[("scale", "i4"), ("y", "i4"), ("x", "i4")])
    rec[:] = [(0, 0, 0), (2, 63, 64), (1, 130, 5)]
    t = P.labels(rec, 3, 131, 129)
    assert t.shape == (3, 3, 3)
    assert t[0, 0, 0] == 1 and t[2, 0, 1] == 1 and t[1, 2, 0] == 1
    assert t.sum() == 3


def test_parameter_count_and_packing():
    assert P.n_params() == 16 * 9 + 16 + 16 * 16 * 9 + 16 + 8 * 16 * 9 + 8 == 3640
    rng = np.random.default_rng(7)
    pr = rand_params(rng)
    back = P.unpack(P.pack(pr))
    for (w, b), (w2, b2) in zip(pr, back):
        np.testing.assert_array_equal(w, w2)
        np.testing.assert_array_equal(b, b2)
