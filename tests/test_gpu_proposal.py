"""The proposal network's kernels against the FP64 oracle (oracle/proposal.py).

Bars (FP32 sums of bf16 x FP32 products against FP64 with the same bf16
weights): pooled frames 1e-6 relative; logits 1e-5 of the largest logit;
gradients 1e-4 of the layer's largest gradient entry; the Adam step exactly
as its formula with the kernel's own gradient; labels bit-exact.
"""
import numpy as np
import pytest

from oracle import proposal as P
from paper_1912_07133_gb300 import synthetic as SY
from tests.parity import to_device

pytestmark = pytest.mark.gpu

LAYERS = [(0, 144), (144, 160), (160, 2464), (2464, 2480), (2480, 3632), (3632, 3640)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def weights(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    params = [(rng.normal(0, scale, w), rng.normal(0, 0.05, b)) for w, b in P.param_shapes()]
    return P.pack(params).astype(np.float32)


def test_pool_matches_the_oracle():
    import torch

    from paper_1912_07133_gb300 import kf
    frames = [SY.tiny_frame(1, 61, 90, 3), SY.counts_frame(seed=2, H=40, W=33, nblobs=2)]
    vs = [1.0, 1.0 / 4095.0]
    ts = [to_device(f) for f in frames]
    n = sum(int(np.prod(kf.pooled_shape(*f.shape))) for f in frames)
    out = torch.full((n,), float("nan"), device="cuda")
    bank = kf.Bank(0)
    kf.kf_proposal_pool(bank.ctx, ts, out, vs)
    got = out.cpu().numpy()
    off = 0
    for f, v in zip(frames, vs):
        ref = P.pool8(f, np.float64(np.float32(v)))
        k = ref.size
        np.testing.assert_allclose(got[off:off + k].reshape(ref.shape), ref, rtol=1e-6, atol=1e-7)
        off += k
    bank.close()


@pytest.mark.parametrize("h,w", [(24, 40), (21, 37)])
def test_logits_match_the_oracle(h, w):
    import torch

    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(h * w)
    x = rng.normal(0, 1, (2, h, w)).astype(np.float32)
    W = weights(3)
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, W)
    th, tw = -(-h // 8), -(-w // 8)
    z = torch.full((2, 8, th, tw), float("nan"), device="cuda")
    kf.kf_proposal_logits(bank.ctx, torch.from_numpy(x).cuda(), z)
    zg = z.cpu().numpy().astype(np.float64)
    params = P.unpack(P.bf16_round(W))
    for n in range(2):
        zo, _ = P.forward(x[n].astype(np.float64), params)
        assert np.abs(zg[n] - zo).max() <= 1e-5 * np.abs(zo).max()
    assert np.array_equal(kf.kf_proposal_get_weights(bank.ctx), W)
    bank.close()


def test_gradient_matches_the_oracle():
    import torch

    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(5)
    h, w = 32, 48
    x = rng.normal(0, 1, (3, h, w)).astype(np.float32)
    t = (rng.uniform(size=(3, 8, 4, 6)) < 0.2).astype(np.uint8)
    W = weights(6)
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, W)
    loss, g = kf.kf_proposal_grad(bank.ctx, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), 5.0)
    lo, go = P.loss_and_grad([xi.astype(np.float64) for xi in x], [ti.astype(np.float64) for ti in t], W, 5.0)
    assert loss == pytest.approx(lo, rel=1e-5)
    for a, b in LAYERS:
        scale = np.abs(go[a:b]).max()
        assert np.abs(g[a:b] - go[a:b]).max() <= 1e-4 * scale, (a, b)
    bank.close()


def test_adam_steps_follow_the_formula():
    """Two steps: the masters move exactly as Adam with the kernel's gradients."""
    import torch

    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.normal(0, 1, (2, 16, 24)).astype(np.float32)).cuda()
    t = torch.from_numpy((rng.uniform(size=(2, 8, 2, 3)) < 0.3).astype(np.uint8)).cuda()
    W = weights(8)
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, W)
    th = W.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for k in (1, 2):
        _, g = kf.kf_proposal_grad(bank.ctx, x, t, 4.0)
        kf.kf_proposal_train_step(bank.ctx, x, t, 4.0, 1e-3)
        th, m, v = P.adam(th, m, v, g.astype(np.float64), k, 1e-3)
        got = kf.kf_proposal_get_weights(bank.ctx).astype(np.float64)
        np.testing.assert_allclose(got, th, rtol=0, atol=2e-6)
    bank.close()


def test_labels_match_the_blob_list():
    import torch

    from paper_1912_07133_gb300 import kf
    frames = [SY.tiny_frame(11, 200, 300, 12), SY.tiny_frame(12, 130, 70, 4)]
    ts = [to_device(f) for f in frames]
    scales = [2.0, 4.0, 8.0]
    bank = kf.Bank(0)
    bank.run(ts, scales, kf.KF_IIR_REPEATED_POLE, 4, threshold=0.05)
    blobs = bank.blobs(0.08)
    sizes = [len(scales) * -(-f.shape[0] // 64) * -(-f.shape[1] // 64) for f in frames]
    lab = torch.full((sum(sizes),), 7, dtype=torch.uint8, device="cuda")
    kf.kf_proposal_labels(bank.ctx, 0.08, lab)
    got = lab.cpu().numpy()
    off = 0
    for i, f in enumerate(frames):
        ref = P.labels(blobs[blobs["frame"] == i], len(scales), *f.shape)
        assert np.array_equal(got[off:off + ref.size].reshape(ref.shape), ref), i
        off += ref.size
    assert got.sum() > 0
    bank.close()


def test_training_reduces_the_loss():
    """Fifty Adam steps on one batch bring the loss down (learning happens)."""
    import torch

    from paper_1912_07133_gb300 import kf
    rng = np.random.default_rng(9)
    x = rng.normal(0, 0.1, (4, 32, 32)).astype(np.float32)
    t = np.zeros((4, 8, 4, 4), np.uint8)
    for n in range(4):  # bright spots mark their tile at channel n
        ty, tx = rng.integers(4, size=2)
        x[n, 8 * ty + 3:8 * ty + 5, 8 * tx + 3:8 * tx + 5] += 2.0
        t[n, n, ty, tx] = 1
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, weights(10, 0.1))
    first = kf.kf_proposal_train_step(bank.ctx, xd, td, 10.0, 3e-3)
    for _ in range(48):
        kf.kf_proposal_train_step(bank.ctx, xd, td, 10.0, 3e-3, want_loss=False)
    last = kf.kf_proposal_train_step(bank.ctx, xd, td, 10.0, 3e-3)
    assert last < 0.5 * first
    bank.close()
