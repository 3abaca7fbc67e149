"""What the trained proposal network gains over the method without it.

The committed network (trained on clustered frames with seeds 1000-2999) gates
the banks on held-out clustered frames (seeds 5000-5003, never seen in
training or in the benchmark): the gated calls must keep at least 99% of the
plain banks' blobs (the spec recall bar), report no blob the plain bank
does not, and run the column pass on strictly fewer tiles -- here a small
fraction of them.  The selected column tiles follow on the host from the
network's logits (kf_proposal_logits) and the gate rule."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEEDS = (5000, 5001, 5002, 5003)
SIZE = 6144
EIGHT = [2.0 * 32.0 ** (s / 7.0) for s in range(8)]
T = 0.3
TW = 30


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as g
    g.build()
    from paper_1912_07133_gb300 import kf as K
    return K


def column_tiles(act, H, W, rows):
    """(selected, total) column tiles of width 30 and `rows` interior rows
    whose interior overlaps an active 64 x 64 tile."""
    sel = tot = 0
    for y0 in range(0, H, rows):
        for x0 in range(0, W, TW):
            y1, x1 = min(y0 + rows, H), min(x0 + TW, W)
            tot += 1
            sel += bool(act[y0 // 64:(y1 - 1) // 64 + 1, x0 // 64:(x1 - 1) // 64 + 1].any())
    return sel, tot


def test_trained_gate_keeps_recall_and_skips_most_column_tiles(kf):
    import torch

    from paper_1912_07133_gb300 import synthetic, train_proposal
    weights, p_gate, stats = train_proposal.load_weights()
    assert not (set(SEEDS) & set(range(stats["seeds"][0], stats["seeds"][1] + 1)))
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, weights)
    zthr = math.log(p_gate / (1 - p_gate))
    plain, gated = set(), set()
    sel_tiles = all_tiles = 0
    for seed in SEEDS:
        X = synthetic.clustered_frame_device(seed, SIZE, SIZE)
        # the gate's tile map on the host, from the network's logits
        pooled = torch.empty(((SIZE + 7) // 8) ** 2, device="cuda")
        kf.kf_proposal_pool(bank.ctx, [X], pooled)
        ph = (SIZE + 7) // 8
        z = torch.empty((1, 8, (ph + 7) // 8, (ph + 7) // 8), device="cuda")
        kf.kf_proposal_logits(bank.ctx, pooled.view(1, ph, ph), z)
        act = (z[0] > zthr).any(dim=0).cpu().numpy()  # KF_GATE_TILES: marked tiles only
        for bi, (ft, order, rows) in enumerate(((kf.KF_FIR_COLORED_SG, 1, 126), (kf.KF_IIR_REPEATED_POLE, 4, 64))):
            bank.run([X], EIGHT, ft, order, threshold=T, fir_kmax=96)
            plain |= {(seed, bi, int(b["scale"]), int(b["y"]), int(b["x"])) for b in bank.blobs()}
            bank.run([X], EIGHT, ft, order, threshold=T, fir_kmax=96, gate=kf.KF_GATE_TILES,
                     gate_threshold=p_gate)
            gated |= {(seed, bi, int(b["scale"]), int(b["y"]), int(b["x"])) for b in bank.blobs()}
            s, t = column_tiles(act, SIZE, SIZE, rows)
            sel_tiles += s
            all_tiles += t
    bank.close()
    assert plain, "the held-out frames have blobs"
    recall = len(plain & gated) / len(plain)
    share = sel_tiles / all_tiles
    print(f"trained gate: recall {recall:.4f} of {len(plain)} blobs, column pass on {share:.3%} of the tiles")
    assert gated <= plain  # every gated blob is the plain bank's blob
    assert recall >= 0.99
    assert sel_tiles < all_tiles and share < 0.5


def test_untrained_network_gains_nothing(kf):
    """The same gate with the network's initial weights (He-normal, the label
    prior as output bias) at the trained threshold: it either marks no tile
    (recall far below 0.99) or fails to skip -- training is what makes the
    gate both selective and faithful."""
    import torch

    from paper_1912_07133_gb300 import synthetic, train_proposal
    _, p_gate, stats = train_proposal.load_weights()
    w0 = train_proposal.init_weights(np.random.default_rng(1000), max(stats["label_prior"], 1e-4))
    bank = kf.Bank(0)
    kf.kf_proposal_set_weights(bank.ctx, w0)
    X = synthetic.clustered_frame_device(SEEDS[0], SIZE, SIZE)
    ft, order = kf.KF_IIR_REPEATED_POLE, 4
    bank.run([X], EIGHT, ft, order, threshold=T, fir_kmax=96)
    plain = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in bank.blobs()}
    bank.run([X], EIGHT, ft, order, threshold=T, fir_kmax=96, gate=kf.KF_GATE_TILES, gate_threshold=p_gate)
    gated = {(int(b["scale"]), int(b["y"]), int(b["x"])) for b in bank.blobs()}
    ph = (SIZE + 7) // 8
    pooled = torch.empty(ph * ph, device="cuda")
    kf.kf_proposal_pool(bank.ctx, [X], pooled)
    z = torch.empty((1, 8, (ph + 7) // 8, (ph + 7) // 8), device="cuda")
    kf.kf_proposal_logits(bank.ctx, pooled.view(1, ph, ph), z)
    share = float((z[0] > math.log(p_gate / (1 - p_gate))).any(dim=0).float().mean())
    bank.close()
    recall = len(plain & gated) / max(len(plain), 1)
    print(f"untrained gate: recall {recall:.4f}, marks {share:.3%} of the tiles")
    assert recall < 0.99 or share > 0.9
