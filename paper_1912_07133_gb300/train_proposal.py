"""Train the gating network of the filter bank on generated frames.

  python -m paper_1912_07133_gb300.train_proposal [--frames 2000] [--size 6144]
         [--epochs 10] [--out paper_1912_07133_gb300/proposal_weights.npz]

Frames: the clustered recipe (1/f background, blob clusters in about 5% of the
64 x 64 tiles), generated on the GPU, seeds 1000, 1001, ...  Labels: the tiles
and scales where the plain colored Savitzky-Golay bank (K <= 96) or the
fourth-order repeated-pole bank, at 8 scales (blob radii 2-64 px) and
threshold 0.3, report a blob (kf_proposal_labels).  At 0.3 the 1/f
background alone (std 0.1) gives no detections; at 0.05 it gives some in
every tile, and there would be nothing to gate.  Input: the 8 x 8 pooled
frame (kf_proposal_pool).  Every forward, backward and Adam step runs in the
library's kernels (kf_proposal_train_step).  The last tenth of the frames is
held out: the saved gate threshold is the largest probability whose dilated
tile map still covers the required share of the labelled tiles there.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "proposal_weights.npz")
SCALES = tuple(2.0 * 32.0 ** (s / 7.0) for s in range(8))
THRESHOLD = 0.3
BANKS = ((2, 1), (0, 4))  # colored SG (K <= 96), repeated pole order 4


def init_weights(rng, prior):
    """He-normal weights, zero biases; the last bias starts at the label prior."""
    out = []
    for co, ci in ((16, 1), (16, 16), (8, 16)):
        out.append(rng.normal(0.0, math.sqrt(2.0 / (ci * 9)), (co, ci, 3, 3)).ravel())
        out.append(np.zeros(co))
    out[-1][:] = math.log(prior / (1.0 - prior))
    return np.concatenate(out).astype(np.float32)


def dilate(active):
    """Tile maps [..., th, tw] (bool tensors): OR over the 3 x 3 neighbourhood."""
    import torch
    a = active.float()
    a = torch.nn.functional.max_pool2d(a.reshape(-1, 1, *a.shape[-2:]), 3, stride=1, padding=1)
    return a.reshape(active.shape) > 0


def make_data(bank, n, size, seed0):
    import torch

    from paper_1912_07133_gb300 import kf, synthetic
    ph = pw = size // 8
    th = tw = size // 64
    pooled = torch.empty((n, ph, pw), dtype=torch.float32, device="cuda")
    labels = torch.zeros((n, 8, th, tw), dtype=torch.uint8, device="cuda")
    tmp = torch.empty(8 * th * tw, dtype=torch.uint8, device="cuda")
    for i in range(n):
        frame = synthetic.clustered_frame_device(seed0 + i, size, size)
        for ft, order in BANKS:
            bank.run([frame], SCALES, ft, order, threshold=THRESHOLD, fir_kmax=96)
            bank.blobs()  # grows the candidate list if it overflowed (repeats the run)
            kf.kf_proposal_labels(bank.ctx, THRESHOLD, tmp)
            labels[i] |= tmp.view(8, th, tw)
        kf.kf_proposal_pool(bank.ctx, [frame], pooled[i].view(-1))
    return pooled, labels


def coverage(bank, pooled, labels, probs):
    """Share of labelled (tile, any scale) covered by the dilated gate map and
    the share of tiles it marks, per probability threshold."""
    import torch

    from paper_1912_07133_gb300 import kf
    n, ph, pw = pooled.shape
    z = torch.empty((n, 8, ph // 8, pw // 8), dtype=torch.float32, device="cuda")
    for i in range(n):
        kf.kf_proposal_logits(bank.ctx, pooled[i:i + 1], z[i:i + 1])
    want = labels.bool().any(dim=1)
    out = []
    for p in probs:
        act = dilate((z > math.log(p / (1 - p))).any(dim=1))
        cov = float((act & want).sum()) / max(float(want.sum()), 1.0)
        out.append((p, cov, float(act.float().mean())))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--frames", type=int, default=2000)
    ap.add_argument("--size", type=int, default=6144)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1000)
    ap.add_argument("--recall", type=float, default=0.995, help="labelled-tile coverage the threshold must keep")
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1912_07133_gb300 import kf

    kf.load()
    bank = kf.Bank(0)
    t0 = time.time()
    pooled, labels = make_data(bank, args.frames, args.size, args.seed)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    n_val = max(1, args.frames // 10)
    n_tr = args.frames - n_val
    prior = float(labels[:n_tr].float().mean())
    pos_weight = float(min(max((1 - prior) / max(prior, 1e-6), 1.0), 50.0))
    rng = np.random.default_rng(args.seed)
    kf.kf_proposal_set_weights(bank.ctx, init_weights(rng, max(prior, 1e-4)))
    steps_per_epoch = n_tr // args.batch
    total = steps_per_epoch * args.epochs
    g = torch.Generator(device="cpu")
    g.manual_seed(args.seed)
    step, losses = 0, []
    t1 = time.time()
    for ep in range(args.epochs):
        perm = torch.randperm(n_tr, generator=g).cuda()
        ep_loss = []
        for b in range(steps_per_epoch):
            idx = perm[b * args.batch:(b + 1) * args.batch]
            lr = args.lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * step / total)))
            want = b % 25 == 0
            loss = kf.kf_proposal_train_step(bank.ctx, pooled[idx].contiguous(), labels[idx].contiguous(),
                                             pos_weight, lr, want_loss=want)
            if want:
                ep_loss.append(loss)
            step += 1
        losses.append(float(np.mean(ep_loss)))
        print(f"epoch {ep}: loss {losses[-1]:.5f}", flush=True)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    probs = [0.02, 0.05, 0.1, 0.15, 0.2, 0.3, 0.4, 0.5]
    cov = coverage(bank, pooled[n_tr:], labels[n_tr:], probs)
    ok = [c for c in cov if c[1] >= args.recall]
    chosen = max(ok, key=lambda c: c[0]) if ok else min(cov, key=lambda c: c[0])
    stats = dict(frames=args.frames, size=args.size, epochs=args.epochs, batch=args.batch, lr=args.lr,
                 pos_weight=pos_weight, label_prior=prior, losses=losses, data_s=round(t_data, 1),
                 train_s=round(t_train, 1), validation=[dict(p=p, tile_recall=c, active=a) for p, c, a in cov],
                 gate_threshold=chosen[0], seeds=[args.seed, args.seed + args.frames - 1])
    np.savez(args.out, weights=kf.kf_proposal_get_weights(bank.ctx), gate_threshold=np.float32(chosen[0]),
             stats=json.dumps(stats))
    print(json.dumps(stats), flush=True)
    bank.close()


def load_weights(path=DEFAULT_OUT):
    """(weights, gate threshold, stats) of a trained network."""
    d = np.load(path)
    return d["weights"], float(d["gate_threshold"]), json.loads(str(d["stats"]))


if __name__ == "__main__":
    main()
