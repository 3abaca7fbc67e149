"""FP64 CPU oracle of the proposal network that gates the filter bank.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the bench's CPU
baseline; never by the product package, and it shares no code with the CUDA
kernels.  The paper (Kennedy, arXiv:1912.07133) has no network; this is the
plain definition of the one the library trains and runs:

  pooled  p[y, x]     = mean of the frame (times its value scale) over the 8 x 8
                        block [8y, 8y+8) x [8x, 8x+8), clipped to the frame
  conv    out[o,y,x]  = b[o] + sum_{i,dy,dx} W[o,i,dy,dx] in[i, y+dy-1, x+dx-1]
                        (cross-correlation, zero outside the input)
  net     a1 = relu(conv(p, W1, b1)), a2 = relu(conv(a1, W2, b2)),
          o3 = conv(a2, W3, b3); channels 1 -> 16 -> 16 -> 8
  logits  z[c, ty, tx] = max of o3[c] over the 8 x 8 block of pooled pixels of
                        tile (ty, tx) (one 64 x 64-pixel tile of the frame); the
                        first maximum in row-major order receives the gradient
  loss    mean over logits of  pw t softplus(-z) + (1 - t) softplus(z)
  labels  t[s, ty, tx] = 1 if a blob of scale s has its centre in the tile
  Adam    m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
          theta -= lr (m / (1-b1^k)) / (sqrt(v / (1-b2^k)) + eps)

The weights used in every product are the bf16 rounding (round to nearest,
ties to even) of the FP32 master weights; gradients are taken with respect to
those rounded weights and applied to the masters.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 16, 16, 8)
TILE = 64   # frame pixels per tile side
POOL = 8    # frame pixels per pooled pixel side; pooled pixels per tile side
B1, B2, EPS = 0.9, 0.999, 1e-8


def param_shapes():
    """[(W shape, b shape)] per layer."""
    return [((co, ci, 3, 3), (co,)) for ci, co in zip(CHANNELS[:-1], CHANNELS[1:])]


def n_params() -> int:
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in param_shapes())


def unpack(flat):
    """Flat parameter vector (W1, b1, W2, b2, W3, b3 in C order) -> list of (W, b)."""
    flat = np.asarray(flat, np.float64)
    out, k = [], 0
    for ws, bs in param_shapes():
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((flat[k:k + nw].reshape(ws), flat[k + nw:k + nw + nb].reshape(bs)))
        k += nw + nb
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def pool8(frame, value_scale=1.0) -> np.ndarray:
    """8 x 8 block means of the frame times its value scale (partial blocks at
    the right and bottom edges average the pixels they contain)."""
    f = np.asarray(frame, np.float64) * value_scale
    H, W = f.shape
    h, w = -(-H // POOL), -(-W // POOL)
    out = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            out[y, x] = f[POOL * y:POOL * y + POOL, POOL * x:POOL * x + POOL].mean()
    return out


def conv3x3(x, W, b) -> np.ndarray:
    """x [Ci, h, w] -> [Co, h, w], cross-correlation with zero padding."""
    Ci, h, w = x.shape
    Co = W.shape[0]
    xp = np.zeros((Ci, h + 2, w + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.empty((Co, h, w))
    for o in range(Co):
        acc = np.full((h, w), float(b[o]))
        for i in range(Ci):
            for dy in range(3):
                for dx in range(3):
                    acc += W[o, i, dy, dx] * xp[i, dy:dy + h, dx:dx + w]
        out[o] = acc
    return out


def conv3x3_backward(x, W, dout, need_dx=True):
    """Gradients of conv3x3 w.r.t. its input, weights and bias."""
    Ci, h, w = x.shape
    Co = W.shape[0]
    xp = np.zeros((Ci, h + 2, w + 2))
    xp[:, 1:-1, 1:-1] = x
    dW = np.empty_like(W)
    for o in range(Co):
        for i in range(Ci):
            for dy in range(3):
                for dx in range(3):
                    dW[o, i, dy, dx] = np.sum(dout[o] * xp[i, dy:dy + h, dx:dx + w])
    db = dout.sum(axis=(1, 2))
    dx = None
    if need_dx:
        dxp = np.zeros((Ci, h + 2, w + 2))
        for o in range(Co):
            for i in range(Ci):
                for dy in range(3):
                    for dx_ in range(3):
                        dxp[i, dy:dy + h, dx_:dx_ + w] += W[o, i, dy, dx_] * dout[o]
        dx = dxp[:, 1:-1, 1:-1]
    return dx, dW, db


def maxpool8(o):
    """o [C, h, w] -> logits [C, ceil(h/8), ceil(w/8)] and the flat index (into
    h x w) of the first maximum of each block in row-major order."""
    C, h, w = o.shape
    th, tw = -(-h // POOL), -(-w // POOL)
    z = np.empty((C, th, tw))
    arg = np.empty((C, th, tw), np.int64)
    for c in range(C):
        for ty in range(th):
            for tx in range(tw):
                blk = o[c, POOL * ty:POOL * ty + POOL, POOL * tx:POOL * tx + POOL]
                k = int(np.argmax(blk))  # first maximum, row-major
                by, bx = divmod(k, blk.shape[1])
                z[c, ty, tx] = blk[by, bx]
                arg[c, ty, tx] = (POOL * ty + by) * w + POOL * tx + bx
    return z, arg


def forward(p, params):
    """p [h, w] pooled frame, params [(W, b)] (already bf16-rounded) ->
    (logits [8, th, tw], cache)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    x = np.asarray(p, np.float64)[None]
    a1 = np.maximum(conv3x3(x, W1, b1), 0.0)
    a2 = np.maximum(conv3x3(a1, W2, b2), 0.0)
    o3 = conv3x3(a2, W3, b3)
    z, arg = maxpool8(o3)
    return z, dict(x=x, a1=a1, a2=a2, o3=o3, arg=arg)


def softplus(v):
    return np.logaddexp(0.0, v)


def bce(z, t, pw):
    """Mean weighted BCE with logits and its gradient (same shapes as z)."""
    z = np.asarray(z, np.float64)
    t = np.asarray(t, np.float64)
    M = z.size
    loss = np.sum(pw * t * softplus(-z) + (1.0 - t) * softplus(z)) / M
    s = 1.0 / (1.0 + np.exp(-z))
    dz = (pw * t * (s - 1.0) + (1.0 - t) * s) / M
    return loss, dz


def backward(params, cache, dz):
    """Gradients [(dW, db)] of a scalar whose gradient w.r.t. the logits is dz."""
    (W1, b1), (W2, b2), (W3, b3) = params
    o3 = cache["o3"]
    C, h, w = o3.shape
    do3 = np.zeros(C * h * w)
    arg = cache["arg"]
    for c in range(C):
        np.add.at(do3, c * h * w + arg[c].ravel(), dz[c].ravel())
    do3 = do3.reshape(C, h, w)
    da2, dW3, db3 = conv3x3_backward(cache["a2"], W3, do3)
    da2 = da2 * (cache["a2"] > 0)
    da1, dW2, db2 = conv3x3_backward(cache["a1"], W2, da2)
    da1 = da1 * (cache["a1"] > 0)
    _, dW1, db1 = conv3x3_backward(cache["x"], W1, da1, need_dx=False)
    return [(dW1, db1), (dW2, db2), (dW3, db3)]


def loss_and_grad(pooled_batch, labels_batch, master_flat, pw):
    """Mean over the batch of the per-frame losses, and its gradient w.r.t. the
    (bf16-rounded) weights, as flat vectors."""
    params = unpack(bf16_round(np.asarray(master_flat, np.float32)))
    total, grad = 0.0, np.zeros(n_params())
    n = len(pooled_batch)
    for p, t in zip(pooled_batch, labels_batch):
        z, cache = forward(p, params)
        loss, dz = bce(z, t, pw)
        total += loss / n
        grad += pack(backward(params, cache, dz / n))
    return total, grad


def adam(master, m, v, g, k, lr):
    """One Adam step (k = 1, 2, ...): returns new (master, m, v)."""
    m = B1 * m + (1 - B1) * g
    v = B2 * v + (1 - B2) * g * g
    mh = m / (1 - B1 ** k)
    vh = v / (1 - B2 ** k)
    return master - lr * mh / (np.sqrt(vh) + EPS), m, v


def labels(blobs, S, H, W):
    """t [S, ceil(H/64), ceil(W/64)] from a blob list (records with scale, y, x)."""
    t = np.zeros((S, -(-H // TILE), -(-W // TILE)), np.uint8)
    for b in blobs:
        t[int(b["scale"]), int(b["y"]) // TILE, int(b["x"]) // TILE] = 1
    return t
