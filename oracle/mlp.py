"""FP64 CPU oracle for the learned link-SDF surrogate (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  The CUDA library never loads it and shares no code with it.

The surrogate has no counterpart in the paper (whose only network approximates
its grid transform, Eq. (5)); it replaces a link's grid lookup (Sec. III-A) by a
small network trained on values of that grid.  Definitions, all in double
precision, matrix products by numpy:

* network (one per link): f(x) = w4 . s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4 with
  s(z) = z / (1 + exp(-z)) (SiLU), x in R^3, hidden width 128;
* parameter vector (one link, PARAMS entries): W1[128][3], b1[128], W2[128][128],
  b2[128], W3[128][128], b3[128], w4[128], b4 -- row-major, output index first;
* input normalisation: x = (p_loc - m) / a, with m the centre of the link's grid box
  [o, o + (n-1)h]^3 and a = (n-1)h/2 its half-span; output scale: distance = a f(x);
* outside the box, the grid path's rule: |p_loc - c| + a f(x(c)), c the nearest box
  point (c = clamp(p_loc));
* quantised form (``quantize=True``): the operands of the two 128 x 128 products
  are rounded to bfloat16 (round to nearest, ties to even) -- W2, W3 and the
  activations entering them, s(z1) and s(z2) -- as the GPU's tensor-core
  products take them; every other quantity stays in full precision;
* loss: mean absolute error over a batch, L = (1/B) sum_b |f(x_b) - y_b|, with
  d|r|/dr = sign(r) (0 at 0); the backward pass is the chain rule, with the
  quantised operands used where the forward used them (the rounding itself is
  treated as the identity, a straight-through gradient).  In the quantised form
  every product of the backward pass also takes bfloat16 operands, as the GPU
  runs each of them on the tensor cores: the pre-activation gradients dz1, dz2,
  dz3, the inputs x and the last hidden layer s(z3) are rounded before they
  enter a product, and each bias gradient is the batch sum of its rounded dz;
* optimiser: Adam (Kingma & Ba, 2015, Algorithm 1): m <- b1 m + (1-b1) g,
  v <- b2 v + (1-b2) g^2, p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
* training batches: step t (from 0) takes samples (t B + j) mod n, j < B;
* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), the counter-based generator
  the GPU's sampler draws its candidate points from.

Parity status: forward and gradient pinned by finite differences and closed
forms, Adam by its first-step closed form, bfloat16 rounding by a library
routine, Philox by its published known-answer vectors (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

H = 128
PARAMS = H * 3 + H + H * H + H + H * H + H + H + 1

_OFF = {}
_o = 0
for _name, _shape in (("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
                      ("b3", (H,)), ("w4", (H,)), ("b4", ()) ):
    _n = int(np.prod(_shape)) if _shape else 1
    _OFF[_name] = (_o, _shape)
    _o += _n
assert _o == PARAMS


def unpack(params) -> dict:
    """Views of one link's parameter vector by name."""
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (PARAMS,)
    out = {}
    for k, (o, shape) in _OFF.items():
        n = int(np.prod(shape)) if shape else 1
        out[k] = p[o:o + n].reshape(shape) if shape else p[o]
    return out


def pack(d: dict) -> np.ndarray:
    p = np.empty(PARAMS, dtype=np.float64)
    for k, (o, shape) in _OFF.items():
        n = int(np.prod(shape)) if shape else 1
        p[o:o + n] = np.asarray(d[k], dtype=np.float64).reshape(-1)
    return p


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.  The value is
    first rounded to float32, then its low 16 bits are rounded away."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _q(a, quantize):
    return bf16_round(a) if quantize else np.asarray(a, dtype=np.float64)


def forward(params, x, quantize: bool = False, cache: bool = False):
    """f(x) for a batch x [B, 3]; with ``cache`` also the intermediate values."""
    P = unpack(params)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = _q(silu(z1), quantize)
    W2 = _q(P["W2"], quantize)
    z2 = h1 @ W2.T + P["b2"]
    h2 = _q(silu(z2), quantize)
    W3 = _q(P["W3"], quantize)
    z3 = h2 @ W3.T + P["b3"]
    h3 = silu(z3)
    f = h3 @ P["w4"] + P["b4"]
    if cache:
        return f, dict(x=x, z1=z1, h1=h1, W2=W2, z2=z2, h2=h2, W3=W3, z3=z3, h3=h3, P=P)
    return f


def loss_and_grad(params, x, y, quantize: bool = False):
    """Mean absolute error over the batch and its gradient (PARAMS entries)."""
    f, c = forward(params, x, quantize, cache=True)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    B = f.shape[0]
    r = f - y
    loss = float(np.mean(np.abs(r)))
    gf = np.sign(r) / B                                  # dL/df
    P = c["P"]
    g = {}
    g["w4"] = _q(c["h3"], quantize).T @ gf
    g["b4"] = np.sum(gf)
    dz3 = np.outer(gf, P["w4"]) * silu_grad(c["z3"])     # [B, H]
    dz3q = _q(dz3, quantize)
    g["b3"] = dz3q.sum(axis=0)
    g["W3"] = dz3q.T @ c["h2"]
    dh2 = dz3q @ c["W3"]
    dz2 = dh2 * silu_grad(c["z2"])
    dz2q = _q(dz2, quantize)
    g["b2"] = dz2q.sum(axis=0)
    g["W2"] = dz2q.T @ c["h1"]
    dh1 = dz2q @ c["W2"]
    dz1 = dh1 * silu_grad(c["z1"])
    dz1q = _q(dz1, quantize)
    g["b1"] = dz1q.sum(axis=0)
    g["W1"] = dz1q.T @ _q(c["x"], quantize)
    return loss, pack(g)


def adam_step(params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (t counts from 1).  Returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def train(params, X, Y, batch: int, steps: int, lr: float, quantize: bool = True, m=None, v=None,
          t0: int = 0):
    """``steps`` Adam steps on sequential batches of (X, Y); returns (params, m, v, losses)."""
    n = X.shape[0]
    p = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros(PARAMS) if m is None else m.copy()
    v = np.zeros(PARAMS) if v is None else v.copy()
    losses = []
    for t in range(t0, t0 + steps):
        idx = (t * batch + np.arange(batch)) % n
        loss, g = loss_and_grad(p, X[idx], Y[idx], quantize)
        p, m, v = adam_step(p, g, m, v, t + 1, lr)
        losses.append(loss)
    return p, m, v, losses


# ---------------------------------------------------------------- link distance

def box_of(meta):
    """(centre m, half-span a, lower corner o, upper corner) of a link's grid box."""
    meta = np.asarray(meta, dtype=np.float64)
    o = meta[0:3]
    h, n = meta[3], int(round(meta[4]))
    a = 0.5 * (n - 1) * h
    return o + a, a, o, o + 2.0 * a


def surrogate_distance(params, meta, p_loc, quantize: bool = True) -> np.ndarray:
    """Surrogate signed distance at link-frame points [N, 3] (the grid path's rule
    outside the box)."""
    m, a, lo, hi = box_of(meta)
    p = np.asarray(p_loc, dtype=np.float64).reshape(-1, 3)
    c = np.clip(p, lo, hi)
    out = np.linalg.norm(p - c, axis=1)
    return out + a * forward(params, (c - m) / a, quantize)


def check(dh, base, params_per_link, metas, q, points, quantize: bool = True):
    """Per-waypoint min over links and points of the surrogate distance, with the
    arg-min (smallest point, then link, on ties): the grid check's reduction
    (Sec. III-A) with the surrogate in place of the grid lookup."""
    from oracle import fk as oracle_fk
    T = oracle_fk(dh, base, q)            # [W, L, 3, 4] world-from-link
    W, L = T.shape[0], T.shape[1]
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    dist = np.full(W, np.inf)
    al = np.full(W, -1, dtype=np.int64)
    ap = np.full(W, -1, dtype=np.int64)
    for w in range(W):
        best = (np.inf, -1, -1)
        for l in range(L):
            R, t = T[w, l, :, :3], T[w, l, :, 3]
            p_loc = (pts - t) @ R
            d = surrogate_distance(params_per_link[l], metas[l], p_loc, quantize)
            d = np.where(np.isnan(d), np.inf, d)
            i = int(np.argmin(d))
            if d[i] < best[0] or (d[i] == best[0] and (i, l) < (best[2], best[1])):
                best = (float(d[i]), l, i)
        dist[w], al[w], ap[w] = best
    return dist, al, ap


# ------------------------------------------------------------------- Philox

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds.  counter [..., 4] and key [..., 2] as uint32;
    returns [..., 4] uint32.  Each round multiplies words 0 and 2 by the two
    constants, and the new words are (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
    hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key grows by the Weyl constants between
    rounds."""
    c = np.asarray(counter, dtype=np.uint64) & 0xFFFFFFFF
    k = np.asarray(key, dtype=np.uint64) & 0xFFFFFFFF
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0] + np.zeros_like(c0), k[..., 1] + np.zeros_like(c0)
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
        p0 = c0 * PHILOX_M0
        p1 = c2 * PHILOX_M1
        hi0, lo0 = p0 >> 32, p0 & 0xFFFFFFFF
        hi1, lo1 = p1 >> 32, p1 & 0xFFFFFFFF
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniform01(u32) -> np.ndarray:
    """The top 24 bits of a uint32 as a float in [0, 1): (u >> 8) * 2^-24."""
    return (np.asarray(u32, dtype=np.uint32) >> 8).astype(np.float64) * (1.0 / 16777216.0)


def sample_candidates(meta, seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Candidate points (link frame) of the surrogate's training sampler: candidate i
    of ``stream`` is lo + u * (hi - lo) with u the first three words of
    Philox4x32-10(counter = (i, stream, 0, 0), key = (seed lo, seed hi)) mapped to
    [0, 1)."""
    _, _, lo, hi = box_of(meta)
    i = np.arange(start, start + count, dtype=np.uint64)
    ctr = np.stack([i & 0xFFFFFFFF, np.full_like(i, stream), np.zeros_like(i), np.zeros_like(i)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    r = philox4x32_10(ctr, key)
    u = uniform01(r[:, :3])
    return lo + u * (hi - lo)
