"""Pins of the surrogate oracle (oracle/mlp.py) against things other than itself:
finite differences of the loss, closed forms of degenerate networks, Adam's first
step, a library bfloat16 conversion and Philox's published known-answer vectors."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mlp

HERE = os.path.dirname(os.path.abspath(__file__))


def _params(rng, scale=1.0):
    p = mlp.unpack(np.zeros(mlp.PARAMS)).copy()
    d = {}
    for k, shape, fan in (("W1", (128, 3), 3), ("b1", (128,), 3), ("W2", (128, 128), 128), ("b2", (128,), 128),
                          ("W3", (128, 128), 128), ("b3", (128,), 128), ("w4", (128,), 128), ("b4", (), 128)):
        b = scale / math.sqrt(fan)
        d[k] = rng.uniform(-b, b, size=shape) if shape else rng.uniform(-b, b)
    return mlp.pack(d)


def test_layout_and_size():
    assert mlp.PARAMS == 33665
    p = np.arange(mlp.PARAMS, dtype=np.float64)
    P = mlp.unpack(p)
    assert P["W1"][0, 0] == 0 and P["W1"][1, 0] == 3       # output index first
    assert P["b1"][0] == 384 and P["W2"][0, 1] == 513 and P["b4"] == mlp.PARAMS - 1
    assert np.array_equal(mlp.pack(P), p)


def test_philox_known_answers():
    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        c = np.array([int(x, 16) for x in v["counter"]], dtype=np.uint64)
        k = np.array([int(x, 16) for x in v["key"]], dtype=np.uint64)
        out = mlp.philox4x32_10(c, k)
        assert [f"{int(x):08x}" for x in out] == v["out"]


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 500), rng.normal(0, 1e4, 500),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8, -1.0 - 2 ** -8,
                         3.0e38, 1e-40, np.inf, -np.inf]]).astype(np.float32)
    ours = mlp.bf16_round(x)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0                  # tie to even (down)
    assert mlp.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6    # tie to even (up)


def test_silu_values():
    assert mlp.silu(0.0) == 0.0 and mlp.silu_grad(0.0) == 0.5
    assert abs(mlp.silu(40.0) - 40.0) < 1e-12 and abs(mlp.silu(-40.0)) < 1e-15
    z = np.linspace(-8, 8, 101)
    e = 1e-6
    fd = (mlp.silu(z + e) - mlp.silu(z - e)) / (2 * e)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng, 2.0)
    x = rng.uniform(-1, 1, (8, 3))
    f = mlp.forward(p, x)
    y = f + np.where(rng.random(8) < 0.5, -1, 1) * rng.uniform(0.5, 1.0, 8)   # residuals far from 0
    loss, g = mlp.loss_and_grad(p, x, y)
    assert abs(loss - np.mean(np.abs(f - y))) < 1e-15
    idx = np.concatenate([np.arange(0, 512), np.arange(mlp.PARAMS - 257, mlp.PARAMS),
                          rng.choice(mlp.PARAMS, 400, replace=False)])
    e = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (np.mean(np.abs(mlp.forward(pp, x) - y)) - np.mean(np.abs(mlp.forward(pm, x) - y))) / (2 * e)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_degenerate_network_closed_forms():
    rng = np.random.default_rng(2)
    P = mlp.unpack(_params(rng))
    P = {k: np.array(v, copy=True) for k, v in P.items()}
    P["W2"][:] = 0.0
    P["W3"][:] = 0.0
    p = mlp.pack(P)
    x = rng.uniform(-1, 1, (16, 3))
    const = sum(P["w4"][j] * P["b3"][j] / (1 + math.exp(-P["b3"][j])) for j in range(128)) + P["b4"]
    assert np.allclose(mlp.forward(p, x), const, rtol=0, atol=1e-12)
    _, g = mlp.loss_and_grad(p, x, np.zeros(16))
    G = mlp.unpack(g)
    assert np.all(G["W1"] == 0) and np.all(G["b1"] == 0) and np.all(G["W2"] == 0) and np.all(G["b2"] == 0)
    assert abs(G["b4"] - np.mean(np.sign(mlp.forward(p, x)))) < 1e-15


def test_single_path_network_indexing():
    # one chain x[2] -> h1[7] -> h2[3] -> h3[5] -> f: a scalar composition
    P = {k: np.zeros_like(v) if np.ndim(v) else 0.0 for k, v in mlp.unpack(np.zeros(mlp.PARAMS)).items()}
    P["W1"][7, 2] = 1.5
    P["b1"][7] = 0.25
    P["W2"][3, 7] = -2.0
    P["b2"][3] = 0.5
    P["W3"][5, 3] = 1.25
    P["b3"][5] = -0.75
    P["w4"][5] = 2.0
    P["b4"] = 0.125
    p = mlp.pack(P)
    s = lambda z: z / (1 + math.exp(-z))
    silu0 = s(0.0)
    for xv in ((0.3, -0.2, 0.9), (-1.0, 1.0, -0.4)):
        h1 = s(1.5 * xv[2] + 0.25)
        h2 = s(-2.0 * h1 + 0.5)
        h3 = s(1.25 * h2 - 0.75)
        # every other unit of layers 2 and 3 sees z = bias = 0 (s(0) = 0) and w4 is zero there
        expect = 2.0 * h3 + 0.125 + 0 * silu0
        assert abs(mlp.forward(p, np.array([xv]))[0] - expect) < 1e-14


def test_quantized_gradient_close_to_exact():
    rng = np.random.default_rng(3)
    p = _params(rng, 2.0)
    x = rng.uniform(-1, 1, (256, 3))
    y = rng.uniform(-0.5, 0.5, 256)
    l0, g0 = mlp.loss_and_grad(p, x, y, quantize=False)
    l1, g1 = mlp.loss_and_grad(p, x, y, quantize=True)
    f0, f1 = mlp.forward(p, x), mlp.forward(p, x, quantize=True)
    # bfloat16 keeps 8 significant bits: relative error 2^-9 per rounding, a few roundings deep
    assert np.max(np.abs(f1 - f0)) < 0.05 * np.max(np.abs(f0)) and np.max(np.abs(f1 - f0)) > 0
    assert np.linalg.norm(g1 - g0) < 0.1 * np.linalg.norm(g0)
    # the quantised operands are bfloat16 values
    _, c = mlp.forward(p, x, quantize=True, cache=True)
    for k in ("h1", "h2", "W2", "W3"):
        assert np.array_equal(c[k], mlp.bf16_round(c[k]))
    assert not np.array_equal(c["h3"], mlp.bf16_round(c["h3"]))     # layer 4 stays in full precision


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(4)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    lr, eps = 1e-3, 1e-8
    p1, m, v = mlp.adam_step(p, g, np.zeros(100), np.zeros(100), 1, lr, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the step at lr (bias correction exact for constant g)
    p2, _, _ = mlp.adam_step(p1, g, m, v, 2, lr, eps=0.0)
    assert np.allclose(p2, p1 - lr * np.sign(g), rtol=0, atol=1e-15)


def test_surrogate_distance_out_of_box_rule():
    rng = np.random.default_rng(5)
    P = {k: np.array(v, copy=True) for k, v in mlp.unpack(_params(rng)).items()}
    P["W2"][:] = 0.0
    P["W3"][:] = 0.0
    p = mlp.pack(P)
    k = float(mlp.forward(p, np.zeros((1, 3)))[0])
    meta = np.array([-0.2, -0.1, -0.3, 0.01, 41, 0, 0, 0, 0.3, 0.05])   # origin, h, n, ...
    m, a, lo, hi = mlp.box_of(meta)
    assert np.allclose(lo, [-0.2, -0.1, -0.3]) and abs(a - 0.2) < 1e-15 and np.allclose(hi, lo + 0.4)
    pts = rng.uniform(-1.0, 1.0, (200, 3))
    box_dist = np.sqrt(np.sum(np.maximum(np.maximum(lo - pts, pts - hi), 0.0) ** 2, axis=1))
    assert np.allclose(mlp.surrogate_distance(p, meta, pts, quantize=False), box_dist + a * k, atol=1e-12)


def test_check_with_constant_networks():
    # link l's network is the constant k_l: inside every box the min is min_l a_l k_l
    import scenegen as sg
    from oracle import fk
    rng = np.random.default_rng(6)
    sc = sg.make_scene("tiny", resolution=16)
    from oracle import grid_meta
    metas = [grid_meta(msh, 16, sc.margin) for msh in sc.meshes]
    L = len(metas)
    ps = []
    for l in range(L):
        P = {k: np.array(v, copy=True) for k, v in mlp.unpack(_params(rng)).items()}
        P["W2"][:] = 0.0
        P["W3"][:] = 0.0
        P["b4"] = 0.1 * (l + 1)
        ps.append(mlp.pack(P))
    q = sc.q[:3]
    T = fk(sc.dh, sc.base, q)
    # points at the centres of the links' boxes, in the world frame, for waypoint 0
    pts = []
    for l in range(L):
        m, _, _, _ = mlp.box_of(metas[l])
        pts.append(T[0, l, :, :3] @ m + T[0, l, :, 3])
    d, al, ap = mlp.check(sc.dh, sc.base, ps, metas, q[:1], np.array(pts), quantize=False)
    vals = [mlp.surrogate_distance(ps[l], metas[l], (np.array(pts) - T[0, l, :, 3]) @ T[0, l, :, :3],
                                   quantize=False) for l in range(L)]
    V = np.array(vals)                                   # [L, N]
    assert abs(d[0] - V.min()) < 1e-12
    assert V[al[0], ap[0]] == V.min()


def test_sample_candidates_in_box_and_uniform():
    meta = np.array([-0.2, -0.1, -0.3, 0.01, 41, 0, 0, 0, 0.3, 0.05])
    c = mlp.sample_candidates(meta, seed=123, stream=0, start=0, count=20000)
    _, _, lo, hi = mlp.box_of(meta)
    assert np.all(c >= lo) and np.all(c < hi)
    u = (c - lo) / (hi - lo)
    assert np.all(np.abs(u.mean(axis=0) - 0.5) < 0.01) and np.all(np.abs(u.var(axis=0) - 1 / 12) < 0.003)
    # counters are positions: a later window continues the same stream
    c2 = mlp.sample_candidates(meta, seed=123, stream=0, start=100, count=5)
    assert np.array_equal(c2, c[100:105])
    assert not np.array_equal(mlp.sample_candidates(meta, 123, 1, 0, 5), c[:5])


def test_training_reduces_loss():
    rng = np.random.default_rng(7)
    p = _params(rng)
    X = rng.uniform(-1, 1, (4096, 3))
    Y = np.linalg.norm(X, axis=1) - 0.5                 # a sphere's SDF in normalised units
    _, _, _, losses = mlp.train(p, X, Y, batch=256, steps=300, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.25 * np.mean(losses[:5])
