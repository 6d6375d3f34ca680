"""Learned surrogate on the GPU against the FP64 oracle (oracle/mlp.py): the
sampler's candidates and labels, the forward pass, the gradient of one batch,
Adam steps, and training that lowers the error against the grid.

Tolerances.  The GPU rounds the products' operands to bfloat16 exactly where the
oracle does, but it computes the values being rounded in FP32 (with a fast
exponential in SiLU), so a value within ~1e-7 relative of a bfloat16 rounding
boundary can round the other way: one bfloat16 ulp (2^-8 relative) on that
operand.  Such flips are rare (about 1e-5 of the operands) and each moves a
product by at most one term's ulp, so results agree to ~1e-3 of their scale,
which is what the assertions allow; everything in FP32 alone agrees to ~1e-5."""
import numpy as np
import pytest

import oracle
import scenegen as sg
from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sdf():
    from paper_2309_12543_gb300 import build
    build.build()
    import paper_2309_12543_gb300 as m
    return m


@pytest.fixture(scope="module")
def env(sdf):
    sc = sg.make_scene("tiny")
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    ctx = sdf.Context(0, torch.cuda.current_stream())
    grids = sdf.sdf_grids_upload(ctx, vals, metas)
    return sc, ctx, grids, np.asarray(vals), [np.asarray(m) for m in metas]


def _dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_sampler_candidates_and_labels(sdf, env):
    sc, ctx, grids, vals, metas = env
    link, n, near10, band, seed = 2, 20000, 7, 0.10, 0x1234_5678_9abc
    x = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    src = torch.empty(n, dtype=torch.int64, device="cuda")
    sdf.sdf_surrogate_sample(ctx, grids, link, n, near10, band, seed, x, y, src)
    assert ctx.synchronize() == 0
    x, y, src = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64), src.cpu().numpy()
    m, a, lo, hi = mlp.box_of(metas[link])
    j = np.arange(n)
    near = (j % 10) < near10
    stream, counter = src >> 40, src & ((1 << 40) - 1)
    assert np.array_equal(stream, np.where(near, 0, 1))
    # uniform samples are the uniform stream in order
    u = (j // 10) * (10 - near10) + (j % 10 - near10)
    assert np.array_equal(counter[~near], u[~near])
    # every sample is its candidate, normalised, and labelled by the grid
    for s_id in (0, 1):
        sel = stream == s_id
        c = np.concatenate([mlp.sample_candidates(metas[link], seed, s_id, int(i), 1) for i in counter[sel][:500]])
        assert np.allclose(x[sel][:500], (c - m) / a, atol=1e-6)
    p = x * a + m
    g = oracle.lookup(vals[link], metas[link], p)
    assert np.max(np.abs(y * a - g)) < 1e-5
    # near samples: the accepted candidates of stream 0 in counter order
    k_counter = counter[near]
    assert np.all(np.diff(k_counter) > 0)
    assert np.all(np.abs(g[near]) <= band + 1e-5)
    skipped = np.setdiff1d(np.arange(k_counter[-1] + 1), k_counter)
    cs = mlp.sample_candidates(metas[link], seed, 0, 0, int(k_counter[-1]) + 1)[skipped]
    assert np.all(np.abs(oracle.lookup(vals[link], metas[link], cs)) > band - 1e-5)


def test_forward_matches_oracle(sdf, env):
    sc, ctx, grids, vals, metas = env
    params = sg.mlp_init(11, len(metas))
    sur = sdf.Surrogate(ctx, grids, params)
    assert np.array_equal(sur.params(), params)          # the layout round-trips
    rng = np.random.default_rng(12)
    for link, n in ((0, 1000), (5, 129), (6, 1)):
        xs = rng.uniform(-1.2, 1.2, (n, 3)).astype(np.float32)
        f = torch.empty(n, dtype=torch.float32, device="cuda")
        sur.eval(link, _dev(xs), n, f)
        assert ctx.synchronize() == 0
        ref = mlp.forward(params[link].astype(np.float64), xs.astype(np.float64), quantize=True)
        err = np.abs(f.cpu().numpy() - ref)
        scale = np.max(np.abs(ref))
        assert err.max() <= 2e-3 * scale + 1e-5, (link, err.max(), scale)
        assert np.median(err) <= 1e-4 * scale + 1e-6


def test_gradient_matches_oracle(sdf, env):
    sc, ctx, grids, vals, metas = env
    params = sg.mlp_init(13, len(metas))
    sur = sdf.Surrogate(ctx, grids, params)
    rng = np.random.default_rng(14)
    for link in (1, 4):
        xs = rng.uniform(-1, 1, (128, 3)).astype(np.float32)
        f0 = mlp.forward(params[link].astype(np.float64), xs.astype(np.float64), quantize=True)
        # labels away from the prediction, so sign(f - y) is the same on both sides
        ys = (f0 + np.where(rng.random(128) < 0.5, -1, 1) * rng.uniform(0.05, 0.5, 128)).astype(np.float32)
        g = torch.empty(sdf.SDF_MLP_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        sur.grad(link, _dev(xs), _dev(ys), g, loss)
        assert ctx.synchronize() == 0
        l_ref, g_ref = mlp.loss_and_grad(params[link].astype(np.float64), xs, ys, quantize=True)
        assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
        G, R = mlp.unpack(g.cpu().numpy().astype(np.float64)), mlp.unpack(g_ref)
        for k in R:
            d = np.abs(np.asarray(G[k]) - np.asarray(R[k]))
            scale = np.max(np.abs(R[k]))
            assert d.max() <= 5e-3 * scale + 1e-7, (link, k, d.max(), scale)
            assert np.linalg.norm(np.asarray(G[k]) - np.asarray(R[k])) <= 2e-3 * np.linalg.norm(R[k]) + 1e-7, k
    assert np.array_equal(sur.params(), params)          # gradient mode changes nothing


def test_adam_steps_match_oracle(sdf, env):
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    params = sg.mlp_init(15, L)
    sur = sdf.Surrogate(ctx, grids, params)
    rng = np.random.default_rng(16)
    n, steps, lr = 384, 3, 1e-3
    X = rng.uniform(-1, 1, (L, n, 3)).astype(np.float32)
    Y = rng.uniform(-0.6, 0.6, (L, n)).astype(np.float32)
    loss = torch.zeros(L, dtype=torch.float32, device="cuda")
    sur.train(_dev(X), _dev(Y), n, 1, steps, lr, loss)
    assert ctx.synchronize() == 0
    got = sur.params().astype(np.float64)
    for link in (0, 3):
        # batches start at index 1 (first_batch = 1); Adam's step counter starts at 1
        p_ref = params[link].astype(np.float64).copy()
        m = np.zeros(mlp.PARAMS)
        v = np.zeros(mlp.PARAMS)
        ls = []
        for s in range(steps):
            idx = ((1 + s) * 128 + np.arange(128)) % n
            lv, gr = mlp.loss_and_grad(p_ref, X[link][idx], Y[link][idx], quantize=True)
            p_ref, m, v = mlp.adam_step(p_ref, gr, m, v, s + 1, lr)
            ls.append(lv)
        assert abs(loss.cpu().numpy()[link] - sum(ls)) <= 1e-3 * sum(ls)
        step_gpu = got[link] - params[link]
        step_ref = p_ref - params[link]
        # each Adam step moves a parameter by about lr; where the gradient is tiny its
        # sign (and so the step) is decided by rounding: compare all but a few
        bad = np.abs(step_gpu - step_ref) > 0.2 * lr
        assert bad.mean() < 0.01, (link, bad.mean())
        assert np.max(np.abs(step_gpu - step_ref)) <= 2 * steps * lr * 1.01


def test_training_lowers_the_error(sdf, env):
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(17, L))
    n = 65536
    X = torch.empty((L, n, 3), dtype=torch.float32, device="cuda")
    Y = torch.empty((L, n), dtype=torch.float32, device="cuda")
    for l in range(L):
        sdf.sdf_surrogate_sample(ctx, grids, l, n, 7, 0.10, 1000 + l, X[l], Y[l])
    before = [sur.error(l, 20000, seed=5)[1] for l in range(L)]
    loss = torch.zeros(L, dtype=torch.float32, device="cuda")
    sur.train(X, Y, n, 0, 3000, 1e-3, loss)
    assert ctx.synchronize() == 0
    after = [sur.error(l, 20000, seed=5) for l in range(L)]
    print("mean error before", before, "after", after)
    for l in range(L):
        assert after[l][1] < 0.2 * before[l], (l, before[l], after[l])


# ----------------------------------------------------------------- surrogate check

def _sur_check(sdf, ctx, robot, sur, q, pts, margin, eps):
    W, N = len(q), len(pts)
    d = torch.full((W,), 7.0, dtype=torch.float32, device="cuda")
    l = torch.full((W,), -7, dtype=torch.int32, device="cuda")
    p = torch.full((W,), -7, dtype=torch.int32, device="cuda")
    rech = torch.full((W,), 9, dtype=torch.uint8, device="cuda")
    sd = torch.full((W,), 7.0, dtype=torch.float32, device="cuda")
    pd = _dev(pts) if N else torch.empty((0, 3), dtype=torch.float32, device="cuda")
    sdf.check_trajectory_surrogate(ctx, robot, sur, _dev(q), W, pd, N, margin, eps, d, l, p, rech, sd)
    assert ctx.synchronize() == 0
    return [t.cpu().numpy() for t in (d, l, p, rech, sd)]


def _grid_check(sdf, ctx, robot, q, pts):
    W = len(q)
    out = [torch.empty(W, dtype=dt, device="cuda") for dt in (torch.float32, torch.int32, torch.int32)]
    sdf.check_trajectory(ctx, robot, _dev(q), W, _dev(pts), len(pts), *out)
    assert ctx.synchronize() == 0
    return [t.cpu().numpy() for t in out]


def _trained(sdf, ctx, grids, L, steps=3000, seed=31):
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(seed, L))
    n = 65536
    X = torch.empty((L, n, 3), dtype=torch.float32, device="cuda")
    Y = torch.empty((L, n), dtype=torch.float32, device="cuda")
    for l in range(L):
        sdf.sdf_surrogate_sample(ctx, grids, l, n, 7, 0.10, 2000 + l, X[l], Y[l])
    sur.train(X, Y, n, 0, steps, 1e-3)
    assert ctx.synchronize() == 0
    return sur


def test_surrogate_check_without_culling_is_the_brute_force_minimum(sdf, env):
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    params = sg.mlp_init(21, L)
    sur = sdf.Surrogate(ctx, grids, params)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q, pts = sc.q[:20].astype(np.float32), sc.points[:400].astype(np.float32)
    d, l, p, rech, sd = _sur_check(sdf, ctx, robot, sur, q, pts, margin=0.0, eps=100.0)   # eps: no culling
    ref_d, ref_l, ref_p = mlp.check(sc.dh, sc.base, params.astype(np.float64), metas, q, pts, quantize=True)
    assert np.max(np.abs(sd - ref_d)) <= 2e-3, np.max(np.abs(sd - ref_d))
    assert np.median(np.abs(sd - ref_d)) <= 2e-4
    # everything is below margin + eps: the grid path decided every waypoint, exactly
    assert np.all(rech == 1)
    g = _grid_check(sdf, ctx, robot, q, pts)
    assert np.array_equal(d.view(np.uint32), g[0].view(np.uint32))
    assert np.array_equal(l, g[1]) and np.array_equal(p, g[2])


@pytest.mark.parametrize("N", [1, 5, 37])
def test_surrogate_check_ragged_seed_tiles(sdf, env, N):
    # seed tiles with fewer valid points than a seed takes (8): the surrogate minimum is
    # still the brute-force one, and the grid path decides every waypoint exactly
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    params = sg.mlp_init(23, L)
    sur = sdf.Surrogate(ctx, grids, params)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q, pts = sc.q[:20].astype(np.float32), sc.points[:N].astype(np.float32)
    d, l, p, rech, sd = _sur_check(sdf, ctx, robot, sur, q, pts, margin=0.0, eps=100.0)   # eps: no culling
    ref_d, ref_l, ref_p = mlp.check(sc.dh, sc.base, params.astype(np.float64), metas, q, pts, quantize=True)
    assert np.max(np.abs(sd - ref_d)) <= 2e-3, np.max(np.abs(sd - ref_d))
    assert np.all(rech == 1)
    g = _grid_check(sdf, ctx, robot, q, pts)
    assert np.array_equal(d.view(np.uint32), g[0].view(np.uint32))
    assert np.array_equal(l, g[1]) and np.array_equal(p, g[2])


def test_surrogate_check_follows_training(sdf, env):
    """The context keeps the networks' weights in the fused kernel's layout between
    checks; a training step in between must reach the next check (the surrogate
    minima match the oracle for the new parameters, not the old ones)."""
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(31, L))
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q, pts = sc.q[:12].astype(np.float32), sc.points[:300].astype(np.float32)
    _, _, _, _, sd0 = _sur_check(sdf, ctx, robot, sur, q, pts, margin=0.0, eps=100.0)
    ref0 = mlp.check(sc.dh, sc.base, sur.params().astype(np.float64), metas, q, pts, quantize=True)[0]
    assert np.max(np.abs(sd0 - ref0)) <= 2e-3
    rng = np.random.default_rng(32)
    n = 256
    X = torch.tensor(rng.uniform(-1, 1, (L, n, 3)).astype(np.float32), device="cuda")
    Y = torch.tensor(rng.uniform(-0.3, 0.3, (L, n)).astype(np.float32), device="cuda")
    sur.train(X, Y, n, 0, 20, 1e-2)
    assert ctx.synchronize() == 0
    _, _, _, _, sd1 = _sur_check(sdf, ctx, robot, sur, q, pts, margin=0.0, eps=100.0)
    ref1 = mlp.check(sc.dh, sc.base, sur.params().astype(np.float64), metas, q, pts, quantize=True)[0]
    assert np.max(np.abs(ref1 - ref0)) > 1e-2          # the training moved the minima
    assert np.max(np.abs(sd1 - ref1)) <= 2e-3


def test_surrogate_check_with_trained_network_and_fallback(sdf, env):
    sc, ctx, grids, vals, metas = env
    L = len(metas)
    sur = _trained(sdf, ctx, grids, L)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    errs = [max(sur.error(k, 50000, 0, seed=77)[0], sur.error(k, 50000, 10, 0.1, seed=78)[0]) for k in range(L)]
    eps = 2.0 * max(errs) + 0.01
    margin = 0.05
    # the cloud beyond 0.8 m from the base: some waypoints come within the margin, some
    # stay far from every point (grid distances 2 cm to 46 cm)
    q = sc.q.astype(np.float32)
    pts = sc.points[np.linalg.norm(sc.points, axis=1) >= 0.8].astype(np.float32)
    d, l, p, rech, sd = _sur_check(sdf, ctx, robot, sur, q, pts, margin, eps)
    params = sur.params().astype(np.float64)
    ref_d, _, _ = mlp.check(sc.dh, sc.base, params, metas, q[:25], pts, quantize=True)
    assert np.max(np.abs(sd[:25] - ref_d)) <= 2e-3
    assert np.array_equal(rech, (sd < np.float32(margin + eps)).astype(np.uint8))
    g = _grid_check(sdf, ctx, robot, q, pts)
    sel = rech == 1
    assert np.array_equal(d[sel].view(np.uint32), g[0][sel].view(np.uint32))
    assert np.array_equal(d[~sel].view(np.uint32), sd[~sel].view(np.uint32))
    # the safety property: every waypoint truly within the margin went to the grid
    assert np.all(rech[g[0] < margin] == 1)
    # and where the surrogate decided, it is within its bound of the grid
    assert 0 < sel.sum() < len(q)
    assert np.all(np.abs(d[~sel] - g[0][~sel]) <= eps)
    print("eps", eps, "rechecked", int(sel.sum()), "of", len(q))
    # without the surrogate-minimum output, waypoints already below margin + eps stop
    # being refined: every output must stay bit-identical
    W, N = len(q), len(pts)
    d2 = torch.full((W,), 7.0, dtype=torch.float32, device="cuda")
    l2 = torch.full((W,), -7, dtype=torch.int32, device="cuda")
    p2 = torch.full((W,), -7, dtype=torch.int32, device="cuda")
    r2 = torch.full((W,), 9, dtype=torch.uint8, device="cuda")
    sdf.check_trajectory_surrogate(ctx, robot, sur, _dev(q), W, _dev(pts), N, margin, eps, d2, l2, p2, r2)
    assert ctx.synchronize() == 0
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), d.view(np.uint32))
    assert np.array_equal(l2.cpu().numpy(), l) and np.array_equal(p2.cpu().numpy(), p)
    assert np.array_equal(r2.cpu().numpy(), rech)


def test_surrogate_check_empty_cloud(sdf, env):
    sc, ctx, grids, vals, metas = env
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(23, len(metas)))
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    d, l, p, rech, sd = _sur_check(sdf, ctx, robot, sur, sc.q[:7].astype(np.float32), np.zeros((0, 3)), 0.05, 0.01)
    assert np.all(np.isinf(d)) and np.all(l == -1) and np.all(p == -1) and np.all(rech == 0)


@pytest.mark.parametrize("warps", [8, 16])
def test_masked_grid_check_writes_only_selected_waypoints(sdf, env, warps):
    # with 16 warps a block holds two interleaved waypoints, the mask read at both
    sc, ctx, grids, vals, metas = env
    ctx.set_option(sdf.SDF_OPT_BLOCK_WARPS, warps)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q, pts = sc.q.astype(np.float32), sc.points.astype(np.float32)
    W = len(q)
    mask = (np.arange(W) % 3 == 1).astype(np.uint8)
    out = [torch.full((W,), 7.0, dtype=torch.float32, device="cuda"),
           torch.full((W,), -7, dtype=torch.int32, device="cuda"), torch.full((W,), -7, dtype=torch.int32, device="cuda")]
    qd, pd, md = _dev(q), _dev(pts), _dev(mask, torch.uint8)
    sdf.check_batch(ctx, [(robot, qd, W, pd, len(pts), *out, md)])
    assert ctx.synchronize() == 0
    d, l, p = [t.cpu().numpy() for t in out]
    g = _grid_check(sdf, ctx, robot, q, pts)
    sel = mask == 1
    assert np.array_equal(d[sel].view(np.uint32), g[0][sel].view(np.uint32))
    assert np.array_equal(l[sel], g[1][sel]) and np.array_equal(p[sel], g[2][sel])
    assert np.all(d[~sel] == 7.0) and np.all(l[~sel] == -7) and np.all(p[~sel] == -7)
    ctx.set_option(sdf.SDF_OPT_BLOCK_WARPS, 0)


def test_surrogate_gain_over_the_grid(sdf):
    """What the trained network gains over the grid form it replaces, at paper scale
    (96^3 grids of about 5 mm): the parameters of a link take 26x less memory than
    its grid, while the mean error against that grid stays about a millimetre, and
    the surrogate form of the check decides waypoints within its error bound of the
    grid form (the fallback decides the rest exactly)."""
    sc = sg.make_scene("paper", W=120, N=6000)
    ctx = sdf.Context(0, torch.cuda.current_stream())
    grids = sdf.sdf_build_grids(ctx, sc.meshes, sc.resolution, sc.margin)
    L = sc.n_links
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(71, L))
    n = 1 << 20
    X = torch.empty((L, n, 3), dtype=torch.float32, device="cuda")
    Y = torch.empty((L, n), dtype=torch.float32, device="cuda")
    for l in range(L):
        sdf.sdf_surrogate_sample(ctx, grids, l, n, 7, 0.10, 3000 + l, X[l], Y[l])
    sur.train(X, Y, n, 0, 8000, 1e-3)
    sur.train(X, Y, n, 8000, 4000, 2e-4)
    assert ctx.synchronize() == 0
    del X, Y
    grid_bytes = sc.resolution ** 3 * 4
    net_bytes = sdf.SDF_MLP_PARAMS * 4
    assert grid_bytes / net_bytes >= 26.0
    errs = [(sur.error(l, 1 << 18, 0, 0.1, seed=4000 + l), sur.error(l, 1 << 18, 10, 0.1, seed=5000 + l))
            for l in range(L)]
    mean = max(max(u[1], v[1]) for u, v in errs)
    eps = max(max(u[0], v[0]) for u, v in errs)
    print(f"memory {grid_bytes / net_bytes:.1f}x smaller, mean error {mean * 1e3:.2f} mm, max {eps * 1e2:.2f} cm")
    assert mean <= 3e-3
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    q, pts = sc.q.astype(np.float32), sc.points.astype(np.float32)
    bound = 2.0 * eps + 0.01          # the sampled maximum, with room for unsampled points
    d, l, p, rech, sd = _sur_check(sdf, ctx, robot, sur, q, pts, 0.0, bound)
    g = _grid_check(sdf, ctx, robot, q, pts)
    keep = rech == 0
    assert np.all(np.abs(d[keep].astype(np.float64) - g[0][keep]) <= bound)
    assert np.array_equal(d[~keep].view(np.uint32), g[0][~keep].view(np.uint32))
