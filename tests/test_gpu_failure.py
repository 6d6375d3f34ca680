"""Failure detection without a GPU fault.

* Bounded device waits: with SDF_OPT_WAIT_POLLS = 0 every bounded wait gives up at
  its first poll.  The check kernel's sphere-staging wait and the surrogate
  kernels' MMA completion waits must then report SDF_ERR_TIMEOUT through
  sdf_ctx_synchronize (each block first drains its own copy or MMAs with a wait of
  the default length, so nothing is left in flight), and the context must stay
  usable: the next call with the default limit passes parity against the oracle.
* Allocation failure, injected on the host: the k-th library allocation fails as
  if memory were exhausted, for every k along a sequence of calls that covers the
  context, grids, robot, scratch growth, host staging, surrogate and server.  Each
  failing call returns SDF_ERR_OOM, and once every object is released the library
  holds exactly what it held before (no leak).
"""
import numpy as np
import pytest

import oracle
import oracle.mlp as mlp
import scenegen as sg
from tests._gpu import assert_parity, device_check

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
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    return sc, ctx, grids, robot, np.asarray(vals), [np.asarray(m) for m in metas]


def test_staging_wait_gives_up_and_the_context_recovers(sdf, env):
    sc, ctx, grids, robot, vals, metas = env
    default = ctx.get_option(sdf.SDF_OPT_WAIT_POLLS)
    assert default == 1 << 22
    ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, 0)
    try:
        rc, d, _, _ = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
        assert rc == sdf.SDF_ERR_TIMEOUT, rc
        assert "bounded device wait" in ctx.last_error()
        # the status was cleared by the synchronisation that reported it
        assert ctx.synchronize() == sdf.SDF_OK
    finally:
        ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, default)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)
    assert rc == sdf.SDF_OK
    assert_parity(sc.dh, sc.base, vals, metas, sc.q, sc.points, d, al, ap)


def test_wait_polls_option_is_validated(sdf, env):
    ctx = env[1]
    with pytest.raises(sdf.SdfError) as e:
        ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, -1)
    assert e.value.code == sdf.SDF_ERR_INVALID_ARG
    with pytest.raises(sdf.SdfError):
        ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, 1 << 32)
    assert ctx.get_option(sdf.SDF_OPT_WAIT_POLLS) == 1 << 22


def test_mma_wait_gives_up_in_evaluation_and_training(sdf, env):
    sc, ctx, grids, robot, vals, metas = env
    L = len(metas)
    params = sg.mlp_init(61, L)
    sur = sdf.Surrogate(ctx, grids, params)
    rng = np.random.default_rng(62)
    n = 300
    xs = rng.uniform(-1.1, 1.1, (n, 3)).astype(np.float32)
    x_dev = torch.tensor(xs, device="cuda")
    f = torch.full((n,), 5.0, device="cuda")
    default = ctx.get_option(sdf.SDF_OPT_WAIT_POLLS)
    # training samples for one step of every link
    X = torch.tensor(rng.uniform(-1, 1, (L, 128, 3)).astype(np.float32), device="cuda")
    Y = torch.tensor(rng.uniform(-0.2, 0.2, (L, 128)).astype(np.float32), device="cuda")
    ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, 0)
    try:
        sur.eval(2, x_dev, n, f)
        assert ctx.synchronize() == sdf.SDF_ERR_TIMEOUT
        sur.train(X, Y, 128, 0, 1, 1e-3)
        assert ctx.synchronize() == sdf.SDF_ERR_TIMEOUT
    finally:
        ctx.set_option(sdf.SDF_OPT_WAIT_POLLS, default)
    # a training step that gave up changed no parameter
    assert np.array_equal(sur.params(), params)
    # with the default limit the same calls complete and match the oracle
    sur.eval(2, x_dev, n, f)
    assert ctx.synchronize() == sdf.SDF_OK
    ref = mlp.forward(params[2].astype(np.float64), xs.astype(np.float64), quantize=True)
    err = np.abs(f.cpu().numpy() - ref)
    assert err.max() <= 2e-3 * np.max(np.abs(ref)) + 1e-5
    sur.train(X, Y, 128, 0, 1, 1e-3)
    assert ctx.synchronize() == sdf.SDF_OK
    assert not np.array_equal(sur.params(), params)
    sur.close()


def _scenario(sdf, sc, vals, metas, held):
    """Every allocating call of the library once, objects appended to `held`."""
    stream = torch.cuda.current_stream()
    ctx = sdf.Context(0, stream)
    held.append(ctx)
    g_built = sdf.sdf_build_grids(ctx, sc.meshes, 10, sc.margin)
    held.append(g_built)
    grids = sdf.sdf_grids_upload(ctx, vals, metas)
    held.append(grids)
    robot = sdf.Robot(ctx, sc.dh, grids, sc.base)
    held.append(robot)
    rc, d, al, ap = device_check(sdf, torch, ctx, robot, sc.q, sc.points)   # grows the scratch
    assert rc == sdf.SDF_OK
    W, N = sc.q.shape[0], sc.points.shape[0]
    out = [np.empty(W, np.float32), np.empty(W, np.int32), np.empty(W, np.int32)]
    sdf.check_trajectory_host(ctx, robot, sc.q.astype(np.float32), W, sc.points.astype(np.float32), N, *out)
    ctx.set_option(sdf.SDF_OPT_STATS, 1)                                   # statistics buffer
    sur = sdf.Surrogate(ctx, grids, sg.mlp_init(63, len(metas)))
    held.append(sur)
    outs = [torch.empty(W, device="cuda"), torch.empty(W, dtype=torch.int32, device="cuda"),
            torch.empty(W, dtype=torch.int32, device="cuda")]
    sdf.check_trajectory_surrogate(ctx, robot, sur, torch.tensor(sc.q, dtype=torch.float32, device="cuda"), W,
                                   torch.tensor(sc.points, dtype=torch.float32, device="cuda"), N, 0.05, 0.3,
                                   *outs)
    srv = sdf.Server(0, slots=2, max_batch=2, max_waypoints=256, max_points=2000, max_dof=sc.dof)
    held.append(srv)
    assert ctx.synchronize() == sdf.SDF_OK
    return d


def test_injected_allocation_failures_return_oom_and_leak_nothing(sdf, env):
    sc0, _, _, _, _, _ = env
    sc = sg.make_scene("tiny", W=12, N=400)
    vals, metas = oracle.build_grids_cached(sc.meshes, sc.resolution, sc.margin)
    base = sdf.sdf_debug_alloc_live()[:2]
    failures = 0
    for k in range(1, 400):
        held = []
        sdf.sdf_debug_fail_alloc(k)
        completed = False
        try:
            d = _scenario(sdf, sc, vals, metas, held)
            completed = True
        except sdf.SdfError as e:
            assert e.code == sdf.SDF_ERR_OOM, (k, e)
            failures += 1
        finally:
            left = sdf.sdf_debug_alloc_live()[2]
            sdf.sdf_debug_fail_alloc(0)
            for obj in reversed(held):
                obj.close()
            torch.cuda.synchronize()
        assert sdf.sdf_debug_alloc_live()[:2] == base, (k, sdf.sdf_debug_alloc_live(), base)
        if completed:
            # the countdown outlived the scenario: every allocation of it has failed once
            assert left > 0, k
            break
    else:
        pytest.fail("the scenario never completed")
    assert failures >= 20, failures
    ref = oracle.check(sc.dh, sc.base, vals, metas, sc.q, sc.points)[0]
    assert np.abs(d.astype(np.float64) - ref).max() <= 1e-5
