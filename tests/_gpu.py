"""Helpers for GPU parity tests: run the CUDA path through the C ABI and compare
with the oracle (test infrastructure)."""
import numpy as np

import oracle

DIST_TOL = 1e-5   # metres, per waypoint (FP32 path vs FP64 oracle)


def device_check(sdf, torch, ctx, robot, q, points, stride=3):
    dev = torch.device("cuda", ctx.device)
    W = int(q.shape[0])
    N = int(points.shape[0])
    qd = torch.tensor(np.asarray(q), dtype=torch.float32, device=dev).contiguous()
    p = np.asarray(points, dtype=np.float32).reshape(N, 3)
    if stride == 4:
        p = np.concatenate([p, np.zeros((N, 1), np.float32)], axis=1)
    pd = torch.tensor(p, device=dev).contiguous()
    dist = torch.full((max(W, 1),), 7.0, dtype=torch.float32, device=dev)
    al = torch.full((max(W, 1),), -7, dtype=torch.int32, device=dev)
    ap = torch.full((max(W, 1),), -7, dtype=torch.int32, device=dev)
    sdf.check_trajectory(ctx, robot, qd, W, pd, N, dist, al, ap)
    rc = ctx.synchronize()
    return rc, dist[:W].cpu().numpy(), al[:W].cpu().numpy(), ap[:W].cpu().numpy()


def assert_parity(dh, base, vals, metas, q, points, dist, al, ap, ref=None, tol=DIST_TOL):
    """dist within tol of the oracle; the reported (link, point) attains the oracle
    minimum within tol (several pairs may tie within FP32 rounding)."""
    d_ref, l_ref, p_ref = ref if ref is not None else oracle.check(dh, base, vals, metas, q, points)
    d = dist.astype(np.float64)
    finite = np.isfinite(d_ref)
    assert np.array_equal(np.isfinite(d), finite)
    err = np.abs(d[finite] - d_ref[finite])
    assert err.max(initial=0.0) <= tol, f"max |dist - oracle| = {err.max():.3g} m"
    W = len(d_ref)
    for w in range(W):
        if not finite[w]:
            assert al[w] == -1 and ap[w] == -1
            continue
        if al[w] == l_ref[w] and ap[w] == p_ref[w]:
            continue
        pv = oracle.pair_values(dh, base, vals, metas, np.asarray(q)[w:w + 1],
                                np.asarray(points)[ap[w]:ap[w] + 1])[0, al[w], 0]
        assert abs(pv - d_ref[w]) <= tol, (w, al[w], ap[w], l_ref[w], p_ref[w], pv, d_ref[w])
    return err.max(initial=0.0)
