"""The seeded synthetic inputs follow the stated recipe: sizes, link meshes, joint
limits, spline end conditions, cloud geometry (2 cm voxel centres of human-like
clusters at their stated distances, in voxel order), the batched size laws and
the drift of the serving clouds.  These fix the workload the parity tests and the
benchmark run on; none of them involves the method's arithmetic."""
import numpy as np
import pytest

import scenegen as sg


@pytest.fixture(scope="module")
def paper():
    return sg.make_scene("paper")


def test_paper_scene_sizes_and_meshes(paper):
    assert paper.q.shape == (500, 6) and paper.points.shape == (20000, 3)
    assert paper.n_links == 7 and paper.resolution == 96 and paper.margin == 0.05
    assert all(m.n_tris == 1968 for m in paper.meshes[1:])
    lo, hi = paper.dh[:, 4], paper.dh[:, 5]
    assert np.all(paper.q >= lo - 1e-12) and np.all(paper.q <= hi + 1e-12)
    assert np.all(-lo >= np.radians(120) - 1e-9) and np.all(hi <= np.radians(170) + 1e-9)


def test_spline_is_clamped_and_passes_its_end_configurations():
    rng = np.random.default_rng(7)
    dh = sg.gen_arm(rng, 6)
    q = sg.spline_trajectory(np.random.default_rng(8), dh, 5, 1001)
    # zero end velocity: the first and last steps are second order in the spacing
    h = 1.0 / 1000
    v0 = np.abs(q[1] - q[0]).max() / h
    vm = np.abs(q[501] - q[500]).max() / h
    assert v0 < 0.05 * max(vm, 1e-3) + 1e-2
    assert np.all(np.abs(q) <= np.abs(dh[:, 4:6]).max(axis=1) + 1e-12)


def test_paper_cloud_is_voxel_centres_of_three_humans_in_voxel_order(paper):
    p = paper.points
    cells = p / 0.02 - 0.5
    assert np.allclose(cells, np.round(cells), atol=1e-9)          # 2 cm voxel centres
    c = np.round(cells).astype(np.int64)
    assert len(np.unique(c, axis=0)) == len(c)                     # without replacement
    off = c - c.min(axis=0)
    ext = off.max(axis=0) + 1
    lin = off[:, 0] + ext[0] * (off[:, 1] + ext[1] * off[:, 2])
    assert np.all(np.diff(lin) > 0)                                # voxel order, x fastest
    r = np.linalg.norm(p[:, :2], axis=1)
    # torso surfaces 0.2-1.5 m from the base axis; limbs reach at most 0.66 m beyond a torso
    assert r.min() > 0.2 - 0.66 - 0.02 and r.max() < 1.5 + 2 * 0.3 + 0.66 + 0.02


def test_tiny_cloud_uniform_in_a_2m_cube():
    sc = sg.make_scene("tiny")
    assert sc.q.shape == (50, 6) and sc.points.shape == (1000, 3) and sc.resolution == 32
    assert np.all(np.abs(sc.points) <= 1.0)
    assert np.all(np.abs(sc.points.mean(axis=0)) < 0.1)


def test_batched_size_laws():
    b = sg.make_batched(n=16, layouts=2)
    assert len(b.instances) == 16 and [a.dof for a in b.arms] == [6, 7]
    for a, q, pts in b.instances:
        assert 50 <= q.shape[0] <= 1000 and q.shape[1] == b.arms[a].dof
        assert 1 <= pts.shape[0] <= 100000


def test_serving_clouds_drift_by_voxel_steps():
    clouds = sg.drifting_clouds(cycles=12)
    assert len(clouds) == 12
    for c in clouds:
        assert 1 <= len(c) <= 80000 and c.dtype == np.float32
        cells = c.astype(np.float64) / 0.02 - 0.5
        assert np.allclose(cells, np.round(cells), atol=1e-4)
    # consecutive clouds overlap: the clusters move by a few voxels per cycle at most
    a = {tuple(x) for x in np.round(clouds[0].astype(np.float64) / 0.02 - 0.5).astype(np.int64)}
    b = {tuple(x) for x in np.round(clouds[1].astype(np.float64) / 0.02 - 0.5).astype(np.int64)}
    assert len(a & b) > 0
