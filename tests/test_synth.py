"""Checks of the seeded input generators (shapes, determinism, mesh validity)."""

import numpy as np

import synth


def test_stream_is_deterministic_and_uniform():
    a = synth.Stream(42).uniform(100000)
    b = synth.Stream(42).uniform(100000)
    np.testing.assert_array_equal(a, b)
    assert abs(a.mean() - 0.5) < 0.005 and a.min() >= 0.0 and a.max() < 1.0
    n = synth.Stream(42, tag=1).normal(200000)
    assert abs(n.mean()) < 0.01 and abs(n.std() - 1.0) < 0.01


def test_splitmix64_known_values():
    # splitmix64 stepping from state 0 (Steele et al.): the first two outputs
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        out = synth.splitmix64(np.array([g, g * np.uint64(2)], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_param_counts():
    assert synth.n_params(synth.Arch(3, 64, 3, -1)) == 8641
    assert synth.n_params(synth.Arch(3, 512, 8, 4)) == 1839614
    shapes = synth.layer_shapes(synth.Arch(3, 512, 8, 4))
    assert shapes[3] == (509, 512) and shapes[4] == (512, 512) and shapes[8] == (1, 512)


def test_points():
    p = synth.body_scale_points(1 << 16, 1)
    assert p.shape == (1 << 16, 4) and p.dtype == np.float32
    assert np.all(p[:, 3] == 0)
    e = (p[:, 0] / 0.3) ** 2 + (p[:, 1] / 0.5) ** 2 + (p[:, 2] / 0.2) ** 2
    near = np.abs(np.sqrt(e) - 1.0) < 0.2
    assert 0.85 < near.mean() < 0.95
    np.testing.assert_array_equal(p, synth.body_scale_points(1 << 16, 1))
    u = synth.uniform_cube_points(4096, 1)
    assert np.abs(u[:, :3]).max() <= 1.0


def _check_watertight(V, F):
    edges = {}
    for f in F:
        for k in range(3):
            e = (int(f[k]), int(f[(k + 1) % 3]))
            edges[e] = edges.get(e, 0) + 1
    for (i, j), c in edges.items():
        assert c == 1 and edges.get((j, i)) == 1   # each edge once each way
    E = len(edges) // 2
    assert len(V) - E + len(F) == 2
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert vol > 0


def test_meshes_are_closed_and_outward():
    V, F = synth.icosphere(5)
    assert V.shape == (10242, 3) and F.shape == (20480, 3)
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-14)
    _check_watertight(*synth.icosphere(2))
    Vd, Fd = synth.displaced_icosphere(level=3)
    r = np.linalg.norm(Vd, axis=1)
    assert 0.45 <= r.min() and r.max() <= 0.55
    _check_watertight(Vd, Fd)
    _check_watertight(*synth.box_mesh())


def test_counts_and_cloth():
    c = synth.grouped_counts()
    assert c.shape == (16,) and c.min() >= 2000 and c.max() < 400000
    np.testing.assert_array_equal(c, synth.grouped_counts())
    P = synth.cloth_grid(8)
    assert P.shape == (64, 4)
    np.testing.assert_allclose(P[1, 0] - P[0, 0], 2.0 / 7, rtol=1e-6)
    assert synth.spring_list(8).shape[0] == 2 * 8 * 7 + 2 * 7 * 7


def test_rigid_transforms_are_rigid_and_seeded():
    T = synth.rigid_transforms(64, seed=3)
    assert T.shape == (64, 4, 4) and T.dtype == np.float32
    R = T[:, :3, :3].astype(np.float64)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape),
                               atol=1e-6)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-6)
    np.testing.assert_array_equal(T[:, 3], np.broadcast_to([0, 0, 0, 1], (64, 4)))
    assert np.abs(T[:, :3, 3]).max() <= 0.5
    np.testing.assert_array_equal(T, synth.rigid_transforms(64, seed=3))
    assert not np.array_equal(T, synth.rigid_transforms(64, seed=4))
