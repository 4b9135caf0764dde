"""GPU parity of the brute-force mesh-SDF kernel and the cloth step vs the oracle."""

import numpy as np
import pytest
import torch

import synth
from oracle import cloth, mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def gpu_mesh_sdf(nsdf, V, F, pts):
    v = torch.from_numpy(V.astype(np.float32)).cuda().contiguous()
    f = torch.from_numpy(F.astype(np.int32)).cuda().contiguous()
    p = torch.from_numpy(pts).cuda()
    out = torch.empty(pts.shape[0], device="cuda")
    nsdf.nsdf_mesh_sdf(v, f, p, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("level,n", [(3, 3000), (5, 700)])
def test_mesh_sdf_matches_oracle(nsdf, level, n):
    V, F = synth.displaced_icosphere(level=level, seed=7)
    V32 = V.astype(np.float32).astype(np.float64)      # both sides see the FP32 mesh
    pts = synth.body_scale_points(n, 3)
    # add points within 1e-4 of the surface, where the FP64 winding number decides
    s = synth.Stream(4)
    k = F[s.u64(64) % np.uint64(F.shape[0])]
    a, b, c = V32[k[:, 0]], V32[k[:, 1]], V32[k[:, 2]]
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    off = s.uniform(64, -1e-4, 1e-4)
    near = (a + b + c) / 3.0 + off[:, None] * nrm
    pts = np.vstack([pts, np.hstack([near, np.zeros((64, 1))]).astype(np.float32)])
    ref = mesh.signed_distance(pts[:, :3].astype(np.float64), V32, F)
    got = gpu_mesh_sdf(nsdf, V, F, pts)
    np.testing.assert_allclose(got, ref, atol=2e-6, rtol=1e-5)
    # the sign is exact wherever the distance is not ~0
    far = np.abs(ref) > 1e-6
    np.testing.assert_array_equal(np.sign(got[far]), np.sign(ref[far]))


def test_mesh_sdf_box_closed_form(nsdf):
    half = (0.3, 0.2, 0.1)
    V, F = synth.box_mesh(half)
    pts = synth.uniform_cube_points(4000, 8)
    pts[:, :3] *= 0.5
    q = np.abs(pts[:, :3].astype(np.float64)) - np.asarray(half)
    ana = np.linalg.norm(np.maximum(q, 0), axis=1) + np.minimum(q.max(1), 0)
    got = gpu_mesh_sdf(nsdf, V, F, pts)
    np.testing.assert_allclose(got, ana, atol=2e-6)


def test_mesh_sdf_ignores_bad_face_indices(nsdf):
    V, F = synth.box_mesh()
    pts = synth.uniform_cube_points(100, 9)
    good = gpu_mesh_sdf(nsdf, V, F, pts)
    Fbad = np.vstack([F, [[0, 1, 999]], [[-5, 2, 3]]])
    bad = gpu_mesh_sdf(nsdf, V, Fbad, pts)
    np.testing.assert_array_equal(good, bad)


def test_cloth_step_matches_oracle(nsdf):
    n = 64
    P = synth.cloth_grid(n)
    S = synth.spring_list(n)
    P64 = P[:, :3].astype(np.float64)
    rest = np.linalg.norm(P64[S[:, 1]] - P64[S[:, 0]], axis=1)
    jitter = synth.Stream(5).normal(n * n * 3, std=1e-3).reshape(n * n, 3)
    X = P.copy()
    X[:, :3] += jitter.astype(np.float32)
    Xp = P.copy()
    Xp[:, 1] += 1e-3
    h = 2.0 / (n - 1)
    # rest lengths exactly as the grid defines them: h along rows and columns,
    # sqrt(2) h on the diagonals
    rest = np.where(np.isclose(rest, h), h, np.sqrt(2.0) * h)
    ref = cloth.verlet_step(X, Xp, S, rest, 1e5, 1e-3)
    x = torch.from_numpy(X).cuda()
    xp = torch.from_numpy(Xp).cuda()
    nsdf.nsdf_cloth_step(x, xp, n, n, h, h, 1e5, 9.81, 1e-3)
    torch.cuda.synchronize()
    got = xp.cpu().numpy()
    np.testing.assert_allclose(got[:, :3], ref, atol=2e-6)
    np.testing.assert_array_equal(got[:, 3], X[:, 3])
