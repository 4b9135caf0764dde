"""GPU parity of the voxel SDF baseline (the comparison system of Sec. 4.3):
the trilinear-lookup collision query against ``oracle.voxel`` on grids made
here (never read back from the GPU), and the grid build against the exact
mesh SDF of ``oracle.mesh`` at sampled nodes.  FP32 lookups: f within 1e-5,
normals within 1e-4 rad where the gradient is not degenerate."""

import numpy as np
import pytest
import torch

import synth
from oracle import mesh, voxel
from parity import normal_angle

pytestmark = pytest.mark.gpu

EPS = 0.002
LO, HI = np.array([-1.0, -0.9, -1.1]), np.array([1.0, 1.1, 0.95])


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def make_grid(n, seed=3):
    """A sphere-like signed distance plus seeded noise, [n, n, n] (z, y, x)."""
    h = (HI - LO) / (n - 1)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x, y, z = LO[0] + h[0] * i, LO[1] + h[1] * j, LO[2] + h[2] * k
    noise = synth.Stream(seed).normal(n ** 3, std=0.01).reshape(n, n, n)
    return (np.sqrt(x * x + (1.3 * y) ** 2 + z * z) - 0.5 + noise).astype(np.float32)


def gpu_collide(nsdf, grid, n, pts):
    g = torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    d = torch.from_numpy(pts).cuda()
    out, ns = torch.full_like(d, -7.0), torch.full_like(d, -7.0)
    hit = torch.full((len(pts),), 9, dtype=torch.uint8, device="cuda")
    nsdf.nsdf_voxel_collide(g, n, LO, HI, d, EPS, out, ns, hit)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ns.cpu().numpy(), hit.cpu().numpy().astype(bool)


@pytest.mark.parametrize("npts", [1, 255, 257, 10000])
def test_lookup_matches_oracle(nsdf, npts):
    n = 33
    grid = make_grid(n)
    pts = np.zeros((npts, 4), dtype=np.float32)
    pts[:, :3] = synth.uniform_cube(npts, 11) * 1.2          # some points outside the box
    pts[:, 3] = 2.5
    out, ns, hit = gpu_collide(nsdf, grid, n, pts)
    f, N, hit_o, x = voxel.collide(grid.astype(np.float64), LO, HI, pts, EPS)
    assert np.abs(ns[:, 3] - f).max() <= 1e-5
    ok = np.linalg.norm(N, axis=1) > 1e-3
    assert normal_angle(N[ok], ns[ok, :3]).max() <= 1e-4
    far = np.abs(f - EPS) > 1e-5
    np.testing.assert_array_equal(hit[far], hit_o[far])
    np.testing.assert_array_equal(hit, ns[:, 3] < EPS)
    exp = pts[:, :3].astype(np.float64).copy()
    exp[hit] += (EPS - ns[hit, 3:4].astype(np.float64)) * ns[hit, :3]
    np.testing.assert_allclose(out[:, :3], exp, atol=2e-6)
    np.testing.assert_array_equal(out[:, 3], pts[:, 3])


def test_nodes_faces_and_nan_points(nsdf):
    n = 9
    grid = make_grid(n, seed=4)
    h = (HI - LO) / (n - 1)
    idx = np.array([[0, 0, 0], [8, 8, 8], [3, 5, 7], [8, 0, 4]])
    pts = np.zeros((6, 4), dtype=np.float32)
    pts[:4, :3] = LO + h * idx
    pts[4, :3] = [np.nan, 0.0, 0.0]
    pts[5, :3] = [np.inf, -np.inf, 0.0]
    out, ns, hit = gpu_collide(nsdf, grid, n, pts)
    np.testing.assert_allclose(ns[:4, 3], grid[idx[:, 2], idx[:, 1], idx[:, 0]], atol=1e-6)
    assert np.isnan(ns[4, 3])                              # reported, read in bounds


def test_grid_build_matches_exact_mesh_sdf(nsdf):
    V, F = synth.displaced_icosphere(level=3, seed=7)
    n = 24
    lo, hi = -0.8 * np.ones(3), 0.8 * np.ones(3)
    g = torch.empty(n ** 3, device="cuda")
    nsdf.nsdf_voxel_build(torch.from_numpy(V.astype(np.float32)).cuda(),
                          torch.from_numpy(F.astype(np.int32)).cuda(), n, lo, hi, g)
    torch.cuda.synchronize()
    grid = g.cpu().numpy().reshape(n, n, n)
    h = (hi - lo) / (n - 1)
    sel = (synth.Stream(12).u64(400) % np.uint64(n ** 3)).astype(np.int64)
    i, j, k = sel % n, (sel // n) % n, sel // (n * n)
    p = np.stack([lo[0] + h[0] * i, lo[1] + h[1] * j, lo[2] + h[2] * k], axis=1)
    V32 = V.astype(np.float32).astype(np.float64)          # the vertices the kernel reads
    d = mesh.signed_distance(p, V32, F)
    np.testing.assert_allclose(grid.ravel()[sel], d, atol=2e-6, rtol=1e-5)


def test_bad_arguments_are_rejected(nsdf):
    grid = torch.zeros(8, device="cuda")
    d = torch.zeros(4, 4, device="cuda")
    out = torch.empty_like(d)
    for n, lo, hi in ((1, LO, HI), (2, HI, LO)):
        with pytest.raises(nsdf.NsdfError) as e:
            nsdf.nsdf_voxel_collide(grid, n, lo, hi, d, EPS, out)
        assert e.value.status == 1
    with pytest.raises(nsdf.NsdfError) as e:                 # host points
        nsdf.nsdf_voxel_collide(grid, 2, LO, HI, torch.zeros(4, 4), EPS, out)
    assert e.value.status == 1
    with pytest.raises(nsdf.NsdfError) as e:                 # misaligned
        nsdf.nsdf_voxel_collide(grid, 2, LO, HI, d.view(-1)[1:13].view(3, 4), EPS, out[:3])
    assert e.value.status == 2
    nsdf.nsdf_voxel_collide(grid, 2, LO, HI, d[:0], EPS, out[:0])     # n = 0: no-op
