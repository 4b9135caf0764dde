"""The paper's own network shape (Sec. 4.3): a Fourier-feature layer, then
ReLU layers of 256 units (8 for the dragon, 4 for the bunny), in the FP32
fused kernel, against the FP64 oracle.

A ReLU slope is a 0/1 decision on the sign of a pre-activation.  Where the
oracle's pre-activation lies within the FP32 rounding of the kernel's (about
1e-6 here), the two can take different decisions and the gradients then
legitimately differ.  So the normal is compared only at points whose every
pre-activation is at least MARGIN from 0 (the decision is the same in any
precision down to FP32); the sdf, which is continuous through a kink, is
compared everywhere.  Tolerances: the FP32 ones, |delta sdf| <= 1e-5,
angle <= 1e-4 rad.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp
from parity import normal_angle

pytestmark = pytest.mark.gpu

DRAGON = synth.Arch(3, 256, 8, -1, 100.0, "relu", 128)
BUNNY = synth.Arch(3, 256, 4, -1, 100.0, "relu", 128)
EPS = 0.002
SDF_TOL, ANG_TOL, MARGIN = 1e-5, 1e-4, 2e-5


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def gpu_collide(nsdf, arch, blob, pts, T=None):
    s = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(blob)
    d = torch.from_numpy(pts).cuda()
    out, ns = torch.empty_like(d), torch.empty_like(d)
    hit = torch.empty(len(pts), dtype=torch.uint8, device="cuda")
    s.collide(d, EPS, T=T, out_pts=out, out_n_sdf=ns, out_hit=hit)
    nsdf.nsdf_sync_status(s.ctx)
    s.close()
    return out.cpu().numpy(), ns.cpu().numpy(), hit.cpu().numpy()


def margins(blob, arch, pts):
    _, zs, _ = mlp.forward(blob, arch, pts[:, :3].astype(np.float64))
    return np.min([np.abs(z).min(axis=1) for z in zs], axis=0)


@pytest.mark.parametrize("arch", [DRAGON, BUNNY], ids=["8x256", "4x256"])
def test_fourier_relu_matches_oracle(nsdf, arch):
    blob = synth.fourier_relu_init(arch, 0)
    pts = synth.body_scale_points(4096, 1)
    out, ns, hit = gpu_collide(nsdf, arch, blob, pts)
    f, N, hit_ref, x = mlp.collide(blob, arch, pts, EPS)
    assert np.abs(ns[:, 3] - f).max() <= SDF_TOL
    safe = margins(blob, arch, pts) > MARGIN
    assert safe.mean() >= 0.95
    assert normal_angle(N[safe], ns[safe, :3]).max() <= ANG_TOL
    far = safe & (np.abs(f - EPS) > 1e-4)
    np.testing.assert_array_equal(hit[far], hit_ref[far])
    np.testing.assert_allclose(out[far, :3], x[far], atol=2e-5)


def test_fourier_relu_with_pose_and_tiles_edge(nsdf):
    """A posed body (Sec. 4.2) and a ragged point count (several tiles and a tail)."""
    blob = synth.fourier_relu_init(BUNNY, 3)
    pts = synth.uniform_cube_points(1000 + 37, 4)
    T = synth.rigid_transforms(1, seed=12)[0]
    out, ns, hit = gpu_collide(nsdf, BUNNY, blob, pts, T=T)
    f, N, _, x = mlp.collide(blob, BUNNY, pts, EPS, T=T)
    assert np.abs(ns[:, 3] - f).max() <= SDF_TOL
    Ti = np.linalg.inv(T.astype(np.float64))
    local = pts[:, :3] @ Ti[:3, :3].T + Ti[:3, 3]
    safe = margins(blob, BUNNY, local) > MARGIN
    assert normal_angle(N[safe], ns[safe, :3]).max() <= ANG_TOL


def test_fourier_relu_grouped_equals_single(nsdf):
    nets = 3
    counts = np.array([500, 0, 1300], dtype=np.int64)
    offs = np.array([0, 500, 500], dtype=np.int64)
    pts = synth.body_scale_points(1800, 5)
    blobs = [synth.fourier_relu_init(BUNNY, k) for k in range(nets)]
    g = nsdf.NeuralSDF(BUNNY, nsdf.NSDF_FP32, n_nets=nets)
    for k, b in enumerate(blobs):
        g.load(b, net=k)
    P = torch.from_numpy(pts).cuda()
    out, ns = torch.zeros_like(P), torch.zeros_like(P)
    nsdf.nsdf_query_grouped(g.ctx, P, torch.from_numpy(offs).cuda(), torch.from_numpy(counts).cuda(),
                            1800, EPS, out, ns)
    nsdf.nsdf_sync_status(g.ctx)
    g.close()
    ns = ns.cpu().numpy()
    for k in (0, 2):
        sl = slice(offs[k], offs[k] + counts[k])
        _, ref_ns, _ = gpu_collide(nsdf, BUNNY, blobs[k], pts[sl].copy())
        np.testing.assert_array_equal(ns[sl], ref_ns)


def test_unsupported_and_invalid_shapes(nsdf):
    with pytest.raises(nsdf.NsdfError) as e:                 # 16-bit ReLU: not offered
        nsdf.NeuralSDF(synth.Arch(3, 512, 8, -1, 100.0, "relu", 0), nsdf.NSDF_BF16)
    assert e.value.status == 6
    with pytest.raises(nsdf.NsdfError) as e:                 # 2m != width
        nsdf.NeuralSDF(synth.Arch(3, 256, 4, -1, 100.0, "relu", 64), nsdf.NSDF_FP32)
    assert e.value.status == 1
    with pytest.raises(nsdf.NsdfError) as e:                 # Fourier features with a skip
        nsdf.NeuralSDF(synth.Arch(3, 256, 4, 2, 100.0, "relu", 128), nsdf.NSDF_FP32)
    assert e.value.status == 1
