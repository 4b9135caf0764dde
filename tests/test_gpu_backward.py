"""GPU checks of the hand-written backward (nsdf_backward) and its autograd wrapper.

Reference: the FP64 oracle's loss_backward (itself pinned to finite
differences) and finite differences of the FP64 oracle loss.  The GPU path is
FP32; gradients are compared relative to their largest component.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu

REL = 2e-4


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def gpu_backward(nsdf, arch, blob, pts, a, v, weights=True, points=True):
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(blob)
    P = torch.from_numpy(pts).cuda()
    A = torch.from_numpy(a.astype(np.float32)).cuda()
    V = None
    if v is not None:
        V = torch.zeros(len(a), 4, device="cuda")
        V[:, :3] = torch.from_numpy(v.astype(np.float32))
    gw = torch.empty(synth.n_params(arch), device="cuda") if weights else None
    gp = torch.empty_like(P) if points else None
    nsdf.nsdf_backward(net.ctx, P, A, V, gw, gp)
    torch.cuda.synchronize()
    net.close()
    return (gw.cpu().numpy() if weights else None), (gp.cpu().numpy()[:, :3] if points else None)


def close(got, ref, rel=REL):
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= rel * scale, (np.abs(got - ref).max(), scale)


@pytest.mark.parametrize("arch,n", [(synth.Arch(3, 64, 3, -1, 100.0), 3001),
                                    (synth.Arch(3, 32, 4, 2, 100.0), 517),
                                    (synth.Arch(3, 32, 3, 1, 50.0), 64)])
def test_weight_and_point_gradients_match_oracle(nsdf, arch, n):
    blob = synth.geometric_init(arch, 1)
    pts = synth.body_scale_points(n, 2)
    s = synth.Stream(5)
    a = s.normal(n) / n
    v = s.normal(3 * n).reshape(n, 3) / n
    gw, gp = gpu_backward(nsdf, arch, blob, pts, a, v)
    rw, rp = mlp.loss_backward(blob, arch, pts, a, v)
    close(gw, rw)
    close(gp, rp)


def test_first_order_penalty_gradient_body_scale(nsdf):
    """d/dp sum max(0, eps - f)^2 = -2 max(0, eps - f) grad f on the 512-wide net."""
    arch = synth.Arch(3, 512, 8, 4, 100.0)
    blob = synth.geometric_init(arch, 0)
    pts = synth.body_scale_points(2048, 3)
    f, _, _ = mlp.forward(blob, arch, pts)
    a = -2.0 * np.maximum(0.0, 0.002 - f)
    _, gp = gpu_backward(nsdf, arch, blob, pts, a, None, weights=False)
    ref = mlp.penalty_grad_closed_form(blob, arch, pts, 0.002)
    assert (np.abs(ref).sum(1) > 0).sum() > 100
    close(gp, ref, 1e-4)


def test_matches_finite_differences_of_oracle_loss(nsdf):
    arch = synth.Arch(3, 32, 2, -1, 20.0)
    blob = synth.geometric_init(arch, 3).astype(np.float64)
    pts = synth.uniform_cube_points(40, 4)
    s = synth.Stream(6)
    a = s.normal(40)
    v = s.normal(120).reshape(40, 3)
    gw, gp = gpu_backward(nsdf, arch, blob.astype(np.float32), pts, a, v)

    def loss(bl):
        f, zs, _ = mlp.forward(bl, arch, pts)
        g = mlp.gradient(bl, arch, pts, zs)
        return a @ f + np.sum(v * g)

    idx = synth.Stream(7).u64(60) % np.uint64(blob.size)
    h = 1e-6
    for i in idx.astype(np.int64):
        e = np.zeros_like(blob)
        e[i] = h
        fd = (loss(blob + e) - loss(blob - e)) / (2 * h)
        assert abs(gw[i] - fd) <= 1e-3 * max(1.0, np.abs(gw).max() * 1e-2) + 1e-3 * abs(fd), (i, gw[i], fd)


def test_deterministic_and_empty(nsdf):
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    blob = synth.geometric_init(arch, 0)
    pts = synth.uniform_cube_points(5000, 1)
    a = np.ones(5000) / 5000
    v = np.full((5000, 3), 0.1)
    g1, p1 = gpu_backward(nsdf, arch, blob, pts, a, v)
    g2, p2 = gpu_backward(nsdf, arch, blob, pts, a, v)
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(p1, p2)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(blob)
    gw = torch.full((synth.n_params(arch),), 7.0, device="cuda")
    nsdf.nsdf_backward(net.ctx, torch.zeros(0, 4, device="cuda"), torch.zeros(0, device="cuda"),
                       None, gw, None)
    torch.cuda.synchronize()
    assert float(gw.abs().max()) == 0.0
    net.close()


def test_unsupported_shapes_report_cleanly(nsdf):
    arch = synth.Arch(3, 512, 8, 4, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(synth.geometric_init(arch, 0))
    P = torch.zeros(8, 4, device="cuda")
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_backward(net.ctx, P, torch.zeros(8, device="cuda"), None,
                           torch.empty(synth.n_params(arch), device="cuda"), None)
    assert e.value.status == 6
    net.close()


def test_autograd_function(nsdf):
    from paper_2110_01614_gb300.autograd import sdf_query
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    blob0 = synth.geometric_init(arch, 0)
    blob = torch.from_numpy(blob0).cuda().requires_grad_(True)
    pts_np = synth.uniform_cube_points(1000, 3)
    pts = torch.from_numpy(pts_np).cuda().requires_grad_(True)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32)
    d = torch.from_numpy((np.linalg.norm(pts_np[:, :3], axis=1) - 0.5).astype(np.float32)).cuda()
    f, g = sdf_query(pts, blob, net)
    loss = (f - d).abs().mean() + 0.1 * ((g.norm(dim=1) - 1.0) ** 2).mean()
    loss.backward()
    # reference: the same loss through the oracle's backward
    fr, zs, _ = mlp.forward(blob0, arch, pts_np)
    gr = mlp.gradient(blob0, arch, pts_np, zs)
    n = len(fr)
    a = np.sign(fr - d.cpu().numpy()) / n
    nr = np.linalg.norm(gr, axis=1, keepdims=True)
    v = 0.1 * 2.0 * (nr - 1.0) * gr / nr / n
    rw, rp = mlp.loss_backward(blob0, arch, pts_np, a, v)
    close(blob.grad.cpu().numpy(), rw, 1e-3)
    close(pts.grad.cpu().numpy()[:, :3], rp, 1e-3)
    net.close()
