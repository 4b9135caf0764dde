"""Support rows on the GPU: fitting a network to a mesh (Sec. 3.1), the collision
penalty gradient at 1M vertices, and the cloth simulation step with collisions
(Sec. 4.1), against the FP64 oracle."""

import os

import numpy as np
import pytest
import torch

import synth
from oracle import cloth as ocloth
from oracle import mlp

pytestmark = pytest.mark.gpu

TINY = synth.Arch(3, 64, 3, -1, 100.0)


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def test_fit_reduces_loss_and_resumes_bit_identically(nsdf, tmp_path):
    from paper_2110_01614_gb300.fit import MeshFit
    V, F = synth.displaced_icosphere(level=3, seed=7)
    fit = MeshFit(TINY, V, F, n_points=20000, lr=2e-3)
    hist, _ = fit.run(40)
    assert hist[-1][1] < 0.6 * hist[0][1]            # L1 term drops
    ck = str(tmp_path / "fit.pt")
    fit.save(ck)
    fit.run(5)
    a = fit.weights().copy()
    other = MeshFit(TINY, V, F, n_points=20000, lr=2e-3)
    other.load(ck)
    other.run(5)
    np.testing.assert_array_equal(other.weights(), a)


def test_pool_fit_reduces_loss_and_resumes_bit_identically(nsdf, tmp_path):
    """The pool mode (points and targets sampled once, seeded batches per step)
    trains, and a checkpoint resumes bit-identically; a checkpoint of the
    other mode is refused."""
    from paper_2110_01614_gb300.fit import MeshFit
    V, F = synth.displaced_icosphere(level=3, seed=7)
    fit = MeshFit(TINY, V, F, n_points=20000, lr=2e-3, pool_points=60000)
    hist, _ = fit.run(40)
    assert hist[-1][1] < 0.6 * hist[0][1]
    ck = str(tmp_path / "pool.pt")
    fit.save(ck)
    fit.run(5)
    a = fit.weights().copy()
    other = MeshFit(TINY, V, F, n_points=20000, lr=2e-3, pool_points=60000)
    other.load(ck)
    other.run(5)
    np.testing.assert_array_equal(other.weights(), a)
    fresh = MeshFit(TINY, V, F, n_points=20000, lr=2e-3)
    with pytest.raises(ValueError):
        fresh.load(ck)


def test_fitted_network_matches_mesh_distances(nsdf):
    from paper_2110_01614_gb300.fit import MeshFit
    V, F = synth.displaced_icosphere(level=3, seed=7)
    fit = MeshFit(TINY, V, F, n_points=50000, lr=3e-3)
    fit.run(150)
    blob = fit.weights()
    pts = synth.training_points(V, F, 2000, seed=99)
    from oracle import mesh
    d = mesh.signed_distance(pts[:, :3].astype(np.float64), V, F)
    f, _, _ = mlp.forward(blob, TINY, pts)
    near = np.abs(d) < 0.05
    assert np.median(np.abs(f[near] - d[near])) < 0.01


def test_penalty_gradient_at_1m_vertices(nsdf):
    from paper_2110_01614_gb300.fit import penalty_gradient
    blob = synth.geometric_init(TINY, 0)
    net = nsdf.NeuralSDF(TINY, nsdf.NSDF_FP32)
    n = 1 << 20
    pts_np = synth.body_scale_points(n, 4)
    g = penalty_gradient(net, torch.from_numpy(blob).cuda(), torch.from_numpy(pts_np).cuda(), 0.002)
    torch.cuda.synchronize()
    idx = np.sort(synth.Stream(3).u64(2048) % np.uint64(n)).astype(np.int64)
    ref = mlp.penalty_grad_closed_form(blob, TINY, pts_np[idx], 0.002)
    got = g.cpu().numpy()[idx, :3]
    assert np.abs(ref).max() > 0
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-9
    net.close()


def test_cloth_steps_match_oracle(nsdf):
    from paper_2110_01614_gb300.cloth_sim import ClothSim
    n, steps = 32, 3
    blob = synth.geometric_init(TINY, 0)
    body = nsdf.NeuralSDF(TINY, nsdf.NSDF_FP32).load(blob)
    sim = ClothSim(n=n, y0=0.3)
    x = sim.x.cpu().numpy().astype(np.float64)
    xp = sim.x_prev.cpu().numpy().astype(np.float64)
    S = synth.spring_list(n)
    h = 2.0 / (n - 1)
    rest = np.where(np.isclose(np.linalg.norm(x[S[:, 1], :3] - x[S[:, 0], :3], axis=1), h), h,
                    np.sqrt(2.0) * h)
    for _ in range(steps):
        sim.step(body)
        xn, hit = ocloth.step(blob, TINY, x, xp, S, rest, 1e5, 1e-3, 0.002)
        xp, x = x[:, :3], xn
    got = sim.x.cpu().numpy()[:, :3]
    assert np.abs(got - x).max() < 2e-5
    body.close()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tensor_core_fit_of_the_512_wide_network_reduces_l1(nsdf, prec):
    """The 512-wide body-scale network fitted with the paper's L1 loss on the
    16-bit path: the loss on the pool drops, and the fitted network's f is
    closer to the mesh distances than the initial one (FP64 oracle on a
    held-out sample)."""
    from paper_2110_01614_gb300.fit import MeshFitTC
    BODY = synth.Arch(3, 512, 8, 4, 100.0)
    V, F = synth.displaced_icosphere(level=3, seed=7)
    p = nsdf.NSDF_BF16 if prec == "bf16" else nsdf.NSDF_FP16
    fit = MeshFitTC(BODY, V, F, precision=p, pool_points=60000, batch=20000, lr=2e-4)
    losses, _ = fit.run(60)
    assert np.mean(losses[-5:]) < 0.7 * np.mean(losses[:5])
    from oracle import mesh
    pts = synth.training_points(V, F, 1000, seed=98)
    d = mesh.signed_distance(pts[:, :3].astype(np.float64), V, F)
    f0, _, _ = mlp.forward(synth.geometric_init(BODY, 0), BODY, pts)
    f1, _, _ = mlp.forward(fit.weights(), BODY, pts)
    assert np.mean(np.abs(f1 - d)) < 0.8 * np.mean(np.abs(f0 - d))
    fit.close()
