"""Gradient of the L1 fitting loss (Sec. 3.1) of the 512-wide body-scale
network on the 16-bit tensor-core path (nsdf_l1_grad), against the FP64
oracle's reverse mode (loss_backward with a_i = sign(f_i - d_i) / n, v = 0).

Targets sit at least 0.01 from the oracle's f, beyond the 16-bit forms' sdf
error (< 5e-3), so sign(f - d) is the same decision on both sides.  Per
layer the gradient is compared in relative Frobenius norm; the bound follows
from the arithmetic: every saved activation and delta is rounded to the
context's 16-bit type (relative 2^-9 for BF16, 2^-12 for FP16) on top of the
errors of the 16-bit chain itself (normal angles up to ~4e-3 rad for BF16,
~5e-4 for FP16), and the products sum over the points with FP32
accumulation, so relative errors of a few 1e-3 (BF16) and a few 1e-4 (FP16)
are expected; the bounds are 2e-2 and 5e-3.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp
from synth.weights import layer_shapes

pytestmark = pytest.mark.gpu

BODY = synth.Arch(3, 512, 8, 4, 100.0)
TOL = {"bf16": 2e-2, "fp16": 5e-3}


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def make_problem(n, seed):
    blob = synth.geometric_init(BODY, 0)
    pts = synth.body_scale_points(n, seed)
    f, _, _ = mlp.forward(blob, BODY, pts[:, :3])
    s = synth.Stream(seed + 1)
    off = s.uniform(n, 0.01, 0.1) * np.where(s.uniform(n) < 0.5, -1.0, 1.0)
    d = (f + off).astype(np.float32)
    a = np.sign(f - d.astype(np.float64)) / n
    g_ref, _ = mlp.loss_backward(blob, BODY, pts[:, :3], a, np.zeros((n, 3)))
    return blob, pts, d, g_ref, np.abs(f - d).mean()


@pytest.fixture(scope="module")
def problem():
    return make_problem(1000, 17)              # several tiles and a ragged tail


@pytest.fixture(scope="module")
def big_problem():
    # more tiles than CTAs: every CTA also walks fully masked tiles
    return make_problem(25_000, 21)


def blocks(arch):
    """(name, slice) of every weight matrix and bias in the blob."""
    out, off = [], 0
    for l, (o, i) in enumerate(layer_shapes(arch)):
        out.append((f"W{l}", slice(off, off + o * i)))
        off += o * i
        out.append((f"b{l}", slice(off, off + o)))
        off += o
    return out


def check_l1_grad(nsdf, problem, prec):
    blob, pts, d, g_ref, loss_ref = problem
    p = nsdf.NSDF_BF16 if prec == "bf16" else nsdf.NSDF_FP16
    net = nsdf.NeuralSDF(BODY, p).load(blob)
    P = torch.from_numpy(pts).cuda()
    D = torch.from_numpy(d).cuda()
    g = torch.full((blob.size,), float("nan"), device="cuda")
    loss = torch.zeros(1, device="cuda")
    nsdf.nsdf_l1_grad(net.ctx, P, D, g, loss)
    nsdf.nsdf_sync_status(net.ctx)
    g1 = g.cpu().numpy().astype(np.float64)
    g2 = torch.empty_like(g)
    nsdf.nsdf_l1_grad(net.ctx, P, D, g2)
    nsdf.nsdf_sync_status(net.ctx)
    net.close()
    assert np.isfinite(g1).all()
    np.testing.assert_array_equal(g2.cpu().numpy(), g1.astype(np.float32))
    assert abs(float(loss) - loss_ref) <= 5e-3 * max(loss_ref, 1e-3) + 1e-3
    worst = 0.0
    for name, sl in blocks(BODY):
        ref = g_ref[sl]
        nrm = np.linalg.norm(ref)
        if nrm == 0.0:
            assert np.abs(g1[sl]).max() <= 1e-6, name
            continue
        err = np.linalg.norm(g1[sl] - ref) / nrm
        worst = max(worst, err)
        assert err <= TOL[prec], (name, err)
    print(prec, len(pts), "points: worst relative layer error", worst)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_l1_grad_matches_oracle_and_is_deterministic(nsdf, problem, prec):
    check_l1_grad(nsdf, problem, prec)


def test_l1_grad_with_more_tiles_than_ctas(nsdf, big_problem):
    check_l1_grad(nsdf, big_problem, "bf16")


def test_l1_grad_rejects_fp32_contexts_and_empty_batches(nsdf, problem):
    blob, pts, d, _, _ = problem
    net = nsdf.NeuralSDF(BODY, nsdf.NSDF_FP32).load(blob)
    P, D = torch.from_numpy(pts).cuda(), torch.from_numpy(d).cuda()
    g = torch.empty(blob.size, device="cuda")
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_l1_grad(net.ctx, P, D, g)
    assert e.value.status == 6
    net.close()
    net = nsdf.NeuralSDF(BODY, nsdf.NSDF_BF16).load(blob)
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_l1_grad(net.ctx, P[:0], D[:0], g)
    assert e.value.status == 1
    net.close()


@pytest.mark.parametrize("arch", [synth.Arch(3, 512, 2, -1, 100.0), synth.Arch(3, 512, 5, 1, 100.0),
                                  synth.Arch(3, 512, 4, 3, 100.0)],
                         ids=["2-layers-no-skip", "5-layers-skip-at-1", "4-layers-skip-at-3"])
def test_l1_grad_other_shapes(nsdf, arch):
    """Other depths and skip positions: the skip layer's p columns, a skip at
    L1 (L0 then feeds it) and no skip at all go through other branches of the
    gradient's assembly."""
    n = 700
    blob = synth.geometric_init(arch, 3)
    pts = synth.body_scale_points(n, 31)
    f, _, _ = mlp.forward(blob, arch, pts[:, :3])
    s = synth.Stream(32)
    d = (f + s.uniform(n, 0.01, 0.1) * np.where(s.uniform(n) < 0.5, -1.0, 1.0)).astype(np.float32)
    g_ref, _ = mlp.loss_backward(blob, arch, pts[:, :3], np.sign(f - d.astype(np.float64)) / n,
                                 np.zeros((n, 3)))
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_BF16).load(blob)
    g = torch.full((blob.size,), float("nan"), device="cuda")
    nsdf.nsdf_l1_grad(net.ctx, torch.from_numpy(pts).cuda(), torch.from_numpy(d).cuda(), g)
    nsdf.nsdf_sync_status(net.ctx)
    net.close()
    g = g.cpu().numpy().astype(np.float64)
    assert np.isfinite(g).all()
    for name, sl in blocks(arch):
        nrm = np.linalg.norm(g_ref[sl])
        if nrm == 0.0:
            assert np.abs(g[sl]).max() <= 1e-6, name
            continue
        assert np.linalg.norm(g[sl] - g_ref[sl]) / nrm <= TOL["bf16"], name
