"""Pins of ``oracle.rounded``: the Fourier-feature ReLU network (Sec. 4.3)
with its tensor-core operands rounded to a 16-bit format.

The rounding itself is checked against library conversions (torch's
float32 -> bfloat16, numpy's float64 -> float16, both round to nearest even).
Each rounding point of the network (weights, activations, deltas of the
reverse chain) is pinned by a network built so that rounding that point, and
no other, changes f or grad f by an amount worked out by hand below; a
dropped or misplaced rounding fails one of them.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp, rounded

M = 128
W = 256


def ff_arch(L):
    return synth.Arch(3, W, L, -1, 100.0, "relu", M)


def blob_of(B, layers):
    parts = [np.asarray(B, dtype=np.float64).ravel()]
    for Wl, bl in layers:
        parts += [np.asarray(Wl, dtype=np.float64).ravel(), np.asarray(bl, dtype=np.float64).ravel()]
    return np.concatenate(parts)


def test_round16_matches_library_conversions():
    s = synth.Stream(21)
    x = s.normal(20000, std=3.0).astype(np.float32)
    # exact ties and near-ties next to 1.0 for both formats, both signs
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11,
                     1 + 2.0 ** -8 + 2.0 ** -20, 2.0 ** -130, 65504.0, 1e-6], dtype=np.float32)
    x = np.concatenate([x, ties, -ties]).astype(np.float32)
    bf = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(rounded.round16(x.astype(np.float64), "bf16"), bf)
    fp = x.astype(np.float64).astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(rounded.round16(x.astype(np.float64), "fp16"), fp)
    assert rounded.round16(np.array([1 + 2.0 ** -8]), "bf16")[0] == 1.0          # tie to even
    assert rounded.round16(np.array([1 + 3 * 2.0 ** -8]), "bf16")[0] == 1 + 2.0 ** -6


def test_weight_rounding():
    """L = 1, B = 0 (gamma = [0]*m + [1]*m), W_0 = 1 + 2^-10 everywhere, no
    bias, w_out = 2^-8: z = m (1 + 2^-10) exactly, f = 256 * 2^-8 * z = z.
    BF16 holds 8 significant bits, so W_0 rounds to 1 and f = 128; FP16
    holds 11 and keeps W_0, f = 128.125."""
    arch = ff_arch(1)
    blob = blob_of(np.zeros((M, 3)), [(np.full((W, 2 * M), 1 + 2.0 ** -10), np.zeros(W)),
                                      (np.full((1, W), 2.0 ** -8), np.zeros(1))])
    p = synth.uniform_cube(5, 1)[:, :3].astype(np.float64)
    f_exact, _ = mlp.query(blob, arch, p, raw_gradient=True)
    np.testing.assert_allclose(f_exact, 128.125, rtol=1e-15)
    f, g, _ = rounded.query_ff_relu(blob, arch, p, "bf16")
    np.testing.assert_array_equal(f, 128.0)
    assert np.abs(g).max() == 0.0
    f, _, _ = rounded.query_ff_relu(blob, arch, p, "fp16")
    np.testing.assert_array_equal(f, 128.125)


def test_activation_rounding():
    """L = 2, B = 0, W_0 = 0 and b_0 = 1 + 2^-9: h_0 = 1 + 2^-9, which BF16
    rounds to 1 (spacing 2^-7) and FP16 keeps.  W_1 = 1/256 (exact), so
    z_1 = h_0 in every unit; f reads the unrounded h_1 through
    w_out = (1, 0, ..., 0): f = 1 in BF16 and 1 + 2^-9 in FP16."""
    arch = ff_arch(2)
    w_out = np.zeros((1, W))
    w_out[0, 0] = 1.0
    blob = blob_of(np.zeros((M, 3)), [(np.zeros((W, 2 * M)), np.full(W, 1 + 2.0 ** -9)),
                                      (np.full((W, W), 1.0 / 256), np.zeros(W)),
                                      (w_out, np.zeros(1))])
    p = synth.uniform_cube(5, 2)[:, :3].astype(np.float64)
    np.testing.assert_allclose(mlp.query(blob, arch, p)[0], 1 + 2.0 ** -9, rtol=1e-15)
    np.testing.assert_array_equal(rounded.query_ff_relu(blob, arch, p, "bf16")[0], 1.0)
    np.testing.assert_array_equal(rounded.query_ff_relu(blob, arch, p, "fp16")[0], 1 + 2.0 ** -9)


def test_delta_rounding_and_feature_jacobian():
    """L = 1 at p = 0 with every frequency b_j = (1, 0, 0): the phases are 0,
    so d sin / dp = 2 pi b_j and d cos / dp = 0.  b_0 = 1 keeps every unit
    on; w_out = 1 + 2^-10 everywhere, so delta_0 = w_out rounds to 1 in
    BF16; W_0 = 2^-8 (exact) gives g_sin,j = 256 * 2^-8 * delta = delta and
    grad f = 2 pi * m * delta * (1, 0, 0) = 256 pi delta e_x."""
    arch = ff_arch(1)
    B = np.zeros((M, 3))
    B[:, 0] = 1.0
    blob = blob_of(B, [(np.full((W, 2 * M), 2.0 ** -8), np.ones(W)),
                       (np.full((1, W), 1 + 2.0 ** -10), np.zeros(1))])
    p = np.zeros((1, 3))
    _, g_exact = mlp.query(blob, arch, p, raw_gradient=True)
    np.testing.assert_allclose(g_exact[0], [256 * np.pi * (1 + 2.0 ** -10), 0, 0], rtol=1e-14)
    _, g, _ = rounded.query_ff_relu(blob, arch, p, "bf16")
    np.testing.assert_allclose(g[0], [256 * np.pi, 0, 0], rtol=1e-14)
    _, g, _ = rounded.query_ff_relu(blob, arch, p, "fp16")
    np.testing.assert_allclose(g[0], g_exact[0], rtol=1e-14)


def test_hidden_delta_rounding():
    """L = 2 at p = 0, b_j = (1, 0, 0), every unit on (b_0 = b_1 = 1).
    W_1 = (1 + 2^-9) / 256 rounds (BF16) to 2^-8 exactly (the spacing at
    2^-8 is 2^-15 and the excess 2^-17 is a quarter of it); w_out = 1, so
    delta_1 = 1 and W_1^T delta_1 = 256 W_1 = 1 in BF16; W_0 = 2^-8 then
    gives g_sin,j = 1 and grad f = 256 pi e_x.  In FP16, W_1 is held
    exactly; W_1^T delta_1 = 1 + 2^-9, which is representable, so grad f =
    256 pi (1 + 2^-9) e_x."""
    arch = ff_arch(2)
    B = np.zeros((M, 3))
    B[:, 0] = 1.0
    blob = blob_of(B, [(np.full((W, 2 * M), 2.0 ** -8), np.ones(W)),
                       (np.full((W, W), (1 + 2.0 ** -9) / 256), np.ones(W)),
                       (np.ones((1, W)), np.zeros(1))])
    p = np.zeros((1, 3))
    _, g, _ = rounded.query_ff_relu(blob, arch, p, "bf16")
    np.testing.assert_allclose(g[0], [256 * np.pi, 0, 0], rtol=1e-14)
    _, g, _ = rounded.query_ff_relu(blob, arch, p, "fp16")
    np.testing.assert_allclose(g[0], [256 * np.pi * (1 + 2.0 ** -9), 0, 0], rtol=1e-14)


@pytest.mark.parametrize("fmt,u", [("bf16", 2.0 ** -9), ("fp16", 2.0 ** -12)])
def test_rounded_network_stays_near_the_exact_one(fmt, u):
    """On the paper's shape the rounded f differs from the exact f by a few
    unit roundoffs u (5-8 u measured), and the typical normal by some tens
    of u.  The tail of the normal's error is not small: near the kinks the
    two take different ReLU decisions."""
    arch = ff_arch(4)
    blob = synth.fourier_relu_init(arch, 0)
    p = synth.body_scale_points(512, 1)[:, :3].astype(np.float64)
    f0, g0 = mlp.query(blob, arch, p, raw_gradient=True)
    f, g, margin = rounded.query_ff_relu(blob, arch, p, fmt)
    assert np.abs(f - f0).max() <= 16 * u
    cos = np.einsum("ij,ij->i", g, g0) / np.linalg.norm(g, axis=1) / np.linalg.norm(g0, axis=1)
    assert np.median(np.arccos(np.clip(cos, -1, 1))) <= 64 * u
    _, zs, _ = mlp.forward(blob, arch, p)
    exact_margin = np.min([np.abs(z).min(axis=1) for z in zs], axis=0)
    assert np.abs(margin - exact_margin).max() <= 16 * u


def test_l1_grad_equals_the_exact_gradient_when_nothing_rounds():
    """A width-8 network (m = 4, two layers) with B = 0 (features 0 and 1),
    weights in {-1, 0, 1} / 8, biases in {-1, 1} / 8 and w_out in {-1, 1} / 8:
    every pre-activation, activation and delta is a multiple of 1/64 below 2
    in magnitude, exact in BF16, so the 16-bit gradient must equal the exact
    one (B, which is not trained, aside)."""
    arch = synth.Arch(3, 8, 2, -1, 100.0, "relu", 4)
    s = synth.Stream(51)

    def pick(n, vals):
        return np.asarray(vals)[(s.u64(n) % np.uint64(len(vals))).astype(np.int64)] / 8.0

    layers = [(pick(64, [-1, 0, 1]).reshape(8, 8), pick(8, [-1, 1])),
              (pick(64, [-1, 0, 1]).reshape(8, 8), pick(8, [-1, 1])),
              (pick(8, [-1, 1]).reshape(1, 8), np.array([0.25]))]
    blob = blob_of(np.zeros((4, 3)), layers)
    p = synth.uniform_cube(20, 52)[:, :3].astype(np.float64)
    a = synth.Stream(53).normal(20)
    exact = mlp.param_gradient(blob, arch, p, a)
    got = rounded.l1_grad_ff_relu(blob, arch, p, a, "bf16")
    np.testing.assert_allclose(got[12:], exact[12:], rtol=1e-13, atol=1e-13)
    assert np.all(got[:12] == 0.0)


def test_l1_grad_near_the_exact_gradient_on_the_paper_shape():
    """On the 4-layer paper shape with random +-1/n weights a_i (as the L1
    loss gives) the 16-bit gradient lies 2.6% (FP16) and 7.2% (BF16) from
    the exact one in relative Frobenius norm: the ReLU decisions that the
    16-bit pre-activations flip move whole per-point contributions, and the
    signed sum cancels most of the rest.  FP16 must be closer than BF16."""
    arch = ff_arch(4)
    blob = synth.fourier_relu_init(arch, 3)
    p = synth.body_scale_points(800, 5)[:, :3].astype(np.float64)
    a = np.sign(synth.Stream(54).normal(800)) / 800
    exact = mlp.param_gradient(blob, arch, p, a)
    off = arch.ff_freqs * 3
    rel = {}
    for fmt in ("fp16", "bf16"):
        got = rounded.l1_grad_ff_relu(blob, arch, p, a, fmt)
        rel[fmt] = np.linalg.norm(got[off:] - exact[off:]) / np.linalg.norm(exact[off:])
    assert rel["fp16"] <= 0.05 and rel["bf16"] <= 0.15, rel
    assert rel["fp16"] < rel["bf16"], rel
