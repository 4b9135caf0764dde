"""Pins of the FP64 network oracle against what the mathematics fixes.

Each test checks ``oracle.mlp`` against something other than itself: a closed
form for an affine network, a symbolic derivative, central finite
differences, or an exact geometric property of the collision solve (Sec. 3.2,
Eqs. 1-3, Sec. 4.2).
"""

import numpy as np
import pytest

import synth
from oracle import mlp


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers]).astype(np.float64)


def random_layers(arch, seed, wscale=1.0, bias=0.0):
    s = synth.Stream(seed, tag=999)
    out = []
    for o, i in synth.layer_shapes(arch):
        W = s.normal(o * i, std=wscale / np.sqrt(i)).reshape(o, i)
        b = s.normal(o, std=0.1) + bias
        out.append((W, b))
    return out


def affine_closed_form(layers, arch):
    """f(p) = c.p + d for a network whose softplus units all act as identity."""
    M = None
    d = None
    k = None
    for l, (W, b) in enumerate(layers[:-1]):
        if l == 0:
            M, d = W.copy(), b.copy()
        elif arch.skip_layer > 0 and l == arch.skip_layer:
            k = W.shape[1] - 3
            M = (W[:, :k] @ M + W[:, k:]) / np.sqrt(2.0)
            d = W[:, :k] @ d / np.sqrt(2.0) + b
        else:
            M, d = W @ M, W @ d + b
    Wo, bo = layers[-1]
    return (Wo @ M)[0], (Wo @ d + bo)[0]


@pytest.mark.parametrize("skip", [-1, 3])
def test_affine_network_matches_closed_form(skip):
    # biases large enough that beta*z > 200 everywhere: softplus(z) = z to 1e-80
    arch = synth.Arch(3, 8, 5, skip, 100.0)
    layers = random_layers(arch, 3, wscale=0.05, bias=5.0)
    blob = pack(layers)
    p = synth.uniform_cube(64, 11)
    f, zs, _ = mlp.forward(blob, arch, p)
    assert min(z.min() for z in zs) * arch.beta > 200
    c, d = affine_closed_form(layers, arch)
    np.testing.assert_allclose(f, p @ c + d, rtol=1e-13, atol=1e-13)
    g = mlp.gradient(blob, arch, p)
    np.testing.assert_allclose(g, np.broadcast_to(c, g.shape), rtol=1e-13, atol=1e-15)


def test_one_hidden_layer_closed_form():
    # f = sum_j v_j softplus_beta(w_j.p + b_j) + c,  grad f = sum_j v_j sigmoid(beta z_j) w_j
    arch = synth.Arch(3, 16, 1, -1, 100.0)
    layers = random_layers(arch, 5)
    blob = pack(layers)
    (W, b), (V, c) = layers
    p = synth.uniform_cube(128, 12, half=0.3)
    z = p @ W.T + b
    sp = np.logaddexp(0.0, arch.beta * z) / arch.beta
    f_ref = sp @ V[0] + c[0]
    sig = 0.5 * (1.0 + np.tanh(0.5 * arch.beta * z))
    g_ref = (sig * V[0]) @ W
    f, n = mlp.query(blob, arch, p, raw_gradient=True)
    np.testing.assert_allclose(f, f_ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(n, g_ref, rtol=1e-11, atol=1e-14)


def test_symbolic_derivative_tiny_network():
    sympy = pytest.importorskip("sympy")
    arch = synth.Arch(3, 5, 3, 2, 100.0)   # skip at L2: L1 has 2 outputs
    layers = random_layers(arch, 21, wscale=2.0)
    blob = pack(layers)
    X = sympy.symbols("x y z")
    beta = sympy.Integer(100)

    def sp(t):
        return sympy.log(1 + sympy.exp(beta * t)) / beta

    def mat(A):
        return sympy.Matrix([[sympy.Float(float(v), 40) for v in row] for row in np.atleast_2d(A)])

    pv = sympy.Matrix(X)
    h = pv
    for l, (W, b) in enumerate(layers[:-1]):
        x = h
        if l == arch.skip_layer:
            x = sympy.Matrix.vstack(h, pv) / sympy.sqrt(2)
        z = mat(W) * x + mat(b).T
        h = z.applyfunc(sp)
    Wo, bo = layers[-1]
    fexpr = (mat(Wo) * h)[0] + sympy.Float(float(bo[0]), 40)
    grads = [sympy.diff(fexpr, v) for v in X]
    pts = np.array([[0.1, -0.2, 0.05], [-0.03, 0.02, 0.01], [0.4, 0.1, -0.3]])
    f, g = mlp.query(blob, arch, pts, raw_gradient=True)
    for i, q in enumerate(pts):
        sub = {X[0]: q[0], X[1]: q[1], X[2]: q[2]}
        assert abs(float(fexpr.evalf(30, subs=sub)) - f[i]) < 1e-12
        for k in range(3):
            assert abs(float(grads[k].evalf(30, subs=sub)) - g[i, k]) < 1e-11


def fd_gradient(blob, arch, p, h=1e-5):
    """Central differences with one Richardson step (error O(h^4))."""
    p = np.asarray(p, dtype=np.float64)[:, :3]

    def D(step):
        out = np.empty_like(p)
        for k in range(3):
            e = np.zeros(3)
            e[k] = step
            fp, _, _ = mlp.forward(blob, arch, p + e)
            fm, _, _ = mlp.forward(blob, arch, p - e)
            out[:, k] = (fp - fm) / (2 * step)
        return out

    return (4.0 * D(h / 2) - D(h)) / 3.0


@pytest.mark.parametrize("which", ["tiny", "skip"])
def test_gradient_matches_finite_differences(which):
    if which == "tiny":
        arch = synth.Arch(3, 64, 3, -1, 100.0)
        pts = synth.uniform_cube_points(48, 1)
    else:
        arch = synth.Arch(3, 32, 8, 4, 100.0)
        pts = synth.body_scale_points(48, 1)
    blob = synth.geometric_init(arch, 0).astype(np.float64)
    g = mlp.gradient(blob, arch, pts)
    fd = fd_gradient(blob, arch, pts)
    rel = np.linalg.norm(g - fd, axis=1) / np.linalg.norm(fd, axis=1)
    assert rel.max() <= 1e-7, rel.max()


def test_gradient_matches_fd_body_scale_network():
    arch = synth.Arch(3, 512, 8, 4, 100.0)
    blob = synth.geometric_init(arch, 0)
    pts = synth.body_scale_points(8, 1)
    g = mlp.gradient(blob, arch, pts)
    fd = fd_gradient(blob, arch, pts)
    rel = np.linalg.norm(g - fd, axis=1) / np.linalg.norm(fd, axis=1)
    assert rel.max() <= 1e-7, rel.max()


def plane_net(normal, offset, arch=synth.Arch(3, 6, 2, -1, 100.0)):
    """A network computing exactly (to 1e-80) the plane SDF n.p + offset, ||n|| = 1.

    L0 = [I; -I] p + 5 (six units, all active), L1 = identity (+0), output
    = 0.5*n.(u - v) with u, v the two halves, minus the constant it adds.
    """
    n = np.asarray(normal, dtype=np.float64)
    W0 = np.vstack([np.eye(3), -np.eye(3)])
    b0 = np.full(6, 5.0)
    W1 = np.eye(6)
    b1 = np.zeros(6)
    Wo = 0.5 * np.concatenate([n, -n])[None, :]
    bo = np.array([offset])
    return pack([(W0, b0), (W1, b1), (Wo, bo)]), arch


def test_projection_lands_on_offset_surface():
    n = np.array([1.0, 2.0, -2.0]) / 3.0
    blob, arch = plane_net(n, -0.1)
    p = synth.uniform_cube(500, 4)
    eps = 0.002
    f, N, hit, x = mlp.collide(blob, arch, p, eps)
    np.testing.assert_allclose(f, p @ n - 0.1, atol=1e-14)
    np.testing.assert_allclose(N, np.broadcast_to(n, N.shape), atol=1e-14)
    assert hit.any() and (~hit).any()
    # Eq. 3: collided points land exactly on f = eps; others are untouched
    np.testing.assert_allclose(x[hit] @ n - 0.1, eps, atol=1e-14)
    np.testing.assert_array_equal(x[~hit], p[~hit])


def test_collision_test_is_strict():
    blob, arch = plane_net(np.array([0.0, 0.0, 1.0]), 0.0)
    p = np.array([[0.1, 0.2, 0.25], [0.1, 0.2, 0.0]])
    f, _, _ = mlp.forward(blob, arch, p)
    _, _, hit, x = mlp.collide(blob, arch, p, eps=f[0])
    assert not hit[0] and hit[1]
    np.testing.assert_array_equal(x[0], p[0])


def test_degenerate_gradient_moves_nothing():
    arch = synth.Arch(3, 8, 2, -1, 100.0)
    layers = random_layers(arch, 8)
    layers[-1] = (np.zeros((1, 8)), np.array([-1.0]))   # f = -1 everywhere, grad f = 0
    blob = pack(layers)
    p = synth.uniform_cube(16, 2)
    f, N, hit, x = mlp.collide(blob, arch, p, 0.002)
    assert hit.all()
    np.testing.assert_array_equal(N, 0.0)
    np.testing.assert_array_equal(x, p)


def rigid(seed):
    s = synth.Stream(seed, tag=5)
    q = s.normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = s.uniform(3, -0.3, 0.3)
    return T


def test_transform_rule_matches_world_frame_derivative():
    # Sec. 4.2: querying T^{-1} p and rotating N by T[:3,:3] must equal the
    # normalised world-frame gradient of x -> f(T^{-1} x), here by FD.
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    blob = synth.geometric_init(arch, 0).astype(np.float64)
    T = rigid(3)
    Ti = np.linalg.inv(T)
    pw = synth.uniform_cube(32, 9, half=0.8)
    f, N, hit, x = mlp.collide(blob, arch, pw, 0.002, T)

    def fw(q):
        return mlp.forward(blob, arch, q @ Ti[:3, :3].T + Ti[:3, 3])[0]

    h = 1e-5
    g = np.stack([(fw(pw + h * e) - fw(pw - h * e)) / (2 * h) for e in np.eye(3)], 1)
    Nfd = g / np.linalg.norm(g, axis=1, keepdims=True)
    np.testing.assert_allclose(N, Nfd, atol=1e-7)
    np.testing.assert_allclose(f, fw(pw), atol=1e-14)
    np.testing.assert_allclose(x[hit], pw[hit] + (0.002 - f[hit])[:, None] * N[hit], atol=1e-14)


def test_plane_under_transform():
    # a plane z = 0 in the body frame, body rotated and moved: the projected
    # world points must sit at body-frame height eps
    blob, arch = plane_net(np.array([0.0, 0.0, 1.0]), 0.0)
    T = rigid(7)
    Ti = np.linalg.inv(T)
    pw = synth.uniform_cube(400, 6)
    f, N, hit, x = mlp.collide(blob, arch, pw, 0.01, T)
    np.testing.assert_allclose(N, np.broadcast_to(T[:3, 2], N.shape), atol=1e-14)
    xb = x @ Ti[:3, :3].T + Ti[:3, 3]
    np.testing.assert_allclose(xb[hit, 2], 0.01, atol=1e-13)


def fd_loss_grads(blob, arch, p, a, v, h=1e-6):
    def loss(bl, pp):
        f, zs, _ = mlp.forward(bl, arch, pp)
        g = mlp.gradient(bl, arch, pp, zs)
        return float(a @ f + np.sum(v * g))

    gb = np.empty(blob.size)
    for i in range(blob.size):
        e = np.zeros(blob.size)
        e[i] = h
        gb[i] = (loss(blob + e, p) - loss(blob - e, p)) / (2 * h)
    gp = np.empty_like(p)
    for i in range(p.shape[0]):
        for k in range(3):
            e = np.zeros_like(p)
            e[i, k] = h
            gp[i, k] = (loss(blob, p + e) - loss(blob, p - e)) / (2 * h)
    return gb, gp


@pytest.mark.parametrize("skip", [-1, 2])
def test_loss_backward_matches_finite_differences(skip):
    arch = synth.Arch(3, 6, 4, skip, 20.0)
    layers = random_layers(arch, 31, wscale=1.5)
    blob = pack(layers)
    p = synth.uniform_cube(5, 13, half=0.5)
    s = synth.Stream(77)
    a = s.normal(5)
    v = s.normal(15).reshape(5, 3)
    gb, gp = mlp.loss_backward(blob, arch, p, a, v)
    fb, fp = fd_loss_grads(blob, arch, p, a, v)
    np.testing.assert_allclose(gb, fb, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(gp, fp, rtol=1e-6, atol=1e-7)


def test_collision_penalty_gradient():
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    blob = synth.geometric_init(arch, 0).astype(np.float64)
    p = synth.uniform_cube(64, 17, half=0.6)
    eps = 0.002
    f, _, _ = mlp.forward(blob, arch, p)
    assert (f < eps).any() and (f >= eps).any()
    closed = mlp.penalty_grad_closed_form(blob, arch, p, eps)
    _, gp = mlp.loss_backward(blob, arch, p, -2.0 * np.maximum(0.0, eps - f), np.zeros((64, 3)))
    np.testing.assert_allclose(gp, closed, rtol=1e-12, atol=1e-15)

    def penalty(pp):
        ff, _, _ = mlp.forward(blob, arch, pp)
        return np.maximum(0.0, eps - ff) ** 2

    h = 1e-6
    fd = np.stack([(penalty(p + h * e) - penalty(p - h * e)) / (2 * h) for e in np.eye(3)], 1)
    np.testing.assert_allclose(closed, fd, rtol=1e-6, atol=1e-9)


def test_geometric_init_is_a_rough_sphere():
    # a sanity property of the seeded weights (not a parity pin): f grows with
    # ||p|| and changes sign inside the unit cube
    for arch in (synth.Arch(3, 64, 3, -1, 100.0), synth.Arch(3, 512, 8, 4, 100.0)):
        blob = synth.geometric_init(arch, 0)
        p = synth.uniform_cube(512, 1)
        f, _, _ = mlp.forward(blob, arch, p)
        r = np.linalg.norm(p, axis=1)
        assert np.corrcoef(r, f)[0, 1] > 0.75
        assert f.min() < 0 < f.max()


# ---- Fourier-feature ReLU networks (the paper's own architecture, Sec. 4.3) ----

RELU = synth.Arch(3, 32, 3, -1, 100.0, "relu", 0)
FFR = synth.Arch(3, 32, 3, -1, 100.0, "relu", 16)


def _with_B(blob, arch, B):
    b = blob.copy()
    b[: arch.ff_freqs * 3] = np.asarray(B, dtype=np.float32).ravel()
    return b


def test_bias_free_relu_network_is_homogeneous_and_satisfies_euler():
    """Zero biases make a ReLU network positively homogeneous of degree 1:
    f(a p) = a f(p) for a > 0, and by Euler's theorem grad f(p) . p = f(p).
    Softplus in place of ReLU, or a wrong slope, breaks both."""
    blob = synth.fourier_relu_init(RELU, 3)           # all biases are zero
    p = synth.uniform_cube(200, 4)[:, :3].astype(np.float64)
    f, _, _ = mlp.forward(blob, RELU, p)
    for a in (0.5, 2.0, 3.7):
        fa, _, _ = mlp.forward(blob, RELU, a * p)
        np.testing.assert_allclose(fa, a * f, rtol=1e-12, atol=1e-12)
    g = mlp.gradient(blob, RELU, p)
    np.testing.assert_allclose(np.einsum("ij,ij->i", g, p), f, rtol=1e-10, atol=1e-12)


def test_fourier_features_are_periodic_for_integer_frequencies():
    """With B integer, gamma(p + e_k) = gamma(p), so f and grad f are
    1-periodic in every coordinate; a missing 2 pi or a mixed-up feature
    breaks the period."""
    s = synth.Stream(5)
    B = np.round(s.normal(16 * 3, std=2.0)).reshape(16, 3)
    blob = _with_B(synth.fourier_relu_init(FFR, 6), FFR, B)
    p = synth.uniform_cube(100, 7)[:, :3].astype(np.float64) * 0.4
    f, g = mlp.query(blob, FFR, p, raw_gradient=True)
    for k in range(3):
        q = p.copy()
        q[:, k] += 1.0
        fq, gq = mlp.query(blob, FFR, q, raw_gradient=True)
        np.testing.assert_allclose(fq, f, atol=1e-10)
        np.testing.assert_allclose(gq, g, atol=1e-8)


def test_fourier_relu_gradient_matches_central_differences():
    """The chain through the feature Jacobian against central differences of
    the forward pass, at points with every pre-activation away from the
    ReLU kink (the difference step never crosses one)."""
    blob = synth.fourier_relu_init(FFR, 8)
    p = synth.uniform_cube(400, 9)[:, :3].astype(np.float64)
    f, zs, _ = mlp.forward(blob, FFR, p)
    margin = np.min([np.abs(z).min(axis=1) for z in zs], axis=0)
    p = p[margin > 1e-4]
    assert len(p) > 20
    g = mlp.gradient(blob, FFR, p)
    h = 1e-7
    fd = np.stack([(mlp.forward(blob, FFR, p + h * e)[0] - mlp.forward(blob, FFR, p - h * e)[0]) / (2 * h)
                   for e in np.eye(3)], axis=1)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_zero_frequencies_give_a_constant_field():
    """B = 0: gamma(p) = [0 ... 0, 1 ... 1] for every p, so f is constant and
    grad f vanishes."""
    blob = _with_B(synth.fourier_relu_init(FFR, 10), FFR, np.zeros((16, 3)))
    p = synth.uniform_cube(50, 11)[:, :3].astype(np.float64)
    f, g = mlp.query(blob, FFR, p, raw_gradient=True)
    np.testing.assert_allclose(f, f[0], atol=1e-14)
    assert np.abs(g).max() == 0.0


def test_relu_slope_is_zero_at_the_kink():
    """The reading of the ReLU derivative at z = 0: no gradient flows."""
    z = np.array([[-1.0, 0.0, 2.0]])
    np.testing.assert_array_equal(mlp.slope(z, RELU), [[0.0, 0.0, 1.0]])
    np.testing.assert_array_equal(mlp.activation(z, RELU), [[0.0, 0.0, 2.0]])


@pytest.mark.parametrize("skip", [-1, 2])
def test_param_gradient_equals_loss_backward_without_tangent(skip):
    """The first-order parameter gradient is loss_backward with v = 0 (pinned
    above by central differences), for softplus networks with and without a
    skip layer."""
    arch = synth.Arch(3, 16, 4, skip, 100.0)
    blob = pack(random_layers(arch, 41))
    p = synth.uniform_cube(40, 42)[:, :3].astype(np.float64)
    a = synth.Stream(43).normal(40)
    g, _ = mlp.loss_backward(blob, arch, p, a, np.zeros((40, 3)))
    np.testing.assert_allclose(mlp.param_gradient(blob, arch, p, a), g, rtol=1e-12, atol=1e-14)


def test_param_gradient_of_fourier_relu_network_matches_central_differences():
    """sum_i a_i f(p_i) differentiated by central differences in sampled
    parameters of every kind (B, W_l, b_l, w_out, b_out), at points whose
    pre-activations all stay away from 0 (no ReLU decision changes within the
    step)."""
    arch = FFR
    blob = synth.fourier_relu_init(arch, 44).astype(np.float64)
    blob += 0.05 * synth.Stream(45).normal(blob.size)          # non-zero biases too
    p = synth.uniform_cube(300, 46)[:, :3].astype(np.float64)
    _, zs, _ = mlp.forward(blob, arch, p)
    p = p[np.min([np.abs(z).min(axis=1) for z in zs], axis=0) > 1e-3]
    assert len(p) > 10
    a = synth.Stream(47).normal(len(p))
    g = mlp.param_gradient(blob, arch, p, a)
    idx = np.unique(synth.Stream(48).u64(60) % np.uint64(blob.size)).astype(np.int64)
    idx = np.concatenate([idx, [0, 5, blob.size - 1, blob.size - 2]])   # B entries, w_out, b_out
    h = 1e-6

    def loss(b):
        return a @ mlp.forward(b, arch, p)[0]

    for i in idx:
        bp, bm = blob.copy(), blob.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(bp) - loss(bm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
