"""FP64 reference for the network query, its gradient and the collision solve.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions followed:

* Eq. 1: f maps a point p in R^3 to a signed distance.  The network is a
  stack of fully connected layers with softplus_beta activations,
  softplus_beta(z) = log(1 + exp(beta z)) / beta, evaluated here in the exact
  stable form max(z, 0) + log1p(exp(-beta |z|)) / beta (no cut-off).  A skip
  layer s reads [h_{s-1}, p] / sqrt(2).
* Eq. 2: the surface normal is grad f / ||grad f||, with grad f obtained by
  back-propagation (Sec. 3.2): delta_l = sigmoid(beta z_l) * g_l,
  g_{l-1} = W_l^T delta_l.
* Sec. 3.2: a vertex collides when f(p) < eps (strict).
* Eq. 3 with the naive solve (Sec. 3.2): the collided vertex moves to the
  contact point p + (eps - f(p)) N_p.  Eq. 3 prints only the displacement
  (eps - f) N; the point itself is p plus that displacement.
* Sec. 4.2: for a body placed by a rigid transform T (4x4), the query uses
  p' = T^{-1} p and the normal is rotated back by T[:3, :3].

* Sec. 4.3 (the paper's own networks): a Fourier-feature input layer
  gamma(p) = [sin(2 pi B p), cos(2 pi B p)] (Tancik et al. 2020; B [m x 3]
  stored in the blob, sines first) followed by ReLU layers.  Its gradient
  multiplies g_gamma = W_0^T delta_0 by the feature Jacobian:
  d sin(2 pi b.p)/dp = 2 pi cos(2 pi b.p) b, d cos(2 pi b.p)/dp =
  -2 pi sin(2 pi b.p) b.  The ReLU slope is 1 where z > 0 and 0 elsewhere
  (at z = 0 the gradient is taken as 0, as TensorFlow does; Sec. 4.3 notes
  that no gradient flows through a ReLU that outputs 0).

Degenerate gradient: when ||grad f|| < 1e-20 the normal is the zero vector,
so a collided vertex is not moved.
"""

import numpy as np

from synth.weights import ff_matrix, unpack

SQRT2 = np.sqrt(2.0)
DEGENERATE_NORM = 1e-20


def softplus(z, beta):
    """softplus_beta(z) = log(1 + e^{beta z}) / beta, exact stable form."""
    return np.maximum(z, 0.0) + np.log1p(np.exp(-beta * np.abs(z))) / beta


def sigmoid(t):
    """1 / (1 + e^{-t}) without overflow for either sign of t."""
    e = np.exp(-np.abs(t))
    return np.where(t >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def _layers(blob, arch):
    return unpack(blob, arch, dtype=np.float64)


def activation(z, arch):
    """softplus_beta (Eq. 1 networks of this build) or ReLU (Sec. 4.3)."""
    return np.maximum(z, 0.0) if arch.activation == "relu" else softplus(z, arch.beta)


def slope(z, arch):
    """Derivative of the activation: sigmoid(beta z), or the ReLU step (0 at 0)."""
    return (z > 0.0).astype(np.float64) if arch.activation == "relu" else sigmoid(arch.beta * z)


def fourier_features(blob, arch, p):
    """gamma(p) = [sin(2 pi B p), cos(2 pi B p)] [n, 2m], and the phases 2 pi B p."""
    B = ff_matrix(blob, arch)
    phase = 2.0 * np.pi * (p @ B.T)
    return np.concatenate([np.sin(phase), np.cos(phase)], axis=1), phase


def _layer_input(l, h, p, arch, blob=None):
    if l == 0:
        if arch.ff_freqs > 0:
            return fourier_features(blob, arch, p)[0]
        return p
    if arch.skip_layer > 0 and l == arch.skip_layer:
        return np.concatenate([h, p], axis=1) / SQRT2
    return h


def forward(blob, arch, p):
    """f(p) for points p [n, 3] (Eq. 1); returns (f [n], zs, xs).

    zs[l] are the pre-activations of hidden layer l and xs[l] its inputs,
    kept for the gradient.
    """
    p = np.asarray(p, dtype=np.float64)[:, :3]
    layers = _layers(blob, arch)
    zs, xs = [], []
    h = p
    for l in range(arch.n_hidden):
        W, b = layers[l]
        x = _layer_input(l, h, p, arch, blob)
        z = x @ W.T + b
        xs.append(x)
        zs.append(z)
        h = activation(z, arch)
    W, b = layers[arch.n_hidden]
    f = (h @ W.T + b)[:, 0]
    return f, zs, xs


def gradient(blob, arch, p, zs=None):
    """grad_p f by the reverse (Jacobian-transpose) chain (Sec. 3.2, Eq. 2)."""
    p = np.asarray(p, dtype=np.float64)[:, :3]
    if zs is None:
        _, zs, _ = forward(blob, arch, p)
    layers = _layers(blob, arch)
    n = p.shape[0]
    w_out = layers[arch.n_hidden][0][0]
    g = np.broadcast_to(w_out, (n, w_out.size))
    direct = np.zeros((n, 3))
    for l in range(arch.n_hidden - 1, -1, -1):
        W, _ = layers[l]
        delta = slope(zs[l], arch) * g
        u = delta @ W
        if l == 0:
            if arch.ff_freqs > 0:
                # u = g_gamma; chain through the feature Jacobian
                m = arch.ff_freqs
                B = ff_matrix(blob, arch)
                _, phase = fourier_features(blob, arch, p)
                coef = u[:, :m] * np.cos(phase) - u[:, m:] * np.sin(phase)
                return 2.0 * np.pi * (coef @ B) + direct
            return u + direct
        if arch.skip_layer > 0 and l == arch.skip_layer:
            k = W.shape[1] - 3
            direct = direct + u[:, k:] / SQRT2
            g = u[:, :k] / SQRT2
        else:
            g = u
    raise AssertionError("unreachable")


def normalise(g):
    """Eq. 2: N = g / ||g||, the zero vector where ||g|| < 1e-20."""
    nrm = np.linalg.norm(g, axis=1, keepdims=True)
    safe = np.where(nrm < DEGENERATE_NORM, 1.0, nrm)
    return np.where(nrm < DEGENERATE_NORM, 0.0, g / safe)


def query(blob, arch, p, raw_gradient=False):
    """(f, n) per point: n = N_p (Eq. 2), or grad f if raw_gradient."""
    f, zs, _ = forward(blob, arch, p)
    g = gradient(blob, arch, p, zs)
    return f, (g if raw_gradient else normalise(g))


def collide(blob, arch, p_world, eps, T=None):
    """Collision test and naive solve (Sec. 3.2, Eq. 3, Sec. 4.2).

    Returns (f, N_world, hit, x_new):
      p' = T^{-1} p (or p), f = f(p'), N = normalise(grad f(p')),
      N_world = T[:3,:3] N, hit = f < eps,
      x_new = p + (eps - f) N_world where hit, else p.
    """
    pw = np.asarray(p_world, dtype=np.float64)[:, :3]
    if T is not None:
        T = np.asarray(T, dtype=np.float64).reshape(4, 4)
        Ti = np.linalg.inv(T)
        pl = pw @ Ti[:3, :3].T + Ti[:3, 3]
    else:
        pl = pw
    f, N = query(blob, arch, pl)
    if T is not None:
        N = N @ T[:3, :3].T
    hit = f < eps
    x_new = pw + np.where(hit[:, None], (eps - f)[:, None] * N, 0.0)
    return f, N, hit, x_new


def loss_backward(blob, arch, p, a, v):
    """Gradients of L = sum_i a_i f(p_i) + v_i . grad f(p_i).

    a [n] and v [n, 3] are the upstream gradients with respect to f and to
    grad f.  Returns (g_blob [n_params] in blob layout, g_p [n, 3]).

    v . grad f is the directional derivative of f along v, so L is computed
    by one forward pass carrying a primal stream (x, z, h) and a tangent
    stream (xd = v at the input, zd = W xd, hd = sigmoid(beta z) * zd), and
    differentiated by plain reverse mode over both streams.  The derivative
    of sigmoid(beta z) is beta s (1 - s); v is a constant, so the tangent
    stream feeds no gradient back to p.
    """
    p = np.asarray(p, dtype=np.float64)[:, :3]
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    beta = arch.beta
    layers = _layers(blob, arch)
    L = arch.n_hidden
    # forward, primal and tangent
    xs, xds, zs, zds, ss = [], [], [], [], []
    h, hd = p, v
    for l in range(L):
        W, b = layers[l]
        if l == 0:
            x, xd = p, v
        elif arch.skip_layer > 0 and l == arch.skip_layer:
            x = np.concatenate([h, p], 1) / SQRT2
            xd = np.concatenate([hd, v], 1) / SQRT2
        else:
            x, xd = h, hd
        z = x @ W.T + b
        zd = xd @ W.T
        s = sigmoid(beta * z)
        xs.append(x); xds.append(xd); zs.append(z); zds.append(zd); ss.append(s)
        h, hd = softplus(z, beta), s * zd
    Wo, _ = layers[L]
    grads = [None] * (L + 1)
    gWo = a @ h + np.ones(p.shape[0]) @ hd          # sum_i (a_i h_i + hd_i)
    grads[L] = (gWo[None, :], np.array([a.sum()]))
    hb = a[:, None] * Wo[0][None, :]                 # dL/dh_{L-1}
    hdb = np.broadcast_to(Wo[0], hb.shape).copy()    # dL/dhd_{L-1}
    pb = np.zeros_like(p)
    for l in range(L - 1, -1, -1):
        W, _ = layers[l]
        s, z, zd = ss[l], zs[l], zds[l]
        zdb = s * hdb
        sb = zd * hdb
        zb = s * hb + sb * beta * s * (1.0 - s)
        gW = zb.T @ xs[l] + zdb.T @ xds[l]
        grads[l] = (gW, zb.sum(0))
        xb = zb @ W
        xdb = zdb @ W
        if l == 0:
            pb += xb
        elif arch.skip_layer > 0 and l == arch.skip_layer:
            k = W.shape[1] - 3
            pb += xb[:, k:] / SQRT2
            hb, hdb = xb[:, :k] / SQRT2, xdb[:, :k] / SQRT2
        else:
            hb, hdb = xb, xdb
    g_blob = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()])
                             for gW, gb in grads])
    return g_blob, pb


def penalty_grad_closed_form(blob, arch, p, eps):
    """Closed form of d/dp sum max(0, eps - f)^2 = -2 max(0, eps - f) grad f."""
    f, zs, _ = forward(blob, arch, p)
    g = gradient(blob, arch, p, zs)
    return (-2.0 * np.maximum(0.0, eps - f))[:, None] * g


def param_gradient(blob, arch, p, a):
    """Gradient of L = sum_i a_i f(p_i) with respect to every parameter, in
    blob layout (first order only; with a_i = sign(f_i - d_i) / n it is the
    gradient of the L1 fitting loss of Sec. 3.1).

    Reverse mode over the forward pass of Eq. 1: delta_l = slope(z_l) * g_l,
    dL/dW_l = sum_i a_i delta_l(i) x_l(i)^T, dL/db_l = sum_i a_i delta_l(i),
    g_{l-1} = W_l^T delta_l (split at the skip layer as in ``gradient``); a
    Fourier-feature layer's frequencies get
    dL/dB_j = sum_i a_i 2 pi (g_sin,j cos(2 pi b_j.p) - g_cos,j sin(2 pi b_j.p)) p_i.
    """
    p = np.asarray(p, dtype=np.float64)[:, :3]
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    layers = _layers(blob, arch)
    L = arch.n_hidden
    _, zs, xs = forward(blob, arch, p)
    h_last = activation(zs[L - 1], arch)
    w_out = layers[L][0][0]
    grads = [None] * (L + 1)
    grads[L] = ((a @ h_last)[None, :], np.array([a.sum()]))
    g = np.broadcast_to(w_out, h_last.shape)
    gB = None
    for l in range(L - 1, -1, -1):
        W, _ = layers[l]
        delta = slope(zs[l], arch) * g
        ad = a[:, None] * delta
        grads[l] = (ad.T @ xs[l], ad.sum(0))
        u = delta @ W
        if l == 0:
            if arch.ff_freqs > 0:
                m = arch.ff_freqs
                _, phase = fourier_features(blob, arch, p)
                coef = u[:, :m] * np.cos(phase) - u[:, m:] * np.sin(phase)
                gB = 2.0 * np.pi * ((a[:, None] * coef).T @ p)
            break
        if arch.skip_layer > 0 and l == arch.skip_layer:
            k = W.shape[1] - 3
            g = u[:, :k] / SQRT2
        else:
            g = u
    parts = [gB.ravel()] if arch.ff_freqs > 0 else []
    parts += [np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads]
    return np.concatenate(parts)
