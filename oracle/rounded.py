"""The Fourier-feature ReLU network (Sec. 4.3) with its tensor-core operands
rounded to a 16-bit format: the arithmetic of the 16-bit kernels, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Why this exists.  A ReLU slope is a 0/1 decision on the sign of a
pre-activation.  Evaluated with 16-bit operands, pre-activations within the
rounding error of 0 take the other decision than in exact arithmetic, and
for a randomly initialised ReLU network each such flip moves grad f by a
large fraction of its length.  So a 16-bit result is compared with this
function, which takes the decisions in the 16-bit precision, and the
distance of this function from the exact one (``mlp.query``) bounds what the
rounding alone may cost.

Rounding points (everything else is exact FP64):

* the features gamma(p) = [sin(2 pi B p), cos(2 pi B p)] (Sec. 4.3),
* every weight matrix W_0 .. W_{L-1} (biases, w_out and B stay FP32 values),
* every activation h_l = max(z_l, 0) that feeds another product (l < L-1),
* every delta of the reverse chain (Sec. 3.2): delta_{L-1} = [z_{L-1} > 0]
  w_out and delta_{l-1} = [z_{l-1} > 0] (W_l^T delta_l).

f = w_out . h_{L-1} + b_out reads the unrounded h_{L-1}, and the input
gradient g_gamma = W_0^T delta_0 goes through the feature Jacobian
unrounded, as in the kernels' FP32 epilogues.
"""

import numpy as np

from synth.weights import ff_matrix, unpack

FORMATS = ("bf16", "fp16")


def round16(x, fmt):
    """Round to the nearest value of a 16-bit format, ties to even.

    bf16: 8 significant bits, the FP32 exponent range; fp16: IEEE binary16.
    Values are rounded from their FP64 value directly (no FP32 step), by
    scaling to an integer significand and rounding half to even (numpy's
    rint).  Overflow saturates to +-inf as in IEEE; the networks here stay
    far from it.
    """
    x = np.asarray(x, dtype=np.float64)
    if fmt not in FORMATS:
        raise ValueError(fmt)
    p, emin, emax = (8, -126, 127) if fmt == "bf16" else (11, -14, 15)
    out = np.zeros_like(x)
    nz = (x != 0) & np.isfinite(x)
    ax = np.abs(x[nz])
    e = np.floor(np.log2(ax))
    # guard the floor of log2 near powers of two
    e = np.where(ax < 2.0 ** e, e - 1, e)
    e = np.where(ax >= 2.0 ** (e + 1), e + 1, e)
    e = np.maximum(e, emin)                      # subnormals share the minimum exponent
    q = 2.0 ** (e - (p - 1))                     # spacing of the format at |x|
    r = np.rint(ax / q) * q
    r = np.where(r >= 2.0 ** (emax + 1), np.inf, r)
    out[nz] = np.sign(x[nz]) * r
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out


def query_ff_relu(blob, arch, p, fmt):
    """(f, grad f, margin) of a Fourier-feature ReLU network at the rounding
    points listed in the module docstring.

    margin[i] is the smallest |z| over all pre-activations of point i: a
    decision with |z| below the kernels' FP32 accumulation error can still
    differ between this function and a kernel.
    """
    assert arch.activation == "relu" and arch.ff_freqs > 0
    p = np.asarray(p, dtype=np.float64)[:, :3]
    layers = unpack(blob, arch, dtype=np.float64)
    L, m = arch.n_hidden, arch.ff_freqs
    B = ff_matrix(blob, arch)
    phase = 2.0 * np.pi * (p @ B.T)
    x = round16(np.concatenate([np.sin(phase), np.cos(phase)], axis=1), fmt)
    Wr = [round16(layers[l][0], fmt) for l in range(L)]
    masks = []
    margin = np.full(p.shape[0], np.inf)
    h = None
    for l in range(L):
        z = x @ Wr[l].T + layers[l][1]
        margin = np.minimum(margin, np.abs(z).min(axis=1))
        masks.append(z > 0.0)
        h = np.where(masks[-1], z, 0.0)
        if l < L - 1:
            x = round16(h, fmt)
    w_out, b_out = layers[L][0][0], layers[L][1][0]
    f = h @ w_out + b_out
    delta = round16(np.where(masks[L - 1], w_out[None, :], 0.0), fmt)
    for l in range(L - 1, 0, -1):
        delta = round16(np.where(masks[l - 1], delta @ Wr[l], 0.0), fmt)
    g_gamma = delta @ Wr[0]
    coef = g_gamma[:, :m] * np.cos(phase) - g_gamma[:, m:] * np.sin(phase)
    return f, 2.0 * np.pi * (coef @ B), margin


def l1_grad_ff_relu(blob, arch, p, a, fmt):
    """sum_i a_i d f(p_i) / d theta in blob layout, from the 16-bit operands a
    tensor-core fitting step saves (the rounding points of the module
    docstring): dL/dW_l = sum_i a_i delta_l(i) x_l(i)^T with x_0 the rounded
    features, x_l = the rounded h_{l-1} and delta_l the rounded deltas;
    dL/db_l = sum_i a_i delta_l(i); dL/dw_out = sum_i a_i h_{L-1}(i) with
    h_{L-1} rounded as it is saved; dL/db_out = sum_i a_i.  The frequencies B
    are not trained (random Fourier features): their entries are 0.
    Sums are exact (FP64).
    """
    assert arch.activation == "relu" and arch.ff_freqs > 0
    p = np.asarray(p, dtype=np.float64)[:, :3]
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    layers = unpack(blob, arch, dtype=np.float64)
    L, m = arch.n_hidden, arch.ff_freqs
    B = ff_matrix(blob, arch)
    phase = 2.0 * np.pi * (p @ B.T)
    x = round16(np.concatenate([np.sin(phase), np.cos(phase)], axis=1), fmt)
    Wr = [round16(layers[l][0], fmt) for l in range(L)]
    xs, masks = [], []
    h = None
    for l in range(L):
        xs.append(x)
        z = x @ Wr[l].T + layers[l][1]
        masks.append(z > 0.0)
        h = np.where(masks[-1], z, 0.0)
        if l < L - 1:
            x = round16(h, fmt)
    w_out = layers[L][0][0]
    grads = [None] * (L + 1)
    grads[L] = ((a @ round16(h, fmt))[None, :], np.array([a.sum()]))
    delta = round16(np.where(masks[L - 1], w_out[None, :], 0.0), fmt)
    for l in range(L - 1, -1, -1):
        ad = a[:, None] * delta
        grads[l] = (ad.T @ xs[l], ad.sum(0))
        if l > 0:
            delta = round16(np.where(masks[l - 1], delta @ Wr[l], 0.0), fmt)
    parts = [np.zeros(m * 3)]
    parts += [np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads]
    return np.concatenate(parts)
