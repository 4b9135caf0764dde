"""Network shapes, the packed weight blob and the geometric initialisation.

Shape convention (the SDF network f: R^3 -> R of Eq. 1):

* ``n_hidden`` hidden layers L0 .. L{n_hidden-1}, each ``width`` wide, then
  the output layer L{n_hidden} (width -> 1).
* With a skip connection at layer ``s`` (``skip_layer = s``), layer L{s-1}
  outputs ``width - in_dim`` units and L{s} reads the concatenation
  ``[h_{s-1}, p] / sqrt(2)``, so every hidden layer keeps ``width`` inputs.
  The 1/sqrt(2) factor is part of the network definition, not of the blob.

Blob layout: for each layer in order, ``W`` row-major ``[out x in]`` followed
by ``b[out]``, all float32.

Fourier-feature networks (the paper's own architecture, Sec. 4.3: a Fourier
feature input layer (Tancik et al., NeurIPS 2020) followed by ReLU layers):
``ff_freqs = m > 0`` maps p to gamma(p) = [sin(2 pi B p), cos(2 pi B p)]
(2m values, sines first) with a fixed frequency matrix B [m x 3] stored at
the start of the blob; L0 then reads the 2m features.  ``activation`` is
"softplus" (softplus_beta) or "relu".

Geometric initialisation (Atzmon & Lipman, "SAL", CVPR 2020, as used by Gropp
et al., "IGR", ICML 2020): hidden weights ~ N(0, 2/fan_out), zero biases; the
output layer has weights ~ N(sqrt(pi)/sqrt(fan_in), 1e-4^2) and bias -r, so
the initial network approximates the sphere SDF ||p|| - r.  The paper (Sec.
3.1) does not say how its networks were initialised; this initialisation only
supplies seeded weights with a meaningful zero level set.
"""

from dataclasses import dataclass

import numpy as np

from .rng import Stream


@dataclass(frozen=True)
class Arch:
    in_dim: int = 3
    width: int = 64
    n_hidden: int = 3
    skip_layer: int = -1
    beta: float = 100.0
    activation: str = "softplus"     # or "relu"
    ff_freqs: int = 0                # m: Fourier-feature input layer of 2m values


def layer_shapes(arch):
    """[(out, in)] for L0 .. L{n_hidden} (the last entry is the output layer)."""
    shapes = []
    for l in range(arch.n_hidden + 1):
        fan_in = (2 * arch.ff_freqs if arch.ff_freqs > 0 else arch.in_dim) if l == 0 else arch.width
        if l == arch.n_hidden:
            fan_out = 1
        elif arch.skip_layer > 0 and l == arch.skip_layer - 1:
            fan_out = arch.width - arch.in_dim
        else:
            fan_out = arch.width
        shapes.append((fan_out, fan_in))
    return shapes


def n_params(arch):
    return arch.ff_freqs * arch.in_dim + sum(o * i + o for o, i in layer_shapes(arch))


def ff_matrix(blob, arch, dtype=np.float64):
    """The Fourier-feature frequency matrix B [m x 3] of a blob (None if m = 0)."""
    if arch.ff_freqs <= 0:
        return None
    m = arch.ff_freqs
    return np.asarray(blob)[: m * arch.in_dim].reshape(m, arch.in_dim).astype(dtype)


def unpack(blob, arch, dtype=np.float64):
    """Split a packed blob into [(W [out x in], b [out])] (B excluded)."""
    blob = np.asarray(blob)
    assert blob.size == n_params(arch), (blob.size, n_params(arch))
    out, off = [], arch.ff_freqs * arch.in_dim
    for o, i in layer_shapes(arch):
        W = blob[off: off + o * i].reshape(o, i).astype(dtype)
        off += o * i
        b = blob[off: off + o].astype(dtype)
        off += o
        out.append((W, b))
    return out


def geometric_init(arch, seed, radius=0.5):
    """Seeded geometric initialisation; returns the float32 blob."""
    parts = []
    shapes = layer_shapes(arch)
    for l, (o, i) in enumerate(shapes):
        s = Stream(seed, tag=1 + l)
        if l == arch.n_hidden:
            W = s.normal(o * i, mean=np.sqrt(np.pi) / np.sqrt(i), std=1e-4)
            b = np.full(o, -radius)
        else:
            W = s.normal(o * i, mean=0.0, std=np.sqrt(2.0) / np.sqrt(o))
            b = np.zeros(o)
        parts += [W, b]
    return np.concatenate(parts).astype(np.float32)


def fourier_relu_init(arch, seed, sigma=2.0):
    """Seeded weights for a Fourier-feature ReLU network; returns the float32 blob.

    B ~ N(0, sigma^2) (the Gaussian mapping of Tancik et al.), hidden weights
    ~ N(0, 2/fan_in) with zero biases (He et al., ICCV 2015, for ReLU), output
    weights ~ N(0, 1/fan_in) and bias 0, so f is O(1) with both signs.  The
    paper's trained networks are not available; these only supply seeded
    weights of the paper's shape.
    """
    assert arch.activation == "relu"
    parts = []
    if arch.ff_freqs > 0:
        parts.append(Stream(seed, tag=900).normal(arch.ff_freqs * arch.in_dim, std=sigma))
    for l, (o, i) in enumerate(layer_shapes(arch)):
        s = Stream(seed, tag=1 + l)
        std = np.sqrt(1.0 / i) if l == arch.n_hidden else np.sqrt(2.0 / i)
        parts += [s.normal(o * i, std=std), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)
