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


def layer_shapes(arch):
    """[(out, in)] for L0 .. L{n_hidden} (the last entry is the output layer)."""
    shapes = []
    for l in range(arch.n_hidden + 1):
        fan_in = arch.in_dim if l == 0 else arch.width
        if l == arch.n_hidden:
            fan_out = 1
        elif arch.skip_layer > 0 and l == arch.skip_layer - 1:
            fan_out = arch.width - arch.in_dim
        else:
            fan_out = arch.width
        shapes.append((fan_out, fan_in))
    return shapes


def n_params(arch):
    return sum(o * i + o for o, i in layer_shapes(arch))


def unpack(blob, arch, dtype=np.float64):
    """Split a packed blob into [(W [out x in], b [out])] without copying data."""
    blob = np.asarray(blob)
    assert blob.size == n_params(arch), (blob.size, n_params(arch))
    out, off = [], 0
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
