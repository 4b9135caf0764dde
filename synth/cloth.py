"""Rectangular quad cloth (Sec. 4.1): a grid of vertices in a horizontal plane.

Vertex (i, j) (row i along z, column j along x) sits at
(-extent + j*h, y0, -extent + i*h) with h = 2*extent/(n-1).  Springs are
structural ((i,j)-(i,j+1), (i,j)-(i+1,j)) and shear ((i,j)-(i+1,j+1),
(i,j+1)-(i+1,j)); rest lengths are the initial distances.
"""

import numpy as np


def cloth_grid(n=1024, y0=0.6, extent=1.0):
    """float32 [n*n, 4] positions (w = 0), row-major over (i, j)."""
    h = 2.0 * extent / (n - 1)
    c = -extent + h * np.arange(n)
    X, Z = np.meshgrid(c, c, indexing="xy")      # X varies along j, Z along i
    P = np.zeros((n * n, 4), dtype=np.float32)
    P[:, 0] = X.ravel()
    P[:, 1] = y0
    P[:, 2] = Z.ravel()
    return P


def spring_list(n):
    """int64 [S, 2] vertex pairs of all structural and shear springs."""
    idx = np.arange(n * n).reshape(n, n)
    pairs = [
        np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
        np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1),
        np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], 1),
        np.stack([idx[:-1, 1:].ravel(), idx[1:, :-1].ravel()], 1),
    ]
    return np.concatenate(pairs)
