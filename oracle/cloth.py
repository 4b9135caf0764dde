"""FP64 reference for one explicit cloth step with neural-SDF collisions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4.1: a rectangular quad cloth integrated with explicit Verlet; Sec. 3.2:
after each step, vertices with f(p) < eps move to their contact point.  The
paper gives no cloth parameters; the mass-spring model here (structural and
shear springs, unit mass, Hooke forces, gravity) is the plain textbook one:

  a_i = g + (1/m) sum_{springs (i,j)} k (|x_j - x_i| - r_ij) (x_j - x_i)/|x_j - x_i|
  x_i(t+dt) = 2 x_i(t) - x_i(t-dt) + dt^2 a_i

then the collision solve of ``oracle.mlp.collide`` on x(t+dt).
"""

import numpy as np

from . import mlp


def spring_accel(x, springs, rest, k_over_m, gravity=(0.0, -9.81, 0.0)):
    x = np.asarray(x, dtype=np.float64)[:, :3]
    i, j = springs[:, 0], springs[:, 1]
    d = x[j] - x[i]
    L = np.linalg.norm(d, axis=1)
    f = (k_over_m * (L - rest) / L)[:, None] * d
    acc = np.zeros_like(x)
    np.add.at(acc, i, f)
    np.add.at(acc, j, -f)
    return acc + np.asarray(gravity)[None, :]


def verlet_step(x, x_prev, springs, rest, k_over_m, dt, gravity=(0.0, -9.81, 0.0)):
    """Explicit position-Verlet update (no collisions)."""
    x = np.asarray(x, dtype=np.float64)[:, :3]
    xp = np.asarray(x_prev, dtype=np.float64)[:, :3]
    return 2.0 * x - xp + dt * dt * spring_accel(x, springs, rest, k_over_m, gravity)


def step(blob, arch, x, x_prev, springs, rest, k_over_m, dt, eps,
         gravity=(0.0, -9.81, 0.0), T=None):
    """Verlet step followed by the naive collision solve; returns (x_new, hit)."""
    xn = verlet_step(x, x_prev, springs, rest, k_over_m, dt, gravity)
    _, _, hit, xc = mlp.collide(blob, arch, xn, eps, T)
    return xc, hit
