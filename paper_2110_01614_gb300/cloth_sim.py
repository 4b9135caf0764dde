"""Cloth dropped onto a body represented by a signed-distance network (Sec. 4.1-4.2).

Each step: one explicit Verlet step of the quad mass-spring cloth
(nsdf_cloth_step), then the collision solve of every vertex against the
network (nsdf_collide: f < eps moves the vertex to its contact point), written
in place.  ``ClothSim.run`` times every step with CUDA events.  A brute-force
reference step evaluates the exact mesh SDF of every vertex instead
(nsdf_mesh_sdf), the plain method the network replaces.
"""

import time

import numpy as np
import torch

import synth

from . import nsdf_cloth_step, nsdf_mesh_sdf


class ClothSim:
    def __init__(self, n=1024, y0=0.6, dt=1e-3, k_over_m=1e5, g=9.81, eps=0.002, v0=-1.0):
        self.n, self.dt, self.k, self.g, self.eps = n, dt, k_over_m, g, eps
        self.h = 2.0 / (n - 1)
        x = torch.from_numpy(synth.cloth_grid(n, y0=y0)).cuda()
        self.x = x
        self.x_prev = x.clone()
        self.x_prev[:, 1] -= v0 * dt               # x(t - dt) for velocity (0, v0, 0)

    def step(self, body):
        # Verlet: x_prev <- x_new, then swap so that x holds the new positions
        nsdf_cloth_step(self.x, self.x_prev, self.n, self.n, self.h, self.h, self.k, self.g, self.dt)
        self.x, self.x_prev = self.x_prev, self.x
        body.collide(self.x, self.eps, out_pts=self.x)   # in place (aliasing allowed)

    def run(self, body, steps):
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            self.step(body)
            e1.record()
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ts]


def mesh_reference_step_ms(V, F, pts, repeats=3):
    """Time of the exact brute-force mesh SDF of every vertex (ms per step)."""
    Vd = torch.from_numpy(np.asarray(V, np.float32)).cuda().contiguous()
    Fd = torch.from_numpy(np.asarray(F, np.int32)).cuda().contiguous()
    out = torch.empty(pts.shape[0], device="cuda")
    nsdf_mesh_sdf(Vd, Fd, pts, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(repeats):
        nsdf_mesh_sdf(Vd, Fd, pts, out)
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0) / repeats, out
