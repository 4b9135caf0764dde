"""Fitting a signed-distance network to a watertight mesh (Sec. 3.1), on the GPU.

Every step: seeded training points (80% near the surface, 20% uniform), exact
signed-distance targets from the brute-force mesh kernel (nsdf_mesh_sdf),
f and grad f from nsdf_query and their gradients from the hand-written
nsdf_backward (through the autograd Function), loss = mean |f - d| + lambda *
mean (||grad f|| - 1)^2, and an Adam update of the packed FP32 weight blob.
The paper trains with the L1 loss alone; the eikonal term keeps grad f a unit
normal away from the samples.  Checkpoints hold the blob, the optimiser state,
the step and the seeds, so a resumed fit continues bit-identically.
"""

import time

import numpy as np
import torch

import synth

from . import NSDF_FP32, NeuralSDF, nsdf_mesh_sdf
from .autograd import sdf_query


class MeshFit:
    def __init__(self, arch, V, F, n_points=250_000, lr=1e-3, eikonal=0.1, init_seed=0,
                 sample_seed=1000, lr_halving=500):
        self.arch = arch
        self.V, self.F = np.asarray(V), np.asarray(F)
        self.n_points = n_points
        self.eikonal = eikonal
        self.sample_seed = sample_seed
        self.net = NeuralSDF(arch, NSDF_FP32)
        self.blob = torch.from_numpy(synth.geometric_init(arch, init_seed)).cuda().requires_grad_(True)
        self.opt = torch.optim.Adam([self.blob], lr=lr)
        self.sched = torch.optim.lr_scheduler.StepLR(self.opt, lr_halving, 0.5)
        self.Vd = torch.from_numpy(self.V.astype(np.float32)).cuda().contiguous()
        self.Fd = torch.from_numpy(self.F.astype(np.int32)).cuda().contiguous()
        self.step_index = 0

    def targets(self, P):
        d = torch.empty(P.shape[0], device="cuda")
        nsdf_mesh_sdf(self.Vd, self.Fd, P, d)
        return d

    def step(self):
        P = torch.from_numpy(synth.training_points(
            self.V, self.F, self.n_points, self.sample_seed + self.step_index)).cuda()
        d = self.targets(P)
        f, g = sdf_query(P, self.blob, self.net)
        l1 = (f - d).abs().mean()
        eik = ((g.norm(dim=1) - 1.0) ** 2).mean()
        loss = l1 + self.eikonal * eik
        self.opt.zero_grad(set_to_none=True)
        loss.backward()
        self.opt.step()
        self.sched.step()
        self.step_index += 1
        return float(loss.detach()), float(l1.detach()), float(eik.detach())

    def run(self, steps, log_every=0):
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            loss, l1, eik = self.step()
            hist.append((loss, l1, eik))
            if log_every and self.step_index % log_every == 0:
                print(f"step {self.step_index}: loss {loss:.5f} l1 {l1:.5f} eik {eik:.5f}", flush=True)
        torch.cuda.synchronize()
        return hist, (time.perf_counter() - t0) / max(steps, 1)

    def state_dict(self):
        return {"blob": self.blob.detach().cpu(), "opt": self.opt.state_dict(),
                "sched": self.sched.state_dict(), "step": self.step_index,
                "sample_seed": self.sample_seed, "eikonal": self.eikonal}

    def save(self, path):
        torch.save(self.state_dict(), path)

    def load(self, path):
        st = torch.load(path, map_location="cuda", weights_only=False)
        with torch.no_grad():
            self.blob.copy_(st["blob"].cuda())
        self.opt.load_state_dict(st["opt"])
        self.sched.load_state_dict(st["sched"])
        self.step_index = st["step"]
        self.sample_seed = st["sample_seed"]
        self.eikonal = st["eikonal"]

    def weights(self):
        return self.blob.detach().cpu().numpy()


def penalty_gradient(net, blob, pts, eps):
    """d/dp sum max(0, eps - f(p))^2 for every vertex (first-order backward path)."""
    P = pts.detach().clone().requires_grad_(True)
    f, _ = sdf_query(P, blob.detach(), net)
    loss = (torch.clamp(eps - f, min=0.0) ** 2).sum()
    loss.backward()
    return P.grad
