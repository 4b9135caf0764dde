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

from . import NSDF_BF16, NSDF_FP32, NeuralSDF, nsdf_l1_grad, nsdf_mesh_sdf
from .autograd import sdf_query


class MeshFit:
    """FP32 fitting with the hand-written backward (L1 + eikonal).

    pool_points=None draws fresh seeded training points every step (the
    targets from the brute-force mesh kernel each time); pool_points=N samples
    N points once, as the paper does (Sec. 3.1 samples a fixed set per shape),
    computes their targets once, and draws a seeded batch of n_points from the
    pool every step.
    """

    def __init__(self, arch, V, F, n_points=250_000, lr=1e-3, eikonal=0.1, init_seed=0,
                 sample_seed=1000, lr_halving=500, pool_points=None):
        self.arch = arch
        self.V, self.F = np.asarray(V), np.asarray(F)
        self.n_points = n_points
        self.eikonal = eikonal
        self.sample_seed = sample_seed
        self.net = NeuralSDF(arch, NSDF_FP32)
        init = synth.fourier_relu_init if getattr(arch, "ff_freqs", 0) > 0 else synth.geometric_init
        self.blob = torch.from_numpy(init(arch, init_seed)).cuda().requires_grad_(True)
        self.opt = torch.optim.Adam([self.blob], lr=lr)
        self.sched = torch.optim.lr_scheduler.StepLR(self.opt, lr_halving, 0.5)
        self.Vd = torch.from_numpy(self.V.astype(np.float32)).cuda().contiguous()
        self.Fd = torch.from_numpy(self.F.astype(np.int32)).cuda().contiguous()
        self.step_index = 0
        self.pool_points = pool_points
        if pool_points:
            self.pool_P = torch.from_numpy(
                synth.training_points(self.V, self.F, pool_points, sample_seed)).cuda()
            self.pool_d = self.targets(self.pool_P)

    def targets(self, P):
        d = torch.empty(P.shape[0], device="cuda")
        nsdf_mesh_sdf(self.Vd, self.Fd, P, d)
        return d

    def batch(self):
        """This step's training points and exact targets."""
        if self.pool_points:
            st = synth.Stream(self.sample_seed + 1 + self.step_index, tag=401)
            idx = torch.from_numpy((st.u64(self.n_points) % np.uint64(self.pool_points)).astype(np.int64))
            idx = idx.cuda()
            return self.pool_P[idx], self.pool_d[idx]
        P = torch.from_numpy(synth.training_points(
            self.V, self.F, self.n_points, self.sample_seed + self.step_index)).cuda()
        return P, self.targets(P)

    def step(self):
        P, d = self.batch()
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
                "sample_seed": self.sample_seed, "eikonal": self.eikonal,
                "pool_points": self.pool_points}

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
        if st.get("pool_points") != self.pool_points:
            raise ValueError("checkpoint was written with pool_points=%r" % st.get("pool_points"))

    def weights(self):
        return self.blob.detach().cpu().numpy()


def penalty_gradient(net, blob, pts, eps):
    """d/dp sum max(0, eps - f(p))^2 for every vertex (first-order backward path)."""
    P = pts.detach().clone().requires_grad_(True)
    f, _ = sdf_query(P, blob.detach(), net)
    loss = (torch.clamp(eps - f, min=0.0) ** 2).sum()
    loss.backward()
    return P.grad


class MeshFitTC:
    """Fitting the 512-wide body-scale network, or one of the paper's
    Fourier-feature ReLU networks (Sec. 4.3), on the 16-bit tensor-core path.

    As in the paper (Sec. 3.1, Sec. 4.3), the training set is sampled once: a
    pool of seeded points (80% near the surface, 20% uniform) with exact
    signed distances from the brute-force mesh kernel; every step draws a
    seeded batch from the pool, repacks the FP32 weight blob into the
    kernel's 16-bit layouts, takes the gradient of the paper's L1 loss from
    nsdf_l1_grad (tensor-core forward and reverse passes, weight-gradient
    products over the batch) and applies Adam to the FP32 blob.
    """

    def __init__(self, arch, V, F, precision=NSDF_BF16, pool_points=1_000_000,
                 batch=250_000, lr=1e-4, init_seed=0, sample_seed=3000, lr_halving=500):
        self.arch = arch
        self.batch = batch
        self.sample_seed = sample_seed
        self.net = NeuralSDF(arch, precision)
        init = synth.fourier_relu_init if getattr(arch, "ff_freqs", 0) > 0 else synth.geometric_init
        self.blob = torch.from_numpy(init(arch, init_seed)).cuda().requires_grad_(True)
        self.opt = torch.optim.Adam([self.blob], lr=lr)
        self.sched = torch.optim.lr_scheduler.StepLR(self.opt, lr_halving, 0.5)
        Vd = torch.from_numpy(np.asarray(V, dtype=np.float32)).cuda().contiguous()
        Fd = torch.from_numpy(np.asarray(F, dtype=np.int32)).cuda().contiguous()
        self.pool_P = torch.from_numpy(synth.training_points(V, F, pool_points, sample_seed)).cuda()
        self.pool_d = torch.empty(pool_points, device="cuda")
        nsdf_mesh_sdf(Vd, Fd, self.pool_P, self.pool_d)
        self.grad = torch.empty_like(self.blob, requires_grad=False)
        self.loss = torch.zeros(1, device="cuda")
        self.step_index = 0

    def step(self):
        s = synth.Stream(self.sample_seed + 1 + self.step_index, tag=402)
        idx = torch.from_numpy((s.u64(self.batch) % np.uint64(self.pool_P.shape[0])).astype(np.int64))
        idx = idx.cuda()
        P, d = self.pool_P[idx], self.pool_d[idx]
        self.net.load(self.blob.detach())
        nsdf_l1_grad(self.net.ctx, P, d, self.grad, self.loss)
        self.blob.grad = self.grad
        self.opt.step()
        self.sched.step()
        self.step_index += 1
        return self.loss

    def run(self, steps):
        """Runs `steps` steps; returns (L1 loss per step, seconds per step)."""
        losses = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            losses.append(self.step().clone())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / max(steps, 1)
        return [float(x) for x in losses], dt

    def weights(self):
        return self.blob.detach().cpu().numpy()

    def close(self):
        self.net.close()
