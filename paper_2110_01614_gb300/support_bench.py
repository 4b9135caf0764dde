"""Timings of the support workloads around the collision query (one JSON line each).

* fit: one fitting step of the 3-64-64-64-1 network to the displaced
  icosphere (20,480 triangles) with 250,000 points: brute-force mesh SDF
  targets + forward + hand-written backward + Adam (Sec. 3.1); fresh seeded
  points every step, and batches drawn from a pool of 1,048,576 points
  sampled once (as the paper samples a fixed set per shape).
* penalty: gradient of sum max(0, eps - f)^2 with respect to 1,048,576 vertices.
* grouped: 16 networks of the 3-64-64-64-1 shape with log-uniform counts in
  [2k, 400k] (616,218 points) in one grouped launch, autotuned, replayed
  from a CUDA graph; also with a rigid pose per body (nsdf_query_grouped_T);
  FP32 kernel and 16-bit tensor-core kernel (BF16, FP16).
* tiny: 4,096 uniform points through the 3-64-64-64-1 network, one launch.
* grouped_paper: the same 16-body scene with every body posed and carrying
  its own network of the paper's dragon shape (Fourier features + 8 ReLU
  layers of 256), BF16 tensor cores against the FP32 grouped kernel.
* cloth: 1024 x 1024 cloth, per-step time of Verlet + collision solve for the
  body-scale network in BF16 / FP16 / FP32 and for the paper's dragon-shaped
  network in BF16, and of the exact brute-force mesh SDF of every vertex
  (20,480 triangles) as the plain reference.

* paper_arch: the paper's own network shapes (Sec. 4.3: a Fourier-feature
  layer of 128 frequencies, then 8 (dragon) or 4 (bunny) ReLU layers of 256
  units), collision query of 1,048,576 body-scale points in the FP32 kernel
  and in the BF16 / FP16 tensor-core kernel; the paper's Table 1 quotes
  255 ms / 350 ms for 1M queries on a Tesla T4 (context only: other
  hardware, other weights).

* fit512: the 512-wide body-scale network fitted with the paper's L1 loss on
  the BF16 tensor-core path (pool of 1,048,576 points with exact targets,
  batches of 250,000): seconds per step and the time of nsdf_l1_grad alone.
* fit_paper: the same for the paper's dragon-shaped Fourier-feature ReLU
  network.
* cloth_fitted: 100 steps of the 1024 x 1024 cloth dropped onto the displaced
  icosphere represented by a body-scale network fitted to it (BF16 tensor-core
  fitting), per-step time in BF16 / FP16 / FP32 and of the brute-force mesh
  SDF of every vertex.
* voxel: the voxel SDF baseline (Sec. 4.3, Table 1) at N = 256 against the
  fitted body-scale network: build time, memory, query time for 1M points
  and error against the exact signed distance near the surface.
* kernels: the brute-force mesh SDF (65,536 points x 20,480 triangles, far
  from and near the surface) and one 1024 x 1024 cloth step, each alone with
  L2 flushed before every launch: pairs per second, and the cloth step's
  bandwidth against the measured copy bandwidth.

Usage: python -m paper_2110_01614_gb300.support_bench [fit penalty grouped grouped_paper cloth
                                                      paper_arch fit512 fit_paper cloth_fitted
                                                      tiny voxel kernels]
"""

import json
import statistics
import sys
import time

import numpy as np
import torch

import synth

from . import (NSDF_BF16, NSDF_FP16, NSDF_FP32, NeuralSDF, nsdf_mesh_sdf, nsdf_query_grouped,
               nsdf_query_grouped_T, nsdf_sync_status)
from .cloth_sim import ClothSim, mesh_reference_step_ms
from .fit import MeshFit, penalty_gradient
from .tune import tuned_grouped

TINY = synth.Arch(3, 64, 3, -1, 100.0)
BODY = synth.Arch(3, 512, 8, 4, 100.0)


def events_ms(fn, reps):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def bench_fit(steps=20):
    V, F = synth.displaced_icosphere(level=5, seed=7)
    fit = MeshFit(TINY, V, F, n_points=250_000)
    fit.run(3)
    hist, per_step = fit.run(steps)
    # the same from a pool of 1,048,576 points sampled (and given targets) once
    pool = MeshFit(TINY, V, F, n_points=250_000, pool_points=1 << 20)
    pool.run(3)
    phist, pool_per_step = pool.run(steps)
    return {"workload": "fit", "points_per_step": 250_000, "triangles": int(F.shape[0]),
            "s_per_step": per_step, "loss_first": hist[0][0], "loss_last": hist[-1][0],
            "pool_s_per_step": pool_per_step, "pool_loss_first": phist[0][0],
            "pool_loss_last": phist[-1][0]}


def bench_penalty(reps=10):
    net = NeuralSDF(TINY, NSDF_FP32)
    blob = torch.from_numpy(synth.geometric_init(TINY, 0)).cuda()
    pts = torch.from_numpy(synth.body_scale_points(1 << 20, 4)).cuda()
    ms = events_ms(lambda: penalty_gradient(net, blob, pts, 0.002), reps)
    net.close()
    return {"workload": "penalty_gradient", "vertices": 1 << 20, "ms": ms}


def bench_grouped(reps=20, precisions=("fp32", "bf16", "fp16")):
    """16 networks of the 3-64-64-64-1 shape, log-uniform counts in [2k, 400k]
    (616,218 points), one autotuned grouped launch replayed from a CUDA graph,
    with and without a rigid pose per body: the FP32 kernel and the 16-bit
    tensor-core kernel (split-BF16 / FP16 operands, FP32 accumulation)."""
    counts = synth.grouped_counts()
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    total = int(counts.sum())
    P = torch.from_numpy(synth.body_scale_points(total, 5)).cuda()
    O = torch.from_numpy(offs).cuda()
    C = torch.from_numpy(counts.astype(np.int64)).cuda()
    Tdev = torch.from_numpy(synth.rigid_transforms(16, seed=77)).cuda()
    out, ns = torch.empty_like(P), torch.empty_like(P)
    res = {"workload": "grouped", "nets": 16, "points": total}
    for name in precisions:
        prec = {"fp32": NSDF_FP32, "bf16": NSDF_BF16, "fp16": NSDF_FP16}[name]
        net = NeuralSDF(TINY, prec, n_nets=16)
        for k in range(16):
            net.load(synth.geometric_init(TINY, k), net=k)
        pt, cps = tuned_grouped(net, P, O, C, total, 0.002, out, ns)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            nsdf_query_grouped(net.ctx, P, O, C, total, 0.002, out, ns)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            nsdf_query_grouped(net.ctx, P, O, C, total, 0.002, out, ns)
        ms = events_ms(g.replay, reps)
        with torch.cuda.stream(s):
            nsdf_query_grouped_T(net.ctx, P, O, C, total, 0.002, Tdev, out, ns)
        s.synchronize()
        gT = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gT, stream=s):
            nsdf_query_grouped_T(net.ctx, P, O, C, total, 0.002, Tdev, out, ns)
        ms_T = events_ms(gT.replay, reps)
        nsdf_sync_status(net.ctx)
        net.close()
        res[name] = {"ms": ms, "queries_per_s": total / (ms * 1e-3), "posed_ms": ms_T,
                     "posed_queries_per_s": total / (ms_T * 1e-3),
                     "tile_points_per_thread": pt, "ctas_per_sm": cps,
                     "kernel": "query_fp32_kernel" if name == "fp32" else f"query_w64_kernel<{name}>"}
    return res


def bench_tiny(reps=50):
    """The tiny workload: 4,096 uniform points through the 3-64-64-64-1
    network, one collision query per launch (latency-bound)."""
    pts = torch.from_numpy(synth.uniform_cube_points(4096, 1)).cuda()
    out, ns = torch.empty_like(pts), torch.empty_like(pts)
    res = {"workload": "tiny", "points": 4096}
    for name, prec in (("fp32", NSDF_FP32), ("bf16", NSDF_BF16), ("fp16", NSDF_FP16)):
        net = NeuralSDF(TINY, prec).load(synth.geometric_init(TINY, 0))
        net.collide(pts, 0.002, out_pts=out, out_n_sdf=ns)
        ms = events_ms(lambda: net.collide(pts, 0.002, out_pts=out, out_n_sdf=ns), reps)
        nsdf_sync_status(net.ctx)
        net.close()
        res[name] = {"ms": ms, "queries_per_s": 4096 / (ms * 1e-3)}
    return res


def bench_grouped_paper(reps=10):
    """16 posed bodies, each with its own network of the paper's dragon shape,
    counts as in the grouped workload (about 1.2M points), CUDA-graph replay:
    BF16 tensor cores against the FP32 grouped kernel."""
    arch = synth.Arch(3, 256, 8, -1, 100.0, "relu", 128)
    counts = synth.grouped_counts()
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    total = int(counts.sum())
    P = torch.from_numpy(synth.body_scale_points(total, 5)).cuda()
    O = torch.from_numpy(offs).cuda()
    C = torch.from_numpy(counts.astype(np.int64)).cuda()
    Tdev = torch.from_numpy(synth.rigid_transforms(16, seed=77)).cuda()
    out, ns = torch.empty_like(P), torch.empty_like(P)
    res = {"workload": "grouped_paper", "nets": 16, "points": total, "shape": "dragon_8x256"}
    for prec, name, r in ((NSDF_BF16, "bf16", reps), (NSDF_FP32, "fp32", 3)):
        net = NeuralSDF(arch, prec, n_nets=16)
        for k in range(16):
            net.load(synth.fourier_relu_init(arch, k), net=k)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            nsdf_query_grouped_T(net.ctx, P, O, C, total, 0.002, Tdev, out, ns)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            nsdf_query_grouped_T(net.ctx, P, O, C, total, 0.002, Tdev, out, ns)
        ms = events_ms(g.replay, r)
        nsdf_sync_status(net.ctx)
        net.close()
        res[name] = {"ms": ms, "queries_per_s": total / (ms * 1e-3)}
    return res


def bench_cloth(steps=20):
    res = {"workload": "cloth", "grid": "1024x1024", "steps": steps}
    blob = synth.geometric_init(BODY, 0)
    for name, prec in (("bf16", NSDF_BF16), ("fp16", NSDF_FP16), ("fp32", NSDF_FP32)):
        body = NeuralSDF(BODY, prec).load(blob)
        sim = ClothSim(n=1024)
        sim.run(body, 2)
        ts = sim.run(body, steps if name != "fp32" else 3)
        res[f"{name}_ms_per_step"] = statistics.median(ts)
        body.close()
    # the same cloth against the paper's dragon-shaped network (Sec. 4.3) in BF16
    ff = synth.Arch(3, 256, 8, -1, 100.0, "relu", 128)
    body = NeuralSDF(ff, NSDF_BF16).load(synth.fourier_relu_init(ff, 0))
    sim = ClothSim(n=1024)
    sim.run(body, 2)
    res["paper_dragon_bf16_ms_per_step"] = statistics.median(sim.run(body, steps))
    body.close()
    V, F = synth.displaced_icosphere(level=5, seed=7)
    sim = ClothSim(n=1024)
    ms, _ = mesh_reference_step_ms(V, F, sim.x, repeats=2)
    res["mesh_bruteforce_sdf_ms_per_step"] = ms
    return res


def bench_paper_arch(reps=10):
    res = {"workload": "paper_arch", "points": 1 << 20}
    pts = torch.from_numpy(synth.body_scale_points(1 << 20, 1)).cuda()
    out, ns = torch.empty_like(pts), torch.empty_like(pts)
    for name, L in (("dragon_8x256", 8), ("bunny_4x256", 4)):
        arch = synth.Arch(3, 256, L, -1, 100.0, "relu", 128)
        blob = synth.fourier_relu_init(arch, 0)
        # algorithmic MAC per query: L0 and L-1 hidden 256x256 products forward,
        # the same transposed backward (incl. W_0^T), plus the output unit
        mac = 2 * L * 256 * 256 + 256
        res[name] = {}
        for prec, pname in ((NSDF_FP32, "fp32"), (NSDF_BF16, "bf16"), (NSDF_FP16, "fp16")):
            net = NeuralSDF(arch, prec).load(blob)
            net.collide(pts, 0.002, out_pts=out, out_n_sdf=ns)
            ms = events_ms(lambda: net.collide(pts, 0.002, out_pts=out, out_n_sdf=ns), reps)
            nsdf_sync_status(net.ctx)
            net.close()
            res[name][pname] = {"ms": ms, "queries_per_s": (1 << 20) / (ms * 1e-3),
                                "tflops": 2 * mac * (1 << 20) / (ms * 1e-3) / 1e12}
    return res


def bench_fit512(steps=20):
    from . import nsdf_l1_grad
    from .fit import MeshFitTC
    V, F = synth.displaced_icosphere(level=5, seed=7)
    fit = MeshFitTC(BODY, V, F, precision=NSDF_BF16, pool_points=1 << 20, batch=250_000)
    fit.run(2)
    losses, s_per_step = fit.run(steps)
    P, d = fit.pool_P[:250_000], fit.pool_d[:250_000]
    ms = events_ms(lambda: nsdf_l1_grad(fit.net.ctx, P, d, fit.grad, fit.loss), 5)
    fit.close()
    # algorithmic work of the gradient: the query's forward and J^T products
    # (3,670,528 MAC per point) plus the weight-gradient products
    # (7 x 512 x 512 MAC per point)
    mac = 3_670_528 + 7 * 512 * 512
    return {"workload": "fit512", "precision": "bf16", "batch": 250_000, "pool": 1 << 20,
            "s_per_step": s_per_step, "l1_grad_ms": ms,
            "l1_grad_tflops": 2 * mac * 250_000 / (ms * 1e-3) / 1e12,
            "loss_first": losses[0], "loss_last": losses[-1]}


def bench_fit_paper(steps=20):
    """The paper's dragon-shaped network (Fourier features + 8 ReLU layers of
    256) fitted with the L1 loss on the BF16 tensor-core path: pool of
    1,048,576 points with exact targets, batches of 250,000."""
    from . import nsdf_l1_grad
    from .fit import MeshFitTC
    arch = synth.Arch(3, 256, 8, -1, 100.0, "relu", 128)
    V, F = synth.displaced_icosphere(level=5, seed=7)
    fit = MeshFitTC(arch, V, F, precision=NSDF_BF16, pool_points=1 << 20, batch=250_000)
    fit.run(2)
    losses, s_per_step = fit.run(steps)
    P, d = fit.pool_P[:250_000], fit.pool_d[:250_000]
    ms = events_ms(lambda: nsdf_l1_grad(fit.net.ctx, P, d, fit.grad, fit.loss), 5)
    fit.close()
    # algorithmic work of the gradient: the query's forward and J^T products
    # (2 x 8 x 256^2 + 256 MAC per point) plus the weight-gradient products
    # (8 x 256^2 MAC per point)
    mac = 3 * 8 * 256 * 256 + 256
    return {"workload": "fit_paper", "shape": "dragon_8x256", "precision": "bf16", "batch": 250_000,
            "pool": 1 << 20, "s_per_step": s_per_step, "l1_grad_ms": ms,
            "l1_grad_tflops": 2 * mac * 250_000 / (ms * 1e-3) / 1e12,
            "loss_first": losses[0], "loss_last": losses[-1]}


def fit_body(fit_steps=300):
    """The body-scale network (3-512x8-1, skip at L4) fitted to the displaced
    icosphere (20,480 triangles) on the BF16 tensor-core path: L1 loss, pool
    of 1,048,576 points, `fit_steps` batches of 250,000.  Returns the FP32
    blob and the fitting record."""
    from .fit import MeshFitTC
    V, F = synth.displaced_icosphere(level=5, seed=7)
    fit = MeshFitTC(BODY, V, F, precision=NSDF_BF16, pool_points=1 << 20, batch=250_000)
    losses, fit_s = fit.run(fit_steps)
    blob = fit.weights()
    fit.close()
    return blob, {"fit_steps": fit_steps, "fit_s_per_step": fit_s, "fit_l1_first": losses[0],
                  "fit_l1_last": losses[-1]}


def bench_cloth_fitted(steps=100, fit_steps=300, fp32_steps=100, fitted=None):
    """Cloth of 1024 x 1024 vertices dropped for `steps` explicit steps onto
    the displaced icosphere represented by the body-scale network fitted to
    it (fit_body); per-step time of Verlet + collision solve in BF16, FP16 and
    FP32, and of the exact brute-force mesh SDF of every vertex."""
    V, F = synth.displaced_icosphere(level=5, seed=7)
    blob, info = fitted if fitted is not None else fit_body(fit_steps)
    res = {"workload": "cloth_fitted_body", "grid": "1024x1024", "steps": steps,
           "body": "3-512x8-1 (skip L4) fitted to the displaced icosphere", **info}
    for name, prec, k in (("bf16", NSDF_BF16, steps), ("fp16", NSDF_FP16, steps),
                          ("fp32", NSDF_FP32, fp32_steps)):
        body = NeuralSDF(BODY, prec).load(blob)
        sim = ClothSim(n=1024)
        ts = sim.run(body, k)
        nsdf_sync_status(body.ctx)
        body.close()
        res[name] = {"steps": k, "ms_per_step_median": statistics.median(ts),
                     "ms_per_step_mean": statistics.mean(ts)}
        if name == "bf16":
            x_final = sim.x
    ms, _ = mesh_reference_step_ms(V, F, x_final, repeats=3)
    res["mesh_bruteforce_sdf_ms_per_step"] = ms
    return res


def bench_voxel(fitted=None, n=256, reps=20):
    """The voxel SDF baseline of Sec. 4.3 (Table 1) on this build's shape: an
    n^3 grid of exact signed distances to the displaced icosphere over
    [-1, 1]^3 against the fitted body-scale network (BF16): build time,
    memory, collision-query time for 1,048,576 points, and |f - d| against
    the exact signed distance d at 262,144 points (80% near the surface)."""
    from . import nsdf_voxel_build, nsdf_voxel_collide
    V, F = synth.displaced_icosphere(level=5, seed=7)
    blob, _ = fitted if fitted is not None else fit_body()
    Vd = torch.from_numpy(V.astype(np.float32)).cuda().contiguous()
    Fd = torch.from_numpy(F.astype(np.int32)).cuda().contiguous()
    lo, hi = -np.ones(3), np.ones(3)
    grid = torch.empty(n ** 3, device="cuda")
    build_ms = events_ms(lambda: nsdf_voxel_build(Vd, Fd, n, lo, hi, grid), 1)
    pts = torch.from_numpy(synth.body_scale_points(1 << 20, 1)).cuda()
    out, ns = torch.empty_like(pts), torch.empty_like(pts)
    vox_ms = events_ms(lambda: nsdf_voxel_collide(grid, n, lo, hi, pts, 0.002, out, ns), reps)
    net = NeuralSDF(BODY, NSDF_BF16).load(blob)
    net_ms = events_ms(lambda: net.collide(pts, 0.002, out_pts=out, out_n_sdf=ns), reps)
    # accuracy against the exact signed distance near the surface
    P = torch.from_numpy(synth.training_points(V, F, 1 << 18, 4242)).cuda()
    d = torch.empty(P.shape[0], device="cuda")
    nsdf_mesh_sdf(Vd, Fd, P, d)
    o2, n2 = torch.empty_like(P), torch.empty_like(P)
    nsdf_voxel_collide(grid, n, lo, hi, P, 0.002, o2, n2)
    ev = (n2[:, 3] - d).abs()
    net.collide(P, 0.002, out_pts=o2, out_n_sdf=n2)
    en = (n2[:, 3] - d).abs()
    nsdf_sync_status(net.ctx)
    net.close()
    params = synth.n_params(BODY)
    return {"workload": "voxel_vs_network", "grid_n": n, "grid_mb": n ** 3 * 4 / 2 ** 20,
            "grid_build_ms": build_ms, "network_params": params,
            "network_mb_fp32": params * 4 / 2 ** 20, "network_mb_16bit_copies": params * 2 / 2 ** 20,
            "query_1M_ms": {"voxel": vox_ms, "network_bf16": net_ms},
            "abs_error_vs_exact": {
                "points": int(P.shape[0]),
                "voxel": {"mean": float(ev.mean()), "p99": float(ev.quantile(0.99)),
                          "max": float(ev.max())},
                "network_bf16": {"mean": float(en.mean()), "p99": float(en.quantile(0.99)),
                                 "max": float(en.max())}}}


def hbm_peak_gbs():
    """The measured copy bandwidth of this GPU model (MEASURED_PEAKS.json at
    the repository root), or None."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def events_ms_flushed(fn, reps, flush):
    """Median CUDA-event time of fn with L2 flushed (a write larger than L2,
    outside the events) before every launch."""
    ts = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def bench_kernels(mesh_reps=3, cloth_reps=20):
    """The support kernels alone, each against its bound, L2 flushed before
    every launch: the brute-force mesh SDF (FP32 ALU + MUFU bound; FP64 for
    undecided winding numbers) of 1,048,576 points against the
    20,480-triangle displaced icosphere, for points far from the surface
    (uniform in the cube: the FP32 winding number decides) and for fitting
    targets (80% within ~0.01 of the surface: many take the FP64 winding
    number), in point-triangle pairs per second (one warm-up launch each);
    and one Verlet step of the 1024 x 1024 cloth (HBM bound: x and x_prev
    read, x_prev written, 48 bytes per vertex; neighbour reads hit the
    caches) against the measured copy bandwidth (three warm-up launches)."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")    # > L2 (129 MB)
    V, F = synth.displaced_icosphere(level=5, seed=7)
    Vd = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    n = 1 << 20
    res = {"workload": "support_kernels", "l2": "flushed before every launch",
           "mesh_reps": mesh_reps, "cloth_reps": cloth_reps}
    for name, P in (("uniform", synth.uniform_cube_points(n, 3)),
                    ("near_surface", synth.training_points(V, F, n, 5))):
        pts = torch.from_numpy(np.ascontiguousarray(P)).cuda()
        out = torch.empty(n, device="cuda")
        fn = lambda: nsdf_mesh_sdf(Vd, Fd, pts, out)     # noqa: E731
        fn()
        ms = events_ms_flushed(fn, mesh_reps, flush)
        pairs = n * int(F.shape[0])
        res[f"mesh_sdf_{name}"] = {"points": n, "triangles": int(F.shape[0]), "ms": ms,
                                   "pairs_per_s": pairs / (ms * 1e-3)}
    from . import nsdf_cloth_step
    sim_n = 1024
    x = torch.from_numpy(synth.cloth_grid(sim_n)).cuda()
    xp = x.clone()
    h = 2.0 / (sim_n - 1)
    fn = lambda: nsdf_cloth_step(x, xp, sim_n, sim_n, h, h, 1e5, 9.81, 1e-3)    # noqa: E731
    for _ in range(3):
        fn()
    ms = events_ms_flushed(fn, cloth_reps, flush)
    bytes_step = 48 * sim_n * sim_n
    gbs = bytes_step / (ms * 1e-3) / 1e9
    peak = hbm_peak_gbs()
    res["cloth_step"] = {"grid": "1024x1024", "ms": ms, "bytes_per_step": bytes_step,
                         "achieved_gbs": gbs, "peak_gbs": peak,
                         "frac": gbs / peak if peak else None,
                         "peak_source": "measured hbm_gbs (copy)" if peak else None}
    return res


def bench_line_support():
    """The support workloads in one bounded pass (about a minute), for the
    benchmark line: grouped launch, penalty gradient, the fitting steps and
    the fitted-body cloth run."""
    out = {}
    for name, fn in (("grouped", lambda: bench_grouped(10)),
                     ("tiny", lambda: bench_tiny(20)),
                     ("penalty_gradient", lambda: bench_penalty(5)),
                     ("fit_width64_fp32", lambda: bench_fit_pool(10)),
                     ("fit512_bf16", lambda: bench_fit512(10)),
                     ("kernels", lambda: bench_kernels(3, 10))):
        out[name] = guarded(fn)
    t0 = time.perf_counter()
    try:
        fitted = fit_body()
    except Exception as e:     # recorded in the line; the headline stands without it
        fitted = None
        out["cloth"] = out["voxel"] = {"error": f"fitting the body: {type(e).__name__}: {e}"}
    if fitted is not None:
        for name, fn in (("cloth", bench_cloth_fitted), ("voxel", bench_voxel)):
            out[name] = guarded(lambda: fn(fitted=fitted), t0)
            t0 = time.perf_counter()
    return out


def guarded(fn, t0=None):
    """fn()'s record with its wall time, or the error it raised (so that one
    failing support workload does not take the benchmark line with it)."""
    t0 = time.perf_counter() if t0 is None else t0
    try:
        r = fn()
    except Exception as e:
        r = {"error": f"{type(e).__name__}: {e}"}
    r["wall_s"] = time.perf_counter() - t0
    return r


def bench_fit_pool(steps=10):
    """Config-1-shaped network fitted (L1 + 0.1 eikonal, FP32 backward) from a
    pool of 1,048,576 points with exact targets, batches of 250,000."""
    V, F = synth.displaced_icosphere(level=5, seed=7)
    pool = MeshFit(TINY, V, F, n_points=250_000, pool_points=1 << 20)
    pool.run(2)
    hist, per_step = pool.run(steps)
    return {"workload": "fit", "points_per_step": 250_000, "pool": 1 << 20,
            "triangles": int(F.shape[0]), "s_per_step": per_step,
            "loss_first": hist[0][0], "loss_last": hist[-1][0]}


def main(argv):
    which = argv or ["fit", "penalty", "grouped", "tiny", "grouped_paper", "cloth", "paper_arch",
                     "fit512", "fit_paper", "cloth_fitted", "voxel"]
    torch.cuda.set_device(0)
    for w in which:
        t0 = time.perf_counter()
        r = {"fit": bench_fit, "penalty": bench_penalty, "grouped": bench_grouped,
             "grouped_paper": bench_grouped_paper, "cloth": bench_cloth,
             "paper_arch": bench_paper_arch, "fit512": bench_fit512, "fit_paper": bench_fit_paper,
             "cloth_fitted": bench_cloth_fitted, "tiny": bench_tiny, "voxel": bench_voxel,
             "kernels": bench_kernels}[w]()
        r["wall_s"] = time.perf_counter() - t0
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
