"""Benchmark of the neural-SDF collision query (SDF + normal + projection).

Workload (one step): the body-scale query -- 1,048,576 points (90% on a
noisy ellipsoid shell, 10% uniform in [-1,1]^3), network 3->512x8->1 with the
input concatenated back at layer 4, softplus beta = 100, eps = 0.002 -- through
nsdf_collide: f, grad f, normal, collision test and contact-point projection
for every point (Eqs. 1-3, Sec. 3.2).  The headline form is BF16 on the
tensor cores with FP32 accumulation; the FP32 CUDA-core form is timed beside
it.  Inputs are synthetic and seeded; weights come from a seeded geometric
initialisation (the paper's meshes and trained networks are not available).

Prints one JSON line.  Single GPU only (--gpus 1).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

N_POINTS = 1 << 20
ARCH = synth.Arch(3, 512, 8, 4, 100.0)
EPS = 0.002
WORKLOAD = ("body-scale collision query: 1,048,576 points (90% noisy ellipsoid shell "
            "0.3/0.5/0.2 + N(0,0.01^2), 10% uniform [-1,1]^3), MLP 3-512x8-1 with input "
            "skip at layer 4, softplus beta=100, eps=0.002; sdf + normal + projection")
METRIC = "SDF+normal queries/s @1M pts (BF16 tensor cores, FP32 accumulate)"
# Algorithmic work per query (Eq. 1 forward + the Jacobian-transpose chain):
# forward 1,835,520 MAC + reverse 1,835,008 MAC = 3,670,528 MAC.
MAC_PER_QUERY = 3_670_528
FLOP_PER_QUERY = 2 * MAC_PER_QUERY

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the tensor-core kernel on this workload, and the share of active cycles its
# tensor pipe was busy (sm__pipe_tensor_cycles_active), from ncu captures
# keyed by the SHA-256 of the kernel's code (query_tc16.cu and its headers
# tc_ptx.cuh, softplus.cuh and f32x2.cuh, comments and blank lines removed)
# they were taken on; reported only while that code is unchanged.
TRAFFIC_CAPTURE = {
    "code_sha256": "0a3c6783a47c08d56a359cb56463f7bfbf7537df188fa8f25ad0c25e3a118f52",
    "bytes_per_launch": 4.003539e9 + 4.895270e9,
    "tensor_pipe_active_pct": 44.9,
}


def code_sha256(text):
    """SHA-256 of C++ source with // comments, trailing blanks and blank lines removed."""
    import hashlib
    import re
    lines = []
    for line in text.splitlines():
        line = re.sub(r"//.*$", "", line).rstrip()
        if line.strip():
            lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


KERNEL_SOURCES = ("query_tc16.cu", "tc_ptx.cuh", "softplus.cuh", "f32x2.cuh")


def kernel_code_sha256():
    text = []
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2110_01614_gb300", "csrc", name)) as f:
            text.append(f.read())
    return code_sha256("\n".join(text))


def captured(key):
    """A figure of the ncu captures, while the kernel's code is the captured code."""
    try:
        h = kernel_code_sha256()
    except OSError:
        return None
    return TRAFFIC_CAPTURE[key] if h == TRAFFIC_CAPTURE["code_sha256"] else None


def traffic_bytes():
    return captured("bytes_per_launch")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("bf16_tflops"), d.get("hbm_gbs"), "measured"
    return 1900.0, 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"nsdf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def single_gpu_only(args):
    """The tensor-core kernels load their weight panels with cluster TMA
    multicast; nothing here runs them on more than one GPU.  Returns the
    reason for refusing this launch, or None for a 1-GPU run."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != 1 or world != 1:
        return (f"single GPU only (--gpus {args.gpus}, WORLD_SIZE {world}): the tensor-core "
                "kernels use cluster TMA multicast on this GPU's own weight copies, so no "
                "code path runs them on 2 or more GPUs")
    return None


def oracle_rate(pts, blob, budget_s):
    """FP64 oracle on the host: queries/s over a bounded sample (test infrastructure)."""
    from oracle import mlp
    t0 = time.perf_counter()
    done = 0
    chunk = 4096
    while True:
        sl = pts[done % pts.shape[0]: done % pts.shape[0] + chunk]
        mlp.collide(blob, ARCH, sl, EPS)
        done += sl.shape[0]
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done / el, done, el


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


SINGLE_THREAD_POINTS = 4096


def single_thread_rate(budget_s):
    """The oracle on one host thread (BLAS pinned to 1 thread in a child
    process): queries/s over the first SINGLE_THREAD_POINTS points of the
    workload, repeated for about budget_s seconds."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", BLIS_NUM_THREADS="1")
    code = ("import json, bench, synth\n"
            f"pts = synth.body_scale_points({N_POINTS}, 1)[:{SINGLE_THREAD_POINTS}]\n"
            "blob = synth.geometric_init(bench.ARCH, 0)\n"
            f"r, d, s = bench.oracle_rate(pts, blob, {budget_s})\n"
            "print(json.dumps([r, d, s]))\n")
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                             text=True, timeout=120 + 4 * budget_s)
        r, d, s = json.loads(out.stdout.strip().splitlines()[-1])
        return {"value": r, "unit": "queries/s", "threads": 1,
                "sample": f"{d} queries over the first {SINGLE_THREAD_POINTS} points of the "
                          f"workload in {s:.1f} s"}
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None


def cpu_baseline(value, cores, sample, single):
    return {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample,
            "single_thread": single}


def run_reference(args):
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0      # the oracle runs on rank 0's host cores only
    pts = synth.body_scale_points(N_POINTS, 1)
    blob = synth.geometric_init(ARCH, 0)
    sample = pts[: 1 << 15]
    for _ in range(max(args.warmup, 0)):
        oracle_rate(sample, blob, 0.5)
    rates, total_pts, total_s = [], 0, 0.0
    # each step is a bounded sample so that the whole run stays near a minute
    per_step = min(args.ref_seconds, 60.0 / max(args.steps, 1))
    for _ in range(args.steps):
        r, d, s = oracle_rate(sample, blob, per_step)
        rates.append(r)
        total_pts += d
        total_s += s
    value = total_pts / total_s
    sample_txt = (f"{total_pts} points of the 1,048,576-point workload over {args.steps} steps "
                  f"of ~{per_step:.1f} s (numpy FP64, BLAS threads as reported)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * N_POINTS / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "points": N_POINTS, "precision": "fp64 oracle",
                   "timed": "each step a bounded sample of the workload; ms_per_step is "
                            "the 1,048,576-point time at the measured rate"},
        "cpu_baseline": cpu_baseline(value, blas_threads(), sample_txt,
                                     single_thread_rate(5.0)),
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# Parity sample of the bench line: this many seeded indices of the 1M points.
PARITY_POINTS = 1 << 16


def parity_sample(n):
    """Seeded distinct indices (sorted) of the points checked against the oracle."""
    k = min(PARITY_POINTS, n)
    if k == n:
        return np.arange(n, dtype=np.int64)
    u = (synth.Stream(99).u64(4 * k) % np.uint64(n)).astype(np.int64)
    _, first = np.unique(u, return_index=True)       # distinct draws, in draw order
    return np.sort(u[np.sort(first)][:k])


def error_stats(ref, out_ns_sample, hit_sample):
    """Errors of one form against the oracle's (f, N) on the parity sample."""
    f, N = ref
    ds = np.abs(out_ns_sample[:, 3].astype(np.float64) - f)
    a, b = N, out_ns_sample[:, :3].astype(np.float64)
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.einsum("ij,ij->i", a, b))
    sel = np.abs(f) > 1e-2
    agree = float(np.mean((f[sel] < EPS) == hit_sample[sel]))
    return {"points": int(len(f)), "sdf_abs_max": float(ds.max()),
            "sdf_abs_p99": float(np.percentile(ds, 99)), "angle_rad_max": float(ang.max()),
            "angle_rad_p99": float(np.percentile(ang, 99)),
            "decision_agreement_abs_sdf_gt_1e-2": agree}


def run_gpu(args):
    refusal = single_gpu_only(args)
    if refusal:
        print(json.dumps({"metric": METRIC, "error": refusal}), flush=True)
        return 2
    import torch
    import paper_2110_01614_gb300 as nsdf
    from paper_2110_01614_gb300 import build as nbuild

    nbuild.ensure_built()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = args.points
    pts_h = synth.body_scale_points(n, 1)
    blob = synth.geometric_init(ARCH, 0)
    pts = torch.from_numpy(pts_h).to(dev)
    out_pts = torch.empty_like(pts)
    out_ns = torch.empty_like(pts)
    out_hit = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def timed_steps(sdf, k, warm):
        for _ in range(warm):
            sdf.collide(pts, EPS, out_pts=out_pts, out_n_sdf=out_ns, out_hit=out_hit)
        torch.cuda.synchronize()
        durs = []
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        for i in range(k):
            flush.fill_(i & 0xFF)                        # evict inputs and weights from L2
            evs[i][0].record(stream)
            sdf.collide(pts, EPS, out_pts=out_pts, out_n_sdf=out_ns, out_hit=out_hit)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        for a, b in evs:
            durs.append(a.elapsed_time(b) / 1e3)
        nsdf.nsdf_sync_status(sdf.ctx)
        return durs

    forms = args.forms.split(",")
    bf = nsdf.NeuralSDF(ARCH, nsdf.NSDF_BF16).load(blob)

    # --- headline: BF16, inputs resident in HBM, one kernel per step ---
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    durs = timed_steps(bf, args.steps, max(args.warmup, 3))
    clk = clocks.stop()
    t_total = sum(durs)
    value = n * args.steps / t_total
    kernel_s = statistics.mean(durs)
    sample_idx = parity_sample(n)
    bf_ns, bf_hit = out_ns.cpu().numpy(), out_hit.cpu().numpy().astype(bool)

    # --- the other forms on the same workload: FP16 tensor cores, FP32 CUDA cores ---
    other = {}
    for name, prec, k in (("fp16", nsdf.NSDF_FP16, args.steps), ("fp32", nsdf.NSDF_FP32, 3)):
        if name not in forms:
            continue
        ctx = nsdf.NeuralSDF(ARCH, prec).load(blob)
        d = timed_steps(ctx, max(2, min(args.steps, k)), 1)
        other[name] = {"value": n / statistics.mean(d), "unit": "queries/s",
                       "ms_per_step": 1e3 * statistics.mean(d),
                       "ns": out_ns.cpu().numpy(), "hit": out_hit.cpu().numpy().astype(bool)}
        if name == "fp32":
            # the FP32 form against the measured FP32 FMA throughput of this GPU
            fma = nsdf.nsdf_debug_fp32_fma_peak()
            tf = FLOP_PER_QUERY * n / statistics.mean(d) / 1e12
            other[name]["roofline"] = {"bound": "fp32 fma", "achieved": tf, "peak": fma,
                                       "unit": "TFLOP/s", "frac": tf / fma,
                                       "peak_source": "measured (nsdf_debug_fp32_fma_peak)"}
        ctx.close()

    # --- the paper's own network shapes (Sec. 4.3) on the same points, BF16 tensor cores ---
    paper = {}
    if "paper" in forms:
        for name, L in (("dragon_8x256", 8), ("bunny_4x256", 4)):
            arch = synth.Arch(3, 256, L, -1, 100.0, "relu", 128)
            ctx = nsdf.NeuralSDF(arch, nsdf.NSDF_BF16).load(synth.fourier_relu_init(arch, 0))
            d = timed_steps(ctx, max(2, min(args.steps, 5)), 1)
            ctx.close()
            t = statistics.mean(d)
            flop = 2 * (2 * L * 256 * 256 + 256) * n
            paper[name] = {"value": n / t, "unit": "queries/s", "ms_per_step": 1e3 * t,
                           "tflops": flop / t / 1e12, "kernel": "query_tc16_ff_kernel<bf16>"}

    # --- end to end through the C ABI with host (pinned) buffers ---
    e2e_value = None
    if not args.no_e2e:
        h_pts = torch.from_numpy(pts_h).pin_memory()
        h_out = torch.empty_like(h_pts).pin_memory()
        h_ns = torch.empty_like(h_pts).pin_memory()
        h_hit = torch.empty(n, dtype=torch.uint8).pin_memory()
        for _ in range(2):
            nsdf.nsdf_collide(bf.ctx, h_pts, EPS, h_out, h_ns, h_hit)
        e2e_t = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            nsdf.nsdf_collide(bf.ctx, h_pts, EPS, h_out, h_ns, h_hit)   # results on host on return
            e2e_t.append(time.perf_counter() - t0)
        e2e_value = n * args.steps / sum(e2e_t)

    support = None
    if args.support:
        from paper_2110_01614_gb300 import support_bench
        support = support_bench.bench_line_support()

    peak_tf, hbm, peak_kind = load_peaks()
    achieved_tf = FLOP_PER_QUERY * n / kernel_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded points, geometric-init weights)",
        "config": {"workload": WORKLOAD, "points": n, "precision": "bf16 x bf16 -> fp32",
                   "l2": "flushed between timed steps (256 MiB write outside the events)",
                   "parallelism": "1 GPU (single-GPU library; no multi-GPU path)"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                     "peak_source": f"{peak_kind} bf16_tflops (burst, cuBLAS)",
                     "traffic": traffic_bytes() if n == N_POINTS else None,
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                     "tensor_pipe_active_pct": (captured("tensor_pipe_active_pct")
                                                if n == N_POINTS else None),
                     "kernel": "query_tc16_kernel<bf16>",
                     "algorithmic_flop_per_launch": FLOP_PER_QUERY * n,
                     "algorithmic_io_bytes_per_launch": 49 * n},
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * (16 + 16 + 1)},
        "forms": {name: {"value": o["value"], "unit": "queries/s", "ms_per_step": o["ms_per_step"],
                         "bf16_speedup_over_this": value / o["value"],
                         **({"roofline": o["roofline"]} if "roofline" in o else {})}
                  for name, o in other.items()},
        "clocks": clk,
    }
    if paper:
        peak_note = f"{peak_kind} bf16_tflops"
        for o in paper.values():
            o["frac_of_peak"] = o["tflops"] / peak_tf
        line["paper_networks"] = {"workload": "the paper's Fourier-feature ReLU shapes (128 "
                                              "frequencies, 8 or 4 layers of 256), same points",
                                  "peak": peak_note, **paper}
    if support is not None:
        line["support"] = support
    from oracle import mlp
    f_ref, N_ref, _, _ = mlp.collide(blob, ARCH, pts_h[sample_idx], EPS)
    ref = (f_ref, N_ref)
    errs = {"bf16": error_stats(ref, bf_ns[sample_idx], bf_hit[sample_idx])}
    for name, o in other.items():
        errs[name] = error_stats(ref, o["ns"][sample_idx], o["hit"][sample_idx])
    line["error_vs_oracle"] = errs
    if not args.no_cpu_baseline:
        r, d, s = oracle_rate(pts_h[: 1 << 15], blob, args.ref_seconds)
        line["cpu_baseline"] = cpu_baseline(
            r, blas_threads(), f"{d} points of the same workload in {s:.1f} s (numpy FP64)",
            single_thread_rate(5.0))
    print(json.dumps(line), flush=True)
    bf.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nsdf", choices=["nsdf", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # profiling conveniences (the defaults are the benchmark)
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--forms", default="bf16,fp16,fp32,paper")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--support", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the support workloads (grouped, fitting, cloth)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
