"""GPU parity of the 16-bit tensor-core kernel for width-64 softplus networks
(query_tc16_w64.cu): the tiny network 3-64-64-64-1 and the grouped
multi-body launch built from it, against the FP64 oracle.

Tolerances: the stated targets (|delta sdf| <= 2e-3, normal angle <= 1e-2 rad,
>= 99.9% collision-decision agreement where |f| > 1e-2) for both forms.  The
BF16 form takes split operands (hi + lo) in its forward products, so its f
is held to 1e-4 as well: one BF16 rounding of the 64-wide weights alone moves
f by up to ~2.8e-3 on these networks (FP64 emulation of the roundings), and a
regression to single operands would fail here.  Grouped launches compute each
point exactly as a single-network launch does, so they are compared bit for
bit with one launch per body.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp
from parity import decision_agreement, normal_angle, report

pytestmark = pytest.mark.gpu

TINY = synth.Arch(3, 64, 3, -1, 100.0)
EPS = 0.002
ANG_TOL, AGREE = 1e-2, 0.999
SDF_TOL = {"bf16": 1e-4, "fp16": 2e-3}


@pytest.fixture(scope="module", params=["bf16", "fp16"])
def prec(request):
    return request.param


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def P(nsdf, prec):
    return nsdf.NSDF_FP16 if prec == "fp16" else nsdf.NSDF_BF16


def collide_gpu(nsdf, prec, arch, blob, pts, T=None):
    s = nsdf.NeuralSDF(arch, P(nsdf, prec)).load(blob)
    d = torch.from_numpy(pts).cuda()
    out_pts, out_ns = torch.full_like(d, -7.0), torch.full_like(d, -7.0)
    out_hit = torch.full((pts.shape[0],), 9, dtype=torch.uint8, device="cuda")
    s.collide(d, EPS, T=T, out_pts=out_pts, out_n_sdf=out_ns, out_hit=out_hit)
    nsdf.nsdf_sync_status(s.ctx)
    s.close()
    return out_pts.cpu().numpy(), out_ns.cpu().numpy(), out_hit.cpu().numpy()


def check(prec, arch, blob, pts, out_pts, out_ns, out_hit, T=None):
    f, N, hit, x = mlp.collide(blob, arch, pts, EPS, T)
    rep = report(f, N, out_ns[:, 3], out_ns[:, :3])
    print(prec, arch.n_hidden, "vs oracle:", rep)
    assert rep["sdf_max"] <= SDF_TOL[prec]
    ok = np.linalg.norm(N, axis=1) > 0
    assert normal_angle(N[ok], out_ns[ok, :3]).max() <= ANG_TOL
    assert decision_agreement(f, out_hit.astype(bool), EPS, 1e-2) >= AGREE
    np.testing.assert_array_equal(out_hit.astype(bool), out_ns[:, 3] < EPS)
    exp = pts[:, :3].astype(np.float64).copy()
    m = out_hit.astype(bool)
    exp[m] += (EPS - out_ns[m, 3:4].astype(np.float64)) * out_ns[m, :3]
    np.testing.assert_allclose(out_pts[:, :3], exp, atol=2e-6)
    np.testing.assert_array_equal(out_pts[:, 3], pts[:, 3])


@pytest.mark.parametrize("n", [1, 127, 128, 129, 255, 256, 257, 4096, 4096 + 17, 40000])
def test_tiny_network_collide(nsdf, prec, n):
    blob = synth.geometric_init(TINY, 0)
    pts = synth.uniform_cube_points(n, 1)
    pts[:, 3] = 5.0
    out_pts, out_ns, out_hit = collide_gpu(nsdf, prec, TINY, blob, pts)
    check(prec, TINY, blob, pts, out_pts, out_ns, out_hit)


@pytest.mark.parametrize("L", [2, 4, 7])
def test_other_depths(nsdf, prec, L):
    arch = synth.Arch(3, 64, L, -1, 100.0)
    blob = synth.geometric_init(arch, 3)
    pts = synth.body_scale_points(3000, 9)
    out_pts, out_ns, out_hit = collide_gpu(nsdf, prec, arch, blob, pts)
    check(prec, arch, blob, pts, out_pts, out_ns, out_hit)


def test_transform_and_raw_gradient(nsdf, prec):
    from test_gpu_query_fp32 import rigid
    blob = synth.geometric_init(TINY, 2)
    pts = synth.body_scale_points(2500, 5)
    T = rigid(3)
    out_pts, out_ns, out_hit = collide_gpu(nsdf, prec, TINY, blob, pts, T)
    check(prec, TINY, blob, pts, out_pts, out_ns, out_hit, T)
    s = nsdf.NeuralSDF(TINY, P(nsdf, prec)).load(blob)
    d = torch.from_numpy(pts).cuda()
    raw = s.query(d, raw_gradient=True).cpu().numpy()
    s.close()
    f, g = mlp.query(blob, TINY, pts, raw_gradient=True)
    assert np.abs(raw[:, 3] - f).max() <= SDF_TOL[prec]
    assert normal_angle(g, raw[:, :3]).max() <= ANG_TOL
    np.testing.assert_allclose(np.linalg.norm(raw[:, :3], axis=1), np.linalg.norm(g, axis=1),
                               rtol=2e-2)


def test_host_buffers_match_device_buffers(nsdf, prec):
    blob = synth.geometric_init(TINY, 0)
    pts = torch.from_numpy(synth.body_scale_points(300000, 3)).pin_memory()
    s = nsdf.NeuralSDF(TINY, P(nsdf, prec)).load(blob)
    h_out, h_ns = torch.empty_like(pts).pin_memory(), torch.empty_like(pts).pin_memory()
    nsdf.nsdf_collide(s.ctx, pts, EPS, h_out, h_ns, None)
    d = pts.cuda()
    d_out, d_ns = torch.empty_like(d), torch.empty_like(d)
    nsdf.nsdf_collide(s.ctx, d, EPS, d_out, d_ns, None)
    torch.cuda.synchronize()
    s.close()
    assert torch.equal(h_out, d_out.cpu()) and torch.equal(h_ns, d_ns.cpu())


# ---------------------------------------------------------------- grouped launches

def make_problem(counts, seed=5):
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    total = int(np.sum(counts))
    return offs, total, synth.body_scale_points(max(total, 1), seed)[:total]


def grouped_net(nsdf, prec, n_nets):
    net = nsdf.NeuralSDF(TINY, P(nsdf, prec), n_nets=n_nets)
    blobs = [synth.geometric_init(TINY, k) for k in range(n_nets)]
    for k, b in enumerate(blobs):
        net.load(b, net=k)
    return net, blobs


def single_launch_reference(nsdf, prec, blobs, offs, counts, pts, T=None):
    out, ns = np.full_like(pts, -7.0), np.full_like(pts, -7.0)
    for k, b in enumerate(blobs):
        if counts[k] == 0:
            continue
        sl = slice(offs[k], offs[k] + counts[k])
        o, n_, _ = collide_gpu(nsdf, prec, TINY, b, pts[sl].copy(), None if T is None else T[k])
        out[sl], ns[sl] = o, n_
    return out, ns


def run_grouped(nsdf, net, pts, offs, counts, total, T=None):
    Pd = torch.from_numpy(pts).cuda()
    O = torch.from_numpy(offs).cuda()
    C = torch.from_numpy(np.asarray(counts, dtype=np.int64)).cuda()
    out, ns = torch.full_like(Pd, -7.0), torch.full_like(Pd, -7.0)
    if T is None:
        nsdf.nsdf_query_grouped(net.ctx, Pd, O, C, total, EPS, out, ns)
    else:
        nsdf.nsdf_query_grouped_T(net.ctx, Pd, O, C, total, EPS, torch.from_numpy(T).cuda(), out, ns)
    nsdf.nsdf_sync_status(net.ctx)
    return out.cpu().numpy(), ns.cpu().numpy()


def test_grouped_equals_single_launches_and_oracle(nsdf, prec):
    counts = (synth.grouped_counts() // 40).astype(np.int64)      # ~30k points, same spread
    counts[3] = 0                                                 # an empty network
    counts[7] = 1                                                 # a one-point network
    offs, total, pts = make_problem(counts)
    net, blobs = grouped_net(nsdf, prec, 16)
    out, ns = run_grouped(nsdf, net, pts, offs, counts, total)
    ref_out, ref_ns = single_launch_reference(nsdf, prec, blobs, offs, counts, pts)
    np.testing.assert_array_equal(out, ref_out)
    np.testing.assert_array_equal(ns, ref_ns)
    for k in range(16):
        if counts[k] == 0:
            continue
        sl = slice(offs[k], offs[k] + counts[k])
        f, N, hit, x = mlp.collide(blobs[k], TINY, pts[sl], EPS)
        assert np.abs(ns[sl, 3] - f).max() <= SDF_TOL[prec]
        ok = np.linalg.norm(N, axis=1) > 0
        assert normal_angle(N[ok], ns[sl][ok, :3]).max() <= ANG_TOL
    net.close()


def test_grouped_posed_scene(nsdf, prec):
    counts = np.array([700, 0, 1500, 64, 2500, 333, 1, 900], dtype=np.int64)
    offs, total, pts = make_problem(counts, seed=21)
    net, blobs = grouped_net(nsdf, prec, 8)
    T = synth.rigid_transforms(8, seed=5)
    out, ns = run_grouped(nsdf, net, pts, offs, counts, total, T)
    for k in range(8):
        if counts[k] == 0:
            continue
        sl = slice(offs[k], offs[k] + counts[k])
        f, N, hit, x = mlp.collide(blobs[k], TINY, pts[sl], EPS, T=T[k])
        assert np.abs(ns[sl, 3] - f).max() <= SDF_TOL[prec]
        ok = np.linalg.norm(N, axis=1) > 0
        assert normal_angle(N[ok], ns[sl][ok, :3]).max() <= ANG_TOL
        # Eq. 3 from the kernel's own f and (world-frame) normal
        m = ns[sl, 3] < EPS
        exp = pts[sl, :3].astype(np.float64).copy()
        exp[m] += (EPS - ns[sl][m, 3:4].astype(np.float64)) * ns[sl][m, :3]
        np.testing.assert_allclose(out[sl, :3], exp, atol=2e-6)
    net.close()


def test_grouped_graph_replay_with_new_counts(nsdf, prec):
    counts0 = np.array([5000, 3000, 11000, 700], dtype=np.int64)
    counts1 = np.array([100, 9000, 0, 8000], dtype=np.int64)
    max_total = 20000
    pts = synth.body_scale_points(max_total, 9)
    net, blobs = grouped_net(nsdf, prec, 4)
    Pd = torch.from_numpy(pts).cuda()
    O = torch.tensor([0, 5000, 8000, 19000], dtype=torch.int64, device="cuda")
    O1 = torch.tensor([0, 100, 9100, 12000], dtype=torch.int64, device="cuda")
    C = torch.from_numpy(counts0).cuda()
    out, ns = torch.zeros_like(Pd), torch.zeros_like(Pd)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nsdf.nsdf_query_grouped(net.ctx, Pd, O, C, max_total, EPS, out, ns)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nsdf.nsdf_query_grouped(net.ctx, Pd, O, C, max_total, EPS, out, ns)
    O0 = O.clone()
    for offs_t, counts in ((O0, counts0), (O1, counts1)):
        O.copy_(offs_t)
        C.copy_(torch.from_numpy(counts))
        out.zero_()
        ns.zero_()
        g.replay()
        torch.cuda.synchronize()
        offs = O.cpu().numpy()
        ref_out, ref_ns = single_launch_reference(nsdf, prec, blobs, offs, counts, pts)
        got_out, got_ns = out.cpu().numpy(), ns.cpu().numpy()
        for k in range(4):
            sl = slice(offs[k], offs[k] + counts[k])
            np.testing.assert_array_equal(got_out[sl], ref_out[sl])
            np.testing.assert_array_equal(got_ns[sl], ref_ns[sl])
    nsdf.nsdf_sync_status(net.ctx)
    net.close()


def test_grouped_autotuner_and_occupancies_agree(nsdf, prec, tmp_path):
    from paper_2110_01614_gb300 import tune
    counts = (synth.grouped_counts() // 20).astype(np.int64)
    offs, total, pts = make_problem(counts, seed=10)
    net, blobs = grouped_net(nsdf, prec, 16)
    Pd = torch.from_numpy(pts).cuda()
    O, C = torch.from_numpy(offs).cuda(), torch.from_numpy(counts).cuda()
    out, ns = torch.empty_like(Pd), torch.empty_like(Pd)
    cache = str(tmp_path / "tune.json")
    pt, cps = tune.tuned_grouped(net, Pd, O, C, total, EPS, out, ns, path=cache)
    assert pt == 0 and cps >= 1
    assert tune.tuned_grouped(net, Pd, O, C, total, EPS, out, ns, path=cache) == (pt, cps)
    outs = []
    for c in (1, 2, 0):
        nsdf.nsdf_set_grouped_config(net.ctx, 0, c)
        outs.append(run_grouped(nsdf, net, pts, offs, counts, total))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
    net.close()


def test_full_size_grouped_workload(nsdf, prec):
    """16 bodies with log-uniform counts in [2k, 400k] (616,218 points): the
    oracle on 2,048 points of every body; properties at every point."""
    counts = synth.grouped_counts().astype(np.int64)
    offs, total, pts = make_problem(counts)
    net, blobs = grouped_net(nsdf, prec, 16)
    out, ns = run_grouped(nsdf, net, pts, offs, counts, total)
    for k in range(16):
        sel = offs[k] + (synth.Stream(40 + k).u64(2048) % np.uint64(counts[k])).astype(np.int64)
        f, N, hit, x = mlp.collide(blobs[k], TINY, pts[sel], EPS)
        assert np.abs(ns[sel, 3] - f).max() <= SDF_TOL[prec]
        ok = np.linalg.norm(N, axis=1) > 0
        assert normal_angle(N[ok], ns[sel][ok, :3]).max() <= ANG_TOL
    assert np.isfinite(ns).all() and np.isfinite(out).all()
    assert np.all(np.abs(np.linalg.norm(ns[:, :3], axis=1) - 1.0) < 1e-5)
    net.close()


def test_bounded_wait_reports_timeout_and_recovers(nsdf, prec):
    """A dropped MMA commit makes the warpgroup's wait run out: the kernel
    must return, the context must report NSDF_ERR_TIMEOUT, and the next call
    must be correct."""
    blob = synth.geometric_init(TINY, 0)
    pts = synth.uniform_cube_points(1000, 2)
    s = nsdf.NeuralSDF(TINY, P(nsdf, prec)).load(blob)
    d = torch.from_numpy(pts).cuda()
    nsdf.nsdf_debug_inject(s.ctx, 0, 20_000_000)
    s.collide(d, EPS)
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_sync_status(s.ctx)
    assert e.value.status == 7
    nsdf.nsdf_debug_inject(s.ctx, -1, 4_000_000_000)
    out_ns = torch.empty_like(d)
    s.collide(d, EPS, out_n_sdf=out_ns)
    nsdf.nsdf_sync_status(s.ctx)
    s.close()
    f, N, _, _ = mlp.collide(blob, TINY, pts, EPS)
    assert np.abs(out_ns.cpu().numpy()[:, 3] - f).max() <= SDF_TOL[prec]
