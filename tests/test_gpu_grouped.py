"""Grouped launch (many bodies' networks in one persistent kernel), its CUDA-graph
replay with changed counts, and the autotuner.

Reference: the single-network nsdf_collide path (same FP32 arithmetic, so the
results must be bitwise equal) and the FP64 oracle on a sample.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import mlp

pytestmark = pytest.mark.gpu

TINY = synth.Arch(3, 64, 3, -1, 100.0)
EPS = 0.002


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def make_problem(counts, seed=5):
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    total = int(np.sum(counts))
    pts = synth.body_scale_points(max(total, 1), seed)[:total]
    return offs, total, pts


def grouped_setup(nsdf, n_nets=16):
    net = nsdf.NeuralSDF(TINY, nsdf.NSDF_FP32, n_nets=n_nets)
    blobs = [synth.geometric_init(TINY, k) for k in range(n_nets)]
    for k, b in enumerate(blobs):
        net.load(b, net=k)
    return net, blobs


def per_net_reference(nsdf, blobs, offs, counts, pts):
    out = np.empty_like(pts)
    ns = np.empty_like(pts)
    for k, b in enumerate(blobs):
        if counts[k] == 0:
            continue
        s = nsdf.NeuralSDF(TINY, nsdf.NSDF_FP32).load(b)
        d = torch.from_numpy(pts[offs[k]: offs[k] + counts[k]].copy()).cuda()
        o, n_ = torch.empty_like(d), torch.empty_like(d)
        s.collide(d, EPS, out_pts=o, out_n_sdf=n_)
        torch.cuda.synchronize()
        out[offs[k]: offs[k] + counts[k]] = o.cpu().numpy()
        ns[offs[k]: offs[k] + counts[k]] = n_.cpu().numpy()
        s.close()
    return out, ns


def run_grouped(nsdf, net, pts, offs, counts, max_total):
    P = torch.from_numpy(pts).cuda()
    O = torch.from_numpy(offs).cuda()
    C = torch.from_numpy(np.asarray(counts, dtype=np.int64)).cuda()
    out = torch.full_like(P, -7.0)
    ns = torch.full_like(P, -7.0)
    nsdf.nsdf_query_grouped(net.ctx, P, O, C, max_total, EPS, out, ns)
    nsdf.nsdf_sync_status(net.ctx)
    return out.cpu().numpy(), ns.cpu().numpy()


def test_grouped_equals_per_network_and_oracle(nsdf):
    counts = (synth.grouped_counts() // 40).astype(np.int64)      # ~30k points, same spread
    counts[3] = 0                                                 # an empty network
    offs, total, pts = make_problem(counts)
    net, blobs = grouped_setup(nsdf)
    out, ns = run_grouped(nsdf, net, pts, offs, counts, total)
    ref_out, ref_ns = per_net_reference(nsdf, blobs, offs, counts, pts)
    np.testing.assert_array_equal(out, ref_out)
    np.testing.assert_array_equal(ns, ref_ns)
    # oracle on a sample of every network
    for k in (0, 5, 15):
        if counts[k] == 0:
            continue
        sl = slice(offs[k], offs[k] + min(counts[k], 300))
        f, N, hit, x = mlp.collide(blobs[k], TINY, pts[sl], EPS)
        assert np.abs(ns[sl, 3] - f).max() <= 1e-5
    net.close()


def test_grouped_tile_shapes_agree(nsdf):
    counts = np.array([1, 63, 64, 65, 1000, 4097], dtype=np.int64)
    offs, total, pts = make_problem(counts, seed=8)
    net, blobs = grouped_setup(nsdf, n_nets=6)
    outs = []
    for pt, cps in ((8, 0), (4, 0), (4, 1), (8, 2)):
        nsdf.nsdf_set_grouped_config(net.ctx, pt, cps)
        outs.append(run_grouped(nsdf, net, pts, offs, counts, total))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
    net.close()


def test_cuda_graph_replay_with_new_counts(nsdf):
    counts0 = np.array([5000, 3000, 11000, 700], dtype=np.int64)
    counts1 = np.array([100, 9000, 0, 8000], dtype=np.int64)
    max_total = 20000
    pts = synth.body_scale_points(max_total, 9)
    net, blobs = grouped_setup(nsdf, n_nets=4)
    P = torch.from_numpy(pts).cuda()
    O = torch.tensor([0, 5000, 8000, 19000], dtype=torch.int64, device="cuda")
    O1 = torch.tensor([0, 100, 9100, 12000], dtype=torch.int64, device="cuda")
    C = torch.from_numpy(counts0).cuda()
    out = torch.zeros_like(P)
    ns = torch.zeros_like(P)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nsdf.nsdf_query_grouped(net.ctx, P, O, C, max_total, EPS, out, ns)   # warm-up (scratch)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nsdf.nsdf_query_grouped(net.ctx, P, O, C, max_total, EPS, out, ns)
    O0 = O.clone()
    for offs_t, counts in ((O0, counts0), (O1, counts1)):
        O.copy_(offs_t)
        C.copy_(torch.from_numpy(counts))
        out.zero_()
        ns.zero_()
        g.replay()
        torch.cuda.synchronize()
        offs = O.cpu().numpy()
        ref_out, ref_ns = per_net_reference(nsdf, blobs, offs, counts, pts)
        got_out, got_ns = out.cpu().numpy(), ns.cpu().numpy()
        for k in range(4):
            sl = slice(offs[k], offs[k] + counts[k])
            np.testing.assert_array_equal(got_out[sl], ref_out[sl])
            np.testing.assert_array_equal(got_ns[sl], ref_ns[sl])
    nsdf.nsdf_sync_status(net.ctx)
    net.close()


def test_autotuner_picks_a_valid_shape_and_caches_it(nsdf, tmp_path):
    from paper_2110_01614_gb300 import tune
    counts = (synth.grouped_counts() // 20).astype(np.int64)
    offs, total, pts = make_problem(counts, seed=10)
    net, blobs = grouped_setup(nsdf)
    P = torch.from_numpy(pts).cuda()
    O = torch.from_numpy(offs).cuda()
    C = torch.from_numpy(counts).cuda()
    out, ns = torch.empty_like(P), torch.empty_like(P)
    cache = str(tmp_path / "tune.json")
    pt, cps = tune.tuned_grouped(net, P, O, C, total, EPS, out, ns, path=cache)
    assert pt in (4, 8) and cps >= 1
    assert tune.tuned_grouped(net, P, O, C, total, EPS, out, ns, path=cache) == (pt, cps)
    got_out, got_ns = run_grouped(nsdf, net, pts, offs, counts, total)
    ref_out, ref_ns = per_net_reference(nsdf, blobs, offs, counts, pts)
    np.testing.assert_array_equal(got_ns, ref_ns)
    net.close()


def test_bad_work_entry_is_reported_not_executed(nsdf):
    counts = np.array([10, 20], dtype=np.int64)
    net, blobs = grouped_setup(nsdf, n_nets=2)
    P = torch.zeros(30, 4, device="cuda")
    O = torch.tensor([0, 25], dtype=torch.int64, device="cuda")      # 25 + 20 > 30
    C = torch.from_numpy(counts).cuda()
    out = torch.full_like(P, 3.0)
    nsdf.nsdf_query_grouped(net.ctx, P, O, C, 30, EPS, out, None)
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_sync_status(net.ctx)
    assert e.value.status == 1
    assert float(out[25:].min()) == 3.0 and float(out[10:25].min()) == 3.0   # untouched
    net.close()


def posed_reference(blobs, offs, counts, pts, T):
    """FP64 oracle per body with its pose."""
    f = np.empty(len(pts))
    N = np.empty((len(pts), 3))
    x = np.empty((len(pts), 3))
    for k, b in enumerate(blobs):
        sl = slice(offs[k], offs[k] + counts[k])
        if counts[k] == 0:
            continue
        f[sl], N[sl], _, x[sl] = mlp.collide(b, TINY, pts[sl], EPS, T=T[k])
    return f, N, x


def test_posed_scene_matches_oracle_and_single_body_path(nsdf):
    from parity import normal_angle
    counts = np.array([700, 0, 1500, 64, 2500, 333, 1, 900], dtype=np.int64)
    offs, total, pts = make_problem(counts, seed=21)
    net, blobs = grouped_setup(nsdf, n_nets=8)
    T = synth.rigid_transforms(8, seed=5)
    P = torch.from_numpy(pts).cuda()
    out = torch.full_like(P, -7.0)
    ns = torch.full_like(P, -7.0)
    nsdf.nsdf_query_grouped_T(net.ctx, P, torch.from_numpy(offs).cuda(),
                              torch.from_numpy(counts).cuda(), total, EPS,
                              torch.from_numpy(T).cuda(), out, ns)
    nsdf.nsdf_sync_status(net.ctx)
    out, ns = out.cpu().numpy(), ns.cpu().numpy()
    f, N, x = posed_reference(blobs, offs, counts, pts, T)
    assert np.abs(ns[:, 3] - f).max() <= 1e-5
    ok = np.linalg.norm(N, axis=1) > 0
    assert normal_angle(N[ok], ns[ok, :3]).max() <= 1e-4
    np.testing.assert_allclose(out[:, :3], x, atol=2e-5)
    np.testing.assert_array_equal(out[:, 3], pts[:, 3])          # w rides along
    # the single-body path with the same pose (its inverse is taken on the host)
    for k in (0, 4):
        s = nsdf.NeuralSDF(TINY, nsdf.NSDF_FP32).load(blobs[k])
        d = torch.from_numpy(pts[offs[k]: offs[k] + counts[k]].copy()).cuda()
        o, n_ = torch.empty_like(d), torch.empty_like(d)
        s.collide(d, EPS, T=T[k], out_pts=o, out_n_sdf=n_)
        torch.cuda.synchronize()
        np.testing.assert_allclose(ns[offs[k]: offs[k] + counts[k]], n_.cpu().numpy(), atol=1e-6)
        s.close()
    net.close()


def test_posed_scene_graph_replays_with_new_poses(nsdf):
    counts = np.array([3000, 2000, 4000], dtype=np.int64)
    offs, total, pts = make_problem(counts, seed=22)
    net, blobs = grouped_setup(nsdf, n_nets=3)
    P = torch.from_numpy(pts).cuda()
    O, C = torch.from_numpy(offs).cuda(), torch.from_numpy(counts).cuda()
    Tdev = torch.from_numpy(synth.rigid_transforms(3, seed=6)).cuda()
    out, ns = torch.zeros_like(P), torch.zeros_like(P)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        nsdf.nsdf_query_grouped_T(net.ctx, P, O, C, total, EPS, Tdev, out, ns)   # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        nsdf.nsdf_query_grouped_T(net.ctx, P, O, C, total, EPS, Tdev, out, ns)
    for seed in (7, 8):
        T = synth.rigid_transforms(3, seed=seed)
        Tdev.copy_(torch.from_numpy(T))
        ns.zero_()
        g.replay()
        torch.cuda.synchronize()
        f, N, x = posed_reference(blobs, offs, counts, pts, T)
        assert np.abs(ns.cpu().numpy()[:, 3] - f).max() <= 1e-5
    nsdf.nsdf_sync_status(net.ctx)
    net.close()


def test_posed_scene_rejects_missing_and_singular_poses(nsdf):
    counts = np.array([100, 50], dtype=np.int64)
    offs, total, pts = make_problem(counts, seed=23)
    net, blobs = grouped_setup(nsdf, n_nets=2)
    P = torch.from_numpy(pts).cuda()
    O, C = torch.from_numpy(offs).cuda(), torch.from_numpy(counts).cuda()
    out = torch.empty_like(P)
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_query_grouped_T(net.ctx, P, O, C, total, EPS, None, out)
    assert e.value.status == 1
    T = synth.rigid_transforms(2, seed=9)
    T[1, :3, :3] = 0.0                                     # singular pose of body 1
    nsdf.nsdf_query_grouped_T(net.ctx, P, O, C, total, EPS, torch.from_numpy(T).cuda(), out)
    with pytest.raises(nsdf.NsdfError) as e:
        nsdf.nsdf_sync_status(net.ctx)
    assert e.value.status == 1
    # body 0 is still answered with its own pose
    f, N, hit, x = mlp.collide(blobs[0], TINY, pts[:100], EPS, T=T[0])
    np.testing.assert_allclose(out.cpu().numpy()[:100, :3], x, atol=2e-5)
    net.close()
