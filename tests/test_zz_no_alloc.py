"""The allocation-free entry point nsdf_collide_noalloc.

For callers that cannot allocate device memory when they query (fixed-budget
simulators, CUDA-graph recording, real-time callbacks): it must give the same
results as nsdf_collide, call after call, while taking its scratch from the
library's fixed device array.  Collected last on purpose (file name), so a
run stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

EPS = 0.002


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


@pytest.mark.parametrize("prec,arch,n", [
    ("bf16", synth.Arch(3, 512, 8, 4, 100.0), 100_003),
    ("fp32", synth.Arch(3, 64, 3, -1, 100.0), 200_001),
    ("bf16", synth.Arch(3, 64, 3, -1, 100.0), 150_001),
])
def test_noalloc_matches_collide_twice(nsdf, prec, arch, n):
    precision = nsdf.NSDF_BF16 if prec == "bf16" else nsdf.NSDF_FP32
    net = nsdf.NeuralSDF(arch, precision).load(synth.geometric_init(arch, 0))
    pts = torch.from_numpy(synth.body_scale_points(n, 11)).cuda()
    ref_pts, ref_ns = torch.empty_like(pts), torch.empty_like(pts)
    ref_hit = torch.empty(n, dtype=torch.uint8, device="cuda")
    nsdf.nsdf_collide(net.ctx, pts, EPS, ref_pts, ref_ns, ref_hit)
    torch.cuda.synchronize()
    for _ in range(2):                      # two calls in a row share the fixed scratch
        out_pts, out_ns = torch.empty_like(pts), torch.empty_like(pts)
        out_hit = torch.empty(n, dtype=torch.uint8, device="cuda")
        nsdf.nsdf_collide_noalloc(net.ctx, pts, EPS, out_pts, out_ns, out_hit)
        nsdf.nsdf_sync_status(net.ctx)
        # each point's result does not depend on the CTA that computed it
        assert torch.equal(out_ns, ref_ns)
        assert torch.equal(out_pts, ref_pts)
        assert torch.equal(out_hit, ref_hit)
    net.close()


def test_noalloc_deepest_network_and_bad_args(nsdf):
    """The deepest network the library accepts (512 wide, 63 hidden layers:
    7.75 MiB of slopes per CTA) still fits the fixed array (4 CTAs) and
    matches nsdf_collide; misuse is reported, not executed."""
    arch = synth.Arch(3, 512, 63, -1, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_BF16)
    pts = torch.from_numpy(synth.body_scale_points(1000, 12)).cuda()
    out = torch.empty_like(pts)
    with pytest.raises(nsdf.NsdfError) as e:    # weights not loaded
        nsdf.nsdf_collide_noalloc(net.ctx, pts, EPS, out)
    assert e.value.status == 3
    net.load(synth.geometric_init(arch, 0))
    ref_ns, got_ns = torch.empty_like(pts), torch.empty_like(pts)
    nsdf.nsdf_collide(net.ctx, pts, EPS, torch.empty_like(pts), ref_ns)
    nsdf.nsdf_collide_noalloc(net.ctx, pts, EPS, out, got_ns)
    nsdf.nsdf_sync_status(net.ctx)
    assert torch.equal(got_ns, ref_ns)
    nsdf.nsdf_collide_noalloc(net.ctx, pts[:0], EPS, out[:0])          # n = 0: no-op
    with pytest.raises(nsdf.NsdfError) as e:                             # misaligned
        nsdf.nsdf_collide_noalloc(net.ctx, pts.view(-1)[1:41].view(10, 4), EPS, out[:10])
    assert e.value.status == 2
    net.close()


def test_noalloc_rejects_host_memory_and_bad_eps(nsdf):
    """Host arrays and a non-finite eps are refused before any launch."""
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(synth.geometric_init(arch, 0))
    lib = nsdf.library()
    host = torch.from_numpy(synth.body_scale_points(256, 13))
    dev = host.cuda()
    out = torch.empty_like(dev)
    # through the C ABI directly (the Python wrapper refuses CPU tensors itself)
    assert lib.nsdf_collide_noalloc(net.ctx, host.data_ptr(), 256, EPS, None, out.data_ptr(),
                                    None, None, None) == 1
    assert lib.nsdf_collide_noalloc(net.ctx, dev.data_ptr(), 256, EPS, None,
                                    torch.empty_like(host).data_ptr(), None, None, None) == 1
    hit = torch.empty(256, dtype=torch.uint8)
    assert lib.nsdf_collide_noalloc(net.ctx, dev.data_ptr(), 256, EPS, None, out.data_ptr(),
                                    None, hit.data_ptr(), None) == 1
    for bad in (float("inf"), float("-inf"), float("nan")):
        assert lib.nsdf_collide_noalloc(net.ctx, dev.data_ptr(), 256, bad, None, out.data_ptr(),
                                        None, None, None) == 1
    with pytest.raises(ValueError):
        nsdf.nsdf_collide_noalloc(net.ctx, host, EPS, out)
    nsdf.nsdf_sync_status(net.ctx)
    net.close()


def test_noalloc_too_large_is_rejected_before_launch(nsdf):
    """With the usable part of the array capped below one CTA's scratch (a
    test-only control: every network the library accepts fits the whole
    array), the call returns NSDF_ERR_TOO_LARGE and launches nothing; with
    the cap lifted the same call runs and matches nsdf_collide."""
    arch = synth.Arch(3, 512, 8, 4, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_BF16).load(synth.geometric_init(arch, 0))
    pts = torch.from_numpy(synth.body_scale_points(5000, 14)).cuda()
    out = torch.full_like(pts, 7.0)
    try:
        nsdf.nsdf_debug_noalloc_limit(64 << 10)      # 64 KiB < 896 KiB of slopes per CTA
        with pytest.raises(nsdf.NsdfError) as e:
            nsdf.nsdf_collide_noalloc(net.ctx, pts, EPS, out)
        assert e.value.status == 8
        torch.cuda.synchronize()
        assert bool((out == 7.0).all())               # nothing was written
    finally:
        nsdf.nsdf_debug_noalloc_limit(0)
    ref, got = torch.empty_like(pts), torch.empty_like(pts)
    nsdf.nsdf_collide(net.ctx, pts, EPS, torch.empty_like(pts), ref)
    nsdf.nsdf_collide_noalloc(net.ctx, pts, EPS, out, got)
    nsdf.nsdf_sync_status(net.ctx)
    assert torch.equal(got, ref)
    net.close()
