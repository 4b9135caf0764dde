"""Every entry point that takes DEVICE pointers refuses host memory with
NSDF_ERR_INVALID_ARG (status 1) before it launches anything, so a host array
passed by mistake never reaches a kernel.  Called through the C ABI directly
(the Python wrappers refuse CPU tensors themselves); each output buffer is
pre-filled and must come back untouched.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

EPS = 0.002
INVALID_ARG = 1


@pytest.fixture(scope="module")
def nsdf(nsdf_lib):
    import paper_2110_01614_gb300 as m
    return m


def untouched(t, value=7.0):
    torch.cuda.synchronize()
    return bool((t == value).all())


def test_backward_rejects_host_memory(nsdf):
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32).load(synth.geometric_init(arch, 0))
    lib = nsdf.library()
    n = 300
    dev = torch.from_numpy(synth.body_scale_points(n, 3)).cuda()
    g_sdf = torch.ones(n, device="cuda")
    g_grad = torch.zeros_like(dev)
    gw = torch.full((nsdf.nsdf_num_params(arch),), 7.0, device="cuda")
    gp = torch.full_like(dev, 7.0)
    host = {"pts": dev.cpu(), "g_sdf": g_sdf.cpu(), "g_grad": g_grad.cpu(),
            "gw": gw.cpu(), "gp": gp.cpu()}
    args = {"pts": dev, "g_sdf": g_sdf, "g_grad": g_grad, "gw": gw, "gp": gp}
    for name in args:
        a = dict(args)
        a[name] = host[name]
        st = lib.nsdf_backward(net.ctx, a["pts"].data_ptr(), n, a["g_sdf"].data_ptr(),
                               a["g_grad"].data_ptr(), a["gw"].data_ptr(), a["gp"].data_ptr(), None)
        assert st == INVALID_ARG, name
    # the first-order route (no g_grad, no g_weights) and the n = 0 route check too
    assert lib.nsdf_backward(net.ctx, host["pts"].data_ptr(), n, g_sdf.data_ptr(), None, None,
                             gp.data_ptr(), None) == INVALID_ARG
    assert lib.nsdf_backward(net.ctx, dev.data_ptr(), 0, g_sdf.data_ptr(), None,
                             host["gw"].data_ptr(), None, None) == INVALID_ARG
    assert untouched(gw) and untouched(gp)
    # and the same arguments on the device still run
    assert lib.nsdf_backward(net.ctx, dev.data_ptr(), n, g_sdf.data_ptr(), g_grad.data_ptr(),
                             gw.data_ptr(), gp.data_ptr(), None) == 0
    nsdf.nsdf_sync_status(net.ctx)
    assert not untouched(gw)
    net.close()


def test_l1_grad_rejects_host_memory(nsdf):
    arch = synth.Arch(3, 256, 4, -1, 100.0, "relu", 128)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_BF16).load(synth.fourier_relu_init(arch, 0))
    lib = nsdf.library()
    n = 1000
    pts = torch.from_numpy(synth.body_scale_points(n, 4)).cuda()
    tgt = torch.zeros(n, device="cuda")
    gw = torch.full((nsdf.nsdf_num_params(arch),), 7.0, device="cuda")
    loss = torch.full((1,), 7.0, device="cuda")
    args = {"pts": pts, "tgt": tgt, "gw": gw, "loss": loss}
    for name in args:
        a = dict(args)
        a[name] = args[name].cpu()
        st = lib.nsdf_l1_grad(net.ctx, a["pts"].data_ptr(), n, a["tgt"].data_ptr(),
                              a["gw"].data_ptr(), a["loss"].data_ptr(), None)
        assert st == INVALID_ARG, name
    assert untouched(gw) and untouched(loss)
    net.close()


def test_grouped_launches_reject_host_memory(nsdf):
    arch = synth.Arch(3, 64, 3, -1, 100.0)
    net = nsdf.NeuralSDF(arch, nsdf.NSDF_FP32, n_nets=2)
    for k in range(2):
        net.load(synth.geometric_init(arch, k), net=k)
    lib = nsdf.library()
    counts = torch.tensor([100, 156], dtype=torch.int64, device="cuda")
    offs = torch.tensor([0, 100], dtype=torch.int64, device="cuda")
    pts = torch.from_numpy(synth.body_scale_points(256, 5)).cuda()
    out = torch.full_like(pts, 7.0)
    ns = torch.full_like(pts, 7.0)
    T = torch.eye(4, device="cuda").repeat(2, 1, 1).contiguous()
    args = {"pts": pts, "offs": offs, "counts": counts, "out": out, "ns": ns, "T": T}
    for name in args:
        a = dict(args)
        a[name] = args[name].cpu()
        if name != "T":
            st = lib.nsdf_query_grouped(net.ctx, a["pts"].data_ptr(), a["offs"].data_ptr(),
                                        a["counts"].data_ptr(), 256, EPS, a["out"].data_ptr(),
                                        a["ns"].data_ptr(), None)
            assert st == INVALID_ARG, name
        st = lib.nsdf_query_grouped_T(net.ctx, a["pts"].data_ptr(), a["offs"].data_ptr(),
                                      a["counts"].data_ptr(), 256, EPS, a["T"].data_ptr(),
                                      a["out"].data_ptr(), a["ns"].data_ptr(), None)
        assert st == INVALID_ARG, name
    chosen = (ctypes.c_int * 2)()
    st = lib.nsdf_autotune_grouped(net.ctx, pts.data_ptr(), offs.cpu().data_ptr(), counts.data_ptr(),
                                   256, EPS, out.data_ptr(), ns.data_ptr(), None, chosen)
    assert st == INVALID_ARG
    assert untouched(out) and untouched(ns)
    net.close()


def test_mesh_sdf_and_cloth_step_reject_host_memory(nsdf):
    lib = nsdf.library()
    V, F = synth.icosphere(2)
    V = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).cuda()
    F = torch.from_numpy(np.ascontiguousarray(F, dtype=np.int32)).cuda()
    pts = torch.from_numpy(synth.body_scale_points(128, 6)).cuda()
    out = torch.full((128,), 7.0, device="cuda")
    args = {"V": V, "F": F, "pts": pts, "out": out}
    for name in args:
        a = dict(args)
        a[name] = args[name].cpu()
        st = lib.nsdf_mesh_sdf(a["V"].data_ptr(), V.shape[0], a["F"].data_ptr(), F.shape[0],
                               a["pts"].data_ptr(), 128, a["out"].data_ptr(), None)
        assert st == INVALID_ARG, name
    assert untouched(out)

    nx, ny = 64, 32
    x = torch.zeros(ny * nx, 4, device="cuda")
    xp = torch.full_like(x, 7.0)
    assert lib.nsdf_cloth_step(x.cpu().data_ptr(), xp.data_ptr(), nx, ny, 0.01, 0.01, 1e5,
                               9.81, 1e-3, None) == INVALID_ARG
    assert lib.nsdf_cloth_step(x.data_ptr(), xp.cpu().data_ptr(), nx, ny, 0.01, 0.01, 1e5,
                               9.81, 1e-3, None) == INVALID_ARG
    assert untouched(xp)
