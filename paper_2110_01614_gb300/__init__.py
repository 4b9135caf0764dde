"""Python binding of the nsdf C ABI (GB300-native neural-SDF collision queries).

Functions carry the names of the C entry points in ``include/nsdf.h`` and
only marshal arguments: tensors become raw pointers, the stream defaults to
PyTorch's current stream, and a non-OK status raises ``NsdfError``.  All
arithmetic runs in the CUDA kernels of ``libnsdf.so``; importing this
package loads that library and fails loudly if it has not been built.

Layouts (see the header for the full contract): points and results are
float32 tensors of shape [n, 4]; weight blobs are float32 vectors in the
packed layout of ``nsdf_num_params``.
"""

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import (NSDF_ACT_RELU, NSDF_ACT_SOFTPLUS, NSDF_BF16, NSDF_FP16, NSDF_FP32,
                   NSDF_RAW_GRADIENT, nsdf_arch)

__all__ = [
    "NsdfError", "NSDF_FP32", "NSDF_BF16", "NSDF_FP16", "NSDF_RAW_GRADIENT", "NSDF_ACT_SOFTPLUS",
    "NSDF_ACT_RELU", "make_arch",
    "nsdf_num_params", "nsdf_create", "nsdf_destroy", "nsdf_load_weights",
    "nsdf_query", "nsdf_collide", "nsdf_collide_noalloc", "nsdf_backward", "nsdf_query_grouped",
    "nsdf_query_grouped_T", "nsdf_l1_grad",
    "nsdf_autotune_grouped", "nsdf_set_grouped_config",
    "nsdf_mesh_sdf", "nsdf_cloth_step", "nsdf_sync_status", "nsdf_debug_inject",
    "nsdf_debug_noalloc_limit", "nsdf_debug_fp32_fma_peak", "nsdf_debug_tc16_one_cta", "nsdf_voxel_build",
    "nsdf_voxel_collide",
    "nsdf_status_string", "NeuralSDF", "library",
]


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _abi.load()


class NsdfError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = library().nsdf_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")


def _check(status, what):
    if status != _abi.NSDF_OK:
        raise NsdfError(status, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("nsdf needs contiguous tensors")
        return t.data_ptr()
    return int(t)


# Argument checks of the binding: the C ABI sees bare pointers and counts, so
# a tensor of the wrong dtype or size would make a kernel read or write past
# its end.  These refuse such tensors (ValueError) before the library is
# called; raw integer pointers pass unchecked.
def _records(t, name, rows=None, optional=False):
    """float4 records: a float32 [n, 4] tensor with at least `rows` rows."""
    if t is None and optional or not isinstance(t, torch.Tensor):
        return
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 4:
        raise ValueError(f"{name} must be a float32 [n, 4] tensor of float4 records, "
                         f"got {t.dtype} {tuple(t.shape)}")
    if rows is not None and t.shape[0] < rows:
        raise ValueError(f"{name} holds {t.shape[0]} records; the call needs {rows}")


def _values(t, name, dtypes, count, optional=False):
    """A tensor of one of `dtypes` with at least `count` elements."""
    if t is None and optional or not isinstance(t, torch.Tensor):
        return
    if t.dtype not in dtypes:
        raise ValueError(f"{name} must be {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} values; the call needs {count}")


def _triangles(verts, faces):
    _values(verts, "verts", (torch.float32,), 0)
    _values(faces, "faces", (torch.int32,), 0)
    for t, name in ((verts, "verts"), (faces, "faces")):
        if isinstance(t, torch.Tensor) and (t.dim() != 2 or t.shape[1] != 3):
            raise ValueError(f"{name} must be [n, 3], got {tuple(t.shape)}")


def _work_list(pts, offsets, counts, max_total, out_pts, out_n_sdf, T=None):
    _records(pts, "pts", max_total)
    _records(out_pts, "out_pts", max_total)
    _records(out_n_sdf, "out_n_sdf", max_total, optional=True)
    _values(offsets, "offsets", (torch.int64,), 0)
    _values(counts, "counts", (torch.int64,), 0)
    if isinstance(offsets, torch.Tensor) and isinstance(counts, torch.Tensor):
        if offsets.numel() != counts.numel():
            raise ValueError("offsets and counts must have one entry per network")
        _values(T, "T", (torch.float32,), 16 * offsets.numel(), optional=True)


_HIT = (torch.uint8, torch.bool)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def make_arch(width, n_hidden, skip_layer=-1, beta=100.0, in_dim=3, activation="softplus",
              ff_freqs=0):
    return nsdf_arch(in_dim, width, n_hidden, skip_layer, beta,
                     NSDF_ACT_RELU if activation == "relu" else NSDF_ACT_SOFTPLUS, ff_freqs)


def _arch(a):
    if isinstance(a, nsdf_arch):
        return a
    return make_arch(a.width, a.n_hidden, a.skip_layer, a.beta, a.in_dim,
                     getattr(a, "activation", "softplus"), getattr(a, "ff_freqs", 0))


def nsdf_status_string(status):
    return library().nsdf_status_string(status).decode()


def nsdf_num_params(arch):
    return int(library().nsdf_num_params(ctypes.byref(_arch(arch))))


def nsdf_create(arch, precision=NSDF_FP32, n_nets=1):
    h = ctypes.c_void_p()
    _check(library().nsdf_create(ctypes.byref(_arch(arch)), int(precision), int(n_nets),
                                 ctypes.byref(h)), "nsdf_create")
    return h.value


def nsdf_destroy(ctx):
    _check(library().nsdf_destroy(ctx), "nsdf_destroy")


def nsdf_load_weights(ctx, net, w, stream=None):
    if w.dtype != torch.float32:
        raise ValueError("weight blob must be float32")
    _check(library().nsdf_load_weights(ctx, int(net), _ptr(w), w.numel(), int(w.is_cuda),
                                       _stream(stream)), "nsdf_load_weights")


def nsdf_query(ctx, pts, out_n_sdf, flags=0, stream=None):
    _records(pts, "pts")
    _records(out_n_sdf, "out_n_sdf", pts.shape[0])
    _check(library().nsdf_query(ctx, _ptr(pts), pts.shape[0], _ptr(out_n_sdf), int(flags),
                                _stream(stream)), "nsdf_query")


def _transform(T):
    if T is None:
        return None
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float32).reshape(16))
    return (ctypes.c_float * 16)(*a.tolist())


def _collide_args(pts, out_pts, out_n_sdf, out_hit):
    _records(pts, "pts")
    n = pts.shape[0]
    _records(out_pts, "out_pts", n)
    _records(out_n_sdf, "out_n_sdf", n, optional=True)
    _values(out_hit, "out_hit", _HIT, n, optional=True)


def nsdf_collide(ctx, pts, eps, out_pts, out_n_sdf=None, out_hit=None, T=None, stream=None):
    _collide_args(pts, out_pts, out_n_sdf, out_hit)
    Tc = _transform(T)
    _check(library().nsdf_collide(ctx, _ptr(pts), pts.shape[0], float(eps),
                                  ctypes.cast(Tc, ctypes.c_void_p) if Tc is not None else None,
                                  _ptr(out_pts), _ptr(out_n_sdf), _ptr(out_hit),
                                  _stream(stream)), "nsdf_collide")


def nsdf_collide_noalloc(ctx, pts, eps, out_pts, out_n_sdf=None, out_hit=None, T=None,
                         stream=None):
    """nsdf_collide with no allocation: scratch from the library's fixed device array.

    Every array must live on the GPU (the library also rejects host memory)."""
    for name, t in (("pts", pts), ("out_pts", out_pts), ("out_n_sdf", out_n_sdf),
                    ("out_hit", out_hit)):
        if t is not None and not getattr(t, "is_cuda", False):
            raise ValueError(f"nsdf_collide_noalloc: {name} must be a CUDA tensor")
    _collide_args(pts, out_pts, out_n_sdf, out_hit)
    Tc = _transform(T)
    _check(library().nsdf_collide_noalloc(ctx, _ptr(pts), pts.shape[0], float(eps),
                                          ctypes.cast(Tc, ctypes.c_void_p) if Tc is not None
                                          else None, _ptr(out_pts), _ptr(out_n_sdf),
                                          _ptr(out_hit), _stream(stream)),
           "nsdf_collide_noalloc")


def nsdf_backward(ctx, pts, g_sdf, g_grad=None, g_weights=None, g_pts=None, stream=None):
    _records(pts, "pts")
    n = pts.shape[0]
    _values(g_sdf, "g_sdf", (torch.float32,), n)
    _records(g_grad, "g_grad", n, optional=True)
    _values(g_weights, "g_weights", (torch.float32,), 0, optional=True)
    _records(g_pts, "g_pts", n, optional=True)
    _check(library().nsdf_backward(ctx, _ptr(pts), pts.shape[0], _ptr(g_sdf), _ptr(g_grad),
                                   _ptr(g_weights), _ptr(g_pts), _stream(stream)),
           "nsdf_backward")


def nsdf_query_grouped(ctx, pts, offsets, counts, max_total, eps, out_pts, out_n_sdf=None,
                       stream=None):
    _work_list(pts, offsets, counts, max_total, out_pts, out_n_sdf)
    _check(library().nsdf_query_grouped(ctx, _ptr(pts), _ptr(offsets), _ptr(counts),
                                        int(max_total), float(eps), _ptr(out_pts),
                                        _ptr(out_n_sdf), _stream(stream)), "nsdf_query_grouped")


def nsdf_query_grouped_T(ctx, pts, offsets, counts, max_total, eps, T, out_pts, out_n_sdf=None,
                         stream=None):
    """nsdf_query_grouped with a device [n_nets, 4, 4] tensor of body poses."""
    _work_list(pts, offsets, counts, max_total, out_pts, out_n_sdf, T)
    _check(library().nsdf_query_grouped_T(ctx, _ptr(pts), _ptr(offsets), _ptr(counts),
                                          int(max_total), float(eps), _ptr(T), _ptr(out_pts),
                                          _ptr(out_n_sdf), _stream(stream)), "nsdf_query_grouped_T")


def nsdf_l1_grad(ctx, pts, targets, g_weights, loss=None, stream=None):
    """Gradient of mean |f(p) - d| for a 16-bit context (Sec. 3.1 fitting loss)."""
    _records(pts, "pts")
    _values(targets, "targets", (torch.float32,), pts.shape[0])
    _values(g_weights, "g_weights", (torch.float32,), 0)
    _values(loss, "loss", (torch.float32,), 1, optional=True)
    _check(library().nsdf_l1_grad(ctx, _ptr(pts), pts.shape[0], _ptr(targets), _ptr(g_weights),
                                  _ptr(loss), _stream(stream)), "nsdf_l1_grad")


def nsdf_autotune_grouped(ctx, pts, offsets, counts, max_total, eps, out_pts, out_n_sdf=None,
                          stream=None):
    """Time the grouped launch's tile shapes on this problem; returns (points/thread, CTAs/SM)."""
    _work_list(pts, offsets, counts, max_total, out_pts, out_n_sdf)
    chosen = (ctypes.c_int * 2)()
    _check(library().nsdf_autotune_grouped(ctx, _ptr(pts), _ptr(offsets), _ptr(counts),
                                           int(max_total), float(eps), _ptr(out_pts),
                                           _ptr(out_n_sdf), _stream(stream), chosen),
           "nsdf_autotune_grouped")
    return int(chosen[0]), int(chosen[1])


def nsdf_set_grouped_config(ctx, points_per_thread, ctas_per_sm):
    _check(library().nsdf_set_grouped_config(ctx, int(points_per_thread), int(ctas_per_sm)),
           "nsdf_set_grouped_config")


def nsdf_mesh_sdf(verts, faces, pts, out_sdf, stream=None):
    _triangles(verts, faces)
    _records(pts, "pts")
    _values(out_sdf, "out_sdf", (torch.float32,), pts.shape[0])
    _check(library().nsdf_mesh_sdf(_ptr(verts), verts.shape[0], _ptr(faces), faces.shape[0],
                                   _ptr(pts), pts.shape[0], _ptr(out_sdf), _stream(stream)),
           "nsdf_mesh_sdf")


def nsdf_cloth_step(x, x_prev, nx, ny, hx, hz, k_over_m, g, dt, stream=None):
    _records(x, "x", int(nx) * int(ny))
    _records(x_prev, "x_prev", int(nx) * int(ny))
    _check(library().nsdf_cloth_step(_ptr(x), _ptr(x_prev), int(nx), int(ny), float(hx),
                                     float(hz), float(k_over_m), float(g), float(dt),
                                     _stream(stream)), "nsdf_cloth_step")


def nsdf_debug_inject(ctx, drop_load=-1, wait_budget_cycles=4_000_000_000):
    """Test-only: drop one weight-panel load and/or shorten the kernel's bounded waits."""
    _check(library().nsdf_debug_inject(ctx, int(drop_load), int(wait_budget_cycles)),
           "nsdf_debug_inject")


def nsdf_debug_tc16_one_cta(enable):
    """Width-512 tensor-core launches after this use one CTA per tile (True) or CTA pairs (False, the default)."""
    _check(library().nsdf_debug_tc16_one_cta(1 if enable else 0), "nsdf_debug_tc16_one_cta")


def nsdf_debug_noalloc_limit(nbytes):
    """Test-only: cap the bytes of nsdf_collide_noalloc's fixed array (0 = all)."""
    _check(library().nsdf_debug_noalloc_limit(int(nbytes)), "nsdf_debug_noalloc_limit")


def _box(lo, hi):
    a = (ctypes.c_float * 3)(*[float(v) for v in lo])
    b = (ctypes.c_float * 3)(*[float(v) for v in hi])
    return a, b


def nsdf_voxel_build(verts, faces, n, lo, hi, grid, stream=None):
    """Fill grid (device float [n^3]) with the exact signed distance of every node."""
    _triangles(verts, faces)
    _values(grid, "grid", (torch.float32,), int(n) ** 3 if int(n) > 0 else 0)
    a, b = _box(lo, hi)
    _check(library().nsdf_voxel_build(_ptr(verts), verts.shape[0], _ptr(faces), faces.shape[0],
                                      int(n), ctypes.cast(a, ctypes.c_void_p),
                                      ctypes.cast(b, ctypes.c_void_p), _ptr(grid),
                                      _stream(stream)), "nsdf_voxel_build")


def nsdf_voxel_collide(grid, n, lo, hi, pts, eps, out_pts, out_n_sdf=None, out_hit=None,
                       stream=None):
    """The collision query answered from a voxel grid (trilinear interpolation)."""
    _values(grid, "grid", (torch.float32,), int(n) ** 3 if int(n) > 0 else 0)
    _collide_args(pts, out_pts, out_n_sdf, out_hit)
    a, b = _box(lo, hi)
    _check(library().nsdf_voxel_collide(_ptr(grid), int(n), ctypes.cast(a, ctypes.c_void_p),
                                        ctypes.cast(b, ctypes.c_void_p), _ptr(pts), pts.shape[0],
                                        float(eps), _ptr(out_pts), _ptr(out_n_sdf), _ptr(out_hit),
                                        _stream(stream)), "nsdf_voxel_collide")


def nsdf_debug_fp32_fma_peak(stream=None):
    """Measured FP32 FMA throughput of the current GPU, TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(library().nsdf_debug_fp32_fma_peak(ctypes.byref(v), _stream(stream)),
           "nsdf_debug_fp32_fma_peak")
    return v.value


def nsdf_sync_status(ctx, stream=None):
    _check(library().nsdf_sync_status(ctx, _stream(stream)), "nsdf_sync_status")


class NeuralSDF:
    """Owns one nsdf context (n_nets networks of one shape) on the current GPU."""

    def __init__(self, arch, precision=NSDF_FP32, n_nets=1):
        self.arch = _arch(arch)
        self.precision = precision
        self.n_nets = n_nets
        self.ctx = nsdf_create(self.arch, precision, n_nets)

    def load(self, blob, net=0, stream=None):
        w = torch.as_tensor(blob, dtype=torch.float32)
        if not w.is_cuda:
            w = w.contiguous()
        nsdf_load_weights(self.ctx, net, w, stream)
        return self

    def query(self, pts, raw_gradient=False, out=None, stream=None):
        out = torch.empty_like(pts) if out is None else out
        nsdf_query(self.ctx, pts, out, NSDF_RAW_GRADIENT if raw_gradient else 0, stream)
        return out

    def collide(self, pts, eps, T=None, out_pts=None, out_n_sdf=None, out_hit=None, stream=None):
        out_pts = torch.empty_like(pts) if out_pts is None else out_pts
        nsdf_collide(self.ctx, pts, eps, out_pts, out_n_sdf, out_hit, T, stream)
        return out_pts

    def close(self):
        if getattr(self, "ctx", None):
            nsdf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
