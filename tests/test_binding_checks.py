"""The binding refuses tensors of the wrong dtype or size before it calls the
library: the C ABI sees bare pointers and counts, so such a tensor would make
a kernel read or write past its end.  CPU only (each call raises before any
library call)."""

import pytest
import torch

import paper_2110_01614_gb300 as nsdf

CTX = 12345     # never dereferenced: every call below raises first


def rec(n, dtype=torch.float32, cols=4):
    return torch.zeros(n, cols, dtype=dtype)


@pytest.mark.parametrize("pts,out", [
    (rec(8, cols=3), rec(8)),                     # float3 rows
    (rec(8, dtype=torch.float16), rec(8)),        # 8-byte rows
    (rec(8, dtype=torch.float64), rec(8)),        # not the ABI's type
    (rec(8), rec(7)),                             # output too short
    (rec(8), rec(8, cols=3)),
])
def test_query_and_collide_refuse_bad_records(pts, out):
    with pytest.raises(ValueError):
        nsdf.nsdf_query(CTX, pts, out)
    with pytest.raises(ValueError):
        nsdf.nsdf_collide(CTX, pts, 0.002, out)


def test_collide_refuses_short_or_wide_outputs():
    pts = rec(8)
    with pytest.raises(ValueError):
        nsdf.nsdf_collide(CTX, pts, 0.002, rec(8), out_n_sdf=rec(4))
    with pytest.raises(ValueError):
        nsdf.nsdf_collide(CTX, pts, 0.002, rec(8), out_hit=torch.zeros(7, dtype=torch.uint8))
    with pytest.raises(ValueError):
        nsdf.nsdf_collide(CTX, pts, 0.002, rec(8), out_hit=torch.zeros(8, dtype=torch.float32))


def test_backward_refuses_bad_arguments():
    pts = rec(8)
    with pytest.raises(ValueError):
        nsdf.nsdf_backward(CTX, pts, torch.zeros(7))                       # g_sdf short
    with pytest.raises(ValueError):
        nsdf.nsdf_backward(CTX, pts, torch.zeros(8, dtype=torch.float64))
    with pytest.raises(ValueError):
        nsdf.nsdf_backward(CTX, pts, torch.zeros(8), g_grad=rec(8, cols=3))
    with pytest.raises(ValueError):
        nsdf.nsdf_backward(CTX, pts, torch.zeros(8), g_weights=torch.zeros(4, dtype=torch.float16))
    with pytest.raises(ValueError):
        nsdf.nsdf_backward(CTX, pts, torch.zeros(8), g_pts=rec(7))


def test_grouped_refuses_bad_work_lists():
    pts, out = rec(100), rec(100)
    off = torch.tensor([0, 50], dtype=torch.int64)
    cnt = torch.tensor([50, 50], dtype=torch.int64)
    with pytest.raises(ValueError):       # int32 offsets would be read as int64
        nsdf.nsdf_query_grouped(CTX, pts, off.int(), cnt, 100, 0.002, out)
    with pytest.raises(ValueError):
        nsdf.nsdf_query_grouped(CTX, pts, off, cnt[:1], 100, 0.002, out)
    with pytest.raises(ValueError):       # fewer points than max_total
        nsdf.nsdf_query_grouped(CTX, rec(99), off, cnt, 100, 0.002, out)
    with pytest.raises(ValueError):
        nsdf.nsdf_query_grouped(CTX, pts, off, cnt, 100, 0.002, rec(99))
    with pytest.raises(ValueError):       # one pose short
        nsdf.nsdf_query_grouped_T(CTX, pts, off, cnt, 100, 0.002, torch.zeros(1, 4, 4), out)
    with pytest.raises(ValueError):
        nsdf.nsdf_query_grouped_T(CTX, pts, off, cnt, 100, 0.002,
                                  torch.zeros(2, 4, 4, dtype=torch.float64), out)
    with pytest.raises(ValueError):
        nsdf.nsdf_autotune_grouped(CTX, pts, off, cnt, 101, 0.002, out)


def test_l1_grad_mesh_cloth_and_voxel_refuse_bad_arguments():
    pts = rec(8)
    with pytest.raises(ValueError):
        nsdf.nsdf_l1_grad(CTX, pts, torch.zeros(7), torch.zeros(10))
    with pytest.raises(ValueError):
        nsdf.nsdf_l1_grad(CTX, pts, torch.zeros(8), torch.zeros(10), loss=torch.zeros(0))
    V, F = torch.zeros(4, 3), torch.zeros(2, 3, dtype=torch.int32)
    with pytest.raises(ValueError):
        nsdf.nsdf_mesh_sdf(V, F.long(), pts, torch.zeros(8))              # int64 faces
    with pytest.raises(ValueError):
        nsdf.nsdf_mesh_sdf(V.reshape(-1), F, pts, torch.zeros(8))
    with pytest.raises(ValueError):
        nsdf.nsdf_mesh_sdf(V, F, pts, torch.zeros(7))
    with pytest.raises(ValueError):
        nsdf.nsdf_cloth_step(rec(15), rec(16), 4, 4, 0.1, 0.1, 1.0, 9.81, 1e-3)
    with pytest.raises(ValueError):
        nsdf.nsdf_voxel_build(V, F, 4, (-1, -1, -1), (1, 1, 1), torch.zeros(63))
    with pytest.raises(ValueError):
        nsdf.nsdf_voxel_collide(torch.zeros(63), 4, (-1, -1, -1), (1, 1, 1), pts, 0.002, rec(8))
    with pytest.raises(ValueError):
        nsdf.nsdf_voxel_collide(torch.zeros(64), 4, (-1, -1, -1), (1, 1, 1), pts, 0.002, rec(6))
