"""The C-ABI library builds, loads and exports every entry point of include/nsdf.h.

CPU-only: these tests make no compute call (no GPU is needed); they check the
host-side logic that runs before any CUDA call.
"""

import ctypes
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    """Every function declared by a header under include/."""
    inc = os.path.join(ROOT, "include")
    names = set()
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(nsdf_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("nsdf_create", "nsdf_destroy", "nsdf_load_weights", "nsdf_query",
                     "nsdf_collide", "nsdf_backward", "nsdf_query_grouped"):
        assert required in names


def test_library_exports_every_declared_symbol(nsdf_lib):
    from paper_2110_01614_gb300 import _abi
    for name in declared_symbols():
        assert hasattr(nsdf_lib, name), name
        assert name in _abi.SIGNATURES, name


def test_num_params_matches_generator(nsdf_lib):
    import paper_2110_01614_gb300 as nsdf
    for a in (synth.Arch(3, 64, 3, -1), synth.Arch(3, 512, 8, 4), synth.Arch(3, 32, 5, 2)):
        assert nsdf.nsdf_num_params(a) == synth.n_params(a)
    assert nsdf.nsdf_num_params(nsdf.make_arch(64, 3, skip_layer=3)) == 0   # skip at output
    assert nsdf.nsdf_num_params(nsdf.make_arch(64, 3, in_dim=2)) == 0


def test_create_rejects_bad_arguments_before_touching_the_device(nsdf_lib):
    import paper_2110_01614_gb300 as nsdf
    h = ctypes.c_void_p()
    bad = nsdf.make_arch(64, 3, beta=-1.0)
    assert nsdf_lib.nsdf_create(ctypes.byref(bad), 0, 1, ctypes.byref(h)) == 1
    good = nsdf.make_arch(64, 3)
    assert nsdf_lib.nsdf_create(ctypes.byref(good), 0, 0, ctypes.byref(h)) == 1
    assert nsdf_lib.nsdf_create(ctypes.byref(good), 7, 1, ctypes.byref(h)) == 1
    odd = nsdf.make_arch(100, 3)
    assert nsdf_lib.nsdf_create(ctypes.byref(odd), 0, 1, ctypes.byref(h)) == 6
    assert nsdf_lib.nsdf_create(ctypes.byref(good), 0, 1, None) == 1


def test_status_strings(nsdf_lib):
    import paper_2110_01614_gb300 as nsdf
    assert nsdf.nsdf_status_string(0) == "ok"
    assert "aligned" in nsdf.nsdf_status_string(2)
    assert nsdf.nsdf_status_string(99) == "unknown status"


def test_null_context_calls_fail_cleanly(nsdf_lib):
    assert nsdf_lib.nsdf_query(None, None, 0, None, 0, None) == 1
    assert nsdf_lib.nsdf_destroy(None) == 1
    assert nsdf_lib.nsdf_sync_status(None, None) == 1
    # n == 0 with no context is still an argument error; with bad sizes too
    assert nsdf_lib.nsdf_mesh_sdf(None, 0, None, 0, None, -1, None, None) == 1
    assert nsdf_lib.nsdf_mesh_sdf(None, 0, None, 0, None, 0, None, None) == 0
    assert nsdf_lib.nsdf_cloth_step(None, None, 0, 4, 0.1, 0.1, 1.0, 9.81, 1e-3, None) == 0


def test_cloth_step_rejects_sizes_beyond_its_index_range(nsdf_lib):
    """Rows beyond the grid's y limit and columns beyond 2^30 are refused
    before any pointer is examined (the addresses here are never touched)."""
    fake_a, fake_b = 1 << 20, 2 << 20
    assert nsdf_lib.nsdf_cloth_step(fake_a, fake_b, 64, 65536, 0.1, 0.1, 1.0, 9.81, 1e-3, None) == 1
    assert nsdf_lib.nsdf_cloth_step(fake_a, fake_b, (1 << 30) + 1, 2, 0.1, 0.1, 1.0, 9.81, 1e-3,
                                    None) == 1
    assert nsdf_lib.nsdf_cloth_step(fake_a, fake_a, 64, 2, 0.1, 0.1, 1.0, 9.81, 1e-3, None) == 1
