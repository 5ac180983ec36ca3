"""The C-ABI library loads and exports every function declared in include/sp2.h
(no compute calls: these run without a GPU)."""
import ctypes

import pytest

import paper_1909_12533_gb300 as sp2


def test_library_exists_and_loads():
    if not sp2.lib_path().exists():
        from paper_1909_12533_gb300 import build
        build.build()
    lib = sp2.load()
    assert isinstance(lib, ctypes.CDLL)


def test_every_declared_symbol_is_exported():
    lib = sp2.load()
    names = sp2.header_functions()
    assert "sp2_create" in names and "sp2_run" in names and "sp2_backward" in names and "sp2_get_D" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    declared = set(sp2.header_functions())
    bound = {n for n, *_ in sp2._SIGS}
    assert declared <= bound, declared - bound


def test_default_params_and_strerror():
    p = sp2.sp2_default_params()
    assert p.mode == 1 and p.stop == 0 and p.trunc == 0 and p.frobinf_part == 4096
    assert p.n_max_cap == 100 and p.ckpt_every == 8 and p.slices == 4 and p.record_masks == 0
    assert sp2.sp2_strerror(0) == "ok"
    assert "bounds" in sp2.sp2_strerror(-2)


def test_struct_sizes_match_header_layout():
    # int64 n, int32 b (+pad), int64 nnzb, 3 pointers, int32 on_device (+pad)
    assert ctypes.sizeof(sp2.sp2_bsr) == 8 + 8 + 8 + 3 * 8 + 8


def test_create_rejects_bad_arguments_before_any_device_work():
    lib = sp2.load()
    out = ctypes.c_void_p()
    # NULL matrix -> invalid argument; no CUDA call is made on this path
    rc = lib.sp2_create(None, 1, -1.0, 1.0, 0.0, None, None, None, ctypes.byref(out))
    assert rc == -1 and not out.value
    bsr = sp2.sp2_bsr(n=64, b=16, nnzb=1, brow=1, bcol=1, val=1, on_device=0)
    assert lib.sp2_create(ctypes.byref(bsr), 1, -1.0, 1.0, 0.0, None, None, None, ctypes.byref(out)) == -1
    bsr.b = 32
    # homo_ub >= lumo_lb -> bounds error
    assert lib.sp2_create(ctypes.byref(bsr), 1, 1.0, -1.0, 0.0, None, None, None, ctypes.byref(out)) == -2
    # NaN bound -> invalid argument
    assert lib.sp2_create(ctypes.byref(bsr), 1, float("nan"), 1.0, 0.0, None, None, None, ctypes.byref(out)) == -1
    # negative tau -> invalid argument
    assert lib.sp2_create(ctypes.byref(bsr), 1, -1.0, 1.0, -1.0, None, None, None, ctypes.byref(out)) == -1
    p = sp2.sp2_default_params(slices=7, precision="split16")
    assert lib.sp2_create(ctypes.byref(bsr), 1, -1.0, 1.0, 0.0, ctypes.byref(p), None, None, ctypes.byref(out)) == -1
    assert lib.sp2_run(None, None) == -1
    assert lib.sp2_get_D(None, None) == -1
