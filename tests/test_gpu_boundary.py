"""The rest of the C ABI against the oracle: dense entry points
(sp2_create_dense, sp2_copy_D_dense), the Python ``run`` call, a caller's
allocator (including one that fails), and the error paths that the library
reports without any fault (bounded-wait timeout and out-of-range slices, both
through the ``selftest`` parameter)."""
import ctypes

import numpy as np
import pytest

from synth import dense_gapped, from_dense, make_config
from tests.helpers import run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def test_create_dense_host_and_device_match_tiles_and_oracle():
    import torch
    import paper_1909_12533_gb300 as sp2
    d = dense_gapped(100, 37, (-2.0, -0.3), (0.4, 2.0), seed=7)   # 3 full tiles and a ragged tail
    F = d["F"]
    o = run_oracle(F, d["nocc"], d["homo_ub"], d["lumo_lb"], 1e-7)
    # host F with a leading dimension larger than n (only the n x n part is read)
    Fld = np.full((100, 104), np.nan)
    Fld[:, :100] = F
    lib = sp2.load()
    ctx = ctypes.c_void_p()
    prm = sp2.sp2_default_params()
    rc = lib.sp2_create_dense(ctypes.c_void_p(Fld.ctypes.data), 100, 104, 0, d["nocc"], d["homo_ub"], d["lumo_lb"],
                              1e-7, ctypes.byref(prm), None, sp2._stream_handle(None), ctypes.byref(ctx))
    assert rc == 0, sp2.sp2_strerror(rc)
    code, st = sp2.sp2_run(ctx)
    assert code == 0 and st.n == o.n
    Dh = np.full((100, 101), 7.0)
    assert lib.sp2_copy_D_dense(ctx, ctypes.c_void_p(Dh.ctypes.data), 101, 0) == 0
    assert np.all(Dh[:, 100] == 7.0)           # outside the n x n part: untouched
    assert np.linalg.norm(Dh[:, :100] - o.D) <= 1e-10
    # the same D as the tile-set entry point, bit for bit
    g = run_gpu(F, d["nocc"], d["homo_ub"], d["lumo_lb"], 1e-7)
    assert np.array_equal(Dh[:, :100], g["D"])
    sp2.sp2_destroy(ctx)
    # device F and device D through the Python call
    Dd, st2 = sp2.run(torch.from_numpy(F).cuda(), d["nocc"], d["homo_ub"], d["lumo_lb"], 1e-7)
    assert Dd.is_cuda and np.array_equal(Dd.cpu().numpy(), g["D"])
    assert st2["n"] == o.n


def test_create_dense_config1_against_projector():
    import oracle.sp2_oracle as O
    import paper_1909_12533_gb300 as sp2
    c = make_config(1)
    D, st = sp2.run(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], 0.0, stop="idempotency")
    assert isinstance(D, np.ndarray) and st["converged"]
    assert np.linalg.norm(D - O.eig_projector(c["F"], c["nocc"])) < 1e-11
    # dense F with exactly zero off-diagonal tiles: they stay out of the pattern
    a = dense_gapped(64, 32, (-1.0, -0.5), (0.5, 1.0), seed=3)["F"]
    F = np.zeros((128, 128))
    F[:64, :64] = a
    F[64:, 64:] = a
    D, st = sp2.run(F, 64, -0.5, 0.5, 0.0, stop="idempotency")
    o = run_oracle(from_dense(F), 64, -0.5, 0.5, 0.0, stop="idempotency")
    assert st["nnzb_hist"][0] == 6 and np.linalg.norm(D - o.D) <= 1e-10


def test_run_on_a_tile_set():
    import paper_1909_12533_gb300 as sp2
    c = make_config("2s")
    (brow, bcol, val), st = sp2.run(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"])
    assert np.array_equal(val, g["val"]) and np.array_equal(brow, g["brow"]) and st["n"] == g["stats"]["n"]


class _CountingAllocator:
    """A caller's device allocator (cudaMalloc / cudaFree through ctypes) that
    fails after ``fail_after`` successful allocations and tracks what is live."""

    def __init__(self, fail_after=None):
        import paper_1909_12533_gb300 as sp2
        self.rt = sp2._cudart()
        self.rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
        self.rt.cudaMalloc.restype = ctypes.c_int
        self.rt.cudaFree.argtypes = [ctypes.c_void_p]
        self.rt.cudaFree.restype = ctypes.c_int
        self.fail_after = fail_after
        self.calls = 0
        self.live = {}
        alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
        self._alloc = alloc_t(self.alloc)
        self._free = free_t(self.free)
        self.struct = sp2.sp2_allocator(alloc=ctypes.cast(self._alloc, ctypes.c_void_p).value,
                                        free=ctypes.cast(self._free, ctypes.c_void_p).value, user=None)

    def alloc(self, nbytes, user):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return None
        p = ctypes.c_void_p()
        if self.rt.cudaMalloc(ctypes.byref(p), nbytes) != 0:
            return None
        self.live[p.value] = nbytes
        return p.value

    def free(self, ptr, user):
        if ptr:
            assert ptr in self.live
            del self.live[ptr]
            self.rt.cudaFree(ptr)


def test_caller_allocator_gives_same_result_and_frees_everything():
    import paper_1909_12533_gb300 as sp2
    c = make_config("2s")
    al = _CountingAllocator()
    ctx = sp2.SP2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], allocator=al.struct,
                  precision="split16")
    st = ctx.run()
    brow, bcol, val = ctx.D_host()
    ctx.close()
    assert al.calls > 10 and not al.live
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16")
    assert np.array_equal(val, g["val"]) and st["n"] == g["stats"]["n"]


@pytest.mark.parametrize("fail_after", [0, 3, 12, 40])
def test_caller_allocator_failure_is_oom_without_leaks(fail_after):
    # an allocator that returns NULL after k allocations: create or run returns
    # SP2_ERR_OOM, and every block it did hand out comes back
    import paper_1909_12533_gb300 as sp2
    c = make_config("2s")
    al = _CountingAllocator(fail_after=fail_after)
    code = 0
    ctx = None
    try:
        ctx = sp2.SP2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], allocator=al.struct)
        ctx.run()
        code = ctx.code
    except sp2.SP2Error as e:
        code = e.code
    finally:
        if ctx is not None:
            ctx.close()
    assert code == -5, code
    assert not al.live
    sp2.sp2_release_memory()


def test_timeout_selftest_then_next_run_succeeds():
    # selftest = 1: the first tensor-core square waits on a barrier that nothing
    # arrives at and gives up after wait_limit_ms (no data moved, no fault); the
    # next run of the same context succeeds and matches a fresh context
    import paper_1909_12533_gb300 as sp2
    c = make_config("2s")
    ctx = sp2.SP2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", selftest=1,
                  wait_limit_ms=200)
    with pytest.raises(sp2.SP2Error) as e:
        ctx.run()
    assert e.value.code == -8
    st = ctx.run()
    assert ctx.code == 0
    _, _, val = ctx.D_host()
    ctx.close()
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16")
    assert np.array_equal(val, g["val"]) and st["n"] == g["stats"]["n"]


def test_range_selftest_reports_range_error_then_next_run_succeeds():
    import paper_1909_12533_gb300 as sp2
    c = make_config("2s")
    ctx = sp2.SP2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", selftest=2)
    with pytest.raises(sp2.SP2Error) as e:
        ctx.run()
    assert e.value.code == -12
    ctx.run()
    assert ctx.code == 0
    ctx.close()
