"""sp2_truncate_noalloc -- the allocation-free truncation entry point for callers
that cannot allocate device memory (graph capture, frameworks that own all
device memory).  Its keep flags must equal those of sp2_truncate on the same
input, on two calls in a row (the shared scratch keeps the previous call's
contents, so the second call checks that it is cleared where it must be)."""
import ctypes

import numpy as np
import pytest

from synth import from_dense

pytestmark = pytest.mark.gpu


def _decaying(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = 0.5 * (A + A.T)
    d = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    A *= np.exp(-d / 30.0)
    return from_dense(A, keep_zero_tiles=True)


def _noalloc(X, tau, mode, part):
    import torch
    import paper_1909_12533_gb300 as sp2
    lib = sp2.load()
    br = torch.from_numpy(X.brow).cuda()
    bc = torch.from_numpy(X.bcol).cuda()
    va = torch.from_numpy(X.val).cuda()
    keep = torch.full((X.nnzb,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sp2_truncate_noalloc(ctypes.c_void_p(br.data_ptr()), ctypes.c_void_p(bc.data_ptr()),
                                  ctypes.c_void_p(va.data_ptr()), X.n, X.nnzb, float(tau),
                                  sp2.TRUNCS[mode], int(part), ctypes.c_void_p(keep.data_ptr()), stream)
    torch.cuda.synchronize()
    assert rc == 0, sp2.sp2_strerror(rc)
    return keep.cpu().numpy()


@pytest.mark.parametrize("mode,part", [("frobenius", 4096), ("frobinf", 128)])
def test_noalloc_matches_allocating_entry_point_twice(mode, part):
    import paper_1909_12533_gb300 as sp2
    first = _decaying(1000, 1)     # 32 tile rows (ragged)
    second = _decaying(700, 2)     # a different size: stale scratch must not leak in
    for X, tau in ((first, 1e-3), (second, 1e-4)):
        ref = sp2.sp2_truncate(X, tau, mode, part)
        got = _noalloc(X, tau, mode, part)
        assert np.array_equal(got, ref)
        assert 0 < ref.sum() < X.nnzb


def test_noalloc_rejects_oversized_input():
    import paper_1909_12533_gb300 as sp2
    lib = sp2.load()
    rc = lib.sp2_truncate_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 10**6,
                                  (1 << 18) + 1, 1e-6, 0, 4096, ctypes.c_void_p(16), None)
    assert rc == -11
    assert "scratch" in sp2.sp2_strerror(rc)
