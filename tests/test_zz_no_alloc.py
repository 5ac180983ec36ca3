"""sp2_truncate_noalloc -- the allocation-free truncation entry point, for
callers that cannot allocate device memory: code that issues work while a CUDA
graph is being captured (an allocation there breaks the capture), callbacks of
frameworks that own all device memory, and processes whose allocator is locked
after start-up.  Its keep flags must equal those of sp2_truncate on the same
input, and the oracle's selection, on two calls in a row: the shared scratch
array keeps the previous call's contents, so the second call (of another size)
checks that everything that must start at zero is cleared.

This file is collected last on purpose (tests/test_zz_*): if it fails, a run
that stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from synth import from_dense, to_dense

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


def _oracle_keep(X, tau, mode, part):
    import oracle.sp2_oracle as O
    pattern = set(zip(X.brow.tolist(), X.bcol.tolist()))
    _, kept, _ = O.truncate_select(to_dense(X), tau, mode, part=part, pattern=pattern)
    ks = set(kept)
    return np.array([1 if (i, j) in ks else 0 for i, j in zip(X.brow.tolist(), X.bcol.tolist())], np.int32)


# Frobenius: 3000 and 2600 rows give 4465 and 3403 upper tiles, above the
# 2048-tile limit of the one-CTA select, so both calls run the multi-launch
# select in the shared scratch array.  Frob-Inf with 128-row super-blocks:
# 64 and 49 segments.
@pytest.mark.parametrize("mode,part,sizes", [("frobenius", 4096, (3000, 2600)), ("frobinf", 128, (1000, 700))])
def test_noalloc_matches_allocating_entry_point_twice(mode, part, sizes):
    import paper_1909_12533_gb300 as sp2
    first = _decaying(sizes[0], 1)
    second = _decaying(sizes[1], 2)     # a different size: stale scratch must not leak in
    if mode == "frobenius":
        assert first.nnzb > 2048 and second.nnzb > 2048
    for X, tau in ((first, 1e-3), (second, 1e-4)):
        ref = sp2.sp2_truncate(X, tau, mode, part)
        got = _noalloc(X, tau, mode, part)
        assert np.array_equal(got, ref)
        assert 0 < ref.sum() < X.nnzb
        assert np.array_equal(got, _oracle_keep(X, tau, mode, part))


def test_noalloc_rejects_oversized_input():
    import paper_1909_12533_gb300 as sp2
    lib = sp2.load()
    rc = lib.sp2_truncate_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 10**6,
                                  (1 << 18) + 1, 1e-6, 0, 4096, ctypes.c_void_p(16), None)
    assert rc == -11
    assert "scratch" in sp2.sp2_strerror(rc)
