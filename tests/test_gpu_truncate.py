"""Truncation step (Eq. (8)) through sp2_truncate against the oracle's selection:
bit-exact keep flags, including exact ties, tau = 0 and the two extremes."""
import numpy as np
import pytest

import oracle.sp2_oracle as O
from synth import BlockSparse, from_dense, to_dense

pytestmark = pytest.mark.gpu


def _decaying(n, seed, ties=False):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = 0.5 * (A + A.T)
    d = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    A *= np.exp(-d / 40.0)
    X = from_dense(A, keep_zero_tiles=True)
    if ties:
        # several tiles with bit-identical values (equal norms): the index decides
        off = np.nonzero(X.brow != X.bcol)[0]
        src = X.val[off[3]].copy()
        for k in off[5:40:3]:
            X.val[k] = src * 1e-3
        # rows and columns past n are padding and stay zero
        r0 = n - 32 * (X.nb - 1)
        X.val[X.bcol == X.nb - 1, :, r0:] = 0.0
        X.val[X.brow == X.nb - 1, r0:, :] = 0.0
    return X


def _oracle_keep(X, tau, mode, part):
    Xd = to_dense(X)
    pattern = set(zip(X.brow.tolist(), X.bcol.tolist()))
    _, kept, _ = O.truncate_select(Xd, tau, mode, part=part, pattern=pattern)
    ks = set(kept)
    return np.array([1 if (i, j) in ks else 0 for i, j in zip(X.brow.tolist(), X.bcol.tolist())], np.int32)


@pytest.mark.parametrize("mode,part", [("frobenius", 4096), ("frobinf", 64), ("frobinf", 128)])
@pytest.mark.parametrize("tau", [0.0, 1e-6, 1e-3, 0.1])
@pytest.mark.parametrize("ties", [False, True])
def test_keep_flags_bit_exact(mode, part, tau, ties):
    import paper_1909_12533_gb300 as sp2
    X = _decaying(331, 17, ties)      # 11 tile rows, ragged tail of 11
    g = sp2.sp2_truncate(X, tau, mode, part)
    o = _oracle_keep(X, tau, mode, part)
    assert np.array_equal(g, o), np.nonzero(g != o)


def test_zero_tiles_and_extremes():
    import paper_1909_12533_gb300 as sp2
    X = _decaying(200, 3)
    X.val[2] = 0.0
    X.val[7] = 0.0
    keep = sp2.sp2_truncate(X, 0.0, "frobenius")
    assert keep.sum() == X.nnzb - 2 and keep[2] == 0 and keep[7] == 0
    assert sp2.sp2_truncate(X, 1e6, "frobenius").sum() == 0          # everything fits
    assert sp2.sp2_truncate(X, 1e-300, "frobenius").sum() == X.nnzb - 2


def test_device_input_matches_host_input():
    import torch
    import paper_1909_12533_gb300 as sp2
    X = _decaying(480, 9)

    class T:
        n = X.n
        brow = torch.from_numpy(X.brow).cuda()
        bcol = torch.from_numpy(X.bcol).cuda()
        val = torch.from_numpy(X.val).cuda()

    kd = sp2.sp2_truncate(T, 1e-4, "frobinf", 128).cpu().numpy()
    kh = sp2.sp2_truncate(X, 1e-4, "frobinf", 128)
    assert np.array_equal(kd, kh)


@pytest.mark.parametrize("n", [2016, 2048, 2017])
@pytest.mark.parametrize("mode", ["frobenius", "frobinf"])
@pytest.mark.parametrize("tau", [0.0, 1e-4, 0.3])
def test_keep_flags_around_one_cta_limit(n, mode, tau):
    """2016 upper tiles (nb = 63) take the one-CTA select, 2080 (nb = 64, also
    with a ragged tail) the multi-launch passes; both match the oracle bit for bit."""
    import paper_1909_12533_gb300 as sp2
    X = _decaying(n, 5, ties=True)
    X.val[11] = 0.0
    g = sp2.sp2_truncate(X, tau, mode, 4096)
    o = _oracle_keep(X, tau, mode, 4096)
    assert np.array_equal(g, o), np.nonzero(g != o)


# ----------------------------------------------------------------- mixed norm (Section 3)
@pytest.mark.parametrize("part", [64, 128, 4096])
@pytest.mark.parametrize("tau", [0.0, 1e-6, 1e-3, 0.1])
@pytest.mark.parametrize("ties", [False, True])
def test_mixed_keep_flags_bit_exact(part, tau, ties):
    # the same integer block sums, bisection and power-step bound on both sides
    import paper_1909_12533_gb300 as sp2
    X = _decaying(331, 17, ties)
    g = sp2.sp2_truncate(X, tau, "mixed", part)
    o = _oracle_keep(X, tau, "mixed", part)
    assert np.array_equal(g, o), np.nonzero(g != o)


@pytest.mark.parametrize("n,part", [(2017, 256), (4000, 128)])
def test_mixed_keep_flags_larger_and_norm_bound(n, part):
    # dropped error: ||E||_2 <= ||E||_m <= tau (exact mixed norm by eigvalsh)
    import paper_1909_12533_gb300 as sp2
    X = _decaying(n, 6)
    tau = 1e-3
    g = sp2.sp2_truncate(X, tau, "mixed", part)
    o = _oracle_keep(X, tau, "mixed", part)
    assert np.array_equal(g, o), np.nonzero(g != o)
    Xd = to_dense(X)
    dropped = [(i, j) for i, j, k in zip(X.brow.tolist(), X.bcol.tolist(), g.tolist()) if not k]
    E = Xd - O.apply_drop(Xd, dropped)
    e = np.append(np.arange(0, n, part), n)
    k = len(e) - 1
    Bm = np.array([[np.linalg.norm(E[e[a]:e[a + 1], e[b]:e[b + 1]]) for b in range(k)] for a in range(k)])
    m = float(np.abs(np.linalg.eigvalsh(Bm)).max())
    assert 0 < len(dropped) and m <= tau * (1 + 1e-12)
