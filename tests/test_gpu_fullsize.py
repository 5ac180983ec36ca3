"""Water-like N = 24000 (1000 molecules, tau = 1e-6), in the launch
configuration bench.py times.  The oracle does not finish this size in
seconds, so the checks are properties that hold at any size (symmetric
storage, trace, idempotency error, D F = F D on sampled tile rows) and the
four-slice tensor-core path against the FP64 path, which is itself compared
element by element with the oracle at smaller sizes."""
import numpy as np
import pytest

from synth import BlockSparse, make_config, to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def water24k():
    import paper_1909_12533_gb300 as sp2
    c = make_config(2)
    out = {}
    for prec in ("split16", "fp64"):
        ctx = sp2.SP2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"],
                      precision=prec, slices=4)
        st = ctx.run()
        out[prec] = (st, ctx.D_host(), ctx.code)
        ctx.close()
    return c, out


@pytest.mark.parametrize("prec", ["split16", "fp64"])
def test_water24k_properties(water24k, prec):
    c, out = water24k
    st, (brow, bcol, val), code = out[prec]
    F = c["F"]
    n, nb = F.n, F.nb
    assert code == 0 and st["converged"]
    assert np.all(brow <= bcol)
    assert np.all(np.diff(brow.astype(np.int64) * nb + bcol) > 0)
    diag = brow == bcol
    np.testing.assert_allclose(val[diag], val[diag].transpose(0, 2, 1), atol=1e-12)
    # padding rows/columns of the last tile row stay zero
    last = np.nonzero(bcol == nb - 1)[0]
    assert not np.any(val[last][:, :, n - (nb - 1) * 32:])
    e_n = st["e"][-1]
    assert e_n < 1e-5
    tr = float(sum(np.trace(v) for v in val[diag]))
    assert abs(tr - c["nocc"]) <= np.sqrt(n) * e_n + 1e-6
    # D commutes with F: compare (D F) and (F D) on six sampled tile rows;
    # the oracle at 101 molecules and the same tau gives 2.4e-7 per row
    Dd = to_dense(BlockSparse(n, brow, bcol, val))
    Fd = to_dense(F)
    rows = np.sort(np.random.default_rng(0).choice(nb, 6, replace=False))
    idx = np.concatenate([np.arange(I * 32, min((I + 1) * 32, n)) for I in rows])
    C = Dd[idx] @ Fd - Fd[idx] @ Dd
    rel = np.linalg.norm(C) / np.linalg.norm(Fd[idx])
    print(f"water N=24000 {prec}: n = {st['n']}, e_n = {e_n:.2e}, trace - nocc = {tr - c['nocc']:.2e}, "
          f"row ||DF-FD|| / ||F|| = {rel:.2e}")
    assert rel < 1e-5


def test_water24k_mixed_matches_fp64(water24k):
    c, out = water24k
    (s1, D1, _), (s2, D2, _) = out["split16"], out["fp64"]
    assert s1["n"] == s2["n"]
    k1 = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(D1[0], D1[1]))}
    k2 = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(D2[0], D2[1]))}
    tot = 0.0
    for key in set(k1) | set(k2):
        w = 1.0 if key[0] == key[1] else 2.0
        a = D1[2][k1[key]] if key in k1 else 0.0
        b = D2[2][k2[key]] if key in k2 else 0.0
        tot += w * float(np.sum((np.asarray(a) - b) ** 2))
    err = np.sqrt(tot)
    print(f"water N=24000: ||D_split16 - D_fp64||_F = {err:.3e}")
    assert err <= 1e-6


# ----------------------------------------------------------------- the headline size: N = 192000, tau = 1e-5
def _symv(brow, bcol, val, v):
    """y = A v for the symmetric matrix whose upper tiles are given (torch, on
    the device): every stored tile (I, J) adds A_IJ v_J to y_I and, off the
    diagonal, A_IJ^T v_I to y_J.  v: [nb * 32, m]."""
    import torch
    nb = v.shape[0] // 32
    V = v.view(nb, 32, -1)
    Y = torch.zeros_like(V)
    I, J = brow.long(), bcol.long()
    for lo in range(0, brow.numel(), 1 << 18):     # chunks keep the temporaries small
        sl = slice(lo, lo + (1 << 18))
        t = val[sl]
        Y.index_add_(0, I[sl], torch.bmm(t, V[J[sl]]))
        off = I[sl] != J[sl]
        Y.index_add_(0, J[sl][off], torch.bmm(t[off].transpose(1, 2), V[I[sl][off]]))
    return Y.view(nb * 32, -1)


def test_water192k_properties_on_the_tensor_path():
    # the bench's workload and path (four FP16 slices): idempotency and D F = F D
    # checked with block-sparse products on random vectors, trace against nocc,
    # symmetric diagonal tiles; the FP64 comparison at this size is in bench.py
    import torch
    import paper_1909_12533_gb300 as sp2
    c = make_config(3)
    F = c["F"]
    n, nb = F.n, F.nb
    ctx = sp2.SP2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision="split16")
    st = ctx.run()
    brow, bcol, val = ctx.D_device()
    ctx.close()
    assert ctx.code == 0 and st["converged"]
    assert bool((brow <= bcol).all())
    diag = brow == bcol
    assert float((val[diag] - val[diag].transpose(1, 2)).abs().max()) <= 1e-12
    tr = float(val[diag].diagonal(dim1=1, dim2=2).sum())
    e_n = st["e"][-1]
    assert abs(tr - c["nocc"]) <= np.sqrt(n) * e_n + 1e-6
    g = torch.Generator("cuda").manual_seed(3)
    v = torch.randn(nb * 32, 4, dtype=torch.float64, device="cuda", generator=g)
    v[n:] = 0.0
    Fb = torch.from_numpy(F.brow).cuda()
    Fc = torch.from_numpy(F.bcol).cuda()
    Fv = torch.from_numpy(F.val).cuda()
    Dv = _symv(brow, bcol, val, v)
    DDv = _symv(brow, bcol, val, Dv)
    idem = float((DDv - Dv).norm() / v.norm())
    comm = float((_symv(brow, bcol, val, _symv(Fb, Fc, Fv, v)) - _symv(Fb, Fc, Fv, Dv)).norm()
                 / _symv(Fb, Fc, Fv, v).norm())
    print(f"water N=192000 split16: n = {st['n']}, e_n = {e_n:.2e}, trace - nocc = {tr - c['nocc']:.2e}, "
          f"||D^2 v - D v|| / ||v|| = {idem:.2e}, ||DFv - FDv|| / ||Fv|| = {comm:.2e}")
    # a random unit vector sees ||D^2 - D||_F / sqrt(N) of the idempotency error
    assert idem <= 10 * e_n / np.sqrt(n) * np.sqrt(4) + 1e-9
    assert comm < 1e-5
