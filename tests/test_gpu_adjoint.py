"""Adjoint (sp2_backward) against the oracle's reverse sweep, central finite
differences through the CUDA forward, and the Daleckii-Krein closed form;
torch.autograd.Function wiring.  Target: 1e-5 relative against finite
differences."""
import numpy as np
import pytest

import oracle.sp2_oracle as O
from synth import BlockSparse, dense_gapped, from_dense, make_config, random_symmetric_on_pattern, to_dense

pytestmark = pytest.mark.gpu


def _sym(rng, n):
    a = rng.standard_normal((n, n))
    return 0.5 * (a + a.T)


def _gpu_grad(Fb, nocc, hub, llb, tau, Wd, **kw):
    import paper_1909_12533_gb300 as sp2
    W = from_dense(Wd, keep_zero_tiles=True)
    ctx = sp2.SP2(Fb, nocc, hub, llb, tau, record_masks=1, **kw)
    st = ctx.run()
    brow, bcol, val = ctx.backward(W)
    ctx.close()
    dF = BlockSparse(n=Fb.n, brow=brow.cpu().numpy(), bcol=bcol.cpu().numpy(), val=val.cpu().numpy())
    return dF, st


def _dense_grad(dF):
    """General-matrix gradient (F_ij and F_ji independent) as a dense array."""
    b = dF.b
    G = np.zeros((dF.nb * b, dF.nb * b))
    for k in range(dF.nnzb):
        i, j = int(dF.brow[k]), int(dF.bcol[k])
        G[i * b:(i + 1) * b, j * b:(j + 1) * b] = dF.val[k]
        if i != j:
            G[j * b:(j + 1) * b, i * b:(i + 1) * b] = dF.val[k].T
    return G[: dF.n, : dF.n]


def _loss_gpu(Fd, nocc, hub, llb, tau, Wd, **kw):
    import paper_1909_12533_gb300 as sp2
    ctx = sp2.SP2(from_dense(Fd), nocc, hub, llb, tau, **kw)
    st = ctx.run()
    brow, bcol, val = ctx.D_host()
    ctx.close()
    D = to_dense(BlockSparse(n=Fd.shape[0], brow=brow, bcol=bcol, val=val))
    return float(np.sum(D * Wd)), st


@pytest.mark.parametrize("n,nocc", [(48, 20), (100, 41)])
def test_adjoint_matches_oracle_dense(n, nocc):
    d = dense_gapped(n, nocc, (-1.5, -0.4), (0.4, 1.5), seed=50 + n)
    W = _sym(np.random.default_rng(n), n)
    dF, st = _gpu_grad(from_dense(d["F"]), nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, stop="idempotency")
    r = O.sp2(d["F"], nocc, d["homo_ub"], d["lumo_lb"], tau=0.0, stop="idempotency")
    G = O.adjoint_sp2(d["F"], r, W)
    Gg = _dense_grad(dF)
    assert st["n"] == r.n
    assert np.linalg.norm(Gg - G) <= 1e-10 * np.linalg.norm(G)


def test_adjoint_central_finite_differences():
    n, nocc = 64, 25
    d = dense_gapped(n, nocc, (-1.5, -0.4), (0.4, 1.5), seed=77)
    W = _sym(np.random.default_rng(3), n)
    kw = dict(stop="idempotency")
    dF, _ = _gpu_grad(from_dense(d["F"]), nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
    G = _dense_grad(dF)
    F = d["F"]
    h = 1e-5
    for (i, j) in [(0, 0), (5, 9), (17, 60), (63, 63), (31, 32)]:
        Fp = F.copy(); Fm = F.copy()
        Fp[i, j] += h; Fm[i, j] -= h
        if i != j:
            Fp[j, i] += h; Fm[j, i] -= h
        Lp, sp = _loss_gpu(Fp, nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
        Lm, sm = _loss_gpu(Fm, nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
        fd = (Lp - Lm) / (2 * h)
        an = G[i, j] + (G[j, i] if i != j else 0.0)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (i, j, fd, an)


def test_adjoint_daleckii_krein():
    n, nocc = 80, 33
    d = dense_gapped(n, nocc, (-1.5, -0.5), (0.5, 1.5), seed=91)
    W = _sym(np.random.default_rng(5), n)
    dF, _ = _gpu_grad(from_dense(d["F"]), nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, stop="idempotency")
    G = _dense_grad(dF)
    lam, V = np.linalg.eigh(d["F"])
    Wt = V.T @ W @ V
    Gt = np.zeros_like(Wt)
    for i in range(nocc):
        for a in range(nocc, n):
            Gt[i, a] = Gt[a, i] = Wt[i, a] / (lam[i] - lam[a])
    ref = V @ Gt @ V.T
    assert np.linalg.norm(G - ref) <= 1e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("ckpt", [1, 3, 8])
def test_adjoint_truncated_helix_prefix_matches_oracle(ckpt):
    # the 64-residue prefix of the helix workload (N = 4096), tau = 1e-6,
    # W with F's tile pattern; checkpoint interval varied
    c = make_config("4s")
    Fb = c["F"]
    Wb = random_symmetric_on_pattern(Fb, seed=4)
    Wd = to_dense(Wb)
    import paper_1909_12533_gb300 as sp2
    ctx = sp2.SP2(Fb, c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], ckpt_every=ckpt, record_masks=1)
    st = ctx.run()
    brow, bcol, val = ctx.backward(Wb)
    ctx.close()
    dF = BlockSparse(n=Fb.n, brow=brow.cpu().numpy(), bcol=bcol.cpu().numpy(), val=val.cpu().numpy())
    Fd = to_dense(Fb)
    r = O.sp2(Fd, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"],
              input_pattern=set(zip(Fb.brow.tolist(), Fb.bcol.tolist())))
    assert st["nnzb_hist"][: r.n + 1] == [len(k) for k in r.kept[: r.n + 1]]
    mask = np.zeros_like(Fd)
    for i, j in zip(Fb.brow.tolist(), Fb.bcol.tolist()):
        mask[i * 32:(i + 1) * 32, j * 32:(j + 1) * 32] = 1
        mask[j * 32:(j + 1) * 32, i * 32:(i + 1) * 32] = 1
    G = O.adjoint_sp2(Fd, r, Wd) * mask
    Gg = _dense_grad(dF)
    assert np.linalg.norm(Gg - G) <= 1e-9 * np.linalg.norm(G)


def test_autograd_function():
    import torch
    import paper_1909_12533_gb300 as sp2
    n, nocc = 70, 30
    d = dense_gapped(n, nocc, (-1.5, -0.4), (0.4, 1.5), seed=13)
    Fb = from_dense(d["F"])
    Fv = torch.from_numpy(Fb.val).cuda().requires_grad_(True)
    br = torch.from_numpy(Fb.brow).cuda()
    bc = torch.from_numpy(Fb.bcol).cuda()
    Fn = sp2.SP2Function
    Dv, Db, Dc = Fn.apply(Fv, br, bc, n, nocc, d["homo_ub"], d["lumo_lb"], 0.0, {"stop": "idempotency"})
    # SP2Function records the masks itself
    # L = sum of stored D tiles weighted by a random tensor
    R = torch.randn(Dv.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    L = (Dv * R).sum()
    L.backward()
    g = Fv.grad.cpu().numpy()
    # finite differences on a few stored entries (symmetric perturbation for
    # off-diagonal tiles: the stored tile stands for both F_IJ and F_JI)
    def loss(Fval):
        Fc = BlockSparse(n=n, brow=Fb.brow, bcol=Fb.bcol, val=Fval)
        ctx = sp2.SP2(Fc, nocc, d["homo_ub"], d["lumo_lb"], 0.0, stop="idempotency")
        ctx.run()
        _, _, dv = ctx.D_device()
        ctx.close()
        return float((dv * R).sum())
    h = 1e-6
    for (t, r_, c_) in [(0, 3, 7), (1, 10, 2), (2, 31, 31)]:
        vp = Fb.val.copy(); vm = Fb.val.copy()
        vp[t, r_, c_] += h; vm[t, r_, c_] -= h
        if Fb.brow[t] == Fb.bcol[t] and r_ != c_:
            vp[t, c_, r_] += h; vm[t, c_, r_] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        an = g[t, r_, c_] + (g[t, c_, r_] if (Fb.brow[t] == Fb.bcol[t] and r_ != c_) else 0.0)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (t, r_, c_, fd, an)


def test_adjoint_split16_matches_oracle_helix_prefix():
    # tensor-core adjoint (G sliced with a power-of-two scale, two-pass G X + X G)
    c = make_config("4s")
    Fb = c["F"]
    Wb = random_symmetric_on_pattern(Fb, seed=4)
    import paper_1909_12533_gb300 as sp2
    ctx = sp2.SP2(Fb, c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=4,
                  record_masks=1)
    st = ctx.run()
    brow, bcol, val = ctx.backward(Wb)
    bms = sp2.stats_dict(sp2.sp2_get_stats(ctx.ctx))["backward_ms"]
    ctx.close()
    dF = BlockSparse(n=Fb.n, brow=brow.cpu().numpy(), bcol=bcol.cpu().numpy(), val=val.cpu().numpy())
    Fd = to_dense(Fb)
    r = O.sp2(Fd, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"],
              input_pattern=set(zip(Fb.brow.tolist(), Fb.bcol.tolist())))
    mask = np.zeros_like(Fd)
    for i, j in zip(Fb.brow.tolist(), Fb.bcol.tolist()):
        mask[i * 32:(i + 1) * 32, j * 32:(j + 1) * 32] = 1
        mask[j * 32:(j + 1) * 32, i * 32:(i + 1) * 32] = 1
    G = O.adjoint_sp2(Fd, r, to_dense(Wb)) * mask
    rel = np.linalg.norm(_dense_grad(dF) - G) / np.linalg.norm(G)
    print(f"split16 adjoint rel err {rel:.2e}, backward {bms:.1f} ms")
    assert st["n"] == r.n
    assert rel <= 1e-6


def test_adjoint_split16_central_finite_differences():
    n, nocc = 64, 25
    d = dense_gapped(n, nocc, (-1.5, -0.4), (0.4, 1.5), seed=78)
    W = _sym(np.random.default_rng(7), n)
    kw = dict(stop="idempotency", idem_tol=1e-11, precision="split16", slices=4)
    dF, _ = _gpu_grad(from_dense(d["F"]), nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
    G = _dense_grad(dF)
    F = d["F"]
    h = 1e-5
    for (i, j) in [(0, 0), (5, 9), (40, 41), (63, 63)]:
        Fp = F.copy(); Fm = F.copy()
        Fp[i, j] += h; Fm[i, j] -= h
        if i != j:
            Fp[j, i] += h; Fm[j, i] -= h
        Lp, _ = _loss_gpu(Fp, nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
        Lm, _ = _loss_gpu(Fm, nocc, d["homo_ub"], d["lumo_lb"], 0.0, W, **kw)
        fd = (Lp - Lm) / (2 * h)
        an = G[i, j] + (G[j, i] if i != j else 0.0)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (i, j, fd, an)


def test_autograd_function_second_backward_and_not_converged():
    # the context stays open until the autograd node is freed: a second
    # backward (retain_graph) runs the same recorded sweep; a forward that ends
    # at n_max without the stop test raises unless allow_not_converged is set
    import torch
    import paper_1909_12533_gb300 as sp2
    n, nocc = 70, 30
    d = dense_gapped(n, nocc, (-1.5, -0.4), (0.4, 1.5), seed=13)
    Fb = from_dense(d["F"])
    Fv = torch.from_numpy(Fb.val).cuda().requires_grad_(True)
    br = torch.from_numpy(Fb.brow).cuda()
    bc = torch.from_numpy(Fb.bcol).cuda()
    Fn = sp2.SP2Function
    Dv, _, _ = Fn.apply(Fv, br, bc, n, nocc, d["homo_ub"], d["lumo_lb"], 0.0, {"stop": "idempotency"})
    R = torch.randn(Dv.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    L = (Dv * R).sum()
    L.backward(retain_graph=True)
    g1 = Fv.grad.clone()
    Fv.grad = None
    L.backward()
    assert torch.equal(Fv.grad, g1)
    with pytest.raises(sp2.SP2Error) as e:
        Fn.apply(Fv, br, bc, n, nocc, d["homo_ub"], d["lumo_lb"], 0.0, {"stop": "idempotency", "n_max_cap": 3})
    assert e.value.code == -7
    Dv3, _, _ = Fn.apply(Fv, br, bc, n, nocc, d["homo_ub"], d["lumo_lb"], 0.0,
                         {"stop": "idempotency", "n_max_cap": 3, "allow_not_converged": True})
    assert torch.isfinite(Dv3).all()
