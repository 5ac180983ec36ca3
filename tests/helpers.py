"""Shared helpers of the parity tests: run the CUDA path through the C ABI and
the CPU oracle on the same seeded input and compare."""
from __future__ import annotations

import numpy as np

from synth import BlockSparse, from_dense, to_dense


def as_blocks(F) -> BlockSparse:
    return F if isinstance(F, BlockSparse) else from_dense(F)


def run_gpu(F, nocc, homo_ub, lumo_lb, tau, **params):
    import paper_1909_12533_gb300 as sp2
    Fb = as_blocks(F)
    ctx = sp2.SP2(Fb, nocc, homo_ub, lumo_lb, tau, **params)
    try:
        st = ctx.run()
        brow, bcol, val = ctx.D_host()
    finally:
        ctx.close()
    D = to_dense(BlockSparse(n=Fb.n, brow=brow, bcol=bcol, val=val))
    return dict(stats=st, code=ctx.code, D=D, brow=brow, bcol=bcol, val=val, Fb=Fb)


def run_oracle(F, nocc, homo_ub, lumo_lb, tau, mode="sp2acc", stop="parameterless", idem_tol=1e-12,
               trunc="frobenius", frobinf_part=4096, gamma=0.0, n_max_cap=100, **_):
    import oracle.sp2_oracle as O
    Fb = as_blocks(F)
    Fd = to_dense(Fb)
    pattern = set(zip(Fb.brow.tolist(), Fb.bcol.tolist()))
    return O.sp2(Fd, nocc, homo_ub, lumo_lb, tau=tau, gamma=gamma if gamma > 0 else None,
                 accelerate=(mode == "sp2acc"), stop=stop, idem_tol=idem_tol, trunc=trunc,
                 frobinf_part=frobinf_part, n_cap=n_max_cap, input_pattern=pattern)


def compare(g, o, d_tol=1e-10):
    """Assert GPU result g == oracle result o within the FP64 tolerance."""
    st = g["stats"]
    sch = o.sched
    assert abs(st["lmin"] - o.lmin) <= 1e-12 * abs(o.lmin) + 1e-14
    assert abs(st["lmax"] - o.lmax) <= 1e-12 * abs(o.lmax) + 1e-14
    assert st["n_max"] == sch.n_max and st["n_min"] == sch.n_min
    assert st["p"][1:] == sch.p[1:]
    np.testing.assert_allclose(st["alpha"][1:], sch.alpha[1:], rtol=1e-14)
    assert st["n"] == o.n, (st["n"], o.n)
    # the numerator of every FLOP/s figure: (I <= J, K) tile triplets over all squares
    assert st["tile_triplets"] == o.tile_triplets, (st["tile_triplets"], o.tile_triplets)
    assert st["squares"] == o.squares
    assert bool(st["converged"]) == o.converged
    ne = len(o.e)
    assert len(st["e"]) == ne
    np.testing.assert_allclose(st["e"], o.e, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(st["t"], o.t, rtol=1e-8, atol=1e-11)
    # integer work bit-exact: the tile pattern of every X~_j and of D
    assert st["nnzb_hist"][: o.n + 1] == [len(k) for k in o.kept[: o.n + 1]]
    kept = sorted(o.kept[o.n])
    assert list(zip(g["brow"].tolist(), g["bcol"].tolist())) == kept
    err = np.linalg.norm(g["D"] - o.D)
    assert err <= d_tol, err
    return err
