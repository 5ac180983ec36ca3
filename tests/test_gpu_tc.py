"""Tensor-core (tcgen05) FP16-slice path against the CPU oracle and the FP64 GPU
path.  Target tolerance of the mixed path: ||D - D_oracle||_F <= 1e-6 with four
slices; the two- and three-slice forms are measured and reported."""
import numpy as np
import pytest

from synth import dense_gapped, from_dense, make_config
from tests.helpers import run_gpu, run_oracle

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def _err(g, o):
    return float(np.linalg.norm(g["D"] - o.D))


@pytest.mark.parametrize("key", [1, "2s", "4s"])
def test_split16_k4_meets_tolerance(key):
    c = make_config(key)
    kw = dict(stop=c["stop"])
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], **kw)
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=4, **kw)
    err = _err(g, o)
    print(f"config {key}: split16 k=4 ||D-Dref||_F = {err:.3e}, n = {g['stats']['n']} (oracle {o.n})")
    assert g["stats"]["prec_hist"][0] == 1
    assert err <= MIXED_TOL
    assert abs(g["stats"]["n"] - o.n) <= 1
    n = g["D"].shape[0]
    assert abs(np.trace(g["D"]) - c["nocc"]) <= 1e-6 * max(1.0, np.sqrt(n))


def test_split16_first_square_matches_fp64_closely():
    # one step only: e_0, t_0 come from S = X~_0^2; slices on a 2^-43 grid.  The
    # tensor path sums ||X~ - S||^2 in FP64 like the FP64 path, so e and t differ
    # only by the products' rounding: |e_a - e_b| <= ||S_a - S_b||_F, each
    # element within ~2^-44 (5.9M elements: < 1e-9 in norm)
    c = make_config("2s")
    a = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], n_max_cap=1)
    b = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], n_max_cap=1, precision="split16", slices=4)
    ea, eb = a["stats"]["e"], b["stats"]["e"]
    # each element of S carries the slicing of ~1000 products (~1e-12), so
    # |e_a - e_b| <= ||S_a - S_b||_F ~ 1e-9 on 5.9M elements (measured 1.4e-9 on
    # e_0 = 11.9, 1.2e-10 relative)
    np.testing.assert_allclose(eb, ea, rtol=1e-9)
    np.testing.assert_allclose(b["stats"]["t"], a["stats"]["t"], rtol=1e-9)
    # 5.9M elements, each within ~1e-12 (2^-44 grid, FP32-exact groups)
    assert np.linalg.norm(a["D"] - b["D"]) < 1e-8


def test_split16_precision_form_config3_analogue():
    # the precision form of the water-like recipe (203 molecules, tau = 1e-5):
    # the tensor path against the oracle at the mixed-path tolerance
    c = make_config("3s")
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=4)
    err = _err(g, o)
    print(f"3s split16: ||D-Dref||_F = {err:.3e}, n = {g['stats']['n']} (oracle {o.n})")
    assert g["code"] == 0 and err <= MIXED_TOL
    assert abs(g["stats"]["n"] - o.n) <= 1


@pytest.mark.parametrize("mixed_from", [1, 8])
def test_split16_narrow_gap_dense_segmented_accumulation(mixed_from):
    # dense N = 1000 with gap 0.05 (the narrow-gap recipe at oracle size);
    # acc_flush_min = 1 cuts every K loop into 16-tile segments, so the
    # per-segment TMEM release and exact fixed-point segment sums run here
    c = make_config("5s")
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision="split16",
                slices=4, acc_flush_min=1, mixed_from=mixed_from)
    g0 = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision="split16",
                 slices=4, acc_flush_min=0, mixed_from=mixed_from)
    err, err0 = _err(g, o), _err(g0, o)
    print(f"5s split16 mixed_from={mixed_from}: segmented {err:.3e}, unsegmented {err0:.3e} (oracle n = {o.n})")
    assert g["code"] == 0 and g["stats"]["converged"]
    assert err <= MIXED_TOL and err0 <= MIXED_TOL


@pytest.mark.parametrize("k", [2, 3])
def test_split16_fewer_slices_reported(k):
    c = make_config("2s")
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=k)
    err = _err(g, o)
    print(f"split16 k={k}: ||D-Dref||_F = {err:.3e}")
    assert np.isfinite(err) and err < 1.0


@pytest.mark.parametrize("n", [33, 100, 129, 300])
def test_split16_ragged_sizes(n):
    d = dense_gapped(n, n // 3, (-2.0, -0.3), (0.4, 2.0), seed=100 + n)
    o = run_oracle(d["F"], d["nocc"], d["homo_ub"], d["lumo_lb"], 0.0, stop="idempotency", idem_tol=1e-11)
    g = run_gpu(d["F"], d["nocc"], d["homo_ub"], d["lumo_lb"], 0.0, stop="idempotency", idem_tol=1e-11,
                precision="split16", slices=4)
    err = _err(g, o)
    assert err <= MIXED_TOL, err


def test_split16_then_fp64_schedule():
    # mixed precision schedule: tensor cores up to iteration 8, FP64 afterwards
    c = make_config("2s")
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=4,
                mixed_until=8)
    ph = g["stats"]["prec_hist"]
    assert ph[0] == 1 and ph[-1] == 0
    assert _err(g, o) <= MIXED_TOL


def test_split16_block_diagonal_sparse_supertiles():
    a = dense_gapped(200, 90, (-1.0, -0.4), (0.4, 1.0), seed=5)["F"]
    b = dense_gapped(190, 80, (-1.0, -0.4), (0.4, 1.0), seed=6)["F"]
    F = np.zeros((390, 390))
    F[:200, :200] = a
    F[200:, 200:] = b
    Fb = from_dense(F)
    o = run_oracle(Fb, 170, -0.4, 0.4, 0.0, stop="idempotency")
    g = run_gpu(Fb, 170, -0.4, 0.4, 0.0, stop="idempotency", precision="split16", slices=4)
    assert _err(g, o) <= MIXED_TOL
    assert list(zip(g["brow"].tolist(), g["bcol"].tolist())) == sorted(o.kept[o.n])


def test_split16_fp64_tail_reaches_idempotency_tolerance():
    # dense N = 512, idempotency stop at 1e-12: the tensor path alone stalls near
    # its rounding floor; the final steps in FP64 reach the tolerance
    c = make_config(1)
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"])
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision="split16",
                slices=4)
    st = g["stats"]
    assert g["code"] == 0 and st["converged"]
    assert st["e"][st["n"]] < 1e-12
    ph = st["prec_hist"]
    assert ph[0] == 1 and ph[-1] == 0 and sorted(ph, reverse=True) == ph   # tensor cores first, FP64 tail
    assert _err(g, o) <= MIXED_TOL
    # fp64_tail = 0: every square on the tensor cores
    g0 = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], stop=c["stop"], precision="split16",
                 slices=4, fp64_tail=0.0, n_max_cap=20)
    assert all(p == 1 for p in g0["stats"]["prec_hist"])


@pytest.mark.parametrize("key,extra", [(1, {}), ("2s", {}), ("3s", {}), ("4s", {}),
                                       ("5s", {"acc_flush_min": 1}), ("2s", {"storage": "general"})])
def test_split_supply_gives_the_same_result(key, extra):
    # the B slices through the copy warps (cp.async) instead of bulk copies: the
    # same bytes land in the same stages, so D is the same bit for bit
    c = make_config(key)
    kw = dict(stop=c["stop"], precision="split16", slices=4, **extra)
    a = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], split_supply=0, **kw)
    b = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], split_supply=1, **kw)
    assert a["code"] == 0 and b["code"] == 0
    assert a["stats"]["n"] == b["stats"]["n"]
    assert np.array_equal(a["brow"], b["brow"]) and np.array_equal(a["val"], b["val"])
    assert a["stats"]["e"] == b["stats"]["e"]


@pytest.mark.parametrize("key,idem_tol,tol", [(1, 1e-10, 1e-8), ("5s", 1e-10, 1e-8), ("2s", None, 1e-9),
                                               ("4s", None, 1e-9)])
def test_split16_five_slices_fp64_grade_without_fp64_squares(key, idem_tol, tol):
    # five 10-bit FP16 slices (finest grid 2^-49) in two launches per square,
    # the diagonal of S in FP64: every square on the tensor cores
    # (fp64_tail = 0).  The idempotency floor of the tensor path on dense rows is
    # ~1e-11 (N = 512), so the dense cases stop at 1e-10 on both sides
    c = make_config(key)
    kw = dict(stop=c["stop"])
    if idem_tol is not None:
        kw["idem_tol"] = idem_tol
    o = run_oracle(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], **kw)
    g = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=5,
                fp64_tail=0.0, **kw)
    err = _err(g, o)
    print(f"config {key}: split16 k=5 ||D-Dref||_F = {err:.3e}, n = {g['stats']['n']} (oracle {o.n})")
    assert g["code"] == 0 and g["stats"]["converged"]
    assert all(p == 1 for p in g["stats"]["prec_hist"])
    assert err <= tol
    assert abs(g["stats"]["n"] - o.n) <= 1


def test_split16_diagonal_of_the_square_in_fp64():
    # the first square of the dense 512 case: the diagonal of S comes from the
    # FP64 row norms, so with five slices S agrees with the FP64 square to
    # ~1e-13 per element (four slices: the 2^-44 slicing, ~2e-11)
    c = make_config(1)
    base = dict(stop=c["stop"], n_max_cap=1)
    a = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], **base)
    for k, tol in ((4, 1e-10), (5, 1e-12)):
        b = run_gpu(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], c["tau"], precision="split16", slices=k,
                    fp64_tail=0.0, **base)
        d = float(np.abs(b["D"] - a["D"]).max())
        print(f"dense 512, first square, {k} slices: max |X_1 - X_1(FP64)| = {d:.3e}")
        assert d <= tol
