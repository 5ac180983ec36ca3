"""Pins of the CPU oracle against things other than itself: eigendecompositions,
closed forms, brute force, the paper's error bound and the values it prints.
All run on the CPU in a few seconds each."""
import itertools
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle.sp2_oracle as O
from synth import dense_gapped, make_config, to_dense

GOLDEN = json.loads((Path(__file__).parent / "golden" / "paper_values.json").read_text())


def _sym(rng, n):
    a = rng.standard_normal((n, n))
    return 0.5 * (a + a.T)


# ----------------------------------------------------------------- paper constants
def test_paper_constants():
    assert O.C_STOP == GOLDEN["stop_constant_C"]["value"]
    assert O.B == GOLDEN["small_block_size"]["value"]
    assert O.FROBINF_PART == GOLDEN["leaf_and_frobinf_block_size"]["value"]


# ----------------------------------------------------------------- Eq. (3)
def test_eig_projector_closed_form_on_diagonal():
    lam = np.array([3.0, -1.0, 0.5, -2.0, 1.5])
    D = O.eig_projector(np.diag(lam), 2)
    np.testing.assert_allclose(D, np.diag([0, 1, 0, 1, 0.0]), atol=1e-15)


def test_eig_projector_invariants():
    rng = np.random.default_rng(1)
    F = _sym(rng, 60)
    D = O.eig_projector(F, 23)
    assert abs(np.trace(D) - 23) < 1e-12
    assert np.linalg.norm(D @ D - D) < 1e-12
    assert np.linalg.norm(D @ F - F @ D) < 1e-12
    np.testing.assert_allclose(D, D.T, atol=1e-15)


# ----------------------------------------------------------------- Algorithm 1
def test_gershgorin_contains_spectrum_and_closed_forms():
    rng = np.random.default_rng(2)
    F = _sym(rng, 40)
    lo, hi = O.gershgorin_bounds(F)
    ev = np.linalg.eigvalsh(F)
    assert lo <= ev[0] and ev[-1] <= hi
    # diagonal matrix: the discs are points
    assert O.gershgorin_bounds(np.diag([2.0, -3.0, 1.0])) == (-3.0, 2.0)
    # 2x2 [[a, b], [b, c]]: discs [a-|b|, a+|b|], [c-|b|, c+|b|]
    lo, hi = O.gershgorin_bounds(np.array([[1.0, -0.25], [-0.25, 3.0]]))
    assert (lo, hi) == (0.75, 3.25)


def test_initial_matrix_maps_spectrum_to_unit_interval_reversed():
    rng = np.random.default_rng(3)
    F = _sym(rng, 30)
    lo, hi = O.gershgorin_bounds(F)
    X = O.initial_matrix(F, lo, hi)
    ev_f = np.linalg.eigvalsh(F)
    ev_x = np.linalg.eigvalsh(X)
    np.testing.assert_allclose(np.sort((hi - ev_f) / (hi - lo)), ev_x, atol=1e-13)
    assert ev_x[0] >= -1e-14 and ev_x[-1] <= 1 + 1e-14
    assert np.linalg.norm(X @ F - F @ X) < 1e-12


# ----------------------------------------------------------------- Algorithm 2 polynomials
@pytest.mark.parametrize("p,alpha", [(1, 1.0), (1, 1.37), (0, 1.0), (0, 1.61)])
def test_polynomial_coefficients_match_matrix_definition(p, alpha):
    rng = np.random.default_rng(4)
    X = _sym(rng, 12) * 0.1 + 0.5 * np.eye(12)
    n = X.shape[0]
    if p == 1:
        Y = (1 - alpha) * np.eye(n) + alpha * X
        want = Y @ Y
    else:
        want = 2 * alpha * X - (alpha * X) @ (alpha * X)
    c0, c1, c2 = O.poly_coeffs(p, alpha)
    np.testing.assert_allclose(c0 * np.eye(n) + c1 * X + c2 * (X @ X), want, atol=1e-14)


# ----------------------------------------------------------------- Step 1 schedule
def test_scale_and_fold_symmetry_closed_form():
    # tau = 0: first step folds [0, l] onto itself: f(0) == f(l) = (l/(2-l))^2 and
    # the occupied bound maps to ((2h - l)/(2 - l))^2
    l, h = 0.3, 0.8   # d0 = 0.3 > d1 = 0.2 -> p = 1
    s = O.schedule(0.0, 1.0, 1.0 - h, 1.0 - l, tau=0.0)
    assert s.p[1] == 1
    a = s.alpha[1]
    assert abs(a - 2.0 / (2.0 - l)) < 1e-15
    f = lambda x: ((1 - a) + a * x) ** 2
    assert abs(f(0.0) - f(l)) < 1e-15
    assert abs(s.vhi[1] - (l / (2 - l)) ** 2) < 1e-15
    assert abs(s.olo[1] - ((2 * h - l) / (2 - l)) ** 2) < 1e-15
    # mirror case p = 0: 1 - h' = (d1/(2 - d1))^2
    l, h = 0.1, 0.6
    s = O.schedule(0.0, 1.0, 1.0 - h, 1.0 - l, tau=0.0)
    assert s.p[1] == 0
    d1 = 1 - h
    assert abs(s.alpha[1] - 2.0 / (2.0 - d1)) < 1e-15
    assert abs((1 - s.olo[1]) - (d1 / (2 - d1)) ** 2) < 1e-15


@pytest.mark.parametrize("accelerate", [True, False])
def test_schedule_bounds_contain_exact_eigenvalue_images(accelerate):
    d = dense_gapped(80, 30, (-2.0, -0.4), (0.3, 2.5), seed=21)
    F = d["F"]
    r = O.sp2(F, d["nocc"], d["homo_ub"], d["lumo_lb"], tau=0.0, stop="idempotency", accelerate=accelerate)
    s = r.sched
    # exact iterates: eigenvalues of X~_i must sit inside the propagated intervals
    X = O.initial_matrix(F, r.lmin, r.lmax)
    for i in range(0, r.n + 1):
        if i >= 1:
            c0, c1, c2 = O.poly_coeffs(s.p[i], s.alpha[i])
            X = c0 * np.eye(80) + c1 * X + c2 * (X @ X)
        ev = np.linalg.eigvalsh(X)
        virt, occ = ev[: 80 - 30], ev[80 - 30:]
        assert virt.max() <= s.vhi[i] + 1e-12, (i, virt.max(), s.vhi[i])
        assert occ.min() >= s.olo[i] - 1e-12, (i, occ.min(), s.olo[i])
    if not accelerate:
        assert s.n_min == 1 and all(a == 1.0 for a in s.alpha[1:])


def test_gamma_mode_tau_satisfies_error_bound_with_equality():
    # Eq. (7): tau_i/(xi_i - tau_i) = gamma/(n_max+1) for every i, so the sum over
    # i = 0..n_max of the bound in Eq. (5) equals gamma
    gamma = 1e-3
    s = O.schedule(-2.0, 3.0, -0.4, 0.4, gamma=gamma)
    terms = [t / (x - t) for t, x in zip(s.tau, s.xi)]
    assert len(terms) == s.n_max + 1
    assert abs(sum(terms) - gamma) < 1e-15


# ----------------------------------------------------------------- truncation
def _E(X, dropped):
    return X - O.apply_drop(X, dropped)


def test_truncation_frobenius_brute_force_maximal():
    rng = np.random.default_rng(5)
    n = 4 * 32 - 7    # 4 tile rows, ragged: 10 upper tiles
    X = _sym(rng, n)
    # tiles of very different sizes
    e = O.tile_grid(n)
    for i in range(4):
        for j in range(i, 4):
            sc = 10.0 ** rng.uniform(-6, -2)
            X[e[i]:e[i + 1], e[j]:e[j + 1]] *= sc
            if i != j:
                X[e[j]:e[j + 1], e[i]:e[i + 1]] *= sc
    nb, tiles = O.upper_tiles(X)
    tau = 3e-4
    _, kept, dropped = O.truncate_select(X, tau, "frobenius")
    assert np.linalg.norm(_E(X, dropped)) <= tau
    # Section 2 (blocks with norms below a threshold are removed): over every
    # threshold -- every set {tiles with (norm, index) below a cut} -- the chosen
    # set is the largest one whose dense ||E||_F stays within tau
    order = sorted(tiles, key=lambda t: (t[2], t[0] * nb + t[1]))
    feasible = [k for k in range(len(order) + 1)
                if np.linalg.norm(_E(X, [(i, j) for i, j, _ in order[:k]])) <= tau]
    best = max(feasible)
    assert sorted(dropped) == sorted((i, j) for i, j, _ in order[:best])
    assert 0 < best < len(order)
    # brute force over all subsets: none with more stored tiles is a threshold set
    ids = [(i, j) for i, j, _ in tiles]
    for k in range(best + 1, len(ids) + 1):
        for S in itertools.combinations(ids, k):
            if np.linalg.norm(_E(X, list(S))) <= tau:
                cut = max((X_n2(tiles, t), t[0] * nb + t[1]) for t in S)
                assert any((X_n2(tiles, t), t[0] * nb + t[1]) < cut and t not in S for t in ids)


def X_n2(tiles, t):
    return next(v for i, j, v in tiles if (i, j) == t)


def _dyadic_tiles(norm2, big):
    """Symmetric 128 x 128 matrix whose upper tile (I, J) has squared Frobenius
    norm norm2[(I, J)] * 2^-60 exactly (integer units; tiles not listed get
    `big`): each tile is a sum of squares of integers a * 2^-30 placed on the
    tile's own diagonal (mirrored for I < J), so every sum below is exact."""
    X = np.zeros((128, 128))
    for I in range(4):
        for J in range(I, 4):
            rem = norm2.get((I, J), big)
            r = 0
            while rem > 0:                      # greedy squares, at most 32 terms
                a = math.isqrt(rem)
                X[32 * I + r, 32 * J + r] = X[32 * J + r, 32 * I + r] = a * 2.0 ** -30
                rem -= a * a
                r += 1
            assert r <= 32
    return X


@pytest.mark.parametrize("slack", ["2^-30", "0"])
def test_truncation_cut_at_the_budget_real_number_rule(slack):
    # Section 2 / Eq. (8), read as: drop the longest prefix (ascending norms)
    # with sum w ||X_IJ||_F^2 <= tau^2.  The oracle sums shares rounded up to
    # units of tau^2 2^-36.  Five candidate tiles (weights 2, 2, 1, 2, 1) sum to
    # tau^2 (1 - 2^-30) or to tau^2 exactly; every share has a fractional part
    tau = 2.0 ** -10                       # tau^2 = 2^-20 = 2^40 units of 2^-60
    cand = [((0, 1), 2, 2 ** 34 + 3), ((0, 2), 2, 2 ** 35 + 5), ((1, 1), 1, 2 ** 35 + 2 ** 34 + 7),
            ((2, 3), 2, 2 ** 36 + 9)]
    target = 2 ** 40 - (2 ** 10 if slack == "2^-30" else 0)
    last = target - sum(w * v for _, w, v in cand)
    assert cand[-1][2] < last < 2 ** 44
    cand.append(((3, 3), 1, last))
    X = _dyadic_tiles({t: v for t, _, v in cand}, big=2 ** 44)
    # the plain rule, in exact integers: all five fit (sum <= tau^2), a sixth does not
    assert sum(w * v for _, w, v in cand) <= 2 ** 40
    assert sum(w * v for _, w, v in cand) + 2 ** 44 > 2 ** 40
    assert all((w * v) % 16 for _, w, v in cand)          # shares (units tau^2 2^-36) are not integers
    _, kept, dropped = O.truncate_select(X, tau, "frobenius")
    E2 = float(np.sum(_E(X, dropped) ** 2))               # exact: multiples of 2^-60 below 2^-20
    assert E2 <= tau * tau
    if slack == "2^-30":
        # 64 units of slack against at most 5 units of rounding: the readings agree
        assert sorted(dropped) == sorted(t for t, _, _ in cand)
        assert E2 == (2 ** 40 - 2 ** 10) * 2.0 ** -60
    else:
        # ||E||_F = tau exactly for the plain rule; the rounded-up shares exceed
        # the budget by at most 5 units, so the oracle keeps the fifth tile (it
        # is conservative by less than one unit per candidate tile)
        assert sorted(dropped) == sorted(t for t, _, _ in cand[:4])
        assert E2 < tau * tau


def test_truncation_tau_zero_drops_only_zero_tiles():
    rng = np.random.default_rng(6)
    X = _sym(rng, 96)
    X[0:32, 64:96] = 0.0
    X[64:96, 0:32] = 0.0
    _, kept, dropped = O.truncate_select(X, 0.0, "frobenius")
    assert dropped == [(0, 2)]


def _block_norm_matrix(A, part):
    n = A.shape[0]
    e = np.append(np.arange(0, n, part), n)
    k = len(e) - 1
    M = np.zeros((k, k))
    for i in range(k):
        for j in range(k):
            M[i, j] = np.linalg.norm(A[e[i]:e[i + 1], e[j]:e[j + 1]])
    return M


def test_truncation_frobinf_norm_chain():
    rng = np.random.default_rng(7)
    n = 320
    X = _sym(rng, n)
    dist = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    X *= np.exp(-dist / 12.0)
    tau = 0.05
    part = 64
    _, kept, dropped = O.truncate_select(X, tau, "frobinf", part=part)
    assert dropped
    E = _E(X, dropped)
    M = _block_norm_matrix(E, part)
    two = np.linalg.norm(E, 2)
    mixed_m = np.linalg.norm(M, 2)          # Frobenius-spectral mixed norm (Eq. (11))
    mixed_M = np.abs(M).sum(axis=1).max()   # Frob-Inf norm (Eq. (13))
    assert two <= mixed_m + 1e-15 <= mixed_M + 2e-15 and mixed_M <= tau * (1 + 1e-12)


@pytest.mark.parametrize("permute", [False, True])
def test_banded_matrix_norm_experiment(permute):
    # Section 3's test matrix: symmetric banded, entries U(0, 1e-3), bandwidth 2*300+1
    g = GOLDEN["banded_norm_test"]
    rng = np.random.default_rng(8)
    n = 3000
    hb = g["half_bandwidth"]
    A = np.triu(rng.uniform(0.0, 1e-3, (n, n)))
    A = np.triu(A) - np.triu(A, hb + 1)
    A = A + np.triu(A, 1).T
    if permute:
        p = rng.permutation(n)
        A = A[np.ix_(p, p)]
    two = np.abs(np.linalg.eigvalsh(A)).max()
    fro = np.linalg.norm(A)
    for bs in g["block_sizes"]:
        M = _block_norm_matrix(A, bs)
        m = np.linalg.norm(M, 2)
        MM = M.sum(axis=1).max()
        assert two <= m * (1 + 1e-12) and m <= MM * (1 + 1e-12)
        if not permute and bs == 100:
            assert MM < 0.6 * fro    # Frob-Inf already well below Frobenius at N = 3000


# ----------------------------------------------------------------- symbolic square
def _random_kept(rng, nb, density, drop_diag=()):
    """A random upper tile pattern (sorted (I, J) list) with the given diagonal
    tiles left out."""
    kept = []
    for i in range(nb):
        for j in range(i, nb):
            if i == j:
                if i not in drop_diag:
                    kept.append((i, j))
            elif rng.random() < density:
                kept.append((i, j))
    return kept


# hand-made cases next to random ones: an isolated coupling (0, 1) with both
# diagonal tiles gone and no K joining them, a chain, a single tile
_HAND = [
    (4, [(0, 1), (2, 2), (2, 3), (3, 3)]),
    (5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    (3, [(1, 1)]),
    (1, [(0, 0)]),
]


@pytest.mark.parametrize("case", range(len(_HAND) + 6))
def test_triplet_count_brute_force(case):
    # the headline's numerator: (I <= J, K) with X~_IK and X~_KJ stored (either
    # triangle), counted by an explicit triple loop
    if case < len(_HAND):
        nb, kept = _HAND[case]
    else:
        rng = np.random.default_rng(100 + case)
        nb = int(rng.integers(2, 9))
        kept = _random_kept(rng, nb, rng.uniform(0.1, 0.9), drop_diag=set(rng.integers(0, nb, 2).tolist()))
    stored = set(kept) | {(j, i) for i, j in kept}
    brute = sum(1 for i in range(nb) for j in range(i, nb) for k in range(nb)
                if (i, k) in stored and (k, j) in stored)
    assert O._triplets(kept, nb) == brute


@pytest.mark.parametrize("case", range(len(_HAND) + 6))
def test_general_storage_triplet_count_brute_force(case):
    # every (I, J) of the square (both triangles) and K with X~_IK, X~_KJ stored
    if case < len(_HAND):
        nb, kept = _HAND[case]
    else:
        rng = np.random.default_rng(300 + case)
        nb = int(rng.integers(2, 9))
        kept = _random_kept(rng, nb, rng.uniform(0.1, 0.9), drop_diag=set(rng.integers(0, nb, 2).tolist()))
    stored = set(kept) | {(j, i) for i, j in kept}
    brute = sum(1 for i in range(nb) for j in range(nb) for k in range(nb)
                if (i, k) in stored and (k, j) in stored)
    assert O.triplets_general(kept, nb) == brute


@pytest.mark.parametrize("case", range(len(_HAND) + 6))
def test_product_pattern_matches_nonzero_tiles_of_the_polynomial(case):
    # the tile pattern of X_i = c0 I + c1 X~ + c2 X~^2 (Algorithm 2), found from
    # the arithmetic itself: positive values on the stored tiles and positive
    # coefficients, so no tile cancels
    if case < len(_HAND):
        nb, kept = _HAND[case]
    else:
        rng = np.random.default_rng(200 + case)
        nb = int(rng.integers(2, 9))
        kept = _random_kept(rng, nb, rng.uniform(0.1, 0.9), drop_diag=set(rng.integers(0, nb, 2).tolist()))
    rng = np.random.default_rng(case)
    b = 4                      # small tiles: the pattern does not depend on the tile size
    X = np.zeros((nb * b, nb * b))
    for i, j in kept:
        blk = rng.uniform(0.5, 1.0, (b, b))
        X[i * b:(i + 1) * b, j * b:(j + 1) * b] = blk
        X[j * b:(j + 1) * b, i * b:(i + 1) * b] = blk.T
    Xi = 0.3 * np.eye(nb * b) + 0.7 * X + 1.1 * (X @ X)
    nz = {(i, j) for i in range(nb) for j in range(i, nb)
          if np.any(Xi[i * b:(i + 1) * b, j * b:(j + 1) * b] != 0.0)}
    assert O.product_pattern(kept, nb) == nz
    if case == 0:
        assert (0, 1) in nz    # kept only through the c1 X~ term


@pytest.mark.parametrize("seed", range(8))
def test_truncation_of_a_psd_matrix_never_isolates_a_coupling_tile(seed):
    # For X >= 0, ||X_IJ||_F <= sqrt(||X_II||_F ||X_JJ||_F) (Hoelder), so the
    # ascending prefix that drops both diagonal tiles of a pair also drops their
    # coupling: the case pattern(X~) not in pattern(X~^2) cannot come out of the
    # Frobenius selection on the (positive semidefinite) iterates.
    rng = np.random.default_rng(seed)
    nb = 4
    n = nb * 32
    Y = rng.standard_normal((n, 6)) * np.repeat(10.0 ** rng.uniform(-4, 0, nb), 32)[:, None]
    X = Y @ Y.T
    _, tiles = O.upper_tiles(X)
    n2 = {(i, j): v for i, j, v in tiles}
    for i in range(nb):
        for j in range(i + 1, nb):
            assert math.sqrt(n2[(i, j)]) <= (n2[(i, i)] * n2[(j, j)]) ** 0.25 * (1 + 1e-12)
    for tau in 10.0 ** np.linspace(-8, 1, 40):
        _, kept, _ = O.truncate_select(X, tau, "frobenius")
        ks = set(kept)
        for i, j in kept:
            if i != j:
                assert (i, i) in ks or (j, j) in ks


# ----------------------------------------------------------------- Algorithms 1 + 2
def test_sp2_tau0_matches_eigendecomposition_projector():
    c = make_config(1)
    r = O.sp2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], tau=0.0, stop="idempotency")
    assert r.converged
    P = O.eig_projector(c["F"], c["nocc"])
    assert np.linalg.norm(r.D - P) < 1e-12
    assert r.e[r.n] < 1e-12


@pytest.mark.parametrize("stop", ["parameterless", "idempotency"])
def test_sp2_small_random_gapped(stop):
    d = dense_gapped(70, 33, (-1.5, -0.2), (0.2, 1.5), seed=31)
    r = O.sp2(d["F"], d["nocc"], d["homo_ub"], d["lumo_lb"], tau=0.0, stop=stop)
    P = O.eig_projector(d["F"], d["nocc"])
    assert np.linalg.norm(r.D - P) < 1e-11
    assert abs(np.trace(r.D) - d["nocc"]) < 1e-11


def test_sp2_invariants_with_truncation():
    c = make_config("2s")
    F = to_dense(c["F"])
    r = O.sp2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"])
    D = r.D
    n = F.shape[0]
    assert r.converged
    np.testing.assert_array_equal(D, D.T)
    idem = np.linalg.norm(D @ D - D)
    assert abs(idem - r.e[r.n]) <= 1e-9 * max(idem, 1e-12) + 1e-14   # e_n is ||X~_n - X~_n^2||_F
    assert abs(np.trace(D) - c["nocc"]) <= math.sqrt(n) * r.e[r.n] + 1e-9
    assert np.linalg.norm(D @ F - F @ D) / np.linalg.norm(F) < 1e-5


def test_error_control_bound_on_occupied_subspace():
    # Section 2: with tau_i from Eq. (7) and ||E_i|| <= tau_i, ||D - P_Xn||_2 <= gamma
    c = make_config("2s")
    F = to_dense(c["F"])
    gamma = 1e-3
    r = O.sp2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], gamma=gamma)
    w, v = np.linalg.eigh(r.D)
    P_Xn = v[:, w > 0.5] @ v[:, w > 0.5].T
    D = O.eig_projector(F, c["nocc"])
    assert P_Xn.shape == D.shape and np.sum(w > 0.5) == c["nocc"]
    assert np.linalg.norm(D - P_Xn, 2) <= gamma
    assert any(len(k) < len(r.kept[0]) + 10**9 for k in r.kept)


def test_paper_iteration_facts_sp2_vs_sp2acc():
    # Section 6: estimated counts exceed obtained ones, SP2ACC needs fewer than SP2
    c = make_config("2s")
    F = to_dense(c["F"])
    a = O.sp2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"], accelerate=True)
    b = O.sp2(F, c["nocc"], c["homo_ub"], c["lumo_lb"], tau=c["tau"], accelerate=False)
    assert a.converged and b.converged
    assert a.n < a.sched.n_max and b.n < b.sched.n_max
    assert a.n < b.n


def test_stopping_criterion_fires_at_noise_floor():
    c = make_config(1)
    r = O.sp2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], tau=0.0, stop="parameterless")
    assert r.converged and r.e[r.n] < 1e-11
    ri = O.sp2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], tau=0.0, stop="idempotency")
    assert abs(r.n - ri.n) <= 2


@pytest.mark.parametrize("accelerate", [False, True])
def test_homo_lumo_estimates_invert_a_single_eigenvalue(accelerate):
    # Section 4 Step 3: the estimate turns r = x - x^2 of an eigenvalue's image
    # x = x_j back into x (the root on the eigenvalue's side of 1/2) and pulls
    # it back through f_j .. f_1 and X_0's map.  The e_j, t_j that one
    # eigenvalue alone produces (its images by poly_scalar, pinned against the
    # matrix polynomials above; steps whose r is below 1e-6, where x - x^2
    # loses its digits in FP64, are left out as below the noise threshold)
    # must give that eigenvalue back
    import dataclasses
    c = make_config(1)
    nocc, ev = c["nocc"], c["eigenvalues"]
    res = O.sp2(c["F"], nocc, c["homo_ub"], c["lumo_lb"], tau=0.0, stop="idempotency", accelerate=accelerate)
    sch = res.sched
    width = sch.lmax - sch.lmin
    for lam, side in ((ev[nocc - 1], 0), (ev[nocc], 1)):
        x = (sch.lmax - lam) / width
        r = [x - x * x]
        for j in range(1, res.n + 1):
            x = O.poly_scalar(sch.p[j], sch.alpha[j], x)
            r.append(x - x * x)
        r = [v if v >= 1e-6 else 0.0 for v in r]
        est = O.homo_lumo_estimates(dataclasses.replace(res, e=list(r), t=list(r)), c["F"].shape[0])
        assert est[side] is not None
        assert abs(est[side] - lam) <= 1e-11 * width, (side, est[side], lam)


def test_homo_lumo_estimates_approximate():
    # approximately pinned: plain SP2 estimates near the exact homo/lumo
    c = make_config(1)
    r = O.sp2(c["F"], c["nocc"], c["homo_ub"], c["lumo_lb"], tau=0.0, stop="idempotency", accelerate=False)
    h, l = r.estimates
    ev = c["eigenvalues"]
    assert abs(h - ev[c["nocc"] - 1]) < 0.02 and abs(l - ev[c["nocc"]]) < 0.02


# ----------------------------------------------------------------- adjoint
def _loss(F, nocc, hub, llb, W, replay, lmin_lmax=None):
    r = O.sp2(F, nocc, hub, llb, tau=0.0, stop="idempotency", replay_kept=replay)
    return float(np.sum(r.D * W)), r


def test_adjoint_central_finite_differences():
    d = dense_gapped(48, 20, (-1.5, -0.4), (0.4, 1.5), seed=41)
    F = d["F"]
    rng = np.random.default_rng(9)
    W = _sym(rng, 48)
    L0, r = _loss(F, d["nocc"], d["homo_ub"], d["lumo_lb"], W, None)
    G = O.adjoint_sp2(F, r, W)
    # hold lambda bounds, schedule and masks fixed: perturb through the same recursion
    for (i, j) in [(0, 0), (3, 7), (10, 40), (47, 47)]:
        h = 1e-6
        Fp = F.copy(); Fm = F.copy()
        Fp[i, j] += h; Fm[i, j] -= h
        if i != j:
            Fp[j, i] += h; Fm[j, i] -= h
        Lp = _fixed(Fp, r, W)
        Lm = _fixed(Fm, r, W)
        fd = (Lp - Lm) / (2 * h)
        an = G[i, j] + (G[j, i] if i != j else 0.0)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (i, j, fd, an)


def _fixed(F, r, W):
    """The recursion of run r (same lambda bounds, p, alpha, masks, n) applied to F."""
    s = r.sched
    X = O.initial_matrix(F, r.lmin, r.lmax)
    Xt = O._mask_tiles(X, r.kept[0])
    for i in range(1, r.n + 1):
        c0, c1, c2 = O.poly_coeffs(s.p[i], s.alpha[i])
        Xt = O._mask_tiles(c0 * np.eye(F.shape[0]) + c1 * Xt + c2 * (Xt @ Xt), r.kept[i])
    return float(np.sum(Xt * W))


def test_adjoint_matches_daleckii_krein_closed_form():
    # tau = 0, converged: dD = sum over occ i, virt a of divided differences of the
    # step function; dL/dF = V Gt V^T with Gt_ai = Gt_ia = (V^T W V)_ai / (lam_i - lam_a)
    d = dense_gapped(40, 17, (-1.5, -0.5), (0.5, 1.5), seed=43)
    F = d["F"]
    rng = np.random.default_rng(10)
    W = _sym(rng, 40)
    _, r = _loss(F, d["nocc"], d["homo_ub"], d["lumo_lb"], W, None)
    G = O.adjoint_sp2(F, r, W)
    lam, V = np.linalg.eigh(F)
    Wt = V.T @ W @ V
    Gt = np.zeros_like(Wt)
    occ = np.arange(40) < 17
    for i in np.nonzero(occ)[0]:
        for a in np.nonzero(~occ)[0]:
            Gt[i, a] = Gt[a, i] = Wt[i, a] / (lam[i] - lam[a])
    ref = V @ Gt @ V.T
    assert np.linalg.norm(G - ref) <= 1e-6 * np.linalg.norm(ref)


# ----------------------------------------------------------------- trace-correcting SP2, two runs
def test_trace_correcting_reaches_eigenprojector():
    # Section 1: the trace-correcting SP2 needs no eigenvalue bounds; at tau = 0
    # it converges to D of Eq. (3)
    c = make_config(1)
    r = O.sp2_trace_correcting(c["F"], c["nocc"], tau=0.0, stop="idempotency")
    assert r.converged and r.e[r.n] < 1e-12
    assert np.linalg.norm(r.D - O.eig_projector(c["F"], c["nocc"])) < 1e-12
    d = dense_gapped(70, 33, (-1.5, -0.2), (0.2, 1.5), seed=31)
    r = O.sp2_trace_correcting(d["F"], d["nocc"], tau=0.0)
    assert r.converged
    assert np.linalg.norm(r.D - O.eig_projector(d["F"], d["nocc"])) < 1e-11


def test_trace_correcting_choices_follow_the_eigenvalue_recursion():
    # the same rule on the eigenvalues of X_0 as scalars: p_i = 1 iff the sum of
    # the images exceeds nocc; compared while the trace is clearly off nocc
    d = dense_gapped(90, 41, (-2.0, -0.1), (0.3, 1.7), seed=8)
    r = O.sp2_trace_correcting(d["F"], d["nocc"], tau=0.0, stop="idempotency")
    x = (r.lmax - d["eigenvalues"]) / (r.lmax - r.lmin)
    compared = 0
    for i in range(1, r.n + 1):
        s = float(np.sum(x))
        if abs(s - d["nocc"]) < 1e-8:
            break
        p = 1 if s > d["nocc"] else 0
        assert r.sched.p[i] == p, i
        compared += 1
        x = O.poly_scalar(p, 1.0, x)
    assert compared >= 10


@pytest.mark.parametrize("key", [1, "2s"])
def test_two_run_bounds_bracket_the_gap(key):
    # Section 6: run 1 (trace-correcting) gives Step 3 estimates; widened by the
    # margin they must be valid bounds (homo_ub >= homo, lumo_lb <= lumo) for
    # the SP2ACC run 2, which then converges in fewer iterations than run 1
    c = make_config(key)
    F = c["F"] if isinstance(c["F"], np.ndarray) else to_dense(c["F"])
    tau1 = 0.0 if key == 1 else 1e-5
    kw = dict(stop=c["stop"])
    r1, r2, (hub, llb) = O.two_run(F, c["nocc"], tau1, tau=c["tau"], **kw)
    ev = np.linalg.eigvalsh(F)
    assert hub >= ev[c["nocc"] - 1] and llb <= ev[c["nocc"]]
    assert r2.converged and r2.n < r1.n
    if key == 1:
        assert np.linalg.norm(r2.D - O.eig_projector(F, c["nocc"])) < 1e-12
    with pytest.raises(ValueError):
        O.bounds_from_estimates(None, 0.5, -1.0, 1.0)


# ----------------------------------------------------------------- mixed-norm truncation (Section 3)
def _exact_mixed(E, part):
    n = E.shape[0]
    e = np.append(np.arange(0, n, part), n)
    k = len(e) - 1
    Bm = np.array([[np.linalg.norm(E[e[i]:e[i + 1], e[j]:e[j + 1]]) for j in range(k)] for i in range(k)])
    return float(np.abs(np.linalg.eigvalsh(Bm)).max())


@pytest.mark.parametrize("seed", range(6))
def test_mixed_norm_bound_is_an_upper_bound_close_to_rho(seed):
    # Collatz-Wielandt: the bound is >= the Perron root of M = sqrt(B2), and the
    # power steps bring it close to it
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 40))
    B = rng.uniform(0.0, 1.0, (k, k)) * (rng.random((k, k)) < 0.5)
    B2 = np.round((B + B.T) ** 2 * 2 ** 20)
    rho = float(np.abs(np.linalg.eigvalsh(np.sqrt(B2))).max())
    ub = O.mixed_norm_bound(B2.astype(np.int64))
    assert ub >= rho * (1 - 1e-12)
    assert ub <= rho * (1 + 1e-6) + 1e-12


@pytest.mark.parametrize("tau,part", [(1e-4, 128), (1e-2, 128), (1e-1, 256), (1.0, 96)])
def test_mixed_truncation_norm_chain_and_near_maximal(tau, part):
    # Section 3: ||E||_2 <= ||E||_m <= tau for the dropped E; dropping the next
    # candidate too would pass tau (the bound is within 1e-6 of ||.||_m)
    rng = np.random.default_rng(17)
    n = 800
    A = _sym(rng, n)
    d = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    A *= np.exp(-d / 40.0)
    _, kept, dropped = O.truncate_select(A, tau, "mixed", part=part)
    E = A - O.apply_drop(A, dropped)
    m = _exact_mixed(E, part)
    assert np.linalg.norm(E, 2) <= m * (1 + 1e-12) and m <= tau * (1 + 1e-12)
    assert len(dropped) > 0
    _, tiles = O.upper_tiles(A)
    n2 = {(i, j): v for i, j, v in tiles}
    nxt = min(kept, key=lambda t: n2[t])
    E2 = A - O.apply_drop(A, dropped + [nxt])
    assert _exact_mixed(E2, part) > tau * (1 - 1e-5)


def test_mixed_truncation_with_one_block_is_the_frobenius_rule():
    # one block: ||E||_m = ||E||_F, and the threshold on the squared norms drops
    # the same tiles as the Frobenius prefix rule (no equal norms here)
    rng = np.random.default_rng(5)
    n = 4 * 32 - 7
    X = _sym(rng, n)
    e = O.tile_grid(n)
    for i in range(4):
        for j in range(i, 4):
            sc = 10.0 ** rng.uniform(-6, -2)
            X[e[i]:e[i + 1], e[j]:e[j + 1]] *= sc
            X[e[j]:e[j + 1], e[i]:e[i + 1]] = X[e[i]:e[i + 1], e[j]:e[j + 1]].T
    for tau in (1e-6, 1e-4, 1e-3, 1e-2):
        a = O.truncate_select(X, tau, "mixed", part=4096)
        b = O.truncate_select(X, tau, "frobenius")
        assert a[1] == b[1]
    assert O.truncate_select(X, 0.0, "mixed", part=64)[2] == []
