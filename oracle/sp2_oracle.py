"""Plain FP64 numpy oracle of the SP2ACC expansion (test infrastructure only).

Header: this module is the parity reference of the CUDA library.  Only the test
suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs may
import it.  It works on dense N x N arrays; tiles of 32 x 32 only matter for
truncation, where the last tile row/column is ragged when 32 does not divide N.

Paper: Kruchinina, Rudberg, Rubensson, "Efficient computation of the density
matrix with error control on distributed computer systems" (arXiv:1909.12533).

What each function follows:
  eig_projector ............. Section 1, Eq. (3): D = sum_{i<=nocc} y_i y_i^T
  gershgorin_bounds, initial_matrix ... Section 4 Step 1 and Algorithm 1
  schedule .................. Section 4 Step 1 (alpha_i, p_i, n_min, n_max, tau_i);
                              the rules for alpha/p/n_min/n_max come from an
                              uncited companion paper, so they are a stated reading
                              (see ``schedule``); tau_i in gamma mode is Eq. (7)
  truncate_* ................ Section 2 (X~_i = X_i + E_i, ||E_i|| <= tau_i, Eqs. (6)-(8))
                              and Section 3 (Frob-Inf norm, Eq. (13); the
                              Frobenius-spectral mixed norm); selection rules are
                              stated readings
  sp2 ....................... Algorithms 1 and 2
  triplets_general .......... Section 5 (general storage: both triangles computed)
  homo_lumo_estimates ....... Section 4 Step 3 (reading; see the function)
  sp2_trace_correcting ...... Section 1 (the original SP2: the polynomial of each
                              iteration chosen from the trace) and Section 6 (the
                              first run, without eigenvalue bounds)
  bounds_from_estimates,
  two_run ................... Section 6: run 1 trace-correcting, its Step 3
                              estimates (with a stated margin) as the bounds of
                              the SP2ACC run 2
  adjoint_sp2 ............... not in the paper: reverse-mode derivative of the
                              recursion for L = trace(D W)

Parity pins: every function above except ``homo_lumo_estimates`` is pinned in
tests/test_oracle.py against eigendecompositions, closed forms, brute force or
invariants.  ``homo_lumo_estimates`` is pinned only approximately (it is an
estimate; it is compared with exact eigenvalues on small cases).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

B = 32                      # tile size (Section 6: small block size 32)
C_STOP = 6.8872             # Algorithm 2, constant of the stopping criterion
FROBINF_PART = 4096         # Section 6: Frob-Inf block size equals leaf size 4096
Q_SCALE = 2.0 ** 36         # resolution of the truncation budget (reading, see truncate_select)
Q_CAP = 2 ** 37             # one tile's budget units are capped here (never removable)


# ----------------------------------------------------------------------------- Section 1
def eig_projector(F: np.ndarray, nocc: int) -> np.ndarray:
    """D = sum_{i=1}^{nocc} y_i y_i^T over the nocc lowest eigenpairs of F (Eq. (3))."""
    w, v = np.linalg.eigh(F)
    y = v[:, :nocc]
    return y @ y.T


# ----------------------------------------------------------------------------- Algorithm 1
def gershgorin_bounds(F: np.ndarray) -> tuple[float, float]:
    """lambda_min <= lambda_1 and lambda_max >= lambda_N from Gershgorin discs
    (Section 4, Step 1): centre F_ii, radius sum_{j != i} |F_ij|."""
    d = np.diag(F)
    r = np.abs(F).sum(axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def initial_matrix(F: np.ndarray, lmin: float, lmax: float) -> np.ndarray:
    """X_0 = (lambda_max I - F) / (lambda_max - lambda_min)  (Algorithm 1)."""
    n = F.shape[0]
    return (lmax * np.eye(n) - F) / (lmax - lmin)


# ----------------------------------------------------------------------------- polynomials
def poly_coeffs(p: int, alpha: float) -> tuple[float, float, float]:
    """X_i = c0 I + c1 X~ + c2 X~^2 for the two polynomials of Algorithm 2:
    p=1: ((1-a) I + a X)^2 = (1-a)^2 I + 2a(1-a) X + a^2 X^2
    p=0: 2 a X - (a X)^2."""
    if p == 1:
        return (1.0 - alpha) ** 2, 2.0 * alpha * (1.0 - alpha), alpha * alpha
    return 0.0, 2.0 * alpha, -(alpha * alpha)


def poly_scalar(p: int, alpha: float, x):
    """The same polynomial applied to scalars (eigenvalues)."""
    if p == 1:
        return ((1.0 - alpha) + alpha * x) ** 2
    return 2.0 * alpha * x - (alpha * x) ** 2


# ----------------------------------------------------------------------------- Step 1 schedule
@dataclass
class Schedule:
    lmin: float
    lmax: float
    p: list = field(default_factory=list)       # p[i], i = 1..n_max (index 0 unused)
    alpha: list = field(default_factory=list)   # alpha[i]
    tau: list = field(default_factory=list)     # tau[i], i = 0..n_max
    n_min: int = 1
    n_max: int = 0
    vhi: list = field(default_factory=list)     # bound on virtual images after step i (incl. truncation slack)
    olo: list = field(default_factory=list)     # bound on occupied images after step i
    xi: list = field(default_factory=list)      # gap lower bound of X_i before truncation (Eq. (7))


def _image(p: int, alpha: float, a: float, b: float) -> tuple[float, float]:
    """Exact range of the quadratic f_i over [a, b]: endpoints plus the vertex."""
    vals = [poly_scalar(p, alpha, a), poly_scalar(p, alpha, b)]
    vertex = (alpha - 1.0) / alpha if p == 1 else 1.0 / alpha
    if a <= vertex <= b:
        vals.append(poly_scalar(p, alpha, vertex))
    return min(vals), max(vals)


def _choose(vlo, vhi, olo, ohi, accelerate: bool, delta_acc: float) -> tuple[int, float, bool]:
    """Reading of Section 4 Step 1 (Algorithm 4 of the stopping-criteria paper is
    not reproduced in this paper):
      d0 = distance of the virtual interval from 0, d1 = of the occupied one from 1;
      p = 1 (the x^2 branch) iff d0 > d1;
      while acceleration is on, alpha folds the interval that p improves onto
      itself around the vertex (scale-and-fold): p=1 maps [vlo, vhi] to an
      interval symmetric about 0 before squaring, p=0 maps [olo, ohi] to one
      symmetric about 1;
      acceleration switches off for good once max(d0, d1) <= delta_acc."""
    d0 = max(vhi, -vlo)
    d1 = max(1.0 - olo, ohi - 1.0)
    p = 1 if d0 > d1 else 0
    if accelerate and max(d0, d1) > delta_acc:
        alpha = 2.0 / (2.0 - vlo - vhi) if p == 1 else 2.0 / (olo + ohi)
        alpha = max(alpha, 1.0)
        return p, alpha, True
    return p, 1.0, False


def schedule(lmin: float, lmax: float, homo_ub: float, lumo_lb: float, tau: float = 0.0,
             gamma: float | None = None, accelerate: bool = True, delta_acc: float = 0.1,
             n_cap: int = 100) -> Schedule:
    """Step 1 of Section 4.

    Images of the eigenvalues under X_0 = (lmax I - F)/w: virtual ones lie in
    [0, (lmax - lumo_lb)/w], occupied ones in [(lmax - homo_ub)/w, 1].

    n_max (reading): the number of steps after which, in exact arithmetic with
    no truncation, both intervals are within 2^-52 of {0, 1}; capped at n_cap.

    p_i, alpha_i (reading, ``_choose``) are chosen on intervals that include the
    truncation slack: after truncation with ||E_i||_2 <= tau_i every eigenvalue
    moves by at most tau_i (Weyl), so each interval is widened by tau_i.

    tau_i: the fixed ``tau`` for every i, or, in gamma mode, Eq. (7) with the
    gap lower bound xi_i = olo_i - vhi_i of X_i.
    """
    w = lmax - lmin
    v0 = (lmax - lumo_lb) / w
    o0 = (lmax - homo_ub) / w
    # n_max from the slack-free propagation
    vlo, vhi, olo, ohi = 0.0, v0, o0, 1.0
    acc = accelerate
    n_max = n_cap
    for i in range(1, n_cap + 1):
        p, a, acc = _choose(vlo, vhi, olo, ohi, acc, delta_acc)
        vlo, vhi = _image(p, a, vlo, vhi)
        olo, ohi = _image(p, a, olo, ohi)
        if max(vhi, -vlo, 1.0 - olo, ohi - 1.0) < 2.0 ** -52:
            n_max = i
            break
    s = Schedule(lmin=lmin, lmax=lmax, n_max=n_max)

    def tau_of(vh, ol):
        if gamma is None:
            return float(tau)
        g = gamma / (n_max + 1)
        return g * (ol - vh) / (1.0 + g)

    vlo, vhi, olo, ohi = 0.0, v0, o0, 1.0
    t0 = tau_of(vhi, olo)
    s.xi.append(olo - vhi)
    s.tau.append(t0)
    vlo, vhi, olo, ohi = vlo - t0, vhi + t0, olo - t0, ohi + t0
    s.p.append(-1)
    s.alpha.append(float("nan"))
    s.vhi.append(vhi)
    s.olo.append(olo)
    acc = accelerate
    s.n_min = 1 if not accelerate else n_max + 1
    for i in range(1, n_max + 1):
        p, a, acc_now = _choose(vlo, vhi, olo, ohi, acc, delta_acc)
        if acc and not acc_now:
            s.n_min = i
        acc = acc_now
        s.p.append(p)
        s.alpha.append(a)
        vlo, vhi = _image(p, a, vlo, vhi)
        olo, ohi = _image(p, a, olo, ohi)
        ti = tau_of(vhi, olo)
        s.xi.append(olo - vhi)
        s.tau.append(ti)
        vlo, vhi, olo, ohi = vlo - ti, vhi + ti, olo - ti, ohi + ti
        s.vhi.append(vhi)
        s.olo.append(olo)
    return s


# ----------------------------------------------------------------------------- truncation
def tile_grid(n: int, b: int = B) -> np.ndarray:
    """Tile edges 0, b, 2b, ..., n (last tile ragged)."""
    return np.append(np.arange(0, n, b), n)


def upper_tiles(X: np.ndarray, b: int = B):
    """All upper tiles (I <= J) of a dense matrix with their squared Frobenius norms,
    in the order sorted by (I, J)."""
    n = X.shape[0]
    e = tile_grid(n, b)
    nb = len(e) - 1
    out = []
    for i in range(nb):
        for j in range(i, nb):
            blk = X[e[i]:e[i + 1], e[j]:e[j + 1]]
            out.append((i, j, float(np.sum(blk * blk))))
    return nb, out


def _prefix_cut(norm2: np.ndarray, weight: np.ndarray, lin: np.ndarray, budget: float) -> np.ndarray:
    """Reading of 'truncate so that ||E|| <= tau' (Section 2, Eq. (8)): sort the
    candidate tiles by (squared norm, linear index) ascending and drop the
    longest prefix whose weighted squared norms fit into the budget tau^2.
    The sum is taken in integer units of budget * 2^-36, each tile's share
    rounded up, so the sum is exact and never understates ||E||_F^2.
    Returns a boolean 'drop' mask in the input order."""
    drop = np.zeros(norm2.shape[0], dtype=bool)
    if norm2.shape[0] == 0:
        return drop
    if budget == 0.0:
        return norm2 == 0.0
    s = Q_SCALE / budget
    q = np.minimum(np.ceil(weight * norm2 * s), Q_CAP).astype(np.int64)
    order = np.lexsort((lin, norm2))
    csum = np.cumsum(q[order])
    k = int(np.searchsorted(csum, int(Q_SCALE), side="right"))
    drop[order[:k]] = True
    return drop


MIXED_POWER_ITERS = 100     # power iterations of the mixed-norm bound (reading, see mixed_norm_bound)
MIXED_MAX_BLOCKS = 512      # largest partition count of the mixed norm


def mixed_norm_bound(B2: np.ndarray) -> float:
    """Upper bound of the spectral norm of the block-norm matrix M = sqrt(B2)
    (B2: symmetric, nonnegative, the squared Frobenius norms of the blocks of a
    symmetric E), i.e. of the Frobenius-spectral mixed norm ||E||_m of Section
    3.  M >= 0, so ||M||_2 = rho(M), and for every positive x the
    Collatz-Wielandt bound rho(M) <= max_i (M x)_i / x_i holds (rows that are
    all zero are isolated and skipped).  Reading: x starts at all ones; each of
    MIXED_POWER_ITERS steps takes the bound u = max_i (M x)_i / x_i, then moves x
    to (M x + u x) / max(M x + u x) -- a power step on M + u I, which keeps x
    positive and converges inside every connected block of M also when M has
    eigenvalues -rho; the smallest bound is returned.  Row sums are sequential
    (the order the library uses)."""
    M = np.sqrt(B2.astype(np.float64))
    live = M.max(axis=1) > 0.0
    if not np.any(live):
        return 0.0
    M = M[np.ix_(live, live)]
    x = np.ones(M.shape[0])
    best = math.inf
    for _ in range(MIXED_POWER_ITERS):
        y = np.cumsum(M * x[None, :], axis=1)[:, -1]
        u = float(np.max(y / x))
        best = min(best, u)
        z = y + u * x
        x = z / float(np.max(z))
    return best


def _mixed_cut(n2, weight, R, C, nsb, tau):
    """Reading of 'truncate so that ||E||_m <= tau' (Section 3): drop every
    candidate tile whose squared norm is at most a threshold theta, for the
    largest theta (found by bisection over the 63-bit patterns of the squared
    norms, which order like the values) whose error matrix has a mixed-norm
    bound (mixed_norm_bound) of at most tau.  Block sums are exact integers in
    units of tau^2 2^-36 with each tile's share rounded up (as in _prefix_cut),
    so the bound never understates ||E||_m.  Returns the boolean 'drop' mask."""
    drop = np.zeros(n2.shape[0], dtype=bool)
    if n2.shape[0] == 0:
        return drop
    if tau == 0.0:
        return n2 == 0.0
    s = Q_SCALE / (tau * tau)
    q = np.minimum(np.ceil(weight * n2 * s), Q_CAP).astype(np.int64)
    bits = n2.view(np.int64)
    limit = 2.0 ** 18          # tau in units of tau 2^-18 (the square root of the unit)

    def bound(theta):
        sel = bits <= theta
        B2 = np.zeros((nsb, nsb), dtype=np.int64)
        np.add.at(B2, (R[sel], C[sel]), q[sel])
        off = sel & (R != C)
        np.add.at(B2, (C[off], R[off]), q[off])
        return mixed_norm_bound(B2)

    lo, hi = 0, 2 ** 63 - 1
    while hi - lo > 1:
        mid = lo + (hi - lo) // 2
        if bound(mid) <= limit:
            lo = mid
        else:
            hi = mid
    return bits <= lo


def truncate_select(X: np.ndarray, tau: float, mode: str = "frobenius", part: int = FROBINF_PART,
                    pattern: set | None = None, b: int = B):
    """Choose the upper tiles to drop from X so that ||E||_F <= tau ("frobenius")
    or ||E||_M <= tau ("frobinf", Eq. (13) with square partition ``part``).

    ``pattern`` restricts the candidates to the stored tiles (tiles outside it
    are exactly zero and not stored); default: all tiles.
    Frob-Inf reading: super-block (R, C) gets the budget tau / max(m_R, m_C) with
    m_R the number of nonzero super-blocks in super-row R; inside it the
    Frobenius prefix rule applies.  Then every super-row sum of ||E_RC||_F is at
    most tau, so ||E||_2 <= ||E||_M <= tau (Eq. (14)).
    Returns (nb, list of kept (I, J) in sorted order, list of dropped (I, J))."""
    nb, tiles = upper_tiles(X, b)
    if pattern is not None:
        tiles = [t for t in tiles if (t[0], t[1]) in pattern]
    ii = np.array([t[0] for t in tiles], dtype=np.int64)
    jj = np.array([t[1] for t in tiles], dtype=np.int64)
    n2 = np.array([t[2] for t in tiles], dtype=np.float64)
    lin = ii * nb + jj
    drop = np.zeros(len(tiles), dtype=bool)
    if mode == "frobenius":
        w = np.where(ii == jj, 1.0, 2.0)
        drop = _prefix_cut(n2, w, lin, float(tau) * float(tau))
    elif mode == "frobinf":
        pt = part // b
        R, Cc = ii // pt, jj // pt
        nsb = (nb + pt - 1) // pt
        nz = np.zeros((nsb, nsb), dtype=bool)
        nz[R, Cc] = True
        nz[Cc, R] = True
        m = nz.sum(axis=1)
        for r in range(nsb):
            for c in range(r, nsb):
                sel = np.nonzero((R == r) & (Cc == c))[0]
                if sel.size == 0:
                    continue
                beta = float(tau) / float(max(m[r], m[c]))
                if r == c:
                    w = np.where(ii[sel] == jj[sel], 1.0, 2.0)
                else:
                    w = np.ones(sel.size)
                drop[sel] = _prefix_cut(n2[sel], w, lin[sel], beta * beta)
    elif mode == "mixed":
        # Frobenius-spectral mixed norm of Section 3 on the partition of `part`
        # rows; weight 2 for an off-diagonal tile inside a diagonal block (its
        # mirror lies in the same block)
        pt = part // b
        R, Cc = ii // pt, jj // pt
        nsb = (nb + pt - 1) // pt
        if nsb > MIXED_MAX_BLOCKS:
            raise ValueError("too many blocks for the mixed norm")
        w = np.where((R == Cc) & (ii != jj), 2.0, 1.0)
        drop = _mixed_cut(n2, w, R, Cc, nsb, float(tau))
    else:
        raise ValueError(mode)
    kept = [(int(a), int(c)) for a, c, d in zip(ii, jj, drop) if not d]
    dropped = [(int(a), int(c)) for a, c, d in zip(ii, jj, drop) if d]
    return nb, kept, dropped


def apply_drop(X: np.ndarray, dropped, b: int = B) -> np.ndarray:
    """X~ = X + E: zero the dropped tiles and their mirrors."""
    e = tile_grid(X.shape[0], b)
    Y = X.copy()
    for i, j in dropped:
        Y[e[i]:e[i + 1], e[j]:e[j + 1]] = 0.0
        Y[e[j]:e[j + 1], e[i]:e[i + 1]] = 0.0
    return Y


def product_pattern(kept, nb: int) -> set:
    """Tile pattern of X_i = c0 I + c1 X~ + c2 X~^2 (Algorithm 2) on the upper
    triangle: (I, J), I <= J, is present iff some K has X~_IK and X~_KJ stored
    (the product X~^2), or X~_IJ itself is stored (the c1 X~ term), or I = J
    (the c0 I term).  Integer work, the exact boolean product."""
    A = np.zeros((nb, nb), dtype=np.int64)
    for i, j in kept:
        A[i, j] = 1
        A[j, i] = 1
    P = ((A @ A) > 0) | (A > 0)
    np.fill_diagonal(P, True)
    iu, ju = np.nonzero(np.triu(P))
    return set(zip(iu.tolist(), ju.tolist()))


# ----------------------------------------------------------------------------- Algorithm 2
@dataclass
class SP2Result:
    D: np.ndarray
    n: int                      # index of the output iterate X~_n
    e: list                     # e_j, j = 0..(last computed)
    t: list                     # t_j
    sched: Schedule
    kept: list                  # kept tiles of X~_j for j = 0..n (list of sorted (I, J) lists)
    converged: bool
    lmin: float
    lmax: float
    squares: int                # number of matrix squares computed
    tile_triplets: int          # sum over squares of the nonzero (I<=J, K) tile triplets
    estimates: tuple | None = None


def _triplets(kept, nb: int) -> int:
    """Number of (I, J, K), I <= J, with X~_IK and X~_KJ stored tiles."""
    A = np.zeros((nb, nb), dtype=np.int64)
    for i, j in kept:
        A[i, j] = 1
        A[j, i] = 1
    C = A @ A
    return int(np.triu(C).sum())


def triplets_general(kept, nb: int) -> int:
    """Number of (I, J, K) over the whole square, both triangles, with X~_IK and
    X~_KJ stored: the tile products of the square in general storage (Section 5:
    the general-matrix implementation stores and computes both triangles)."""
    A = np.zeros((nb, nb), dtype=np.int64)
    for i, j in kept:
        A[i, j] = 1
        A[j, i] = 1
    return int((A @ A).sum())


def sp2(F: np.ndarray, nocc: int, homo_ub: float, lumo_lb: float, tau: float = 0.0,
        gamma: float | None = None, accelerate: bool = True, stop: str = "parameterless",
        idem_tol: float = 1e-12, trunc: str = "frobenius", delta_acc: float = 0.1,
        n_cap: int = 100, replay_kept=None, input_pattern=None, b: int = B,
        frobinf_part: int = FROBINF_PART) -> SP2Result:
    """Algorithms 1 and 2 in the paper's order.

    e_j = ||X~_j - X~_j^2||_F and t_j = trace(X~_j - X~_j^2) need X~_j^2, which is
    also the product that forms X_{j+1}; so the loop at step i computes
    S = X~_{i-1}^2 once, takes e_{i-1}, t_{i-1} from it, runs the stopping test on
    index i-1 and only then forms X_i.  Stopping at index j returns X~_j.

    Parameterless stop (Algorithm 2): j >= n_min, p_j != p_{j-1} and
    e_j > C e_{j-2}^2, with the reading j >= 2 (e_{j-2} and p_{j-1} must exist).
    Idempotency stop: e_j < idem_tol.

    ``input_pattern``: the set of stored tiles of F (the pattern of X_0 is that
    set plus the diagonal); default all nonzero tiles.
    ``replay_kept``: optional per-iteration kept lists (mask replay) used instead
    of a fresh selection.
    """
    n = F.shape[0]
    lmin, lmax = gershgorin_bounds(F)
    sch = schedule(lmin, lmax, homo_ub, lumo_lb, tau=tau, gamma=gamma, accelerate=accelerate,
                   delta_acc=delta_acc, n_cap=n_cap)
    X = initial_matrix(F, lmin, lmax)
    nb = (n + b - 1) // b
    if input_pattern is None:
        _, tl = upper_tiles(F, b)
        input_pattern = {(i, j) for i, j, v in tl if v != 0.0 or i == j}
    else:
        input_pattern = set(input_pattern) | {(i, i) for i in range(nb)}

    def trunc_step(Xi, ti, pattern, it):
        if replay_kept is not None:
            kept = sorted(replay_kept[it])
            dropped = sorted(pattern - set(kept))
            return kept, apply_drop(Xi, dropped, b)
        _, kept, dropped = truncate_select(Xi, ti, trunc, part=frobinf_part, pattern=pattern, b=b)
        return kept, apply_drop(Xi, dropped, b)

    kept, Xt = trunc_step(X, sch.tau[0], input_pattern, 0)
    kept_hist = [kept]
    e, t = [], []
    squares = 0
    trip = 0
    converged = False
    n_out = None
    for i in range(1, sch.n_max + 2):
        S = Xt @ Xt
        squares += 1
        trip += _triplets(kept, nb)
        R = Xt - S
        e.append(float(np.sqrt(np.sum(R * R))))
        t.append(float(np.trace(Xt) - np.trace(S)))
        j = i - 1
        if stop == "parameterless":
            if j >= max(sch.n_min, 2) and sch.p[j] != sch.p[j - 1] and e[j] > C_STOP * e[j - 2] ** 2:
                converged, n_out = True, j
                break
        elif stop == "idempotency":
            if e[j] < idem_tol:
                converged, n_out = True, j
                break
        else:
            raise ValueError(stop)
        if i == sch.n_max + 1:
            n_out = j
            break
        c0, c1, c2 = poly_coeffs(sch.p[i], sch.alpha[i])
        Xi = c0 * np.eye(n) + c1 * Xt + c2 * S
        pattern = product_pattern(kept, nb)
        kept, Xt = trunc_step(Xi, sch.tau[i], pattern, i)
        kept_hist.append(kept)
    res = SP2Result(D=Xt, n=n_out, e=e, t=t, sched=sch, kept=kept_hist, converged=converged,
                    lmin=lmin, lmax=lmax, squares=squares, tile_triplets=trip)
    res.estimates = homo_lumo_estimates(res, n)
    return res


# ----------------------------------------------------------------------------- Step 3
def _pull_back(sch: Schedule, j: int, x: float) -> float:
    """Invert f_j, ..., f_1 on the branch next to the gap; then undo X_0's map."""
    for i in range(j, 0, -1):
        p, a = sch.p[i], sch.alpha[i]
        y = min(max(x, 0.0), 1.0)
        if p == 1:
            x = (math.sqrt(y) + a - 1.0) / a
        else:
            x = (1.0 - math.sqrt(1.0 - y)) / a
    return sch.lmax - x * (sch.lmax - sch.lmin)


def homo_lumo_estimates(res: SP2Result, n: int):
    """Reading of Section 4 Step 3 (Algorithm 3 of the interior-eigenvalue paper
    is not reproduced here).  Each eigenvalue image x of X~_j adds r = x - x^2 to
    t_j and r^2 to e_j^2.  A step with x^2 (p_j = 1) squares r on the virtual
    side (x near 0) and roughly doubles it on the occupied side, so right after
    it the occupied side carries e_j and t_j; after 2x - x^2 (p_j = 0) the
    virtual side does.  On the dominant side r_max is estimated by
    e_j^2 / t_j (the r-weighted mean of its r values, exact when the leading
    values are equal), x = (1 +/- sqrt(1 - 4 r)) / 2 next to the gap, and x is
    pulled back through f_j..f_1 and X_0's map (each pull-back through a
    squaring step halves the relative error of 1 - x or x).  For each side the
    largest j with e_j above 100 f, t_j and r above 10 f (f = tau_j + sqrt(N) 2^-52,
    the truncation and rounding noise in e_j and t_j) and r < 1/4 is used.
    Returns (homo_estimate, lumo_estimate); a side without such a j gives None."""
    sch = res.sched
    homo = lumo = None
    for j in range(len(res.t) - 1, 0, -1):
        if j >= len(sch.p):
            continue
        f = sch.tau[min(j, len(sch.tau) - 1)] + math.sqrt(n) * 2.0 ** -52
        e, t = res.e[j], res.t[j]
        if not (e > 100.0 * f and t > 10.0 * f):
            continue
        r = e * e / t
        if not (10.0 * f < r < 0.25):
            continue
        if sch.p[j] == 1 and homo is None:
            homo = _pull_back(sch, j, (1.0 + math.sqrt(1.0 - 4.0 * r)) / 2.0)
        elif sch.p[j] == 0 and lumo is None:
            lumo = _pull_back(sch, j, (1.0 - math.sqrt(1.0 - 4.0 * r)) / 2.0)
        if homo is not None and lumo is not None:
            break
    return homo, lumo


# ----------------------------------------------------------------------------- Section 1 / 6: trace-correcting
def sp2_trace_correcting(F: np.ndarray, nocc: int, tau: float = 0.0, stop: str = "parameterless",
                         idem_tol: float = 1e-12, trunc: str = "frobenius", n_cap: int = 100,
                         input_pattern=None, b: int = B, frobinf_part: int = FROBINF_PART) -> SP2Result:
    """The SP2 expansion whose polynomial is chosen from the trace (Section 1:
    the original SP2 algorithm; Section 6: the first run, where nothing is known
    about the eigenvalues).  X_0 maps the occupied eigenvalues near 1 (Algorithm
    1), so x^2 lowers the trace and 2x - x^2 raises it: p_i = 1 iff
    trace(X~_{i-1}) > nocc (a tie takes 2x - x^2).  No acceleration (alpha_i =
    1, n_min = 1), n_max = n_cap, the fixed truncation threshold tau for every
    iteration; truncation, e_i, t_i and the stop tests as in Algorithm 2.
    The returned schedule holds the p_i that were taken, so Step 3 estimates
    follow the same reading as for SP2ACC."""
    n = F.shape[0]
    lmin, lmax = gershgorin_bounds(F)
    sch = Schedule(lmin=lmin, lmax=lmax, n_max=n_cap, n_min=1)
    sch.p.append(-1)
    sch.alpha.append(float("nan"))
    sch.tau = [float(tau)] * (n_cap + 1)
    X = initial_matrix(F, lmin, lmax)
    nb = (n + b - 1) // b
    if input_pattern is None:
        _, tl = upper_tiles(F, b)
        input_pattern = {(i, j) for i, j, v in tl if v != 0.0 or i == j}
    else:
        input_pattern = set(input_pattern) | {(i, i) for i in range(nb)}
    _, kept, dropped = truncate_select(X, tau, trunc, part=frobinf_part, pattern=input_pattern, b=b)
    Xt = apply_drop(X, dropped, b)
    kept_hist = [kept]
    e, t = [], []
    squares = 0
    trip = 0
    converged = False
    n_out = None
    for i in range(1, n_cap + 2):
        if i <= n_cap:
            p = 1 if float(np.trace(Xt)) > nocc else 0
            sch.p.append(p)
            sch.alpha.append(1.0)
        S = Xt @ Xt
        squares += 1
        trip += _triplets(kept, nb)
        R = Xt - S
        e.append(float(np.sqrt(np.sum(R * R))))
        t.append(float(np.trace(Xt) - np.trace(S)))
        j = i - 1
        if stop == "parameterless":
            if j >= 2 and sch.p[j] != sch.p[j - 1] and e[j] > C_STOP * e[j - 2] ** 2:
                converged, n_out = True, j
                break
        elif stop == "idempotency":
            if e[j] < idem_tol:
                converged, n_out = True, j
                break
        else:
            raise ValueError(stop)
        if i == n_cap + 1:
            n_out = j
            break
        c0, c1, c2 = poly_coeffs(sch.p[i], 1.0)
        Xi = c0 * np.eye(n) + c1 * Xt + c2 * S
        pattern = product_pattern(kept, nb)
        _, kept, dropped = truncate_select(Xi, tau, trunc, part=frobinf_part, pattern=pattern, b=b)
        Xt = apply_drop(Xi, dropped, b)
        kept_hist.append(kept)
    res = SP2Result(D=Xt, n=n_out, e=e, t=t, sched=sch, kept=kept_hist, converged=converged,
                    lmin=lmin, lmax=lmax, squares=squares, tile_triplets=trip)
    res.estimates = homo_lumo_estimates(res, n)
    return res


def bounds_from_estimates(homo: float, lumo: float, lmin: float, lmax: float, margin: float = 0.1):
    """Bounds for the second run from the first run's Step 3 estimates (Section
    6).  The estimates are not bounds, so each moves away from the gap by
    margin * (lumo - homo) (a stated reading; the paper gives no margin), and
    stays inside the Gershgorin interval [lmin, lmax]."""
    if homo is None or lumo is None or not (lumo > homo):
        raise ValueError("no usable homo/lumo estimates")
    d = margin * (lumo - homo)
    return max(homo + d, lmin), min(lumo - d, lmax)


def two_run(F: np.ndarray, nocc: int, tau1: float, tau: float = 0.0, gamma: float | None = None,
            margin: float = 0.1, **kw):
    """Section 6: run 1 is the trace-correcting expansion with the threshold
    tau1; its Step 3 estimates, widened by the margin, are the homo/lumo bounds
    of run 2, the SP2ACC expansion (tau or gamma as given).  Returns
    (run1, run2, (homo_ub, lumo_lb))."""
    pattern_kw = {k: kw[k] for k in ("input_pattern", "trunc", "frobinf_part", "n_cap", "stop", "idem_tol")
                  if k in kw}
    r1 = sp2_trace_correcting(F, nocc, tau=tau1, **pattern_kw)
    hub, llb = bounds_from_estimates(r1.estimates[0], r1.estimates[1], r1.lmin, r1.lmax, margin)
    r2 = sp2(F, nocc, hub, llb, tau=tau, gamma=gamma, **kw)
    return r1, r2, (hub, llb)


# ----------------------------------------------------------------------------- adjoint
def adjoint_sp2(F: np.ndarray, res: SP2Result, W: np.ndarray,
                F_pattern_mask: np.ndarray | None = None) -> np.ndarray:
    """Reverse-mode derivative of L = trace(D W) through the recursion (not in
    the paper).  With G = dL/dX for symmetric X and a symmetric step
    X' = c0 I + c1 X + c2 X^2 the chain rule gives G_prev = c1 G + c2 (G X + X G);
    the truncation of each step is a fixed mask (tiles kept), applied to G;
    X_0 = (lmax I - F)/w gives dL/dF = -G_0 / w.  lmin, lmax, alpha_i, p_i and the
    masks are held constant (they are piecewise constant in F).
    Returns dF as a dense array, restricted to ``F_pattern_mask`` if given."""
    sch = res.sched
    n = res.D.shape[0]
    X = initial_matrix(F, res.lmin, res.lmax)
    # recompute the forward iterates with the stored masks
    xs = []
    Xt = _mask_tiles(X, res.kept[0])
    xs.append(Xt)
    for i in range(1, res.n + 1):
        c0, c1, c2 = poly_coeffs(sch.p[i], sch.alpha[i])
        Xi = c0 * np.eye(n) + c1 * Xt + c2 * (Xt @ Xt)
        Xt = _mask_tiles(Xi, res.kept[i])
        xs.append(Xt)
    G = 0.5 * (W + W.T)
    G = _mask_tiles(G, res.kept[res.n])
    for i in range(res.n, 0, -1):
        c0, c1, c2 = poly_coeffs(sch.p[i], sch.alpha[i])
        Xp = xs[i - 1]
        G = c1 * G + c2 * (G @ Xp + Xp @ G)
        G = _mask_tiles(G, res.kept[i - 1])
    dF = -G / (sch.lmax - sch.lmin)
    if F_pattern_mask is not None:
        dF = dF * F_pattern_mask
    return dF


def _mask_tiles(X: np.ndarray, kept, b: int = B) -> np.ndarray:
    e = tile_grid(X.shape[0], b)
    M = np.zeros_like(X)
    for i, j in kept:
        M[e[i]:e[i + 1], e[j]:e[j + 1]] = X[e[i]:e[i + 1], e[j]:e[j + 1]]
        M[e[j]:e[j + 1], e[i]:e[i + 1]] = X[e[j]:e[j + 1], e[i]:e[i + 1]]
    return M
