"""Seeded synthetic Fock matrices with the shapes of the paper's workloads.

The paper's own matrices (HF/3-21G water clusters, a Glu-Ala helix, Section 6)
are not available, so these generators stand in for them:

* ``dense_gapped``  -- F = Q diag(lam) Q^T with Q from the QR factorisation of
  a seeded N(0,1) matrix (dense reference cases).
* ``water_like``    -- molecules of 24 basis functions placed uniformly at
  random in a cube at 0.0334 molecules per cubic Angstrom, sorted along a 3-D
  Morton curve so that 32x32 tiles are spatially local; diagonal molecule
  blocks Q_b diag(occupied, virtual) Q_b^T; off-diagonal molecule blocks
  N(0,1) * exp(-r / 2 A) for centre distance r < 10 A, scaled once so that
  every row sum of |off-block part| is at most 0.25.
* ``helix_like``    -- the same construction on a 1-D chain (1.5 A spacing,
  64 basis functions per residue, exp(-d / 3 A) for d < 15 A).

Every random draw comes from ``numpy.random.Generator(PCG64(seed))`` in the
order written in each function.  The homo/lumo bounds returned with each
matrix follow from Weyl's inequality: the block-diagonal part has a known
spectrum and the off-block part has spectral norm at most its largest row sum.

Block-sparse layout (the one the C ABI takes): tiles of b x b = 32 x 32, only
tiles with block row I <= block column J are stored, sorted by (I, J); the
values of a tile are row-major; diagonal tiles are stored in full (both
triangles); when N is not a multiple of b the last tile row/column is padded
with zeros.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BLOCK = 32


@dataclass
class BlockSparse:
    """Upper-triangle block-sparse symmetric matrix (see module docstring)."""

    n: int
    brow: np.ndarray  # int32 [nnzb]
    bcol: np.ndarray  # int32 [nnzb]
    val: np.ndarray  # float64 [nnzb, b, b]
    b: int = BLOCK
    meta: dict = field(default_factory=dict)

    @property
    def nb(self) -> int:
        return (self.n + self.b - 1) // self.b

    @property
    def nnzb(self) -> int:
        return int(self.brow.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_dense(m: BlockSparse) -> np.ndarray:
    """Expand the stored upper tiles (and their mirrors) to a dense N x N array."""
    b, nb = m.b, m.nb
    full = np.zeros((nb * b, nb * b))
    for k in range(m.nnzb):
        i, j = int(m.brow[k]), int(m.bcol[k])
        full[i * b:(i + 1) * b, j * b:(j + 1) * b] = m.val[k]
        if i != j:
            full[j * b:(j + 1) * b, i * b:(i + 1) * b] = m.val[k].T
    return full[: m.n, : m.n].copy()


def from_dense(a: np.ndarray, b: int = BLOCK, keep_zero_tiles: bool = False,
               force_diag: bool = True) -> BlockSparse:
    """Tile a dense symmetric array; keeps every upper tile that is not all zero
    (plus all diagonal tiles when ``force_diag``)."""
    n = a.shape[0]
    nb = (n + b - 1) // b
    pad = np.zeros((nb * b, nb * b))
    pad[:n, :n] = a
    tiles = pad.reshape(nb, b, nb, b).transpose(0, 2, 1, 3)
    iu, ju = np.triu_indices(nb)
    t = tiles[iu, ju]
    keep = np.ones(len(iu), dtype=bool) if keep_zero_tiles else np.any(t != 0.0, axis=(1, 2))
    if force_diag:
        keep |= iu == ju
    return BlockSparse(n=n, brow=iu[keep].astype(np.int32), bcol=ju[keep].astype(np.int32),
                       val=np.ascontiguousarray(t[keep]), b=b)


# --------------------------------------------------------------------------- dense
def dense_gapped(n: int, nocc: int, occ: tuple, virt: tuple, seed: int) -> dict:
    """F = Q diag(lam) Q^T.  Draw order: A (n x n standard normal), occupied
    eigenvalues (nocc uniform in ``occ``), virtual eigenvalues (n - nocc
    uniform in ``virt``).  Q from numpy's QR of A."""
    rng = _rng(seed)
    a = rng.standard_normal((n, n))
    lam_occ = rng.uniform(occ[0], occ[1], nocc)
    lam_virt = rng.uniform(virt[0], virt[1], n - nocc)
    q, _ = np.linalg.qr(a)
    lam = np.concatenate([lam_occ, lam_virt])
    f = (q * lam) @ q.T
    f = 0.5 * (f + f.T)
    return dict(F=f, n=n, nocc=nocc, homo_ub=float(lam_occ.max()), lumo_lb=float(lam_virt.min()),
                eigenvalues=np.sort(lam))


# --------------------------------------------------------------------------- molecular
def _morton3(q: np.ndarray) -> np.ndarray:
    """Interleave the bits of three 10-bit integer coordinates."""
    code = np.zeros(q.shape[0], dtype=np.int64)
    for bit in range(10):
        for ax in range(3):
            code |= ((q[:, ax].astype(np.int64) >> bit) & 1) << (3 * bit + ax)
    return code


def _assemble(n: int, nbf: int, diag_blocks: np.ndarray, pairs: np.ndarray, pair_blocks: np.ndarray,
              b: int = BLOCK) -> BlockSparse:
    """Scatter molecule blocks into 32x32 upper tiles.

    diag_blocks: [nmol, nbf, nbf] full symmetric blocks; pairs: [npair, 2] with
    A < B; pair_blocks: [npair, nbf, nbf] = F[rows of A, cols of B]."""
    nmol = diag_blocks.shape[0]
    nb = (n + b - 1) // b
    # tiles touched by each molecule
    first = (np.arange(nmol) * nbf) // b
    last = (np.arange(nmol) * nbf + nbf - 1) // b
    span = int((last - first).max()) + 1
    cand = []
    for di in range(span):
        for dj in range(span):
            ii = first + di
            jj = first + dj
            ok = (ii <= last) & (jj <= last) & (ii <= jj)
            cand.append(np.stack([ii[ok], jj[ok]], axis=1))
            if pairs.shape[0]:
                pa, pb = pairs[:, 0], pairs[:, 1]
                ii = first[pa] + di
                jj = first[pb] + dj
                ok = (ii <= last[pa]) & (jj <= last[pb])
                cand.append(np.stack([ii[ok], jj[ok]], axis=1))
                # mirrored part of a pair can fall into a diagonal tile
                ii = first[pb] + di
                jj = first[pa] + dj
                ok = (ii <= last[pb]) & (jj <= last[pa]) & (ii == jj)
                cand.append(np.stack([ii[ok], jj[ok]], axis=1))
    tiles = np.unique(np.concatenate(cand).astype(np.int64) @ np.array([nb, 1], dtype=np.int64))
    brow = (tiles // nb).astype(np.int32)
    bcol = (tiles % nb).astype(np.int32)
    lookup = np.full(nb * nb, -1, dtype=np.int32)
    lookup[tiles] = np.arange(tiles.shape[0], dtype=np.int32)
    val = np.zeros((tiles.shape[0], b, b))
    flat = val.reshape(-1)
    loc = np.arange(nbf)

    def scatter(r0, c0, blocks, mirror_only_diag=False, transpose=False):
        # r0, c0: [m] first global row / col; blocks [m, nbf, nbf]
        rr = r0[:, None, None] + loc[None, :, None]
        cc = c0[:, None, None] + loc[None, None, :]
        rr, cc = np.broadcast_arrays(rr, cc)
        vv = blocks
        if transpose:
            rr, cc = cc, rr
        ti, tj = rr // b, cc // b
        keep = ti <= tj
        if mirror_only_diag:
            keep = ti == tj
        tid = lookup[ti[keep].astype(np.int64) * nb + tj[keep]]
        flat[tid.astype(np.int64) * (b * b) + (rr[keep] % b) * b + (cc[keep] % b)] = vv[keep]

    chunk = 20000
    r0 = np.arange(nmol) * nbf
    for s in range(0, nmol, chunk):
        scatter(r0[s:s + chunk], r0[s:s + chunk], diag_blocks[s:s + chunk])
    for s in range(0, pairs.shape[0], chunk):
        pa, pb = pairs[s:s + chunk, 0], pairs[s:s + chunk, 1]
        scatter(r0[pa], r0[pb], pair_blocks[s:s + chunk])
        scatter(r0[pa], r0[pb], pair_blocks[s:s + chunk], mirror_only_diag=True, transpose=True)
    return BlockSparse(n=n, brow=brow, bcol=bcol, val=val, b=b)


def _molecular(pos: np.ndarray, rng: np.random.Generator, nbf: int, nocc_per: int, occ: tuple, virt: tuple,
               cutoff: float, decay: float, rowsum: float, pairs: np.ndarray) -> tuple:
    nmol = pos.shape[0]
    # draw order: per molecule (in final order) A_b (nbf x nbf), occupied, virtual eigenvalues
    diag = np.empty((nmol, nbf, nbf))
    occ_max, virt_min = -np.inf, np.inf
    for m in range(nmol):
        a = rng.standard_normal((nbf, nbf))
        lo = rng.uniform(occ[0], occ[1], nocc_per)
        lv = rng.uniform(virt[0], virt[1], nbf - nocc_per)
        q, _ = np.linalg.qr(a)
        lam = np.concatenate([lo, lv])
        blk = (q * lam) @ q.T
        diag[m] = 0.5 * (blk + blk.T)
        occ_max = max(occ_max, lo.max())
        virt_min = min(virt_min, lv.min())
    # then all pair blocks at once, pairs in lexicographic order
    if pairs.shape[0]:
        dist = np.linalg.norm(pos[pairs[:, 0]] - pos[pairs[:, 1]], axis=1)
        blocks = rng.standard_normal((pairs.shape[0], nbf, nbf)) * np.exp(-dist / decay)[:, None, None]
        rs = np.zeros(nmol * nbf)
        absb = np.abs(blocks)
        np.add.at(rs, (pairs[:, 0][:, None] * nbf + np.arange(nbf)[None, :]).ravel(), absb.sum(axis=2).ravel())
        np.add.at(rs, (pairs[:, 1][:, None] * nbf + np.arange(nbf)[None, :]).ravel(), absb.sum(axis=1).ravel())
        maxrow = float(rs.max())
        scale = min(1.0, rowsum / maxrow) if maxrow > 0 else 1.0
        blocks *= scale
        offnorm = maxrow * scale
    else:
        blocks = np.zeros((0, nbf, nbf))
        offnorm = 0.0
    return diag, blocks, float(occ_max + offnorm), float(virt_min - offnorm)


def water_like(nmol: int, seed: int, density: float = 0.0334, nbf: int = 24, nocc_per: int = 12,
               occ=(-1.5, -0.5), virt=(0.5, 2.5), cutoff: float = 10.0, decay: float = 2.0,
               rowsum: float = 0.25) -> dict:
    """Water-cluster-like F.  Draw order: positions (nmol x 3 uniform in the
    cube), then per molecule (after the Morton sort) its 24x24 normal matrix,
    12 occupied and 12 virtual eigenvalues, then the pair blocks."""
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    side = (nmol / density) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, side, (nmol, 3))
    q = np.clip(np.floor(pos / side * 1024.0), 0, 1023).astype(np.int64)
    order = np.argsort(_morton3(q), kind="stable")
    pos = pos[order]
    pairs = cKDTree(pos).query_pairs(r=cutoff, output_type="ndarray")
    if pairs.shape[0]:
        pairs = np.sort(pairs, axis=1)
        d = np.linalg.norm(pos[pairs[:, 0]] - pos[pairs[:, 1]], axis=1)
        pairs = pairs[d < cutoff]
        pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    diag, blocks, homo_ub, lumo_lb = _molecular(pos, rng, nbf, nocc_per, occ, virt, cutoff, decay, rowsum, pairs)
    n = nmol * nbf
    f = _assemble(n, nbf, diag, pairs, blocks)
    f.meta = dict(kind="water_like", nmol=nmol, side=side, npairs=int(pairs.shape[0]))
    return dict(F=f, n=n, nocc=nmol * nocc_per, homo_ub=homo_ub, lumo_lb=lumo_lb)


def helix_like(nres: int, seed: int, nbf: int = 64, nocc_per: int = 32, spacing: float = 1.5,
               occ=(-1.5, -0.5), virt=(0.5, 2.5), cutoff: float = 15.0, decay: float = 3.0,
               rowsum: float = 0.25) -> dict:
    """Helix-like 1-D chain.  Draw order: per residue its 64x64 normal matrix,
    32 occupied and 32 virtual eigenvalues, then the pair blocks."""
    rng = _rng(seed)
    pos = np.zeros((nres, 3))
    pos[:, 0] = spacing * np.arange(nres)
    reach = int(np.ceil(cutoff / spacing))
    pa, pb = [], []
    for k in range(1, reach + 1):
        if k * spacing < cutoff:
            i = np.arange(nres - k)
            pa.append(i)
            pb.append(i + k)
    pairs = np.stack([np.concatenate(pa), np.concatenate(pb)], axis=1) if pa else np.zeros((0, 2), np.int64)
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    diag, blocks, homo_ub, lumo_lb = _molecular(pos, rng, nbf, nocc_per, occ, virt, cutoff, decay, rowsum, pairs)
    n = nres * nbf
    f = _assemble(n, nbf, diag, pairs, blocks)
    f.meta = dict(kind="helix_like", nres=nres, npairs=int(pairs.shape[0]))
    return dict(F=f, n=n, nocc=nres * nocc_per, homo_ub=homo_ub, lumo_lb=lumo_lb)


def random_symmetric_on_pattern(m: BlockSparse, seed: int) -> BlockSparse:
    """Seeded symmetric N(0,1) matrix on the tile pattern of ``m`` (padding zero)."""
    rng = _rng(seed)
    val = rng.standard_normal(m.val.shape)
    diag = m.brow == m.bcol
    val[diag] = 0.5 * (val[diag] + val[diag].transpose(0, 2, 1))
    pad = m.nb * m.b - m.n
    if pad:
        last = m.nb - 1
        val[m.bcol == last, :, m.b - pad:] = 0.0
        val[m.brow == last, m.b - pad:, :] = 0.0
    return BlockSparse(n=m.n, brow=m.brow.copy(), bcol=m.bcol.copy(), val=val, b=m.b)


# --------------------------------------------------------------------------- configs
SEED_BASE = 1909_12533 * 10

CONFIGS = {
    # the five workloads
    1: dict(kind="dense", n=512, nocc=256, occ=(-2.0, -0.5), virt=(0.5, 3.0), tau=0.0, stop="idempotency"),
    2: dict(kind="water", nmol=1000, tau=1e-6, stop="parameterless"),
    3: dict(kind="water", nmol=8000, tau=1e-5, stop="parameterless"),
    4: dict(kind="helix", nres=2000, tau=1e-6, stop="parameterless"),
    5: dict(kind="dense", n=16384, nocc=8192, occ=(-2.0, -0.025), virt=(0.025, 3.0), tau=0.0, stop="idempotency"),
    # reduced versions of the same recipes, small enough for the CPU oracle
    "2s": dict(kind="water", nmol=101, tau=1e-6, stop="parameterless"),
    "2m": dict(kind="water", nmol=400, tau=1e-6, stop="parameterless"),
    # the precision form's threshold on 1000 molecules (profiling size)
    "3m": dict(kind="water", nmol=1000, tau=1e-5, stop="parameterless"),
    "3s": dict(kind="water", nmol=203, tau=1e-5, stop="parameterless"),
    "4s": dict(kind="helix", nres=64, tau=1e-6, stop="parameterless"),
    "5s": dict(kind="dense", n=1000, nocc=500, occ=(-2.0, -0.025), virt=(0.025, 3.0), tau=0.0, stop="idempotency"),
}


def _seed_of(key) -> int:
    if isinstance(key, int):
        return SEED_BASE + key
    return SEED_BASE + 100 + int(str(key)[0])


def make_config(key, seed: int | None = None) -> dict:
    """Build one of ``CONFIGS`` (integers are the five workloads, "Ns" their
    reduced versions).  Returns a dict with F (dense array for kind="dense",
    BlockSparse otherwise), n, nocc, homo_ub, lumo_lb, tau and stop."""
    c = CONFIGS[key]
    s = _seed_of(key) if seed is None else seed
    if c["kind"] == "dense":
        out = dense_gapped(c["n"], c["nocc"], c["occ"], c["virt"], s)
    elif c["kind"] == "water":
        out = water_like(c["nmol"], s)
    else:
        out = helix_like(c["nres"], s)
    out.update(tau=c["tau"], stop=c["stop"], key=key, seed=s)
    return out
