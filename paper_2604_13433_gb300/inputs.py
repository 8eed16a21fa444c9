"""Seeded synthetic inputs shaped like the paper's test matrices.

This module builds sparse matrices and vectors only. It holds none of the
PackSELL arithmetic (no quantisation, no delta encoding, no packing, no SpMV),
so both the CUDA path and the CPU oracle can take their inputs from it.

Every generator takes an explicit seed and uses numpy's PCG64 generator, so a
run reproduces its inputs exactly.

Workload shapes (paper §5):

* ``poisson5(L)``: 2-D 5-point Dirichlet Laplacian on an L x L grid,
  lexicographic order, diagonal 4 and off-diagonals -1.
* ``stencil27(N, seed)``: the 27-point pattern of the HPCG benchmark on N^3
  (the paper's HPCG_x_y_z matrices, §5.2, Table 2), diagonal 26 and
  off-diagonals -(1 + U(-0.1, 0.1)).
* ``poisson7_varcoef(N, seed)``: 3-D 7-point variable-coefficient Poisson with
  log-normal face coefficients and Dirichlet boundary faces, symmetrically
  scaled to a unit diagonal as the paper scales its solver matrices (§5.2).
* ``poisson5_varcoef(L, seed)``: 2-D 5-point variable-coefficient Poisson,
  unscaled, returned together with its face list so that gradients with
  respect to face coefficients can be formed.
* ``zipf_irregular(n, m, seed)``: non-symmetric matrix with power-law row
  lengths and columns clustered around the diagonal (a high-RSD matrix in the
  sense of §5.1.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """Compressed sparse rows with sorted, strictly increasing columns per row."""

    n: int
    m: int
    rowptr: np.ndarray  # int64 [n + 1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float32 or float64 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def _from_offsets(n: int, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Build CSR from an [n, k] table of candidate columns (-1 = absent).

    The k candidate columns of a row must already be in increasing order.
    """
    mask = cols >= 0
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n=n, m=n, rowptr=rowptr, col=cols[mask].astype(np.int32), val=vals[mask])


# --------------------------------------------------------------------------
# stencils
# --------------------------------------------------------------------------
def poisson5(L: int, dtype=np.float32) -> CSR:
    """5-point Dirichlet Laplacian on an L x L grid; row r*L + c is cell (r, c)."""
    n = L * L
    i = np.arange(n, dtype=np.int64)
    r, c = i // L, i % L
    offs = [(-L, r > 0), (-1, c > 0), (0, np.ones(n, bool)), (1, c < L - 1), (L, r < L - 1)]
    cols = np.full((n, 5), -1, dtype=np.int64)
    vals = np.zeros((n, 5), dtype=dtype)
    for k, (o, ok) in enumerate(offs):
        cols[ok, k] = i[ok] + o
        vals[ok, k] = 4.0 if o == 0 else -1.0
    csr = _from_offsets(n, cols, vals)
    csr.meta = {"kind": "poisson5", "L": L}
    return csr


def stencil27(N, seed: int = 0) -> CSR:
    """HPCG 27-point pattern on an nx x ny x nz grid (row z*ny*nx + y*nx + x).

    ``N`` is an int (cube) or a tuple (nx, ny, nz). Diagonal 26; each
    off-diagonal entry is -(1 + u) with u ~ U(-0.1, 0.1) drawn independently
    per entry, in CSR order.
    """
    nx, ny, nz = (N, N, N) if np.isscalar(N) else tuple(int(v) for v in N)
    n = nx * ny * nz
    i = np.arange(n, dtype=np.int64)
    z, y, x = i // (nx * ny), (i // nx) % ny, i % nx
    cols = np.full((n, 27), -1, dtype=np.int32)
    k = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = ((z + dz >= 0) & (z + dz < nz) & (y + dy >= 0) & (y + dy < ny)
                      & (x + dx >= 0) & (x + dx < nx))
                cols[ok, k] = (i[ok] + dz * nx * ny + dy * nx + dx).astype(np.int32)
                k += 1
    del z, y, x
    mask = cols >= 0
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[mask]
    del cols, mask
    rng = _rng(seed)
    u = rng.uniform(-0.1, 0.1, size=col.size)
    val = (-(1.0 + u)).astype(np.float32)
    del u
    row = np.repeat(np.arange(n, dtype=np.int64), counts)
    val[col == row] = 26.0
    csr = CSR(n=n, m=n, rowptr=rowptr, col=col, val=val)
    csr.meta = {"kind": "stencil27", "grid": (nx, ny, nz), "seed": seed}
    return csr


def _face_coefficients(shape_faces, rng, sigma):
    return np.exp(sigma * rng.standard_normal(shape_faces))


def poisson7_varcoef(N: int, seed: int = 0, sigma: float = 1.0, scale: bool = True) -> CSR:
    """7-point variable-coefficient Poisson on N^3 with Dirichlet boundary faces.

    A = sum_f theta_f (e_u - e_v)(e_u - e_v)^T + sum_b theta_b e_u e_u^T with
    theta ~ exp(N(0, sigma^2)) per interior face f = (u, v) and per boundary
    face b of cell u. The result is SPD. With ``scale`` the matrix is returned
    as G^-1 A G^-1 with g_i = sqrt(a_ii) (unit diagonal), the symmetric
    scaling the paper applies to every solver matrix (§5.2). Values float64.
    """
    n = N ** 3
    rng = _rng(seed)
    thx = _face_coefficients((N, N, N - 1), rng, sigma)  # (z, y, x)-(z, y, x+1)
    thy = _face_coefficients((N, N - 1, N), rng, sigma)
    thz = _face_coefficients((N - 1, N, N), rng, sigma)
    bnd = [_face_coefficients((N, N), rng, sigma) for _ in range(6)]
    diag = np.zeros((N, N, N))
    diag[:, :, :-1] += thx
    diag[:, :, 1:] += thx
    diag[:, :-1, :] += thy
    diag[:, 1:, :] += thy
    diag[:-1, :, :] += thz
    diag[1:, :, :] += thz
    diag[:, :, 0] += bnd[0]
    diag[:, :, -1] += bnd[1]
    diag[:, 0, :] += bnd[2]
    diag[:, -1, :] += bnd[3]
    diag[0, :, :] += bnd[4]
    diag[-1, :, :] += bnd[5]
    # coefficient of the face to the +1 neighbour in each axis, 0 where absent
    cx = np.zeros((N, N, N)); cx[:, :, :-1] = thx
    cy = np.zeros((N, N, N)); cy[:, :-1, :] = thy
    cz = np.zeros((N, N, N)); cz[:-1, :, :] = thz
    del thx, thy, thz, bnd
    cx, cy, cz, diag = (a.reshape(n) for a in (cx, cy, cz, diag))
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    cols = np.full((n, 7), -1, dtype=np.int32)
    vals = np.zeros((n, 7))
    plan = [
        (-N * N, z > 0, lambda ok: cz[i[ok] - N * N]),
        (-N, y > 0, lambda ok: cy[i[ok] - N]),
        (-1, x > 0, lambda ok: cx[i[ok] - 1]),
        (0, None, None),
        (1, x < N - 1, lambda ok: cx[i[ok]]),
        (N, y < N - 1, lambda ok: cy[i[ok]]),
        (N * N, z < N - 1, lambda ok: cz[i[ok]]),
    ]
    for k, (o, ok, coef) in enumerate(plan):
        if o == 0:
            cols[:, k] = i.astype(np.int32)
            vals[:, k] = diag
        else:
            cols[ok, k] = (i[ok] + o).astype(np.int32)
            vals[ok, k] = -coef(ok)
    del x, y, z, cx, cy, cz
    if scale:
        g = np.sqrt(diag)
        safe = np.where(cols >= 0, cols, 0)
        vals = vals / g[:, None] / g[safe]
        del safe
    csr = _from_offsets(n, cols, vals)
    csr.meta = {"kind": "poisson7_varcoef", "N": N, "seed": seed, "sigma": sigma,
                "scaled": scale}
    return csr


def poisson5_varcoef(L: int, seed: int = 0, sigma: float = 0.5):
    """2-D 5-point variable-coefficient Poisson on L x L, with its face list.

    Returns (csr, faces) where csr has float64 values and ``faces`` is a dict:

    * ``u``, ``v``: int64 [F] cells of interior face f (u < v);
    * ``pos_uu``, ``pos_vv``, ``pos_uv``, ``pos_vu``: int64 [F] CSR positions
      of a_uu, a_vv, a_uv, a_vu;
    * ``bu``: int64 [B] cell of boundary face b; ``pos_b``: CSR position of
      a_{bu,bu};
    * ``theta``: float64 [F + B] coefficients, interior faces first.

    A = sum_f theta_f (e_u - e_v)(e_u - e_v)^T + sum_b theta_b e_bu e_bu^T,
    theta ~ exp(N(0, sigma^2)).
    """
    n = L * L
    rng = _rng(seed)
    th_h = np.exp(sigma * rng.standard_normal((L, L - 1)))  # (r, c)-(r, c+1)
    th_v = np.exp(sigma * rng.standard_normal((L - 1, L)))  # (r, c)-(r+1, c)
    th_b = np.exp(sigma * rng.standard_normal(4 * L))  # left, right, top, bottom
    idx = np.arange(n, dtype=np.int64).reshape(L, L)
    u_h, v_h = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    u_v, v_v = idx[:-1, :].ravel(), idx[1:, :].ravel()
    u = np.concatenate([u_h, u_v])
    v = np.concatenate([v_h, v_v])
    th_f = np.concatenate([th_h.ravel(), th_v.ravel()])
    bu = np.concatenate([idx[:, 0], idx[:, -1], idx[0, :], idx[-1, :]])
    base = poisson5(L, dtype=np.float64)
    rowptr, col = base.rowptr, base.col
    val = np.zeros(base.nnz)
    # CSR position of (r, c): rows and columns are sorted, so the key r*n + c
    # is increasing along the CSR arrays and a binary search finds it
    row_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    key = row_of * n + col.astype(np.int64)  # sorted, since rows and cols are

    def find(r, c):
        p = np.searchsorted(key, r * n + c)
        assert np.all(key[p] == r * n + c)
        return p

    pos_uu, pos_vv = find(u, u), find(v, v)
    pos_uv, pos_vu = find(u, v), find(v, u)
    pos_b = find(bu, bu)
    np.add.at(val, pos_uu, th_f)
    np.add.at(val, pos_vv, th_f)
    np.add.at(val, pos_uv, -th_f)
    np.add.at(val, pos_vu, -th_f)
    np.add.at(val, pos_b, th_b)
    csr = CSR(n=n, m=n, rowptr=rowptr, col=col, val=val)
    csr.meta = {"kind": "poisson5_varcoef", "L": L, "seed": seed, "sigma": sigma}
    faces = {"u": u, "v": v, "pos_uu": pos_uu, "pos_vv": pos_vv, "pos_uv": pos_uv,
             "pos_vu": pos_vu, "bu": bu, "pos_b": pos_b,
             "theta": np.concatenate([th_f, th_b])}
    return csr, faces


# --------------------------------------------------------------------------
# irregular (high-RSD) matrices
# --------------------------------------------------------------------------
def _zipf_lengths(rng, n, a, lmax):
    k = np.arange(1, lmax + 1, dtype=np.float64)
    p = k ** (-a)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    return (np.searchsorted(cdf, rng.random(n), side="right") + 1).astype(np.int64)


def zipf_irregular(n: int, m: int | None = None, seed: int = 0, zipf_a: float = 2.0,
                   max_len: int = 4096, sigma_col: float = 1000.0,
                   frac_uniform: float = 0.05) -> CSR:
    """Non-symmetric irregular matrix with power-law row lengths.

    Row length L_i ~ Zipf(zipf_a) truncated to [1, max_len] (clamped to m).
    Each column is, with probability 1 - frac_uniform, round(N(i, sigma_col))
    clamped to [0, m), else uniform on [0, m). Duplicates within a row are
    redrawn until the row has L_i distinct columns. Values N(0, 1) float32.
    """
    m = n if m is None else m
    rng = _rng(seed)
    lengths = np.minimum(_zipf_lengths(rng, n, zipf_a, max_len), m)
    total = int(lengths.sum())
    row = np.repeat(np.arange(n, dtype=np.int64), lengths)

    def draw(rows):
        g = np.rint(rows + sigma_col * rng.standard_normal(rows.size))
        g = np.clip(g, 0, m - 1).astype(np.int64)
        uni = rng.random(rows.size) < frac_uniform
        g[uni] = rng.integers(0, m, size=int(uni.sum()))
        return g

    key = row * m + draw(row)
    for it in range(60):
        key.sort()
        dup = np.zeros(total, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        rows = key[dup] // m
        key[dup] = rows * m + (draw(rows) if it < 40 else rng.integers(0, m, size=nd))
    else:
        # rows that still repeat a column (nearly full rows of small matrices)
        # are drawn again whole, as a uniform subset without replacement
        key.sort()
        dup = np.zeros(total, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        rowptr0 = np.concatenate([[0], np.cumsum(lengths)])
        for r in np.unique(key[dup] // m):
            a, b = rowptr0[r], rowptr0[r + 1]
            key[a:b] = r * m + np.sort(rng.choice(m, size=b - a, replace=False))
        key.sort()
    col = key % m
    del key, row
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=rowptr[1:])
    val = rng.standard_normal(total).astype(np.float32)
    csr = CSR(n=n, m=m, rowptr=rowptr, col=col.astype(np.int32), val=val)
    csr.meta = {"kind": "zipf_irregular", "seed": seed, "zipf_a": zipf_a,
                "max_len": max_len, "sigma_col": sigma_col, "frac_uniform": frac_uniform}
    return csr


def zipf_batch(count: int = 256, seed: int = 0, nmin: int = 1000, nmax: int = 100000):
    """``count`` irregular square matrices with log-uniform sizes in [nmin, nmax]."""
    rng = _rng(seed)
    sizes = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=count)).astype(np.int64)
    seeds = rng.integers(0, 2 ** 31, size=count)
    return [zipf_irregular(int(s), seed=int(sd), sigma_col=min(1000.0, s / 8.0))
            for s, sd in zip(sizes, seeds)]


def poisson5_varcoef_batch(count: int = 512, seed: int = 6, lmin: int = 32, lmax: int = 256,
                           sigma: float = 0.5):
    """``count`` SPD 5-point variable-coefficient systems on L x L grids, L
    uniform on [lmin, lmax], assembled block-diagonally. Returns (csr, parts):
    csr has the block-diagonal pattern and values; parts holds, per system,
    its row offset ``row0``, side ``L``, nonzero offset ``nz0``, face dict
    (positions local to the system) and the seed it was drawn with, plus the
    concatenated global position arrays ``pos_uu/vv/uv/vu`` (interior faces of
    every system, in system order), ``pos_b`` (boundary terms) and
    ``theta_f``/``theta_b`` (their coefficients)."""
    rng = _rng(seed)
    sides = rng.integers(lmin, lmax + 1, size=count)
    rows, cols, vals, systems = [], [], [], []
    glob = {k: [] for k in ("pos_uu", "pos_vv", "pos_uv", "pos_vu", "pos_b")}
    th_f, th_b = [], []
    r0 = z0 = 0
    for i, L in enumerate(sides):
        c, f = poisson5_varcoef(int(L), seed=1000 + i, sigma=sigma)
        rows.append(c.rowptr[:-1] + z0)
        cols.append(c.col.astype(np.int64) + r0)
        vals.append(c.val)
        for k in glob:
            glob[k].append(f[k] + z0)
        F = f["u"].size
        th_f.append(f["theta"][:F])
        th_b.append(f["theta"][F:])
        systems.append({"row0": r0, "L": int(L), "nz0": z0, "faces": f, "csr": c})
        r0 += c.n
        z0 += c.nnz
    rowptr = np.append(np.concatenate(rows), z0).astype(np.int64)
    csr = CSR(n=r0, m=r0, rowptr=rowptr, col=np.concatenate(cols).astype(np.int32),
              val=np.concatenate(vals), meta={"kind": "poisson5_varcoef_batch", "count": count})
    parts = {k: np.concatenate(v) for k, v in glob.items()}
    parts.update(theta_f=np.concatenate(th_f), theta_b=np.concatenate(th_b), systems=systems)
    return csr, parts


# --------------------------------------------------------------------------
# vectors and small random matrices
# --------------------------------------------------------------------------
def uniform(n: int, seed: int = 0, lo: float = -1.0, hi: float = 1.0, dtype=np.float32):
    return _rng(seed).uniform(lo, hi, size=n).astype(dtype)


def normal(n: int, seed: int = 0, std: float = 1.0, dtype=np.float64):
    return (std * _rng(seed).standard_normal(n)).astype(dtype)


def random_csr(n: int, m: int, density: float, seed: int = 0, dtype=np.float32,
               empty_rows: float = 0.0, long_gaps: bool = False) -> CSR:
    """Small random CSR for edge-case tests.

    ``empty_rows`` is the fraction of rows forced empty; ``long_gaps`` spreads
    columns over the whole range so that deltas overflow small delta fields.
    """
    rng = _rng(seed)
    dense = rng.random((n, m)) < density
    if long_gaps and m > 4:
        dense[:, : m // 2] &= rng.random((n, m // 2)) < 0.2
    if empty_rows > 0:
        dense[rng.random(n) < empty_rows, :] = False
    r, c = np.nonzero(dense)
    counts = np.bincount(r, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    val = rng.standard_normal(r.size).astype(dtype)
    return CSR(n=n, m=m, rowptr=rowptr, col=c.astype(np.int32), val=val,
               meta={"kind": "random", "seed": seed})


def spd_from_pattern(csr: CSR, shift: float = 1.0) -> CSR:
    """Make a symmetric, strictly diagonally dominant (hence SPD) matrix.

    Input pattern is symmetrised; off-diagonals are -|a|, the diagonal is the
    absolute row sum plus ``shift``. Values float64.
    """
    n = csr.n
    row = np.repeat(np.arange(n, dtype=np.int64), csr.row_lengths())
    col = csr.col.astype(np.int64)
    keep = col < n
    r = np.concatenate([row[keep], col[keep], np.arange(n)])
    c = np.concatenate([col[keep], row[keep], np.arange(n)])
    w = np.concatenate([np.abs(csr.val[keep]), np.abs(csr.val[keep]), np.zeros(n)])
    key = r * n + c
    order = np.argsort(key, kind="stable")
    key, w = key[order], w[order]
    uk, first = np.unique(key, return_index=True)
    wsum = np.add.reduceat(w, first)
    ur, uc = uk // n, uk % n
    off = ur != uc
    val = np.where(off, -0.5 * wsum, 0.0)
    rowsum = np.bincount(ur[off], weights=-val[off], minlength=n)
    val[~off] = rowsum[ur[~off]] + shift
    counts = np.bincount(ur, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n=n, m=n, rowptr=rowptr, col=uc.astype(np.int32), val=val,
               meta={"kind": "spd_from_pattern"})


def diag_scaled(csr: CSR) -> CSR:
    """The symmetric diagonal scaling the paper applies before its solver runs
    (§5.2): G^-1 A G^-1 with g_i = sqrt(|a_ii|) (1 where the diagonal is
    absent), values in float64."""
    row = np.repeat(np.arange(csr.n), np.diff(csr.rowptr))
    val = np.asarray(csr.val, np.float64)
    d = np.ones(csr.n)
    on = csr.col == row
    d[row[on]] = np.abs(val[on])
    d[d == 0] = 1.0
    g = 1.0 / np.sqrt(d)
    out = CSR(n=csr.n, m=csr.m, rowptr=csr.rowptr, col=csr.col, val=val * g[row] * g[csr.col])
    out.meta = dict(csr.meta, scaled=True)
    return out
