"""Seeded synthetic inputs: stencil matrices in CSR form and right-hand sides.

This module is the one place that both the CUDA path's tests/benchmark and the
oracle's tests draw their inputs from.  It holds none of the solver's
arithmetic (no SpMV, factorisation, level scheduling or Krylov step); it only
assembles matrices and vectors from a documented recipe with numpy's PCG64
generator (``numpy.random.default_rng(seed)``).

The workloads stand in for the paper's test matrices (Section 3: the
3D_Poisson 150^3 matrix of Table 2, and reservoir-like diffusion systems):

* ``poisson2d_5pt(N)`` / ``poisson3d_7pt(N)`` -- constant-coefficient Poisson,
  unscaled (diagonal 4 / 6, off-diagonals -1), Dirichlet boundary, natural
  lexicographic order with x fastest.
* ``diffusion2d_5pt_lognormal`` / ``diffusion3d_7pt_lognormal`` -- cell-centred
  finite-volume diffusion with one coefficient kappa_f = exp(sigma * g),
  g ~ N(0, 1), per cell face (boundary faces included).  A_ij = -kappa_f for the
  face shared by cells i and j; A_ii = sum of the kappa of all faces of cell i
  (a boundary face acts as a Dirichlet face).  The result is symmetric, an
  M-matrix and positive definite.
* ``stencil27_irregular`` -- 27-point stencil with off-diagonals -1, plus a
  fraction of rows that receive extra random off-diagonal entries (values
  N(0, variance)), with the diagonal set to a multiple of the off-diagonal
  absolute row sum (strictly diagonally dominant).
* ``rhs_uniform(n, seed)`` -- right-hand side uniform on [-1, 1].
* ``stencil27_lognormal(N, sigma, seed)`` -- symmetric 27-point coupling on
  N^3 with one log-normal coefficient per neighbour pair (and per missing
  neighbour at the boundary, added to the diagonal only): an M-matrix,
  symmetric positive definite.
* ``serving_requests(count, seed)`` -- the request mix of the serving
  workload (sizes log-uniform, stencil and ILU level drawn per request).
* ``batch_diffusion2d(nsys, smin, smax, sigma, seed)`` -- a batch of
  independent 2D log-normal diffusion systems with square sides drawn
  uniformly from [smin, smax], concatenated (system offsets, int64 row
  pointers, local column indices).

All matrices come back as ``(row_ptr int32[n+1], col int32[nnz], val
float64[nnz])`` with strictly ascending column indices in every row and the
diagonal present.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR",
    "poisson2d_5pt",
    "poisson3d_7pt",
    "diffusion2d_5pt_lognormal",
    "diffusion3d_7pt_lognormal",
    "stencil27_irregular",
    "rhs_uniform",
    "tridiagonal",
    "random_sparse",
    "batch_diffusion2d",
    "Batch",
    "stencil27_lognormal",
    "serving_requests",
    "serving_matrix",
]


class CSR:
    """A square CSR matrix: ``row_ptr`` (int32, n+1), ``col`` (int32), ``val`` (float64)."""

    __slots__ = ("n", "row_ptr", "col", "val")

    def __init__(self, row_ptr, col, val):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _assemble(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Sort (row, col) pairs and build CSR.  Pairs must be unique."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    vals = vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return CSR(row_ptr.astype(np.int32), cols.astype(np.int32), vals)


def _stencil_csr(dims, offsets, weights) -> CSR:
    """Constant-coefficient stencil on a box grid (x fastest), Dirichlet.

    ``offsets`` are per-axis displacement tuples (dx, dy[, dz]); ``weights``
    the matrix value for each.  Offsets are visited in ascending linear
    order so columns come out sorted without a sort.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    nd = len(dims)
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    lin = [sum(o[a] * strides[a] for a in range(nd)) for o in offsets]
    order = np.argsort(lin, kind="stable")
    coords = np.unravel_index(np.arange(n), dims[::-1])[::-1]  # coords[a] for axis a (x first)
    rows_l, cols_l, vals_l = [], [], []
    idx = np.arange(n, dtype=np.int64)
    for oi in order:
        o = offsets[oi]
        mask = np.ones(n, dtype=bool)
        for a in range(nd):
            c = coords[a] + o[a]
            mask &= (c >= 0) & (c < dims[a])
        r = idx[mask]
        rows_l.append(r)
        cols_l.append(r + lin[oi])
        vals_l.append(np.full(r.shape[0], weights[oi], dtype=np.float64))
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = np.concatenate(vals_l)
    return _assemble(n, rows, cols, vals)


def poisson2d_5pt(N: int) -> CSR:
    """2D 5-point Poisson on an N x N grid: n = N^2, nnz = 5N^2 - 4N."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    w = [4.0, -1.0, -1.0, -1.0, -1.0]
    return _stencil_csr((N, N), offs, w)


def poisson3d_7pt(N: int) -> CSR:
    """3D 7-point Poisson on an N^3 grid: n = N^3, nnz = 7N^3 - 6N^2."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    w = [6.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0]
    return _stencil_csr((N, N, N), offs, w)


def _face_assembly(dims, faces) -> CSR:
    """Finite-volume assembly from per-axis face coefficient arrays.

    ``faces[a]`` has the grid shape (z, y, x order, reversed dims) with axis
    a extended by one: face index f along axis a sits between cells f-1 and
    f; faces 0 and dims[a] are boundary faces.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    shape = dims[::-1]  # numpy shape, slowest axis first
    diag = np.zeros(shape, dtype=np.float64)
    rows_l, cols_l, vals_l = [], [], []
    idx = np.arange(n, dtype=np.int64).reshape(shape)
    for a in range(nd):
        ax = nd - 1 - a  # numpy axis for grid axis a
        k = faces[a]
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[ax] = slice(0, dims[a])
        hi[ax] = slice(1, dims[a] + 1)
        diag += k[tuple(lo)] + k[tuple(hi)]
        inner = [slice(None)] * nd
        inner[ax] = slice(1, dims[a])
        kin = k[tuple(inner)]  # faces between cell f-1 and f, f = 1..dims-1
        left = [slice(None)] * nd
        right = [slice(None)] * nd
        left[ax] = slice(0, dims[a] - 1)
        right[ax] = slice(1, dims[a])
        il = idx[tuple(left)].ravel()
        ir = idx[tuple(right)].ravel()
        kv = kin.ravel()
        rows_l += [il, ir]
        cols_l += [ir, il]
        vals_l += [-kv, -kv]
    rows_l.append(idx.ravel())
    cols_l.append(idx.ravel())
    vals_l.append(diag.ravel())
    return _assemble(n, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(vals_l))


def diffusion2d_5pt_lognormal(N: int, sigma: float, seed: int, Ny: int | None = None) -> CSR:
    """2D 5-point diffusion, log-normal(0, sigma) face coefficients.

    Draw order from ``default_rng(seed)``: x-faces (shape Ny x (N+1)), then
    y-faces ((Ny+1) x N), each as standard normals scaled by sigma.
    """
    Nx, Ny = int(N), int(N if Ny is None else Ny)
    rng = np.random.default_rng(seed)
    fx = np.exp(sigma * rng.standard_normal((Ny, Nx + 1)))
    fy = np.exp(sigma * rng.standard_normal((Ny + 1, Nx)))
    return _face_assembly((Nx, Ny), [fx, fy])


def diffusion3d_7pt_lognormal(N: int, sigma: float, seed: int) -> CSR:
    """3D 7-point diffusion on N^3 with log-normal(0, sigma) face coefficients.

    Draw order from ``default_rng(seed)``: x-faces (N, N, N+1), y-faces
    (N, N+1, N), z-faces (N+1, N, N), numpy shapes in (z, y, x) order.
    n = N^3, nnz = 7N^3 - 6N^2.
    """
    rng = np.random.default_rng(seed)
    fx = np.exp(sigma * rng.standard_normal((N, N, N + 1)))
    fy = np.exp(sigma * rng.standard_normal((N, N + 1, N)))
    fz = np.exp(sigma * rng.standard_normal((N + 1, N, N)))
    return _face_assembly((N, N, N), [fx, fy, fz])


def stencil27_irregular(N: int, struct_seed: int, value_seed: int, frac: float = 0.02,
                        extra_min: int = 30, extra_max: int = 120, variance: float = 0.01,
                        diag_factor: float = 1.1) -> CSR:
    """3D 27-point stencil (off-diagonals -1) on N^3 plus irregular rows.

    ``round(frac * n)`` rows, chosen uniformly without replacement with
    ``default_rng(struct_seed)``, each receive U{extra_min..extra_max} extra
    distinct off-diagonal columns drawn uniformly among the columns the row
    does not hold yet.  Their values are N(0, variance) from
    ``default_rng(value_seed)`` (variance, i.e. standard deviation
    sqrt(variance)).  The diagonal is diag_factor times the off-diagonal
    absolute row sum.
    """
    offs, w = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offs.append((dx, dy, dz))
                w.append(0.0 if (dx, dy, dz) == (0, 0, 0) else -1.0)
    base = _stencil_csr((N, N, N), offs, w)
    n = base.n
    srng = np.random.default_rng(struct_seed)
    vrng = np.random.default_rng(value_seed)
    nrows = int(round(frac * n))
    chosen = np.sort(srng.choice(n, size=nrows, replace=False))
    counts = srng.integers(extra_min, extra_max + 1, size=nrows)
    ex_rows, ex_cols = [], []
    for r, c in zip(chosen.tolist(), counts.tolist()):
        have = set(base.col[base.row_ptr[r]:base.row_ptr[r + 1]].tolist())
        picked: list[int] = []
        while len(picked) < c:
            cand = srng.integers(0, n, size=2 * c)
            for j in cand.tolist():
                if j not in have:
                    have.add(j)
                    picked.append(j)
                    if len(picked) == c:
                        break
        ex_rows.append(np.full(c, r, dtype=np.int64))
        ex_cols.append(np.asarray(picked, dtype=np.int64))
    ex_rows = np.concatenate(ex_rows) if ex_rows else np.zeros(0, np.int64)
    ex_cols = np.concatenate(ex_cols) if ex_cols else np.zeros(0, np.int64)
    ex_vals = vrng.normal(0.0, np.sqrt(variance), size=ex_rows.shape[0])
    brows = np.repeat(np.arange(n, dtype=np.int64), np.diff(base.row_ptr))
    rows = np.concatenate([brows, ex_rows])
    cols = np.concatenate([base.col.astype(np.int64), ex_cols])
    vals = np.concatenate([base.val, ex_vals])
    offdiag = rows != cols
    absrow = np.bincount(rows[offdiag], weights=np.abs(vals[offdiag]), minlength=n)
    vals = np.where(offdiag, vals, diag_factor * absrow[rows])
    return _assemble(n, rows, cols, vals)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform on [-1, 1] from ``default_rng(seed)``."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def tridiagonal(n: int, seed: int) -> CSR:
    """Random strictly diagonally dominant tridiagonal matrix (nonsymmetric)."""
    rng = np.random.default_rng(seed)
    lo = rng.uniform(-1.0, 1.0, n - 1)
    up = rng.uniform(-1.0, 1.0, n - 1)
    d = 2.5 + rng.uniform(0.0, 1.0, n)
    rows = np.concatenate([np.arange(1, n), np.arange(n), np.arange(n - 1)])
    cols = np.concatenate([np.arange(n - 1), np.arange(n), np.arange(1, n)])
    vals = np.concatenate([lo, d, up])
    return _assemble(n, rows.astype(np.int64), cols.astype(np.int64), vals)


def random_sparse_rows(n: int, per_row: int, seed: int, dominance: float = 1.5) -> CSR:
    """Random nonsymmetric sparse matrix for large n: every row draws
    ``per_row`` off-diagonal columns uniformly (duplicates merged), values
    uniform on [-1, 1], diagonal ``dominance`` * off-diagonal abs row sum + 1."""
    rng = np.random.default_rng(seed)
    r = np.repeat(np.arange(n, dtype=np.int64), per_row)
    c = rng.integers(0, n, size=r.shape[0])
    keep = r != c
    r, c = r[keep], c[keep]
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    v = rng.uniform(-1.0, 1.0, size=r.shape[0])
    absrow = np.bincount(r, weights=np.abs(v), minlength=n)
    rows = np.concatenate([r, np.arange(n)])
    cols = np.concatenate([c, np.arange(n)])
    vals = np.concatenate([v, dominance * absrow + 1.0])
    return _assemble(n, rows, cols, vals)


def random_powerlaw_rows(n: int, scale: float, alpha: float, max_len: int, seed: int,
                         dominance: float = 1.5) -> CSR:
    """Random nonsymmetric sparse matrix whose row lengths are heavy-tailed,
    the shape that separates ELL, CSR and hybrid formats: row i draws
    min(max_len, max(1, round(scale * u^(-1/alpha)))) off-diagonal columns
    (u uniform on (0, 1], a Pareto law of shape alpha), uniformly among the
    other columns (duplicates merged); values uniform on [-1, 1]; diagonal
    ``dominance`` * off-diagonal abs row sum + 1."""
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)
    lens = np.minimum(max_len, np.maximum(1, np.rint(scale * u ** (-1.0 / alpha)))).astype(np.int64)
    r = np.repeat(np.arange(n, dtype=np.int64), lens)
    c = rng.integers(0, n, size=r.shape[0])
    keep = r != c
    r, c = r[keep], c[keep]
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    v = rng.uniform(-1.0, 1.0, size=r.shape[0])
    absrow = np.bincount(r, weights=np.abs(v), minlength=n)
    rows = np.concatenate([r, np.arange(n)])
    cols = np.concatenate([c, np.arange(n)])
    vals = np.concatenate([v, dominance * absrow + 1.0])
    return _assemble(n, rows, cols, vals)


def random_sparse(n: int, density: float, seed: int, dominance: float = 1.5,
                  integer: bool = False) -> CSR:
    """Random nonsymmetric sparse matrix with full diagonal.

    Off-diagonal positions are Bernoulli(density); values uniform on [-1, 1]
    (or integers in [-3, 3] \\ {0} if ``integer``).  The diagonal is
    ``dominance`` times the off-diagonal absolute row sum plus one, so every
    ILU(k) of it has nonzero pivots.
    """
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < density
    np.fill_diagonal(mask, False)
    r, c = np.nonzero(mask)
    if integer:
        v = rng.integers(1, 4, size=r.shape[0]) * rng.choice([-1.0, 1.0], size=r.shape[0])
    else:
        v = rng.uniform(-1.0, 1.0, size=r.shape[0])
    absrow = np.bincount(r, weights=np.abs(v), minlength=n)
    d = np.floor(dominance * absrow) + 1.0 if integer else dominance * absrow + 1.0
    rows = np.concatenate([r, np.arange(n)])
    cols = np.concatenate([c, np.arange(n)])
    vals = np.concatenate([v, d])
    return _assemble(n, rows.astype(np.int64), cols.astype(np.int64), vals.astype(np.float64))


class Batch:
    """Independent systems concatenated: system s owns rows
    ``sys_ptr[s]:sys_ptr[s+1]``; ``row_ptr`` (int64) indexes ``col`` (local
    column indices, int32) and ``val``."""

    __slots__ = ("sys_ptr", "row_ptr", "col", "val", "sides")

    def __init__(self, sys_ptr, row_ptr, col, val, sides=None):
        self.sys_ptr = np.ascontiguousarray(sys_ptr, dtype=np.int64)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.sides = sides

    @property
    def nsys(self) -> int:
        return int(self.sys_ptr.shape[0] - 1)

    @property
    def rows(self) -> int:
        return int(self.sys_ptr[-1])

    def system(self, s: int) -> CSR:
        r0, r1 = int(self.sys_ptr[s]), int(self.sys_ptr[s + 1])
        e0 = int(self.row_ptr[r0])
        return CSR(self.row_ptr[r0:r1 + 1] - e0, self.col[e0:self.row_ptr[r1]],
                   self.val[e0:self.row_ptr[r1]])


def batch_diffusion2d(nsys: int, smin: int, smax: int, sigma: float, seed: int) -> Batch:
    """``nsys`` systems ``diffusion2d_5pt_lognormal(s_i, sigma, c_i)``.

    From ``default_rng(seed)``: the sides s_i = integers(smin, smax + 1, nsys)
    (uniform on [smin, smax]), then the coefficient seeds
    c_i = integers(0, 2**31 - 1, nsys).
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(smin, smax + 1, nsys)
    cseeds = rng.integers(0, 2 ** 31 - 1, nsys)
    mats = [diffusion2d_5pt_lognormal(int(n), sigma, int(c)) for n, c in zip(sides, cseeds)]
    ns = np.array([A.n for A in mats], dtype=np.int64)
    nnz = np.array([A.nnz for A in mats], dtype=np.int64)
    sys_ptr = np.zeros(nsys + 1, dtype=np.int64)
    sys_ptr[1:] = np.cumsum(ns)
    eoff = np.zeros(nsys + 1, dtype=np.int64)
    eoff[1:] = np.cumsum(nnz)
    row_ptr = np.empty(int(sys_ptr[-1]) + 1, dtype=np.int64)
    for i, A in enumerate(mats):
        row_ptr[sys_ptr[i]:sys_ptr[i + 1]] = A.row_ptr[:-1].astype(np.int64) + eoff[i]
    row_ptr[-1] = eoff[-1]
    col = np.concatenate([A.col for A in mats])
    val = np.concatenate([A.val for A in mats])
    return Batch(sys_ptr, row_ptr, col, val, sides)


_OFF27 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
          if (dz, dy, dx) > (0, 0, 0)]  # the 13 "forward" neighbour offsets


def stencil27_lognormal(N: int, sigma: float, seed: int) -> CSR:
    """27-point coupling on N^3 (x fastest), log-normal(0, sigma) coefficients.

    From ``default_rng(seed)``: G of shape (13, N, N, N) -- G[o, cell] couples
    cell and cell + offset_o (offsets in the order of ``_OFF27``) -- then H of
    the same shape, the coupling of cell with a missing neighbour at
    cell - offset_o.  Off-diagonal A_ij = -kappa_ij; A_ii = sum of the
    kappa of all 26 neighbour slots of cell i (a slot outside the grid keeps
    its coefficient on the diagonal, like a Dirichlet neighbour).  Both draws
    are exp(sigma * standard normal)."""
    rng = np.random.default_rng(seed)
    G = np.exp(sigma * rng.standard_normal((13, N, N, N)))
    Hh = np.exp(sigma * rng.standard_normal((13, N, N, N)))
    n = N ** 3
    idx = np.arange(n, dtype=np.int64).reshape(N, N, N)  # (z, y, x)
    diag = np.zeros((N, N, N))
    rows_l, cols_l, vals_l = [], [], []
    for o, (dx, dy, dz) in enumerate(_OFF27):
        # forward neighbour: cell + (dx, dy, dz)
        zs = slice(max(0, -dz), N - max(0, dz))
        ys = slice(max(0, -dy), N - max(0, dy))
        xs = slice(max(0, -dx), N - max(0, dx))
        zt = slice(max(0, dz), N - max(0, -dz))
        yt = slice(max(0, dy), N - max(0, -dy))
        xt = slice(max(0, dx), N - max(0, -dx))
        k = G[o][zs, ys, xs]
        a = idx[zs, ys, xs].ravel()
        b = idx[zt, yt, xt].ravel()
        rows_l += [a, b]
        cols_l += [b, a]
        vals_l += [-k.ravel(), -k.ravel()]
        diag[zs, ys, xs] += k
        diag[zt, yt, xt] += k
        # forward slot leaving the grid: G keeps its value on the diagonal
        m = np.ones((N, N, N), dtype=bool)
        m[zs, ys, xs] = False
        diag[m] += G[o][m]
        # backward slot leaving the grid: H
        m = np.ones((N, N, N), dtype=bool)
        m[zt, yt, xt] = False
        diag[m] += Hh[o][m]
    rows_l.append(idx.ravel())
    cols_l.append(idx.ravel())
    vals_l.append(diag.ravel())
    return _assemble(n, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(vals_l))


def serving_requests(count: int, seed: int, nmin: float = 1e3, nmax: float = 1e6):
    """The request mix: from ``default_rng(seed)``, per request in order --
    log10(n) uniform on [log10 nmin, log10 nmax]; stencil uniform over
    (5, 7, 27); ILU level 0 or 1 with probability 1/2; a coefficient seed
    (integers below 2^31 - 1).  The grid side is round(n^(1/d)) (at least 2).
    Returns dicts {stencil, side, n, k, seed}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = 10.0 ** rng.uniform(np.log10(nmin), np.log10(nmax))
        st = int(rng.choice([5, 7, 27]))
        k = int(rng.integers(0, 2))
        cs = int(rng.integers(0, 2 ** 31 - 1))
        d = 2 if st == 5 else 3
        side = max(2, int(round(n ** (1.0 / d))))
        out.append({"stencil": st, "side": side, "n": side ** d, "k": k, "seed": cs})
    return out


def serving_matrix(req, sigma: float = 2.0) -> CSR:
    """The matrix of one request of ``serving_requests``."""
    if req["stencil"] == 5:
        return diffusion2d_5pt_lognormal(req["side"], sigma, req["seed"])
    if req["stencil"] == 7:
        return diffusion3d_7pt_lognormal(req["side"], sigma, req["seed"])
    return stencil27_lognormal(req["side"], sigma, req["seed"])
