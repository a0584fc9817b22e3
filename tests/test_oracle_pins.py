"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types an oracle formula: each compares the oracle with
a closed form, a brute-force literal execution on tiny inputs, a textbook or
library routine in a case where the method reduces to it exactly, or an
invariant.  They run without a GPU.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1606_00545_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers
def dense_iluk_literal(Ad, pattern, k):
    """Algorithm 2 executed literally on dense arrays (brute force, O(n^3)).

    Levels follow Eq. 9 (0 on the pattern, infinity elsewhere) and Eq. 10;
    after the p loop of row i the positions with level > k are zeroed and
    their level reset to infinity.
    """
    A = Ad.astype(np.float64).copy()
    n = A.shape[0]
    L = np.where(pattern, 0.0, np.inf)
    for i in range(1, n):
        for p in range(i):
            if L[i, p] <= k:
                A[i, p] = A[i, p] / A[p, p]
                A[i, p + 1:] = A[i, p + 1:] - A[i, p] * A[p, p + 1:]
                L[i, p + 1:] = np.minimum(L[i, p + 1:], L[i, p] + L[p, p + 1:] + 1)
        drop = L[i, :] > k
        A[i, drop] = 0.0
        L[i, drop] = np.inf
    return A, L


def pattern_of(A):
    P = np.zeros((A.n, A.n), dtype=bool)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    P[rows, A.col] = True
    return P


def fixpoint_levels(n, row_ptr, col, upper):
    """Brute force for Eq. 11: sweep in the *wrong* order until nothing changes."""
    lev = np.zeros(n, dtype=np.int64)
    changed = True
    sweeps = 0
    while changed:
        changed = False
        sweeps += 1
        order = range(n) if upper else range(n - 1, -1, -1)
        for i in order:
            cols = col[row_ptr[i]:row_ptr[i + 1]]
            deps = cols[cols > i] if upper else cols[cols < i]
            new = 1 + (lev[deps].max() if deps.size else 0)
            if new != lev[i]:
                lev[i] = new
                changed = True
        assert sweeps <= n + 2
    return lev


def lu_nopivot_checked(D):
    """scipy LU; asserts that no row exchange happened (so it is Doolittle LU)."""
    P, L, U = sla.lu(D)
    assert np.array_equal(P, np.eye(D.shape[0]))
    return L, U


# --------------------------------------------------------------------------- generator vs Table 2
def test_table2_poisson_sizes_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_poisson_sizes.txt"))
            if l.strip() and not l.startswith("#")]
    for name, side, n, nnz, mib in rows:
        side, n, nnz = int(side), int(n), int(nnz)
        # n and nnz of the 7-point stencil: count without building the 3.4M-row matrix
        assert side ** 3 == n
        assert 7 * side ** 3 - 6 * side ** 2 == nnz
        if mib != "-":
            assert round((nnz * 12 + (n + 1) * 4) / 2 ** 20) == int(mib)
    small = synth.poisson3d_7pt(12)
    assert small.nnz == 7 * 12 ** 3 - 6 * 12 ** 2


# --------------------------------------------------------------------------- O1: SpMV
@pytest.mark.parametrize("N", [7, 12])
def test_spmv_poisson2d_eigenpairs(orc, N):
    A = synth.poisson2d_5pt(N)
    x = np.arange(1, N + 1)
    h = np.pi / (N + 1)
    for p, q in [(1, 1), (2, 3), (N, 1), (N - 1, N)]:
        v = np.outer(np.sin(q * h * x), np.sin(p * h * x)).ravel()  # (y, x) with x fastest
        lam = 4 - 2 * np.cos(p * h) - 2 * np.cos(q * h)
        Av = orc.spmv(A, v)
        assert np.max(np.abs(Av - lam * v)) <= 1e-12 * max(1.0, lam)


def test_spmv_poisson3d_eigenpairs(orc):
    N = 6
    A = synth.poisson3d_7pt(N)
    x = np.arange(1, N + 1)
    h = np.pi / (N + 1)
    for p, q, r in [(1, 1, 1), (2, 5, 3), (6, 6, 6)]:
        v = np.einsum("k,j,i->kji", np.sin(r * h * x), np.sin(q * h * x), np.sin(p * h * x)).ravel()
        lam = 6 - 2 * (np.cos(p * h) + np.cos(q * h) + np.cos(r * h))
        assert np.max(np.abs(orc.spmv(A, v) - lam * v)) <= 1e-12 * lam


def test_spmv_integer_exact_and_epilogue(orc):
    A = synth.random_sparse(150, 0.05, seed=11, integer=True)
    rng = np.random.default_rng(3)
    x = rng.integers(-5, 6, size=A.n).astype(np.float64)
    y = rng.integers(-5, 6, size=A.n).astype(np.float64)
    Ai = A.to_dense().astype(np.int64)
    exact = 2 * (Ai @ x.astype(np.int64)) - 3 * y.astype(np.int64)
    got = orc.spmv(A, x, alpha=2.0, beta=-3.0, y=y)
    assert np.array_equal(got, exact.astype(np.float64))


def test_spmv_diffusion_rowsum_is_boundary_flux(orc):
    # A 1 = sum of the boundary-face coefficients of each cell (interior faces cancel)
    N, sigma, seed = 5, 2.0, 9
    A = synth.diffusion3d_7pt_lognormal(N, sigma, seed)
    rng = np.random.default_rng(seed)
    fx = np.exp(sigma * rng.standard_normal((N, N, N + 1)))
    fy = np.exp(sigma * rng.standard_normal((N, N + 1, N)))
    fz = np.exp(sigma * rng.standard_normal((N + 1, N, N)))
    bnd = np.zeros((N, N, N))
    bnd[:, :, 0] += fx[:, :, 0]
    bnd[:, :, -1] += fx[:, :, -1]
    bnd[:, 0, :] += fy[:, 0, :]
    bnd[:, -1, :] += fy[:, -1, :]
    bnd[0, :, :] += fz[0, :, :]
    bnd[-1, :, :] += fz[-1, :, :]
    got = orc.spmv(A, np.ones(A.n))
    assert np.allclose(got, bnd.ravel(), rtol=1e-12, atol=1e-12 * np.abs(A.val).max())


def test_vector_ops_exact(orc):
    rng = np.random.default_rng(5)
    x = rng.integers(-9, 10, 1000).astype(np.float64)
    y = rng.integers(-9, 10, 1000).astype(np.float64)
    assert orc.dot(x, y) == float(np.sum(x.astype(np.int64) * y.astype(np.int64)))
    assert orc.nrm2(np.array([3.0, 4.0])) == 5.0
    assert np.array_equal(orc.axpby(2.0, x, -1.0, y), 2 * x - y)
    assert np.array_equal(orc.waxpby(-3.0, x, 4.0, y), -3 * x + 4 * y)


# --------------------------------------------------------------------------- O2/O3: ILU(k)
def _check_against_literal(orc, A, k):
    F = orc.iluk(A, k)
    Ad = A.to_dense()
    D, Lev = dense_iluk_literal(Ad, pattern_of(A), k)
    keep = np.isfinite(Lev)
    rows = np.repeat(np.arange(A.n), np.diff(F.row_ptr))
    got_pat = np.zeros_like(keep)
    got_pat[rows, F.col] = True
    assert np.array_equal(got_pat, keep), "fill pattern differs from literal Algorithm 2"
    assert np.array_equal(F.lev, Lev[rows, F.col].astype(np.int32)), "fill levels differ"
    assert np.array_equal(F.val, D[rows, F.col]), "values differ from literal Algorithm 2"
    return F


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("seed", [1, 2])
def test_iluk_matches_literal_algorithm2_random(orc, k, seed):
    A = synth.random_sparse(90, 0.04, seed=seed)
    _check_against_literal(orc, A, k)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_iluk_matches_literal_algorithm2_stencils(orc, k):
    _check_against_literal(orc, synth.poisson2d_5pt(9), k)
    _check_against_literal(orc, synth.diffusion3d_7pt_lognormal(4, 2.0, 1), k)
    _check_against_literal(orc, synth.stencil27_irregular(4, 1, 2, frac=0.1, extra_min=3,
                                                          extra_max=8), k)


def test_ilu0_reproduces_A_on_its_pattern(orc):
    for A in (synth.random_sparse(120, 0.05, seed=4), synth.diffusion3d_7pt_lognormal(5, 2.0, 3)):
        F = orc.iluk(A, 0)
        (Lrp, Lc, Lv), (Urp, Uc, Uv) = F.split()
        Ld = np.eye(A.n)
        Ud = np.zeros((A.n, A.n))
        Ld[np.repeat(np.arange(A.n), np.diff(Lrp)), Lc] = Lv
        Ud[np.repeat(np.arange(A.n), np.diff(Urp)), Uc] = Uv
        Ad = A.to_dense()
        P = pattern_of(A)
        assert np.array_equal(np.repeat(np.arange(A.n), np.diff(F.row_ptr)),
                              np.repeat(np.arange(A.n), np.diff(A.row_ptr)))
        LU = Ld @ Ud
        scale = np.abs(Ad).max()
        assert np.max(np.abs(LU[P] - Ad[P])) <= 1e-13 * scale


def test_ilu0_tridiagonal_equals_dense_lu(orc):
    A = synth.tridiagonal(200, seed=8)
    F = orc.iluk(A, 0)
    L, U = lu_nopivot_checked(A.to_dense())
    D = F.to_dense()
    assert np.allclose(np.tril(D, -1), np.tril(L, -1), rtol=0, atol=1e-14)
    assert np.allclose(np.triu(D), U, rtol=0, atol=1e-14 * np.abs(U).max())


def test_iluk_high_level_equals_dense_lu(orc):
    # 2D Poisson N x N: full LU fills inside the band |i-j| <= N; a level beyond
    # the maximum fill level reproduces exact LU (pattern and values).
    N = 6
    A = synth.poisson2d_5pt(N)
    L, U = lu_nopivot_checked(A.to_dense())
    F = orc.iluk(A, 3 * N)
    D = F.to_dense()
    band = np.abs(np.subtract.outer(np.arange(A.n), np.arange(A.n))) <= N
    rows = np.repeat(np.arange(A.n), np.diff(F.row_ptr))
    pat = np.zeros((A.n, A.n), bool)
    pat[rows, F.col] = True
    lu_nz = (np.tril(L, -1) + U) != 0
    assert np.all(pat[lu_nz]) and not np.any(pat & ~band)
    # the same result as any larger level
    assert np.array_equal(orc.iluk(A, 5 * N).to_dense(), D)
    assert np.allclose(np.tril(D, -1), np.tril(L, -1), atol=1e-13)
    assert np.allclose(np.triu(D), U, atol=1e-13)


def test_iluk_fill_offsets_2d_and_3d(orc):
    N = 8
    A = synth.poisson2d_5pt(N)
    F = orc.iluk(A, 1)
    rows = np.repeat(np.arange(A.n), np.diff(F.row_ptr))
    offs = set(np.unique(F.col - rows).tolist())
    assert offs == {-N, -(N - 1), -1, 0, 1, N - 1, N}
    fill = F.lev == 1
    assert set(np.unique((F.col - rows)[fill]).tolist()) == {-(N - 1), N - 1}
    assert F.row_ptr[-1] == A.nnz + 2 * (N - 1) ** 2
    M = 5
    B = synth.poisson3d_7pt(M)
    G = orc.iluk(B, 1)
    rows = np.repeat(np.arange(B.n), np.diff(G.row_ptr))
    fill_offs = set(np.unique((G.col - rows)[G.lev == 1]).tolist())
    assert fill_offs == {-(M - 1), M - 1, -(M * M - 1), M * M - 1, -(M * M - M), M * M - M}
    assert G.lev.max() == 1


def test_iluk_zero_pivot_and_invalid(orc):
    A = synth.CSR(np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([0.0, 1.0, 1.0, 0.0]))
    with pytest.raises(orc.OracleError) as e:
        orc.iluk(A, 0)
    assert e.value.status == orc.ERR_ZERO_PIVOT
    B = synth.CSR(np.array([0, 2, 3]), np.array([1, 0, 1]), np.array([1.0, 2.0, 3.0]))
    with pytest.raises(orc.OracleError) as e:
        orc.iluk(B, 0)
    assert e.value.status == orc.ERR_INVALID


# --------------------------------------------------------------------------- O5: levels
@pytest.mark.parametrize("k", [0, 1, 2])
def test_levels_match_fixpoint(orc, k):
    for A in (synth.random_sparse(150, 0.03, seed=21), synth.stencil27_irregular(
            5, 3, 4, frac=0.05, extra_min=2, extra_max=6)):
        F = orc.iluk(A, k)
        for upper in (False, True):
            lev, nlev = orc.levels(F.n, F.row_ptr, F.col, upper)
            ref = fixpoint_levels(F.n, F.row_ptr, F.col, upper)
            assert np.array_equal(lev, ref)
            assert nlev == ref.max()


def test_levels_closed_forms(orc):
    N = 9
    F = orc.iluk(synth.poisson2d_5pt(N), 0)
    lev, nlev = orc.levels(F.n, F.row_ptr, F.col, False)
    y, x = np.divmod(np.arange(N * N), N)
    assert nlev == 2 * N - 1
    assert np.array_equal(lev, x + y + 1)
    ulev, unlev = orc.levels(F.n, F.row_ptr, F.col, True)
    assert unlev == 2 * N - 1
    assert np.array_equal(ulev, (N - 1 - x) + (N - 1 - y) + 1)
    M = 5
    G = orc.iluk(synth.poisson3d_7pt(M), 0)
    lev, nlev = orc.levels(G.n, G.row_ptr, G.col, False)
    z, r = np.divmod(np.arange(M ** 3), M * M)
    y, x = np.divmod(r, M)
    assert nlev == 3 * M - 2
    assert np.array_equal(lev, x + y + z + 1)
    # diagonal -> 1 level, bidiagonal -> n levels
    n = 10
    lev, nlev = orc.levels(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), False)
    assert nlev == 1 and np.all(lev == 1)
    rp = np.concatenate([[0], 1 + 2 * np.arange(n)]).astype(np.int32)
    col = np.concatenate([[0]] + [[i - 1, i] for i in range(1, n)]).astype(np.int32)
    lev, nlev = orc.levels(n, rp, col, False)
    assert nlev == n and np.array_equal(lev, np.arange(1, n + 1))


def test_level_sets_are_canonical(orc):
    F = orc.iluk(synth.random_sparse(80, 0.05, seed=2), 1)
    lev, nlev = orc.levels(F.n, F.row_ptr, F.col, False)
    ptr, rows = orc.level_sets(lev, nlev)
    assert ptr[-1] == F.n and np.all(np.diff(ptr) > 0)
    for l in range(nlev):
        seg = rows[ptr[l]:ptr[l + 1]]
        assert np.all(np.diff(seg) > 0) and np.all(lev[seg] == l + 1)


# --------------------------------------------------------------------------- O6: triangular solves
def test_triangular_solves_vs_scipy(orc):
    A = synth.random_sparse(200, 0.03, seed=6)
    F = orc.iluk(A, 1)
    D = F.to_dense()
    b = synth.rhs_uniform(A.n, 3)
    y = orc.lsolve_unit(F, b)
    yr = sla.solve_triangular(np.tril(D, -1) + np.eye(A.n), b, lower=True, unit_diagonal=True)
    assert np.max(np.abs(y - yr)) <= 1e-13 * np.abs(yr).max()
    z = orc.usolve(F, y)
    zr = sla.solve_triangular(np.triu(D), y, lower=False)
    assert np.max(np.abs(z - zr)) <= 1e-13 * np.abs(zr).max()


# --------------------------------------------------------------------------- O4: RAS
def test_ras_single_block_is_plain_ilu(orc):
    A = synth.diffusion3d_7pt_lognormal(6, 2.0, 5)
    r = synth.rhs_uniform(A.n, 1)
    M = orc.RAS(A, 1, 1, 0)
    F = orc.iluk(A, 1)
    assert np.array_equal(M.apply(r), orc.usolve(F, orc.lsolve_unit(F, r)))


def test_ras_block_diagonal_equals_global_ilu(orc):
    blocks = [synth.random_sparse(40, 0.08, seed=s) for s in range(4)]
    n = 160
    rows, cols, vals = [], [], []
    for b, B in enumerate(blocks):
        rr = np.repeat(np.arange(40), np.diff(B.row_ptr)) + 40 * b
        rows.append(rr)
        cols.append(B.col + 40 * b)
        vals.append(B.val)
    A = synth._assemble(n, np.concatenate(rows).astype(np.int64),
                        np.concatenate(cols).astype(np.int64), np.concatenate(vals))
    r = synth.rhs_uniform(n, 2)
    F = orc.iluk(A, 2)
    ref = orc.usolve(F, orc.lsolve_unit(F, r))
    for ov in (0, 1, 3):
        assert np.array_equal(orc.RAS(A, 2, 4, ov).apply(r), ref)


def test_ras_large_overlap_equals_global_ilu(orc):
    A = synth.poisson2d_5pt(8)
    r = synth.rhs_uniform(A.n, 4)
    F = orc.iluk(A, 0)
    ref = orc.usolve(F, orc.lsolve_unit(F, r))
    M = orc.RAS(A, 0, 4, 2 * 8)  # overlap >= graph diameter: every block is the whole matrix
    for b in range(4):
        assert M.block(b)[0].shape[0] == A.n
    assert np.array_equal(M.apply(r), ref)


def test_ras_apply_is_the_schwarz_sum(orc):
    # z = sum_b R0_b (L_b U_b)^{-1} R_b r computed with dense algebra
    A = synth.random_sparse(120, 0.03, seed=9)
    M = orc.RAS(A, 1, 5, 1)
    r = synth.rhs_uniform(A.n, 5)
    z = np.full(A.n, np.nan)
    owned = np.zeros(A.n, int)
    for b in range(5):
        rows, lo, hi, F = M.block(b)
        D = F.to_dense()
        Lb = np.tril(D, -1) + np.eye(rows.shape[0])
        Ub = np.triu(D)
        zb = np.linalg.solve(Lb @ Ub, r[rows])
        sel = (rows >= lo) & (rows < hi)
        z[rows[sel]] = zb[sel]
        owned[rows[sel]] += 1
    assert np.all(owned == 1)
    got = M.apply(r)
    assert np.max(np.abs(got - z)) <= 1e-10 * np.abs(z).max()


def test_ras_overlap_sets_closed_form(orc):
    # 7-point stencil, N^3 grid, nb = N/2 blocks of 2 z-planes, overlap 1:
    # V_b = planes 2b-1 .. 2b+2 (clipped to the grid)
    N = 6
    A = synth.poisson3d_7pt(N)
    nb = N // 2
    M = orc.RAS(A, 1, nb, 1)
    P = N * N
    for b in range(nb):
        rows, lo, hi, F = M.block(b)
        assert (lo, hi) == (2 * b * P, (2 * b + 2) * P)
        z0, z1 = max(0, 2 * b - 1), min(N, 2 * b + 3)
        assert np.array_equal(rows, np.arange(z0 * P, z1 * P))


def test_ras_every_owned_row_written_once(orc):
    A = synth.stencil27_irregular(6, 1, 2, frac=0.05, extra_min=3, extra_max=10)
    M = orc.RAS(A, 0, 7, 1)
    z = M.apply(np.ones(A.n))
    assert np.all(np.isfinite(z))
    covered = np.zeros(A.n, int)
    for b in range(7):
        rows, lo, hi, F = M.block(b)
        covered[lo:hi] += 1
    assert np.all(covered == 1)


# --------------------------------------------------------------------------- O7: BiCGSTAB
def test_bicgstab_exact_preconditioner_one_iteration(orc):
    A = synth.tridiagonal(300, seed=3)
    b = synth.rhs_uniform(A.n, 1)
    x, info = orc.bicgstab(A, b, M=orc.RAS(A, 0, 1, 0), tol=1e-12)
    assert info.status == orc.OK and info.iters == 1 and info.rel_resid <= 1e-12
    B = synth.poisson2d_5pt(7)
    b = synth.rhs_uniform(B.n, 2)
    x, info = orc.bicgstab(B, b, M=orc.RAS(B, 100, 1, 0), tol=1e-12)
    assert info.iters == 1 and info.rel_resid <= 1e-12


@pytest.mark.parametrize("nb,ov,k", [(1, 0, 0), (4, 1, 1), (3, 0, 2)])
def test_bicgstab_manufactured_solution(orc, nb, ov, k):
    A = synth.diffusion2d_5pt_lognormal(24, 1.0, seed=4)
    xs = synth.rhs_uniform(A.n, 7)
    b = orc.spmv(A, xs)
    x, info = orc.bicgstab(A, b, M=orc.RAS(A, k, nb, ov), tol=1e-10, maxit=500)
    assert info.status == orc.OK and info.rel_resid <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-6


def test_bicgstab_unpreconditioned_and_breakdown(orc):
    A = synth.random_sparse(100, 0.05, seed=12)
    b = synth.rhs_uniform(A.n, 3)
    x, info = orc.bicgstab(A, b, tol=1e-10)
    assert info.status == orc.OK
    assert np.allclose(x, np.linalg.solve(A.to_dense(), b), atol=1e-8)
    # skew-symmetric: (r0, A r0) = 0, so alpha is undefined at the first step
    S = synth.CSR(np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([0.0, 1.0, -1.0, 0.0]))
    x, info = orc.bicgstab(S, np.array([1.0, 2.0]), tol=1e-10)
    assert info.status == orc.BREAKDOWN


def test_bicgstab_zero_rhs(orc):
    A = synth.poisson2d_5pt(4)
    x, info = orc.bicgstab(A, np.zeros(A.n), x0=np.ones(A.n))
    assert info.iters == 0 and np.all(x == 0)


def diag_inverse(A):
    d = np.zeros(A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    on = rows == A.col
    d[rows[on]] = A.val[on]
    return 1.0 / d


@pytest.mark.parametrize("prec", ["none", "jacobi", "ras"])
def test_bicgstab_iterates_match_scipy(orc, prec):
    """The first iterates equal SciPy's BiCGSTAB (van der Vorst's right-preconditioned
    recurrences, shadow residual r0) with the same preconditioner: a wrong sign or a
    swapped alpha/omega in any update moves x_k off SciPy's x_k at once."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = synth.diffusion2d_5pt_lognormal(14, 1.0, seed=6)
    b = synth.rhs_uniform(A.n, 4)
    As = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n, A.n))
    if prec == "none":
        M, Ms = None, None
    elif prec == "jacobi":
        dinv = diag_inverse(A)
        M = orc.Jacobi(A, 1.0)
        Ms = spla.LinearOperator((A.n, A.n), matvec=lambda r: dinv * r)
    else:
        M = orc.RAS(A, 0, 3, 1)
        Ms = spla.LinearOperator((A.n, A.n), matvec=M.apply)
    hist = []
    spla.bicgstab(As, b, rtol=1e-300, atol=0.0, maxiter=6, M=Ms,
                  callback=lambda xk: hist.append(xk.copy()))
    assert len(hist) == 6
    for k in range(1, 7):
        x, info = orc.bicgstab(A, b, M=M, tol=1e-300, maxit=k)
        assert info.iters == k
        xs = hist[k - 1]
        assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs), k


# --------------------------------------------------------------------------- O8: GMRES
def min_residual_iterate(Ad, Minv, b, x0, k):
    """argmin ||b - A x|| over x in x0 + M^{-1} K_k(A M^{-1}, r0), by dense least squares
    over an orthonormalised power basis (the defining property of GMRES)."""
    B = Ad @ Minv
    r0 = b - Ad @ x0
    K = np.empty((len(b), k))
    v = r0 / np.linalg.norm(r0)
    for j in range(k):
        K[:, j] = v
        v = B @ v
        v /= np.linalg.norm(v)
    W, _ = np.linalg.qr(K)
    c = np.linalg.lstsq(B @ W, r0, rcond=None)[0]
    return x0 + Minv @ (W @ c)


@pytest.mark.parametrize("prec", ["none", "ras"])
def test_gmres_iterates_minimise_the_residual_over_the_krylov_space(orc, prec):
    """Each x_k (k steps inside one cycle) is the minimal-residual point of the
    right-preconditioned Krylov space; after a restart the same holds from the
    restart point. A dropped Givens term, a wrong back substitution or a missing
    M^{-1} in the update each give a larger residual than the minimum."""
    A = synth.diffusion2d_5pt_lognormal(12, 1.5, seed=8)
    b = synth.rhs_uniform(A.n, 5)
    Ad = A.to_dense()
    if prec == "none":
        M, Minv = None, np.eye(A.n)
    else:
        M = orc.RAS(A, 0, 2, 1)
        Minv = np.column_stack([M.apply(e) for e in np.eye(A.n)])
    for k in range(1, 7):
        x, info = orc.gmres(A, b, M=M, tol=1e-300, maxit=k, restart=8)
        assert info.iters == k and info.restarts == 1
        xr = min_residual_iterate(Ad, Minv, b, np.zeros(A.n), k)
        res, res_ref = np.linalg.norm(b - Ad @ x), np.linalg.norm(b - Ad @ xr)
        assert res <= res_ref * (1 + 1e-9), k
        assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr), k
        assert abs(info.est_resid - res / np.linalg.norm(b)) <= 1e-10
    # two cycles of GMRES(3): the second minimises from the first cycle's end point
    x3, _ = orc.gmres(A, b, M=M, tol=1e-300, maxit=3, restart=3)
    x5, info = orc.gmres(A, b, M=M, tol=1e-300, maxit=5, restart=3)
    assert info.restarts == 2
    xr = min_residual_iterate(Ad, Minv, b, x3, 2)
    assert np.linalg.norm(x5 - xr) <= 1e-8 * np.linalg.norm(xr)


def test_gmres_finite_termination(orc):
    A = synth.poisson2d_5pt(6)
    b = synth.rhs_uniform(A.n, 1)
    x, info = orc.gmres(A, b, tol=1e-10, maxit=A.n, restart=A.n)
    assert info.status == orc.OK and info.iters <= A.n and info.rel_resid <= 1e-10
    # an exact LU preconditioner solves in one Arnoldi step
    x, info = orc.gmres(A, b, M=orc.RAS(A, 100, 1, 0), tol=1e-12, restart=5)
    assert info.iters == 1 and info.rel_resid <= 1e-12


def test_gmres_givens_estimate_is_true_residual(orc):
    A = synth.diffusion2d_5pt_lognormal(16, 1.0, seed=2)
    b = synth.rhs_uniform(A.n, 9)
    for M in (None, orc.RAS(A, 0, 2, 1)):
        x, info = orc.gmres(A, b, M=M, tol=1e-6, maxit=400, restart=400)
        assert info.restarts == 1
        assert abs(info.est_resid - info.rel_resid) <= 1e-9


@pytest.mark.parametrize("restart", [5, 30])
def test_gmres_manufactured_solution(orc, restart):
    A = synth.random_sparse(150, 0.04, seed=15)
    xs = synth.rhs_uniform(A.n, 2)
    b = orc.spmv(A, xs)
    x, info = orc.gmres(A, b, M=orc.RAS(A, 0, 3, 1), tol=1e-10, maxit=600, restart=restart)
    assert info.status == orc.OK and info.rel_resid <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8
    if restart == 5:
        assert info.restarts > 1


def test_gmres_maxit(orc):
    A = synth.diffusion2d_5pt_lognormal(20, 2.0, seed=1)
    b = synth.rhs_uniform(A.n, 1)
    x, info = orc.gmres(A, b, tol=1e-14, maxit=7, restart=3)
    assert info.status == orc.MAXIT and info.iters == 7


# --------------------------------------------------------------------------- damped Jacobi, CG
def dense_csr(D):
    """A dense matrix as CSR with every entry stored (zeros included on the diagonal)."""
    n = D.shape[0]
    rows, cols = np.nonzero((D != 0) | np.eye(n, dtype=bool))
    return synth.CSR(np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]), cols,
                     D[rows, cols])


def test_jacobi_on_a_diagonal_matrix_is_the_scaled_exact_solve(orc):
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 3.0, 40) * rng.choice([-1.0, 1.0], 40)
    A = dense_csr(np.diag(d))
    r = rng.standard_normal(40)
    for omega in (1.0, 0.6):
        z = orc.Jacobi(A, omega).apply(r)
        np.testing.assert_allclose(z, omega * np.linalg.solve(np.diag(d), r), rtol=1e-15)
    # with omega = 1 the preconditioner is exact: one iteration of each solver
    b = rng.standard_normal(40)
    for solve in (orc.bicgstab, orc.cg):
        x, info = solve(dense_csr(np.diag(np.abs(d))), b, M=orc.Jacobi(dense_csr(np.diag(np.abs(d)))),
                        tol=1e-13)
        assert info.status == orc.OK and info.iters == 1


def test_damped_jacobi_iteration_contracts_at_the_closed_form_rate(orc):
    # x <- x + M (b - A x) with M = omega D^{-1} on tridiag(-1, 2, -1): the error
    # contracts by the spectral radius max_k |1 - omega (1 - cos(k pi / (n+1)))|
    n, omega = 20, 2.0 / 3.0
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = dense_csr(T)
    M = orc.Jacobi(A, omega)
    xs = np.linspace(-1, 1, n) ** 2 + 0.3
    b = T @ xs
    x = np.zeros(n)
    errs = []
    for _ in range(700):
        x = x + M.apply(b - T @ x)
        errs.append(np.linalg.norm(x - xs))
    rate = errs[-1] / errs[-2]
    k = np.arange(1, n + 1)
    rho = np.max(np.abs(1 - omega * (1 - np.cos(k * np.pi / (n + 1)))))
    assert abs(rate - rho) <= 1e-6


def test_jacobi_zero_diagonal_and_bad_omega(orc):
    D = np.diag([1.0, 0.0, 2.0])
    D[1, 0] = 1.0
    with pytest.raises(orc.OracleError) as e:
        orc.Jacobi(dense_csr(D))
    assert e.value.status == orc.ERR_ZERO_PIVOT
    with pytest.raises(orc.OracleError):
        orc.Jacobi(dense_csr(np.eye(3)), 0.0)


def test_cg_iterates_minimise_the_energy_norm_over_the_krylov_space(orc):
    # x_k = argmin over K_k(A, b) of ||x - x*||_A, computed by a dense projection
    A = synth.diffusion2d_5pt_lognormal(6, 0.5, seed=3)
    T = A.to_dense()
    b = synth.rhs_uniform(A.n, 4)
    K = np.empty((A.n, 0))
    v = b.copy()
    for k in range(1, 7):
        K = np.column_stack([K, v])
        v = T @ v
        Q, _ = np.linalg.qr(K)
        xk = Q @ np.linalg.solve(Q.T @ T @ Q, Q.T @ b)
        x, info = orc.cg(A, b, tol=0.0, maxit=k)
        assert info.iters == k and info.status == orc.MAXIT
        assert np.linalg.norm(x - xk) <= 1e-9 * np.linalg.norm(xk)


def test_cg_converges_in_as_many_steps_as_distinct_eigenvalues(orc):
    rng = np.random.default_rng(8)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    lam = np.repeat([1.0, 4.0, 9.0], 10)
    A = dense_csr(Q @ np.diag(lam) @ Q.T)
    b = rng.standard_normal(30)
    x, info = orc.cg(A, b, tol=1e-10, maxit=10)
    assert info.status == orc.OK and info.iters == 3


def test_cg_exact_preconditioner_and_finite_termination(orc):
    A = synth.poisson2d_5pt(6)
    b = synth.rhs_uniform(A.n, 1)
    x, info = orc.cg(A, b, tol=1e-10, maxit=A.n)
    assert info.status == orc.OK and info.iters <= A.n and info.rel_resid <= 1e-10
    x, info = orc.cg(A, b, M=orc.RAS(A, 100, 1, 0), tol=1e-12)
    assert info.iters == 1 and info.rel_resid <= 1e-12


@pytest.mark.parametrize("prec", ["none", "ilu0", "jacobi"])
def test_cg_manufactured_solution(orc, prec):
    A = synth.diffusion2d_5pt_lognormal(20, 1.0, seed=6)
    xs = synth.rhs_uniform(A.n, 3)
    b = orc.spmv(A, xs)
    M = {"none": None, "ilu0": orc.RAS(A, 0, 1, 0), "jacobi": orc.Jacobi(A, 0.8)}[prec]
    x, info = orc.cg(A, b, M=M, tol=1e-11, maxit=2000)
    assert info.status == orc.OK and info.rel_resid <= 1e-11
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-7


def test_cg_breakdown_and_zero_rhs(orc):
    A = dense_csr(np.diag([1.0, -1.0]))
    x, info = orc.cg(A, np.array([1.0, 1.0]), tol=1e-12, maxit=5)
    assert info.status == orc.BREAKDOWN
    B = synth.poisson2d_5pt(4)
    x, info = orc.cg(B, np.zeros(B.n), x0=np.ones(B.n))
    assert info.status == orc.OK and np.all(x == 0) and info.iters == 0


def test_spmv_on_host_threads_is_the_same_row_loop(orc):
    # the all-cores CPU baseline splits the oracle's row loop over threads
    A = synth.stencil27_irregular(16, 2, 3)
    x = synth.rhs_uniform(A.n, 5)
    for t in (1, 3, 8):
        assert np.array_equal(orc.spmv_threads(A, x, t), orc.spmv(A, x))
