"""The seeded input recipes hold the structure their documentation states.

The parity tests and the benchmark draw every input from ``synth.py``; these
checks pin what its docstrings promise about each workload (entry counts in
closed form, sorted CSR with the diagonal present, symmetry, M-matrix and
positive definiteness, the request mix's distribution, the batch assembly),
so that a change of recipe cannot slip through as a change of workload.
No GPU.
"""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth


def well_formed(A):
    """Sorted, duplicate-free rows with the diagonal present (the CSR form every
    generator returns)."""
    assert A.row_ptr[0] == 0 and A.row_ptr[-1] == len(A.col) == len(A.val)
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def spd_m_matrix(A):
    D = A.to_dense()
    off = D - np.diag(np.diag(D))
    assert np.array_equal(D, D.T)
    assert np.all(off <= 0) and np.all(np.diag(D) > 0)
    # weakly diagonally dominant, strictly on the rows with a boundary face
    slack = np.diag(D) + off.sum(axis=1)
    assert np.all(slack >= -1e-12 * np.diag(D)) and np.any(slack > 0)
    assert np.linalg.eigvalsh(D).min() > 0


@pytest.mark.parametrize("N", [2, 5, 9])
def test_diffusion_stencils_entry_counts_and_spd(N):
    A2 = synth.diffusion2d_5pt_lognormal(N, 2.0, seed=N)
    assert A2.n == N * N and A2.nnz == 5 * N * N - 4 * N
    A3 = synth.diffusion3d_7pt_lognormal(N, 2.0, seed=N)
    assert A3.n == N ** 3 and A3.nnz == 7 * N ** 3 - 6 * N ** 2
    for A in (A2, A3):
        well_formed(A)
        spd_m_matrix(A)


def test_headline_system_size_from_the_closed_form():
    """The 128^3 system: n = 2,097,152 and nnz = 7N^3 - 6N^2 = 14,581,760 (the
    figures every byte count of the benchmark is built on)."""
    N = 128
    assert N ** 3 == 2_097_152 and 7 * N ** 3 - 6 * N ** 2 == 14_581_760


@pytest.mark.parametrize("N", [2, 4, 6])
def test_stencil27_lognormal_is_a_full_27_point_spd_m_matrix(N):
    A = synth.stencil27_lognormal(N, 2.0, seed=3)
    # every cell couples to each in-grid neighbour: (3N - 2) per axis
    assert A.n == N ** 3 and A.nnz == (3 * N - 2) ** 3
    well_formed(A)
    spd_m_matrix(A)
    # a slot outside the grid puts its coefficient on the diagonal only: the
    # row sum is zero on interior cells and positive on every boundary cell
    D = A.to_dense()
    slack = D.sum(axis=1)
    z, y, x = np.unravel_index(np.arange(A.n), (N, N, N))
    boundary = (np.minimum.reduce([x, y, z]) == 0) | (np.maximum.reduce([x, y, z]) == N - 1)
    assert np.all(slack[boundary] > 0)
    assert np.allclose(slack[~boundary], 0, atol=1e-12 * np.abs(np.diag(D)).max())


def test_lognormal_coefficients_have_the_stated_spread():
    """Face coefficients exp(sigma g), g ~ N(0, 1): the off-diagonals of a 3D
    system are -kappa, so log(-a_ij) has mean 0 and standard deviation sigma."""
    A = synth.diffusion3d_7pt_lognormal(24, 2.0, seed=2)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = A.val[rows != A.col]
    g = np.log(-off)
    assert abs(g.mean()) < 0.05 and abs(g.std() - 2.0) < 0.05


def test_stencil27_irregular_extra_rows_and_dominance():
    A = synth.stencil27_irregular(8, 4, 5, frac=0.1, extra_min=30, extra_max=40)
    well_formed(A)
    lens = np.diff(A.row_ptr)
    interior = 27
    # about 10% of rows carry 30-40 extra entries beyond their stencil part
    assert 0.05 < np.mean(lens > interior) < 0.15
    assert lens.max() <= interior + 40
    D = A.to_dense()
    d = np.diag(D)
    offsum = np.abs(D).sum(axis=1) - np.abs(d)
    assert np.allclose(d, 1.1 * offsum)  # the diagonal is 1.1 x the off-diagonal |row sum|


def test_serving_request_mix_distribution():
    reqs = synth.serving_requests(3000, 8)
    st = np.array([r["stencil"] for r in reqs])
    k = np.array([r["k"] for r in reqs])
    n = np.array([r["n"] for r in reqs], dtype=np.float64)
    for s in (5, 7, 27):
        assert abs(np.mean(st == s) - 1 / 3) < 0.04
    assert set(k) == {0, 1} and abs(k.mean() - 0.5) < 0.04
    # log10 n uniform on [3, 6] before the side is rounded
    ln = np.log10(n)
    assert 2.9 < ln.min() and ln.max() < 6.05
    for q in (0.25, 0.5, 0.75):
        assert abs(np.quantile(ln, q) - (3 + 3 * q)) < 0.12
    for r in reqs:
        d = 2 if r["stencil"] == 5 else 3
        assert r["n"] == r["side"] ** d and r["side"] >= 2
    # the same seed gives the same stream
    assert synth.serving_requests(50, 8) == reqs[:50]


def test_batch_assembly_matches_its_systems():
    B = synth.batch_diffusion2d(6, 16, 24, 2.0, 7)
    assert B.nsys == 6 and B.row_ptr.dtype == np.int64
    assert np.all((B.sides >= 16) & (B.sides <= 24))
    rng = np.random.default_rng(7)
    sides = rng.integers(16, 25, 6)
    seeds = rng.integers(0, 2 ** 31 - 1, 6)
    assert np.array_equal(B.sides, sides)
    for s in range(B.nsys):
        A = B.system(s)
        ref = synth.diffusion2d_5pt_lognormal(int(sides[s]), 2.0, int(seeds[s]))
        assert A.n == ref.n
        assert np.array_equal(A.row_ptr, ref.row_ptr) and np.array_equal(A.col, ref.col)
        assert np.array_equal(A.val, ref.val)
    assert B.rows == int(np.sum(B.sides.astype(np.int64) ** 2))
