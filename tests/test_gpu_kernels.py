"""GPU parity of the CUDA kernels against the FP64 oracle, through the C ABI.

Tolerances (the two sides differ only in rounding):
  * SpMV (Eq. 2): per entry |y - y_ref| <= 1e-12 * (sum_j |a_ij x_j| + |beta y_i|),
    i.e. relative to the magnitude the sum is formed from; bit-exact for
    small-integer data (every partial sum is exact in FP64).
  * dot / norm (Eqs. 5-6): 1e-13 relative to sum |x_i y_i|.
  * preconditioner apply: per entry, |z - z_ref| <= the sum of the rounding
    bounds of both sides (tests/ras_bound.py: local errors of every row,
    propagated through the comparison-matrix triangular solves; FP64, or FP32
    for the FP32 layout), i.e. relative to the magnitudes each z_i is built
    from.
"""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth
from ras_bound import check_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    from paper_1606_00545_gb300 import build
    build.build()
    from paper_1606_00545_gb300 import hecgpu
    hecgpu.load_library()
    torch.cuda.set_device(0)
    return hecgpu


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def absmat(A):
    return synth.CSR(A.row_ptr, A.col, np.abs(A.val))


SPMV_CASES = {
    "poisson2d_64": lambda: (synth.poisson2d_5pt(64), 0),
    "diffusion3d_24": lambda: (synth.diffusion3d_7pt_lognormal(24, 2.0, 2), 0),
    "irregular27_12": lambda: (synth.stencil27_irregular(12, 4, 5), 0),
    "random_forced_tail": lambda: (synth.random_sparse(1500, 0.01, seed=3), 2),
    "n1": lambda: (synth.CSR(np.array([0, 1]), np.array([0]), np.array([3.0])), 0),
    "n3": lambda: (synth.tridiagonal(3, seed=1), 0),
    "n513": lambda: (synth.random_sparse(513, 0.01, seed=4), 0),
    "n1025_tail": lambda: (synth.random_sparse(1025, 0.02, seed=5), 4),
    # the format ablation's splits: K = 1 (almost all CSR tail), K = the
    # longest row (pure ELL), on heavy-tailed and irregular rows
    "powerlaw_csr": lambda: (synth.random_powerlaw_rows(20000, 2.5, 1.5, 600, 3), 1),
    "powerlaw_hec": lambda: (synth.random_powerlaw_rows(20000, 2.5, 1.5, 600, 3), 0),
    "powerlaw_ell": lambda: (synth.random_powerlaw_rows(3000, 2.5, 1.5, 200, 4), 201),
    "irregular27_csr": lambda: (synth.stencil27_irregular(12, 4, 5), 1),
    "irregular27_ell": lambda: (synth.stencil27_irregular(12, 4, 5), 160),
}


@pytest.mark.parametrize("case", sorted(SPMV_CASES))
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.5, 0.0), (-1.0, 1.0), (0.5, -3.0)])
def test_spmv_parity(H, orc, case, alpha, beta):
    A, K = SPMV_CASES[case]()
    x = synth.rhs_uniform(A.n, 11)
    y0 = synth.rhs_uniform(A.n, 12)
    M = H.hec_build(A.row_ptr, A.col, A.val, ell_width=K)
    xd, yin = dev(x), dev(y0)
    yout = dev(np.zeros(A.n))
    H.hec_spmv(M, alpha, xd, beta, yin if beta != 0 else None, yout)
    got = host(yout)
    ref = orc.spmv(A, x, alpha=alpha, beta=beta, y=y0)
    scale = abs(alpha) * orc.spmv(absmat(A), np.abs(x)) + abs(beta) * np.abs(y0)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-12 * scale + 1e-300), (case, err.max())
    # in place: y_in == y_out
    if beta != 0:
        H.hec_spmv(M, alpha, xd, beta, yin, yin)
        assert np.array_equal(host(yin), got)


def test_spmv_integer_bit_exact(H, orc):
    for K in (0, 3):
        A = synth.random_sparse(2000, 0.004, seed=9, integer=True)
        rng = np.random.default_rng(1)
        x = rng.integers(-7, 8, A.n).astype(np.float64)
        y0 = rng.integers(-7, 8, A.n).astype(np.float64)
        M = H.hec_build(A.row_ptr, A.col, A.val, ell_width=K)
        out = dev(np.zeros(A.n))
        H.hec_spmv(M, 3.0, dev(x), -2.0, dev(y0), out)
        assert np.array_equal(host(out), orc.spmv(A, x, alpha=3.0, beta=-2.0, y=y0))


def test_spmv_fused_dots_deterministic(H, orc):
    import torch
    A = synth.stencil27_irregular(10, 1, 2)
    x = synth.rhs_uniform(A.n, 3)
    w = synth.rhs_uniform(A.n, 4)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    y = dev(np.zeros(A.n))
    dots = dev(np.zeros(2))
    H.hec_spmv(M, 1.0, dev(x), 0.0, None, y, w=dev(w), dots=dots)
    d1 = host(dots).copy()
    yr = orc.spmv(A, x)
    assert abs(d1[0] - orc.dot(w, yr)) <= 1e-13 * np.sum(np.abs(w * yr))
    assert abs(d1[1] - orc.dot(yr, yr)) <= 1e-13 * np.sum(yr * yr)
    for _ in range(3):
        H.hec_spmv(M, 1.0, dev(x), 0.0, None, y, w=dev(w), dots=dots)
        assert np.array_equal(host(dots), d1)  # fixed summation order
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [1, 7, 1000, 300001])
def test_vector_ops(H, orc, n):
    x = synth.rhs_uniform(n, 1)
    y = synth.rhs_uniform(n, 2)
    xd, yd = dev(x), dev(y)
    H.hec_axpby(1.5, xd, -0.25, yd)
    ref = orc.axpby(1.5, x, -0.25, y)
    assert np.max(np.abs(host(yd) - ref)) <= 1e-15 * (1.5 * np.abs(x) + 0.25 * np.abs(y)).max()
    z = dev(np.zeros(n))
    H.hec_waxpby(-2.0, xd, 3.0, dev(y), z)
    ref = orc.waxpby(-2.0, x, 3.0, y)
    assert np.max(np.abs(host(z) - ref)) <= 1e-15 * (2 * np.abs(x) + 3 * np.abs(y)).max()
    r = dev(np.zeros(1))
    H.hec_dot(xd, dev(y), r)
    assert abs(host(r)[0] - orc.dot(x, y)) <= 1e-13 * np.sum(np.abs(x * y))
    H.hec_nrm2(xd, r)
    assert abs(host(r)[0] - orc.nrm2(x)) <= 1e-14 * orc.nrm2(x)


@pytest.mark.parametrize("k", [1, 7, 33])
def test_multidot(H, orc, k):
    n = 100003
    ldv = n + 5
    rng = np.random.default_rng(k)
    V = rng.uniform(-1, 1, (k, ldv))
    w = rng.uniform(-1, 1, n)
    h = dev(np.zeros(k))
    H.hec_multidot(n, k, dev(V.ravel()), ldv, dev(w), h)
    got = host(h)
    for i in range(k):
        ref = orc.dot(V[i, :n].copy(), w)
        assert abs(got[i] - ref) <= 1e-13 * np.sum(np.abs(V[i, :n] * w))


PRECOND_CASES = {
    "c1_poisson64_ilu0": lambda: (synth.poisson2d_5pt(64), 0, 1, 0),
    "diffusion3d_16_ilu1_ras8": lambda: (synth.diffusion3d_7pt_lognormal(16, 2.0, 2), 1, 8, 1),
    "random_ilu2_ras3_ov2": lambda: (synth.random_sparse(3000, 0.002, seed=2), 2, 3, 2),
    "irregular27_ilu0_ras4": lambda: (synth.stencil27_irregular(10, 4, 5), 0, 4, 1),
    "tridiag_exact": lambda: (synth.tridiagonal(5000, seed=3), 0, 1, 0),
    "wide_window_global": lambda: (synth.random_sparse_rows(24000, 6, seed=6), 0, 1, 0),
    "many_blocks": lambda: (synth.diffusion2d_5pt_lognormal(40, 2.0, 5), 1, 200, 1),
}


# cases whose blocks the resident-vector kernel takes (rows of at most 8
# entries, the block's vector in shared memory)
RESIDENT_FITS = {"c1_poisson64_ilu0", "diffusion3d_16_ilu1_ras8", "tridiag_exact", "many_blocks"}
KERNEL_MODES = {"auto": (0, 0), "streamed1": (1, 1), "streamed2": (1, 2), "streamed8": (1, 8),
                "resident": (2, 0)}


@pytest.mark.parametrize("mode", sorted(KERNEL_MODES))
@pytest.mark.parametrize("case", sorted(PRECOND_CASES))
def test_precond_apply_parity(H, orc, case, mode):
    """FP64 and FP32 applies against the oracle, entry by entry: the automatic
    choice, the streamed kernel with one CTA per block and with blocks forced
    into chains of 2 and 8 thread-block-cluster CTAs (where the dependencies
    allow it), and the resident-vector kernel where the blocks fit."""
    import torch
    kernel, parts = KERNEL_MODES[mode]
    if kernel == H.TRSV_RESIDENT and case not in RESIDENT_FITS:
        pytest.skip("rows too long or block too large for the resident kernel")
    A, k, nb, ov = PRECOND_CASES[case]()
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P, parts=parts, kernel=kernel)
    inf = P.info()
    assert inf["trsv_resident"] == (1 if kernel == H.TRSV_RESIDENT else
                                    0 if kernel == H.TRSV_STREAMED else inf["trsv_resident"])
    R = orc.RAS(A, k, nb, ov)
    for seed in (1, 2):
        r = synth.rhs_uniform(A.n, seed)
        z = dev(np.full(A.n, np.nan))
        H.hec_precond_apply(P, dev(r), z)
        assert H.hec_precond_status(P) == H.OK
        check_apply(orc, R, r, host(z), what="%s %s" % (case, mode))
        z32 = torch.full((A.n,), float("nan"), dtype=torch.float32, device="cuda:0")
        H.hec_precond_apply_f32(P, torch.tensor(r, dtype=torch.float32, device="cuda:0"), z32)
        assert H.hec_precond_status(P) == H.OK
        check_apply(orc, R, r, host(z32), fp32=True, what="%s %s fp32" % (case, mode))
    inf = P.info()
    if case == "wide_window_global" and kernel == H.TRSV_STREAMED:
        assert inf["global_passes"] > 0
    if case in ("c1_poisson64_ilu0", "diffusion3d_16_ilu1_ras8"):
        assert inf["global_passes"] == 0
        if mode == "auto" and case == "c1_poisson64_ilu0":
            assert inf["trsv_resident"] == 1  # levels of at most 64 rows
    if parts > 1 and case in ("c1_poisson64_ilu0", "diffusion3d_16_ilu1_ras8"):
        assert inf["split_blocks"] == nb  # the chained path ran


def test_precond_exact_on_tridiagonal(H, orc):
    # ILU(0) of a tridiagonal matrix is its LU: M^{-1} A x = x
    A = synth.tridiagonal(4000, seed=5)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    x = synth.rhs_uniform(A.n, 1)
    z = dev(np.zeros(A.n))
    H.hec_precond_apply(P, dev(orc.spmv(A, x)), z)
    assert np.max(np.abs(host(z) - x)) <= 1e-13


@pytest.mark.parametrize("kernel", [1, 2])
def test_precond_bounded_wait_reports_timeout(H, orc, kernel):
    """A wait on a barrier that nothing completes runs out, the kernel reports
    HEC_ERR_TIMEOUT, and the context stays usable (streamed and resident
    kernels)."""
    A = synth.poisson2d_5pt(32)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 2, 1)
    H.level_schedule(P, kernel=kernel)
    assert P.info()["trsv_resident"] == (kernel == H.TRSV_RESIDENT)
    r = synth.rhs_uniform(A.n, 1)
    z = dev(np.zeros(A.n))
    H.hec_precond_apply(P, dev(r), z, spin_limit=-1000)  # stall: nothing issued
    assert H.hec_precond_status(P) == H.ERR_TIMEOUT
    assert H.hec_precond_status(P) == H.OK  # the status was cleared
    H.hec_precond_apply(P, dev(r), z)
    assert H.hec_precond_status(P) == H.OK
    ref = orc.RAS(A, 0, 2, 1).apply(r)
    assert np.max(np.abs(host(z) - ref)) <= 1e-12 * np.abs(ref).max()
