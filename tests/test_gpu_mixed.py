"""Mixed precision: FP32 inner GMRES cycles (FP32 SpMV, FP32 ILU(k) solves, FP32
Krylov basis) inside FP64 iterative refinement, checked against the FP64 oracle.

Tolerances:
  * FP32 SpMV, per row i with k_i stored entries: |y - y_ref| <= (k_i + 2) u
    sum_j |a_ij x_j| (u = 2^-24): the first-order bound of a k-term dot product
    whose inputs are rounded to FP32 once and whose products and sums are FP32.
  * FP32 preconditioner apply: per entry, |z - z_ref| <= the FP32 rounding
    bound of the apply plus the oracle's FP64 one (tests/ras_bound.py: local
    errors of every row with u = 2^-24, factors and r rounded to FP32,
    propagated through the comparison-matrix triangular solves).
  * Mixed solves: the FP64 residual reaches tol (1e-8) and the solution agrees
    with the oracle's FP64 solution to 1e-6 relative.
"""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth
from ras_bound import check_apply

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def H():
    import torch
    from paper_1606_00545_gb300 import build
    build.build()
    from paper_1606_00545_gb300 import hecgpu
    hecgpu.load_library()
    torch.cuda.set_device(0)
    return hecgpu


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float64, device="cuda:0")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("ab", [(1.0, 0.0), (-0.5, 0.0), (-1.0, 1.0)])
@pytest.mark.parametrize("case", ["poisson2d", "irregular27", "random_tail", "ragged_tail"])
def test_spmv_f32_within_fp32_bound(H, orc, case, ab):
    """FP32 SpMV (four rows per thread) against the FP64 oracle, entry by
    entry, within the first-order bound of a k-term FP32 dot product plus the
    alpha/beta epilogue's roundings.  The ragged case has n = 5003 rows (not a
    multiple of four, five row blocks) and a CSR tail."""
    import torch
    alpha, beta = ab
    A, K = {"poisson2d": (synth.poisson2d_5pt(64), 0),
            "irregular27": (synth.stencil27_irregular(12, 4, 5), 0),
            "random_tail": (synth.random_sparse(1200, 0.02, seed=2), 3),
            "ragged_tail": (synth.random_sparse(5003, 0.002, seed=3), 2)}[case]
    x = synth.rhs_uniform(A.n, 5)
    yin = synth.rhs_uniform(A.n, 6).astype(np.float32).astype(np.float64)
    M = H.hec_build(A.row_ptr, A.col, A.val, ell_width=K)
    y = torch.tensor(yin, dtype=torch.float32, device="cuda:0")
    H.hec_spmv_f32(M, alpha, dev(x, torch.float32), beta, y if beta else None, y)
    got = host(y)
    ref = alpha * orc.spmv(A, x) + beta * yin
    scale = orc.spmv(synth.CSR(A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    bound = (A.row_lengths() + 4) * U32 * (abs(alpha) * scale + abs(beta) * np.abs(yin)) * 1.01 \
        + 1e-300
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)


@pytest.mark.parametrize("case", ["c1_poisson64_ilu0", "diffusion3d_ilu1_ras8", "irregular_ras4"])
def test_precond_f32_vs_fp64_oracle(H, orc, case):
    import torch
    A, k, nb, ov = {"c1_poisson64_ilu0": (synth.poisson2d_5pt(64), 0, 1, 0),
                    "diffusion3d_ilu1_ras8": (synth.diffusion3d_7pt_lognormal(16, 2.0, 2), 1, 8, 1),
                    "irregular_ras4": (synth.stencil27_irregular(10, 4, 5), 0, 4, 1)}[case]
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    r = synth.rhs_uniform(A.n, 1)
    z = torch.full((A.n,), float("nan"), dtype=torch.float32, device="cuda:0")
    H.hec_precond_apply_f32(P, dev(r, torch.float32), z)
    assert H.hec_precond_status(P) == H.OK
    got = host(z)
    R = orc.RAS(A, k, nb, ov)
    ref = R.apply(r)
    err = np.max(np.abs(got - ref)) / np.abs(ref).max()
    print("fp32 preconditioner, %s: max error / max|z| = %.2e" % (case, err))
    check_apply(orc, R, r, got, fp32=True, what=case, ref=ref)


def test_precond_global_scratch_after_nan_apply(H, orc):
    """A pass whose dependency window exceeds the shared-memory ring reads its
    dependencies from a global scratch that keeps the previous apply's values.
    In the uniform-width FP32 layout the padding of a dependency-free row
    points at a position not yet written in the current apply; after an apply
    of an all-NaN right-hand side (which leaves NaN in every scratch slot) the
    next apply must still be exact, in FP32 and FP64."""
    import torch
    A = synth.random_sparse_rows(24000, 6, seed=6)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    assert P.info()["global_passes"] > 0
    r = synth.rhs_uniform(A.n, 3)
    R = orc.RAS(A, 0, 1, 0)
    ref = R.apply(r)
    for fp32 in (True, False):
        dt = torch.float32 if fp32 else torch.float64
        apply = H.hec_precond_apply_f32 if fp32 else H.hec_precond_apply
        z = torch.empty(A.n, dtype=dt, device="cuda:0")
        apply(P, torch.full((A.n,), float("nan"), dtype=dt, device="cuda:0"), z)
        assert H.hec_precond_status(P) == H.OK
        assert not np.any(np.isfinite(host(z)))
        apply(P, dev(r, dt), z)
        assert H.hec_precond_status(P) == H.OK
        got = host(z)
        assert np.all(np.isfinite(got)), fp32
        check_apply(orc, R, r, got, fp32=fp32, what="after a NaN apply", ref=ref)
    assert P.layout(fp32=True)["fixed_width"] > 0  # the uniform-width kernel ran


def test_mixed_gmres_c1(H, orc):
    """64x64 Poisson, ILU(0), mixed GMRES(30): FP64 residual 1e-8."""
    A = synth.poisson2d_5pt(64)
    b = synth.rhs_uniform(A.n, 1)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=2000, restart=30, method=H.GMRES,
                          flags=H.MIXED_FP32)
    xg = host(x)
    assert info["status"] == H.OK and info["rel_resid"] <= 1e-8, info
    assert np.linalg.norm(b - orc.spmv(A, xg)) / np.linalg.norm(b) <= 1e-8
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) <= 1e-6


@pytest.mark.parametrize("k,nb,ov,m", [(1, 8, 1, 30), (0, 1, 0, 50)])
def test_mixed_matches_fp64_oracle_solution(H, orc, k, nb, ov, m):
    A = synth.diffusion3d_7pt_lognormal(20, 2.0, 2)
    b = synth.rhs_uniform(A.n, 3)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=5000, restart=m, method=H.GMRES,
                          flags=H.MIXED_FP32)
    xr, ir = orc.gmres(A, b, M=orc.RAS(A, k, nb, ov), tol=1e-8, maxit=5000, restart=m)
    xg = host(x)
    assert info["status"] == H.OK and info["rel_resid"] <= 1e-8, info
    err = np.linalg.norm(xg - xr) / np.linalg.norm(xr)
    print("mixed GMRES(%d): %d steps (oracle FP64: %d), error vs oracle %.2e"
          % (m, info["iters"], ir.iters, err))
    assert err <= 1e-6


def test_mixed_unpreconditioned(H, orc):
    A = synth.poisson2d_5pt(16)
    b = synth.rhs_uniform(A.n, 2)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, None, dev(b), x, tol=1e-9, maxit=4000, restart=40, method=H.GMRES,
                          flags=H.MIXED_FP32)
    assert info["status"] == H.OK
    assert np.linalg.norm(b - orc.spmv(A, host(x))) / np.linalg.norm(b) <= 1e-9


def test_mixed_rejects_bicgstab(H):
    A = synth.poisson2d_5pt(8)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    with pytest.raises(H.HecError):
        H.krylov_solve(M, None, dev(np.ones(A.n)), dev(np.zeros(A.n)), method=H.BICGSTAB,
                       flags=H.MIXED_FP32)


def test_c3_irregular_96_mixed_gmres50(H, orc):
    """96^3 27-point + 2% irregular rows (30-120 extra entries, N(0, 0.01)),
    diagonal 1.1 x off-diagonal row sum; ILU(0) on 64 RAS blocks; FP32 inner
    GMRES(50) with FP64 refinement to 1e-8.  Manufactured solution x*."""
    A = synth.stencil27_irregular(96, 4, 5)
    xs = synth.rhs_uniform(A.n, 6)
    b = orc.spmv(A, xs)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    inf = M.info()
    assert inf["tail_rows"] > 0  # the HEC tail is exercised
    P = H.ilu_k_setup(M, 0, 64, 1)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=5000, restart=50, method=H.GMRES,
                          flags=H.MIXED_FP32)
    xg = host(x)
    assert info["status"] == H.OK and info["rel_resid"] <= 1e-8, info
    assert np.linalg.norm(b - orc.spmv(A, xg)) / np.linalg.norm(b) <= 1e-8
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= 1e-6


def test_mixed_ill_conditioned_converges(H, orc):
    """An ill-conditioned 859^2 2D log-normal (sigma = 2) system with ILU(1)
    on RAS blocks (about 4,000 GMRES(30) steps): the mixed solve reaches the
    FP64 residual 1e-8, by FP32 refinement alone or with an FP64 finish."""
    req = synth.serving_requests(24, 8)[16]
    A = synth.serving_matrix(req)
    b = synth.rhs_uniform(A.n, 16)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, req["k"], 46, 1)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=20000, restart=30, method=H.GMRES,
                          flags=H.MIXED_FP32 | H.X0_ZERO)
    print("ill-conditioned mixed solve:", info)
    assert info["status"] == H.OK, info
    assert np.linalg.norm(b - orc.spmv(A, host(x))) <= 1e-8 * np.linalg.norm(b)


def test_mixed_unreachable_tol_switches_to_fp64(H):
    """A tolerance below what the arithmetic reaches: the mixed solve
    stagnates, switches to FP64 and ends at maxit."""
    A = synth.diffusion2d_5pt_lognormal(48, 2.0, 3)
    b = synth.rhs_uniform(A.n, 4)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-17, maxit=1500, restart=30, method=H.GMRES,
                          flags=H.MIXED_FP32 | H.X0_ZERO)
    assert info["fp64_finish"] == 1 and info["status"] == H.MAXIT and info["iters"] == 1500
    assert info["rel_resid"] < 1e-11
