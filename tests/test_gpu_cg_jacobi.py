"""Preconditioned CG (Section 2.7 lists it among the Krylov solvers) and the
damped-Jacobi preconditioner z = omega D^{-1} r (Section 2.8) on the GPU,
through the C ABI, against the FP64 oracle on the same seeded inputs.

Bars: the Jacobi apply is one FP64 multiply by the same omega / a_ii on both
sides, so it is bit-exact; solves reach relative residual <= tol (recomputed
by the oracle's SpMV), the solution is within 1e-6 of the oracle's, and
iteration counts agree within 10% (the fused reductions sum in another
order, so iterates are not bit-equal).
"""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth

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


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), device="cuda:0", dtype=dtype or torch.float64)


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_resid(orc, A, b, x):
    return np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)


def close_iters(a, b):
    return abs(a - b) <= max(2, 0.1 * b)


@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_jacobi_apply_bit_exact(H, orc, omega):
    A = synth.stencil27_irregular(12, 4, 5)
    r = synth.rhs_uniform(A.n, 2)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.jacobi_setup(M, omega)
    H.level_schedule(P)  # a no-op for Jacobi
    z = dev(np.zeros(A.n))
    H.hec_precond_apply(P, dev(r), z)
    zr = orc.Jacobi(A, omega).apply(r)
    assert np.array_equal(host(z), zr)
    assert H.hec_precond_status(P) == H.OK
    # the allocation-free entry point takes a Jacobi handle too
    z2 = dev(np.zeros(A.n))
    H.hec_precond_apply_noalloc(P, dev(r), z2)
    assert np.array_equal(host(z2), zr)
    # FP32: one rounding of omega / a_ii and of r, one FP32 multiply
    import torch
    z32 = dev(np.zeros(A.n), torch.float32)
    H.hec_precond_apply_f32(P, dev(r, torch.float32), z32)
    ref32 = (zr.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(host(z32) - ref32) / np.abs(ref32)) <= 3 * 2.0 ** -24
    info = P.info()
    assert info["k"] == -1 and info["nblocks"] == 0 and info["apply_bytes"] == 24 * A.n


def test_jacobi_rejects_zero_diagonal_and_bad_omega(H):
    # a zero diagonal entry stored explicitly
    A = synth.CSR(np.array([0, 2, 3]), np.array([0, 1, 1]), np.array([1.0, 2.0, 0.0]))
    M = H.hec_build(A.row_ptr, A.col, A.val)
    with pytest.raises(H.HecError) as e:
        H.jacobi_setup(M, 1.0)
    assert e.value.status == H.ERR_ZERO_PIVOT
    B = synth.poisson2d_5pt(4)
    MB = H.hec_build(B.row_ptr, B.col, B.val)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(H.HecError):
            H.jacobi_setup(MB, bad)


@pytest.mark.parametrize("prec", ["none", "ilu0", "ilu1", "jacobi"])
def test_cg_c1_poisson64(H, orc, prec):
    """64x64 5-point Poisson (the small workload), rhs uniform[-1,1] seed 1, tol 1e-8."""
    A = synth.poisson2d_5pt(64)
    b = synth.rhs_uniform(A.n, 1)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    if prec == "jacobi":
        P, R = H.jacobi_setup(M, 0.8), orc.Jacobi(A, 0.8)
    elif prec.startswith("ilu"):
        k = int(prec[-1])
        P, R = H.ilu_k_setup(M, k, 1, 0), orc.RAS(A, k, 1, 0)
        H.level_schedule(P)
    else:
        P, R = None, None
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=2000, method=H.CG)
    xr, ir = orc.cg(A, b, M=R, tol=1e-8, maxit=2000)
    xg = host(x)
    assert info["status"] == H.OK and ir.status == orc.OK
    assert info["rel_resid"] <= 1e-8 and rel_resid(orc, A, b, xg) <= 1e-8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    assert close_iters(info["iters"], ir.iters), (info["iters"], ir.iters)


def test_cg_diffusion3d_lognormal_manufactured(H, orc):
    A = synth.diffusion3d_7pt_lognormal(24, 1.0, 11)
    xs = synth.rhs_uniform(A.n, 4)
    b = orc.spmv(A, xs)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-10, maxit=3000, method=H.CG)
    xr, ir = orc.cg(A, b, M=orc.RAS(A, 0, 1, 0), tol=1e-10, maxit=3000)
    xg = host(x)
    assert info["status"] == H.OK and rel_resid(orc, A, b, xg) <= 1e-10
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) <= 1e-6
    assert close_iters(info["iters"], ir.iters), (info["iters"], ir.iters)


def test_cg_eager_equals_graph(H):
    A = synth.diffusion2d_5pt_lognormal(40, 1.0, 2)
    b = synth.rhs_uniform(A.n, 5)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.jacobi_setup(M, 1.0)
    x1, x2 = dev(np.zeros(A.n)), dev(np.zeros(A.n))
    i1 = H.krylov_solve(M, P, dev(b), x1, tol=1e-9, maxit=3000, method=H.CG)
    i2 = H.krylov_solve(M, P, dev(b), x2, tol=1e-9, maxit=3000, method=H.CG,
                        flags=H.SOLVE_EAGER)
    assert i1["iters"] == i2["iters"] and np.array_equal(host(x1), host(x2))


def test_cg_maxit_breakdown_zero_rhs(H, orc):
    A = synth.poisson2d_5pt(32)
    b = synth.rhs_uniform(A.n, 6)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, None, dev(b), x, tol=1e-12, maxit=7, method=H.CG)
    xr, ir = orc.cg(A, b, tol=1e-12, maxit=7)
    assert info["status"] == H.MAXIT and info["iters"] == 7 and ir.iters == 7
    assert np.linalg.norm(host(x) - xr) <= 1e-10 * np.linalg.norm(xr)
    # an indefinite matrix: (A p, p) = 0 at the first pass
    D = synth.CSR(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, -1.0]))
    MD = H.hec_build(D.row_ptr, D.col, D.val)
    xd = dev(np.zeros(2))
    info = H.krylov_solve(MD, None, dev([1.0, 1.0]), xd, tol=1e-12, maxit=5, method=H.CG)
    assert info["status"] == H.BREAKDOWN
    # b = 0 gives x = 0
    x0 = dev(np.ones(A.n))
    info = H.krylov_solve(M, None, dev(np.zeros(A.n)), x0, tol=1e-8, maxit=50, method=H.CG)
    assert info["status"] == H.OK and np.all(host(x0) == 0)


@pytest.mark.parametrize("method", ["bicgstab", "gmres", "gmres_mixed"])
def test_jacobi_preconditions_every_solver(H, orc, method):
    A = synth.diffusion2d_5pt_lognormal(48, 1.0, 9)
    b = synth.rhs_uniform(A.n, 2)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.jacobi_setup(M, 1.0)
    R = orc.Jacobi(A, 1.0)
    x = dev(np.zeros(A.n))
    if method == "bicgstab":
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=3000, method=H.BICGSTAB)
        xr, ir = orc.bicgstab(A, b, M=R, tol=1e-8, maxit=3000)
    else:
        flags = H.MIXED_FP32 if method == "gmres_mixed" else 0
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=6000, restart=30,
                              method=H.GMRES, flags=flags)
        xr, ir = orc.gmres(A, b, M=R, tol=1e-8, maxit=6000, restart=30)
    xg = host(x)
    assert info["status"] == H.OK and ir.status == orc.OK
    assert rel_resid(orc, A, b, xg) <= 1e-8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    if method != "gmres_mixed":
        assert close_iters(info["iters"], ir.iters), (info["iters"], ir.iters)
