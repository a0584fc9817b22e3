"""GPU Krylov solves (BiCGSTAB, Algorithm 4; restarted GMRES(m)) through the C
ABI, checked against the FP64 oracle's solves on the same seeded inputs.

Bars: relative residual <= tol (recomputed from scratch by the oracle's SpMV
on the returned x), solution relative error <= 1e-6 against the oracle's
solution (or a manufactured / dense solution), iteration counts within 10%
of the oracle's (the two round differently, so iterates are not bit-equal).
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


def dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def true_rel_resid(orc, A, b, x):
    return np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)


def setup(H, A, k, nb, ov):
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    return M, P


def close_iters(a, b):
    return abs(a - b) <= max(2, 0.1 * b)


def test_c1_poisson64_ilu0_gmres30(H, orc):
    """64x64 5-point Poisson, rhs uniform[-1,1] seed 1, ILU(0) + GMRES(30), tol 1e-8."""
    A = synth.poisson2d_5pt(64)
    b = synth.rhs_uniform(A.n, 1)
    M, P = setup(H, A, 0, 1, 0)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=1000, restart=30, method=H.GMRES)
    xr, ir = orc.gmres(A, b, M=orc.RAS(A, 0, 1, 0), tol=1e-8, maxit=1000, restart=30)
    xg = host(x)
    assert info["status"] == H.OK and ir.status == orc.OK
    assert info["rel_resid"] <= 1e-8 and true_rel_resid(orc, A, b, xg) <= 1e-8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) <= 1e-6
    assert close_iters(info["iters"], ir.iters), (info["iters"], ir.iters)
    assert info["kernel_launches"] > info["iters"]


@pytest.mark.parametrize("method", ["bicgstab", "gmres"])
@pytest.mark.parametrize("k,nb,ov", [(0, 1, 0), (1, 8, 1), (2, 4, 0)])
def test_diffusion3d_solves_match_oracle(H, orc, method, k, nb, ov):
    A = synth.diffusion3d_7pt_lognormal(20, 2.0, 2)
    b = synth.rhs_uniform(A.n, 3)
    M, P = setup(H, A, k, nb, ov)
    R = orc.RAS(A, k, nb, ov)
    x = dev(np.zeros(A.n))
    if method == "bicgstab":
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=2000, method=H.BICGSTAB)
        xr, ir = orc.bicgstab(A, b, M=R, tol=1e-8, maxit=2000)
    else:
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=2000, restart=30, method=H.GMRES)
        xr, ir = orc.gmres(A, b, M=R, tol=1e-8, maxit=2000, restart=30)
    xg = host(x)
    assert info["status"] == H.OK, info
    assert true_rel_resid(orc, A, b, xg) <= 1e-8
    if method == "gmres":
        assert info["rel_resid"] <= 1e-8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    assert close_iters(info["iters"], ir.iters), (info["iters"], ir.iters)


@pytest.mark.parametrize("method", [0, 1])
def test_manufactured_solution_irregular(H, orc, method):
    A = synth.stencil27_irregular(14, 4, 5)
    xs = synth.rhs_uniform(A.n, 6)
    b = orc.spmv(A, xs)
    M, P = setup(H, A, 0, 4, 1)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-10, maxit=1000, restart=50, method=method)
    assert info["status"] == H.OK
    assert np.linalg.norm(host(x) - xs) / np.linalg.norm(xs) <= 1e-6


def test_host_buffers_match_device_path(H, orc):
    A = synth.diffusion2d_5pt_lognormal(40, 2.0, 1)
    b = synth.rhs_uniform(A.n, 2)
    M, P = setup(H, A, 1, 4, 1)
    for method in (H.BICGSTAB, H.GMRES):
        xd = dev(np.zeros(A.n))
        i1 = H.krylov_solve(M, P, dev(b), xd, tol=1e-9, maxit=500, method=method)
        xh = np.zeros(A.n)
        i2 = H.krylov_solve(M, P, b.copy(), xh, tol=1e-9, maxit=500, method=method)
        assert np.array_equal(host(xd), xh)  # same kernels, same order
        assert i1["iters"] == i2["iters"]
        assert i2["h2d_bytes"] == 2 * 8 * A.n and i2["d2h_bytes"] == 8 * A.n
        assert i1["h2d_bytes"] == 0 and i1["d2h_bytes"] == 0


def test_eager_solve_matches_graph_solve(H):
    """HEC_SOLVE_EAGER runs the same kernels from a host loop: identical results."""
    A = synth.diffusion2d_5pt_lognormal(30, 2.0, 3)
    b = synth.rhs_uniform(A.n, 6)
    M, P = setup(H, A, 1, 3, 1)
    for method in (H.BICGSTAB, H.GMRES):
        xg = dev(np.zeros(A.n))
        ig = H.krylov_solve(M, P, dev(b), xg, tol=1e-9, maxit=500, restart=8, method=method)
        xe = dev(np.zeros(A.n))
        ie = H.krylov_solve(M, P, dev(b), xe, tol=1e-9, maxit=500, restart=8, method=method,
                            flags=H.SOLVE_EAGER)
        assert np.array_equal(host(xg), host(xe))
        assert ig["iters"] == ie["iters"] and ig["restarts"] == ie["restarts"]
        assert ig["status"] == ie["status"] == H.OK


def test_repeat_solves_are_identical(H):
    A = synth.poisson2d_5pt(30)
    b = synth.rhs_uniform(A.n, 4)
    M, P = setup(H, A, 0, 2, 1)
    outs = []
    for _ in range(3):
        x = dev(np.zeros(A.n))
        H.krylov_solve(M, P, dev(b), x, tol=1e-10, maxit=500, method=H.BICGSTAB)
        outs.append(host(x))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_unpreconditioned_and_initial_guess(H, orc):
    A = synth.poisson2d_5pt(10)
    b = synth.rhs_uniform(A.n, 5)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    for method in (H.BICGSTAB, H.GMRES):
        x = dev(np.zeros(A.n))
        info = H.krylov_solve(M, None, dev(b), x, tol=1e-10, maxit=1000, restart=A.n,
                              method=method)
        assert info["status"] == H.OK
        assert true_rel_resid(orc, A, b, host(x)) <= 1e-10
    # GMRES(n) without preconditioner terminates within n steps
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, None, dev(b), x, tol=1e-10, maxit=A.n, restart=A.n, method=H.GMRES)
    assert info["status"] == H.OK and info["iters"] <= A.n
    # starting from the solution: zero iterations
    xs = dev(np.linalg.solve(A.to_dense(), b))
    info = H.krylov_solve(M, None, dev(b), xs, tol=1e-8, maxit=100, method=H.BICGSTAB)
    assert info["iters"] == 0 and info["status"] == H.OK


def test_exact_preconditioner_one_step(H):
    A = synth.tridiagonal(3000, seed=2)
    b = synth.rhs_uniform(A.n, 1)
    M, P = setup(H, A, 0, 1, 0)
    for method in (H.BICGSTAB, H.GMRES):
        x = dev(np.zeros(A.n))
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-12, maxit=10, method=method)
        assert info["iters"] == 1 and info["rel_resid"] <= 1e-12


def test_maxit_zero_rhs_and_breakdown(H):
    A = synth.diffusion2d_5pt_lognormal(20, 2.0, 1)
    b = synth.rhs_uniform(A.n, 1)
    M, P = setup(H, A, 0, 1, 0)
    for method in (H.BICGSTAB, H.GMRES):
        x = dev(np.zeros(A.n))
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-14, maxit=3, restart=2, method=method)
        assert info["status"] == H.MAXIT and info["iters"] == 3
        x = dev(np.ones(A.n))
        info = H.krylov_solve(M, P, dev(np.zeros(A.n)), x, tol=1e-8, maxit=10, method=method)
        assert info["status"] == H.OK and info["iters"] == 0 and np.all(host(x) == 0)
    # skew-symmetric 2x2: (r0, A r0) = 0 -> BiCGSTAB breakdown
    S = H.hec_build(np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([0.0, 1.0, -1.0, 0.0]))
    x = dev(np.zeros(2))
    info = H.krylov_solve(S, None, dev(np.array([1.0, 2.0])), x, tol=1e-10, maxit=10,
                          method=H.BICGSTAB)
    assert info["status"] == H.BREAKDOWN


def test_invalid_arguments(H):
    A = synth.poisson2d_5pt(8)
    M, P = setup(H, A, 0, 1, 0)
    b = dev(np.ones(A.n))
    x = dev(np.zeros(A.n))
    with pytest.raises(H.HecError):
        H.krylov_solve(M, P, b, x, restart=0, method=H.GMRES)
    with pytest.raises(H.HecError):
        H.krylov_solve(M, P, b, x, restart=500, method=H.GMRES)
    B = H.hec_build(A.row_ptr, A.col, A.val)
    with pytest.raises(H.HecError):
        H.krylov_solve(B, P, b, x)  # preconditioner of another matrix


@pytest.mark.parametrize("method,flags", [("bicgstab", 0), ("gmres", 0), ("gmres", "mixed"),
                                          ("cg", 0)])
def test_nan_rhs_ends_in_breakdown(H, orc, method, flags):
    """Fault injected on the host: a NaN in b ends the solve with
    HEC_BREAKDOWN (no hang, no device error); a clean solve on the same
    handles still works afterwards."""
    A = synth.diffusion2d_5pt_lognormal(32, 1.0, 4)
    M, P = setup(H, A, 0, 1, 0)
    b = synth.rhs_uniform(A.n, 8)
    bad = b.copy()
    bad[A.n // 3] = np.nan
    m = {"bicgstab": H.BICGSTAB, "gmres": H.GMRES, "cg": H.CG}[method]
    fl = H.MIXED_FP32 if flags == "mixed" else 0
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(bad), x, tol=1e-8, maxit=200, restart=30, method=m,
                          flags=fl)
    assert info["status"] == H.BREAKDOWN
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=2000, restart=30, method=m, flags=fl)
    assert info["status"] == H.OK
    assert true_rel_resid(orc, A, b, host(x)) <= 1e-8


def test_workspace_bytes_zero_once_solved(H):
    """hec_workspace_bytes counts what the first solve with given arguments
    allocates; once that solve has run, its workspace (and, for the mixed
    form, the FP32 copies) stays cached in the handles and the count is 0."""
    A = synth.diffusion2d_5pt_lognormal(30, 1.0, 2)
    b = synth.rhs_uniform(A.n, 3)
    M, P = setup(H, A, 0, 2, 1)
    for method, restart, flags in ((H.GMRES, 20, 0), (H.GMRES, 20, H.MIXED_FP32),
                                   (H.BICGSTAB, 0, 0)):
        assert H.hec_workspace_bytes(M, P, restart, method, flags) > 0
        x = dev(np.zeros(A.n))
        info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=500, restart=max(restart, 1),
                              method=method, flags=flags)
        assert info["status"] == H.OK
        assert H.hec_workspace_bytes(M, P, restart, method, flags) == 0
    assert H.hec_workspace_bytes(M, P, 25, H.GMRES) > 0  # another restart length
    assert H.hec_workspace_bytes(M, None, 0, H.CG) > 0  # no preconditioner: its own cache
