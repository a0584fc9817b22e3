"""Numeric refactorisation on the GPU (hec_refactor): the same sparsity
pattern with new values.  The GPU elimination performs the host's operations
in the host's order, so factors, layouts and applies must equal those of a
preconditioner built from scratch on the new matrix bit for bit, and the
factors must equal the oracle's ILU(k) of the new blocks."""
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


def factors(H, P):
    return [P.factor(b) for b in range(P.info()["nblocks"])]


@pytest.mark.parametrize("k,nb,ov", [(0, 1, 0), (1, 8, 1), (2, 4, 0)])
def test_refactor_equals_fresh_setup_bit_for_bit(H, orc, k, nb, ov):
    import torch
    A0 = synth.diffusion3d_7pt_lognormal(14, 2.0, 2)
    A1 = synth.diffusion3d_7pt_lognormal(14, 2.0, 5)  # same pattern, new values
    assert np.array_equal(A0.col, A1.col) and not np.array_equal(A0.val, A1.val)
    M = H.hec_build(A0.row_ptr, A0.col, A0.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    r = synth.rhs_uniform(A0.n, 3)
    z32 = dev(np.zeros(A0.n), torch.float32)
    H.hec_precond_apply_f32(P, dev(r, torch.float32), z32)  # builds the FP32 layout
    H.hec_refactor(M, P, A1.val)
    # a preconditioner built from scratch on the new matrix
    M1 = H.hec_build(A1.row_ptr, A1.col, A1.val)
    P1 = H.ilu_k_setup(M1, k, nb, ov)
    H.level_schedule(P1)
    for b in range(nb):
        f_ref, f_got = P1.factor(b), P.factor(b)
        assert np.array_equal(f_got[1], f_ref[1]) and np.array_equal(f_got[2], f_ref[2]), b
    # the oracle's ILU(k) of the new blocks
    R1 = orc.RAS(A1, k, nb, ov)
    for b in range(nb):
        _, _, _, F = R1.block(b)
        assert np.array_equal(P.factor(b)[2], F.val), b
    # applies: FP64 and FP32 layouts refilled on the device
    z, z1 = dev(np.zeros(A0.n)), dev(np.zeros(A0.n))
    H.hec_precond_apply(P, dev(r), z)
    H.hec_precond_apply(P1, dev(r), z1)
    assert np.array_equal(host(z), host(z1))
    z32b = dev(np.zeros(A0.n), torch.float32)
    H.hec_precond_apply_f32(P, dev(r, torch.float32), z32)
    H.hec_precond_apply_f32(P1, dev(r, torch.float32), z32b)
    assert np.array_equal(host(z32), host(z32b))
    # the layouts refilled on the device equal those packed from scratch, byte for byte
    for fp32 in (False, True):
        la, lb = P.layout(fp32=fp32), P1.layout(fp32=fp32)
        assert np.array_equal(la["chunks"], lb["chunks"]) and np.array_equal(la["programs"],
                                                                              lb["programs"])
        assert np.array_equal(la["pack"], lb["pack"]), fp32
    # SpMV on the new values
    y = dev(np.zeros(A0.n))
    H.hec_spmv(M, 1.0, dev(r), 0.0, None, y)
    ref = orc.spmv(A1, r)
    scale = orc.spmv(synth.CSR(A1.row_ptr, A1.col, np.abs(A1.val)), np.abs(r))
    assert np.all(np.abs(host(y) - ref) <= 1e-12 * scale)
    # and back to the first matrix
    H.hec_refactor(M, P, dev(A0.val))
    P0 = H.ilu_k_setup(H.hec_build(A0.row_ptr, A0.col, A0.val), k, nb, ov)
    for b in range(nb):
        assert np.array_equal(P.factor(b)[2], P0.factor(b)[2])


def test_refactored_solve_matches_oracle(H, orc):
    A0 = synth.diffusion3d_7pt_lognormal(20, 2.0, 2)
    A1 = synth.diffusion3d_7pt_lognormal(20, 2.0, 9)
    b = synth.rhs_uniform(A0.n, 4)
    M = H.hec_build(A0.row_ptr, A0.col, A0.val)
    P = H.ilu_k_setup(M, 1, 8, 1)
    H.level_schedule(P)
    x = dev(np.zeros(A0.n))
    H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=500, method=H.BICGSTAB)  # graph built
    H.hec_refactor(M, P, A1.val)
    x = dev(np.zeros(A0.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=500, method=H.BICGSTAB)
    xr, ir = orc.bicgstab(A1, b, M=orc.RAS(A1, 1, 8, 1), tol=1e-8, maxit=500)
    xg = host(x)
    assert info["status"] == H.OK and ir.status == orc.OK
    assert np.linalg.norm(b - orc.spmv(A1, xg)) / np.linalg.norm(b) <= 1e-8
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-6
    assert abs(info["iters"] - ir.iters) <= max(2, 0.1 * ir.iters)


def test_refactor_jacobi_and_matrix_only(H, orc):
    A0 = synth.diffusion2d_5pt_lognormal(30, 1.0, 1)
    A1 = synth.diffusion2d_5pt_lognormal(30, 1.0, 3)
    M = H.hec_build(A0.row_ptr, A0.col, A0.val)
    J = H.jacobi_setup(M, 0.7)
    H.hec_refactor(M, J, dev(A1.val))
    r = synth.rhs_uniform(A0.n, 2)
    z = dev(np.zeros(A0.n))
    H.hec_precond_apply(J, dev(r), z)
    assert np.array_equal(host(z), orc.Jacobi(A1, 0.7).apply(r))
    # the matrix alone; its host export follows
    H.hec_refactor(M, None, A0.val)
    y = dev(np.zeros(A0.n))
    H.hec_spmv(M, 1.0, dev(r), 0.0, None, y)
    assert np.allclose(host(y), orc.spmv(A0, r), rtol=1e-13, atol=0)
    ex, ex0 = M.export(), H.hec_build(A0.row_ptr, A0.col, A0.val).export()
    assert np.array_equal(ex["ell_val"], ex0["ell_val"])
    assert np.array_equal(ex["tail_val"], ex0["tail_val"])


def test_refactor_zero_pivot_and_bad_handles(H):
    A = synth.tridiagonal(50, seed=2)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    bad = A.val.copy()
    bad[A.row_ptr[0]] = 0.0  # a_00 = 0: the first pivot
    with pytest.raises(H.HecError) as e:
        H.hec_refactor(M, P, bad)
    assert e.value.status == H.ERR_ZERO_PIVOT
    H.hec_refactor(M, P, A.val)  # usable again
    z = dev(np.zeros(A.n))
    H.hec_precond_apply(P, dev(np.ones(A.n)), z)
    assert H.hec_precond_status(P) == H.OK
    other = H.hec_build(A.row_ptr, A.col, A.val)
    with pytest.raises(H.HecError):
        H.hec_refactor(other, P, A.val)
