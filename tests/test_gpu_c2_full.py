"""The benchmark's own workload at full size, in the launch configuration
bench.py times: 128^3 7-point diffusion with log-normal (sigma = 2) face
coefficients (seed 2), ILU(1) on 64 RAS blocks with overlap 1, BiCGSTAB.

The oracle computes what it can in seconds: SpMV rows in sampled ranges,
the whole RAS/ILU(1) apply, and the first BiCGSTAB iterations; the full
solve is checked through its true residual (the oracle's SpMV).  Bars as
elsewhere: SpMV 1e-12 of sum |a_ij x_j| per row, FP64 and FP32 applies
entry by entry within the rounding bounds of tests/ras_bound.py, iterates
after 5 passes 1e-9, residual 1e-8.  The triangular solve runs as bench.py
runs it: every RAS block split over a chain of thread-block-cluster CTAs."""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth
from ras_bound import check_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1606_00545_gb300 import build
    build.build()
    from paper_1606_00545_gb300 import hecgpu as H
    H.load_library()
    torch.cuda.set_device(0)
    A = synth.diffusion3d_7pt_lognormal(128, 2.0, 2)
    b = synth.rhs_uniform(A.n, 3)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 1, 64, 1)
    H.level_schedule(P)
    assert P.info()["split_blocks"] == 64
    return H, A, b, M, P


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), device="cuda:0", dtype=dtype or torch.float64)


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_c2_spmv_sampled_rows(setup, orc):
    H, A, b, M, P = setup
    x = synth.rhs_uniform(A.n, 11)
    y = dev(np.zeros(A.n))
    H.hec_spmv(M, 1.0, dev(x), 0.0, None, y)
    got = host(y)
    rng = np.random.default_rng(0)
    absA = synth.CSR(A.row_ptr, A.col, np.abs(A.val))
    for lo in np.concatenate([[0, A.n - 4096], rng.integers(0, A.n - 4096, 6)]):
        sub = slice(int(lo), int(lo) + 4096)
        ref = orc.spmv_rows(A, x, int(lo), int(lo) + 4096)
        scale = orc.spmv_rows(absA, np.abs(x), int(lo), int(lo) + 4096)
        assert np.all(np.abs(got[sub] - ref) <= 1e-12 * scale)


def test_c2_precond_apply_full(setup, orc):
    import torch
    H, A, b, M, P = setup
    r = synth.rhs_uniform(A.n, 7)
    z = dev(np.zeros(A.n))
    H.hec_precond_apply(P, dev(r), z)
    assert H.hec_precond_status(P) == H.OK
    R = orc.RAS(A, 1, 64, 1)
    zr = R.apply(r)
    check_apply(orc, R, r, host(z), what="C2 FP64", ref=zr)
    z32 = dev(np.zeros(A.n), torch.float32)
    H.hec_precond_apply_f32(P, dev(r, torch.float32), z32)
    assert H.hec_precond_status(P) == H.OK
    check_apply(orc, R, r, host(z32), fp32=True, what="C2 FP32", ref=zr)


def test_c2_bicgstab_first_iterates_and_full_solve(setup, orc):
    H, A, b, M, P = setup
    R = orc.RAS(A, 1, 64, 1)
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-30, maxit=5, method=H.BICGSTAB)
    xr, ir = orc.bicgstab(A, b, M=R, tol=1e-30, maxit=5)
    assert info["status"] == H.MAXIT and info["iters"] == 5 == ir.iters
    assert np.linalg.norm(host(x) - xr) <= 1e-9 * np.linalg.norm(xr)
    # the full solve, as the benchmark runs it
    x = dev(np.zeros(A.n))
    info = H.krylov_solve(M, P, dev(b), x, tol=1e-8, maxit=20000, method=H.BICGSTAB,
                          flags=H.X0_ZERO)
    xg = host(x)
    assert info["status"] == H.OK and info["rel_resid"] <= 1e-8
    assert np.linalg.norm(b - orc.spmv(A, xg)) / np.linalg.norm(b) <= 1e-8
