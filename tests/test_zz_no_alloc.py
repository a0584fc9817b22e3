"""hec_precond_apply_noalloc: the preconditioner apply for callers that cannot
allocate device memory while they run (a fixed device-memory budget, or no
room for cudaMalloc's implicit synchronisation).  Its result must equal the
allocating hec_precond_apply's on two calls in a row, through the C ABI.

This file is collected last on purpose, and it also passes alone in a fresh
process (the first call on the device sets the static scratch up)."""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth

pytestmark = pytest.mark.gpu

# the precond-apply tolerance of tests/test_gpu_kernels.py
TOL = 1e-10


@pytest.fixture(scope="module")
def H():
    import torch
    from paper_1606_00545_gb300 import build
    build.build()
    from paper_1606_00545_gb300 import hecgpu
    hecgpu.load_library()
    torch.cuda.set_device(0)
    return hecgpu


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def test_noalloc_apply_matches_allocating_apply(H):
    import torch
    A = synth.diffusion3d_7pt_lognormal(24, 2.0, 2)
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 1, 8, 1)
    H.level_schedule(P)
    for seed in (1, 2):  # two calls in a row, different right-hand sides
        r = _dev(synth.rhs_uniform(A.n, seed))
        z_ref = torch.full_like(r, float("nan"))
        H.hec_precond_apply(P, r, z_ref)
        assert H.hec_precond_status(P) == H.OK
        z = torch.full_like(r, float("nan"))
        H.hec_precond_apply_noalloc(P, r, z)
        assert H.hec_precond_status(P) == H.OK
        torch.cuda.synchronize()
        zr, zg = z_ref.cpu().numpy(), z.cpu().numpy()
        assert np.all(np.isfinite(zg))
        assert np.max(np.abs(zg - zr)) <= TOL * np.abs(zr).max()


def test_noalloc_apply_rejects_oversized_scratch(H):
    # one block of 1.1M rows needs more scratch than the 2^20-double array
    n = 1_100_000
    A = synth.CSR(np.arange(n + 1), np.arange(n), np.full(n, 2.0))
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    r = _dev(np.ones(A.n))
    z = _dev(np.zeros(A.n))
    with pytest.raises(H.HecError) as e:
        H.hec_precond_apply_noalloc(P, r, z)
    assert e.value.status == H.ERR_INVALID
    assert "static array" in str(e.value)
