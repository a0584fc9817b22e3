"""hec_precond_apply_noalloc: the preconditioner apply for callers that cannot
allocate device memory while they run (a fixed device-memory budget, or no
room for cudaMalloc's implicit synchronisation).  Its result must equal the
allocating hec_precond_apply's on two calls in a row, through the C ABI.

This file is collected last on purpose, and it also passes alone in a fresh
process (the first call on the device sets the static scratch up)."""
import numpy as np
import pytest

from paper_1606_00545_gb300 import synth
from ras_bound import apply_bound

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


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def _same(orc, R, r, zg, zr):
    """The apply tolerance of the other parity tests: per entry, the FP64
    rounding bound of one apply, twice (tests/ras_bound.py)."""
    assert np.all(np.isfinite(zg))
    bound = 2 * apply_bound(orc, R, r)
    assert np.all(np.abs(zg - zr) <= bound)


def _setup(H, A, k, nb, ov):
    M = H.hec_build(A.row_ptr, A.col, A.val)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    return M, P


def _both(H, P, r):
    import torch
    z_ref = torch.full_like(r, float("nan"))
    H.hec_precond_apply(P, r, z_ref)
    assert H.hec_precond_status(P) == H.OK
    z = torch.full_like(r, float("nan"))
    H.hec_precond_apply_noalloc(P, r, z)
    assert H.hec_precond_status(P) == H.OK
    torch.cuda.synchronize()
    return z.cpu().numpy(), z_ref.cpu().numpy()


def test_noalloc_apply_matches_allocating_apply(H, orc):
    A = synth.diffusion3d_7pt_lognormal(24, 2.0, 2)
    M, P = _setup(H, A, 1, 8, 1)
    R = orc.RAS(A, 1, 8, 1)
    for seed in (1, 2):  # two calls in a row, different right-hand sides
        r = synth.rhs_uniform(A.n, seed)
        zg, zr = _both(H, P, _dev(r))
        _same(orc, R, r, zg, zr)


def test_noalloc_apply_with_global_scratch_pass(H, orc):
    """The static array keeps whatever the last call left in it.  A
    preconditioner whose dependency window does not fit shared memory reads
    dependencies from that array: after a call with an all-NaN right-hand
    side (which leaves NaN in every slot it writes), a call with a finite one
    must match the allocating apply, and so must a call on a second,
    different preconditioner after it."""
    import torch
    A = synth.random_sparse_rows(24000, 6, seed=6)
    M, P = _setup(H, A, 0, 1, 0)
    assert P.info()["global_passes"] > 0
    R = orc.RAS(A, 0, 1, 0)
    z = torch.zeros(A.n, dtype=torch.float64, device="cuda:0")
    H.hec_precond_apply_noalloc(P, _dev(np.full(A.n, np.nan)), z)
    assert H.hec_precond_status(P) == H.OK
    assert not np.any(np.isfinite(z.cpu().numpy()))
    r = synth.rhs_uniform(A.n, 4)
    zg, zr = _both(H, P, _dev(r))
    _same(orc, R, r, zg, zr)
    A2 = synth.diffusion3d_7pt_lognormal(20, 2.0, 3)
    M2, P2 = _setup(H, A2, 1, 4, 1)
    r2 = synth.rhs_uniform(A2.n, 5)
    zg, zr = _both(H, P2, _dev(r2))
    _same(orc, orc.RAS(A2, 1, 4, 1), r2, zg, zr)


def test_noalloc_apply_allocates_nothing(H):
    """After a first call (which looks the array's address up), further calls
    change neither the device's free memory nor the memory PyTorch's
    allocator holds."""
    import torch
    A = synth.diffusion3d_7pt_lognormal(24, 2.0, 2)
    M, P = _setup(H, A, 1, 8, 1)
    r = _dev(synth.rhs_uniform(A.n, 1))
    z = torch.zeros_like(r)
    H.hec_precond_apply_noalloc(P, r, z)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(5):
        H.hec_precond_apply_noalloc(P, r, z)
    assert H.hec_precond_status(P) == H.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def _diag(n):
    return synth.CSR(np.arange(n + 1), np.arange(n), np.full(n, 2.0))


def test_noalloc_apply_scratch_limit(H):
    """A diagonal matrix's y scratch holds one value per row: 2^20 rows fit
    the 2^20-double array exactly and are accepted; one row more is
    rejected before any device work."""
    import torch
    n = 1 << 20
    M, P = _setup(H, _diag(n), 0, 1, 0)
    r = _dev(np.ones(n))
    z = torch.zeros_like(r)
    H.hec_precond_apply_noalloc(P, r, z)
    assert H.hec_precond_status(P) == H.OK
    assert np.all(z.cpu().numpy() == 0.5)
    M, P = _setup(H, _diag(n + 1), 0, 1, 0)
    r = _dev(np.ones(n + 1))
    z = _dev(np.zeros(n + 1))
    with pytest.raises(H.HecError) as e:
        H.hec_precond_apply_noalloc(P, r, z)
    assert e.value.status == H.ERR_INVALID
    assert "static array" in str(e.value)
