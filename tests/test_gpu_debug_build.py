"""The library compiled with HEC_DEBUG: the triangular-solve kernel checks every
chunk header against the position its program has reached, every gathered
index against n and every dependency slot against its ring, and records the
first violation (hec_debug_record); the resident-vector kernel checks every
dependency and row slot against the block's vector and every gathered index
against n.  The small preconditioner parity cases, streamed with 1, 2 and 8
CTAs per RAS block and resident where the blocks fit, in FP64 and FP32, must
run with no violation and still match the oracle within the entry-wise
rounding bound.

A process loads one copy of the library, so the debug build runs in a child
process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C, os, sys
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
import numpy as np
import torch
from paper_1606_00545_gb300 import build, synth
build.build(debug=True)
from paper_1606_00545_gb300 import hecgpu as H
lib = H.load_library(H.DEBUG_LIB_PATH)
import oracle as orc
orc.build()
from ras_bound import check_apply
torch.cuda.set_device(0)
rec = (C.c_int32 * 8)()
assert lib.hec_debug_record(rec, 1) == H.OK  # a debug build
cases = {
    "poisson64_ilu0": (synth.poisson2d_5pt(64), 0, 1, 0),
    "diffusion3d_16_ilu1_ras8": (synth.diffusion3d_7pt_lognormal(16, 2.0, 2), 1, 8, 1),
    "random_ilu2_ras3_ov2": (synth.random_sparse(3000, 0.002, seed=2), 2, 3, 2),
    "wide_window_global": (synth.random_sparse_rows(24000, 6, seed=6), 0, 1, 0),
    "many_blocks": (synth.diffusion2d_5pt_lognormal(40, 2.0, 5), 1, 200, 1),
}
for name, (A, k, nb, ov) in cases.items():
    M = H.hec_build(A.row_ptr, A.col, A.val)
    R = orc.RAS(A, k, nb, ov)
    r = synth.rhs_uniform(A.n, 3)
    modes = [(H.TRSV_STREAMED, 1), (H.TRSV_STREAMED, 2), (H.TRSV_STREAMED, 8)]
    if name in ("poisson64_ilu0", "diffusion3d_16_ilu1_ras8", "many_blocks"):
        modes.append((H.TRSV_RESIDENT, 0))
    for kernel, parts in modes:
        P = H.ilu_k_setup(M, k, nb, ov)
        H.level_schedule(P, parts=parts, kernel=kernel)
        for fp32 in (False, True):
            dt = torch.float32 if fp32 else torch.float64
            ap = H.hec_precond_apply_f32 if fp32 else H.hec_precond_apply
            z = torch.full((A.n,), float("nan"), dtype=dt, device="cuda:0")
            ap(P, torch.tensor(r, dtype=dt, device="cuda:0"), z)
            st = H._lib.hec_precond_status(P.handle, None)
            assert lib.hec_debug_record(rec, 1) == H.OK
            assert list(rec) == [0] * 8, (name, parts, fp32, list(rec))
            assert st == H.OK, (name, parts, fp32, st)
            check_apply(orc, R, r, z.double().cpu().numpy(), fp32=fp32,
                        what="debug build %s parts=%d fp32=%d" % (name, parts, fp32))
print("DEBUG_BUILD_OK")
'''


def test_debug_build_runs_the_parity_cases_without_violations():
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0 and "DEBUG_BUILD_OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
