"""CPU tests of the CUDA library's host side: the shared library loads and
exports every symbol of include/hecgpu.h, and the host setup (HEC layout,
RAS blocks, ILU(k), level schedule) matches the oracle bit for bit.  No call
here touches a GPU (handles are built with HEC_HOST_ONLY)."""
import os
import re

import numpy as np
import pytest

from paper_1606_00545_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_1606_00545_gb300 import build
    build.build()
    from paper_1606_00545_gb300 import hecgpu
    hecgpu.load_library()
    return hecgpu


def header_functions():
    src = open(os.path.join(ROOT, "include", "hecgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^(?:int|void|double|const char\s*\*)\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_header_symbol(H):
    import ctypes
    names = header_functions()
    assert "krylov_solve" in names and "hec_build" in names and len(names) >= 20
    lib = ctypes.CDLL(H.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(H.exported_symbols()) == names


def test_status_strings(H):
    lib = H.load_library()
    for s in (0, -1, -2, -3, -4, -5, -6, 1, 2):
        assert lib.hec_status_string(s)


def _reassemble(ex, n):
    K, ld = ex["K"], ex["ld"]
    rows, cols, vals = [], [], []
    tail_of = {r: t for t, r in enumerate(ex["tail_rows"])}
    for i in range(n):
        c = list(ex["ell_col"][:, i])
        v = list(ex["ell_val"][:, i])
        if i in tail_of:
            t = tail_of[i]
            c += list(ex["tail_col"][ex["tail_ptr"][t]:ex["tail_ptr"][t + 1]])
            v += list(ex["tail_val"][ex["tail_ptr"][t]:ex["tail_ptr"][t + 1]])
        for cc, vv in zip(c, v):
            rows.append(i)
            cols.append(cc)
            vals.append(vv)
    return np.array(rows), np.array(cols), np.array(vals)


@pytest.mark.parametrize("case", ["poisson2d", "irregular", "forced_k"])
def test_hec_layout_reassembles_csr(H, case):
    if case == "poisson2d":
        A, K = synth.poisson2d_5pt(20), 0
    elif case == "irregular":
        A, K = synth.stencil27_irregular(6, 1, 2, frac=0.05, extra_min=30, extra_max=60), 0
    else:
        A, K = synth.random_sparse(300, 0.03, seed=5), 3
    M = H.hec_build(A.row_ptr, A.col, A.val, ell_width=K, host_only=True)
    inf = M.info()
    ex = M.export()
    assert inf["ell_ld"] % 256 == 0 and inf["ell_ld"] >= A.n
    lens = A.row_lengths()
    if K == 0:
        # auto width: the largest K that at least a third of the rows reach
        Kx = max(k for k in range(1, lens.max() + 1) if 3 * np.sum(lens >= k) >= A.n)
        assert inf["ell_width"] == Kx
    else:
        assert inf["ell_width"] == K
    assert inf["tail_rows"] == int(np.sum(lens > inf["ell_width"]))
    r, c, v = _reassemble(ex, A.n)
    dense = np.zeros((A.n, A.n))
    np.add.at(dense, (r, c), v)
    assert np.array_equal(dense, A.to_dense())
    # every slab position beyond a row's length is padding (value 0, own row)
    Kw = inf["ell_width"]
    for i in range(A.n):
        for k in range(lens[i], Kw):
            assert ex["ell_col"][k, i] == i and ex["ell_val"][k, i] == 0.0


@pytest.mark.parametrize("k,nb,ov", [(0, 1, 0), (1, 4, 1), (2, 3, 2)])
def test_ras_ilu_levels_match_oracle(H, orc, k, nb, ov):
    for A in (synth.diffusion3d_7pt_lognormal(6, 2.0, 3),
              synth.random_sparse(200, 0.02, seed=7),
              synth.stencil27_irregular(5, 2, 3, frac=0.05, extra_min=3, extra_max=9)):
        Mh = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
        P = H.ilu_k_setup(Mh, k, nb, ov)
        H.level_schedule(P)
        R = orc.RAS(A, k, nb, ov)
        for b in range(nb):
            rows, lo, hi, F = R.block(b)
            grows, glo, ghi = P.block(b)
            assert (glo, ghi) == (lo, hi)
            assert np.array_equal(grows, rows)
            rp, ci, va, lev = P.factor(b)
            assert np.array_equal(rp, F.row_ptr) and np.array_equal(ci, F.col)
            assert np.array_equal(lev, F.lev)
            assert np.array_equal(va, F.val)  # same operations in the same order
            for which, upper in ((H.FACTOR_L, False), (H.FACTOR_U, True)):
                lv, nlev = orc.levels(F.n, F.row_ptr, F.col, upper)
                ptr_ref, rows_ref = orc.level_sets(lv, nlev)
                ptr, lrows = P.levels(b, which)
                assert np.array_equal(ptr, ptr_ref) and np.array_equal(lrows, rows_ref)
        inf = P.info()
        assert inf["scheduled"] == 1 and inf["apply_bytes"] > 0


def test_setup_errors(H):
    A = synth.CSR(np.array([0, 2, 4]), np.array([0, 1, 0, 1]), np.array([0.0, 1.0, 1.0, 0.0]))
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    with pytest.raises(H.HecError) as e:
        H.ilu_k_setup(M, 0, 1, 0)
    assert e.value.status == H.ERR_ZERO_PIVOT
    with pytest.raises(H.HecError) as e:
        H.hec_build(np.array([0, 2, 3]), np.array([1, 0, 1]), np.array([1.0, 2.0, 3.0]),
                    host_only=True)
    assert e.value.status == H.ERR_UNSORTED_CSR
    B = synth.CSR(np.array([0, 1, 2]), np.array([1, 0]), np.array([1.0, 1.0]))
    Mb = H.hec_build(B.row_ptr, B.col, B.val, host_only=True)
    with pytest.raises(H.HecError) as e:
        H.ilu_k_setup(Mb, 0, 1, 0)
    assert e.value.status == H.ERR_INVALID
    with pytest.raises(H.HecError):
        H.ilu_k_setup(Mb, 0, 3, 0)  # more blocks than rows
