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
    # row_ptr past nnz in the middle (rejected before any column is read),
    # decreasing row_ptr, a column out of range, a last entry that is not nnz
    for rp, ci in (([0, 10, 5], [0, 1, 0, 1, 1]), ([0, 3, 2, 5], [0, 1, 2, 0, 2]),
                   ([0, 2, 4], [0, 2, 0, 1]), ([0, 2, 3], [0, 1, 1, 0])):
        with pytest.raises(H.HecError) as e:
            H.hec_build(np.array(rp), np.array(ci), np.ones(len(ci)), host_only=True)
        assert e.value.status in (H.ERR_INVALID, H.ERR_UNSORTED_CSR)


def test_cpp_exception_does_not_cross_the_abi(H):
    """An ELL slab larger than a host vector can hold makes the C++ setup
    throw; the entry point returns an error code with a message instead (the
    process keeps running, the next call works)."""
    A = synth.poisson2d_5pt(4)
    with pytest.raises(H.HecError) as e:
        H.hec_build(A.row_ptr, A.col, A.val, ell_width=2 ** 31 - 1,
                    ell_ld_align=2 ** 31 - 32, host_only=True)
    assert e.value.status in (H.ERR_INVALID, H.ERR_OOM)
    assert "hec_build" in str(e.value)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    assert M.info()["n"] == A.n


# ------------------------------------------------------------------ factor layout
# The level-major chunk layout that the triangular-solve kernel streams,
# executed on the host from its bytes: a check of the packer (positions,
# dependencies, ring window, padding, row maps, algorithmic bytes) that needs
# no GPU.

def _seg_stride(w, nr):
    left = nr - 32 * w
    return 32 if left >= 32 else (left + 3) & ~3


def run_layout(lay, n, r):
    """z = M^{-1} r by the chunk program of every RAS block, as the kernel
    runs it: L chunks then U chunks, the rows of a chunk in parallel,
    dependencies from the shared-memory ring (zeroed at launch, slot =
    position mod ring size) or from the global scratch.  The scratch starts
    as NaN here (the kernel never clears it), so a read of a position the
    pass has not produced yet shows up; the kernel skips entries of value 0
    of a uniform-width layout there.  Returns z and how often each row of z
    was written."""
    pack, chunks, R = lay["pack"], lay["chunks"], lay["ring_slots"]
    FW, vb = lay["fixed_width"], lay["vbytes"]
    dt = np.float64 if vb == 8 else np.float32
    mask = R - 1
    z = np.full(n, np.nan, dt)
    writes = np.zeros(n, np.int64)
    rv = r.astype(dt)
    for c0, cm, c1, ring_l, ring_u, _, _ in lay["blocks"]:
        ring = np.zeros(R, dt)
        held = np.full(R, -1, np.int64)  # the position whose value a slot holds
        y = None
        for upass, lo, hi, use_ring in ((False, c0, cm, ring_l), (True, cm, c1, ring_u)):
            heads = [np.frombuffer(pack, np.int32, 24, int(chunks[c, 0]) * 16) for c in range(lo, hi)]
            npos = int(heads[-1][2] + heads[-1][0]) if heads else 0
            sol = np.full(npos, np.nan, dt)
            nxt = 0
            for c, h in zip(range(lo, hi), heads):
                base = int(chunks[c, 0]) * 16
                nr, nw, q, flags = (int(v) for v in h[:4])
                assert (flags & 1) == int(upass) and q == nxt and 0 < nr <= 256
                assert nw == (nr + 31) // 32 and int(chunks[c, 1]) % 16 == 0
                nxt = q + nr
                src = np.frombuffer(pack, np.int32, nr, base + int(h[20]))
                if upass:
                    assert np.all((src >= 0) & (src < len(y)))
                    acc = y[src].copy()
                else:
                    acc = rv[src].copy()
                for w in range(nw):
                    wd, so, ls = int(h[4 + w]), int(h[12 + w]), _seg_stride(w, nr)
                    m = min(32, nr - 32 * w)
                    if FW:  # the kernel computes these offsets at compile time
                        assert wd == FW and so == 96 + w * FW * 32 * (vb + 4)
                    if wd == 0:
                        continue
                    val = np.frombuffer(pack, dt, wd * ls, base + so).reshape(wd, ls)[:, :m]
                    dep = np.frombuffer(pack, np.int32, wd * ls,
                                        base + so + wd * ls * vb).reshape(wd, ls)[:, :m]
                    rows = slice(32 * w, 32 * w + m)
                    for k in range(wd):
                        d, live = dep[k], val[k] != 0
                        # rows of a chunk share a level: every dependency is earlier
                        assert np.all((d >= 0) & (d <= q)) and np.all(d[live] < q)
                        if use_ring:
                            assert np.all(held[d[live] & mask] == d[live])  # in the window
                            assert np.all(nxt - 1 - d[live] < R)  # not overwritten by the chunk
                            yk = ring[d & mask]
                        else:
                            yk = sol[d]
                            if FW:
                                yk = np.where(live, yk, dt(0))
                        acc[rows] -= val[k] * yk
                if upass:
                    acc *= np.frombuffer(pack, dt, nr, base + int(h[22]))
                pos = np.arange(q, nxt)
                sol[pos] = acc
                if use_ring:
                    ring[pos & mask] = acc
                    held[pos & mask] = pos
                if upass:
                    dst = np.frombuffer(pack, np.int32, nr, base + int(h[21]))
                    own = dst >= 0
                    z[dst[own]] = acc[own]
                    np.add.at(writes, dst[own], 1)
            assert nxt == npos and np.all(np.isfinite(sol))
            if not upass:
                y = sol
    return z, writes


def needed_rows(rp, ci, rows, lo, hi):
    """Rows of block V_b that can reach its owned part of z: the U solve needs
    the owned rows and, transitively, their U dependencies; the L solve needs
    those and, transitively, their L dependencies."""
    nv = len(rows)
    owned = (rows >= lo) & (rows < hi)
    need_u = owned.copy()
    for i in range(nv):
        if need_u[i]:
            cols = ci[rp[i]:rp[i + 1]]
            need_u[cols[cols > i]] = True
    need_l = need_u.copy()
    for i in range(nv - 1, -1, -1):
        if need_l[i]:
            cols = ci[rp[i]:rp[i + 1]]
            need_l[cols[cols < i]] = True
    return owned, need_l, need_u


LAYOUT_CASES = {
    "poisson2d_ilu0": (lambda: synth.poisson2d_5pt(24), 0, 1, 0),
    "diffusion3d_ilu1_ras4": (lambda: synth.diffusion3d_7pt_lognormal(10, 2.0, 2), 1, 4, 1),
    "random_ilu2_ras3_ov2": (lambda: synth.random_sparse(600, 0.01, seed=2), 2, 3, 2),
    "irregular27_ras2": (lambda: synth.stencil27_irregular(6, 2, 3, frac=0.05, extra_min=3,
                                                           extra_max=9), 0, 2, 1),
    "wide_window_global": (lambda: synth.random_sparse_rows(24000, 6, seed=6), 0, 1, 0),
}


@pytest.mark.parametrize("case", sorted(LAYOUT_CASES))
def test_factor_layout_runs_to_the_oracle_apply(H, orc, case):
    make, k, nb, ov = LAYOUT_CASES[case]
    A = make()
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P)
    ref = orc.RAS(A, k, nb, ov).apply(synth.rhs_uniform(A.n, 1))
    r = synth.rhs_uniform(A.n, 1)
    for fp32 in (False, True):
        lay = H.Precond.layout(P, fp32=fp32)
        vb = lay["vbytes"]
        z, writes = run_layout(lay, A.n, r)
        assert np.all(writes == 1)  # every row of z written once, by its owner
        err = np.max(np.abs(z - ref)) / np.abs(ref).max()
        assert err <= (1e-5 if fp32 else 1e-13), (case, fp32, err)
        # algorithmic bytes of one apply, counted from the factors
        alg = 0
        for b in range(nb):
            rows, lo, hi = P.block(b)
            rp, ci, _, _ = P.factor(b)
            owned, need_l, need_u = needed_rows(rp, ci, rows, lo, hi)
            c0, cm, c1 = (int(v) for v in lay["blocks"][b, :3])
            npos = []
            for a, e in ((c0, cm), (cm, c1)):
                h = np.frombuffer(lay["pack"], np.int32, 4, int(lay["chunks"][e - 1, 0]) * 16)
                npos.append(int(h[2] + h[0]))
            assert npos == [int(need_l.sum()), int(need_u.sum())]
            for i in range(len(rows)):
                cols = ci[rp[i]:rp[i + 1]]
                if need_l[i]:
                    alg += (4 + vb) * int(np.sum(cols < i)) + 2 * vb + 4
                if need_u[i]:
                    alg += (4 + vb) * int(np.sum(cols > i)) + 2 * vb + 8 + (vb if owned[i] else 0)
        inf = P.info()
        assert alg == inf["apply_bytes_f32" if fp32 else "apply_bytes"]
        if fp32:
            assert lay["fixed_width"] in (0, 4, 6, 8)
        else:
            assert lay["fixed_width"] == 0
    if case == "wide_window_global":
        assert P.info()["global_passes"] > 0
        assert H.Precond.layout(P, fp32=True)["fixed_width"] > 0


def test_factor_layout_errors(H):
    A = synth.poisson2d_5pt(8)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 0, 1, 0)
    with pytest.raises(H.HecError):
        P.layout()  # before level_schedule
    H.level_schedule(P)
    assert P.layout()["chunks"].shape[0] > 0


def test_workspace_bytes_query(H):
    """hec_workspace_bytes on host-only handles: each extra GMRES restart step
    costs one padded basis vector (FP64, or FP32 in the mixed form), BiCGSTAB
    keeps four vectors more than CG, and the mixed count drops by exactly
    the FP32 layout's device bytes once that layout exists."""
    A = synth.diffusion3d_7pt_lognormal(9, 2.0, 1)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 1, 3, 1)
    H.level_schedule(P)
    nv = (A.n + 31) // 32 * 32
    q = H.hec_workspace_bytes
    assert q(M, P, 50, H.GMRES) - q(M, P, 30, H.GMRES) == 20 * nv * 8
    assert q(M, P, 0, H.BICGSTAB) - q(M, P, 0, H.CG) == 4 * nv * 8
    assert q(M, None, 0, H.CG) == q(M, P, 0, H.CG)
    m30 = q(M, P, 30, H.GMRES, H.MIXED_FP32)
    assert q(M, P, 50, H.GMRES, H.MIXED_FP32) - m30 == 20 * nv * 4
    lay = P.layout(fp32=True)  # packs the FP32 layout (host-only: nothing uploaded)
    heads = [np.frombuffer(lay["pack"], np.int32, 4, int(c) * 16) for c in lay["chunks"][:, 0]]
    ysz = zsz = 0
    for c0, cm, c1, _, ring_u, _, _ in lay["blocks"]:
        ysz += int(heads[cm - 1][2] + heads[cm - 1][0])
        if not ring_u:
            zsz += int(heads[c1 - 1][2] + heads[c1 - 1][0])
    layout_bytes = (len(lay["pack"]) + 8 * len(lay["chunks"]) + 40 * len(lay["blocks"]) +
                    4 * max(ysz, 1) + 4 * max(zsz, 1))
    assert m30 - q(M, P, 30, H.GMRES, H.MIXED_FP32) == layout_bytes
    for bad in (dict(restart=0, method=H.GMRES), dict(restart=500, method=H.GMRES),
                dict(restart=0, method=H.BICGSTAB, flags=H.MIXED_FP32), dict(restart=30, method=7)):
        with pytest.raises(H.HecError):
            q(M, P, **bad)


def test_spmv_rejects_misaligned_output(H):
    """The SpMV stores two adjacent rows per thread with one vector store, so
    y_out must be 16-byte (FP64) or 8-byte (FP32) aligned; a misaligned
    output is rejected before any device work (the addresses below are
    never dereferenced)."""
    import ctypes
    A = synth.poisson2d_5pt(4)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    lib = H.load_library()
    x = ctypes.c_void_p(0x10000)
    for y, f32 in ((0x20008, False), (0x20004, True)):
        if f32:
            rc = lib.hec_spmv_f32(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(y), None)
        else:
            rc = lib.hec_spmv(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(y), None, None, None)
        assert rc == H.ERR_INVALID
        assert b"aligned" in lib.hec_last_error()
    # aligned: rejected for the host-only handle instead, after the alignment check
    rc = lib.hec_spmv(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(0x20010), None, None, None)
    assert rc == H.ERR_INVALID and b"host-only" in lib.hec_last_error()
