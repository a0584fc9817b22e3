"""CPU tests of the CUDA library's host side: the shared library loads and
exports every symbol of include/hecgpu.h, and the host setup (HEC layout,
RAS blocks, ILU(k), level schedule) matches the oracle bit for bit.  No call
here touches a GPU (handles are built with HEC_HOST_ONLY)."""
import os
import re

import numpy as np
import pytest

from paper_1606_00545_gb300 import synth
from ras_bound import check_apply

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


def _chunk(pack, chunks, c):
    base = int(chunks[c, 0]) * 16
    return base, np.frombuffer(pack, np.int32, 28, base)


def parse_chunk(pack, chunks, c, vb):
    """One chunk of either format: header fields, per-warp (rows, val, dep)
    and per-row src, dst, dinv, exp (None where the format has none)."""
    dt = np.float64 if vb == 8 else np.float32
    base, h = _chunk(pack, chunks, c)
    nr, nw, q, flags = (int(v) for v in h[:4])
    upass, fixed = bool(flags & 1), bool(flags & 8)
    out = dict(nr=nr, nw=nw, q=q, flags=flags, upass=upass, fixed=fixed, warps=[])
    assert 0 < nr <= 256 and nw == (nr + 31) // 32 and int(chunks[c, 1]) % 16 == 0
    if fixed:
        FW, exps = int(h[6]), bool(flags & 16)
        out.update(need_prev=int(h[4]), need_next=int(h[5]), FW=FW, xend=int(h[7]))
        VW = 16 // vb
        NV, ND = (FW + VW - 1) // VW, (FW + 3) // 4
        blk = (NV + ND) * 512 + 128 + (32 * vb + 128 if upass else 0) + (128 if exps else 0)
        assert int(chunks[c, 1]) == 32 + nw * blk
        src, dst, dinv, exp = [], [], [], []
        for w in range(nw):
            o = base + 32 + w * blk
            m = min(32, nr - 32 * w)
            # [NV][32 lanes][VW] -> [entry][lane]
            v = np.frombuffer(pack, dt, NV * 32 * VW, o).reshape(NV, 32, VW)
            val = v.transpose(0, 2, 1).reshape(NV * VW, 32)[:FW]
            d = np.frombuffer(pack, np.int32, ND * 128, o + NV * 512).reshape(ND, 32, 4)
            dep = d.transpose(0, 2, 1).reshape(ND * 4, 32)[:FW]
            o2 = o + (NV + ND) * 512
            if upass:
                dinv.append(np.frombuffer(pack, dt, 32, o2)[:m])
                o2 += 32 * vb
            src.append(np.frombuffer(pack, np.int32, 32, o2)[:m])
            o2 += 128
            if upass:
                dst.append(np.frombuffer(pack, np.int32, 32, o2)[:m])
                o2 += 128
            if exps:
                exp.append(np.frombuffer(pack, np.int32, 32, o2)[:m])
            out["warps"].append((slice(32 * w, 32 * w + m), val[:, :m], dep[:, :m]))
        out["src"] = np.concatenate(src)
        out["dst"] = np.concatenate(dst) if upass else None
        out["dinv"] = np.concatenate(dinv) if upass else None
        out["exp"] = np.concatenate(exp) if exps else None
        return out
    out.update(need_prev=int(h[24]), need_next=int(h[25]), FW=0, xend=int(h[26]))
    for w in range(nw):
        wd, so, ls = int(h[4 + w]), int(h[12 + w]), _seg_stride(w, nr)
        m = min(32, nr - 32 * w)
        val = np.frombuffer(pack, dt, wd * ls, base + so).reshape(wd, ls)[:, :m]
        dep = np.frombuffer(pack, np.int32, wd * ls, base + so + wd * ls * vb).reshape(wd, ls)[:, :m]
        out["warps"].append((slice(32 * w, 32 * w + m), val, dep))
    out["src"] = np.frombuffer(pack, np.int32, nr, base + int(h[20]))
    out["dst"] = np.frombuffer(pack, np.int32, nr, base + int(h[21])) if upass else None
    out["dinv"] = np.frombuffer(pack, dt, nr, base + int(h[22])) if upass else None
    out["exp"] = np.frombuffer(pack, np.int32, nr, base + int(h[23])) if flags & 2 else None
    return out


def parse_resident_chunk(pack, chunks, c, vb):
    """One chunk of the resident kernel's format: per warp (rows, val, dep)
    with dependency slots, and per row its own slot and (U) dinv."""
    dt = np.float64 if vb == 8 else np.float32
    base, h = _chunk(pack, chunks, c)
    nr, nw, q, flags = (int(v) for v in h[:4])
    upass = bool(flags & 1)
    assert flags & 8 and flags & 32
    assert 0 < nr <= 256 and nw == (nr + 31) // 32 and int(chunks[c, 1]) % 16 == 0
    FW = int(h[6])
    VW = 16 // vb
    NV, NI = (FW + VW - 1) // VW, (FW + 1 + 7) // 8
    blk = (NV + NI) * 512 + 32 * vb  # every chunk has a block per solving warp of the kernel
    assert (int(chunks[c, 1]) - 32) % blk == 0 and (int(chunks[c, 1]) - 32) // blk >= nw
    pad_slots = []  # warps past the rows: values 0, every slot padding
    for w in range(nw, (int(chunks[c, 1]) - 32) // blk):
        o = base + 32 + w * blk
        assert not np.any(np.frombuffer(pack, dt, NV * 32 * VW, o))
        pad_slots.append(np.frombuffer(pack, np.uint16, NI * 256, o + NV * 512))
    out = dict(nr=nr, nw=nw, q=q, upass=upass, FW=FW, flags=flags, warps=[], pad_slots=pad_slots)
    own, dinv = [], []
    for w in range(nw):
        o = base + 32 + w * blk
        m = min(32, nr - 32 * w)
        v = np.frombuffer(pack, dt, NV * 32 * VW, o).reshape(NV, 32, VW)
        val = v.transpose(0, 2, 1).reshape(NV * VW, 32)[:FW]
        ix = np.frombuffer(pack, np.uint16, NI * 256, o + NV * 512).reshape(NI, 32, 8)
        ix = ix.transpose(0, 2, 1).reshape(NI * 8, 32).astype(np.int64)
        dep = ix[:FW]
        own.append(ix[FW])
        if upass:
            dinv.append(np.frombuffer(pack, dt, 32, o + (NV + NI) * 512))
        out["warps"].append((w, val, dep, m))
    out["own"] = np.concatenate(own)
    out["dinv"] = np.concatenate(dinv) if upass else None
    return out


def run_resident(lay, P, n, r, nb):
    """z = M^{-1} r by the resident kernel's programs, as it runs them: block
    b's vector x starts as r on V_b with slot nv = 0; every chunk's rows
    update their own slot in place from the slots of their dependencies
    (which must hold values of this pass already), the U pass multiplies by
    dinv; z on the owned rows is x at the end.  Padding entries must have
    value 0 and slot nv, padding rows own slot nv.  Returns z and the writes
    per row."""
    pack, chunks, vb = lay["pack"], lay["chunks"], lay["vbytes"]
    dt = np.float64 if vb == 8 else np.float32
    z = np.full(n, np.nan, dt)
    writes = np.zeros(n, np.int64)
    rv = r.astype(dt)
    progs = lay["programs"]
    assert lay["parts"] == 1 and len(progs) == nb
    voff = 0
    for b in range(nb):
        rows, lo, hi = P.block(b)
        nv = len(rows)
        c0, cm, c1, _, _, yoff, _, links = (int(v) for v in progs[b])
        assert yoff == voff and links == 0
        voff += nv
        x = np.concatenate([rv[rows], [dt(0)]])
        solved = [np.zeros(nv + 1, bool), np.zeros(nv + 1, bool)]
        pos = [0, 0]
        gbytes, gchunks = 0, 0  # the group of consecutive chunks being streamed
        gstart = int(chunks[c0, 0]) * 16
        for c in range(c0, c1):
            C = parse_resident_chunk(pack, chunks, c, vb)
            gbytes += int(chunks[c, 1])
            gchunks += 1
            h = _chunk(pack, chunks, c)[1]
            if C["flags"] & 64 or c == c1 - 1:  # one bulk copy of at most 16 KB
                assert C["flags"] & 64 and (gbytes <= 16384 or gchunks == 1)
                gbytes, gchunks = 0, 0
                gstart = int(chunks[c, 0]) * 16 + int(chunks[c, 1])
            if c + 1 < c1:  # the next chunk's place in its group's stage and its warps
                hn = _chunk(pack, chunks, c + 1)[1]
                assert int(h[4]) == int(chunks[c + 1, 0]) * 16 - gstart and int(h[5]) == int(hn[1])
            upass = C["upass"]
            assert upass == (c >= cm) and C["q"] == pos[int(upass)]
            pos[int(upass)] += C["nr"]
            own = C["own"]
            assert np.all(own[C["nr"]:] == nv) and np.all(own[:C["nr"]] < nv)
            assert all(np.all(p == nv) for p in C["pad_slots"])
            acc = x[own].copy()
            done = solved[int(upass)]
            for w, val, dep, m in C["warps"]:
                assert np.all(val[:, m:] == 0) and np.all(dep[:, m:] == nv)
                for k in range(val.shape[0]):
                    d, live = dep[k], val[k] != 0
                    assert np.all((d >= 0) & (d <= nv))
                    # a dependency was solved by an earlier chunk of the pass
                    assert np.all(done[d[:m][live[:m]]])
                    acc[32 * w:32 * w + 32] -= val[k] * x[d]
            if upass:
                acc *= C["dinv"]
            mine = own[:C["nr"]]
            assert not np.any(done[mine])  # every row once per pass
            if upass:  # a U row starts from its y: the L pass solved it
                assert np.all(solved[0][mine])
            x[mine] = acc[:C["nr"]]
            done[mine] = True
        o0 = int(np.searchsorted(rows, lo))
        o1 = int(np.searchsorted(rows, hi))
        assert solved[1][o0:o1].all() and solved[0][o0:o1].all()
        z[rows[o0:o1]] = x[o0:o1]
        writes[rows[o0:o1]] += 1
    return z, writes


def run_layout(lay, n, r, eager=True, who=None, sols=None):
    """z = M^{-1} r by the chunk programs of every RAS block, as the kernel
    runs them.  A block has P programs (its parts, one CTA each); each runs
    its L chunks then its U chunks, the rows of a chunk in parallel.
    Dependencies come from the CTA's shared-memory ring (own slots below R,
    zeroed at launch; slots from R on receive the values the neighbouring
    part exports, NaN until written) or, in a pass whose window does not fit,
    from the global scratch by position.  A chunk runs only once the
    neighbours have completed the chunk counts in its header.  eager=True
    runs every part as far as it can before the next one gets a turn (a
    leading part gets as far ahead as its thresholds allow); eager=False
    runs one chunk per part per turn.  The scratch starts as NaN (the kernel
    never clears it), so a read of a position the pass has not produced yet
    shows up; the kernel skips entries of value 0 of a uniform-width layout
    there.  Returns z and how often each row of z was written (who, if
    given, receives the program index that wrote each row)."""
    pack, chunks = lay["pack"], lay["chunks"]
    R, RI, P = lay["ring_slots"], lay["import_slots"], lay["parts"]
    FW, vb = lay["fixed_width"], lay["vbytes"]
    dt = np.float64 if vb == 8 else np.float32
    z = np.full(n, np.nan, dt)
    writes = np.zeros(n, np.int64)
    rv = r.astype(dt)
    progs = lay["programs"]
    assert len(progs) % P == 0 and R >= 32 and (R & (R - 1)) == 0
    assert RI == 0 or (RI & (RI - 1)) == 0
    for b0 in range(0, len(progs), P):
        parts = []
        for p in range(P):
            c0, cm, c1, ring_l, ring_u, _, _, links = (int(v) for v in progs[b0 + p])
            assert c0 <= cm <= c1
            npos = []
            for lo, hi in ((c0, cm), (cm, c1)):
                h = _chunk(pack, chunks, hi - 1)[1] if hi > lo else None
                npos.append(int(h[2] + h[0]) if h is not None else 0)
            parts.append(dict(c0=c0, cm=cm, c1=c1, ring=(ring_l, ring_u), links=links,
                              buf=np.concatenate([np.zeros(R, dt), np.full(RI, np.nan, dt)]),
                              sol=[np.full(npos[0], np.nan, dt), np.full(npos[1], np.nan, dt)],
                              done=0, nxt=0))
        for p in range(P):  # links are symmetric
            if parts[p]["links"] & 2:
                assert p + 1 < P and parts[p + 1]["links"] & 1
        for p in range(P):
            if parts[p]["links"] & 1:
                assert p > 0 and parts[p - 1]["links"] & 2

        def run_chunk(p):
            st = parts[p]
            c = st["c0"] + st["done"]
            upass = c >= st["cm"]
            if c == st["cm"]:
                st["nxt"] = 0
            use_ring = st["ring"][int(upass)]
            sol = st["sol"][int(upass)]
            C = parse_chunk(pack, chunks, c, vb)
            nr, q, flags = C["nr"], C["q"], C["flags"]
            assert C["upass"] == upass and q == st["nxt"]
            assert C["fixed"] == (FW > 0) and C["FW"] == FW
            nxt = st["nxt"] = q + nr
            src = C["src"]
            if upass:
                y = st["sol"][0]
                assert np.all((src >= 0) & (src < len(y)))
                acc = y[src].copy()
            else:
                acc = rv[src].copy()
            buf = st["buf"]
            for rows, val, dep in C["warps"]:
                for k in range(val.shape[0]):
                    d, live = dep[k], val[k] != 0
                    if use_ring:
                        assert np.all((d >= 0) & (d < R + RI))
                        yk = buf[d]
                        assert np.all(np.isfinite(yk[live]))  # imports arrive first
                    else:
                        # rows of a chunk share a level: every dependency is earlier
                        assert np.all((d >= 0) & (d <= q)) and np.all(d[live] < q)
                        yk = sol[d]
                        if FW:
                            yk = np.where(live, yk, dt(0))
                    acc[rows] -= val[k] * yk
            if upass:
                acc *= C["dinv"]
            pos = np.arange(q, nxt)
            sol[pos] = acc
            if use_ring:
                buf[pos & (R - 1)] = acc
            exp = C["exp"]
            if exp is not None and np.any(exp >= 0):  # exports into the neighbour's ring
                assert RI > 0 and (flags & 2)
                tgt = p - 1 if upass else p + 1
                assert st["links"] & (1 if upass else 2)
                e = exp >= 0
                # export positions run on through the pass, chunk after chunk
                xs = st.setdefault("xend", {})
                lo = xs.get(upass, 0)
                assert np.all((exp[e] >= lo) & (exp[e] < C["xend"]))
                xs[upass] = C["xend"]
                parts[tgt]["buf"][R + (exp[e] & (RI - 1))] = acc[e]
            else:
                assert not (flags & 2)
                assert C["xend"] == st.setdefault("xend", {}).get(upass, 0)
            if upass:
                dst = C["dst"]
                own = dst >= 0
                z[dst[own]] = acc[own]
                np.add.at(writes, dst[own], 1)
                if who is not None:  # (block, part) that wrote each row of z
                    who[dst[own]] = (b0 // P) * P + p
            st["done"] += 1

        def ready(p):
            st = parts[p]
            if st["c0"] + st["done"] >= st["c1"]:
                return False
            C = parse_chunk(pack, chunks, st["c0"] + st["done"], vb)
            prev = parts[p - 1]["done"] if p > 0 else 0
            nxt = parts[p + 1]["done"] if p + 1 < P else 0
            assert (C["need_prev"] == 0 or st["links"] & 1)
            assert (C["need_next"] == 0 or st["links"] & 2)
            return C["need_prev"] <= prev and C["need_next"] <= nxt

        moved = True
        while moved:
            moved = False
            for p in range(P):
                while ready(p):
                    run_chunk(p)
                    moved = True
                    if not eager:
                        break
        for p, st in enumerate(parts):
            assert st["c0"] + st["done"] == st["c1"]  # no part is left waiting
            assert all(np.all(np.isfinite(v)) for v in st["sol"])
            if sols is not None:  # every program's L and U results by position
                sols[b0 + p] = st["sol"]
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
    "diffusion3d_ilu1_slab": (lambda: synth.diffusion3d_7pt_lognormal(12, 2.0, 4), 1, 2, 1),
}


@pytest.mark.parametrize("parts", [1, 2, 4, 8])
@pytest.mark.parametrize("case", sorted(LAYOUT_CASES))
def test_factor_layout_runs_to_the_oracle_apply(H, orc, case, parts):
    """The streamed kernel's layout (ring of recent values, blocks split over
    `parts` CTAs where the dependencies allow) run on the host."""
    make, k, nb, ov = LAYOUT_CASES[case]
    A = make()
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P, parts=parts, kernel=H.TRSV_STREAMED)
    assert P.info()["trsv_resident"] == 0
    R = orc.RAS(A, k, nb, ov)
    r = synth.rhs_uniform(A.n, 1)
    inf = P.info()
    assert inf["trsv_parts"] in (1, 2, 4, 8) and inf["trsv_parts"] <= parts
    for fp32 in (False, True):
        lay = H.Precond.layout(P, fp32=fp32)
        vb = lay["vbytes"]
        Pn = lay["parts"]
        assert lay["programs"].shape == (nb * Pn, 8)
        z, writes = run_layout(lay, A.n, r)
        assert np.all(writes == 1)  # every row of z written once, by its owner
        # the host run rounds like the kernel (FP32 layout: FP32 values and
        # arithmetic), so the entry-wise rounding bound holds for it too
        worst = check_apply(orc, R, r, z, fp32=fp32, what="%s fp32=%d" % (case, fp32))
        if fp32:
            assert worst > 1e-3  # the FP32 bound is not vacuous here
        # the same result when the parts take turns chunk by chunk
        z2, _ = run_layout(lay, A.n, r, eager=False)
        assert np.array_equal(z, z2)
        # algorithmic bytes of one apply, counted from the factors
        alg = 0
        for b in range(nb):
            rows, lo, hi = P.block(b)
            rp, ci, _, _ = P.factor(b)
            owned, need_l, need_u = needed_rows(rp, ci, rows, lo, hi)
            npos = [0, 0]
            for prog in lay["programs"][b * Pn:(b + 1) * Pn]:
                c0, cm, c1 = (int(v) for v in prog[:3])
                for j, (a, e) in enumerate(((c0, cm), (cm, c1))):
                    if e > a:
                        h = _chunk(lay["pack"], lay["chunks"], e - 1)[1]
                        npos[j] += int(h[2] + h[0])
            assert npos == [int(need_l.sum()), int(need_u.sum())]
            for i in range(len(rows)):
                cols = ci[rp[i]:rp[i + 1]]
                if need_l[i]:
                    alg += (4 + vb) * int(np.sum(cols < i)) + 2 * vb + 4
                if need_u[i]:
                    alg += (4 + vb) * int(np.sum(cols > i)) + 2 * vb + 8 + (vb if owned[i] else 0)
        inf = P.info()
        assert alg == inf["apply_bytes_f32" if fp32 else "apply_bytes"]
        assert lay["fixed_width"] in (0, 4, 6, 8)
        assert (lay["import_slots"] > 0) == (inf["split_blocks"] > 0)
    if case == "wide_window_global":
        assert P.info()["global_passes"] > 0
        assert H.Precond.layout(P, fp32=True)["fixed_width"] > 0
    if case in ("poisson2d_ilu0", "diffusion3d_ilu1_slab") and parts > 1:
        # dependencies reach only the next part: every block is split
        assert P.info()["split_blocks"] == nb


RESIDENT_CASES = ["poisson2d_ilu0", "diffusion3d_ilu1_ras4", "diffusion3d_ilu1_slab",
                  "random_ilu0_ras3_ov2", "poisson2d_64_ilu0"]


@pytest.mark.parametrize("case", RESIDENT_CASES)
def test_resident_layout_runs_to_the_oracle_apply(H, orc, case):
    """The resident kernel's layout (one CTA per block, the block's vector in
    shared memory, updated in place) run on the host, FP64 and FP32: every
    owned row written once, the entry-wise rounding bound against the
    oracle's RAS apply, the rows of every pass solved once in level order,
    the algorithmic bytes counted as for the streamed layout."""
    if case == "poisson2d_64_ilu0":  # the 64 x 64 single-block ILU(0) solve
        A, k, nb, ov = synth.poisson2d_5pt(64), 0, 1, 0
    elif case == "random_ilu0_ras3_ov2":  # irregular rows, 2 overlap layers
        A, k, nb, ov = synth.random_sparse(600, 0.004, seed=5), 0, 3, 2
    else:
        make, k, nb, ov = LAYOUT_CASES[case]
        A = make()
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P, kernel=H.TRSV_RESIDENT)
    inf = P.info()
    assert inf["trsv_resident"] == 1 and inf["trsv_parts"] == 1
    R = orc.RAS(A, k, nb, ov)
    r = synth.rhs_uniform(A.n, 1)
    for fp32 in (False, True):
        lay = H.Precond.layout(P, fp32=fp32)
        assert lay["fixed_width"] in (2, 3, 4, 6, 8)
        z, writes = run_resident(lay, P, A.n, r, nb)
        assert np.all(writes == 1)
        check_apply(orc, R, r, z, fp32=fp32, what="%s resident fp32=%d" % (case, fp32))
    # the automatic choice: resident where no level holds more than 128 rows
    # (the blocks fit and are not split); both count the same algorithmic bytes
    widest = max(int(np.max(np.diff(P.levels(b, which)[0])))
                 for b in range(nb) for which in (H.FACTOR_L, H.FACTOR_U))
    P2 = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P2)
    assert P2.info()["trsv_resident"] == (1 if widest <= 128 else 0)
    assert P2.info()["apply_bytes"] == inf["apply_bytes"]


def _diagonal(n):
    return synth.CSR(np.arange(n + 1), np.arange(n), 1.5 + np.arange(n) % 3)


def _lower_bidiagonal(n):
    rows = np.concatenate([np.arange(n), np.arange(1, n)])
    cols = np.concatenate([np.arange(n), np.arange(n - 1)])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0)])
    o = np.lexsort((cols, rows))
    return synth.CSR(np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]),
                     cols[o], vals[o])


DEGENERATE_CASES = {
    "n1": (lambda: _diagonal(1), 0, 1, 0),                    # one row, one level
    "diagonal_3_blocks": (lambda: _diagonal(300), 0, 3, 1),   # no dependencies at all
    "bidiagonal_chain": (lambda: _lower_bidiagonal(300), 0, 1, 0),  # L: 300 levels of 1 row
    "one_row_per_block": (lambda: synth.tridiagonal(16, 3), 0, 16, 1),
    "overlap_covers_all": (lambda: synth.tridiagonal(40, 4), 1, 4, 50),
}


@pytest.mark.parametrize("kernel", ["streamed", "resident"])
@pytest.mark.parametrize("case", sorted(DEGENERATE_CASES))
def test_degenerate_layouts_run_to_the_oracle_apply(H, orc, case, kernel):
    """The edge cases of the method: a single row, rows with no dependency,
    a chain with one row per level, blocks of one owned row, and an overlap
    that covers the whole matrix; both kernels' layouts run on the host,
    FP64 and FP32, every owned row written once and within the rounding bound
    of the oracle's RAS apply."""
    make, k, nb, ov = DEGENERATE_CASES[case]
    A = make()
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P, kernel=H.TRSV_RESIDENT if kernel == "resident" else H.TRSV_STREAMED)
    assert P.info()["trsv_resident"] == (1 if kernel == "resident" else 0)
    R = orc.RAS(A, k, nb, ov)
    r = synth.rhs_uniform(A.n, 2)
    for fp32 in (False, True):
        lay = H.Precond.layout(P, fp32=fp32)
        if kernel == "resident":
            z, writes = run_resident(lay, P, A.n, r, nb)
        else:
            z, writes = run_layout(lay, A.n, r)
            z2, _ = run_layout(lay, A.n, r, eager=False)
            assert np.array_equal(z, z2)
        assert np.all(writes == 1)
        check_apply(orc, R, r, z, fp32=fp32, what="%s %s fp32=%d" % (case, kernel, fp32))
    # the automatic choice: resident unless a level holds more than 128 rows
    # (the chain's U is diagonal: one level of 300 rows)
    widest = max(int(np.max(np.diff(P.levels(b, which)[0])))
                 for b in range(nb) for which in (H.FACTOR_L, H.FACTOR_U))
    P2 = H.ilu_k_setup(M, k, nb, ov)
    H.level_schedule(P2)
    assert P2.info()["trsv_resident"] == (1 if widest <= 128 else 0)
    assert (widest > 128) == (case == "bidiagonal_chain")


def test_resident_kernel_refused_where_it_does_not_fit(H):
    """Rows longer than 8 entries (a random matrix with ILU(2) fill) cannot
    take the resident kernel: asking for it fails at level_schedule, the
    automatic choice streams."""
    A = synth.random_sparse(600, 0.01, seed=2)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 2, 3, 2)
    with pytest.raises(H.HecError):
        H.level_schedule(P, kernel=H.TRSV_RESIDENT)
    P = H.ilu_k_setup(M, 2, 3, 2)
    H.level_schedule(P)
    assert P.info()["trsv_resident"] == 0
    lib = H.load_library()
    assert lib.hec_precond_set_trsv_kernel(P.handle, H.TRSV_RESIDENT) != H.OK  # too late
    P = H.ilu_k_setup(M, 2, 3, 2)
    assert lib.hec_precond_set_trsv_kernel(P.handle, 7) != H.OK


def test_trsv_parts_choice(H):
    """Automatic parts: split while the widest block's levels hold more than
    128 rows per CTA and the CTAs fit on the device (host-only handles count
    152 SMs).  A random matrix has dependencies that skip parts of a 4-way
    split; any 2-way split is admissible, so it falls back to 2 parts."""
    A = synth.poisson2d_5pt(24)  # 576 rows, 47 levels: 12 rows per level
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    # levels of at most 24 rows on an unsplit block: the resident kernel
    assert P.info()["trsv_parts"] == 1 and P.info()["trsv_resident"] == 1
    A = synth.poisson2d_5pt(400)  # 160,000 rows, 799 levels: 200 rows per level
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    # split over 2 CTAs (and too large for shared memory anyway): streamed
    assert P.info()["trsv_parts"] == 2 and P.info()["split_blocks"] == 1
    assert P.info()["trsv_resident"] == 0
    A = synth.poisson2d_5pt(160)  # 25,600 rows, levels up to 160 rows: streamed, 1 CTA
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 0, 1, 0)
    H.level_schedule(P)
    assert P.info()["trsv_parts"] == 1 and P.info()["trsv_resident"] == 0
    A = synth.random_sparse(600, 0.01, seed=2)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    P = H.ilu_k_setup(M, 2, 1, 0)
    H.level_schedule(P, parts=4)
    assert P.info()["trsv_parts"] == 2 and P.info()["split_blocks"] == 1
    P = H.ilu_k_setup(M, 0, 1, 0)
    with pytest.raises(H.HecError):
        H.level_schedule(P, parts=3)
    H.level_schedule(P)
    assert H.load_library().hec_precond_set_trsv_parts(P.handle, 2) != H.OK  # too late


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
    resident = P.info()["trsv_resident"] == 1  # (the FP32 layout follows the FP64 choice)
    for c0, cm, c1, _, ring_u, _, _, _ in lay["programs"]:
        if resident:  # no scratch; the kernel's row list holds every block's V_b
            continue
        if cm > c0:
            ysz += int(heads[cm - 1][2] + heads[cm - 1][0])
        if not ring_u and c1 > cm:
            zsz += int(heads[c1 - 1][2] + heads[c1 - 1][0])
    rows = sum(len(P.block(b)[0]) for b in range(3)) if resident else 0
    groups = 0
    if resident:  # chunk groups: a group ends at every chunk with flag bit 6
        groups = sum(1 for h in heads if h[3] & 64)
    # per program 56 bytes (chunk range, ring flags, scratch offsets, links,
    # the resident kernel's row count, owned range and group count)
    layout_bytes = (len(lay["pack"]) + 8 * len(lay["chunks"]) + 56 * len(lay["programs"]) +
                    4 * max(ysz, 1) + 4 * max(zsz, 1) + 4 * rows + (8 * groups if resident else 0))
    assert m30 - q(M, P, 30, H.GMRES, H.MIXED_FP32) == layout_bytes
    for bad in (dict(restart=0, method=H.GMRES), dict(restart=500, method=H.GMRES),
                dict(restart=0, method=H.BICGSTAB, flags=H.MIXED_FP32), dict(restart=30, method=7)):
        with pytest.raises(H.HecError):
            q(M, P, **bad)


def test_spmv_rejects_misaligned_output(H):
    """The SpMV stores its adjacent rows (two in FP64, four in FP32) with one
    16-byte vector store, so y_out must be 16-byte aligned; a misaligned
    output is rejected before any device work (the addresses below are
    never dereferenced)."""
    import ctypes
    A = synth.poisson2d_5pt(4)
    M = H.hec_build(A.row_ptr, A.col, A.val, host_only=True)
    lib = H.load_library()
    x = ctypes.c_void_p(0x10000)
    for y, f32 in ((0x20008, False), (0x20004, True), (0x20008, True)):
        if f32:
            rc = lib.hec_spmv_f32(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(y), None)
        else:
            rc = lib.hec_spmv(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(y), None, None, None)
        assert rc == H.ERR_INVALID
        assert b"aligned" in lib.hec_last_error()
    # aligned: rejected for the host-only handle instead, after the alignment check
    rc = lib.hec_spmv(M.handle, 1.0, x, 0.0, None, ctypes.c_void_p(0x20010), None, None, None)
    assert rc == H.ERR_INVALID and b"host-only" in lib.hec_last_error()
