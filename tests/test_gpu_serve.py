"""The solve server: continuous batching over lanes, admission by device
memory, keyed residency, results independent of the mix.

Tolerance: every solve reaches the true FP64 relative residual 1e-8 (checked
with the oracle's SpMV); the same request gives a bit-identical solution
alone and in a mix (each request's arithmetic is fixed by the request)."""
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


def mix():
    """Requests on both paths (one-CTA batched for <= 32768 unknowns, the
    single-system RAS path above), all three stencils, ILU(0) and ILU(1)."""
    reqs = []
    for i, (st, side, k) in enumerate([(5, 20, 0), (7, 12, 1), (27, 9, 0), (5, 90, 1),
                                       (7, 40, 0), (27, 33, 1), (5, 200, 0), (7, 16, 0),
                                       (27, 14, 1), (5, 64, 0)]):
        A = synth.serving_matrix({"stencil": st, "side": side, "k": k, "seed": 100 + i})
        reqs.append((A, synth.rhs_uniform(A.n, 200 + i), k))
    return reqs


def run_all(H, reqs, lanes, budget=0, keys=None, flags=None):
    flags = H.MIXED_FP32 if flags is None else flags
    out = {}
    with H.Server(lanes=lanes, device_budget=budget, flags=flags) as S:
        tickets = []
        for i, (A, b, k) in enumerate(reqs):
            tickets.append(S.submit(A, b, ilu_k=k, key=(keys[i] if keys else 0), tag=i))
        got = []
        while len(got) < len(reqs):
            got += S.poll(wait_ms=200)
        for r in got:
            out[r["tag"]] = (r, S.solution(r["ticket"], reqs[r["tag"]][0].n))
    return out


def test_serve_mix_converges(H, orc):
    reqs = mix()
    res = run_all(H, reqs, lanes=6)
    assert sorted(res) == list(range(len(reqs)))
    for i, (A, b, k) in enumerate(reqs):
        r, x = res[i]
        assert r["status"] == H.OK, r
        assert np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b) <= 1e-8
        assert r["t_submit"] <= r["t_start"] <= r["t_setup"] <= r["t_done"]
    # the lanes overlapped: some request started before another one finished
    iv = sorted((res[i][0]["t_start"], res[i][0]["t_done"]) for i in res)
    assert any(iv[j + 1][0] < iv[j][1] for j in range(len(iv) - 1))


def test_serve_result_identical_alone_and_in_mix(H):
    reqs = mix()
    together = run_all(H, reqs, lanes=8)
    for i in (0, 3, 5, 6):
        alone = run_all(H, [reqs[i]], lanes=1)
        assert np.array_equal(alone[0][1], together[i][1]), i
        assert alone[0][0]["iters"] == together[i][0]["iters"]


def test_serve_admission_by_device_memory(H, orc):
    """A budget below two requests' footprint: requests still all complete,
    one at a time."""
    reqs = [r for r in mix() if r[0].n > 5000][:4]
    res = run_all(H, reqs, lanes=4, budget=1)
    iv = sorted((res[i][0]["t_start"], res[i][0]["t_done"]) for i in res)
    assert all(iv[j + 1][0] >= iv[j][1] for j in range(len(iv) - 1))
    for i, (A, b, k) in enumerate(reqs):
        assert res[i][0]["status"] == H.OK
        assert np.linalg.norm(b - orc.spmv(A, res[i][1])) <= 1e-8 * np.linalg.norm(b)


def test_serve_keyed_reuse(H, orc):
    A = synth.serving_matrix({"stencil": 7, "side": 36, "k": 1, "seed": 5})
    bs = [synth.rhs_uniform(A.n, s) for s in (1, 2, 3)]
    with H.Server(lanes=2, flags=H.MIXED_FP32) as S:
        t = [S.submit(A, b, ilu_k=1, key=77, tag=i) for i, b in enumerate(bs)]
        got = []
        while len(got) < 3:
            got += S.poll(wait_ms=200)
        got.sort(key=lambda r: r["tag"])
        assert [r["reused"] for r in got] == [0, 1, 1]
        # one key serves one request at a time
        assert got[1]["t_start"] >= got[0]["t_done"] and got[2]["t_start"] >= got[1]["t_done"]
        for r, b in zip(got, bs):
            x = S.solution(r["ticket"], A.n)
            assert r["status"] == H.OK
            assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)
        assert S.stats()["reserved"] > 0  # the keyed system stays resident
        # a keyed request without its matrix uses the resident system
        t = S.submit(None, bs[0], ilu_k=1, key=77, tag=5)
        r = []
        while not r:
            r = S.poll(wait_ms=200)
        assert r[0]["status"] == H.OK and r[0]["reused"] == 1
        S.solution(t, A.n)
        S.submit(None, np.ones(5), ilu_k=0, key=78, tag=6)  # nothing resident under 78
        r = []
        while not r:
            r = S.poll(wait_ms=200)
        assert r[0]["status"] == H.ERR_INVALID
        # the same key with another matrix is refused per request
        B = synth.serving_matrix({"stencil": 5, "side": 10, "k": 1, "seed": 6})
        S.submit(B, np.ones(B.n), ilu_k=1, key=77, tag=9)
        r = []
        while not r:
            r = S.poll(wait_ms=200)
        assert r[0]["status"] == H.ERR_INVALID


def test_serve_fp64_and_invalid(H, orc):
    reqs = mix()[:3]
    res = run_all(H, reqs, lanes=2, flags=0)
    for i, (A, b, k) in enumerate(reqs):
        assert res[i][0]["status"] == H.OK
        assert np.linalg.norm(b - orc.spmv(A, res[i][1])) <= 1e-8 * np.linalg.norm(b)
    with pytest.raises(H.HecError):
        H.Server(restart=40)
    with H.Server(lanes=1) as S:
        with pytest.raises(H.HecError):
            S.solution(12345, 10)


def test_serve_keyed_new_values_refactor_on_device(H, orc):
    """A keyed request carrying new values of the resident pattern is
    refactored on the GPU (hec_refactor) instead of set up again; its result
    is bit-identical to a cold solve of the new matrix.  A one-CTA batched
    system with new values is set up again."""
    big0 = synth.serving_matrix({"stencil": 7, "side": 36, "k": 1, "seed": 5})
    big1 = synth.serving_matrix({"stencil": 7, "side": 36, "k": 1, "seed": 8})
    small0 = synth.serving_matrix({"stencil": 5, "side": 40, "k": 0, "seed": 2})
    small1 = synth.serving_matrix({"stencil": 5, "side": 40, "k": 0, "seed": 3})
    assert np.array_equal(big0.col, big1.col) and not np.array_equal(big0.val, big1.val)
    b_big = synth.rhs_uniform(big0.n, 4)
    b_small = synth.rhs_uniform(small0.n, 5)

    def solve_all(items):
        out = []
        with H.Server(lanes=1, flags=H.MIXED_FP32) as S:
            for i, (A, b, k, key) in enumerate(items):
                t = S.submit(A, b, ilu_k=k, key=key, tag=i)
                r = []
                while not r:
                    r = S.poll(wait_ms=200)
                out.append((r[0], S.solution(t, A.n)))
        return out

    keyed = solve_all([(big0, b_big, 1, 90), (big1, b_big, 1, 90),
                       (small0, b_small, 0, 91), (small1, b_small, 0, 91)])
    cold = solve_all([(big1, b_big, 1, 0), (small1, b_small, 0, 0)])
    assert keyed[1][0]["reused"] == 1 and keyed[1][0]["refactored"] == 1
    assert keyed[3][0]["reused"] == 1 and keyed[3][0]["refactored"] == 0
    for (r, x), (rc, xc), (A, b) in ((keyed[1], cold[0], (big1, b_big)),
                                     (keyed[3], cold[1], (small1, b_small))):
        assert r["status"] == H.OK and rc["status"] == H.OK
        assert np.array_equal(x, xc)
        assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)


def test_serve_failed_refactor_drops_the_resident_system(H, orc):
    """New values of the resident pattern with a zero first pivot: the
    refactor fails (the request's status), the key's system is dropped
    rather than kept half-updated, a request with the key alone then finds
    nothing resident, and the key set up again from a matrix solves."""
    A = synth.serving_matrix({"stencil": 7, "side": 36, "k": 1, "seed": 5})
    b = synth.rhs_uniform(A.n, 4)
    r0, r1 = int(A.row_ptr[0]), int(A.row_ptr[1])
    bad_val = A.val.copy()
    bad_val[r0 + int(np.flatnonzero(A.col[r0:r1] == 0)[0])] = 0.0
    bad = synth.CSR(A.row_ptr, A.col, bad_val)

    def one(S, M, key, tag):
        t = S.submit(M, b, ilu_k=1, key=key, tag=tag)
        r = []
        while not r:
            r = S.poll(wait_ms=200)
        return t, r[0]

    with H.Server(lanes=1, flags=H.MIXED_FP32) as S:
        t, r = one(S, A, 92, 0)
        assert r["status"] == H.OK and r["reused"] == 0
        S.solution(t, A.n)
        assert S.stats()["reserved"] > 0
        _, r = one(S, bad, 92, 1)
        assert r["reused"] == 1 and r["refactored"] == 1
        assert r["status"] == H.ERR_ZERO_PIVOT
        assert S.stats()["reserved"] == 0
        _, r = one(S, None, 92, 2)
        assert r["status"] == H.ERR_INVALID
        t, r = one(S, A, 92, 3)
        assert r["status"] == H.OK and r["reused"] == 0
        x = S.solution(t, A.n)
        assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-8 * np.linalg.norm(b)
