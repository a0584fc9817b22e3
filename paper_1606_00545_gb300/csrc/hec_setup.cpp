// hec_setup.cpp -- host setup: HEC conversion (Section 2.1), RAS blocks
// (Section 2.5), ILU(k) (Section 2.4, Eqs. 9-10, Algorithm 2), level schedule
// (Section 2.6, Eq. 11) and the chunk layout of the triangular-solve kernel.
#include "hec_setup.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>

#include "../../include/hecgpu.h"

namespace hec {

void parallel_for(int count, const std::function<void(int)> &f)
{
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::min<unsigned>(hw ? hw : 1, 32u);
    nt = std::min(nt, count);
    if (nt <= 1) {
        for (int i = 0; i < count; ++i)
            f(i);
        return;
    }
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&]() {
            for (int i = next++; i < count; i = next++)
                f(i);
        });
    for (auto &t : th)
        t.join();
}

int check_csr(int n, const int *rp, const int *ci, int nnz, bool need_diag, std::string &msg)
{
    if (n < 1 || !rp || (nnz > 0 && !ci)) {
        msg = "matrix must have n >= 1 and non-null arrays";
        return HEC_ERR_INVALID;
    }
    if (rp[0] != 0 || rp[n] != nnz) {
        msg = "row_ptr[0] must be 0 and row_ptr[n] must equal nnz";
        return HEC_ERR_INVALID;
    }
    for (int i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) {
            msg = "row_ptr decreases at row " + std::to_string(i);
            return HEC_ERR_INVALID;
        }
        bool diag = false;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n) {
                msg = "column index out of range in row " + std::to_string(i);
                return HEC_ERR_UNSORTED_CSR;
            }
            if (e > rp[i] && ci[e] <= ci[e - 1]) {
                msg = "columns not strictly ascending in row " + std::to_string(i);
                return HEC_ERR_UNSORTED_CSR;
            }
            diag |= (ci[e] == i);
        }
        if (need_diag && !diag) {
            msg = "diagonal entry missing in row " + std::to_string(i);
            return HEC_ERR_INVALID;
        }
    }
    return HEC_OK;
}

// ---------------------------------------------------------------- HEC

// Width of the ELL slab: the largest K such that at least a third of the rows
// hold K or more entries (the ELL/COO split criterion of Bell and Garland that
// Section 2.1 cites for its ELL/CSR boundary).
int ell_width_auto(const HostCSR &A)
{
    int maxlen = 0;
    for (int i = 0; i < A.n; ++i)
        maxlen = std::max(maxlen, A.rp[i + 1] - A.rp[i]);
    std::vector<int64_t> atleast(maxlen + 2, 0);
    for (int i = 0; i < A.n; ++i)
        atleast[A.rp[i + 1] - A.rp[i]]++;
    for (int k = maxlen - 1; k >= 0; --k)
        atleast[k] += atleast[k + 1];
    int K = 0;
    for (int k = 1; k <= maxlen; ++k)
        if (3 * atleast[k] >= (int64_t)A.n)
            K = k;
    return std::max(K, 1);
}

void build_hec(const HostCSR &A, int K, int align, HecHost &H)
{
    const int n = A.n;
    H.n = n;
    H.K = K;
    H.ld = (int)(((int64_t)n + align - 1) / align * align);
    H.ell_col.assign((size_t)K * H.ld, 0);
    H.ell_val.assign((size_t)K * H.ld, 0.0);
    H.tail_rows.clear();
    H.tail_ptr.assign(1, 0);
    H.tail_col.clear();
    H.tail_val.clear();
    for (int i = 0; i < H.ld; ++i) {
        const int len = i < n ? A.rp[i + 1] - A.rp[i] : 0;
        for (int k = 0; k < K; ++k) {
            size_t o = (size_t)k * H.ld + i;
            if (k < len) {
                H.ell_col[o] = A.ci[A.rp[i] + k];
                H.ell_val[o] = A.va[A.rp[i] + k];
            } else {
                H.ell_col[o] = i < n ? i : 0; // padding: value 0, own row
                H.ell_val[o] = 0.0;
            }
        }
        if (len > K) {
            H.tail_rows.push_back(i);
            for (int e = A.rp[i] + K; e < A.rp[i + 1]; ++e) {
                H.tail_col.push_back(A.ci[e]);
                H.tail_val.push_back(A.va[e]);
            }
            H.tail_ptr.push_back((int)H.tail_col.size());
        }
    }
    const int ntiles = (n + kSpmvTile - 1) / kSpmvTile;
    H.tile_tail.assign(ntiles + 1, 0);
    size_t t = 0;
    for (int tile = 0; tile <= ntiles; ++tile) {
        const int64_t start = (int64_t)tile * kSpmvTile;
        while (t < H.tail_rows.size() && H.tail_rows[t] < start)
            ++t;
        H.tile_tail[tile] = (int)t;
    }
}

// ---------------------------------------------------------------- RAS blocks

// Section 2.5 on one device.  Owned rows: the sequence partition (Section
// 2.2) W_b = [floor(b n / nb), floor((b+1) n / nb)).  Overlap: `overlap`
// breadth-first layers of the row-pattern graph around W_b.  A_b =
// A[V_b, V_b] with V_b in ascending order; entries leaving the block dropped.
void ras_blocks(const HostCSR &A, int nblocks, int overlap, std::vector<BlockFactor> &out)
{
    const int n = A.n;
    out.assign(nblocks, BlockFactor());
    parallel_for(nblocks, [&](int b) {
        BlockFactor &B = out[b];
        B.own_lo = (int)((int64_t)b * n / nblocks);
        B.own_hi = (int)((int64_t)(b + 1) * n / nblocks);
        std::vector<int> frontier, members;
        std::vector<char> in;
        // grow by layers; membership kept in a hash-free sorted merge when small
        in.assign(n, 0);
        for (int i = B.own_lo; i < B.own_hi; ++i) {
            in[i] = 1;
            frontier.push_back(i);
        }
        members = frontier;
        for (int d = 0; d < overlap; ++d) {
            std::vector<int> next;
            for (int i : frontier)
                for (int e = A.rp[i]; e < A.rp[i + 1]; ++e) {
                    const int j = A.ci[e];
                    if (!in[j]) {
                        in[j] = 1;
                        next.push_back(j);
                    }
                }
            members.insert(members.end(), next.begin(), next.end());
            frontier.swap(next);
        }
        std::sort(members.begin(), members.end());
        B.rows = members;
        // global -> local through binary search over the sorted member list
        const int nv = (int)B.rows.size();
        B.F.n = nv;
        B.F.rp.assign(nv + 1, 0);
        B.F.ci.clear();
        B.F.va.clear();
        for (int t = 0; t < nv; ++t) {
            const int i = B.rows[t];
            for (int e = A.rp[i]; e < A.rp[i + 1]; ++e) {
                const int j = A.ci[e];
                if (!in[j])
                    continue;
                const int lj = (int)(std::lower_bound(B.rows.begin(), B.rows.end(), j) - B.rows.begin());
                B.F.ci.push_back(lj);
                B.F.va.push_back(A.va[e]);
            }
            B.F.rp[t + 1] = (int)B.F.ci.size();
        }
    });
}

// ---------------------------------------------------------------- ILU(k)

// Symbolic phase: the fill pattern and levels of ILU(k) (Eqs. 9-10).  Row i
// is a sorted linked list that starts from the pattern of A (level 0); every
// pivot p < i of the list merges the kept upper part of row p, a position
// being admitted only with a level <= k (a level above k can never become a
// pivot nor lower another level to <= k, so pruning it early changes
// nothing).  Numeric phase: the IKJ elimination of Algorithm 2 restricted to
// that pattern -- every kept position receives exactly the updates Algorithm
// 2 applies to it, in the same pivot order.
int iluk_block(BlockFactor &B, int k, std::string &msg)
{
    HostCSR &A = B.F;
    const int n = A.n;
    std::vector<int> frp(n + 1, 0), fci, flev, fdiag(n, -1);
    fci.reserve(A.ci.size() * 2);
    flev.reserve(A.ci.size() * 2);
    std::vector<int> nxt(n, -1), lv(n, 0), stamp(n, -1);
    for (int i = 0; i < n; ++i) {
        int head = -1, tail = -1;
        for (int e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int j = A.ci[e];
            lv[j] = 0;
            stamp[j] = i;
            nxt[j] = -1;
            if (tail < 0)
                head = j;
            else
                nxt[tail] = j;
            tail = j;
        }
        for (int p = head; p >= 0 && p < i; p = nxt[p]) {
            const int lp = lv[p];
            int cursor = p;
            for (int e = fdiag[p] + 1; e < frp[p + 1]; ++e) {
                const int j = fci[e];
                const int cand = lp + flev[e] + 1;
                if (stamp[j] == i) {
                    if (cand < lv[j])
                        lv[j] = cand;
                    cursor = j;
                    continue;
                }
                if (cand > k)
                    continue;
                while (nxt[cursor] >= 0 && nxt[cursor] < j)
                    cursor = nxt[cursor];
                stamp[j] = i;
                lv[j] = cand;
                nxt[j] = nxt[cursor];
                nxt[cursor] = j;
                cursor = j;
            }
        }
        for (int j = head; j >= 0; j = nxt[j]) {
            if (j == i)
                fdiag[i] = (int)fci.size();
            fci.push_back(j);
            flev.push_back(lv[j]);
        }
        frp[i + 1] = (int)fci.size();
        if (fdiag[i] < 0) {
            msg = "diagonal entry missing";
            return HEC_ERR_INVALID;
        }
    }
    // numeric phase
    std::vector<double> fva(fci.size(), 0.0), w(n, 0.0);
    std::vector<int> mark(n, -1);
    for (int i = 0; i < n; ++i) {
        for (int e = frp[i]; e < frp[i + 1]; ++e) {
            w[fci[e]] = 0.0;
            mark[fci[e]] = i;
        }
        for (int e = A.rp[i]; e < A.rp[i + 1]; ++e)
            w[A.ci[e]] = A.va[e];
        for (int e = frp[i]; e < fdiag[i]; ++e) {
            const int p = fci[e];
            const double upp = fva[fdiag[p]];
            if (upp == 0.0) {
                msg = "zero pivot at local row " + std::to_string(p);
                return HEC_ERR_ZERO_PIVOT;
            }
            const double lip = w[p] / upp;
            w[p] = lip;
            for (int f = fdiag[p] + 1; f < frp[p + 1]; ++f) {
                const int j = fci[f];
                if (mark[j] == i)
                    w[j] = w[j] - lip * fva[f];
            }
        }
        for (int e = frp[i]; e < frp[i + 1]; ++e)
            fva[e] = w[fci[e]];
        if (fva[fdiag[i]] == 0.0) {
            msg = "zero pivot at local row " + std::to_string(i);
            return HEC_ERR_ZERO_PIVOT;
        }
    }
    A.rp.swap(frp);
    A.ci.swap(fci);
    A.va.swap(fva);
    B.lev.swap(flev);
    B.diag.swap(fdiag);
    return HEC_OK;
}

// ---------------------------------------------------------------- levels (Eq. 11)

static void level_sets(const std::vector<int> &lev, int nlev, std::vector<int> &ptr,
                       std::vector<int> &rows)
{
    ptr.assign(nlev + 1, 0);
    for (int l : lev)
        ptr[l]++;
    for (int l = 0; l < nlev; ++l)
        ptr[l + 1] += ptr[l];
    rows.assign(lev.size(), 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < (int)lev.size(); ++i) // ascending rows inside a level
        rows[fill[lev[i] - 1]++] = i;
}

void levels_block(BlockFactor &B)
{
    const HostCSR &F = B.F;
    const int n = F.n;
    B.levL.assign(n, 0);
    B.levU.assign(n, 0);
    B.nlevL = B.nlevU = 0;
    for (int i = 0; i < n; ++i) {
        int m = 0;
        for (int e = F.rp[i]; e < B.diag[i]; ++e)
            m = std::max(m, B.levL[F.ci[e]]);
        B.levL[i] = m + 1;
        B.nlevL = std::max(B.nlevL, m + 1);
    }
    for (int i = n - 1; i >= 0; --i) {
        int m = 0;
        for (int e = B.diag[i] + 1; e < F.rp[i + 1]; ++e)
            m = std::max(m, B.levU[F.ci[e]]);
        B.levU[i] = m + 1;
        B.nlevU = std::max(B.nlevU, m + 1);
    }
    level_sets(B.levL, B.nlevL, B.lptrL, B.lrowsL);
    level_sets(B.levU, B.nlevU, B.lptrU, B.lrowsU);
}

// ---------------------------------------------------------------- chunk layout

namespace {

inline int r2(int x) { return (x + 1) & ~1; }
inline int r4(int x) { return (x + 3) & ~3; }

size_t chunk_bytes(int nrows, int width, bool upass)
{
    size_t b = 16 + (size_t)width * (8 * r2(nrows) + 4 * r4(nrows)) + 4 * (size_t)r4(nrows);
    if (upass)
        b += 4 * (size_t)r4(nrows) + 8 * (size_t)r2(nrows);
    return (b + 15) & ~(size_t)15;
}

struct PassRows {
    std::vector<int> order;     // needed rows in level-major order
    std::vector<int> level_end; // end offsets into order, one per level
};

} // namespace

// Which rows a block must solve: the U solve needs the owned rows and,
// transitively, the rows they depend on through U (higher local indices);
// the L solve needs every row whose y the U solve reads and, transitively,
// their L dependencies.  The other rows cannot influence the owned part of
// the result and are left out of the device program (the result on the
// owned rows is unchanged).
int pack_trsv(const std::vector<BlockFactor> &Bs, int n, int stage_bytes, int max_ring,
              TrsvPack &P, std::string &msg)
{
    (void)n;
    const int nb = (int)Bs.size();
    P.pack.clear();
    P.chunks.clear();
    P.blocks.assign(nb, TrsvBlock());
    P.ysz = P.zsz = 0;
    P.alg_bytes = 0;
    P.rows_L = P.rows_U = 0;
    int ring_need = 32;
    struct BlockOut {
        std::vector<unsigned char> bytes;
        std::vector<uint2> chunks; // offsets relative to this block
        int nL = 0, nU = 0, spanL = 0, spanU = 0;
        int64_t alg = 0;
        std::string err;
    };
    std::vector<BlockOut> outs(nb);
    parallel_for(nb, [&](int b) {
        const BlockFactor &B = Bs[b];
        const HostCSR &F = B.F;
        const int nv = F.n;
        BlockOut &O = outs[b];
        std::vector<char> needU(nv, 0), needL(nv, 0), owned(nv, 0);
        for (int i = 0; i < nv; ++i)
            owned[i] = (B.rows[i] >= B.own_lo && B.rows[i] < B.own_hi);
        for (int i = 0; i < nv; ++i) {
            needU[i] |= owned[i];
            if (needU[i])
                for (int e = B.diag[i] + 1; e < F.rp[i + 1]; ++e)
                    needU[F.ci[e]] = 1;
        }
        for (int i = nv - 1; i >= 0; --i) {
            needL[i] |= needU[i];
            if (needL[i])
                for (int e = F.rp[i]; e < B.diag[i]; ++e)
                    needL[F.ci[e]] = 1;
        }
        std::vector<int> posL(nv, -1), posU(nv, -1);
        auto order_pass = [&](bool upass, std::vector<int> &pos) {
            const std::vector<int> &ptr = upass ? B.lptrU : B.lptrL;
            const std::vector<int> &rows = upass ? B.lrowsU : B.lrowsL;
            const std::vector<char> &need = upass ? needU : needL;
            PassRows pr;
            for (size_t l = 0; l + 1 < ptr.size(); ++l) {
                for (int q = ptr[l]; q < ptr[l + 1]; ++q)
                    if (need[rows[q]]) {
                        pos[rows[q]] = (int)pr.order.size();
                        pr.order.push_back(rows[q]);
                    }
                pr.level_end.push_back((int)pr.order.size());
            }
            return pr;
        };
        PassRows pl = order_pass(false, posL);
        PassRows pu = order_pass(true, posU);
        O.nL = (int)pl.order.size();
        O.nU = (int)pu.order.size();
        auto emit = [&](bool upass, const PassRows &pr, const std::vector<int> &pos, int &span) {
            int start = 0;
            span = 0;
            for (int end : pr.level_end) {
                int q = start;
                while (q < end) {
                    // greedy chunk: rows [q, q2) of this level
                    int q2 = q, width = 0;
                    while (q2 < end && q2 - q < kThreads) {
                        const int i = pr.order[q2];
                        const int len = upass ? F.rp[i + 1] - B.diag[i] - 1 : B.diag[i] - F.rp[i];
                        const int w2 = std::max(width, len);
                        if (chunk_bytes(q2 - q + 1, w2, upass) > (size_t)stage_bytes)
                            break;
                        width = w2;
                        ++q2;
                    }
                    if (q2 == q) {
                        O.err = "a factor row is too long for one shared-memory stage";
                        return;
                    }
                    const int nr = q2 - q, n2 = r2(nr), n4 = r4(nr);
                    const size_t bytes = chunk_bytes(nr, width, upass);
                    const size_t off = O.bytes.size();
                    O.bytes.resize(off + bytes, 0);
                    unsigned char *ch = O.bytes.data() + off;
                    int hdr[4] = {nr, width, q, upass ? 1 : 0};
                    std::memcpy(ch, hdr, 16);
                    double *val = reinterpret_cast<double *>(ch + 16);
                    int *dep = reinterpret_cast<int *>(val + (size_t)width * n2);
                    int *src = dep + (size_t)width * n4;
                    int *dst = src + n4;
                    double *dinv = reinterpret_cast<double *>(dst + n4);
                    int mindep = q;
                    for (int t = 0; t < nr; ++t) {
                        const int i = pr.order[q + t];
                        const int e0 = upass ? B.diag[i] + 1 : F.rp[i];
                        const int e1 = upass ? F.rp[i + 1] : B.diag[i];
                        const int len = e1 - e0;
                        if (len == 0 && width > 0) {
                            // a row of level >= 2 always has a dependency
                            O.err = "internal: dependency-free row in a dependent level";
                            return;
                        }
                        for (int kk = 0; kk < width; ++kk) {
                            // padding repeats the first dependency with value 0
                            const int e = kk < len ? e0 + kk : e0;
                            const int d = (upass ? posU : posL)[F.ci[e]];
                            dep[(size_t)kk * n4 + t] = d;
                            val[(size_t)kk * n2 + t] = kk < len ? F.va[e] : 0.0;
                            if (len > 0)
                                mindep = std::min(mindep, d);
                        }
                        if (upass) {
                            src[t] = posL[i];
                            dst[t] = owned[i] ? B.rows[i] : -1;
                            dinv[t] = 1.0 / F.va[B.diag[i]];
                            O.alg += 12ll * len + 8 /*y*/ + 8 /*dinv*/ + 4 /*src*/ + 4 /*dst*/ +
                                     (owned[i] ? 8 : 0);
                        } else {
                            src[t] = B.rows[i];
                            O.alg += 12ll * len + 8 /*r*/ + 8 /*y*/ + 4 /*src*/;
                        }
                    }
                    span = std::max(span, (q + nr) - mindep);
                    O.chunks.push_back(make_uint2((unsigned)(off / 16), (unsigned)bytes));
                    q = q2;
                }
                start = end;
            }
        };
        emit(false, pl, posL, O.spanL);
        if (!O.err.empty())
            return;
        emit(true, pu, posU, O.spanU);
    });
    for (int b = 0; b < nb; ++b)
        if (!outs[b].err.empty()) {
            msg = outs[b].err;
            return HEC_ERR_INVALID;
        }
    // ring size: the largest window that fits, power of two
    auto pow2 = [](int v) {
        int p = 32;
        while (p < v)
            p <<= 1;
        return p;
    };
    for (int b = 0; b < nb; ++b) {
        if (pow2(outs[b].spanL + 1) <= max_ring)
            ring_need = std::max(ring_need, pow2(outs[b].spanL + 1));
        if (pow2(outs[b].spanU + 1) <= max_ring)
            ring_need = std::max(ring_need, pow2(outs[b].spanU + 1));
    }
    P.ring_slots = ring_need;
    size_t total = 0;
    for (auto &O : outs)
        total += O.bytes.size();
    P.pack.resize(total);
    size_t off = 0;
    int64_t yoff = 0, zoff = 0;
    bool any_global_u = false;
    for (int b = 0; b < nb; ++b) {
        BlockOut &O = outs[b];
        TrsvBlock &T = P.blocks[b];
        T.chunk_begin = (int)P.chunks.size();
        for (const uint2 &c : O.chunks)
            P.chunks.push_back(make_uint2((unsigned)(c.x + off / 16), c.y));
        T.chunk_end = (int)P.chunks.size();
        std::memcpy(P.pack.data() + off, O.bytes.data(), O.bytes.size());
        off += O.bytes.size();
        T.ring_L = (O.spanL + 1 <= ring_need) ? 1 : 0;
        T.ring_U = (O.spanU + 1 <= ring_need) ? 1 : 0;
        T.yoff = yoff;
        yoff += O.nL;
        T.zoff = zoff;
        if (!T.ring_U) {
            zoff += O.nU;
            any_global_u = true;
        }
        P.alg_bytes += O.alg;
        P.rows_L += O.nL;
        P.rows_U += O.nU;
    }
    if (off / 16 > 0xffffffffull) {
        msg = "factor layout exceeds 64 GiB";
        return HEC_ERR_INVALID;
    }
    P.ysz = yoff;
    P.zsz = any_global_u ? zoff : 0;
    return HEC_OK;
}

} // namespace hec
