// hec_setup.cpp -- host setup: HEC conversion (Section 2.1), RAS blocks
// (Section 2.5), ILU(k) (Section 2.4, Eqs. 9-10, Algorithm 2), level schedule
// (Section 2.6, Eq. 11).  The triangular-solve layout is in trsv_layout.cpp.
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
        // checked before row i's columns are read: they must lie in [0, nnz)
        if (rp[i + 1] < rp[i] || rp[i + 1] > nnz) {
            msg = "row_ptr decreases or exceeds nnz at row " + std::to_string(i);
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
    // The tail schedule.  A tile's short tail rows are read by groups of g
    // lanes (g = 4..32, a power of two near half their mean length, so that
    // a warp is busy on rows of a few entries as on rows of a hundred); rows
    // longer than kSpmvLongRow are read by the whole CTA, one at a time.
    H.tile_group.assign(ntiles, 32);
    H.tile_long.assign(ntiles + 1, 0);
    H.tail_long.clear();
    for (int tile = 0; tile < ntiles; ++tile) {
        H.tile_long[tile] = (int)H.tail_long.size();
        int64_t len_sum = 0, nshort = 0;
        for (int q = H.tile_tail[tile]; q < H.tile_tail[tile + 1]; ++q) {
            const int len = H.tail_ptr[q + 1] - H.tail_ptr[q];
            if (len > kSpmvLongRow) {
                H.tail_long.push_back(q);
            } else {
                len_sum += len;
                ++nshort;
            }
        }
        int g = 4;
        if (nshort > 0)
            while (g < 32 && 2 * (int64_t)g * nshort < len_sum)
                g *= 2;
        H.tile_group[tile] = g;
    }
    H.tile_long[ntiles] = (int)H.tail_long.size();
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
        // grow by breadth-first layers over the graph of A; membership is a byte map
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

} // namespace hec
