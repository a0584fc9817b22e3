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

// ---------------------------------------------------------------- chunk layout

namespace {

constexpr int kWarpRows = 32;
constexpr int kMaxWarps = kThreads / kWarpRows;
// counts, one width and one segment offset per warp, section offsets
constexpr int kChunkHeader = 16 + 4 * kMaxWarps + 4 * kMaxWarps + 16;

inline int r32(int x) { return (x + kWarpRows - 1) & ~(kWarpRows - 1); }

// Lane stride of warp w's segment: 32 for a full warp, the row count rounded
// up to 4 for the last, partial one.
inline int seg_stride(int w, int nrows)
{
    const int left = nrows - w * kWarpRows;
    return left >= kWarpRows ? kWarpRows : (left + 3) & ~3;
}

// Chunk layout (offsets in bytes, every section 16-byte aligned):
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass)
//   [16, 48)  width of every warp's segment (entries per row, uniform in the warp)
//   [48, 80)  byte offset of every warp's segment
//   [80, 96)  byte offsets of src, dst, dinv, and 0
//   per warp w < nwarps: val[width_w][stride_w] (value), dep[width_w][stride_w] (int32)
//   src[r32(nrows)] (int32), and for U: dst[r32(nrows)] (int32), dinv[r32(nrows)] (value)
// Values are vb bytes: 8 (FP64 layout) or 4 (FP32 layout of the mixed-precision
// mode).  Row t of the chunk is handled by thread t (warp t / 32, lane t % 32).
size_t chunk_bytes(const std::vector<int> &widths, int nrows, bool upass, int vb)
{
    size_t b = kChunkHeader;
    for (size_t w = 0; w < widths.size(); ++w)
        b += (size_t)widths[w] * seg_stride((int)w, nrows) * (vb + 4);
    b += 4 * (size_t)r32(nrows);
    if (upass)
        b += (4 + vb) * (size_t)r32(nrows);
    return (b + 15) & ~(size_t)15;
}

inline void put_value(unsigned char *base, size_t i, double v, int vb)
{
    if (vb == 8)
        reinterpret_cast<double *>(base)[i] = v;
    else
        reinterpret_cast<float *>(base)[i] = (float)v;
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
int max_factor_width(const std::vector<BlockFactor> &Bs, bool upass)
{
    int w = 0;
    for (const BlockFactor &B : Bs)
        for (int i = 0; i < B.F.n; ++i)
            w = std::max(w, upass ? B.F.rp[i + 1] - B.diag[i] - 1 : B.diag[i] - B.F.rp[i]);
    return w;
}

int pack_trsv(const std::vector<BlockFactor> &Bs, int n, int stage_bytes, int max_ring, int vb,
              TrsvPack &P, std::string &msg, int uniform_width)
{
    (void)n;
    if (vb != 8 && vb != 4) {
        msg = "value size must be 8 or 4 bytes";
        return HEC_ERR_INVALID;
    }
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
        int nL = 0, nU = 0, spanL = 0, spanU = 0, nchunksL = 0;
        std::vector<int> rows_per_chunk, rm_start, rm_len, rm_diag; // block-local entries
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
        // off-diagonal entries of row i in the L (upass false) or U factor
        auto row_len = [&](bool upass, int i) {
            return upass ? F.rp[i + 1] - B.diag[i] - 1 : B.diag[i] - F.rp[i];
        };
        auto order_pass = [&](bool upass, std::vector<int> &pos) {
            const std::vector<int> &ptr = upass ? B.lptrU : B.lptrL;
            const std::vector<int> &rows = upass ? B.lrowsU : B.lrowsL;
            const std::vector<char> &need = upass ? needU : needL;
            PassRows pr;
            std::vector<int> lvl;
            for (size_t l = 0; l + 1 < ptr.size(); ++l) {
                lvl.clear();
                for (int q = ptr[l]; q < ptr[l + 1]; ++q)
                    if (need[rows[q]])
                        lvl.push_back(rows[q]);
                // inside a level rows are independent: longest first, so each
                // warp's segment pads little (stable: ties keep row order)
                std::stable_sort(lvl.begin(), lvl.end(), [&](int x, int y) {
                    return row_len(upass, x) > row_len(upass, y);
                });
                for (int i : lvl) {
                    pos[i] = (int)pr.order.size();
                    pr.order.push_back(i);
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
            (void)pos;
            int start = 0;
            span = 0;
            std::vector<int> widths;
            for (int end : pr.level_end) {
                int q = start;
                while (q < end) {
                    // greedy chunk: rows [q, q2) of this level, warp w takes rows
                    // 32w .. 32w+31; rows are sorted longest first, so a warp's
                    // width is the length of its first row
                    int q2 = q;
                    widths.clear();
                    while (q2 < end && q2 - q < kThreads) {
                        const int j = q2 - q;
                        if (j % kWarpRows == 0)
                            widths.push_back(uniform_width > 0 ? uniform_width
                                                               : row_len(upass, pr.order[q2]));
                        if (chunk_bytes(widths, j + 1, upass, vb) > (size_t)stage_bytes) {
                            if (j % kWarpRows == 0)
                                widths.pop_back();
                            break;
                        }
                        ++q2;
                    }
                    if (q2 == q) {
                        O.err = "a factor row is too long for one shared-memory stage";
                        return;
                    }
                    const int nr = q2 - q, npad = r32(nr), nw = (int)widths.size();
                    const size_t bytes = chunk_bytes(widths, nr, upass, vb);
                    const size_t off = O.bytes.size();
                    O.bytes.resize(off + bytes, 0);
                    unsigned char *ch = O.bytes.data() + off;
                    int hdr[kChunkHeader / 4] = {nr, nw, q, upass ? 1 : 0};
                    int segoff = kChunkHeader;
                    for (int w = 0; w < nw; ++w) {
                        hdr[4 + w] = widths[w];
                        hdr[4 + kMaxWarps + w] = segoff;
                        segoff += widths[w] * seg_stride(w, nr) * (vb + 4);
                    }
                    hdr[4 + 2 * kMaxWarps + 0] = segoff;                  // src
                    hdr[4 + 2 * kMaxWarps + 1] = segoff + 4 * npad;       // dst
                    hdr[4 + 2 * kMaxWarps + 2] = segoff + 8 * npad;       // dinv
                    std::memcpy(ch, hdr, kChunkHeader);
                    unsigned char *seg = ch + kChunkHeader;
                    int *src = nullptr;
                    int mindep = q;
                    for (int w = 0; w < nw; ++w) {
                        const int wd = widths[w];
                        const int ls = seg_stride(w, nr);
                        unsigned char *val = seg;
                        int *dep = reinterpret_cast<int *>(seg + (size_t)wd * ls * vb);
                        for (int lane = 0; lane < ls; ++lane) {
                            const int t = w * kWarpRows + lane;
                            if (t >= nr) {
                                // rows past the chunk: never read, keep them valid
                                for (int kk = 0; kk < wd; ++kk) {
                                    dep[(size_t)kk * ls + lane] = q;
                                    put_value(val, (size_t)kk * ls + lane, 0.0, vb);
                                }
                                continue;
                            }
                            const int i = pr.order[q + t];
                            const int e0 = upass ? B.diag[i] + 1 : F.rp[i];
                            const int len = row_len(upass, i);
                            if (len == 0 && wd > 0 && uniform_width == 0) {
                                // a row of level >= 2 always has a dependency
                                O.err = "internal: dependency-free row in a dependent level";
                                return;
                            }
                            for (int kk = 0; kk < wd; ++kk) {
                                // padding repeats the first dependency with value 0
                                // (a row without one -- level 1 of a uniform-width
                                // layout -- points at the chunk's first position:
                                // in the ring that slot holds a value of this
                                // apply or 0; from the global scratch the kernel
                                // does not read entries of value 0)
                                const int e = kk < len ? e0 + kk : e0;
                                const int d = len > 0 ? (upass ? posU : posL)[F.ci[e]] : q;
                                dep[(size_t)kk * ls + lane] = d;
                                put_value(val, (size_t)kk * ls + lane, kk < len ? F.va[e] : 0.0, vb);
                                mindep = std::min(mindep, d);
                            }
                        }
                        seg += (size_t)wd * ls * (vb + 4);
                    }
                    O.rows_per_chunk.push_back(nr);
                    for (int t = 0; t < nr; ++t) {
                        const int i = pr.order[q + t];
                        O.rm_start.push_back(upass ? B.diag[i] + 1 : F.rp[i]);
                        O.rm_len.push_back(row_len(upass, i));
                        O.rm_diag.push_back(upass ? B.diag[i] : -1);
                    }
                    src = reinterpret_cast<int *>(seg);
                    int *dst = src + npad;
                    unsigned char *dinv = reinterpret_cast<unsigned char *>(dst + npad);
                    for (int t = 0; t < nr; ++t) {
                        const int i = pr.order[q + t];
                        const int len = row_len(upass, i);
                        if (upass) {
                            src[t] = posL[i];
                            dst[t] = owned[i] ? B.rows[i] : -1;
                            put_value(dinv, t, 1.0 / F.va[B.diag[i]], vb);
                            O.alg += (4ll + vb) * len + vb /*y*/ + vb /*dinv*/ + 4 /*src*/ +
                                     4 /*dst*/ + (owned[i] ? vb : 0);
                        } else {
                            src[t] = B.rows[i];
                            O.alg += (4ll + vb) * len + vb /*r*/ + vb /*y*/ + 4 /*src*/;
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
        O.nchunksL = (int)O.chunks.size();
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
    P.chunk_row0.clear();
    P.rm_start.clear();
    P.rm_len.clear();
    P.rm_diag.clear();
    {
        int64_t ent0 = 0, r0 = 0;
        for (int b = 0; b < nb; ++b) {
            const BlockOut &O = outs[b];
            for (int nr : O.rows_per_chunk) {
                P.chunk_row0.push_back(r0);
                r0 += nr;
            }
            for (size_t q = 0; q < O.rm_start.size(); ++q) {
                P.rm_start.push_back((int)(ent0 + O.rm_start[q]));
                P.rm_len.push_back(O.rm_len[q]);
                P.rm_diag.push_back(O.rm_diag[q] < 0 ? -1 : (int)(ent0 + O.rm_diag[q]));
            }
            ent0 += (int64_t)Bs[b].F.ci.size();
        }
        P.chunk_row0.push_back(r0);
    }
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
        T.chunk_mid = T.chunk_begin + O.nchunksL;
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
