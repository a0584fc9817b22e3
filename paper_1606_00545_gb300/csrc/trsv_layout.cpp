// trsv_layout.cpp -- the chunk layout that the RAS/ILU(k) triangular-solve
// kernel streams (Sections 2.5-2.6, Eq. 11).
//
// Every RAS block's rows are solved level by level (Eq. 11): the L pass
// visits the levels of L_b, the U pass those of U_b.  A block may be split
// into a chain of P "parts" -- contiguous ranges of its local rows, each
// solved by one CTA of a thread-block cluster.  L_b is lower triangular in the
// block's local order, so in the L pass part p depends only on parts <= p;
// the layout admits a split only when every dependency stays inside a part or
// reaches the adjacent one (p - 1 in the L pass, p + 1 in the U pass).  A
// part solves its own rows of every level and pushes the values its
// neighbour reads into that neighbour's shared memory ("exports"; the
// neighbour's "imports"), so the CTAs of one block work on different rows of
// the same levels at once: the leading part (part 0 for L, the last part for
// U) never waits for the others, and a trailing part waits only when the
// values it imports are not there yet.
//
// Each part's program is a list of chunks -- rows of one level, at most one
// CTA's worth -- first of its L pass, then of its U pass.  Chunk headers carry
// two progress thresholds (the neighbours' completed-chunk counts this chunk
// must wait for): one for the values it imports, one so that its exports do
// not overwrite import slots the neighbour still has to read.  The planner
// runs every part's program against these thresholds on the host and accepts
// a split only if the chain cannot deadlock.
#include <algorithm>
#include <cstring>

#include "hec_setup.h"

#include "../../include/hecgpu.h"

namespace hec {

namespace {

constexpr int kWarpRows = 32;
constexpr int kMaxWarps = kThreads / kWarpRows;
// [0,16) counts, [16,48) widths, [48,80) segment offsets, [80,96) section
// offsets, [96,112) progress thresholds
constexpr int kChunkHeader = 112;
constexpr int kMaxParts = 8;
constexpr int kNarrowRow = 8; // rows the kernel holds in registers (flag bit 2)

constexpr int kFixedHeader = 32;

inline int r32(int x) { return (x + kWarpRows - 1) & ~(kWarpRows - 1); }

// Lane stride of warp w's segment: 32 for a full warp, the row count rounded
// up to 4 for the last, partial one.
inline int seg_stride(int w, int nrows)
{
    const int left = nrows - w * kWarpRows;
    return left >= kWarpRows ? kWarpRows : (left + 3) & ~3;
}

inline int pow2_at_least(int v, int lo)
{
    int p = lo;
    while (p < v)
        p <<= 1;
    return p;
}

// Chunk layout (offsets in bytes, every section 16-byte aligned):
//   [0, 16)    nrows, nwarps, first position, flags (bit 0: U pass, bit 1: exports,
//              bit 2: every warp segment at most kNarrowRow entries wide)
//   [16, 48)   width of every warp's segment (entries per row, uniform in the warp)
//   [48, 80)   byte offset of every warp's segment
//   [80, 96)   byte offsets of src, dst, dinv, exp
//   [96, 112)  need_prev, need_next (completed chunks of part p - 1 / p + 1 to
//              wait for), xend (exports of the pass up to this chunk), 0
//   per warp w < nwarps: val[width_w][stride_w] (value), dep[width_w][stride_w] (int32)
//   src[r32(nrows)] (int32); for U: dst[r32(nrows)] (int32), dinv[r32(nrows)]
//   (value); with exports: exp[r32(nrows)] (int32)
// A dependency is a shared-memory slot when the pass reads the ring: own
// values at position & (R - 1), imported ones at R + (import position & (RI - 1));
// otherwise the position in the block's global scratch.  exp[t] is row t's
// export position (its value goes to slot R + (exp & (RI - 1)) of the
// neighbour's ring), -1 when nobody imports it.
// Values are vb bytes: 8 (FP64 layout) or 4 (FP32 layout of the
// mixed-precision mode).  Row t of the chunk is handled by thread t.
size_t chunk_bytes(const std::vector<int> &widths, int nrows, bool upass, bool exp, int vb)
{
    size_t b = kChunkHeader;
    for (size_t w = 0; w < widths.size(); ++w)
        b += (size_t)widths[w] * seg_stride((int)w, nrows) * (vb + 4);
    b += 4 * (size_t)r32(nrows);
    if (upass)
        b += (4 + vb) * (size_t)r32(nrows);
    if (exp)
        b += 4 * (size_t)r32(nrows);
    return (b + 15) & ~(size_t)15;
}

// Fixed-slot format (layouts of one uniform width FW <= 8): every row's data
// sits at an offset that depends only on its thread, and a thread reads its
// row with 16-byte loads, so the kernel can copy the next chunk's row into
// registers without reading the header first.  VW = 16 / vb values per vector.
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass, bit 1:
//             exports, bit 2: narrow, bit 3: fixed-slot format, bit 4: the
//             blocks carry exp arrays)
//   [16, 32)  need_prev, need_next, FW, xend (exports of the pass so far)
//   per warp w < nwarps, a block of fixed_block() bytes, lane l = row 32w + l:
//     val: ceil(FW / VW) vectors of 32 lanes x 16 bytes (vector v of lane l:
//          entries v VW .. v VW + VW - 1); dep: ceil(FW / 4) vectors of 32
//          lanes x 4 int32; U: dinv[32] (value); src[32] (int32); U: dst[32]
//          (int32); with exp arrays: exp[32] (int32)
// Entries past FW in the last vector and rows past nrows in the last warp
// are padding (value 0, dependency = the chunk's padding slot, dst = exp = -1).
inline int fixed_vw(int vb) { return 16 / vb; }
inline int fixed_nv(int FW, int vb) { return (FW + fixed_vw(vb) - 1) / fixed_vw(vb); }
inline int fixed_nd(int FW) { return (FW + 3) / 4; }

size_t fixed_block(int FW, bool upass, bool exps, int vb)
{
    size_t b = (size_t)(fixed_nv(FW, vb) + fixed_nd(FW)) * 512 + 128;
    if (upass)
        b += (size_t)32 * vb + 128;
    if (exps)
        b += 128;
    return b;
}

size_t chunk_bytes_fixed(int FW, int nrows, bool upass, bool exps, int vb)
{
    return kFixedHeader + (size_t)((nrows + kWarpRows - 1) / kWarpRows) * fixed_block(FW, upass, exps, vb);
}

inline void put_value(unsigned char *base, size_t i, double v, int vb)
{
    if (vb == 8)
        reinterpret_cast<double *>(base)[i] = v;
    else
        reinterpret_cast<float *>(base)[i] = (float)v;
}

struct ChunkPlan {
    bool upass = false, exp = false;
    int q = 0, nr = 0;          // first position and row count in the part's pass order
    std::vector<int> widths;    // per warp
    int need_prev = 0, need_next = 0;
};

struct PassOrder {
    std::vector<int> order;     // local rows in level-major order
    std::vector<int> level_end; // end offsets into order, one per level
};

struct PartPlan {
    PassOrder L, U;
    std::vector<ChunkPlan> chunks; // the program: L chunks, then U chunks
    int nchunksL = 0;
    int spanL = 0, spanU = 0;      // own ring windows (positions)
    std::vector<int> expL, expU;   // exported rows by import position
};

struct BlockPlan {
    int nparts = 1;
    std::vector<char> owned, needL, needU;
    std::vector<int> part;            // part of every local row
    std::vector<int> posL, posU;      // position in its part's pass order (-1: not solved)
    std::vector<int> chunkL, chunkU;  // program chunk of every solved row
    std::vector<int> iposL, iposU;    // import position of exported rows (-1: not exported)
    std::vector<int> lastL, lastU;    // last importing chunk of exported rows
    std::vector<PartPlan> parts;
    std::string err;
};

inline int row_len(const BlockFactor &B, bool upass, int i)
{
    const HostCSR &F = B.F;
    return upass ? F.rp[i + 1] - B.diag[i] - 1 : B.diag[i] - F.rp[i];
}
inline int row_first(const BlockFactor &B, bool upass, int i)
{
    return upass ? B.diag[i] + 1 : B.F.rp[i];
}

// Rows a block must solve: the U solve needs the owned rows and,
// transitively, the rows they depend on through U (higher local indices);
// the L solve needs every row whose y the U solve reads and, transitively,
// their L dependencies.  The other rows cannot influence the owned part of
// the result and are left out of the device program.
void needed_rows(const BlockFactor &B, BlockPlan &bp)
{
    const HostCSR &F = B.F;
    const int nv = F.n;
    bp.owned.assign(nv, 0);
    bp.needL.assign(nv, 0);
    bp.needU.assign(nv, 0);
    for (int i = 0; i < nv; ++i)
        bp.owned[i] = (B.rows[i] >= B.own_lo && B.rows[i] < B.own_hi);
    for (int i = 0; i < nv; ++i) {
        bp.needU[i] |= bp.owned[i];
        if (bp.needU[i])
            for (int e = B.diag[i] + 1; e < F.rp[i + 1]; ++e)
                bp.needU[F.ci[e]] = 1;
    }
    for (int i = nv - 1; i >= 0; --i) {
        bp.needL[i] |= bp.needU[i];
        if (bp.needL[i])
            for (int e = F.rp[i]; e < B.diag[i]; ++e)
                bp.needL[F.ci[e]] = 1;
    }
}

// Split the needed rows into P contiguous ranges of about equal size;
// false if a dependency skips a part.
bool assign_parts(const BlockFactor &B, BlockPlan &bp, int P)
{
    const HostCSR &F = B.F;
    const int nv = F.n;
    int cnt = 0;
    for (int i = 0; i < nv; ++i)
        cnt += bp.needL[i];
    bp.part.assign(nv, 0);
    int seen = 0;
    for (int i = 0; i < nv; ++i) {
        bp.part[i] = cnt > 0 ? std::min(P - 1, (int)((int64_t)seen * P / cnt)) : 0;
        seen += bp.needL[i];
    }
    for (int i = 0; i < nv; ++i) {
        if (bp.needL[i])
            for (int e = F.rp[i]; e < B.diag[i]; ++e)
                if (bp.part[F.ci[e]] < bp.part[i] - 1)
                    return false;
        if (bp.needU[i])
            for (int e = B.diag[i] + 1; e < F.rp[i + 1]; ++e)
                if (bp.part[F.ci[e]] > bp.part[i] + 1)
                    return false;
    }
    return true;
}

// Level-major order of part p's rows in one pass; inside a level rows are
// independent and sorted longest first, so each warp's segment pads little.
void order_pass(const BlockFactor &B, BlockPlan &bp, int p, bool upass, PassOrder &po,
                std::vector<int> &pos)
{
    const std::vector<int> &ptr = upass ? B.lptrU : B.lptrL;
    const std::vector<int> &rows = upass ? B.lrowsU : B.lrowsL;
    const std::vector<char> &need = upass ? bp.needU : bp.needL;
    std::vector<int> lvl;
    po.order.clear();
    po.level_end.clear();
    for (size_t l = 0; l + 1 < ptr.size(); ++l) {
        lvl.clear();
        for (int q = ptr[l]; q < ptr[l + 1]; ++q)
            if (need[rows[q]] && bp.part[rows[q]] == p)
                lvl.push_back(rows[q]);
        std::stable_sort(lvl.begin(), lvl.end(), [&](int x, int y) {
            return row_len(B, upass, x) > row_len(B, upass, y);
        });
        for (int i : lvl) {
            pos[i] = (int)po.order.size();
            po.order.push_back(i);
        }
        if (!lvl.empty())
            po.level_end.push_back((int)po.order.size());
    }
}

// Greedy chunks of one pass: rows of one level, at most kThreads of them and
// one shared-memory stage of bytes; warp w takes rows 32w .. 32w+31.
bool chunk_pass(const BlockFactor &B, const BlockPlan &bp, bool upass, const PassOrder &po,
                const std::vector<int> &ipos, int stage_bytes, int vb, int uniform_width,
                bool exps, std::vector<ChunkPlan> &out)
{
    int start = 0;
    std::vector<int> widths;
    for (int end : po.level_end) {
        int q = start;
        while (q < end) {
            int q2 = q;
            bool exp = false;
            widths.clear();
            while (q2 < end && q2 - q < kThreads) {
                const int j = q2 - q, i = po.order[q2];
                if (j % kWarpRows == 0)
                    widths.push_back(uniform_width > 0 ? uniform_width : row_len(B, upass, i));
                const bool e2 = exp || ipos[i] >= 0;
                const size_t need = uniform_width > 0
                                        ? chunk_bytes_fixed(uniform_width, j + 1, upass, exps, vb)
                                        : chunk_bytes(widths, j + 1, upass, e2, vb);
                if (need > (size_t)stage_bytes) {
                    if (j % kWarpRows == 0)
                        widths.pop_back();
                    break;
                }
                exp = e2;
                ++q2;
            }
            if (q2 == q)
                return false;
            ChunkPlan c;
            c.upass = upass;
            c.exp = exp;
            c.q = q;
            c.nr = q2 - q;
            c.widths = widths;
            out.push_back(std::move(c));
            q = q2;
        }
        start = end;
    }
    (void)bp;
    return true;
}

// Plan block B with P parts: orders, chunks, exports, own ring windows.
bool plan_parts(const BlockFactor &B, BlockPlan &bp, int P, int stage_bytes, int vb,
                int uniform_width, bool exps)
{
    const HostCSR &F = B.F;
    const int nv = F.n;
    bp.nparts = P;
    bp.parts.assign(P, PartPlan());
    bp.posL.assign(nv, -1);
    bp.posU.assign(nv, -1);
    bp.chunkL.assign(nv, -1);
    bp.chunkU.assign(nv, -1);
    bp.iposL.assign(nv, -1);
    bp.iposU.assign(nv, -1);
    bp.lastL.assign(nv, -1);
    bp.lastU.assign(nv, -1);
    for (int p = 0; p < P; ++p) {
        order_pass(B, bp, p, false, bp.parts[p].L, bp.posL);
        order_pass(B, bp, p, true, bp.parts[p].U, bp.posU);
    }
    // exported rows: L values read by part p + 1, U values read by part p - 1
    std::vector<char> xL(nv, 0), xU(nv, 0);
    for (int i = 0; i < nv; ++i) {
        if (bp.needL[i])
            for (int e = F.rp[i]; e < B.diag[i]; ++e)
                if (bp.part[F.ci[e]] != bp.part[i])
                    xL[F.ci[e]] = 1;
        if (bp.needU[i])
            for (int e = B.diag[i] + 1; e < F.rp[i + 1]; ++e)
                if (bp.part[F.ci[e]] != bp.part[i])
                    xU[F.ci[e]] = 1;
    }
    for (int p = 0; p < P; ++p) {
        PartPlan &pp = bp.parts[p];
        for (int i : pp.L.order)
            if (xL[i]) {
                bp.iposL[i] = (int)pp.expL.size();
                pp.expL.push_back(i);
            }
        for (int i : pp.U.order)
            if (xU[i]) {
                bp.iposU[i] = (int)pp.expU.size();
                pp.expU.push_back(i);
            }
        if (!chunk_pass(B, bp, false, pp.L, bp.iposL, stage_bytes, vb, uniform_width, exps,
                        pp.chunks))
            return false;
        pp.nchunksL = (int)pp.chunks.size();
        if (!chunk_pass(B, bp, true, pp.U, bp.iposU, stage_bytes, vb, uniform_width, exps,
                        pp.chunks))
            return false;
        for (int c = 0; c < (int)pp.chunks.size(); ++c) {
            const ChunkPlan &ch = pp.chunks[c];
            const PassOrder &po = ch.upass ? pp.U : pp.L;
            std::vector<int> &chunk = ch.upass ? bp.chunkU : bp.chunkL;
            const std::vector<int> &pos = ch.upass ? bp.posU : bp.posL;
            int mindep = ch.q;
            for (int t = 0; t < ch.nr; ++t) {
                const int i = po.order[ch.q + t];
                chunk[i] = c;
                const int e0 = row_first(B, ch.upass, i), len = row_len(B, ch.upass, i);
                for (int e = e0; e < e0 + len; ++e)
                    if (bp.part[F.ci[e]] == p)
                        mindep = std::min(mindep, pos[F.ci[e]]);
            }
            int &span = ch.upass ? pp.spanU : pp.spanL;
            span = std::max(span, (ch.q + ch.nr) - mindep);
        }
    }
    // last chunk of the importing part that reads each exported row
    for (int p = 0; p < P; ++p) {
        const PartPlan &pp = bp.parts[p];
        for (int c = 0; c < (int)pp.chunks.size(); ++c) {
            const ChunkPlan &ch = pp.chunks[c];
            const PassOrder &po = ch.upass ? pp.U : pp.L;
            std::vector<int> &last = ch.upass ? bp.lastU : bp.lastL;
            for (int t = 0; t < ch.nr; ++t) {
                const int i = po.order[ch.q + t];
                const int e0 = row_first(B, ch.upass, i), len = row_len(B, ch.upass, i);
                for (int e = e0; e < e0 + len; ++e)
                    if (bp.part[F.ci[e]] != p)
                        last[F.ci[e]] = std::max(last[F.ci[e]], c);
            }
        }
    }
    return true;
}

// Progress thresholds of every chunk for an import ring of RI slots, then a
// host run of the parts against them, by the kernel's rule: true if every
// part's program can run to its end.  A part only waits for counters that
// never decrease, so if the most eager run finishes, every interleaving does.
bool set_thresholds(const BlockFactor &B, BlockPlan &bp, int RI)
{
    const HostCSR &F = B.F;
    const int P = bp.nparts;
    for (int p = 0; p < P; ++p) {
        PartPlan &pp = bp.parts[p];
        for (ChunkPlan &ch : pp.chunks) {
            const PassOrder &po = ch.upass ? pp.U : pp.L;
            ch.need_prev = ch.need_next = 0;
            for (int t = 0; t < ch.nr; ++t) {
                const int i = po.order[ch.q + t];
                const int e0 = row_first(B, ch.upass, i), len = row_len(B, ch.upass, i);
                // imports: the producing chunk of the neighbour has completed
                for (int e = e0; e < e0 + len; ++e) {
                    const int j = F.ci[e];
                    if (bp.part[j] == p)
                        continue;
                    if (ch.upass)
                        ch.need_next = std::max(ch.need_next, bp.chunkU[j] + 1);
                    else
                        ch.need_prev = std::max(ch.need_prev, bp.chunkL[j] + 1);
                }
                // exports: the slot's previous value has been read by its last reader
                const int ip = ch.upass ? bp.iposU[i] : bp.iposL[i];
                if (ip >= RI) {
                    const int old = (ch.upass ? pp.expU : pp.expL)[ip - RI];
                    if (ch.upass)
                        ch.need_prev = std::max(ch.need_prev, bp.lastU[old] + 1);
                    else
                        ch.need_next = std::max(ch.need_next, bp.lastL[old] + 1);
                }
            }
        }
    }
    // The kernel completes chunk k only after chunks k + 1 and k + 2 of the
    // same pass have been handed over too (the first is loaded, the second
    // confirmed, before chunk k's barrier), so completing k needs all three
    // chunks' thresholds met.
    std::vector<int> done(P, 0);
    auto met = [&](int p, const ChunkPlan &ch) {
        return ch.need_prev <= (p > 0 ? done[p - 1] : 0) &&
               ch.need_next <= (p + 1 < P ? done[p + 1] : 0);
    };
    for (bool moved = true; moved;) {
        moved = false;
        for (int p = 0; p < P; ++p) {
            const PartPlan &pp = bp.parts[p];
            const std::vector<ChunkPlan> &cs = pp.chunks;
            while (done[p] < (int)cs.size()) {
                const int k = done[p];
                const int pass_end = k < pp.nchunksL ? pp.nchunksL : (int)cs.size();
                bool ok = true;
                for (int j = k; j < std::min(k + 3, pass_end) && ok; ++j)
                    ok = met(p, cs[j]);
                if (!ok)
                    break;
                ++done[p];
                moved = true;
            }
        }
    }
    for (int p = 0; p < P; ++p)
        if (done[p] < (int)bp.parts[p].chunks.size())
            return false;
    return true;
}

bool all_ring(const BlockPlan &bp, int R)
{
    for (const PartPlan &pp : bp.parts)
        if (pp.spanL + 1 > R || pp.spanU + 1 > R)
            return false;
    return true;
}

struct BlockOut {
    std::vector<unsigned char> bytes;
    std::vector<std::vector<uint2>> chunks; // per part, offsets relative to this block
    std::vector<int> nchunksL, nL, nU;      // per part
    std::vector<int> ringL, ringU;          // per part
    std::vector<int> rows_per_chunk, rm_start, rm_len, rm_diag; // block-local entries
    int64_t alg = 0;
};

void emit_block(const BlockFactor &B, const BlockPlan &bp, int R, int RI, int vb,
                int uniform_width, bool exps, int P, BlockOut &O)
{
    const HostCSR &F = B.F;
    O.chunks.assign(P, {});
    O.nchunksL.assign(P, 0);
    O.nL.assign(P, 0);
    O.nU.assign(P, 0);
    O.ringL.assign(P, 1);
    O.ringU.assign(P, 1);
    for (int p = 0; p < bp.nparts; ++p) {
        const PartPlan &pp = bp.parts[p];
        O.nchunksL[p] = pp.nchunksL;
        O.nL[p] = (int)pp.L.order.size();
        O.nU[p] = (int)pp.U.order.size();
        O.ringL[p] = pp.spanL + 1 <= R;
        O.ringU[p] = pp.spanU + 1 <= R;
        bool xpass = false;
        int xcount = 0;
        for (const ChunkPlan &ch : pp.chunks) {
            const bool upass = ch.upass;
            const PassOrder &po = upass ? pp.U : pp.L;
            const std::vector<int> &pos = upass ? bp.posU : bp.posL;
            const std::vector<int> &ipos = upass ? bp.iposU : bp.iposL;
            const bool ring = upass ? O.ringU[p] : O.ringL[p];
            const int q = ch.q, nr = ch.nr, npad = r32(nr), nw = (int)ch.widths.size();
            // the slot (ring) or scratch position (global) a dependency is read from
            auto dep_of = [&](int j) {
                if (bp.part[j] != p)
                    return R + (ipos[j] & (RI - 1));
                return ring ? (pos[j] & (R - 1)) : pos[j];
            };
            const int pad_dep = ring ? (q & (R - 1)) : q;
            // per row: refill maps and algorithmic bytes
            auto account = [&](int i) {
                const int len = row_len(B, upass, i);
                O.rm_start.push_back(row_first(B, upass, i));
                O.rm_len.push_back(len);
                O.rm_diag.push_back(upass ? B.diag[i] : -1);
                if (upass)
                    O.alg += (4ll + vb) * len + vb /*y*/ + vb /*dinv*/ + 4 /*src*/ + 4 /*dst*/ +
                             (bp.owned[i] ? vb : 0);
                else
                    O.alg += (4ll + vb) * len + vb /*r*/ + vb /*y*/ + 4 /*src*/;
            };
            // exports of this pass up to and including this chunk (export
            // positions follow the pass's level-major order)
            auto export_end = [&]() {
                if (upass != xpass) {
                    xpass = upass;
                    xcount = 0;
                }
                for (int t = 0; t < nr; ++t)
                    if (ipos[po.order[q + t]] >= 0)
                        xcount = std::max(xcount, ipos[po.order[q + t]] + 1);
                return xcount;
            };
            if (uniform_width > 0) {
                const int FW = uniform_width;
                const size_t blk = fixed_block(FW, upass, exps, vb);
                const size_t bytes = chunk_bytes_fixed(FW, nr, upass, exps, vb);
                const size_t off = O.bytes.size();
                O.bytes.resize(off + bytes, 0);
                unsigned char *cb = O.bytes.data() + off;
                const int xend = export_end();
                const int hdr[kFixedHeader / 4] = {
                    nr, nw, q, (upass ? 1 : 0) | (ch.exp ? 2 : 0) | 4 | 8 | (exps ? 16 : 0),
                    ch.need_prev, ch.need_next, FW, xend};
                std::memcpy(cb, hdr, kFixedHeader);
                const int VW = fixed_vw(vb), NV = fixed_nv(FW, vb), ND = fixed_nd(FW);
                for (int w = 0; w < nw; ++w) {
                    unsigned char *base = cb + kFixedHeader + w * blk;
                    unsigned char *val = base;                          // [NV][32][VW]
                    int *dep = reinterpret_cast<int *>(base + NV * 512); // [ND][32][4]
                    size_t o = (size_t)(NV + ND) * 512;
                    unsigned char *dinv = base + o;
                    if (upass)
                        o += (size_t)32 * vb;
                    int *src = reinterpret_cast<int *>(base + o);
                    o += 128;
                    int *dst = reinterpret_cast<int *>(base + o);
                    if (upass)
                        o += 128;
                    int *exp = reinterpret_cast<int *>(base + o);
                    auto at_val = [&](int k, int lane) {
                        return (size_t)(k / VW) * 32 * VW + (size_t)lane * VW + k % VW;
                    };
                    auto at_dep = [&](int k, int lane) {
                        return (size_t)(k / 4) * 128 + (size_t)lane * 4 + k % 4;
                    };
                    for (int lane = 0; lane < kWarpRows; ++lane) {
                        const int t = w * kWarpRows + lane;
                        const int i = t < nr ? po.order[q + t] : -1;
                        const int e0 = i >= 0 ? row_first(B, upass, i) : 0;
                        const int len = i >= 0 ? row_len(B, upass, i) : 0;
                        for (int kk = 0; kk < NV * VW; ++kk) {
                            // padding repeats the first dependency with value 0 (a row
                            // without one, or a padding row, points at the padding slot)
                            const int e = kk < len ? e0 + kk : e0;
                            put_value(val, at_val(kk, lane), kk < len ? F.va[e] : 0.0, vb);
                        }
                        for (int kk = 0; kk < ND * 4; ++kk) {
                            const int e = kk < len ? e0 + kk : e0;
                            dep[at_dep(kk, lane)] = len > 0 ? dep_of(F.ci[e]) : pad_dep;
                        }
                        if (i < 0) { // padding rows: never used
                            src[lane] = 0;
                            if (upass) {
                                dst[lane] = -1;
                                put_value(dinv, lane, 0.0, vb);
                            }
                            if (exps)
                                exp[lane] = -1;
                            continue;
                        }
                        if (upass) {
                            src[lane] = bp.posL[i];
                            dst[lane] = bp.owned[i] ? B.rows[i] : -1;
                            put_value(dinv, lane, 1.0 / F.va[B.diag[i]], vb);
                        } else {
                            src[lane] = B.rows[i];
                        }
                        if (exps)
                            exp[lane] = ipos[i];
                        account(i);
                    }
                }
                O.rows_per_chunk.push_back(nr);
                O.chunks[p].push_back(make_uint2((unsigned)(off / 16), (unsigned)bytes));
                continue;
            }
            const size_t bytes = chunk_bytes(ch.widths, nr, upass, ch.exp, vb);
            const size_t off = O.bytes.size();
            O.bytes.resize(off + bytes, 0);
            unsigned char *cb = O.bytes.data() + off;
            const int widest = nw > 0 ? *std::max_element(ch.widths.begin(), ch.widths.end()) : 0;
            int hdr[kChunkHeader / 4] = {nr, nw, q,
                                         (upass ? 1 : 0) | (ch.exp ? 2 : 0) |
                                             (widest <= kNarrowRow ? 4 : 0)};
            int segoff = kChunkHeader;
            for (int w = 0; w < nw; ++w) {
                hdr[4 + w] = ch.widths[w];
                hdr[4 + kMaxWarps + w] = segoff;
                segoff += ch.widths[w] * seg_stride(w, nr) * (vb + 4);
            }
            const int src_off = segoff, dst_off = src_off + 4 * npad,
                      dinv_off = dst_off + 4 * npad,
                      exp_off = upass ? dinv_off + vb * npad : dst_off;
            hdr[4 + 2 * kMaxWarps + 0] = src_off;
            hdr[4 + 2 * kMaxWarps + 1] = upass ? dst_off : 0;
            hdr[4 + 2 * kMaxWarps + 2] = upass ? dinv_off : 0;
            hdr[4 + 2 * kMaxWarps + 3] = ch.exp ? exp_off : 0;
            hdr[24] = ch.need_prev;
            hdr[25] = ch.need_next;
            hdr[26] = export_end();
            std::memcpy(cb, hdr, kChunkHeader);
            unsigned char *seg = cb + kChunkHeader;
            for (int w = 0; w < nw; ++w) {
                const int wd = ch.widths[w], ls = seg_stride(w, nr);
                unsigned char *val = seg;
                int *dep = reinterpret_cast<int *>(seg + (size_t)wd * ls * vb);
                for (int lane = 0; lane < ls; ++lane) {
                    const int t = w * kWarpRows + lane;
                    if (t >= nr) { // rows past the chunk: never read, keep them valid
                        for (int kk = 0; kk < wd; ++kk) {
                            dep[(size_t)kk * ls + lane] = pad_dep;
                            put_value(val, (size_t)kk * ls + lane, 0.0, vb);
                        }
                        continue;
                    }
                    const int i = po.order[q + t];
                    const int e0 = row_first(B, upass, i), len = row_len(B, upass, i);
                    for (int kk = 0; kk < wd; ++kk) {
                        // padding repeats the first dependency with value 0 (a
                        // row without one -- level 1 of a uniform-width layout
                        // -- points at the chunk's first position: in the ring
                        // that slot holds a value of this apply or 0; from the
                        // global scratch the kernel skips entries of value 0)
                        const int e = kk < len ? e0 + kk : e0;
                        dep[(size_t)kk * ls + lane] = len > 0 ? dep_of(F.ci[e]) : pad_dep;
                        put_value(val, (size_t)kk * ls + lane, kk < len ? F.va[e] : 0.0, vb);
                    }
                }
                seg += (size_t)wd * ls * (vb + 4);
            }
            O.rows_per_chunk.push_back(nr);
            int *src = reinterpret_cast<int *>(cb + src_off);
            int *dst = reinterpret_cast<int *>(cb + dst_off);
            unsigned char *dinv = cb + dinv_off;
            int *exp = reinterpret_cast<int *>(cb + exp_off);
            for (int t = 0; t < nr; ++t) {
                const int i = po.order[q + t];
                account(i);
                if (upass) {
                    src[t] = bp.posL[i];
                    dst[t] = bp.owned[i] ? B.rows[i] : -1;
                    put_value(dinv, t, 1.0 / F.va[B.diag[i]], vb);
                } else {
                    src[t] = B.rows[i];
                }
                if (ch.exp)
                    exp[t] = ipos[i];
            }
            if (ch.exp)
                for (int t = nr; t < npad; ++t)
                    exp[t] = -1;
            O.chunks[p].push_back(make_uint2((unsigned)(off / 16), (unsigned)bytes));
        }
    }
}

// ------------------------------------------------------------------ resident format
// (k_trsv_res: the block's whole right-hand side stays in shared memory and is
// overwritten in place, so dependencies are local row slots; see k_trsv.cu)
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass, bit 3:
//             fixed slots, bit 5: resident format)
//   [16, 32)  the next chunk's byte offset in its group's stage and its warp
//             count (0, 0 for the last chunk), FW, 0
//   per warp w < NW (the kernel's solving warps: every chunk has the same
//   size, so the kernel finds chunk k of a group at k times that size), a
//   block of res_block() bytes, lane l = row 32w + l:
//     val: ceil(FW / VW) vectors of 32 lanes x 16 bytes; idx: ceil((FW + 1) /
//     8) vectors of 32 lanes x 8 uint16 (FW dependency slots, then the row's
//     own slot); dinv[32] (value; used by the U pass)
// Padding entries have value 0 and slot nv (which holds 0); padding rows and
// the warps past the chunk's rows have own slot nv.  Every group of G =
// kResGroupBytes / (chunk size) consecutive chunks of a block's program (at
// least one) is streamed by one bulk copy into one stage; flag bit 6 marks
// the last chunk of a group.
inline int res_ni(int FW) { return (FW + 1 + 7) / 8; }
constexpr size_t kResGroupBytes = 16384;

size_t res_block(int FW, int vb)
{
    return (size_t)(fixed_nv(FW, vb) + res_ni(FW)) * 512 + (size_t)32 * vb;
}

size_t chunk_bytes_res(int FW, int NW, int vb)
{
    return kFixedHeader + (size_t)NW * res_block(FW, vb);
}

struct ResOut {
    std::vector<unsigned char> bytes;
    std::vector<uint2> chunks; // offsets relative to this block
    std::vector<uint2> groups; // the same for the groups of consecutive chunks
    int nchunksL = 0, nL = 0, nU = 0, own0 = 0, own1 = 0;
    std::vector<int> rows_per_chunk, rm_start, rm_len, rm_diag;
    size_t largest = 0; // bytes of the largest group
    int group = 1;      // chunks per group
    int64_t alg = 0;
};

void emit_resident(const BlockFactor &B, int FW, int vb, int NW, ResOut &O)
{
    const HostCSR &F = B.F;
    const int nv = F.n;
    BlockPlan bp;
    needed_rows(B, bp);
    bp.part.assign(nv, 0);
    bp.posL.assign(nv, -1);
    bp.posU.assign(nv, -1);
    PassOrder po[2];
    order_pass(B, bp, 0, false, po[0], bp.posL);
    order_pass(B, bp, 0, true, po[1], bp.posU);
    O.nL = (int)po[0].order.size();
    O.nU = (int)po[1].order.size();
    O.own0 = (int)(std::lower_bound(B.rows.begin(), B.rows.end(), B.own_lo) - B.rows.begin());
    O.own1 = (int)(std::lower_bound(B.rows.begin(), B.rows.end(), B.own_hi) - B.rows.begin());
    const int VW = fixed_vw(vb), NV = fixed_nv(FW, vb), NI = res_ni(FW);
    for (int pass = 0; pass < 2; ++pass) {
        const bool upass = pass == 1;
        const PassOrder &P = po[pass];
        const size_t blk = res_block(FW, vb);
        int start = 0;
        for (int end : P.level_end) {
            for (int q = start; q < end; q += NW * kWarpRows) {
                const int nr = std::min(NW * kWarpRows, end - q);
                const int nw = (nr + kWarpRows - 1) / kWarpRows;
                const size_t bytes = chunk_bytes_res(FW, NW, vb);
                const size_t off = O.bytes.size();
                O.bytes.resize(off + bytes, 0);
                O.largest = std::max(O.largest, bytes);
                unsigned char *cb = O.bytes.data() + off;
                const int hdr[kFixedHeader / 4] = {nr, nw, q, (upass ? 1 : 0) | 8 | 32, 0, 0, FW, 0};
                std::memcpy(cb, hdr, kFixedHeader);
                for (int w = 0; w < NW; ++w) {
                    unsigned char *base = cb + kFixedHeader + w * blk;
                    uint16_t *idx = reinterpret_cast<uint16_t *>(base + (size_t)NV * 512);
                    unsigned char *dinv = base + (size_t)(NV + NI) * 512;
                    auto at_val = [&](int k, int lane) {
                        return (size_t)(k / VW) * 32 * VW + (size_t)lane * VW + k % VW;
                    };
                    auto at_idx = [&](int k, int lane) {
                        return (size_t)(k / 8) * 256 + (size_t)lane * 8 + k % 8;
                    };
                    for (int lane = 0; lane < kWarpRows; ++lane) {
                        const int t = w * kWarpRows + lane;
                        const int i = t < nr ? P.order[q + t] : -1;
                        const int e0 = i >= 0 ? row_first(B, upass, i) : 0;
                        const int len = i >= 0 ? row_len(B, upass, i) : 0;
                        for (int k = 0; k < NV * VW; ++k)
                            put_value(base, at_val(k, lane), k < len ? F.va[e0 + k] : 0.0, vb);
                        for (int k = 0; k < NI * 8; ++k)
                            idx[at_idx(k, lane)] = (uint16_t)(k < len ? F.ci[e0 + k] : nv);
                        idx[at_idx(FW, lane)] = (uint16_t)(i >= 0 ? i : nv);
                        put_value(dinv, lane, upass && i >= 0 ? 1.0 / F.va[B.diag[i]] : 0.0, vb);
                        if (i < 0)
                            continue;
                        O.rm_start.push_back(e0);
                        O.rm_len.push_back(len);
                        O.rm_diag.push_back(upass ? B.diag[i] : -1);
                        if (upass)
                            O.alg += (4ll + vb) * len + vb /*y*/ + vb /*dinv*/ + 4 /*src*/ +
                                     4 /*dst*/ + (bp.owned[i] ? vb : 0);
                        else
                            O.alg += (4ll + vb) * len + vb /*r*/ + vb /*y*/ + 4 /*src*/;
                    }
                }
                O.rows_per_chunk.push_back(nr);
                O.chunks.push_back(make_uint2((unsigned)(off / 16), (unsigned)bytes));
            }
            start = end;
        }
        if (!upass)
            O.nchunksL = (int)O.chunks.size();
    }
    // groups of G consecutive chunks, one bulk copy each
    const size_t cbytes = chunk_bytes_res(FW, NW, vb);
    O.group = std::max<int>(1, (int)(kResGroupBytes / cbytes));
    const int nch = (int)O.chunks.size();
    for (int g0 = 0; g0 < nch; g0 += O.group) {
        const int g1 = std::min(nch, g0 + O.group);
        O.groups.push_back(make_uint2(O.chunks[g0].x, (unsigned)((size_t)(g1 - g0) * cbytes)));
        reinterpret_cast<int *>(O.bytes.data() + (size_t)O.chunks[g1 - 1].x * 16)[3] |= 64;
    }
    // every chunk names the next one's byte offset in its group's stage and
    // its warp count, so the kernel loads it without waiting for its header
    size_t gstart = 0;
    for (size_t c = 0; c < O.chunks.size(); ++c) {
        int *h = reinterpret_cast<int *>(O.bytes.data() + (size_t)O.chunks[c].x * 16);
        const size_t end = (size_t)O.chunks[c].x * 16 + O.chunks[c].y;
        if (h[3] & 64)
            gstart = end; // the next chunk opens a group
        if (c + 1 < O.chunks.size()) {
            const int *hn = reinterpret_cast<const int *>(O.bytes.data() +
                                                          (size_t)O.chunks[c + 1].x * 16);
            h[4] = (int)((size_t)O.chunks[c + 1].x * 16 - gstart);
            h[5] = hn[1];
        }
    }
    O.largest = (size_t)O.group * cbytes;
}

} // namespace

int trsv_resident_width(int longest_row)
{
    for (int w : {2, 3, 4, 6, 8})
        if (longest_row <= w)
            return w;
    return 0;
}

int pack_trsv_resident(const std::vector<BlockFactor> &Bs, int width, int vb, TrsvPack &P,
                       std::string &msg)
{
    if ((vb != 8 && vb != 4) || trsv_resident_width(width) != width) {
        msg = "resident layout: value size 8 or 4 and width 2, 3, 4, 6 or 8";
        return HEC_ERR_INVALID;
    }
    const int nb = (int)Bs.size();
    for (const BlockFactor &B : Bs)
        if (B.F.n >= 65535) {
            msg = "resident layout: a block has 65535 rows or more";
            return HEC_ERR_INVALID;
        }
    // solving warps: enough for the widest level (wider levels take several
    // chunks of 8 warps)
    int widest = 1;
    for (const BlockFactor &B : Bs) {
        for (size_t l = 0; l + 1 < B.lptrL.size(); ++l)
            widest = std::max(widest, B.lptrL[l + 1] - B.lptrL[l]);
        for (size_t l = 0; l + 1 < B.lptrU.size(); ++l)
            widest = std::max(widest, B.lptrU[l + 1] - B.lptrU[l]);
    }
    const int NW = widest <= 2 * kWarpRows ? 2 : widest <= 4 * kWarpRows ? 4 : 8;
    std::vector<ResOut> outs(nb);
    parallel_for(nb, [&](int b) { emit_resident(Bs[b], width, vb, NW, outs[b]); });
    P = TrsvPack();
    P.resident = 1;
    P.res_warps = NW;
    P.parts = 1;
    P.ring_slots = 32;
    size_t total = 0, largest = 16;
    for (const ResOut &O : outs) {
        total += O.bytes.size();
        largest = std::max(largest, O.largest);
    }
    if (total / 16 > 0xffffffffull) {
        msg = "factor layout exceeds 64 GiB";
        return HEC_ERR_INVALID;
    }
    P.stage_bytes = (int)((largest + 127) & ~(size_t)127);
    P.res_group = nb > 0 ? outs[0].group : 1;
    P.pack.resize(total);
    P.blocks.assign(nb, TrsvBlock());
    int64_t ent0 = 0, r0 = 0;
    size_t off = 0;
    for (int b = 0; b < nb; ++b) {
        const ResOut &O = outs[b];
        TrsvBlock &T = P.blocks[b];
        T.chunk_begin = (int)P.chunks.size();
        for (const uint2 &c : O.chunks)
            P.chunks.push_back(make_uint2((unsigned)(c.x + off / 16), c.y));
        T.chunk_end = (int)P.chunks.size();
        T.chunk_mid = T.chunk_begin + O.nchunksL;
        T.links = 0;
        T.ring_L = T.ring_U = 1;
        T.yoff = (int64_t)P.vrows.size();
        T.zoff = (int64_t)P.groups.size();
        T.ngroups = (int)O.groups.size();
        for (const uint2 &g : O.groups)
            P.groups.push_back(make_uint2((unsigned)(g.x + off / 16), g.y));
        T.nv = Bs[b].F.n;
        T.own0 = O.own0;
        T.own1 = O.own1;
        P.vrows.insert(P.vrows.end(), Bs[b].rows.begin(), Bs[b].rows.end());
        P.res_slots = std::max(P.res_slots, T.nv + 1);
        P.rows_L += O.nL;
        P.rows_U += O.nU;
        for (int nr : O.rows_per_chunk) {
            P.chunk_row0.push_back(r0);
            r0 += nr;
        }
        for (size_t k = 0; k < O.rm_start.size(); ++k) {
            P.rm_start.push_back((int)(ent0 + O.rm_start[k]));
            P.rm_len.push_back(O.rm_len[k]);
            P.rm_diag.push_back(O.rm_diag[k] < 0 ? -1 : (int)(ent0 + O.rm_diag[k]));
        }
        ent0 += (int64_t)Bs[b].F.ci.size();
        std::memcpy(P.pack.data() + off, O.bytes.data(), O.bytes.size());
        off += O.bytes.size();
        P.alg_bytes += O.alg;
    }
    P.chunk_row0.push_back(r0);
    return HEC_OK;
}

int max_factor_width(const std::vector<BlockFactor> &Bs, bool upass)
{
    int w = 0;
    for (const BlockFactor &B : Bs)
        for (int i = 0; i < B.F.n; ++i)
            w = std::max(w, row_len(B, upass, i));
    return w;
}

int trsv_auto_parts(const std::vector<BlockFactor> &Bs, int sm_count, int rows_per_part)
{
    // rows per level of the widest block (L pass, all rows)
    double per_level = 0;
    for (const BlockFactor &B : Bs)
        if (B.nlevL > 0)
            per_level = std::max(per_level, (double)B.F.n / B.nlevL);
    int P = 1;
    while (2 * P <= kMaxParts && (int64_t)Bs.size() * 2 * P <= sm_count &&
           per_level / P > rows_per_part)
        P *= 2;
    return P;
}

int pack_trsv(const std::vector<BlockFactor> &Bs, int n, int stage_bytes, int max_ring, int vb,
              TrsvPack &P, std::string &msg, int uniform_width, int parts)
{
    (void)n;
    if (vb != 8 && vb != 4) {
        msg = "value size must be 8 or 4 bytes";
        return HEC_ERR_INVALID;
    }
    if (parts < 1 || parts > kMaxParts || (parts & (parts - 1)) != 0) {
        msg = "parts must be 1, 2, 4 or 8";
        return HEC_ERR_INVALID;
    }
    const int nb = (int)Bs.size();
    // fixed-slot chunks carry export slots whenever blocks may be split, and
    // a stage holds the largest one (the kernel reads every warp's slots)
    const bool exps = parts > 1;
    if (uniform_width > 0) {
        if (uniform_width > kNarrowRow) {
            msg = "uniform width above 8";
            return HEC_ERR_INVALID;
        }
        const size_t most = chunk_bytes_fixed(uniform_width, kThreads, true, exps, vb);
        stage_bytes = std::max<int>(stage_bytes, (int)((most + 127) & ~(size_t)127));
    }
    std::vector<BlockPlan> plans(nb);
    std::vector<int> want(nb, parts);
    std::vector<char> failed(nb, 0);
    // plan every block with the parts it may have, halving where a split is
    // not admissible (a dependency skips a part, or a pass does not fit one
    // shared-memory stage)
    auto plan = [&](int b) {
        const BlockFactor &B = Bs[b];
        BlockPlan &bp = plans[b];
        if (bp.owned.empty())
            needed_rows(B, bp);
        for (int p = want[b]; p >= 1; p /= 2) {
            if (p > 1 && !assign_parts(B, bp, p))
                continue;
            if (p == 1)
                bp.part.assign(B.F.n, 0);
            if (plan_parts(B, bp, p, stage_bytes, vb, uniform_width, exps)) {
                want[b] = p;
                return;
            }
            if (p == 1)
                break;
        }
        failed[b] = 1;
    };
    parallel_for(nb, plan);
    for (int b = 0; b < nb; ++b)
        if (failed[b]) {
            msg = "a factor row is too long for one shared-memory stage";
            return HEC_ERR_INVALID;
        }
    // own ring: the largest window that fits (power of two); a split block
    // must read every pass from the ring, else it is planned again with
    // fewer parts.  Import ring: the smallest size for which every split
    // block's chain runs through, doubled for slack.
    int R = 32, RI = 0;
    for (;;) {
        R = 32;
        for (const BlockPlan &bp : plans)
            for (const PartPlan &pp : bp.parts)
                for (int s : {pp.spanL, pp.spanU})
                    if (pow2_at_least(s + 1, 32) <= max_ring)
                        R = std::max(R, pow2_at_least(s + 1, 32));
        std::vector<int> redo;
        for (int b = 0; b < nb; ++b)
            if (plans[b].nparts > 1 && !all_ring(plans[b], R))
                redo.push_back(b);
        if (redo.empty()) {
            bool any_split = false;
            for (const BlockPlan &bp : plans)
                any_split |= bp.nparts > 1;
            if (!any_split) {
                RI = 0;
                break;
            }
            auto run_all = [&](int ri, std::vector<char> &ok) {
                ok.assign(nb, 1);
                parallel_for(nb, [&](int b) {
                    if (plans[b].nparts > 1)
                        ok[b] = set_thresholds(Bs[b], plans[b], ri) ? 1 : 0;
                });
                return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
            };
            std::vector<char> ok;
            int found = 0;
            for (int ri = 256; ri <= max_ring && !found; ri *= 2)
                if (run_all(ri, ok))
                    found = ri;
            if (found) {
                // twice the smallest size, for slack between the parts, if it runs too
                RI = (2 * found <= max_ring && run_all(2 * found, ok)) ? 2 * found : found;
                run_all(RI, ok); // the thresholds of the size kept
                break;
            }
            for (int b = 0; b < nb; ++b) // still stuck at the largest size
                if (!ok[b])
                    redo.push_back(b);
        }
        for (int b : redo) {
            want[b] = plans[b].nparts / 2;
            plan(b);
            if (failed[b]) {
                msg = "a factor row is too long for one shared-memory stage";
                return HEC_ERR_INVALID;
            }
        }
    }
    int nparts = 1;
    for (const BlockPlan &bp : plans)
        nparts = std::max(nparts, bp.nparts);
    std::vector<BlockOut> outs(nb);
    parallel_for(nb, [&](int b) {
        emit_block(Bs[b], plans[b], R, std::max(RI, 1), vb, uniform_width, exps, nparts, outs[b]);
    });

    P.pack.clear();
    P.chunks.clear();
    P.parts = nparts;
    P.stage_bytes = stage_bytes;
    P.exp_arrays = exps && uniform_width > 0 ? 1 : 0;
    P.ring_slots = R;
    P.import_slots = RI;
    P.blocks.assign((size_t)nb * nparts, TrsvBlock());
    P.ysz = P.zsz = 0;
    P.alg_bytes = 0;
    P.rows_L = P.rows_U = 0;
    size_t total = 0;
    for (auto &O : outs)
        total += O.bytes.size();
    if (total / 16 > 0xffffffffull) {
        msg = "factor layout exceeds 64 GiB";
        return HEC_ERR_INVALID;
    }
    P.pack.resize(total);
    P.chunk_row0.clear();
    P.rm_start.clear();
    P.rm_len.clear();
    P.rm_diag.clear();
    int64_t ent0 = 0, r0 = 0;
    size_t off = 0;
    int64_t yoff = 0, zoff = 0;
    bool any_global_u = false;
    for (int b = 0; b < nb; ++b) {
        BlockOut &O = outs[b];
        // the row maps follow the chunks: parts in order, each L then U
        for (int p = 0; p < nparts; ++p) {
            TrsvBlock &T = P.blocks[(size_t)b * nparts + p];
            T.chunk_begin = (int)P.chunks.size();
            for (const uint2 &c : O.chunks[p])
                P.chunks.push_back(make_uint2((unsigned)(c.x + off / 16), c.y));
            T.chunk_end = (int)P.chunks.size();
            T.chunk_mid = T.chunk_begin + O.nchunksL[p];
            T.links = (p > 0 && p < plans[b].nparts ? 1 : 0) |
                      (p + 1 < plans[b].nparts ? 2 : 0);
            T.ring_L = O.ringL[p];
            T.ring_U = O.ringU[p];
            T.yoff = yoff;
            yoff += O.nL[p];
            T.zoff = zoff;
            if (!T.ring_U) {
                zoff += O.nU[p];
                any_global_u = true;
            }
            P.rows_L += O.nL[p];
            P.rows_U += O.nU[p];
        }
        for (int nr : O.rows_per_chunk) {
            P.chunk_row0.push_back(r0);
            r0 += nr;
        }
        for (size_t k = 0; k < O.rm_start.size(); ++k) {
            P.rm_start.push_back((int)(ent0 + O.rm_start[k]));
            P.rm_len.push_back(O.rm_len[k]);
            P.rm_diag.push_back(O.rm_diag[k] < 0 ? -1 : (int)(ent0 + O.rm_diag[k]));
        }
        ent0 += (int64_t)Bs[b].F.ci.size();
        std::memcpy(P.pack.data() + off, O.bytes.data(), O.bytes.size());
        off += O.bytes.size();
        P.alg_bytes += O.alg;
    }
    P.chunk_row0.push_back(r0);
    P.ysz = yoff;
    P.zsz = any_global_u ? zoff : 0;
    return HEC_OK;
}

} // namespace hec
