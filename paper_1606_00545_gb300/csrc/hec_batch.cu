// hec_batch.cu -- host side of the batched solver (batch.cuh, k_batch.cu):
// per-system setup (ILU(k) and level sets, Sections 2.4-2.6), the device
// layout (HEC slab and tail per system, Section 2.1; level-ordered factor
// chunks), the autotuner, and the batched entry points of include/hecgpu.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/hecgpu.h"
#include "batch.cuh"
#include "hec_setup.h"
#include "runtime.h"

using namespace hec;

namespace {

constexpr long long kBatchSpin = 1ll << 24;

struct SysHost {
    HostCSR A;      // natural order, local column indices
    BlockFactor F;  // ILU(k) factor of A and the level sets of L and U
};

// One system's share of the device layout, before concatenation.
struct SysLayout {
    int K = 0, ld = 0;
    std::vector<int> rop, pos, upos;  // row of position; position / U position of row
    std::vector<int> ell_col;
    std::vector<double> ell_val;
    std::vector<int> tail_rows;
    std::vector<long long> tail_ptr;  // local offsets, ntail + 1
    std::vector<int> tail_col;
    std::vector<double> tail_val;
    int need = 0;  // dependency window (positions) of the triangular passes
    double cost = 0.0;
};

// Chunks of one triangular pass of one system: (first position, rows, level).
struct ChunkPlan {
    int first, nrows, width;
};

struct FacArena {
    bool built = false;
    int ent_bytes = 16;
    std::vector<int> chL, chU;  // per system: first chunk of the L / U pass
    DevBuf d_chunks, d_fac;
    int64_t bytes = 0;
};

} // namespace

struct hec_batch_s {
    int nsys = 0;
    int64_t rows = 0, nnz = 0, factor_nnz = 0;
    int max_n = 0;
    int ilu_k = -1;
    hec_batch_config_t cfg{};
    std::vector<SysHost> sys;
    std::vector<int64_t> sys_ptr;
    // layout
    bool layout_ok = false;
    std::vector<SysLayout> lay;
    std::vector<ChunkPlan> plan;          // all chunks, systems in order, L then U
    std::vector<int> planL, planU, nplanL, nplanU;
    int ring_slots = 32;
    std::vector<BatchSys> host_sys;
    DevBuf d_sys, d_order, d_ell_col, d_ell_val64, d_ell_val32, d_tail_rows, d_tail_ptr,
        d_tail_col, d_tail_val64, d_tail_val32, d_rop;
    FacArena fac[2];  // [0] FP32 values, [1] FP64 values
    // solve scratch
    DevBuf ws, queue, err, res;
    int64_t device_bytes() const
    {
        int64_t t = 0;
        for (const DevBuf *d : {&d_sys, &d_order, &d_ell_col, &d_ell_val64, &d_ell_val32,
                                &d_tail_rows, &d_tail_ptr, &d_tail_col, &d_tail_val64,
                                &d_tail_val32, &d_rop, &ws, &queue, &err, &res})
            t += (int64_t)d->bytes;
        for (const FacArena &f : fac)
            t += (int64_t)(f.d_chunks.bytes + f.d_fac.bytes);
        return t;
    }
};

namespace {

int r4(int x) { return (x + 3) & ~3; }
int64_t r16(int64_t x) { return (x + 15) & ~(int64_t)15; }

int check_config(const hec_batch_config_t &c)
{
    if (c.threads != 0 && c.threads != 128 && c.threads != 256 && c.threads != 512)
        return fail(HEC_ERR_INVALID, "threads must be 128, 256 or 512");
    if (c.ctas_per_sm < 0 || c.ell_width < 0 || c.nstages < 0 || c.nstages > 16)
        return fail(HEC_ERR_INVALID, "bad batch configuration");
    return HEC_OK;
}

// ------------------------------------------------------------------ layout
// Positions, HEC slab and tail, and dependency window of system s.
void layout_system(const hec_batch_s *B, int s, SysLayout &L)
{
    const SysHost &S = B->sys[s];
    const HostCSR &A = S.A;
    const int n = A.n;
    const bool fac = B->ilu_k >= 0;
    L.rop.resize(n);
    L.pos.resize(n);
    L.upos.assign(n, 0);
    if (fac) {
        L.rop = S.F.lrowsL;  // level order of L, rows ascending within a level
        for (int p = 0; p < n; ++p)
            L.upos[S.F.lrowsU[p]] = p;
    } else {
        std::iota(L.rop.begin(), L.rop.end(), 0);
    }
    for (int p = 0; p < n; ++p)
        L.pos[L.rop[p]] = p;
    // HEC: rows with at most K entries in the slab, longer rows whole in the tail
    L.K = B->cfg.ell_width > 0 ? B->cfg.ell_width : ell_width_auto(A);
    L.ld = (n + 31) & ~31;
    L.ell_col.assign((size_t)L.K * L.ld, 0);
    L.ell_val.assign((size_t)L.K * L.ld, 0.0);
    L.tail_ptr.assign(1, 0);
    for (int p = 0; p < L.ld; ++p)
        for (int k = 0; k < L.K; ++k)
            L.ell_col[(size_t)k * L.ld + p] = p < n ? p : 0;
    for (int p = 0; p < n; ++p) {
        const int r = L.rop[p];
        const int len = A.rp[r + 1] - A.rp[r];
        if (len <= L.K) {
            for (int e = A.rp[r], k = 0; e < A.rp[r + 1]; ++e, ++k) {
                L.ell_col[(size_t)k * L.ld + p] = L.pos[A.ci[e]];
                L.ell_val[(size_t)k * L.ld + p] = A.va[e];
            }
        } else {
            L.ell_col[p] = -1;
            L.tail_rows.push_back(p);
            for (int e = A.rp[r]; e < A.rp[r + 1]; ++e) {
                L.tail_col.push_back(L.pos[A.ci[e]]);
                L.tail_val.push_back(A.va[e]);
            }
            L.tail_ptr.push_back((long long)L.tail_col.size());
        }
    }
    // dependency window: a level's rows read positions >= end_of_level - need
    L.need = 0;
    if (fac) {
        const BlockFactor &F = S.F;
        for (int l = 0; l < F.nlevL; ++l) {
            const int a = F.lptrL[l], b = F.lptrL[l + 1];
            int lo = a;
            for (int p = a; p < b; ++p) {
                const int r = L.rop[p];
                for (int e = F.F.rp[r]; e < F.diag[r]; ++e)
                    lo = std::min(lo, L.pos[F.F.ci[e]]);
            }
            L.need = std::max(L.need, b - lo);
        }
        for (int l = 0; l < F.nlevU; ++l) {
            const int a = F.lptrU[l], b = F.lptrU[l + 1];
            int lo = a;
            for (int q = a; q < b; ++q) {
                const int r = F.lrowsU[q];
                for (int e = F.diag[r] + 1; e < F.F.rp[r + 1]; ++e)
                    lo = std::min(lo, L.upos[F.F.ci[e]]);
            }
            L.need = std::max(L.need, b - lo);
        }
    }
    const double nnzf = fac ? (double)S.F.F.ci.size() : 0.0;
    const double depth = fac ? (double)(S.F.nlevL + S.F.nlevU) : std::sqrt((double)n);
    L.cost = ((double)A.ci.size() + nnzf + 40.0 * n) * depth;
}

// Chunks of the L and U passes of system s.
void plan_system(const hec_batch_s *B, int s, std::vector<ChunkPlan> &L, std::vector<ChunkPlan> &U)
{
    const BlockFactor &F = B->sys[s].F;
    const SysLayout &Ly = B->lay[s];
    auto add = [](std::vector<ChunkPlan> &out, int a, int b, const std::function<int(int)> &width) {
        for (int c = a; c < b; c += kBatchChunkRows) {
            ChunkPlan p{c, std::min(kBatchChunkRows, b - c), 0};
            for (int q = p.first; q < p.first + p.nrows; ++q)
                p.width = std::max(p.width, width(q));
            out.push_back(p);
        }
    };
    for (int l = 0; l < F.nlevL; ++l)
        add(L, F.lptrL[l], F.lptrL[l + 1], [&](int p) {
            const int r = Ly.rop[p];
            return F.diag[r] - F.F.rp[r];
        });
    for (int l = 0; l < F.nlevU; ++l)
        add(U, F.lptrU[l], F.lptrU[l + 1], [&](int q) {
            const int r = F.lrowsU[q];
            return F.F.rp[r + 1] - F.diag[r] - 1;
        });
}

int64_t chunk_bytes(const ChunkPlan &c, bool upass, int vb)
{
    const int st = r4(c.nrows);
    return r16(16 + 4ll * st * (1 + c.width) + (int64_t)vb * st * (c.width + (upass ? 1 : 0)));
}

// Writes the block of chunk c of system s at dst.
void fill_chunk(const hec_batch_s *B, int s, const ChunkPlan &c, bool upass, int vb,
                unsigned char *dst)
{
    const BlockFactor &F = B->sys[s].F;
    const SysLayout &Ly = B->lay[s];
    const int st = r4(c.nrows), W = c.width, mask = B->ring_slots - 1, zero = B->ring_slots;
    int *hdr = reinterpret_cast<int *>(dst);
    hdr[0] = c.nrows;
    hdr[1] = W;
    hdr[2] = c.first;
    hdr[3] = upass ? 1 : 0;
    int *dsti = hdr + 4;
    int *dep = dsti + st;
    unsigned char *valp = reinterpret_cast<unsigned char *>(dep + (size_t)W * st);
    auto put = [&](unsigned char *base, size_t idx, double v) {
        if (vb == 8)
            reinterpret_cast<double *>(base)[idx] = v;
        else
            reinterpret_cast<float *>(base)[idx] = (float)v;
    };
    for (int i = 0; i < st; ++i) {
        dsti[i] = 0;
        for (int k = 0; k < W; ++k) {
            dep[(size_t)k * st + i] = zero;
            put(valp, (size_t)k * st + i, 0.0);
        }
        if (upass)
            put(valp, (size_t)W * st + i, 0.0);
    }
    for (int i = 0; i < c.nrows; ++i) {
        const int q = c.first + i;
        if (!upass) {
            const int r = Ly.rop[q];
            dsti[i] = Ly.upos[r];
            int k = 0;
            for (int e = F.F.rp[r]; e < F.diag[r]; ++e, ++k) {
                dep[(size_t)k * st + i] = Ly.pos[F.F.ci[e]] & mask;
                put(valp, (size_t)k * st + i, F.F.va[e]);
            }
        } else {
            const int r = F.lrowsU[q];
            dsti[i] = Ly.pos[r];
            int k = 0;
            for (int e = F.diag[r] + 1; e < F.F.rp[r + 1]; ++e, ++k) {
                dep[(size_t)k * st + i] = Ly.upos[F.F.ci[e]] & mask;
                put(valp, (size_t)k * st + i, F.F.va[e]);
            }
            put(valp, (size_t)W * st + i, 1.0 / F.F.va[F.diag[r]]);
        }
    }
}

// HEC slabs, tails, positions and system descriptors (value-type independent).
int build_layout(hec_batch_s *B, cudaStream_t st)
{
    if (B->layout_ok)
        return HEC_OK;
    const int ns = B->nsys;
    B->lay.assign(ns, SysLayout());
    parallel_for(ns, [&](int s) { layout_system(B, s, B->lay[s]); });
    int need = 0;
    for (const SysLayout &L : B->lay)
        need = std::max(need, L.need);
    int R = 32;
    while (R < need)
        R <<= 1;
    B->ring_slots = R;
    // chunk plans
    std::vector<std::vector<ChunkPlan>> pl(ns), pu(ns);
    if (B->ilu_k >= 0)
        parallel_for(ns, [&](int s) { plan_system(B, s, pl[s], pu[s]); });
    B->plan.clear();
    B->planL.assign(ns, 0);
    B->planU.assign(ns, 0);
    B->nplanL.assign(ns, 0);
    B->nplanU.assign(ns, 0);
    for (int s = 0; s < ns; ++s) {
        B->planL[s] = (int)B->plan.size();
        B->nplanL[s] = (int)pl[s].size();
        B->plan.insert(B->plan.end(), pl[s].begin(), pl[s].end());
        B->planU[s] = (int)B->plan.size();
        B->nplanU[s] = (int)pu[s].size();
        B->plan.insert(B->plan.end(), pu[s].begin(), pu[s].end());
    }
    // concatenation
    std::vector<BatchSys> ds(ns);
    int64_t ell = 0, tail = 0, tptr = 0, tent = 0, perm = 0;
    for (int s = 0; s < ns; ++s) {
        const SysLayout &L = B->lay[s];
        BatchSys &d = ds[s];
        d.n = B->sys[s].A.n;
        d.K = L.K;
        d.ld = L.ld;
        d.ntail = (int)L.tail_rows.size();
        d.chL = B->planL[s];
        d.nchL = B->nplanL[s];
        d.chU = B->planU[s];
        d.nchU = B->nplanU[s];
        d.row0 = B->sys_ptr[s];
        d.ell = ell;
        d.tail = tail;
        d.tptr = tptr;
        d.perm = perm;
        ell += (int64_t)L.K * L.ld;
        tail += d.ntail;
        tptr += d.ntail + 1;
        tent += (int64_t)L.tail_col.size();
        perm += d.n;
    }
    std::vector<int> ell_col(ell), tail_rows(tail), tail_col(tent), rop(perm);
    std::vector<double> ell_val(ell), tail_val(tent);
    std::vector<long long> tail_ptr(tptr);
    std::vector<int64_t> tent0(ns + 1, 0);
    for (int s = 0; s < ns; ++s)
        tent0[s + 1] = tent0[s] + (int64_t)B->lay[s].tail_col.size();
    parallel_for(ns, [&](int s) {
        const SysLayout &L = B->lay[s];
        const BatchSys &d = ds[s];
        std::copy(L.ell_col.begin(), L.ell_col.end(), ell_col.begin() + d.ell);
        std::copy(L.ell_val.begin(), L.ell_val.end(), ell_val.begin() + d.ell);
        std::copy(L.tail_rows.begin(), L.tail_rows.end(), tail_rows.begin() + d.tail);
        for (size_t i = 0; i < L.tail_ptr.size(); ++i)
            tail_ptr[d.tptr + i] = L.tail_ptr[i] + tent0[s];
        std::copy(L.tail_col.begin(), L.tail_col.end(), tail_col.begin() + tent0[s]);
        std::copy(L.tail_val.begin(), L.tail_val.end(), tail_val.begin() + tent0[s]);
        std::copy(L.rop.begin(), L.rop.end(), rop.begin() + d.perm);
    });
    std::vector<int> order(ns);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return B->lay[x].cost > B->lay[y].cost; });
    std::vector<float> ell_val32(ell_val.begin(), ell_val.end());
    std::vector<float> tail_val32(tail_val.begin(), tail_val.end());
    HEC_TRY(upload(B->d_sys, ds, st));
    HEC_TRY(upload(B->d_order, order, st));
    HEC_TRY(upload(B->d_ell_col, ell_col, st));
    HEC_TRY(upload(B->d_ell_val64, ell_val, st));
    HEC_TRY(upload(B->d_ell_val32, ell_val32, st));
    HEC_TRY(upload(B->d_tail_rows, tail_rows, st));
    HEC_TRY(upload(B->d_tail_ptr, tail_ptr, st));
    HEC_TRY(upload(B->d_tail_col, tail_col, st));
    HEC_TRY(upload(B->d_tail_val64, tail_val, st));
    HEC_TRY(upload(B->d_tail_val32, tail_val32, st));
    HEC_TRY(upload(B->d_rop, rop, st));
    HEC_CK(cudaStreamSynchronize(st));
    B->host_sys = ds;
    B->fac[0].built = B->fac[1].built = false;
    B->layout_ok = true;
    return HEC_OK;
}

// The factor arena with vb-byte values (4: FP32, 8: FP64).
int build_factors(hec_batch_s *B, int vb, cudaStream_t st)
{
    FacArena &A = B->fac[vb == 4 ? 0 : 1];
    if (A.built)
        return HEC_OK;
    const size_t nc = B->plan.size();
    std::vector<int64_t> off(nc + 1, 0);
    std::vector<char> isU(nc, 0);
    for (int s = 0; s < B->nsys; ++s)
        for (int c = 0; c < B->nplanU[s]; ++c)
            isU[B->planU[s] + c] = 1;
    int64_t maxb = 16;
    for (size_t c = 0; c < nc; ++c) {
        const int64_t b = chunk_bytes(B->plan[c], isU[c], vb);
        off[c + 1] = off[c] + b;
        maxb = std::max(maxb, b);
    }
    if (off[nc] / 16 > (int64_t)0x7fffffff)
        return fail(HEC_ERR_INVALID, "factor arena of %lld bytes is too large", (long long)off[nc]);
    std::vector<unsigned char> fac((size_t)std::max<int64_t>(off[nc], 16), 0);
    std::vector<BChunk> ch(nc);
    parallel_for(B->nsys, [&](int s) {
        for (int c = B->planL[s]; c < B->planU[s] + B->nplanU[s]; ++c) {
            fill_chunk(B, s, B->plan[c], isU[c], vb, fac.data() + off[c]);
            ch[c] = BChunk{(int)(off[c] / 16), (int)(off[c + 1] - off[c]), B->plan[c].first,
                           B->plan[c].nrows};
        }
    });
    HEC_TRY(upload(A.d_fac, fac, st));
    HEC_TRY(upload(A.d_chunks, ch, st));
    HEC_CK(cudaStreamSynchronize(st));
    A.ent_bytes = (int)maxb;
    A.bytes = off[nc];
    A.built = true;
    return HEC_OK;
}

// ------------------------------------------------------------------ launch
struct Launch {
    bool fp32 = true;
    int NR = 1, threads = 256, ctas = 1, grid = 1, nstages = 8, stage_bytes = 0, smem = 0;
    int sstages = 2, sbytes = 0;
};

int resolve_launch(hec_batch_s *B, bool fp32, int nrhs, int m, Launch &L)
{
    L.fp32 = fp32;
    L.NR = nrhs <= 1 ? 1 : nrhs == 2 ? 2 : 4;
    const int tsz = fp32 ? 4 : 8;
    L.threads = B->cfg.threads ? B->cfg.threads : 256;
    L.nstages = B->cfg.nstages ? B->cfg.nstages : 8;
    const FacArena &F = B->fac[fp32 ? 0 : 1];
    L.stage_bytes = (int)r16(F.ent_bytes + batch_rhs_area(L.NR, tsz));
    const int optin = device_smem_optin();
    // A configuration that does not fit the shared memory gives up, in this
    // order: triangular-solve stages (down to 2), the second basis-tile stage,
    // half the CTA size (down to 128).
    for (;;) {
        // basis tiles: m + 1 slots of one CTA-size tile; a third stage when it
        // fits in the triangular-solve stages' share of the region
        L.sbytes = (m + 1) * L.threads * tsz;
        L.sstages = 3 * L.sbytes <= L.nstages * L.stage_bytes ? 3 : 2;
        auto total = [&]() {
            return batch_smem(L.nstages, L.stage_bytes, L.sstages, L.sbytes, B->ring_slots, L.NR,
                              tsz, m, L.threads).total;
        };
        while (total() > optin && L.nstages > 2)
            --L.nstages;
        if (total() > optin)
            L.sstages = 1;
        L.smem = total();
        if (L.smem <= optin || L.threads <= 128)
            break;
        L.threads /= 2;
    }
    if (L.smem > optin)
        return fail(HEC_ERR_INVALID,
                    "batched solve needs %d bytes of shared memory (dependency window of %d "
                    "positions); the device allows %d",
                    L.smem, B->ring_slots, optin);
    const int occ = batch_occupancy(fp32, L.NR, L.threads, L.smem);
    if (occ <= 0)
        return fail(HEC_ERR_CUDA, "batched kernel does not fit an SM (%d threads, %d bytes)",
                    L.threads, L.smem);
    L.ctas = B->cfg.ctas_per_sm ? std::min(B->cfg.ctas_per_sm, occ) : std::min(occ, 4);
    L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(B->nsys, (int64_t)device_sms() * L.ctas));
    return HEC_OK;
}

// Runs the batched kernel once; b and x are device arrays.  ms: device time.
int run_batch(hec_batch_s *B, int op, bool fp32, const double *b, double *x, int nrhs, double tol,
              int maxit, int m, double inner_rtol, bool x0_zero, long long spin, cudaStream_t st,
              float *ms, const unsigned char *only = nullptr)
{
    HEC_TRY(build_layout(B, st));
    const bool need_fac = B->ilu_k >= 0;
    if (need_fac)
        HEC_TRY(build_factors(B, fp32 ? 4 : 8, st));
    Launch L;
    HEC_TRY(resolve_launch(B, fp32, nrhs, m, L));
    const int tsz = fp32 ? 4 : 8;
    const int64_t E = ((int64_t)B->max_n * L.NR + L.threads - 1) / L.threads * L.threads;
    auto al = [](int64_t v) { return (v + 255) & ~(int64_t)255; };
    const int64_t offZ = al((int64_t)(m + 1) * E * tsz);
    const int64_t offY = offZ + al(E * tsz);
    const int64_t offX = offY + al(E * tsz);
    const int64_t offB = offX + al(E * 8);
    const int64_t offR = offB + al(E * 8);
    const int64_t stride = offR + al((int64_t)L.NR * (m + 1) * (m + 1) * 8);
    const size_t wsb = (size_t)stride * L.grid;
    if (B->ws.bytes < wsb)
        HEC_TRY(B->ws.alloc(wsb, st));
    if (!B->queue.p)
        HEC_TRY(B->queue.alloc(16, st));
    if (!B->err.p)
        HEC_TRY(B->err.alloc(16, st));
    if (B->res.bytes < sizeof(BatchResult) * (size_t)B->nsys)
        HEC_TRY(B->res.alloc(sizeof(BatchResult) * (size_t)B->nsys, st));
    HEC_CK(cudaMemsetAsync(B->queue.p, 0, 16, st));
    HEC_CK(cudaMemsetAsync(B->err.p, 0, 16, st));
    BatchArgs a{};
    a.nsys = B->nsys;
    a.nrhs = nrhs;
    a.m = m;
    a.maxit = maxit;
    a.tol = tol;
    a.inner_rtol = inner_rtol;
    a.x0_zero = x0_zero ? 1 : 0;
    a.op = op;
    a.sys = B->d_sys.as<BatchSys>();
    a.order = B->d_order.as<int>();
    const FacArena &F = B->fac[fp32 ? 0 : 1];
    a.chunks = need_fac ? F.d_chunks.as<BChunk>() : nullptr;
    a.fac = need_fac ? F.d_fac.as<unsigned char>() : nullptr;
    a.ell_col = B->d_ell_col.as<int>();
    a.ell_val64 = B->d_ell_val64.as<double>();
    a.ell_val = fp32 ? B->d_ell_val32.p : B->d_ell_val64.p;
    a.tail_rows = B->d_tail_rows.as<int>();
    a.tail_ptr = B->d_tail_ptr.as<long long>();
    a.tail_col = B->d_tail_col.as<int>();
    a.tail_val64 = B->d_tail_val64.as<double>();
    a.tail_val = fp32 ? B->d_tail_val32.p : B->d_tail_val64.p;
    a.row_of_pos = B->d_rop.as<int>();
    a.b = b;
    a.x = x;
    a.ws = B->ws.as<unsigned char>();
    a.ws_stride = stride;
    a.E = E;
    a.offZ = offZ;
    a.offY = offY;
    a.offX = offX;
    a.offB = offB;
    a.offR = offR;
    a.ring_mask = B->ring_slots - 1;
    a.nstages = L.nstages;
    a.stage_bytes = L.stage_bytes;
    a.ent_bytes = (int)r16(F.ent_bytes);
    a.sstages = L.sstages;
    a.sbytes = L.sbytes;
    a.spin_limit = spin;
    a.queue = B->queue.as<int>();
    a.err = B->err.as<int>();
    a.res = B->res.as<BatchResult>();
    a.only = only;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        HEC_CK(cudaEventCreate(&e0));
        HEC_CK(cudaEventCreate(&e1));
        HEC_CK(cudaEventRecord(e0, st));
    }
    const int rc = launch_batch(a, fp32, L.NR, L.threads, L.grid, L.smem, st);
    if (rc != 0) {
        if (ms) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        return fail(HEC_ERR_CUDA, "batched kernel launch: %s", cudaGetErrorString((cudaError_t)rc));
    }
    if (ms) {
        HEC_CK(cudaEventRecord(e1, st));
        HEC_CK(cudaEventSynchronize(e1));
        HEC_CK(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int herr = 0;
    HEC_CK(cudaMemcpyAsync(&herr, B->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HEC_CK(cudaStreamSynchronize(st));
    if (herr != 0)
        return fail(herr, "batched kernel: a bounded device wait ran out");
    return HEC_OK;
}

// A batch made of some of B's systems (for the autotuner's trials).
std::unique_ptr<hec_batch_s> sub_batch(const hec_batch_s *B, const std::vector<int> &idx)
{
    auto S = std::make_unique<hec_batch_s>();
    S->nsys = (int)idx.size();
    S->ilu_k = B->ilu_k;
    S->cfg = B->cfg;
    S->sys_ptr.assign(1, 0);
    for (int i : idx) {
        S->sys.push_back(B->sys[i]);
        S->sys_ptr.push_back(S->sys_ptr.back() + B->sys[i].A.n);
        S->rows += B->sys[i].A.n;
        S->nnz += (int64_t)B->sys[i].A.ci.size();
        S->max_n = std::max(S->max_n, B->sys[i].A.n);
    }
    return S;
}

bool valid_handle(const hec_batch_s *B) { return B != nullptr && B->nsys > 0; }

} // namespace

// ====================================================================== ABI
int hec_build_batched(const hec_batch_csr_t *A, const hec_batch_config_t *cfg, void *stream,
                      hec_batch_t *out)
{
    return abi_guard(__func__, [&]() -> int {
        (void)stream;
        if (!A || !out || !A->sys_ptr || !A->row_ptr || !A->col || !A->val)
            return fail(HEC_ERR_INVALID, "null argument");
        *out = nullptr;
        if (A->nsys < 1)
            return fail(HEC_ERR_INVALID, "nsys must be >= 1");
        hec_batch_config_t c{};
        if (cfg)
            c = *cfg;
        HEC_TRY(check_config(c));
        if (A->sys_ptr[0] != 0 || A->row_ptr[0] != 0)
            return fail(HEC_ERR_INVALID, "sys_ptr[0] and row_ptr[0] must be 0");
        for (int s = 0; s < A->nsys; ++s) {
            const int64_t n = A->sys_ptr[s + 1] - A->sys_ptr[s];
            if (n < 1 || n > (1 << 30))
                return fail(HEC_ERR_INVALID, "system %d has %lld rows", s, (long long)n);
        }
        auto B = std::make_unique<hec_batch_s>();
        B->nsys = A->nsys;
        B->cfg = c;
        B->sys.resize(A->nsys);
        B->sys_ptr.assign(A->sys_ptr, A->sys_ptr + A->nsys + 1);
        std::vector<int> rc(A->nsys, HEC_OK);
        std::vector<std::string> msg(A->nsys);
        parallel_for(A->nsys, [&](int s) {
            const int64_t r0 = A->sys_ptr[s], r1 = A->sys_ptr[s + 1];
            HostCSR &H = B->sys[s].A;
            H.n = (int)(r1 - r0);
            H.rp.resize(H.n + 1);
            const int64_t e0 = A->row_ptr[r0];
            for (int64_t i = r0; i <= r1; ++i) {
                const int64_t e = A->row_ptr[i] - e0;
                if (e < 0 || e > (int64_t)0x7fffffff || (i > r0 && A->row_ptr[i] < A->row_ptr[i - 1])) {
                    rc[s] = HEC_ERR_INVALID;
                    msg[s] = "row_ptr is not non-decreasing";
                    return;
                }
                H.rp[i - r0] = (int)e;
            }
            const int64_t nnz = A->row_ptr[r1] - e0;
            H.ci.assign(A->col + e0, A->col + e0 + nnz);
            H.va.assign(A->val + e0, A->val + e0 + nnz);
            rc[s] = check_csr(H.n, H.rp.data(), H.ci.data(), (int)nnz, true, msg[s]);
        });
        for (int s = 0; s < A->nsys; ++s)
            if (rc[s] != HEC_OK)
                return fail(rc[s], "system %d: %s", s, msg[s].c_str());
        for (const SysHost &S : B->sys) {
            B->rows += S.A.n;
            B->nnz += (int64_t)S.A.ci.size();
            B->max_n = std::max(B->max_n, S.A.n);
        }
        *out = B.release();
        return HEC_OK;
    });
}

int ilu_k_setup_batched(hec_batch_t B, int32_t k)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B))
            return fail(HEC_ERR_INVALID, "invalid batch handle");
        if (k < 0)
            return fail(HEC_ERR_INVALID, "k must be >= 0");
        std::vector<int> rc(B->nsys, HEC_OK);
        std::vector<std::string> msg(B->nsys);
        parallel_for(B->nsys, [&](int s) {
            SysHost &S = B->sys[s];
            BlockFactor &F = S.F;
            F = BlockFactor();
            F.own_lo = 0;
            F.own_hi = S.A.n;
            F.rows.resize(S.A.n);
            std::iota(F.rows.begin(), F.rows.end(), 0);
            F.F = S.A;
            rc[s] = iluk_block(F, k, msg[s]);
            if (rc[s] == HEC_OK)
                levels_block(F);
        });
        for (int s = 0; s < B->nsys; ++s)
            if (rc[s] != HEC_OK) {
                B->ilu_k = -1;
                return fail(rc[s], "system %d: %s", s, msg[s].c_str());
            }
        B->factor_nnz = 0;
        for (const SysHost &S : B->sys)
            B->factor_nnz += (int64_t)S.F.F.ci.size();
        B->ilu_k = k;
        B->layout_ok = false;
        return HEC_OK;
    });
}

int hec_batch_info(hec_batch_t B, hec_batch_info_t *info)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B) || !info)
            return fail(HEC_ERR_INVALID, "invalid argument");
        std::memset(info, 0, sizeof(*info));
        info->nsys = B->nsys;
        info->ilu_k = B->ilu_k;
        info->rows = B->rows;
        info->nnz = B->nnz;
        info->factor_nnz = B->factor_nnz;
        info->max_n = B->max_n;
        info->ring_slots = B->layout_ok ? B->ring_slots : 0;
        info->device_bytes = B->device_bytes();
        info->config = B->cfg;
        return HEC_OK;
    });
}

int hec_batch_set_config(hec_batch_t B, const hec_batch_config_t *cfg)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B) || !cfg)
            return fail(HEC_ERR_INVALID, "invalid argument");
        HEC_TRY(check_config(*cfg));
        if (cfg->ell_width != B->cfg.ell_width)
            B->layout_ok = false;
        B->cfg = *cfg;
        return HEC_OK;
    });
}

int hec_batch_autotune(hec_batch_t B, int32_t nrhs, int32_t restart, const hec_solve_opts_t *opts,
                       void *stream, hec_batch_config_t *chosen)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B) || nrhs < 1 || restart < 1 || restart > kBatchMaxRestart)
            return fail(HEC_ERR_INVALID, "invalid argument");
        cudaStream_t st = (cudaStream_t)stream;
        const bool fp32 = opts && (opts->flags & HEC_MIXED_FP32);
        // sample: about eight systems per SM, evenly spaced over the size ranking,
        // so that every CTA of a trial works through several systems as in the
        // full batch (a trial of one system per CTA would time the largest
        // system's latency, not the throughput)
        std::vector<int> bysize(B->nsys);
        std::iota(bysize.begin(), bysize.end(), 0);
        std::stable_sort(bysize.begin(), bysize.end(),
                         [&](int x, int y) { return B->sys[x].A.n > B->sys[y].A.n; });
        const int want = std::min(B->nsys, 8 * device_sms());
        std::vector<int> idx;
        for (int i = 0; i < want; ++i)
            idx.push_back(bysize[(int64_t)i * B->nsys / want]);
        auto S = sub_batch(B, idx);
        S->factor_nnz = 0;
        for (SysHost &h : S->sys)
            S->factor_nnz += (int64_t)h.F.F.ci.size();
        DevBuf db, dx;
        const size_t vb = (size_t)S->rows * nrhs * sizeof(double);
        HEC_TRY(db.alloc(vb, st));
        HEC_TRY(dx.alloc(vb, st));
        {
            std::vector<double> ones((size_t)S->rows * nrhs, 1.0);
            HEC_CK(cudaMemcpyAsync(db.p, ones.data(), vb, cudaMemcpyHostToDevice, st));
        }
        // ELL width candidates: per-system choice, and the largest row length
        std::vector<int> kc = {0};
        int maxlen = 0;
        for (const SysHost &h : S->sys)
            for (int i = 0; i < h.A.n; ++i)
                maxlen = std::max(maxlen, h.A.rp[i + 1] - h.A.rp[i]);
        bool differs = false;
        for (const SysHost &h : S->sys)
            differs |= ell_width_auto(h.A) != maxlen;
        if (differs)
            kc.push_back(maxlen);
        hec_batch_config_t best = B->cfg;
        float best_ms = 1e30f;
        const int maxit = restart;  // one cycle per system
        for (int K : kc) {
            for (int threads : {128, 256, 512}) {
                for (int ctas : {1, 2, 3, 4}) {
                    if (threads * ctas > 2048)
                        continue;
                    for (int ns : {4, 8}) {
                        hec_batch_config_t c{threads, ctas, K, ns};
                        if (S->cfg.ell_width != K)
                            S->layout_ok = false;
                        S->cfg = c;
                        Launch L;
                        HEC_TRY(build_layout(S.get(), st));
                        if (S->ilu_k >= 0)
                            HEC_TRY(build_factors(S.get(), fp32 ? 4 : 8, st));
                        if (resolve_launch(S.get(), fp32, nrhs, restart, L) != HEC_OK || L.ctas < ctas)
                            continue;  // does not fit
                        float ms = 0.f;
                        const int rc = run_batch(S.get(), BOP_SOLVE, fp32, db.as<double>(), dx.as<double>(),
                                                 nrhs, 1e-30, maxit, restart, fp32 ? 1e-5 : 0.0, true,
                                                 kBatchSpin, st, &ms);
                        if (rc < 0)
                            return rc;
                        if (ms < best_ms) {
                            best_ms = ms;
                            best = c;
                        }
                    }
                }
            }
        }
        if (best.ell_width != B->cfg.ell_width)
            B->layout_ok = false;
        B->cfg = best;
        if (chosen)
            *chosen = best;
        return HEC_OK;
    });
}

int krylov_solve_batched(hec_batch_t B, const double *b, double *x, int32_t nrhs, double tol,
                         int32_t maxit, int32_t restart, const hec_solve_opts_t *opts,
                         void *stream, hec_solve_info_t *info, hec_batch_sys_info_t *sys_info)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B) || !b || !x)
            return fail(HEC_ERR_INVALID, "invalid argument");
        if (nrhs < 1 || restart < 1 || restart > kBatchMaxRestart || maxit < 0 || !(tol >= 0.0))
            return fail(HEC_ERR_INVALID, "nrhs >= 1, 1 <= restart <= %d, maxit >= 0, tol >= 0",
                        kBatchMaxRestart);
        cudaStream_t st = (cudaStream_t)stream;
        hec_solve_opts_t o{};
        if (opts)
            o = *opts;
        const bool fp32 = (o.flags & HEC_MIXED_FP32) != 0;
        const long long spin = o.spin_limit > 0 ? o.spin_limit : kBatchSpin;
        const size_t nb = (size_t)B->rows * nrhs * sizeof(double);
        const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
        DevBuf sb, sx;
        const double *db = b;
        double *dx = x;
        int64_t h2d = 0, d2h = 0;
        if (!bdev) {
            HEC_TRY(sb.alloc(nb, st));
            HEC_CK(cudaMemcpyAsync(sb.p, b, nb, cudaMemcpyHostToDevice, st));
            db = sb.as<double>();
            h2d += (int64_t)nb;
        }
        if (!xdev) {
            HEC_TRY(sx.alloc(nb, st));
            if (!(o.flags & HEC_X0_ZERO)) {
                HEC_CK(cudaMemcpyAsync(sx.p, x, nb, cudaMemcpyHostToDevice, st));
                h2d += (int64_t)nb;
            }
            dx = sx.as<double>();
        }
        HEC_TRY(run_batch(B, BOP_SOLVE, fp32, db, dx, nrhs, tol, maxit, restart, fp32 ? 1e-5 : 0.0,
                          (o.flags & HEC_X0_ZERO) != 0, spin, st, nullptr));
        std::vector<BatchResult> res(B->nsys);
        HEC_CK(cudaMemcpyAsync(res.data(), B->res.p, sizeof(BatchResult) * res.size(),
                               cudaMemcpyDeviceToHost, st));
        HEC_CK(cudaStreamSynchronize(st));
        // systems whose FP32 cycles stopped refining: finish them in FP64, from
        // their current x, in one more launch restricted to them
        std::vector<unsigned char> only(B->nsys, 0);
        int nstag = 0;
        for (int s = 0; s < B->nsys; ++s)
            if (res[s].status == kBatchStagnated) {
                only[s] = 1;
                ++nstag;
            }
        int launches = 1;
        if (nstag > 0) {
            DevBuf donly;
            HEC_TRY(upload(donly, only, st));
            HEC_TRY(run_batch(B, BOP_SOLVE, false, db, dx, nrhs, tol, maxit, restart, 0.0, false, spin,
                              st, nullptr, donly.as<unsigned char>()));
            std::vector<BatchResult> r64(B->nsys);
            HEC_CK(cudaMemcpyAsync(r64.data(), B->res.p, sizeof(BatchResult) * r64.size(),
                                   cudaMemcpyDeviceToHost, st));
            HEC_CK(cudaStreamSynchronize(st));
            for (int s = 0; s < B->nsys; ++s)
                if (only[s]) {
                    res[s].iters += r64[s].iters;
                    res[s].cycles += r64[s].cycles;
                    res[s].reorth += r64[s].reorth;
                    res[s].status = r64[s].status;
                    res[s].rel_resid = r64[s].rel_resid;
                }
            launches = 2;
        }
        if (!xdev) {
            HEC_CK(cudaMemcpyAsync(x, dx, nb, cudaMemcpyDeviceToHost, st));
            d2h += (int64_t)nb;
        }
        HEC_CK(cudaStreamSynchronize(st));
        int status = HEC_OK;
        hec_solve_info_t I{};
        I.fp64_finish = nstag;
        for (int s = 0; s < B->nsys; ++s) {
            const BatchResult &r = res[s];
            I.iters += r.iters;
            I.restarts += r.cycles;
            I.rel_resid = std::max(I.rel_resid, r.rel_resid);
            if (status == HEC_OK && r.status != HEC_OK)
                status = r.status;
            if (sys_info) {
                sys_info[s].iters = r.iters;
                sys_info[s].cycles = r.cycles;
                sys_info[s].status = r.status;
                sys_info[s].reorth = r.reorth;
                sys_info[s].rel_resid = r.rel_resid;
            }
        }
        I.status = status;
        I.kernel_launches = launches;
        I.h2d_bytes = h2d;
        I.d2h_bytes = d2h;
        if (info)
            *info = I;
        return status;
    });
}

int hec_batch_apply(hec_batch_t B, int32_t op, const double *b, double *x, int32_t nrhs, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!valid_handle(B) || !b || !x || nrhs < 1 || op < 0 || op > 3)
            return fail(HEC_ERR_INVALID, "invalid argument");
        if ((op == 2 || op == 3) && B->ilu_k < 0)
            return fail(HEC_ERR_INVALID, "no factors: call ilu_k_setup_batched first");
        static const int kop[4] = {BOP_SPMV64, BOP_SPMV_IN, BOP_PRECOND, BOP_PRECOND};
        const bool fp32 = op == 1 || op == 2;
        return run_batch(B, kop[op], fp32, b, x, nrhs, 0.0, 0, 1, 0.0, true, kBatchSpin,
                         (cudaStream_t)stream, nullptr);
    });
}

void hec_batch_destroy(hec_batch_t B) { delete B; }
