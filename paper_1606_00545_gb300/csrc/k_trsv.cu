// k_trsv.cu -- z = M^{-1} r for the RAS/ILU(k) preconditioner (Sections
// 2.5-2.6): for every RAS block, gather r on V_b, solve L_b y = r_b level by
// level (Eq. 11, Algorithm 3), solve U_b z = y level by level, write z on the
// rows the block owns.
//
// Design for sm_103a.  Each RAS block is solved by one CTA, or by a chain of
// P CTAs of one thread-block cluster ("parts": contiguous ranges of the
// block's rows, see trsv_layout.cpp).  A CTA walks its "program": its rows of
// every level of L_b, then of U_b, packed level-major into chunks (a chunk
// holds rows of one level only; rows inside a level are independent).  A
// chunk is one contiguous byte range in HBM holding, for its rows, the factor
// entries (value, dependency slot), the source index of the right-hand side,
// for U the destination row and the inverted diagonal, and for rows a
// neighbouring part reads, the slot they go to there.  Two chunk formats:
//   - fixed-slot (every row padded to one width FW <= 8): each thread's data
//     sits at a compile-time offset from the stage, so the solving warps copy
//     their rows of the next chunk into registers while the current chunk's
//     multiply-add chain runs -- a level's critical path is then the ring
//     loads, the chain and the barrier;
//   - generic (wider rows): per-warp widths, rows solved from shared memory.
// Nothing on a level's critical path waits for HBM:
//   - an issuer warp streams chunks into a ring of shared-memory stages with
//     cp.async.bulk (the TMA bulk-copy engine, evict-first in L2) completing
//     on mbarriers, S chunks ahead of the solving warps;
//   - two gatherer warps, taking chunks in turn, gather each landed chunk's
//     right-hand sides (L pass: from r; U pass: from the L results, once the
//     L pass is complete) with 4- or 8-byte cp.async, one chunk ahead, and
//     hand the chunk over (a per-stage release-add counter) once the copies
//     have completed and the neighbouring parts have completed the chunks its
//     thresholds name;
//   - solved values of the last few levels live in a shared-memory ring
//     indexed by level-major position (the setup checks that every
//     dependency of a chunk lies within the ring's window; passes whose
//     window does not fit read dependencies from the global scratch); values
//     a neighbouring part reads are also stored straight into that part's
//     import ring (distributed shared memory);
//   - a signaller warp forwards the completed-chunk count to the neighbouring
//     parts (a release at cluster scope, then the count stored into their
//     shared memory), off the solving warps' path.
// Levels are separated by a barrier of the solving warps only -- no
// grid-wide synchronisation.  Every wait is bounded: a wait that runs out
// sets the device error word, one thread waits (bounded) for the copies still
// in flight, and the CTA returns.
#include <mutex>
#include <type_traits>

#include "ptx.cuh"
#include "reduce.cuh"

namespace hec {

// Shared memory of one CTA: S stages, S right-hand-side slots of kThreads
// values, the ring (own and import slots: ring_slots in all), 2 S + 1
// mbarriers and two progress counters.  vbytes: 8 (FP64) or 4 (FP32).
size_t trsv_smem_bytes(int stage_bytes, int nstages, int ring_slots, int vbytes)
{
    const size_t ring = ((size_t)ring_slots * vbytes + 7) & ~(size_t)7;
    return (size_t)stage_bytes * nstages + (size_t)nstages * kThreads * vbytes + ring +
           (size_t)(2 * nstages + 1) * sizeof(uint64_t) + 2 * sizeof(uint32_t);
}

// Gatherer warps of a CTA: each takes every other chunk and keeps two
// chunks' right-hand-side gathers in flight.  (Three and four gatherers
// were measured on the 128^3 case: no faster.)
constexpr int kGatherers = 2;

int trsv_stages_for(int stage_bytes, int ring_slots, int vbytes)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    int S = 8;
    while (S > 3 && trsv_smem_bytes(stage_bytes, S, ring_slots, vbytes) > (size_t)optin)
        --S;
    return S;
}

// ------------------------------------------------------------------ debug build
// Compiled with HEC_DEBUG, the kernel checks what it reads before it uses it:
// every chunk's header against the position the program has reached, every
// gathered index against the array it indexes, every dependency slot against
// the ring.  A failed check records the first violation (code, program,
// chunk, thread, value, bound), sets the error word to HEC_ERR_DEBUG and
// skips the access; nothing traps.
__device__ int g_trsv_debug[8];

#ifdef HEC_DEBUG
__device__ __noinline__ void debug_fail(int *err, int code, int c, int val, int bound)
{
    if (atomicCAS(&g_trsv_debug[0], 0, code) == 0) {
        g_trsv_debug[1] = (int)blockIdx.x;
        g_trsv_debug[2] = c;
        g_trsv_debug[3] = (int)threadIdx.x;
        g_trsv_debug[4] = val;
        g_trsv_debug[5] = bound;
    }
    atomicExch(err, HEC_ERR_DEBUG);
}
#define HEC_CHECK(cond, code, c, val, bound)                                                     \
    ((cond) ? true : (debug_fail(a.err, (code), (c), (int)(val), (int)(bound)), false))
#else
#define HEC_CHECK(cond, code, c, val, bound) true
#endif

// Drain bound for copies already issued when a wait ran out: copies complete
// in microseconds, this only guarantees that the CTA never waits forever.
constexpr long long kDrainPolls = 1ll << 24;

// A chunk in shared memory (layout written by trsv_layout.cpp; T is the
// value type, double or float):
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass, bit 1: exports)
//   [16, 48)  width of every warp's segment
//   [48, 80)  byte offset of every warp's segment
//   [80, 96)  byte offsets of src, dst, dinv, exp
//   [96, 112) need_prev, need_next: completed chunks of part p - 1 / p + 1 to wait for
//   per warp w < nwarps: val[width_w][stride_w] (T), dep[width_w][stride_w] (int32),
//     stride_w = 32 for a full warp, the row count rounded up to 4 for the last one
//   src[r32(nrows)] (int32); for U: dst[r32(nrows)] (int32), dinv[r32(nrows)] (T);
//   with exports: exp[r32(nrows)] (int32), the row's slot in the neighbour's ring
// A dependency is a slot of the ring in ring mode (own values below R,
// imported ones from R on), else a position in the block's global scratch.
constexpr int kWarpRows = 32;
constexpr int kMaxWarps = kThreads / kWarpRows;
constexpr int kFeedThreads = 32 * (kGatherers + 2); // issuer, gatherers and the signaller
constexpr int kMaxStages = 8;

__device__ __forceinline__ int seg_stride(int w, int nrows)
{
    const int left = nrows - w * kWarpRows;
    return left >= kWarpRows ? kWarpRows : (left + 3) & ~3;
}

template <class T> struct ChunkView {
    int nrows, nwarps, base;
    bool upass, exports;
    const int *src, *dst, *exp;
    const T *dinv;
};

template <class T> __device__ __forceinline__ ChunkView<T> view_chunk(const unsigned char *ch)
{
    ChunkView<T> v;
    const int4 hdr = *reinterpret_cast<const int4 *>(ch);
    const int4 off = *reinterpret_cast<const int4 *>(ch + 16 + 8 * kMaxWarps);
    v.nrows = hdr.x;
    v.nwarps = hdr.y;
    v.base = hdr.z;
    v.upass = (hdr.w & 1) != 0;
    v.exports = (hdr.w & 2) != 0;
    v.src = reinterpret_cast<const int *>(ch + off.x);
    v.dst = reinterpret_cast<const int *>(ch + off.y);
    v.dinv = reinterpret_cast<const T *>(ch + off.z);
    v.exp = reinterpret_cast<const int *>(ch + off.w);
    return v;
}

// The segment of warp w: entry k of lane l at val[k * stride + l], dep[k * stride + l].
template <class T> struct Segment {
    int width, stride;
    const T *val;
    const int *dep;
};

template <class T>
__device__ __forceinline__ Segment<T> warp_segment(const unsigned char *ch, int nrows, int w)
{
    const int *hdr = reinterpret_cast<const int *>(ch);
    Segment<T> g;
    g.width = hdr[4 + w];
    g.stride = seg_stride(w, nrows);
    g.val = reinterpret_cast<const T *>(ch + hdr[4 + kMaxWarps + w]);
    g.dep = reinterpret_cast<const int *>(g.val + (size_t)g.width * g.stride);
    return g;
}

// s - sum_k val[k] * y[dep[k]] for one row in ascending column order (y: the
// ring slot dep[k], or the global-scratch position dep[k]), width W
// known at compile time: every shared-memory load of the row is issued before
// the first multiply.  One accumulator: in FP64 the pipe's throughput, not
// the 64-cycle latency of a dependent DFMA, bounds a level once several warps
// are busy, and a second accumulator would cost one more FP64 add per row.
template <int W, bool RING, class T>
__device__ __forceinline__ T row_solve(const Segment<T> &g, int lane, const T *ring, const T *gdep,
                                       T s)
{
    if constexpr (W == 0) {
        return s;
    } else {
        T l[W], y[W];
        int d[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            l[k] = g.val[k * g.stride + lane];
            d[k] = g.dep[k * g.stride + lane];
        }
#pragma unroll
        for (int k = 0; k < W; ++k)
            y[k] = RING ? ring[d[k]] : gdep[d[k]];
#pragma unroll
        for (int k = 0; k < W; ++k)
            s = fma(-l[k], y[k], s);
        return s;
    }
}

template <bool RING, class T>
__device__ __forceinline__ T row_solve_any(const Segment<T> &g, int lane, const T *ring,
                                           const T *gdep, T s)
{
    switch (g.width) {
    case 0: return s;
    case 1: return row_solve<1, RING>(g, lane, ring, gdep, s);
    case 2: return row_solve<2, RING>(g, lane, ring, gdep, s);
    case 3: return row_solve<3, RING>(g, lane, ring, gdep, s);
    case 4: return row_solve<4, RING>(g, lane, ring, gdep, s);
    case 5: return row_solve<5, RING>(g, lane, ring, gdep, s);
    case 6: return row_solve<6, RING>(g, lane, ring, gdep, s);
    case 7: return row_solve<7, RING>(g, lane, ring, gdep, s);
    case 8: return row_solve<8, RING>(g, lane, ring, gdep, s);
    default: {
        // wide rows: loads in blocks of 8 entries
        int k = 0;
        for (; k + 8 <= g.width; k += 8) {
            T l[8], y[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                l[q] = g.val[(k + q) * g.stride + lane];
                const int d = g.dep[(k + q) * g.stride + lane];
                y[q] = RING ? ring[d] : gdep[d];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                s = fma(-l[q], y[q], s);
        }
        for (; k < g.width; ++k) {
            const int d = g.dep[k * g.stride + lane];
            s = fma(-g.val[k * g.stride + lane], RING ? ring[d] : gdep[d], s);
        }
        return s;
    }
    }
}

// Barrier of the consumer warps only (named barrier 1), AND-reducing a flag.
__device__ __forceinline__ int consumer_sync_and(int flag)
{
    int all;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.s32 p, %1, 0;\n\t"
                 "barrier.cta.red.and.pred q, 1, %2, p;\n\t"
                 "selp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(all)
                 : "r"(flag), "n"(kThreads)
                 : "memory");
    return all;
}

// ------------------------------------------------------------------ generic format
// The row of a chunk solved from shared memory: s - sum_k l_k y_dep(k), times
// dinv in the U pass.
template <class T>
__device__ __forceinline__ T solve_row_smem(const unsigned char *ch, const ChunkView<T> &v, int t,
                                            bool rm, const T *ring, const T *gdep, T sacc)
{
    const Segment<T> g = warp_segment<T>(ch, v.nrows, t / kWarpRows);
    const int lane = t % kWarpRows;
    sacc = rm ? row_solve_any<true, T>(g, lane, ring, gdep, sacc)
              : row_solve_any<false, T>(g, lane, ring, gdep, sacc);
    if (v.upass)
        sacc *= v.dinv[t];
    return sacc;
}

// ------------------------------------------------------------------ fixed-slot format
// (written by trsv_layout.cpp; every row padded to FW entries)
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass, bit 1: exports)
//   [16, 32)  need_prev, need_next, FW, xend (exports of the pass so far)
//   per warp w < nwarps a block, lane l = row 32w + l: val (ceil(FW / VW)
//   vectors of 32 lanes x 16 bytes, VW = 16 / sizeof(T)), dep (ceil(FW / 4)
//   vectors of 32 lanes x 4 int32), U: dinv[32] (T), src[32] (int32), U:
//   dst[32] (int32), exp[32] (int32 export positions, -1: none) in launches
//   with exp_arrays
constexpr int kFixedHeader = 32;

template <class T> struct Vec16;
template <> struct Vec16<double> {
    using type = double2;
    __device__ static double get(const double2 &v, int j) { return j == 0 ? v.x : v.y; }
};
template <> struct Vec16<float> {
    using type = float4;
    __device__ static float get(const float4 &v, int j)
    {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    }
};
__device__ __forceinline__ int get4(const int4 &v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

template <class T, int FW> struct Fixed {
    static constexpr int VW = 16 / (int)sizeof(T);
    static constexpr int NV = (FW + VW - 1) / VW; // value vectors per lane
    static constexpr int ND = (FW + 3) / 4;       // dependency vectors per lane
    __device__ static constexpr int dep() { return NV * 512; }
    __device__ static constexpr int dinv() { return (NV + ND) * 512; }
    __device__ static constexpr int src(bool u) { return dinv() + (u ? 32 * (int)sizeof(T) : 0); }
    __device__ static constexpr int dst(bool u) { return src(u) + 128; }
    __device__ static constexpr int exp(bool u) { return src(u) + 128 + (u ? 128 : 0); }
    __device__ static constexpr int block(bool u, bool e) { return exp(u) + (e ? 128 : 0); }
};

// A solving thread's copy of its row of one fixed-slot chunk, with the
// chunk's header fields.
template <class T, int FW> struct RowRegs {
    int nrows, nwarps, base, flags;
    typename Vec16<T>::type lv[Fixed<T, FW>::NV];
    int4 dv[Fixed<T, FW>::ND];
    T rhs, dinv;
    int dst, exp;
    __device__ T l(int k) const { return Vec16<T>::get(lv[k / Fixed<T, FW>::VW], k % Fixed<T, FW>::VW); }
    __device__ int d(int k) const { return get4(dv[k / 4], k % 4); }
};

// Every address below depends only on the stage, the thread and the pass,
// never on a value read from the stage: all loads issue back to back, 16
// bytes each for the row's entries.
template <class T, int FW>
__device__ __forceinline__ void load_fixed(const unsigned char *ch, const T *rslot, int w, int lane,
                                           int t, bool upass, bool exps, RowRegs<T, FW> &R)
{
    using F = Fixed<T, FW>;
    const int4 hdr = *reinterpret_cast<const int4 *>(ch);
    R.nrows = hdr.x;
    R.nwarps = hdr.y;
    R.base = hdr.z;
    R.flags = hdr.w;
    const unsigned char *blk = ch + kFixedHeader + (size_t)w * F::block(upass, exps);
    const typename Vec16<T>::type *val = reinterpret_cast<const typename Vec16<T>::type *>(blk) + lane;
#pragma unroll
    for (int v = 0; v < F::NV; ++v)
        R.lv[v] = val[v * 32];
    const int4 *dep = reinterpret_cast<const int4 *>(blk + F::dep()) + lane;
#pragma unroll
    for (int v = 0; v < F::ND; ++v)
        R.dv[v] = dep[v * 32];
    R.rhs = rslot[t];
    if (upass) {
        R.dinv = reinterpret_cast<const T *>(blk + F::dinv())[lane];
        R.dst = reinterpret_cast<const int *>(blk + F::dst(true))[lane];
    }
    R.exp = exps ? reinterpret_cast<const int *>(blk + F::exp(upass))[lane] : -1;
}

// The issuer warp of both kernels: streams chunk c of the program into stage
// c mod S once the consumers released chunk c - S.  The factor layout is read
// once per apply, so its lines are marked first to leave L2, which keeps the
// gathered right-hand sides and the y scratch there (measured on the 128^3
// case: FP32 apply 0.321 -> 0.286 ms, FP64 unchanged).  (Copying a chunk with
// lane-parallel 16-byte cp.async instead of one cp.async.bulk was measured
// there too: 1.3x slower in FP64, 2x in FP32.)  Returns false when a wait ran
// out.
__device__ __forceinline__ bool issue_chunks(const uint2 *chunks, int nch, int S, int stage_bytes,
                                             const unsigned char *pack, unsigned char *stages,
                                             uint64_t *full, uint64_t *empty, long long limit,
                                             int lane, int *s_issued)
{
    uint2 win = make_uint2(0, 0);
    int wbase = -64;
    int s = 0;
    uint32_t par = 1; // parity of the release of the stage's previous chunk
    const uint64_t pol = l2_evict_first_policy();
    for (int c = 0; c < nch; ++c) {
        if (c >= wbase + 32) { // 32 descriptors per warp-wide load
            wbase = c;
            win = (c + lane < nch) ? chunks[c + lane] : make_uint2(0, 0);
        }
        const unsigned off16 = __shfl_sync(0xffffffffu, win.x, c - wbase);
        const unsigned bytes = __shfl_sync(0xffffffffu, win.y, c - wbase);
        // every wait decision is a warp vote: the lanes must stay converged
        if (c >= S && __any_sync(0xffffffffu, !bounded_wait(&empty[s], par, limit)))
            return false;
        if (lane == 0) {
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s_hint(stages + (size_t)s * stage_bytes, pack + (size_t)off16 * 16, bytes,
                          &full[s], pol);
            *s_issued = c + 1;
        }
        if (++s == S) {
            s = 0;
            par ^= 1u;
        }
    }
    return true;
}

// Release-add by one thread to a shared counter (the handover of a chunk).
__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v)
                 : "memory");
}

// Warp-specialised CTA: warps 0-7 solve rows (one row per thread per chunk),
// warps 8-11 feed them.  Per chunk c in stage s = c mod S:
//   issuer (warp 8): wait empty[s] (chunk c - S released) -> arm full[s] with
//             the chunk's byte count -> cp.async.bulk the chunk;
//   gatherers (warps 9 and 10, chunks alternating): wait full[s] -> gather
//             the chunk's right-hand sides into slot s with cp.async, one
//             commit group per chunk (a U chunk waits for ldone first: its
//             right-hand side is the L pass's output) -> once the group has
//             completed (waited for while the warp's next chunk is gathered)
//             and lane 0 has seen the neighbouring parts' progress counters
//             reach the chunk's thresholds, every lane adds 1 to the stage's
//             handover counter (release): 32 per chunk;
//   consumers: fixed-slot chunks are software-pipelined by one chunk: after
//             issuing chunk c's dependency loads, every thread copies its row
//             of chunk c + 1 into registers, then runs chunk c's multiply-add
//             chain.  The level's results go to the ring (and, for exports,
//             into the neighbour's import ring).  Before the level's barrier
//             the last thread -- whose warp holds the shortest rows --
//             confirms that chunk c + 2 has been handed over (an acquire load
//             of the counter; the barrier orders everybody's later loads
//             after it), and after the barrier it frees chunk c + 1's stage
//             and publishes the completed count.  Generic chunks are solved
//             from shared memory, one at a time;
//   signaller (warp 11): for a split block, forwards the completed count to
//             the neighbouring parts (a release at cluster scope, then the
//             count stored into their shared memory) as often as the fence
//             allows -- the count may jump several chunks at once.
// T = double: the FP64 path; T = float: the FP32 inner solves of the
// mixed-precision mode (FP32 factors, products and accumulation).
template <class T, int FW>
__global__ void __launch_bounds__(kThreads + kFeedThreads, 1) k_trsv_ras(TrsvArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    count_launch(a.st);
    if (a.st && a.st->skip)
        return; // uniform over the grid: no CTA of a cluster reaches a cluster barrier
    const T *r = reinterpret_cast<const T *>(a.r);
    if (a.r_from_j)
        r += (int64_t)a.st->j * a.ldv;

    const bool clustered = a.parts > 1;
    const int part = clustered ? (int)cluster_ctarank() : 0;
    const TrsvBlock blk = a.blocks[blockIdx.x];
    const int S = a.nstages;
    unsigned char *stages = smem;
    T *rhs = reinterpret_cast<T *>(smem + (size_t)S * a.stage_bytes);
    T *ring = rhs + (size_t)S * kThreads;
    const int nown = a.ring_mask + 1;
    const int RI = a.import_slots;
    const int nring = nown + RI; // own values, then values imported from a neighbour
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(ring) +
                                                  (((size_t)nring * sizeof(T) + 7) & ~(size_t)7));
    uint64_t *empty = full + S;
    uint64_t *ldone = empty + S;
    uint32_t *ctr = reinterpret_cast<uint32_t *>(ldone + 1); // [0]: from part p - 1, [1]: from p + 1
    const int nch = blk.chunk_end - blk.chunk_begin;
    const int nL = blk.chunk_mid - blk.chunk_begin; // chunks of the L pass
    const bool has_prev = (blk.links & 1) != 0, has_next = (blk.links & 2) != 0;
    const bool signal = has_prev || has_next;
    const bool exps = FW > 0 && a.exp_arrays != 0;
    const bool stall_test = a.spin_limit < 0;       // fault injection: nothing is issued
    const long long limit = stall_test ? -a.spin_limit : a.spin_limit;
    const uint2 *chunks = a.chunks + blk.chunk_begin;
    T *ysc_w = reinterpret_cast<T *>(a.ysc) + blk.yoff;
    const T *ysc = ysc_w;
    T *zsc = a.zsc ? reinterpret_cast<T *>(a.zsc) + blk.zoff : nullptr;
    T *z = reinterpret_cast<T *>(a.z);
    const int t = threadIdx.x;
    // shared state of the roles (written before the final barrier)
    __shared__ int s_issued, s_err;
    __shared__ uint32_t s_done;             // chunks the consumers have completed
    __shared__ uint32_t s_hand[kMaxStages]; // handover count of every stage: 32 per chunk

    if (t == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(ldone, 1);
        ctr[0] = ctr[1] = 0;
        s_issued = 0;
        s_err = 0;
        s_done = 0;
        fence_mbar_init();
    }
    if (t < kMaxStages)
        s_hand[t] = 0;
    for (int i = t; i < nown; i += blockDim.x)
        ring[i] = T(0);
    __syncthreads();
    // the neighbours store into this CTA's ring and counters only after they
    // are initialised
    if (clustered)
        cluster_sync_all();
    int failed = 0;

    if (t >= kThreads && t < kThreads + 32 && !stall_test) {
        // ------------------------------------------------------------ issuer warp
        if (!issue_chunks(chunks, nch, S, a.stage_bytes, a.pack, stages, full, empty, limit,
                          t - kThreads, &s_issued))
            failed = 1;
    } else if (t >= kThreads + 32 && t < kThreads + 32 * (1 + kGatherers) && !stall_test) {
        // ------------------------------------------------------------ gatherer warps
        // follow the chunks as they land (even chunks: warp 9, odd: warp 10):
        // gather each one's right-hand sides as one cp.async group, and hand
        // the chunk over once its group has completed and the neighbours'
        // progress allows it.  Each warp keeps one chunk's gathers in flight
        // while it issues the next one's.  Every lane hands over for itself,
        // after waiting for its own copies (an arrive-on-completion of the
        // copies, measured on this GPU, did not make them visible to the
        // solving warps in time).
        const int gw = (t - kThreads - 32) / 32;
        const int lane = t % 32;
        bool ldone_seen = false;
        int sg = gw; // S >= 3: chunk gw lies in stage gw, phase 0
        uint32_t par = 0;
        int gp = -1, sgp = 0; // the chunk whose gathers are in flight, and its stage
        // hand chunk gp over: lane 0 first waits for the neighbours' progress
        auto finish = [&]() -> bool {
            int late = 0;
            if (lane == 0 && clustered) {
                // the values this chunk imports are in the ring, and the
                // import slots its exports overwrite have been read
                const unsigned char *ch = stages + (size_t)sgp * a.stage_bytes;
                const int2 need = *reinterpret_cast<const int2 *>(ch + (FW > 0 ? 16 : 96));
                long long it = 0;
                // polls back off, leaving the issue slots to the solving warps
                if (need.x > 0)
                    while ((int)ld_acquire_cluster_u32(&ctr[0]) < need.x && ++it < limit)
                        __nanosleep(32);
                if (need.y > 0)
                    while ((int)ld_acquire_cluster_u32(&ctr[1]) < need.y && ++it < limit)
                        __nanosleep(32);
                late = it >= limit;
            }
            if (__any_sync(0xffffffffu, late))
                return false;
            red_release_add(&s_hand[sgp], 1u); // this lane's gathers of chunk gp have landed
            return true;
        };
        for (int g = gw; g < nch; g += kGatherers) {
            // a chunk in flight is handed over first when the next one has not landed
            if (gp >= 0 && !__all_sync(0xffffffffu, mbar_test_wait(&full[sg], par))) {
                cp_async_wait_group<0>();
                if (!finish()) {
                    failed = 1;
                    break;
                }
                gp = -1;
            }
            if (__any_sync(0xffffffffu, !bounded_wait(&full[sg], par, limit))) {
                failed = 1;
                break;
            }
            const unsigned char *ch = stages + (size_t)sg * a.stage_bytes;
            int4 hdr = *reinterpret_cast<const int4 *>(ch);
            const bool upass = (hdr.w & 1) != 0;
            if (!HEC_CHECK(upass == (g >= nL), 1, g, hdr.w, nL) ||
                !HEC_CHECK(hdr.x >= 1 && hdr.x <= kThreads, 2, g, hdr.x, kThreads))
                hdr.x = 0; // nothing gathered from a chunk that is not the expected one
            if (upass && !ldone_seen) {
                if (gp >= 0) { // the last L chunk in flight goes first
                    cp_async_wait_group<0>();
                    if (!finish()) {
                        failed = 1;
                        break;
                    }
                    gp = -1;
                }
                if (__any_sync(0xffffffffu, !bounded_wait(ldone, 0u, limit))) {
                    failed = 1;
                    break;
                }
                ldone_seen = true;
            }
            T *slot = rhs + (size_t)sg * kThreads;
            const T *from = upass ? ysc : r;
            if constexpr (FW > 0) {
                const int blkb = Fixed<T, FW>::block(upass, exps);
                const unsigned char *src = ch + kFixedHeader + Fixed<T, FW>::src(upass) + 4 * lane;
                for (int i = lane, j = 0; i < hdr.x; i += 32, ++j) {
                    const int si = *reinterpret_cast<const int *>(src + (size_t)j * blkb);
                    if (HEC_CHECK(si >= 0 && (upass || si < a.n), 3, g, si, a.n))
                        cp_async_v<sizeof(T)>(&slot[i], from + si);
                }
            } else {
                const ChunkView<T> v = view_chunk<T>(ch);
                for (int i = lane; i < hdr.x; i += 32)
                    if (HEC_CHECK(v.src[i] >= 0 && (upass || v.src[i] < a.n), 3, g, v.src[i], a.n))
                        cp_async_v<sizeof(T)>(&slot[i], from + v.src[i]);
            }
            cp_async_commit();
            if (gp >= 0) { // the previous chunk's group: all but the newest have completed
                cp_async_wait_group<1>();
                if (!finish()) {
                    failed = 1;
                    break;
                }
            }
            gp = g;
            sgp = sg;
            sg += kGatherers;
            if (sg >= S) {
                sg -= S;
                par ^= 1u;
            }
        }
        if (!failed && gp >= 0) {
            cp_async_wait_group<0>();
            if (!finish())
                failed = 1;
        }
        cp_async_wait_all();
    } else if (t >= kThreads + 32 * (1 + kGatherers)) {
        // ------------------------------------------------------------ signaller warp
        // publishes the completed-chunk count to the neighbours: the release
        // at cluster scope covers the consumers' stores into the neighbours'
        // import rings, ordered before the count by the consumer barrier
        if (signal && t == kThreads + 32 * (1 + kGatherers)) {
            const uint32_t to_prev = has_prev ? mapa_shared(smem_u32(&ctr[1]), part - 1) : 0;
            const uint32_t to_next = has_next ? mapa_shared(smem_u32(&ctr[0]), part + 1) : 0;
            uint32_t pub = 0;
            long long it = 0;
            while (pub < (uint32_t)nch) {
                const uint32_t v = ld_acquire_cta_u32(&s_done);
                if (v > pub) {
                    fence_acq_rel_cluster();
                    if (has_prev)
                        st_relaxed_cluster_u32(to_prev, v);
                    if (has_next)
                        st_relaxed_cluster_u32(to_next, v);
                    pub = v;
                    it = 0;
                } else if (*reinterpret_cast<volatile int *>(&s_err) || ++it >= limit) {
                    failed = 1;
                    break;
                } else {
                    __nanosleep(64);
                }
            }
        }
    } else if (t < kThreads) {
    // ---------------------------------------------------------------- consumer warps
    volatile int *verr = &s_err;
    // the neighbours' import rings: L values go to part p + 1, U values to p - 1
    const uint32_t imp_next =
        has_next ? mapa_shared(smem_u32(ring + nown), part + 1) : 0;
    const uint32_t imp_prev =
        has_prev ? mapa_shared(smem_u32(ring + nown), part - 1) : 0;
    int s = 0;         // stage of chunk c
    uint32_t hneed = 32; // the stage's handover count once chunk c is handed over
    int err = 0;
    // wait (bounded) until chunk c, in stage s, has been handed over
    auto handed = [&](int st, uint32_t need) -> bool {
        long long it = 0;
        while (ld_acquire_cta_u32(&s_hand[st]) < need) {
            if (++it >= limit)
                return false;
            __nanosleep(16);
        }
        return true;
    };
    // a solved row leaves: ring or scratch, neighbour's import ring; returns
    // where its global copy goes (written after the level's barrier)
    auto put = [&](bool upass, bool rm, int pos, int dst, int e, T acc) -> T * {
        T *gout = nullptr;
        if (upass) {
            if (rm)
                ring[pos & a.ring_mask] = acc;
            else
                zsc[pos] = acc; // read by later levels of this pass
            if (dst >= 0)
                gout = z + dst;
        } else if (rm) {
            ring[pos & a.ring_mask] = acc;
            gout = ysc_w + pos;
        } else {
            ysc_w[pos] = acc; // read by later levels of this pass
        }
        if (e >= 0)
            st_cluster((upass ? imp_prev : imp_next) + (uint32_t)((e & (RI - 1)) * sizeof(T)),
                       acc);
        return gout;
    };
    // after the level's barrier: global copies, end of the L pass, progress
    auto close = [&](int c, T *gout, T out) {
        if (gout)
            *gout = out;
        if (c == nL - 1) {
            // every y of the L pass is written before the gatherers read
            // the U pass's right-hand sides from them
            consumer_sync_and(1);
            if (t == kThreads - 1)
                mbar_arrive(ldone);
        }
        if (t == kThreads - 1 && signal)
            st_release_cta_u32(&s_done, (uint32_t)(c + 1));
    };
    if constexpr (FW > 0) {
        const int w = t / kWarpRows, lane = t % kWarpRows;
        RowRegs<T, FW> A, B;
        // one pass: chunks [c0, c1), U: the upper-triangular pass.  Before a
        // level's barrier every thread has copied its row of the next chunk
        // of the pass into registers, so that chunk's stage is free after
        // the barrier, and the next level starts with its dependencies.
        auto run = [&](auto Ucst, int c0, int c1) -> bool {
            constexpr bool U = decltype(Ucst)::value;
            if (c0 >= c1)
                return false;
            const bool rm = U ? blk.ring_U : blk.ring_L;
            const T *gdep = U ? zsc : ysc;
            T *scr = U ? zsc : ysc_w;
            const uint32_t imp = U ? imp_prev : imp_next;
            // stage and handover count of the chunk after a given one
            auto next = [&](int &st, uint32_t &h) {
                if (++st == S) {
                    st = 0;
                    h += 32;
                }
            };
            // the last thread confirms the handovers (acquire) before a
            // barrier, so the other threads' loads after it need no check:
            // chunks c0 and c0 + 1 now, chunk c + 2 at level c
            int s1 = s, s2;
            uint32_t h1 = hneed, h2;
            next(s1, h1);
            s2 = s1;
            h2 = h1;
            next(s2, h2);
            int err = 0;
            if (t == kThreads - 1)
                err = !handed(s, hneed) || (c0 + 1 < c1 && !handed(s1, h1));
            if (!consumer_sync_and(!err)) {
                *verr = 1;
                return true;
            }
            load_fixed<T, FW>(stages + (size_t)s * a.stage_bytes, rhs + (size_t)s * kThreads, w,
                              lane, t, U, exps, A);
#ifdef HEC_DEBUG
            int xbase = 0; // position the program has reached in its pass
#endif
            // level c: cur holds chunk c, nxt receives chunk c + 1; s, s1, s2
            // are the stages of chunks c, c + 1, c + 2
            auto level = [&](int c, RowRegs<T, FW> &cur, RowRegs<T, FW> &nxt) -> bool {
                const bool more = c + 1 < c1, more2 = c + 2 < c1;
                bool rows = w < cur.nwarps; // warps past the chunk's last one hold no rows
#ifdef HEC_DEBUG
                rows = rows && HEC_CHECK(cur.base == xbase, 4, c, cur.base, xbase) &&
                       HEC_CHECK((cur.flags & 1) == (U ? 1 : 0), 1, c, cur.flags, nL) &&
                       HEC_CHECK(cur.nrows >= 1 && cur.nrows <= kThreads &&
                                     cur.nwarps == (cur.nrows + 31) / 32,
                                 2, c, cur.nrows, cur.nwarps);
                if (rows)
                    for (int k = 0; k < FW; ++k)
                        rows &= rm ? HEC_CHECK(cur.d(k) >= 0 && cur.d(k) < nring, 5, c, cur.d(k),
                                               nring)
                                   : HEC_CHECK(cur.l(k) == T(0) ||
                                                   (cur.d(k) >= 0 && cur.d(k) < cur.base),
                                               6, c, cur.d(k), cur.base);
                if (rows && t < cur.nrows && U)
                    rows &= HEC_CHECK(cur.dst < a.n, 7, c, cur.dst, a.n);
                xbase += cur.nrows;
#endif
                // this level's dependencies (the previous level's barrier has
                // passed); padding lanes of the last warp carry valid slots
                T y[FW];
                if (rows) {
                    if (rm) {
#pragma unroll
                        for (int k = 0; k < FW; ++k)
                            y[k] = ring[cur.d(k)];
                    } else {
                        // global scratch: padding of a dependency-free row
                        // points at a position this apply has not written (it
                        // may hold NaN); entries of value 0 are not read
#pragma unroll
                        for (int k = 0; k < FW; ++k)
                            y[k] = cur.l(k) != T(0) ? gdep[cur.d(k)] : T(0);
                    }
                }
                // the next chunk's rows (handed over, confirmed before the
                // previous barrier): loads only, first used after this barrier
                if (more)
                    load_fixed<T, FW>(stages + (size_t)s1 * a.stage_bytes,
                                      rhs + (size_t)s1 * kThreads, w, lane, t, U, exps, nxt);
                T out = T(0);
                T *gout = nullptr;
                if (rows) { // warps without rows issue no multiply-adds
                    T acc = cur.rhs;
#pragma unroll
                    for (int k = 0; k < FW; ++k)
                        acc = fma(-cur.l(k), y[k], acc);
                    if (U)
                        acc *= cur.dinv;
                    if (t < cur.nrows) {
                        const int pos = cur.base + t;
                        if (rm)
                            ring[pos & a.ring_mask] = acc;
                        else
                            scr[pos] = acc; // read by later levels of this pass
                        if (U)
                            gout = cur.dst >= 0 ? z + cur.dst : nullptr;
                        else if (rm)
                            gout = ysc_w + pos;
                        if (cur.exp >= 0) // exports (-1 without export slots)
                            st_cluster(imp + (uint32_t)((cur.exp & (RI - 1)) * sizeof(T)), acc);
                        out = acc;
                    }
                }
                int bad = 0;
                if (t == kThreads - 1 && more2)
                    bad = !handed(s2, h2);
                if (!consumer_sync_and(!bad))
                    return true; // a feeding warp's wait ran out
                // every thread holds its rows of chunks c and c + 1: their
                // stages are free (chunk c's only now at the pass's first level)
                if (t == kThreads - 1) {
                    if (c == c0)
                        mbar_arrive(&empty[s]);
                    if (more)
                        mbar_arrive(&empty[s1]);
                    if (signal)
                        st_release_cta_u32(&s_done, (uint32_t)(c + 1));
                }
                if (gout)
                    *gout = out;
                s = s1;
                hneed = h1;
                s1 = s2;
                h1 = h2;
                next(s2, h2);
                return false;
            };
            for (int c = c0; c < c1; c += 2) {
                if (level(c, A, B)) {
                    *verr = 1;
                    return true;
                }
                if (c + 1 < c1 && level(c + 1, B, A)) {
                    *verr = 1;
                    return true;
                }
            }
            return false;
        };

        if (run(std::integral_constant<bool, false>(), 0, nL)) {
            failed = 1;
        } else {
            if (nL > 0) {
                // every y of the L pass is written before the gatherers read
                // the U pass's right-hand sides from them
                consumer_sync_and(1);
                if (t == kThreads - 1)
                    mbar_arrive(ldone);
            }
            if (run(std::integral_constant<bool, true>(), nL, nch))
                failed = 1;
        }

    } else {
        for (int c = 0; c < nch; ++c) {
            if (!handed(s, hneed)) {
                err = 1;
                *verr = 1;
            }
            T out = T(0);
            T *gout = nullptr;
            if (!err) {
                const unsigned char *ch = stages + (size_t)s * a.stage_bytes;
                const ChunkView<T> v = view_chunk<T>(ch);
                if (t < v.nrows) {
                    const bool rm = v.upass ? blk.ring_U : blk.ring_L;
                    const T acc = solve_row_smem<T>(ch, v, t, rm, ring, v.upass ? zsc : ysc,
                                                    rhs[(size_t)s * kThreads + t]);
                    gout = put(v.upass, rm, v.base + t, v.upass ? v.dst[t] : -1,
                               v.exports ? v.exp[t] : -1, acc);
                    out = acc;
                }
            }
            if (!consumer_sync_and(!err)) {
                failed = 1; // the feeding warps' own waits run out
                break;
            }
            if (t == kThreads - 1)
                mbar_arrive(&empty[s]); // stage s and its right-hand-side slot are free
            close(c, gout, out);
            if (++s == S) {
                s = 0;
                hneed += 32;
            }
        }
    }
    }
    // every role has left its loop: drain the copies still in flight, report
    __syncthreads();
    if (t == kThreads) {
        const int issued = s_issued;
        const int first = issued - S > 0 ? issued - S : 0;
        for (int c = first; c < issued; ++c)
            bounded_wait(&full[c % S], (uint32_t)(c / S) & 1u, kDrainPolls);
    }
    if (failed) {
        atomicExch(a.err, HEC_ERR_TIMEOUT);
        if (a.st)
            a.st->err = HEC_ERR_TIMEOUT;
    }
    // no CTA leaves while a neighbour may still store into its shared memory
    if (clustered)
        cluster_sync_all();
}

// ------------------------------------------------------------------ resident-vector kernel
// A RAS block whose right-hand side fits in shared memory next to the chunk
// stages is solved in place, by one CTA, with nothing on a level's critical
// path but shared memory: xs[i] starts as r[V_b[i]] (all local rows, gathered
// once at launch), the L pass overwrites it with y_i, the U pass with z_i, and
// the owned rows are written to z at the end.  A row's right-hand side is its
// own slot and its dependencies are the slots of its columns (local row
// indices), so there are no gatherer warps, no global scratch and no handover
// counters: one issuer warp streams the chunks (rows of one level) into the
// stages S chunks ahead with cp.async.bulk, and the solving warps run
//   level c: read the dependencies and the right-hand side of chunk c's rows
//            from xs, copy chunk c + 1's rows into registers, run the
//            multiply-add chain, store the results into xs; the last thread
//            confirms that chunk c + 2 has landed; barrier; chunk c + 1's stage
//            is released.
// The per-level critical path is a shared-memory load, the row's dependent
// multiply-adds (for U, the multiply by 1/u_ii) and a barrier of the solving
// warps.  This is the latency-first form for small systems (a single ILU block
// of a few thousand rows has hundreds of levels of a few dozen rows each).
//
// Chunk format (trsv_layout.cpp, flag bits 3 and 5): [0, 16) nrows, nwarps,
// first position, flags (bit 0: U pass); [16, 32) 0, 0, FW, 0; then per warp
// w < nwarps a block: val (ceil(FW / VW) 16-byte vectors of 32 lanes), idx
// (ceil((FW + 1) / 8) 16-byte vectors of 32 lanes x 8 uint16: the FW
// dependency slots, then the row's own slot), for U dinv[32].  Padding
// entries have value 0 and slot nv (a slot that holds 0); padding rows have
// row slot nv and are not stored.
template <class T, int FW> struct Res {
    static constexpr int VW = 16 / (int)sizeof(T);
    static constexpr int NV = (FW + VW - 1) / VW; // value vectors per lane
    static constexpr int NI = (FW + 1 + 7) / 8;   // index vectors per lane
    __device__ static constexpr int idx() { return NV * 512; }
    __device__ static constexpr int dinv() { return (NV + NI) * 512; }
    __device__ static constexpr int block() { return dinv() + 32 * (int)sizeof(T); }
};

template <class T, int FW> struct ResRow {
    int nrows, nwarps, flags;
    int next_off, next_nw; // the next chunk's offset in its group's stage and its warps
    typename Vec16<T>::type lv[Res<T, FW>::NV];
    uint4 iv[Res<T, FW>::NI];
    T dinv;
    __device__ T l(int k) const { return Vec16<T>::get(lv[k / Res<T, FW>::VW], k % Res<T, FW>::VW); }
    // uint16 k of the index vectors: dependency slot k < FW, the row's slot at FW
    __device__ int slot(int k) const
    {
        const uint4 &v = iv[k / 8];
        const int q = (k % 8) / 2;
        const uint32_t word = q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
        return (int)((word >> (16 * (k % 2))) & 0xffffu);
    }
};

// A solving thread's row of a resident-format chunk.  Every chunk has a block
// for each of the kernel's NW solving warps (padding rows beyond its rows), so
// a warp reads its block without waiting for the chunk's header; nw limits
// the reads all the same (the header's warp count of a chunk is at most NW).
template <class T, int FW, bool U>
__device__ __forceinline__ void load_res(const unsigned char *ch, int w, int lane, int nw,
                                         ResRow<T, FW> &R)
{
    using F = Res<T, FW>;
    const int4 hdr = *reinterpret_cast<const int4 *>(ch);
    const int4 nxt = *reinterpret_cast<const int4 *>(ch + 16);
    R.nrows = hdr.x;
    R.nwarps = hdr.y;
    R.flags = hdr.w;
    R.next_off = nxt.x;
    R.next_nw = nxt.y;
    if (w >= nw)
        return;
    const unsigned char *blk = ch + kFixedHeader + (size_t)w * F::block();
    const typename Vec16<T>::type *val = reinterpret_cast<const typename Vec16<T>::type *>(blk) + lane;
#pragma unroll
    for (int v = 0; v < F::NV; ++v)
        R.lv[v] = val[v * 32];
    const uint4 *idx = reinterpret_cast<const uint4 *>(blk + F::idx()) + lane;
#pragma unroll
    for (int v = 0; v < F::NI; ++v)
        R.iv[v] = idx[v * 32];
    if (U)
        R.dinv = reinterpret_cast<const T *>(blk + F::dinv())[lane];
}

// Barrier of the NT solving threads of a resident-kernel CTA (named barrier
// 1), AND-reducing a flag.
template <int NT> __device__ __forceinline__ int solvers_sync_and(int flag)
{
    int all;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.s32 p, %1, 0;\n\t"
                 "barrier.cta.red.and.pred q, 1, %2, p;\n\t"
                 "selp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(all)
                 : "r"(flag), "n"(NT)
                 : "memory");
    return all;
}

// NW solving warps (chunks of at most 32 NW rows, NW sized at setup to the
// widest level) and one issuer warp.
template <class T, int FW, int NW>
__global__ void __launch_bounds__(NW * 32 + 32, 1) k_trsv_res(TrsvArgs a)
{
    constexpr int NT = NW * 32; // solving threads
    extern __shared__ __align__(128) unsigned char smem[];
    count_launch(a.st);
    if (a.st && a.st->skip)
        return; // uniform over the grid
    const T *r = reinterpret_cast<const T *>(a.r);
    if (a.r_from_j)
        r += (int64_t)a.st->j * a.ldv;
    T *z = reinterpret_cast<T *>(a.z);
    const TrsvBlock blk = a.blocks[blockIdx.x];
    const int S = a.nstages;
    unsigned char *stages = smem;
    T *xs = reinterpret_cast<T *>(smem + (size_t)S * a.stage_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(xs) +
                                                  (((size_t)a.res_slots * sizeof(T) + 7) & ~(size_t)7));
    uint64_t *empty = full + S;
    const int nch = blk.chunk_end - blk.chunk_begin;
    const int nL = blk.chunk_mid - blk.chunk_begin;
    const int *vrows = a.vrows + blk.yoff; // V_b: the global row of every local slot
    const bool stall_test = a.spin_limit < 0; // fault injection: nothing is issued
    const long long limit = stall_test ? -a.spin_limit : a.spin_limit;
    const int t = threadIdx.x;
    __shared__ int s_issued;
    if (t == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        s_issued = 0;
        fence_mbar_init();
    }
    __syncthreads();
    int failed = 0;
    if (t >= NT) {
        // ------------------------------------------------------------ issuer warp
        if (!stall_test &&
            !issue_chunks(a.groups + blk.zoff, blk.ngroups, S, a.stage_bytes, a.pack, stages,
                          full, empty, limit, t - NT, &s_issued))
            failed = 1;
    } else {
        // ------------------------------------------------------------ solving warps
        // r on V_b into the resident vector; slot nv holds 0 (padding)
        for (int i = t; i < blk.nv; i += NT) {
            const int g = vrows[i];
            xs[i] = HEC_CHECK(g >= 0 && g < a.n, 3, 0, g, a.n) ? r[g] : T(0);
        }
        if (t == 0)
            xs[blk.nv] = T(0);
        const int w = t / kWarpRows, lane = t % kWarpRows;
        // Chunks arrive in groups of G (one bulk copy each) in stage order, all
        // of one size CB: chunk k of a group sits at k CB in its group's stage.
        // A chunk's place is that stage s, the stage's phase parity and k.
        constexpr int CB = kFixedHeader + NW * Res<T, FW>::block();
        const int G = a.res_group;
        struct Loc {
            int s;
            uint32_t ph;
            int k;
        };
        auto next = [&](Loc l) -> Loc {
            if (++l.k == G) {
                l.k = 0;
                if (++l.s == S) {
                    l.s = 0;
                    l.ph ^= 1u;
                }
            }
            return l;
        };
        auto landed = [&](const Loc &l) -> bool { return bounded_wait(&full[l.s], l.ph, limit); };
        auto load = [&](bool U, const Loc &l, ResRow<T, FW> &R) {
            const unsigned char *ch = stages + (size_t)l.s * a.stage_bytes + (size_t)l.k * CB;
            if (U)
                load_res<T, FW, true>(ch, w, lane, NW, R);
            else
                load_res<T, FW, false>(ch, w, lane, NW, R);
        };
        const Loc l0{0, 0u, 0};
        int bad = 0;
        if (t == NT - 1 && nch > 0)
            bad = !landed(l0);
        // the gather above is complete and the first group has landed
        if (!solvers_sync_and<NT>(!bad)) {
            failed = 1;
        } else if (nch > 0) {
            ResRow<T, FW> A, B;
            load(0 >= nL, l0, A);
            Loc ln = next(l0); // chunk 1
            bad = (t == NT - 1 && nch > 1 && ln.k == 0) ? !landed(ln) : 0;
            if (!solvers_sync_and<NT>(!bad))
                failed = 1;
            // level c: cur holds chunk c's rows, nxt receives chunk c + 1's
            // (found at ln); every place is known without reading a header
            auto level = [&](int c, ResRow<T, FW> &cur, ResRow<T, FW> &nxt) -> bool {
                const bool U = c >= nL;
                const bool rows = w < cur.nwarps; // warps past the chunk's last one idle
                T y[FW];
                T acc = T(0);
                int me = blk.nv;
                if (rows) {
#pragma unroll
                    for (int k = 0; k < FW; ++k) {
                        const int d = cur.slot(k);
                        y[k] = HEC_CHECK(d <= blk.nv, 5, c, d, blk.nv) ? xs[d] : T(0);
                    }
                    me = cur.slot(FW);
                    if (!HEC_CHECK(me <= blk.nv, 7, c, me, blk.nv))
                        me = blk.nv;
                    acc = xs[me];
                }
                const Loc l2 = next(ln); // chunk c + 2
                const bool more = c + 1 < nch;
                if (more) // its group landed: confirmed before the previous barrier
                    load(c + 1 >= nL, ln, nxt);
                // chunk c + 2 opens a group: the last thread confirms it landed
                int late = 0;
                if (t == NT - 1 && c + 2 < nch && l2.k == 0)
                    late = !landed(l2);
                if (rows) {
#pragma unroll
                    for (int k = 0; k < FW; ++k)
                        acc = fma(-cur.l(k), y[k], acc);
                    if (U)
                        acc *= cur.dinv;
                    if (t < cur.nrows && me < blk.nv)
                        xs[me] = acc;
                }
                if (!solvers_sync_and<NT>(!late))
                    return false;
                // every thread holds chunks up to c + 1 in registers: the group
                // that chunk closes has a free stage
                if (t == NT - 1) {
                    if (c == 0 && (G == 1 || nch == 1))
                        mbar_arrive(&empty[0]);
                    if (more && (ln.k == G - 1 || c + 1 == nch - 1))
                        mbar_arrive(&empty[ln.s]);
                }
                ln = l2;
                return true;
            };
            for (int c = 0; c < nch && !failed; c += 2) {
                if (!level(c, A, B))
                    failed = 1;
                else if (c + 1 < nch && !level(c + 1, B, A))
                    failed = 1;
            }
            if (!failed)
                for (int i = blk.own0 + t; i < blk.own1; i += NT)
                    z[vrows[i]] = xs[i];
        }
    }
    // every role has left its loop: drain the copies still in flight, report
    __syncthreads();
    if (t == NT) {
        const int issued = s_issued;
        const int first = issued - S > 0 ? issued - S : 0;
        for (int c = first; c < issued; ++c)
            bounded_wait(&full[c % S], (uint32_t)(c / S) & 1u, kDrainPolls);
    }
    if (failed) {
        atomicExch(a.err, HEC_ERR_TIMEOUT);
        if (a.st)
            a.st->err = HEC_ERR_TIMEOUT;
    }
}

// The dynamic shared memory limit is a process-wide attribute of the kernel:
// raised once to the device's opt-in maximum, so that launches of different
// sizes from several host threads never race on it.
template <class T, int FW, bool RES, int NW = 8> static cudaError_t prepare_trsv()
{
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, []() {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaFuncAttributes fa{};
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) {
            if constexpr (RES)
                e = cudaFuncGetAttributes(&fa, k_trsv_res<T, FW, NW>);
            else
                e = cudaFuncGetAttributes(&fa, k_trsv_ras<T, FW>);
        }
        if (e == cudaSuccess) { // the opt-in limit covers static and dynamic shared memory
            if constexpr (RES)
                e = cudaFuncSetAttribute(k_trsv_res<T, FW, NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes);
            else
                e = cudaFuncSetAttribute(k_trsv_ras<T, FW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes);
        }
    });
    return e;
}

template <class T, int FW> static int launch_t(const TrsvArgs &a, cudaStream_t s)
{
    const size_t smem =
        trsv_smem_bytes(a.stage_bytes, a.nstages, a.ring_mask + 1 + a.import_slots, sizeof(T));
    if (prepare_trsv<T, FW, false>() != cudaSuccess)
        return -1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)a.nblocks);
    cfg.blockDim = dim3(kThreads + kFeedThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.parts;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.parts > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_trsv_ras<T, FW>, a) == cudaSuccess ? 0 : -1;
}

template <class T, int FW, int NW> static int launch_res(const TrsvArgs &a, cudaStream_t s)
{
    const size_t smem = trsv_res_smem_bytes(a.stage_bytes, a.nstages, a.res_slots, sizeof(T));
    if (prepare_trsv<T, FW, true, NW>() != cudaSuccess)
        return -1;
    k_trsv_res<T, FW, NW><<<a.nblocks, NW * 32 + 32, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class T, int FW> static int launch_res_w(const TrsvArgs &a, cudaStream_t s)
{
    switch (a.res_warps) {
    case 2: return launch_res<T, FW, 2>(a, s);
    case 4: return launch_res<T, FW, 4>(a, s);
    case 8: return launch_res<T, FW, 8>(a, s);
    default: return -1;
    }
}

size_t trsv_res_smem_bytes(int stage_bytes, int nstages, int res_slots, int vbytes)
{
    return (size_t)stage_bytes * nstages + (((size_t)res_slots * vbytes + 7) & ~(size_t)7) +
           (size_t)2 * nstages * sizeof(uint64_t);
}

int trsv_res_stages_for(int stage_bytes, int res_slots, int vbytes)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    optin -= 1024; // static shared memory of the kernel
    for (int S = 8; S >= 3; --S)
        if (trsv_res_smem_bytes(stage_bytes, S, res_slots, vbytes) <= (size_t)optin)
            return S;
    return 0;
}

int trsv_debug_read(int *out, bool clear)
{
    if (cudaMemcpyFromSymbol(out, g_trsv_debug, sizeof(g_trsv_debug)) != cudaSuccess)
        return -1;
    if (clear) {
        static const int zero[8] = {};
        if (cudaMemcpyToSymbol(g_trsv_debug, zero, sizeof(zero)) != cudaSuccess)
            return -1;
    }
    return 0;
}

bool trsv_debug_build()
{
#ifdef HEC_DEBUG
    return true;
#else
    return false;
#endif
}

int launch_trsv(const TrsvArgs &a, cudaStream_t s, bool fp32)
{
    if (a.resident) {
#define HEC_RES_CASE(W)                                                                          \
    case W: return fp32 ? launch_res_w<float, W>(a, s) : launch_res_w<double, W>(a, s);
        switch (a.fixed_width) {
            HEC_RES_CASE(2)
            HEC_RES_CASE(3)
            HEC_RES_CASE(4)
            HEC_RES_CASE(6)
            HEC_RES_CASE(8)
        default: return -1;
        }
#undef HEC_RES_CASE
    }
    // fixed-slot layouts by their uniform width; generic layouts
    if (!fp32) {
        switch (a.fixed_width) {
        case 4: return launch_t<double, 4>(a, s);
        case 6: return launch_t<double, 6>(a, s);
        case 8: return launch_t<double, 8>(a, s);
        default: return launch_t<double, 0>(a, s);
        }
    }
    switch (a.fixed_width) {
    case 4: return launch_t<float, 4>(a, s);
    case 6: return launch_t<float, 6>(a, s);
    case 8: return launch_t<float, 8>(a, s);
    default: return launch_t<float, 0>(a, s);
    }
}

int trsv_uniform_width(int longest_row)
{
    return longest_row <= 4 ? 4 : longest_row <= 6 ? 6 : longest_row <= 8 ? 8 : 0;
}

} // namespace hec
