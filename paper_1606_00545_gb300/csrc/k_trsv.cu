// k_trsv.cu -- z = M^{-1} r for the RAS/ILU(k) preconditioner (Sections
// 2.5-2.6): for every RAS block, gather r on V_b, solve L_b y = r_b level by
// level (Eq. 11, Algorithm 3), solve U_b z = y level by level, write z on the
// rows the block owns.
//
// Design for sm_103a.  One persistent CTA per RAS block walks the block's
// "program": the rows of every level of L_b, then of U_b, packed level-major
// into chunks (a chunk holds rows of one level only; rows inside a level are
// independent).  A chunk is one contiguous byte range in HBM holding, for its
// rows, the factor entries column-major (value, dependency position), the
// source index of the right-hand side, and for U the destination row and the
// inverted diagonal.  Rows of a level are sorted longest first and every warp
// gets its own segment width, so little FP64 work is spent on padding.
// Nothing on a level's critical path waits for HBM:
//   - an issuer warp streams chunks into a ring of shared-memory stages with
//     cp.async.bulk (the TMA bulk-copy engine) completing on mbarriers, S
//     chunks ahead of the solving warps;
//   - a gatherer warp, once a chunk has landed, gathers its right-hand sides
//     (L pass: from r; U pass: from the L results, once the L pass is
//     complete) with 4- or 8-byte cp.async completing on a per-stage
//     mbarrier -- a separate warp, so that a stage the issuer waits to
//     refill never holds back the gathers of chunks already in flight;
//   - solved values of the last few levels live in a shared-memory ring
//     indexed by level-major position (the setup checks that every
//     dependency of a chunk lies within the ring's window; passes whose
//     window does not fit read dependencies from the global scratch).
// Levels are separated by a barrier of the solving warps only -- no
// grid-wide synchronisation.  Every wait is bounded: a wait that runs out
// sets the device error word, one thread waits (bounded) for the copies still
// in flight, and the CTA returns.
#include <mutex>

#include "ptx.cuh"
#include "reduce.cuh"

namespace hec {

// Barrier of the consumer warps only (named barrier 1), OR-reducing a flag.
__device__ __forceinline__ int consumer_sync_or(int flag)
{
    int any;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.s32 p, %1, 0;\n\t"
                 "barrier.cta.red.or.pred q, 1, %2, p;\n\t"
                 "selp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(any)
                 : "r"(flag), "n"(kThreads)
                 : "memory");
    return any;
}

// Shared memory of one CTA: S stages, S right-hand-side slots of kThreads
// values, the ring, and 3 S + 1 mbarriers.  vbytes: 8 (FP64) or 4 (FP32).
size_t trsv_smem_bytes(int stage_bytes, int nstages, int ring_slots, int vbytes)
{
    return (size_t)stage_bytes * nstages + (size_t)nstages * kThreads * vbytes +
           (size_t)ring_slots * vbytes + (size_t)(3 * nstages + 1) * sizeof(uint64_t);
}

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

// Drain bound for copies already issued when a wait ran out: copies complete
// in microseconds, this only guarantees that the CTA never waits forever.
constexpr long long kDrainPolls = 1ll << 24;

// A chunk in shared memory (layout written by the setup's packer; T is the
// value type, double or float):
//   [0, 16)   nrows, nwarps, first position, flags (bit 0: U pass)
//   [16, 48)  width of every warp's segment
//   [48, 80)  byte offset of every warp's segment
//   [80, 96)  byte offsets of src, dst, dinv
//   per warp w < nwarps: val[width_w][stride_w] (T), dep[width_w][stride_w] (int32),
//     stride_w = 32 for a full warp, the row count rounded up to 4 for the last one
//   src[r32(nrows)] (int32), and for U: dst[r32(nrows)] (int32), dinv[r32(nrows)] (T)
constexpr int kWarpRows = 32;
constexpr int kMaxWarps = kThreads / kWarpRows;

__device__ __forceinline__ int seg_stride(int w, int nrows)
{
    const int left = nrows - w * kWarpRows;
    return left >= kWarpRows ? kWarpRows : (left + 3) & ~3;
}

template <class T> struct ChunkView {
    int nrows, nwarps, base;
    bool upass;
    const int *src, *dst;
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
    v.src = reinterpret_cast<const int *>(ch + off.x);
    v.dst = reinterpret_cast<const int *>(ch + off.y);
    v.dinv = reinterpret_cast<const T *>(ch + off.z);
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

// s - sum_k val[k] * y[dep[k]] for one row in ascending column order, width W
// known at compile time: every shared-memory load of the row is issued before
// the first multiply.  One accumulator: in FP64 the pipe's throughput, not
// the 64-cycle latency of a dependent DFMA, bounds a level once several warps
// are busy, and a second accumulator would cost one more FP64 add per row.
template <int W, bool RING, class T>
__device__ __forceinline__ T row_solve(const Segment<T> &g, int lane, const T *ring, int mask,
                                       const T *gdep, T s)
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
            y[k] = RING ? ring[d[k] & mask] : gdep[d[k]];
#pragma unroll
        for (int k = 0; k < W; ++k)
            s = fma(-l[k], y[k], s);
        return s;
    }
}

template <bool RING, class T>
__device__ __forceinline__ T row_solve_any(const Segment<T> &g, int lane, const T *ring, int mask,
                                           const T *gdep, T s)
{
    switch (g.width) {
    case 0: return s;
    case 1: return row_solve<1, RING>(g, lane, ring, mask, gdep, s);
    case 2: return row_solve<2, RING>(g, lane, ring, mask, gdep, s);
    case 3: return row_solve<3, RING>(g, lane, ring, mask, gdep, s);
    case 4: return row_solve<4, RING>(g, lane, ring, mask, gdep, s);
    case 5: return row_solve<5, RING>(g, lane, ring, mask, gdep, s);
    case 6: return row_solve<6, RING>(g, lane, ring, mask, gdep, s);
    case 7: return row_solve<7, RING>(g, lane, ring, mask, gdep, s);
    case 8: return row_solve<8, RING>(g, lane, ring, mask, gdep, s);
    default: {
        // wide rows: loads in blocks of 8 entries
        int k = 0;
        for (; k + 8 <= g.width; k += 8) {
            T l[8], y[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                l[q] = g.val[(k + q) * g.stride + lane];
                const int d = g.dep[(k + q) * g.stride + lane];
                y[q] = RING ? ring[d & mask] : gdep[d];
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                s = fma(-l[q], y[q], s);
        }
        for (; k < g.width; ++k) {
            const int d = g.dep[k * g.stride + lane];
            s = fma(-g.val[k * g.stride + lane], RING ? ring[d & mask] : gdep[d], s);
        }
        return s;
    }
    }
}

// Warp-specialised CTA: warps 0-7 solve rows (one row per thread per chunk),
// warps 8 and 9 feed them.  Per chunk c in stage s = c mod S:
//   issuer (warp 8): wait empty[s] (chunk c - S released) -> arm full[s] with
//             the chunk's byte count -> cp.async.bulk the chunk;
//   gatherer (warp 9): wait full[s] -> gather the chunk's right-hand sides
//             into slot s with cp.async (a U chunk waits for ldone first: its
//             right-hand side is the L pass's output); ready[s] completes
//             when the 32 lanes' gathers have landed (cp.async arrivals) and
//             lane 0 -- which has seen the chunk's data land -- has arrived,
//             so one barrier covers both;
//   consumers: wait ready[s] -> solve -> consumer barrier ->
//             one thread releases empty[s] (and ldone after the last L chunk).
// T = double: the FP64 path; T = float: the FP32 inner solves of the
// mixed-precision mode (FP32 factors, products and accumulation).
template <class T, int FW>
__global__ void __launch_bounds__(kThreads + 64, 1) k_trsv_ras(TrsvArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    count_launch(a.st);
    if (a.st && a.st->skip)
        return;
    const T *r = reinterpret_cast<const T *>(a.r);
    if (a.r_from_j)
        r += (int64_t)a.st->j * a.ldv;

    const TrsvBlock blk = a.blocks[blockIdx.x];
    const int S = a.nstages;
    unsigned char *stages = smem;
    T *rhs = reinterpret_cast<T *>(smem + (size_t)S * a.stage_bytes);
    T *ring = rhs + (size_t)S * kThreads;
    const int mask = a.ring_mask;
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + mask + 1);
    uint64_t *empty = full + S;
    uint64_t *ready = empty + S;
    uint64_t *ldone = ready + S;
    const int nch = blk.chunk_end - blk.chunk_begin;
    const int nL = blk.chunk_mid - blk.chunk_begin; // chunks of the L pass
    const bool stall_test = a.spin_limit < 0;       // fault injection: nothing is issued
    const long long limit = stall_test ? -a.spin_limit : a.spin_limit;
    const uint2 *chunks = a.chunks + blk.chunk_begin;
    T *ysc_w = reinterpret_cast<T *>(a.ysc) + blk.yoff;
    const T *ysc = ysc_w;
    T *zsc = a.zsc ? reinterpret_cast<T *>(a.zsc) + blk.zoff : nullptr;
    T *z = reinterpret_cast<T *>(a.z);
    const int t = threadIdx.x;

    if (t == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&ready[s], 33); // 32 gather arrivals + 1 data arrival
        }
        mbar_init(ldone, 1);
        fence_mbar_init();
    }
    for (int i = t; i <= mask; i += blockDim.x)
        ring[i] = T(0);
    __syncthreads();

    // shared state of the two feeding warps (written before the final barrier)
    __shared__ int s_issued;
    if (t == 0)
        s_issued = 0;
    __syncthreads();
    int failed = 0;

    if (t >= kThreads && t < kThreads + 32 && !stall_test) {
        // ------------------------------------------------------------ issuer warp
        // streams chunk c into stage c mod S once the consumers released it
        const int lane = t - kThreads;
        uint2 win = make_uint2(0, 0);
        int wbase = -64;
        for (int c = 0; c < nch; ++c) {
            const int s = c % S;
            if (c >= wbase + 32) { // 32 descriptors per warp-wide load
                wbase = c;
                win = (c + lane < nch) ? chunks[c + lane] : make_uint2(0, 0);
            }
            const unsigned off16 = __shfl_sync(0xffffffffu, win.x, c - wbase);
            const unsigned bytes = __shfl_sync(0xffffffffu, win.y, c - wbase);
            // every wait decision is a warp vote: the lanes must stay converged
            if (c >= S &&
                __any_sync(0xffffffffu,
                           !bounded_wait(&empty[s], (uint32_t)((c / S) - 1) & 1u, limit))) {
                failed = 1;
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(stages + (size_t)s * a.stage_bytes, a.pack + (size_t)off16 * 16, bytes,
                         &full[s]);
                s_issued = c + 1;
            }
        }
    } else if (t >= kThreads + 32 && !stall_test) {
        // ------------------------------------------------------------ gatherer warp
        // follows the chunks as they land: gathers each one's right-hand sides
        const int lane = t - kThreads - 32;
        bool ldone_seen = false;
        for (int g = 0; g < nch; ++g) {
            const int sg = g % S;
            if (__any_sync(0xffffffffu, !bounded_wait(&full[sg], (uint32_t)(g / S) & 1u, limit))) {
                failed = 1;
                break;
            }
            const ChunkView<T> v = view_chunk<T>(stages + (size_t)sg * a.stage_bytes);
            if (v.upass && !ldone_seen) {
                if (__any_sync(0xffffffffu, !bounded_wait(ldone, 0u, limit))) {
                    failed = 1;
                    break;
                }
                ldone_seen = true;
            }
            T *slot = rhs + (size_t)sg * kThreads;
            for (int i = lane; i < v.nrows; i += 32)
                cp_async_v<sizeof(T)>(&slot[i], v.upass ? ysc + v.src[i] : r + v.src[i]);
            cp_async_arrive_noinc(&ready[sg]); // when this lane's gathers land
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&ready[sg]); // the chunk's data has landed (seen above)
        }
        cp_async_wait_all();
    } else if (t < kThreads) {
    // ---------------------------------------------------------------- consumer warps
    int err = 0;
    int s = 0;
    uint32_t par = 0;
    for (int c = 0; c < nch; ++c) {
        if (!bounded_wait(&ready[s], par, limit))
            err = 1;
        // results leave the critical path: global stores are issued after the
        // stage is released, so the release does not wait for them
        T out = T(0);
        T *gout = nullptr;
        if (!err) {
            const unsigned char *ch = stages + (size_t)s * a.stage_bytes;
            const ChunkView<T> v = view_chunk<T>(ch);
            if (t < v.nrows) {
                const bool rm = v.upass ? blk.ring_U : blk.ring_L;
                const T *gdep = v.upass ? zsc : ysc;
                const int lane = t % kWarpRows;
                T sacc = rhs[(size_t)s * kThreads + t];
                if constexpr (FW > 0) {
                    // uniform-width layout: every warp's segment is FW entries
                    // wide, so this thread's entries sit at a compile-time
                    // offset from the chunk (all warps before the last are
                    // full) and the row needs no width dispatch
                    const int w = t / kWarpRows;
                    const int stride = seg_stride(w, v.nrows);
                    const T *val = reinterpret_cast<const T *>(
                                       ch + 96 + (size_t)w * FW * kWarpRows * (sizeof(T) + 4)) +
                                   lane;
                    const int *dep = reinterpret_cast<const int *>(val - lane + FW * stride) + lane;
                    T l[FW], y[FW];
                    int d[FW];
#pragma unroll
                    for (int k = 0; k < FW; ++k) {
                        l[k] = val[k * stride];
                        d[k] = dep[k * stride];
                    }
                    if (rm) {
#pragma unroll
                        for (int k = 0; k < FW; ++k)
                            y[k] = ring[d[k] & mask];
                    } else {
                        // the padding of a dependency-free row points at the
                        // chunk's first position, which this apply has not
                        // written yet in the global scratch (it may hold
                        // anything, NaN included): entries of value 0 are
                        // not read
#pragma unroll
                        for (int k = 0; k < FW; ++k)
                            y[k] = l[k] != T(0) ? gdep[d[k]] : T(0);
                    }
#pragma unroll
                    for (int k = 0; k < FW; ++k)
                        sacc = fma(-l[k], y[k], sacc);
                } else {
                    const Segment<T> g = warp_segment<T>(ch, v.nrows, t / kWarpRows);
                    sacc = rm ? row_solve_any<true, T>(g, lane, ring, mask, gdep, sacc)
                              : row_solve_any<false, T>(g, lane, ring, mask, gdep, sacc);
                }
                const int pos = v.base + t;
                if (v.upass) {
                    sacc *= v.dinv[t];
                    if (rm)
                        ring[pos & mask] = sacc;
                    else
                        zsc[pos] = sacc; // read by later levels of this pass
                    const int d = v.dst[t];
                    if (d >= 0)
                        gout = z + d;
                } else {
                    if (rm) {
                        ring[pos & mask] = sacc;
                        gout = ysc_w + pos;
                    } else {
                        ysc_w[pos] = sacc; // read by later levels of this pass
                    }
                }
                out = sacc;
            }
        }
        if (consumer_sync_or(err)) {
            failed = 1; // the feeding warps' own waits run out
            break;
        }
        // the release falls to the last thread: warp 7 holds the shortest rows
        if (t == kThreads - 1)
            mbar_arrive(&empty[s]); // stage s and its right-hand-side slot are free
        if (gout)
            *gout = out;
        if (c == nL - 1) {
            // every y of the L pass is written before the gatherer reads
            // the U pass's right-hand sides from them
            consumer_sync_or(0);
            if (t == kThreads - 1)
                mbar_arrive(ldone);
        }
        if (++s == S) {
            s = 0;
            par ^= 1u;
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
}

// The dynamic shared memory limit is a process-wide attribute of the kernel:
// raised once to the device's opt-in maximum, so that launches of different
// sizes from several host threads never race on it.
template <class T, int FW> static cudaError_t prepare_trsv()
{
    static std::once_flag once;
    static cudaError_t e = cudaSuccess;
    std::call_once(once, []() {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaFuncAttributes fa{};
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, k_trsv_ras<T, FW>);
        if (e == cudaSuccess)  // the opt-in limit covers static and dynamic shared memory
            e = cudaFuncSetAttribute(k_trsv_ras<T, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
    });
    return e;
}

template <class T, int FW> static int launch_t(const TrsvArgs &a, cudaStream_t s)
{
    const size_t smem = trsv_smem_bytes(a.stage_bytes, a.nstages, a.ring_mask + 1, sizeof(T));
    if (prepare_trsv<T, FW>() != cudaSuccess)
        return -1;
    k_trsv_ras<T, FW><<<a.nblocks, kThreads + 64, smem, s>>>(a);
    return 0;
}

int launch_trsv(const TrsvArgs &a, cudaStream_t s, bool fp32)
{
    if (!fp32)
        return launch_t<double, 0>(a, s);
    switch (a.fixed_width) { // FP32 layouts padded to a uniform width
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
