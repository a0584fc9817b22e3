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
// inverted diagonal.  Chunks stream into a ring of shared-memory stages with
// cp.async.bulk (the TMA bulk-copy engine) completing on mbarriers, several
// chunks ahead of the wavefront, so the factor bytes are in shared memory
// when their level becomes ready.  Solved values of the last few levels live
// in a shared-memory ring indexed by level-major position (the setup checks
// that every dependency of a level lies within the ring's window); blocks
// whose window does not fit read dependencies from the global scratch
// instead.  Levels are separated by CTA barriers only -- no grid-wide
// synchronisation.  Every wait is bounded: a wait that runs out sets the
// device error word, the CTA waits (bounded) for its own copies in flight,
// and returns.
#include "reduce.cuh"

namespace hec {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                 "%2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool bounded_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

size_t trsv_smem_bytes(int stage_bytes, int nstages, int ring_slots)
{
    return (size_t)stage_bytes * nstages + (size_t)ring_slots * sizeof(double) +
           (size_t)nstages * sizeof(uint64_t);
}

// Drain bound for copies already issued when a wait ran out: copies complete
// in microseconds, this only guarantees that the CTA never waits forever.
constexpr long long kDrainPolls = 1ll << 24;

__global__ void __launch_bounds__(kThreads, 1) k_trsv_ras(TrsvArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    count_launch(a.st);
    if (a.st && a.st->skip)
        return;
    const double *r = a.r;
    if (a.r_from_j)
        r += (int64_t)a.st->j * a.ldv;

    const TrsvBlock blk = a.blocks[blockIdx.x];
    const int S = a.nstages;
    unsigned char *stages = smem;
    double *ring = reinterpret_cast<double *>(smem + (size_t)S * a.stage_bytes);
    const int mask = a.ring_mask;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ring + mask + 1);
    const int nch = blk.chunk_end - blk.chunk_begin;
    const bool stall_test = a.spin_limit < 0; // fault-injection: nothing is issued
    const long long limit = stall_test ? -a.spin_limit : a.spin_limit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s)
            mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i <= mask; i += blockDim.x)
        ring[i] = 0.0;
    __syncthreads();

    if (threadIdx.x == 0 && !stall_test) {
        const int pro = nch < S ? nch : S;
        for (int c = 0; c < pro; ++c) {
            const uint2 d = a.chunks[blk.chunk_begin + c];
            mbar_arrive_expect_tx(&bar[c], d.y);
            bulk_g2s(stages + (size_t)c * a.stage_bytes, a.pack + (size_t)d.x * 16, d.y, &bar[c]);
        }
    }

    const double *ysc = a.ysc + blk.yoff;
    double *ysc_w = a.ysc + blk.yoff;
    double *zsc = a.zsc ? a.zsc + blk.zoff : nullptr;

    int failed_at = -1;
    for (int c = 0; c < nch; ++c) {
        const int s = c % S;
        const uint32_t par = (uint32_t)(c / S) & 1u;
        int err = bounded_wait(&bar[s], par, limit) ? 0 : 1;
        if (!err) {
            const unsigned char *ch = stages + (size_t)s * a.stage_bytes;
            const int4 hdr = *reinterpret_cast<const int4 *>(ch);
            const int nrows = hdr.x, width = hdr.y, base = hdr.z;
            const bool upass = (hdr.w & 1) != 0;
            const int nr2 = (nrows + 1) & ~1, nr4 = (nrows + 3) & ~3;
            const double *val = reinterpret_cast<const double *>(ch + 16);
            const int *dep = reinterpret_cast<const int *>(val + (size_t)width * nr2);
            const int *src = dep + (size_t)width * nr4;
            const int *dst = src + nr4;
            const double *dinv = reinterpret_cast<const double *>(dst + nr4);
            const bool rm = upass ? blk.ring_U : blk.ring_L;
            const double *gdep = upass ? zsc : ysc;
            for (int t = threadIdx.x; t < nrows; t += blockDim.x) {
                double sacc = upass ? ysc[src[t]] : r[src[t]];
                if (rm) {
                    for (int k = 0; k < width; ++k)
                        sacc = fma(-val[k * nr2 + t], ring[dep[k * nr4 + t] & mask], sacc);
                } else {
                    for (int k = 0; k < width; ++k)
                        sacc = fma(-val[k * nr2 + t], gdep[dep[k * nr4 + t]], sacc);
                }
                const int pos = base + t;
                if (upass) {
                    sacc *= dinv[t];
                    if (rm)
                        ring[pos & mask] = sacc;
                    else
                        zsc[pos] = sacc;
                    const int d = dst[t];
                    if (d >= 0)
                        a.z[d] = sacc;
                } else {
                    if (rm)
                        ring[pos & mask] = sacc;
                    ysc_w[pos] = sacc;
                }
            }
        }
        if (__syncthreads_or(err)) {
            failed_at = c;
            break;
        }
        if (threadIdx.x == 0 && c + S < nch) {
            fence_proxy_async_smem(); // generic reads of stage s before the async write
            const uint2 d = a.chunks[blk.chunk_begin + c + S];
            mbar_arrive_expect_tx(&bar[s], d.y);
            bulk_g2s(stages + (size_t)s * a.stage_bytes, a.pack + (size_t)d.x * 16, d.y, &bar[s]);
        }
    }
    if (failed_at >= 0) {
        // copies issued for chunks failed_at .. failed_at + S - 1 may be in flight
        if (threadIdx.x == 0) {
            if (!stall_test) {
                const int last = (failed_at + S < nch) ? failed_at + S : nch;
                for (int c = failed_at; c < last; ++c)
                    bounded_wait(&bar[c % S], (uint32_t)(c / S) & 1u, kDrainPolls);
            }
            atomicExch(a.err, HEC_ERR_TIMEOUT);
            if (a.st)
                a.st->err = HEC_ERR_TIMEOUT;
        }
        __syncthreads();
    }
}

int launch_trsv(const TrsvArgs &a, cudaStream_t s)
{
    const size_t smem = trsv_smem_bytes(a.stage_bytes, a.nstages, a.ring_mask + 1);
    cudaError_t e = cudaFuncSetAttribute(k_trsv_ras, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return -1;
    k_trsv_ras<<<a.nblocks, kThreads, smem, s>>>(a);
    return 0;
}

} // namespace hec
