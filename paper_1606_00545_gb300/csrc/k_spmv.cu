// k_spmv.cu -- SpMV on the HEC format (Section 2.1-2.2, Algorithm 1, Eq. 2).
//
// The paper runs the ELL part with one thread per row and then the CSR part
// with one thread per row.  Here one launch does both.  A thread owns RPT
// adjacent rows -- 2 in FP64, 4 in FP32 -- so each slab column is read with
// one 16-byte load of values (double2 / float4) and one load of column
// indices (int2 / int4), coalesced across the warp because the slab is
// column-major with a leading dimension that is a multiple of 32 rows, and
// streamed with an evict-first L2 policy so that x stays in L2.  A CTA
// walks row blocks of kThreads * RPT rows (one 512-row tile in FP64, two in
// FP32).  Tail rows of a block (rows longer than the slab width K) are summed
// first into shared memory, then added to the slab sum of their row: short
// tail rows by groups of 4-32 lanes (the group size the setup chose for the
// tile from its mean tail length) with xor-shuffle sums, rows longer than
// kSpmvLongRow by the whole CTA in a fixed order.  The result goes through
// the Eq. 2 epilogue and, optionally, up to two dot products of the output
// are reduced in the same launch (deterministic order, see reduce.cuh).
// T = double is the FP64 path; T = float is the FP32 inner solve of the
// mixed-precision mode (FP32 products and accumulation; the dots' cross-CTA
// sums in FP64).
#include "reduce.cuh"

namespace hec {

// Loads of the slab stream: no L1 allocation and an evict-first L2 policy,
// so the slab (read once per SpMV) does not push x -- gathered at random,
// and small enough to stay in L2 -- out of it.  Measured on the 128^3 and
// 96^3 cases: 9-12% faster in FP64, 17% in FP32.
__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ double2 ld_stream(const double2 *p, uint64_t pol)
{
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4 *p, uint64_t pol)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int2 ld_stream(const int2 *p, uint64_t pol)
{
    int2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int4 ld_stream(const int4 *p, uint64_t pol)
{
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
    return v;
}

// RPT adjacent rows per thread, read with 16-byte value vectors.
template <class T> struct RowVec;
template <> struct RowVec<double> {
    static constexpr int RPT = 2;
    using V = double2;
    using C = int2;
    __device__ static double get(const V &v, int j) { return j == 0 ? v.x : v.y; }
    __device__ static int col(const C &c, int j) { return j == 0 ? c.x : c.y; }
    __device__ static void put(double *p, const double *y) { *reinterpret_cast<V *>(p) = make_double2(y[0], y[1]); }
};
template <> struct RowVec<float> {
    static constexpr int RPT = 4;
    using V = float4;
    using C = int4;
    __device__ static float get(const V &v, int j)
    {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    }
    __device__ static int col(const C &c, int j)
    {
        return j == 0 ? c.x : j == 1 ? c.y : j == 2 ? c.z : c.w;
    }
    __device__ static void put(float *p, const float *y)
    {
        *reinterpret_cast<V *>(p) = make_float4(y[0], y[1], y[2], y[3]);
    }
};

template <class T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row blocks of one CTA pass: kThreads * RPT rows, i.e. RPT / 2 SpMV tiles.
template <class T> constexpr int spmv_tiles_per_block() { return RowVec<T>::RPT / 2; }

template <int MODE, int NDOT, bool TAIL, class T>
__global__ void __launch_bounds__(kThreads) k_spmv_hec(SpmvArgs a)
{
    using RV = RowVec<T>;
    constexpr int RPT = RV::RPT, TPB = RPT / 2, BR = kThreads * RPT;
    count_launch(a.st);
    if (a.st && a.st->skip)
        return; // uniform across the grid: set before this launch
    __shared__ T s_tail[TAIL ? BR : 1];
    T acc[NDOT > 0 ? NDOT : 1];
#pragma unroll
    for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d)
        acc[d] = T(0);
    const typename RV::V *__restrict__ valv = reinterpret_cast<const typename RV::V *>(a.ell_val);
    const typename RV::C *__restrict__ colv = reinterpret_cast<const typename RV::C *>(a.ell_col);
    const T *__restrict__ x = reinterpret_cast<const T *>(a.x);
    const T *y_in = reinterpret_cast<const T *>(a.y_in);
    T *y_out = reinterpret_cast<T *>(a.y_out);
    const T *tail_val = reinterpret_cast<const T *>(a.tail_val);
    const T alpha = T(a.alpha), beta = T(a.beta);
    const int ldv = a.ld / RPT; // the leading dimension is a multiple of 32 rows
    const int nblk = (a.ntiles + TPB - 1) / TPB;

    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int base = blk * BR;
        const int r0 = base + RPT * threadIdx.x;
        if (TAIL) {
#pragma unroll
            for (int j = 0; j < RPT; ++j)
                s_tail[RPT * threadIdx.x + j] = T(0);
            __syncthreads();
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            const int tile0 = blk * TPB, tile1 = min(tile0 + TPB, a.ntiles);
            for (int tile = tile0; tile < tile1; ++tile) {
                // short rows: groups of g lanes, 32 / g rows per warp at a
                // time, reduced by xor shuffles inside each aligned group
                const int t0 = a.tile_tail[tile], t1 = a.tile_tail[tile + 1];
                const int g = a.tile_group[tile];
                const int rpw = 32 / g, gid = lane / g, lig = lane % g;
                for (int tb = t0 + wid * rpw; tb < t1; tb += (kThreads / 32) * rpw) {
                    const int t = tb + gid;
                    T s = T(0);
                    bool mine = false;
                    if (t < t1) {
                        const int e0 = a.tail_ptr[t], e1 = a.tail_ptr[t + 1];
                        mine = e1 - e0 <= kSpmvLongRow;
                        if (mine)
                            for (int e = e0 + lig; e < e1; e += g)
                                s += tail_val[e] * __ldg(&x[a.tail_col[e]]);
                    }
                    for (int o = g >> 1; o > 0; o >>= 1)
                        s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (mine && lig == 0)
                        s_tail[a.tail_rows[t] - base] = s;
                }
            }
            // long rows: the whole CTA, one row at a time, fixed-order sum
            for (int q = a.tile_long[tile0]; q < a.tile_long[tile1]; ++q) {
                const int t = a.tail_long[q];
                T s = T(0);
                for (int e = a.tail_ptr[t] + threadIdx.x; e < a.tail_ptr[t + 1]; e += kThreads)
                    s += tail_val[e] * __ldg(&x[a.tail_col[e]]);
                s = warp_sum_t(s);
                __shared__ T s_red[kThreads / 32];
                __syncthreads(); // s_red of the previous long row is read
                if (lane == 0)
                    s_red[wid] = s;
                __syncthreads();
                if (threadIdx.x == 0) {
                    T tot = T(0);
                    for (int w = 0; w < kThreads / 32; ++w)
                        tot += s_red[w];
                    s_tail[a.tail_rows[t] - base] = tot;
                }
            }
            __syncthreads();
        }
        if (r0 < a.n) {
            T s[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j)
                s[j] = T(0);
            const int p0 = r0 / RPT;
            const uint64_t pol = evict_first_policy();
#pragma unroll 4
            for (int k = 0; k < a.K; ++k) {
                const typename RV::V v = ld_stream(&valv[(size_t)k * ldv + p0], pol);
                const typename RV::C c = ld_stream(&colv[(size_t)k * ldv + p0], pol);
#pragma unroll
                for (int j = 0; j < RPT; ++j)
                    s[j] = fma(RV::get(v, j), __ldg(&x[RV::col(c, j)]), s[j]);
            }
            const int nr = min(RPT, a.n - r0); // rows of this thread inside the matrix
            T y[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                if (TAIL)
                    s[j] += s_tail[RPT * threadIdx.x + j];
                if (MODE == 0)
                    y[j] = s[j];
                else if (MODE == 1)
                    y[j] = alpha * s[j];
                else
                    y[j] = j < nr ? fma(alpha, s[j], beta * y_in[r0 + j]) : T(0);
            }
            if (nr == RPT) {
                RV::put(&y_out[r0], y);
            } else {
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    if (j < nr)
                        y_out[r0 + j] = y[j];
                    else
                        y[j] = T(0);
                }
            }
#pragma unroll
            for (int d = 0; d < NDOT; ++d) {
                const T *w = reinterpret_cast<const T *>(d == 0 ? a.w0 : a.w1);
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const T q = j < nr ? (w ? w[r0 + j] : y[j]) : T(0);
                    acc[d] = fma(q, y[j], acc[d]);
                }
            }
        }
        if (TAIL)
            __syncthreads(); // s_tail is rewritten by the next row block
    }
    if constexpr (NDOT > 0) {
        double v[NDOT];
#pragma unroll
        for (int d = 0; d < NDOT; ++d)
            v[d] = double(acc[d]);
        reduce_and_finalize<NDOT>(v, a.red, a.op, a.result, a.st);
    }
}

template <int MODE, int NDOT, class T>
static void launch_t(const SpmvArgs &a, bool tail, int grid, cudaStream_t s)
{
    if (tail)
        k_spmv_hec<MODE, NDOT, true, T><<<grid, kThreads, 0, s>>>(a);
    else
        k_spmv_hec<MODE, NDOT, false, T><<<grid, kThreads, 0, s>>>(a);
}

int launch_spmv(const SpmvArgs &a, int mode, int ndot, bool has_tail, int grid, cudaStream_t s,
                bool fp32)
{
#define HEC_SPMV_CASE(M, D)                                                                      \
    if (mode == M && ndot == D) {                                                                \
        if (fp32)                                                                                \
            launch_t<M, D, float>(a, has_tail, grid, s);                                         \
        else                                                                                     \
            launch_t<M, D, double>(a, has_tail, grid, s);                                        \
        return 0;                                                                                \
    }
    HEC_SPMV_CASE(0, 0)
    HEC_SPMV_CASE(0, 1)
    HEC_SPMV_CASE(0, 2)
    HEC_SPMV_CASE(1, 0)
    HEC_SPMV_CASE(1, 1)
    HEC_SPMV_CASE(1, 2)
    HEC_SPMV_CASE(2, 0)
    HEC_SPMV_CASE(2, 1)
    HEC_SPMV_CASE(2, 2)
#undef HEC_SPMV_CASE
    return -1;
}

} // namespace hec
