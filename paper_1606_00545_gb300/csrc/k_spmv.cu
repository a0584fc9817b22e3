// k_spmv.cu -- SpMV on the HEC format (Section 2.1-2.2, Algorithm 1, Eq. 2).
//
// The paper runs the ELL part with one thread per row and then the CSR part
// with one thread per row.  Here one launch does both: every CTA walks tiles
// of 512 consecutive rows; a thread owns two adjacent rows, so each slab
// column is read with one vector load of values (double2 / float2) and one
// 64-bit load of column indices (int2), coalesced across the warp because the
// slab is column-major with a leading dimension that is a multiple of 256
// rows.  Tail rows of a tile (rows longer than the slab width K) are summed
// first, one warp per row with a shuffle reduction, into shared memory, then
// added to the slab sum of their row.  The result goes through the Eq. 2
// epilogue and, optionally, up to two dot products of the output are reduced
// in the same launch (deterministic order, see reduce.cuh).  T = double is
// the FP64 path; T = float is the FP32 inner solve of the mixed-precision
// mode (FP32 products and accumulation; the dots' cross-CTA sums in FP64).
#include "reduce.cuh"

namespace hec {

template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

template <class T>
__device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int MODE, int NDOT, bool TAIL, class T>
__global__ void __launch_bounds__(kThreads) k_spmv_hec(SpmvArgs a)
{
    using T2 = typename Vec2<T>::type;
    count_launch(a.st);
    if (a.st && a.st->skip)
        return; // uniform across the grid: set before this launch
    __shared__ T s_tail[TAIL ? kSpmvTile : 1];
    T acc[NDOT > 0 ? NDOT : 1];
#pragma unroll
    for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d)
        acc[d] = T(0);
    const T2 *__restrict__ val2 = reinterpret_cast<const T2 *>(a.ell_val);
    const int2 *__restrict__ col2 = reinterpret_cast<const int2 *>(a.ell_col);
    const T *__restrict__ x = reinterpret_cast<const T *>(a.x);
    const T *y_in = reinterpret_cast<const T *>(a.y_in);
    T *y_out = reinterpret_cast<T *>(a.y_out);
    const T *tail_val = reinterpret_cast<const T *>(a.tail_val);
    const T alpha = T(a.alpha), beta = T(a.beta);
    const int ld2 = a.ld >> 1;

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int base = tile * kSpmvTile;
        const int r0 = base + 2 * threadIdx.x;
        if (TAIL) {
            s_tail[2 * threadIdx.x] = T(0);
            s_tail[2 * threadIdx.x + 1] = T(0);
            __syncthreads();
            const int t0 = a.tile_tail[tile], t1 = a.tile_tail[tile + 1];
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            // short rows: groups of g lanes, 32 / g rows per warp at a time,
            // reduced by xor shuffles inside each aligned group of g lanes
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
            // long rows: the whole CTA, one row at a time, fixed-order sum
            for (int q = a.tile_long[tile]; q < a.tile_long[tile + 1]; ++q) {
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
            T s0 = T(0), s1 = T(0);
            const int p0 = r0 >> 1;
#pragma unroll 4
            for (int k = 0; k < a.K; ++k) {
                const T2 v = __ldg(&val2[(size_t)k * ld2 + p0]);
                const int2 c = __ldg(&col2[(size_t)k * ld2 + p0]);
                s0 = fma(v.x, __ldg(&x[c.x]), s0);
                s1 = fma(v.y, __ldg(&x[c.y]), s1);
            }
            if (TAIL) {
                s0 += s_tail[2 * threadIdx.x];
                s1 += s_tail[2 * threadIdx.x + 1];
            }
            const bool two = (r0 + 1 < a.n);
            T y0, y1;
            if (MODE == 0) {
                y0 = s0;
                y1 = s1;
            } else if (MODE == 1) {
                y0 = alpha * s0;
                y1 = alpha * s1;
            } else {
                y0 = fma(alpha, s0, beta * y_in[r0]);
                y1 = two ? fma(alpha, s1, beta * y_in[r0 + 1]) : T(0);
            }
            if (two) {
                T2 out;
                out.x = y0;
                out.y = y1;
                *reinterpret_cast<T2 *>(&y_out[r0]) = out;
            } else {
                y_out[r0] = y0;
                y1 = T(0);
            }
            if (NDOT >= 1) {
                const T *w = reinterpret_cast<const T *>(a.w0);
                T q0 = w ? w[r0] : y0;
                T q1 = two ? (w ? w[r0 + 1] : y1) : T(0);
                acc[0] = fma(q0, y0, acc[0]);
                acc[0] = fma(q1, y1, acc[0]);
            }
            if (NDOT >= 2) {
                const T *w = reinterpret_cast<const T *>(a.w1);
                T q0 = w ? w[r0] : y0;
                T q1 = two ? (w ? w[r0 + 1] : y1) : T(0);
                acc[1] = fma(q0, y0, acc[1]);
                acc[1] = fma(q1, y1, acc[1]);
            }
        }
        if (TAIL)
            __syncthreads(); // s_tail is rewritten by the next tile
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
