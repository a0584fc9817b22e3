// k_spmv.cu -- SpMV on the HEC format (Section 2.1-2.2, Algorithm 1, Eq. 2).
//
// The paper runs the ELL part with one thread per row and then the CSR part
// with one thread per row.  Here one launch does both: every CTA walks tiles
// of 512 consecutive rows; a thread owns two adjacent rows, so each slab
// column is read with one 128-bit load of values (double2) and one 64-bit
// load of column indices (int2), coalesced across the warp because the slab
// is column-major with a leading dimension that is a multiple of 256 rows.
// Tail rows of a tile (rows longer than the slab width K) are summed first,
// one warp per row with a shuffle reduction, into shared memory, then added
// to the slab sum of their row.  The result goes through the Eq. 2 epilogue
// and, optionally, up to two dot products of the output are reduced in the
// same launch (deterministic order, see reduce.cuh).
#include "reduce.cuh"

namespace hec {

template <int MODE, int NDOT, bool TAIL>
__global__ void __launch_bounds__(kThreads) k_spmv_hec(SpmvArgs a)
{
    count_launch(a.st);
    if (a.st && a.st->skip)
        return; // uniform across the grid: set before this launch
    __shared__ double s_tail[TAIL ? kSpmvTile : 1];
    double acc[NDOT > 0 ? NDOT : 1];
#pragma unroll
    for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d)
        acc[d] = 0.0;
    const double2 *__restrict__ val2 = reinterpret_cast<const double2 *>(a.ell_val);
    const int2 *__restrict__ col2 = reinterpret_cast<const int2 *>(a.ell_col);
    const double *__restrict__ x = a.x;
    const int ld2 = a.ld >> 1;

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int base = tile * kSpmvTile;
        const int r0 = base + 2 * threadIdx.x;
        if (TAIL) {
            s_tail[2 * threadIdx.x] = 0.0;
            s_tail[2 * threadIdx.x + 1] = 0.0;
            __syncthreads();
            const int t0 = a.tile_tail[tile], t1 = a.tile_tail[tile + 1];
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            for (int t = t0 + wid; t < t1; t += kThreads / 32) {
                double s = 0.0;
                for (int e = a.tail_ptr[t] + lane; e < a.tail_ptr[t + 1]; e += 32)
                    s += a.tail_val[e] * __ldg(&x[a.tail_col[e]]);
                s = warp_sum(s);
                if (lane == 0)
                    s_tail[a.tail_rows[t] - base] = s;
            }
            __syncthreads();
        }
        if (r0 < a.n) {
            double s0 = 0.0, s1 = 0.0;
            const int p0 = r0 >> 1;
#pragma unroll 4
            for (int k = 0; k < a.K; ++k) {
                const double2 v = __ldg(&val2[(size_t)k * ld2 + p0]);
                const int2 c = __ldg(&col2[(size_t)k * ld2 + p0]);
                s0 = fma(v.x, __ldg(&x[c.x]), s0);
                s1 = fma(v.y, __ldg(&x[c.y]), s1);
            }
            if (TAIL) {
                s0 += s_tail[2 * threadIdx.x];
                s1 += s_tail[2 * threadIdx.x + 1];
            }
            const bool two = (r0 + 1 < a.n);
            double y0, y1;
            if (MODE == 0) {
                y0 = s0;
                y1 = s1;
            } else if (MODE == 1) {
                y0 = a.alpha * s0;
                y1 = a.alpha * s1;
            } else {
                y0 = fma(a.alpha, s0, a.beta * a.y_in[r0]);
                y1 = two ? fma(a.alpha, s1, a.beta * a.y_in[r0 + 1]) : 0.0;
            }
            if (two) {
                *reinterpret_cast<double2 *>(&a.y_out[r0]) = make_double2(y0, y1);
            } else {
                a.y_out[r0] = y0;
                y1 = 0.0;
            }
            if (NDOT >= 1) {
                const double *w = a.w0;
                double q0 = w ? w[r0] : y0;
                double q1 = two ? (w ? w[r0 + 1] : y1) : 0.0;
                acc[0] = fma(q0, y0, acc[0]);
                acc[0] = fma(q1, y1, acc[0]);
            }
            if (NDOT >= 2) {
                const double *w = a.w1;
                double q0 = w ? w[r0] : y0;
                double q1 = two ? (w ? w[r0 + 1] : y1) : 0.0;
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
            v[d] = acc[d];
        reduce_and_finalize<NDOT>(v, a.red, a.op, a.result, a.st);
    }
}

template <int MODE, int NDOT>
static void launch_t(const SpmvArgs &a, bool tail, int grid, cudaStream_t s)
{
    if (tail)
        k_spmv_hec<MODE, NDOT, true><<<grid, kThreads, 0, s>>>(a);
    else
        k_spmv_hec<MODE, NDOT, false><<<grid, kThreads, 0, s>>>(a);
}

int launch_spmv(const SpmvArgs &a, int mode, int ndot, bool has_tail, int grid, cudaStream_t s)
{
#define HEC_SPMV_CASE(M, D)                                                                      \
    if (mode == M && ndot == D) {                                                                \
        launch_t<M, D>(a, has_tail, grid, s);                                                     \
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
