// k_refactor.cu -- numeric refactorisation on the GPU: a matrix with the same
// sparsity pattern and new values replaces the old one without a host round
// trip.  The HEC slab and tail take the new values (Section 2.1), every RAS
// block's ILU(k) factor is recomputed on its existing fill pattern by the
// IKJ elimination of Algorithm 2 (the pattern -- Eqs. 9-10 -- does not depend
// on the values), scheduled by the L level sets of Eq. 11 (a row's
// elimination reads only rows of lower levels), and the triangular-solve
// layouts get the new factor values.
//
// The elimination performs exactly the host's operations in the host's
// order -- per row, pivots p ascending; l_ip = a_ip / u_pp; a_ij -= l_ip u_pj
// for the j of row p's U part that row i holds -- with separately rounded
// multiply and subtract (no contraction, as the host code is compiled), so
// the factors are bit-identical to a host factorisation of the new matrix.
#include "reduce.cuh"

namespace hec {

// New CSR values -> slab / tail slots: slot >= 0 is an ELL slot, slot < 0 the
// tail entry -slot - 1.
__global__ void k_scatter_hec(int64_t nnz, const double *val, const int64_t *slot, double *ell,
                              double *tail)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = slot[e];
        if (s >= 0)
            ell[s] = val[e];
        else
            tail[-s - 1] = val[e];
    }
}

__global__ void k_cast_f32(int64_t n, const double *x, float *y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

// Factor entries start from A's values on the original pattern, 0 on fill.
__global__ void k_gather_factor(int64_t nent, const double *val, const int *src, double *f)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nent;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = src[e];
        f[e] = s >= 0 ? val[s] : 0.0;
    }
}

// Rows of at most kLocalRow entries are eliminated in per-thread arrays:
// the row is read once and written once, and its merges against the pivot
// rows read only the pivot rows from memory.  Longer rows run the same steps
// on global memory.
constexpr int kLocalRow = 48;

__device__ __forceinline__ bool eliminate_row_local(const RefactorArgs &a, int row0, int r)
{
    const int b0 = a.rp[r], len = a.rp[r + 1] - b0, nl = a.dg[r] - b0;
    int ci[kLocalRow];
    double f[kLocalRow];
    for (int q = 0; q < len; ++q) {
        ci[q] = a.ci[b0 + q];
        f[q] = a.f[b0 + q];
    }
    bool ok = true;
    for (int k = 0; k < nl; ++k) {
        const int p = row0 + ci[k]; // pivot row
        const int dp = a.dg[p], ep = a.rp[p + 1];
        const double upp = a.f[dp];
        if (upp == 0.0) {
            ok = false;
            break;
        }
        const double lip = __ddiv_rn(f[k], upp);
        f[k] = lip;
        // row i's entries right of p against row p's U part (both ascending)
        int x = k + 1, y = dp + 1;
        int cy = y < ep ? a.ci[y] : 0x7fffffff;
        double fy = y < ep ? a.f[y] : 0.0;
        while (x < len && y < ep) {
            const int cx = ci[x];
            if (cx == cy) {
                f[x] = __dsub_rn(f[x], __dmul_rn(lip, fy));
                ++x;
                ++y;
                if (y < ep) {
                    cy = a.ci[y];
                    fy = a.f[y];
                }
            } else if (cx < cy) {
                ++x;
            } else {
                ++y;
                if (y < ep) {
                    cy = a.ci[y];
                    fy = a.f[y];
                }
            }
        }
    }
    for (int q = 0; q < len; ++q)
        a.f[b0 + q] = f[q];
    return ok && f[nl] != 0.0;
}

__device__ __forceinline__ bool eliminate_row_global(const RefactorArgs &a, int row0, int r)
{
    double *f = a.f;
    const int end_i = a.rp[r + 1];
    for (int e = a.rp[r]; e < a.dg[r]; ++e) {
        const int p = row0 + a.ci[e]; // pivot row
        const double upp = f[a.dg[p]];
        if (upp == 0.0)
            return false;
        const double lip = __ddiv_rn(f[e], upp);
        f[e] = lip;
        int x = e + 1, y = a.dg[p] + 1;
        const int end_p = a.rp[p + 1];
        while (x < end_i && y < end_p) {
            const int cx = a.ci[x], cy = a.ci[y];
            if (cx == cy) {
                f[x] = __dsub_rn(f[x], __dmul_rn(lip, f[y]));
                ++x;
                ++y;
            } else if (cx < cy) {
                ++x;
            } else {
                ++y;
            }
        }
    }
    return f[a.dg[r]] != 0.0;
}

// One CTA per RAS block, one thread per row of the current L level, a CTA
// barrier between levels.  Row data is global-entry indexed: row r (global
// over all blocks) holds entries [rp[r], rp[r+1]), local columns ci, its
// diagonal at dg[r].  Within a row the pivots are taken in ascending order
// and each update is a separately rounded multiply and subtract: the host's
// operations in the host's order.
__global__ void __launch_bounds__(kThreads) k_iluk_numeric(RefactorArgs a)
{
    const int b = blockIdx.x;
    const int row0 = a.blk_row0[b];
    const int *lptr = a.lptr + a.blk_lev0[b];
    const int nlev = a.blk_lev0[b + 1] - a.blk_lev0[b] - 1;
    const int *lrows = a.lrows + row0;
    for (int l = 0; l < nlev; ++l) {
        for (int q = lptr[l] + threadIdx.x; q < lptr[l + 1]; q += blockDim.x) {
            const int r = row0 + lrows[q];
            const bool ok = (a.rp[r + 1] - a.rp[r] <= kLocalRow)
                                ? eliminate_row_local(a, row0, r)
                                : eliminate_row_global(a, row0, r);
            if (!ok)
                atomicExch(a.err, HEC_ERR_ZERO_PIVOT);
        }
        __syncthreads();
    }
}

// The triangular-solve layout's value slots from the new factor values: one
// CTA per chunk, thread t on row t.  Row t of chunk c takes the factor
// entries [start, start + len) of its pass (L: the multipliers; U: the
// entries right of the diagonal) and, for U, 1 / u_tt.  The chunk formats
// of trsv_layout.cpp: fixed-slot (flag bit 3: every row padded to FW entries,
// 16-byte vectors per lane in per-warp blocks; bit 5: the resident kernel's
// blocks, with 16-bit slots) and generic (per-warp widths).
template <class T> __global__ void __launch_bounds__(kThreads) k_fill_pack(FillArgs a)
{
    const int c = blockIdx.x;
    unsigned char *ch = a.pack + (size_t)a.chunks[c].x * 16;
    const int *hdr = reinterpret_cast<const int *>(ch);
    const int nrows = hdr[0];
    const bool upass = (hdr[3] & 1) != 0;
    const int t = threadIdx.x;
    if (t >= nrows)
        return;
    const int w = t / 32, lane = t % 32;
    const int64_t q = a.chunk_row0[c] + t;
    const int start = a.rm_start[q], len = a.rm_len[q];
    if (hdr[3] & 8) { // fixed-slot: 16-byte vectors of VW values per lane
        const int FW = hdr[6];
        constexpr int vb = (int)sizeof(T), VW = 16 / vb;
        const int NV = (FW + VW - 1) / VW;
        int blk, dinv_off;
        if (hdr[3] & 32) { // resident format: index vectors of 8 uint16, every block with dinv
            const int NI = (FW + 1 + 7) / 8;
            dinv_off = (NV + NI) * 512;
            blk = dinv_off + 32 * vb;
        } else {
            const bool exps = (hdr[3] & 16) != 0;
            const int ND = (FW + 3) / 4;
            dinv_off = (NV + ND) * 512;
            blk = dinv_off + 128 + (upass ? 32 * vb + 128 : 0) + (exps ? 128 : 0);
        }
        T *val = reinterpret_cast<T *>(ch + 32 + (size_t)w * blk);
        for (int k = 0; k < NV * VW; ++k)
            val[(k / VW) * 32 * VW + lane * VW + k % VW] = k < len ? T(a.f[start + k]) : T(0);
        if (upass)
            reinterpret_cast<T *>(ch + 32 + (size_t)w * blk + dinv_off)[lane] =
                T(__ddiv_rn(1.0, a.f[a.rm_diag[q]]));
        return;
    }
    const int left = nrows - w * 32;
    const int stride = left >= 32 ? 32 : (left + 3) & ~3;
    const int width = hdr[4 + w];
    T *val = reinterpret_cast<T *>(ch + hdr[4 + 8 + w]);
    for (int k = 0; k < width; ++k)
        val[k * stride + lane] = k < len ? T(a.f[start + k]) : T(0);
    if (upass) {
        T *dinv = reinterpret_cast<T *>(ch + hdr[4 + 16 + 2]);
        dinv[t] = T(__ddiv_rn(1.0, a.f[a.rm_diag[q]]));
    }
}

__global__ void k_jacobi_dinv(int n, const double *val, const int64_t *diag, double omega,
                              double *dinv, float *dinv32, int *err)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = val[diag[i]];
        if (d == 0.0)
            atomicExch(err, HEC_ERR_ZERO_PIVOT);
        const double v = __ddiv_rn(omega, d);
        dinv[i] = v;
        if (dinv32)
            dinv32[i] = (float)v;
    }
}

static int grid_of(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 4096); }

int launch_scatter_hec(int64_t nnz, const double *val, const int64_t *slot, double *ell,
                       double *tail, cudaStream_t s)
{
    k_scatter_hec<<<grid_of(nnz), 256, 0, s>>>(nnz, val, slot, ell, tail);
    return 0;
}

int launch_cast_f32(int64_t n, const double *x, float *y, cudaStream_t s)
{
    if (n > 0)
        k_cast_f32<<<grid_of(n), 256, 0, s>>>(n, x, y);
    return 0;
}

int launch_refactor(const RefactorArgs &a, int nblocks, cudaStream_t s)
{
    k_gather_factor<<<grid_of(a.nent), 256, 0, s>>>(a.nent, a.val, a.src, a.f);
    k_iluk_numeric<<<nblocks, kThreads, 0, s>>>(a);
    return 0;
}

int launch_fill_pack(const FillArgs &a, int nchunks, bool fp32, cudaStream_t s)
{
    if (nchunks <= 0)
        return 0;
    if (fp32)
        k_fill_pack<float><<<nchunks, kThreads, 0, s>>>(a);
    else
        k_fill_pack<double><<<nchunks, kThreads, 0, s>>>(a);
    return 0;
}

int launch_jacobi_dinv(int n, const double *val, const int64_t *diag, double omega, double *dinv,
                       float *dinv32, int *err, cudaStream_t s)
{
    k_jacobi_dinv<<<grid_of(n), 256, 0, s>>>(n, val, diag, omega, dinv, dinv32, err);
    return 0;
}

} // namespace hec
