// k_batch.cu -- the batched solver: one persistent launch solves many
// independent systems, one system (and up to NR right-hand sides of it in
// lockstep) per CTA, start to finish, with no further launch and no grid-wide
// synchronisation.
//
// Per system, a CTA runs right-preconditioned restarted GMRES(m) (Section
// 2.7) on A_s M_s^{-1}, M_s = L_s U_s the ILU(k) factors of A_s (Eqs. 9-10,
// Algorithm 2), as FP64 iterative refinement around inner cycles in the inner
// type T (float for the mixed form, double for the plain one):
//   cycle:  r = b - A x in FP64, beta = ||r||;  v_0 = r / beta in T
//           Arnoldi in T: z = M^{-1} v_j (level-scheduled L and U passes,
//           Eq. 11, Algorithm 3), w = A z (HEC: ELL slab + CSR tail, Eq. 2,
//           Algorithm 1), classical Gram-Schmidt with a second projection
//           when the first leaves ||w'|| < ||w|| / sqrt(2) (the Daniel-
//           Gragg-Kaufman-Stewart test; the first update and the second
//           projection's dot products share one read of the basis), Givens
//           rotations and least squares in FP64;
//           the cycle ends when |g_{j+1}| <= max(inner_rtol beta, tol ||b||)
//           x += M^{-1} (V y) with the update added in FP64.
// The basis is kept unnormalised: v_i = sig_i * V_i, and sig_i is applied
// where v_i is read (in the dot products, the update coefficients and the
// scaling of the L pass's right-hand side), so no pass rescales a vector.
//
// Vectors hold the system's unknowns in the level order of L, NR values
// (one per right-hand side) per position, so a level's rows are consecutive:
// the right-hand sides of a triangular-solve chunk are one contiguous slice
// that the bulk-copy engine fetches with the chunk's factor entries, S chunks
// ahead; solved values live in a shared-memory ring indexed by position.
// The Krylov basis is stored tile-interleaved (tile = CTA-size elements of
// every slot, contiguous), so the Gram-Schmidt passes stream whole tiles of
// all slots into shared memory with one bulk copy each, several tiles ahead:
// the bytes in flight per SM do not depend on registers.  One thread issues
// every bulk copy: lane 0 of the last warp, which holds no row of a chunk of
// up to (CTA size - 32) rows, so issuing stays off the solving threads' path.
// Every wait is bounded; a wait that runs out sets the error word, drains the
// copies in flight and ends the CTA.
#include <mutex>
#include <set>

#include "../../include/hecgpu.h"
#include "batch.cuh"
#include "ptx.cuh"

namespace hec {
namespace {

constexpr long long kBatchDrainPolls = 1ll << 24;

// Scalars of a right-hand side's state.
enum { SC_BETA = 0, SC_BNORM, SC_BCYCLE, SC_EST, SC_WW, SC_W2, SC_ACTIVE, SC_BROKE,
       SC_RUN = 8 /* cycles in a row whose true residual exceeded 10x the estimate */,
       SC_STAG = 9 };
// Shared integers.
enum { MI_SYS = 0, MI_STOP };

template <class T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void ld(const float *p, float (&v)[4])
    {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        v[0] = f.x;
        v[1] = f.y;
        v[2] = f.z;
        v[3] = f.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void ld(const double *p, double (&v)[4])
    {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&v)[4])
    {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

// The NR values of one position.
template <class T, int NR> __device__ __forceinline__ void ldn(const T *p, T (&v)[NR])
{
    if constexpr (NR == 4) {
        Vec4<T>::ld(p, v);
    } else if constexpr (NR == 2) {
        if constexpr (sizeof(T) == 4) {
            const float2 f = *reinterpret_cast<const float2 *>(p);
            v[0] = f.x;
            v[1] = f.y;
        } else {
            const double2 f = *reinterpret_cast<const double2 *>(p);
            v[0] = f.x;
            v[1] = f.y;
        }
    } else {
        v[0] = *p;
    }
}

template <class T, int NR> __device__ __forceinline__ void stn(T *p, const T (&v)[NR])
{
    if constexpr (NR == 4) {
        Vec4<T>::st(p, v);
    } else if constexpr (NR == 2) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        else
            *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

// Sums N values (N a power of two <= 32) over a warp: lane l returns the warp
// sum of v[l % N].  N - 1 shuffles halve the vector at every step (each lane
// keeps the half its lane bit selects), then the lanes holding equal indices
// are summed.  Fixed order: deterministic.
template <int N, class V> __device__ __forceinline__ V warp_transpose_sum(V (&v)[N], int lane)
{
#pragma unroll
    for (int off = N / 2; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const V send = up ? v[i] : v[i + off];
            const V keep = up ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    V s = v[0];
#pragma unroll
    for (int off = N; off < 32; off <<= 1)
        s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

template <class V> __device__ __forceinline__ V warp_allsum(V x)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// A ring of bulk-copy stages.  Every thread keeps the consumer state (next
// stage, parity of each stage's next completion, copies consumed); the
// issuing thread also keeps its own stage cursor and issue count.
struct Pipe {
    int S = 1, cst = 0, ist = 0, issued = 0, consumed = 0;
    uint32_t cpar = 0;
    __device__ void start_pass()
    {
        issued = 0;
        consumed = 0;
    }
    __device__ int next_issue()
    {
        const int s = ist;
        ist = ist + 1 == S ? 0 : ist + 1;
        ++issued;
        return s;
    }
    __device__ void advance()
    {
        cpar ^= 1u << cst;
        cst = cst + 1 == S ? 0 : cst + 1;
        ++consumed;
    }
};

template <class T, int NR> struct Batch {
    const BatchArgs &a;
    int tid, nt, lane, warp, nw, tshift, issuer;
    unsigned char *stages;
    T *ring;
    uint64_t *full, *full2;
    void *red;
    void *out;
    T *coef;
    double *dbl;
    int *misc;
    T *V, *z, *yU;
    double *xp, *bp, *R;
    Pipe tp, sp;
    BatchSys s;
    long long nE, Ep;
    int ntiles;

    __device__ Batch(const BatchArgs &args, unsigned char *smem) : a(args)
    {
        tid = threadIdx.x;
        nt = blockDim.x;
        lane = tid & 31;
        warp = tid >> 5;
        nw = nt >> 5;
        tshift = 31 - __clz(nt);
        issuer = nt - 32;  // lane 0 of the last warp: rows of a chunk go to the first threads
        const BatchSmem L = batch_smem(a.nstages, a.stage_bytes, a.sstages, a.sbytes,
                                       a.ring_mask + 1, NR, (int)sizeof(T), a.m, nt);
        stages = smem + L.stage;
        ring = reinterpret_cast<T *>(smem + L.ring);
        full = reinterpret_cast<uint64_t *>(smem + L.bar);
        full2 = reinterpret_cast<uint64_t *>(smem + L.bar2);
        red = smem + L.red;
        out = smem + L.out;
        coef = reinterpret_cast<T *>(smem + L.coef);
        dbl = reinterpret_cast<double *>(smem + L.dbl);
        misc = reinterpret_cast<int *>(smem + L.misc);
        unsigned char *w = a.ws + (size_t)blockIdx.x * a.ws_stride;
        V = reinterpret_cast<T *>(w);
        z = reinterpret_cast<T *>(w + a.offZ);
        yU = reinterpret_cast<T *>(w + a.offY);
        xp = reinterpret_cast<double *>(w + a.offX);
        bp = reinterpret_cast<double *>(w + a.offB);
        R = reinterpret_cast<double *>(w + a.offR);
        tp.S = a.nstages;
        sp.S = a.sstages;
    }

    // The basis is tile-interleaved: tile t (nt elements) of slots 0..m is
    // one contiguous block, so one bulk copy brings every slot of a tile.
    __device__ T *vel(int slot, long long e) const
    {
        return V + ((((size_t)(e >> tshift)) * (a.m + 1) + slot) << tshift) + (e & (nt - 1));
    }

    struct RhsView {
        double *h, *h2, *cs, *sn, *g, *y, *sig, *sc;
    };
    __device__ RhsView rv(int r) const
    {
        const int m = a.m;
        double *p = dbl + (size_t)r * batch_rhs_doubles(m);
        RhsView v;
        v.h = p;
        v.h2 = v.h + (m + 2);
        v.cs = v.h2 + (m + 2);
        v.sn = v.cs + (m + 1);
        v.g = v.sn + (m + 1);
        v.y = v.g + (m + 2);
        v.sig = v.y + (m + 1);
        v.sc = v.sig + (m + 2);
        return v;
    }

    // Block-wide sums of N values per thread (N <= 32, power of two) into
    // out[0..N); ends with a barrier, out is then readable by every thread.
    template <int N, class W> __device__ void block_sum(W (&v)[N])
    {
        W *rd = reinterpret_cast<W *>(red);
        W *o = reinterpret_cast<W *>(out);
        const W s_ = warp_transpose_sum<N, W>(v, lane);
        if (lane < N)
            rd[warp * N + lane] = s_;
        __syncthreads();
        if (tid < N) {
            W t = 0;
            for (int w = 0; w < nw; ++w)
                t += rd[w * N + tid];
            o[tid] = t;
        }
        __syncthreads();
    }

    // Sums v[i] (i < 32) over the threads of each right-hand side (a thread's
    // elements all belong to right-hand side tid % NR) into out[i * NR + q].
    // Halving over the lane bits above log2(NR) leaves lane l with NR values,
    // indices c + (l & ~(NR - 1)), summed over the lanes of its right-hand
    // side; the warps' values are then added in a fixed order.
    __device__ void reduce32(T (&v)[32])
    {
        T *rd = reinterpret_cast<T *>(red);
        T *o = reinterpret_cast<T *>(out);
#pragma unroll
        for (int off = 16; off >= NR; off >>= 1) {
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < off; ++i) {
                const T send = up ? v[i] : v[i + off];
                const T keep = up ? v[i + off] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c)
            rd[(warp * 32 + lane) * NR + c] = v[c];
        __syncthreads();
        for (int k = tid; k < 32 * NR; k += nt) {
            const int i = k / NR, q = k % NR;
            const int l = (i & ~(NR - 1)) | q, c = i & (NR - 1);
            T t = T(0);
            for (int w = 0; w < nw; ++w)
                t += rd[(w * 32 + l) * NR + c];
            o[k] = t;
        }
        __syncthreads();
    }

    // ------------------------------------------------------------- HEC SpMV
    // y = bvec - A x in FP64 (bvec may be null: y = -A x); y is written to
    // basis slot `slot` (ys == null) or to the plain array ys; per-rhs partial
    // sums of y^2 in part.  Rows of the slab one per thread, rows of the tail
    // one per warp with a shuffle reduction.
    template <class TO>
    __device__ void resid64(const double *bvec, const double *x, int slot, TO *ys, double (&part)[NR])
    {
        const int *col = a.ell_col + s.ell;
        const double *val = a.ell_val64 + s.ell;
        auto put = [&](int p, const double (&acc)[NR]) {
            TO o[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                o[r] = (TO)acc[r];
                part[r] += acc[r] * acc[r];
            }
            if (ys)
                stn<TO, NR>(ys + (size_t)p * NR, o);
            else
                stn<TO, NR>(reinterpret_cast<TO *>(vel(slot, (long long)p * NR)), o);
        };
        for (int p = tid; p < s.n; p += nt) {
            const int c0 = col[p];
            if (c0 < 0)
                continue;
            double acc[NR];
            if (bvec)
                ldn<double, NR>(bvec + (size_t)p * NR, acc);
            else
                for (int r = 0; r < NR; ++r)
                    acc[r] = 0.0;
#pragma unroll 4
            for (int k = 0; k < s.K; ++k) {
                const int cc = k ? col[(size_t)k * s.ld + p] : c0;
                const double v = val[(size_t)k * s.ld + p];
                double xv[NR];
                ldn<double, NR>(x + (size_t)cc * NR, xv);
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    acc[r] -= v * xv[r];
            }
            put(p, acc);
        }
        const int *trow = a.tail_rows + s.tail;
        const long long *tptr = a.tail_ptr + s.tptr;
        for (int t = warp; t < s.ntail; t += nw) {
            const int p = trow[t];
            double acc[NR];
            for (int r = 0; r < NR; ++r)
                acc[r] = 0.0;
            for (long long e = tptr[t] + lane; e < tptr[t + 1]; e += 32) {
                const double v = a.tail_val64[e];
                double xv[NR];
                ldn<double, NR>(x + (size_t)a.tail_col[e] * NR, xv);
                for (int r = 0; r < NR; ++r)
                    acc[r] += v * xv[r];
            }
            for (int r = 0; r < NR; ++r)
                acc[r] = warp_allsum(acc[r]);
            if (lane == 0) {
                double bv[NR];
                if (bvec)
                    ldn<double, NR>(bvec + (size_t)p * NR, bv);
                for (int r = 0; r < NR; ++r)
                    acc[r] = (bvec ? bv[r] : 0.0) - acc[r];
                put(p, acc);
            }
        }
    }

    // Basis slot `slot` = A x in the inner type (x: a plain array).
    __device__ void spmv_in(const T *x, int slot)
    {
        const int *col = a.ell_col + s.ell;
        const T *val = static_cast<const T *>(a.ell_val) + s.ell;
        for (int p = tid; p < s.n; p += nt) {
            const int c0 = col[p];
            if (c0 < 0)
                continue;
            T acc[NR];
            for (int r = 0; r < NR; ++r)
                acc[r] = T(0);
#pragma unroll 4
            for (int k = 0; k < s.K; ++k) {
                const int cc = k ? col[(size_t)k * s.ld + p] : c0;
                const T v = val[(size_t)k * s.ld + p];
                T xv[NR];
                ldn<T, NR>(x + (size_t)cc * NR, xv);
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    acc[r] += v * xv[r];
            }
            stn<T, NR>(vel(slot, (long long)p * NR), acc);
        }
        const int *trow = a.tail_rows + s.tail;
        const long long *tptr = a.tail_ptr + s.tptr;
        const T *tval = static_cast<const T *>(a.tail_val);
        for (int t = warp; t < s.ntail; t += nw) {
            const int p = trow[t];
            T acc[NR];
            for (int r = 0; r < NR; ++r)
                acc[r] = T(0);
            for (long long e = tptr[t] + lane; e < tptr[t + 1]; e += 32) {
                const T v = tval[e];
                T xv[NR];
                ldn<T, NR>(x + (size_t)a.tail_col[e] * NR, xv);
                for (int r = 0; r < NR; ++r)
                    acc[r] += v * xv[r];
            }
            for (int r = 0; r < NR; ++r)
                acc[r] = warp_allsum(acc[r]);
            if (lane == 0)
                stn<T, NR>(vel(slot, (long long)p * NR), acc);
        }
    }

    // ------------------------------------------------- bulk-copy pipes
    // The issuing thread, after a wait ran out: wait (bounded) for every copy
    // still in flight so that none lands after the CTA has left.
    __device__ void drain(const Pipe &P, uint64_t *bars)
    {
        if (tid != issuer)
            return;
        int st = P.cst;
        for (int k = P.consumed; k < P.issued; ++k) {
            bounded_wait(&bars[st], (P.cpar >> st) & 1u, kBatchDrainPolls);
            st = st + 1 == P.S ? 0 : st + 1;
        }
        atomicExch(a.err, HEC_ERR_TIMEOUT);
    }

    // Right-hand side of a triangular pass: a basis slot or a plain array.
    struct Src {
        const T *base;
        int slot;  // >= 0: basis slot; < 0: base
    };

    __device__ void issue_chunk(const BChunk &ch, const Src &src)
    {
        const int st = tp.next_issue();
        unsigned char *dst = stages + (size_t)st * a.stage_bytes;
        constexpr long long epb = 16 / sizeof(T);  // elements per 16 bytes
        const long long e0 = (long long)ch.first * NR, e1 = (long long)(ch.first + ch.nrows) * NR;
        const long long lo = e0 & ~(epb - 1), hi = (e1 + epb - 1) & ~(epb - 1);
        mbar_arrive_expect_tx(&full[st], (uint32_t)(ch.bytes + (hi - lo) * sizeof(T)));
        bulk_g2s(dst, a.fac + (size_t)ch.off16 * 16, (uint32_t)ch.bytes, &full[st]);
        unsigned char *rd = dst + a.ent_bytes;
        if (src.slot < 0) {
            bulk_g2s(rd, src.base + lo, (uint32_t)((hi - lo) * sizeof(T)), &full[st]);
        } else {
            // a slice of a basis slot: one copy per tile it touches
            for (long long p = lo; p < hi;) {
                const long long tend = ((p >> tshift) + 1) << tshift;
                const long long q = tend < hi ? tend : hi;
                bulk_g2s(rd + (p - lo) * sizeof(T), vel(src.slot, p), (uint32_t)((q - p) * sizeof(T)),
                         &full[st]);
                p = q;
            }
        }
    }

    // One pass over chunks [c0, c0 + nch): rows of the chunk solve
    //   L: y = scale * rhs - sum l_ij y_j          (unit diagonal)
    //   U: z = (rhs - sum u_ij z_j) / u_ii
    // reading dependencies from the ring and writing every result to the ring
    // and to outv at the chunk's destination positions.  Returns false after
    // a wait ran out (the CTA must then end).
    template <bool UP>
    __device__ bool tri_pass(int c0, int nch, const Src &src, const T (&scale)[NR], T *outv,
                             bool fence_out)
    {
        const int S = tp.S;
        tp.start_pass();
        BChunk nxt{};
        if (tid == issuer) {
            const int pre = nch < S ? nch : S;
            for (int i = 0; i < pre; ++i)
                issue_chunk(a.chunks[c0 + i], src);
            if (pre < nch)
                nxt = a.chunks[c0 + pre];
        }
        constexpr long long epb = 16 / sizeof(T);
        for (int i = 0; i < nch; ++i) {
            const int st = tp.cst;
            const bool ok = bounded_wait(&full[st], (tp.cpar >> st) & 1u, a.spin_limit);
            if (ok) {
                const unsigned char *spp = stages + (size_t)st * a.stage_bytes;
                const int4 hdr = *reinterpret_cast<const int4 *>(spp);
                const int nrows = hdr.x, width = hdr.y, first = hdr.z;
                const int stride = (nrows + 3) & ~3;
                const int *dst = reinterpret_cast<const int *>(spp + 16);
                const int *dep = dst + stride;
                const T *val = reinterpret_cast<const T *>(dep + (size_t)width * stride);
                const T *dinv = val + (size_t)width * stride;
                const T *rhs = reinterpret_cast<const T *>(spp + a.ent_bytes) +
                               (((long long)first * NR) & (epb - 1));
                for (int r_ = tid; r_ < nrows; r_ += nt) {
                    T acc[NR];
                    ldn<T, NR>(rhs + (size_t)r_ * NR, acc);
                    if (!UP) {
#pragma unroll
                        for (int r = 0; r < NR; ++r)
                            acc[r] *= scale[r];
                    }
                    for (int k = 0; k < width; ++k) {
                        const int d = dep[k * stride + r_];
                        const T v = val[k * stride + r_];
                        T pv[NR];
                        ldn<T, NR>(ring + (size_t)d * NR, pv);
#pragma unroll
                        for (int r = 0; r < NR; ++r)
                            acc[r] -= v * pv[r];
                    }
                    if (UP) {
                        const T di = dinv[r_];
#pragma unroll
                        for (int r = 0; r < NR; ++r)
                            acc[r] *= di;
                    }
                    stn<T, NR>(ring + (size_t)((first + r_) & a.ring_mask) * NR, acc);
                    stn<T, NR>(outv + (size_t)dst[r_] * NR, acc);
                }
            }
            if (fence_out && i == nch - 1)
                fence_proxy_async_global();
            if (__syncthreads_or(!ok)) {
                drain(tp, full);
                return false;
            }
            tp.advance();
            if (tid == issuer && i + S < nch) {
                issue_chunk(nxt, src);
                if (i + S + 1 < nch)
                    nxt = a.chunks[c0 + i + S + 1];
            }
        }
        return true;
    }

    // z = M^{-1} (scale * src): L pass into yU, U pass into z.
    __device__ bool precond(const Src &src, const T (&scale)[NR])
    {
        if (s.nchL == 0) {  // no factor: z = scale * src
            for (long long e = tid; e < nE; e += nt)
                z[e] = (src.slot < 0 ? src.base[e] : *vel(src.slot, e)) * scale[e % NR];
            __syncthreads();
            return true;
        }
        if (!tri_pass<false>(s.chL, s.nchL, src, scale, yU, true))
            return false;
        return tri_pass<true>(s.chU, s.nchU, Src{yU, -1}, scale, z, false);
    }

    // Streams basis tiles 0 .. ntiles-1 (slots [0, nv) of each) through the
    // stage ring; body(stage, tile) runs on every thread, thread tid owning
    // element tid of the tile.
    __device__ void issue_tile(int t, uint32_t bytes)
    {
        const int st = sp.next_issue();
        mbar_arrive_expect_tx(&full2[st], bytes);
        bulk_g2s(stages + (size_t)st * a.sbytes, V + ((size_t)t * (a.m + 1) << tshift), bytes,
                 &full2[st]);
    }

    template <class F> __device__ bool stream(int nv, F &&body)
    {
        const uint32_t bytes = (uint32_t)((size_t)nv * sizeof(T)) << tshift;
        const int S = sp.S;
        sp.start_pass();
        if (tid == issuer)
            for (int t = 0; t < S && t < ntiles; ++t)
                issue_tile(t, bytes);
        for (int t = 0; t < ntiles; ++t) {
            const int st = sp.cst;
            const bool ok = bounded_wait(&full2[st], (sp.cpar >> st) & 1u, a.spin_limit);
            if (ok)
                body(reinterpret_cast<const T *>(stages + (size_t)st * a.sbytes), t);
            if (__syncthreads_or(!ok)) {
                drain(sp, full2);
                return false;
            }
            sp.advance();
            if (tid == issuer && t + S < ntiles)
                issue_tile(t + S, bytes);
        }
        return true;
    }

    // coef[i][u] = c_r[i] * sig_r[i], r = u % NR, from c = h, h2 or y.
    __device__ void set_coef(int cnt, int which)
    {
        for (int t = tid; t < cnt * 4; t += nt) {
            const int i = t / 4, r = (t % 4) % NR;
            RhsView v = rv(r);
            const double c = which == 0 ? v.h[i] : which == 1 ? v.h2[i] : v.y[i];
            coef[t] = (T)(c * v.sig[i]);
        }
        __syncthreads();
    }

    // h (or h2)[r][i] = sig[r][i] * sum, and the extra value 31 into sc[x]
    // (||w||^2 before or after the projection), from reduce32's out.
    __device__ void take_dots(int j, bool second, int scx)
    {
        const T *o = reinterpret_cast<const T *>(out);
        for (int k = tid; k < (j + 1) * NR; k += nt) {
            const int i = k / NR, r = k % NR;
            RhsView v = rv(r);
            (second ? v.h2 : v.h)[i] = v.sig[i] * (double)o[i * NR + r];
        }
        if (tid < NR)
            rv(tid).sc[scx] = (double)o[31 * NR + tid];
        __syncthreads();
    }

    // One Arnoldi step's orthogonalisation of w = basis slot j + 1 against
    // slots 0..j: classical Gram-Schmidt, projected twice unless the first
    // projection kept ||w'|| >= ||w|| / sqrt(2) for every right-hand side.
    //   pass 1: h = V^T w, ||w||^2
    //   pass 2: w' = w - V h; h2 = V^T w', ||w'||^2       (one read of V)
    //   pass 3: w'' = w' - V h2, ||w''||^2; h += h2       (when needed)
    __device__ bool orthogonalise(int j, int &reorth_steps)
    {
        const int u4 = tid & 3;
        const int wi = (j + 1) << tshift;
        {
            T acc[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                acc[i] = T(0);
            if (!stream(j + 2, [&](const T *st, int) {
                    const T w = st[wi + tid];
#pragma unroll
                    for (int i = 0; i < 31; ++i)
                        if (i <= j)
                            acc[i] += st[(i << tshift) + tid] * w;
                    acc[31] += w * w;
                }))
                return false;
            reduce32(acc);
            take_dots(j, false, SC_WW);
        }
        set_coef(j + 1, 0);
        {
            T acc[32];
#pragma unroll
            for (int i = 0; i < 32; ++i)
                acc[i] = T(0);
            if (!stream(j + 2, [&](const T *st, int t) {
                    T w = st[wi + tid];
#pragma unroll
                    for (int i = 0; i < 31; ++i)
                        if (i <= j)
                            w -= coef[i * 4 + u4] * st[(i << tshift) + tid];
#pragma unroll
                    for (int i = 0; i < 31; ++i)
                        if (i <= j)
                            acc[i] += st[(i << tshift) + tid] * w;
                    acc[31] += w * w;
                    V[(((size_t)t * (a.m + 1) + j + 1) << tshift) + tid] = w;
                }))
                return false;
            fence_proxy_async_global();
            reduce32(acc);
            take_dots(j, true, SC_W2);
        }
        bool reorth = false;
        for (int r = 0; r < NR; ++r) {
            RhsView v = rv(r);
            reorth |= v.sc[SC_ACTIVE] != 0.0 && v.sc[SC_W2] < 0.5 * v.sc[SC_WW];
        }
        if (reorth) {
            ++reorth_steps;
            set_coef(j + 1, 1);
            T w2[4] = {T(0), T(0), T(0), T(0)};
            if (!stream(j + 2, [&](const T *st, int t) {
                    T w = st[wi + tid];
#pragma unroll
                    for (int i = 0; i < 31; ++i)
                        if (i <= j)
                            w -= coef[i * 4 + u4] * st[(i << tshift) + tid];
                    w2[u4] += w * w;
                    V[(((size_t)t * (a.m + 1) + j + 1) << tshift) + tid] = w;
                }))
                return false;
            fence_proxy_async_global();
            block_sum<4, T>(w2);
            if (tid < NR) {
                const T *o = reinterpret_cast<const T *>(out);
                RhsView v = rv(tid);
                double t = 0.0;
                for (int u = 0; u < 4; ++u)
                    if (u % NR == tid)
                        t += (double)o[u];
                v.sc[SC_W2] = t;
                for (int i = 0; i <= j; ++i)
                    v.h[i] += v.h2[i];
            }
            __syncthreads();
        }
        return true;
    }

    // --------------------------------------------------------- one system
    __device__ void load_group(int g0)
    {
        const int *rop = a.row_of_pos + s.perm;
        for (long long e = tid; e < Ep; e += nt) {
            const long long p = e / NR;
            const int rr = g0 * NR + (int)(e % NR);
            double bv = 0.0, xv = 0.0;
            if (p < s.n && rr < a.nrhs) {
                const long long row = s.row0 + rop[p];
                bv = a.b[row * a.nrhs + rr];
                if (a.op == BOP_SOLVE && !a.x0_zero)
                    xv = a.x[row * a.nrhs + rr];
            }
            bp[e] = bv;
            xp[e] = xv;
        }
        // padding of every basis slot stays zero for the tile passes
        const long long pad = Ep - nE;
        for (long long t = tid; t < (long long)(a.m + 1) * pad; t += nt)
            *vel((int)(t / pad), nE + t % pad) = T(0);
        __syncthreads();
    }

    template <class G> __device__ void store_group(int g0, G &&get)
    {
        const int *rop = a.row_of_pos + s.perm;
        for (long long e = tid; e < nE; e += nt) {
            const long long p = e / NR;
            const int rr = g0 * NR + (int)(e % NR);
            if (rr < a.nrhs)
                a.x[(s.row0 + rop[p]) * a.nrhs + rr] = get(e);
        }
    }

    // Solves right-hand sides g0 * NR ... of the current system.  Returns
    // false when a wait ran out.  res: accumulated over the groups.
    __device__ bool solve_group(int g0, BatchResult &res)
    {
        load_group(g0);
        // ||b|| per right-hand side
        {
            double bb[4] = {0.0, 0.0, 0.0, 0.0};
            for (long long e = tid; e < Ep; e += nt)
                bb[e & 3] += bp[e] * bp[e];
            block_sum<4, double>(bb);
            if (tid < NR) {
                const double *o = reinterpret_cast<const double *>(out);
                double t = 0.0;
                for (int u = 0; u < 4; ++u)
                    if (u % NR == tid)
                        t += o[u];
                rv(tid).sc[SC_BNORM] = sqrt(t);
            }
            __syncthreads();
            // b = 0: the solution is 0
            for (long long e = tid; e < Ep; e += nt)
                if (rv((int)(e % NR)).sc[SC_BNORM] == 0.0)
                    xp[e] = 0.0;
            __syncthreads();
        }
        const int m = a.m;
        int steps = 0, cycles = 0, status = HEC_OK, reorth_steps = 0;
        double worst = 0.0;
        for (;;) {
            // ---- true residual in FP64; v_0 (unnormalised) in T
            {
                double part[NR];
                for (int r = 0; r < NR; ++r)
                    part[r] = 0.0;
                resid64<T>(bp, xp, 0, nullptr, part);
                fence_proxy_async_global();
                double pv[4] = {0.0, 0.0, 0.0, 0.0};
                for (int r = 0; r < NR; ++r)
                    pv[r] = part[r];
                block_sum<4, double>(pv);
            }
            if (tid < NR) {
                RhsView v = rv(tid);
                const double beta = sqrt(reinterpret_cast<const double *>(out)[tid]);
                const double bn = v.sc[SC_BNORM];
                const bool act = bn > 0.0 && !(beta <= a.tol * bn);
                // the previous FP32 cycle promised a residual of SC_EST: a
                // true FP64 residual far above it with less than a halving
                // over the cycle, two cycles in a row, means the FP32
                // arithmetic limits the refinement
                if (cycles == 0)
                    v.sc[SC_RUN] = 0.0;
                else if (v.sc[SC_ACTIVE] != 0.0)
                    v.sc[SC_RUN] = (v.sc[SC_EST] > 0.0 && beta > 10.0 * v.sc[SC_EST] &&
                                    beta > 0.5 * v.sc[SC_BCYCLE])
                                       ? v.sc[SC_RUN] + 1.0
                                       : 0.0;
                v.sc[SC_STAG] = (sizeof(T) == 4 && act && v.sc[SC_RUN] >= 2.0) ? 1.0 : 0.0;
                v.sc[SC_BETA] = beta;
                v.sc[SC_ACTIVE] = act ? 1.0 : 0.0;
                v.sc[SC_BCYCLE] = beta;
                v.sc[SC_BROKE] = 0.0;
                v.sig[0] = act ? 1.0 / beta : 0.0;
                v.g[0] = act ? beta : 0.0;
            }
            __syncthreads();
            bool any = false, bad = false, stag = false;
            worst = 0.0;
            for (int r = 0; r < NR; ++r) {
                RhsView v = rv(r);
                any |= v.sc[SC_ACTIVE] != 0.0;
                stag |= v.sc[SC_STAG] != 0.0;
                bad |= !isfinite(v.sc[SC_BETA]);
                const double rel = v.sc[SC_BNORM] > 0.0 ? v.sc[SC_BETA] / v.sc[SC_BNORM] : 0.0;
                worst = rel > worst ? rel : worst;
            }
            if (bad) {
                status = HEC_BREAKDOWN;
                break;
            }
            if (!any)
                break;
            if (stag) {
                status = kBatchStagnated;
                break;
            }
            if (steps >= a.maxit) {
                status = HEC_MAXIT;
                break;
            }
            ++cycles;
            int j = 0;
            for (;;) {
                T scale[NR];
                for (int r = 0; r < NR; ++r)
                    scale[r] = (T)rv(r).sig[j];
                if (!precond(Src{nullptr, j}, scale))
                    return false;
                spmv_in(z, j + 1);
                fence_proxy_async_global();
                __syncthreads();
                if (!orthogonalise(j, reorth_steps))
                    return false;
                // ---- Givens rotations and least-squares residual, FP64
                if (tid < NR) {
                    RhsView v = rv(tid);
                    if (v.sc[SC_ACTIVE] != 0.0) {
                        const double hn = sqrt(v.sc[SC_W2] > 0.0 ? v.sc[SC_W2] : 0.0);
                        const double tiny = (sizeof(T) == 4 ? 4.8e-7 : 8.9e-16) * sqrt(v.sc[SC_WW]);
                        const bool brk = !(hn > tiny);
                        v.sig[j + 1] = brk ? 0.0 : 1.0 / hn;
                        double *h = v.h;
                        for (int i = 0; i < j; ++i) {
                            const double t0 = v.cs[i] * h[i] + v.sn[i] * h[i + 1];
                            h[i + 1] = -v.sn[i] * h[i] + v.cs[i] * h[i + 1];
                            h[i] = t0;
                        }
                        const double den = hypot(h[j], hn);
                        const double c = den > 0.0 ? h[j] / den : 1.0;
                        const double sn = den > 0.0 ? hn / den : 0.0;
                        h[j] = den;
                        v.cs[j] = c;
                        v.sn[j] = sn;
                        v.g[j + 1] = -sn * v.g[j];
                        v.g[j] = c * v.g[j];
                        double *Rc = R + ((size_t)tid * (m + 1) + j) * (m + 1);
                        for (int i = 0; i <= j; ++i)
                            Rc[i] = h[i];
                        v.sc[SC_EST] = fabs(v.g[j + 1]);
                        v.sc[SC_BROKE] = brk ? 1.0 : 0.0;
                    } else {
                        v.sig[j + 1] = 0.0;
                    }
                }
                __syncthreads();
                ++steps;
                ++j;
                bool done = true;
                for (int r = 0; r < NR; ++r) {
                    RhsView v = rv(r);
                    if (v.sc[SC_ACTIVE] == 0.0 || v.sc[SC_BROKE] != 0.0)
                        continue;
                    const double lim1 = a.inner_rtol * v.sc[SC_BCYCLE];
                    const double lim2 = a.tol * v.sc[SC_BNORM];
                    if (!(v.sc[SC_EST] <= (lim1 > lim2 ? lim1 : lim2)))
                        done = false;
                }
                if (done || j == m || steps >= a.maxit)
                    break;
            }
            // ---- y = R^{-1} g per right-hand side (warp r), FP64
            if (warp < NR) {
                RhsView v = rv(warp);
                const bool act = v.sc[SC_ACTIVE] != 0.0;
                const double *Rr = R + (size_t)warp * (m + 1) * (m + 1);
                for (int i = j - 1; i >= 0; --i) {
                    double yi = 0.0;
                    if (lane == 0) {
                        const double d = Rr[(size_t)i * (m + 1) + i];
                        yi = act && d != 0.0 ? v.g[i] / d : 0.0;
                        v.y[i] = yi;
                    }
                    yi = __shfl_sync(0xffffffffu, yi, 0);
                    for (int k = lane; k < i; k += 32)
                        v.g[k] -= Rr[(size_t)i * (m + 1) + k] * yi;
                    __syncwarp();
                }
            }
            __syncthreads();
            // ---- u = sum y_i v_i (T) into slot j, z = M^{-1} u, x += z in FP64
            set_coef(j, 2);
            {
                const int u4 = tid & 3, jj = j;
                if (!stream(jj, [&](const T *st, int t) {
                        T u = T(0);
#pragma unroll
                        for (int i = 0; i < 31; ++i)
                            if (i < jj)
                                u += coef[i * 4 + u4] * st[(i << tshift) + tid];
                        V[(((size_t)t * (a.m + 1) + jj) << tshift) + tid] = u;
                    }))
                    return false;
                fence_proxy_async_global();
                __syncthreads();
                T one[NR];
                for (int r = 0; r < NR; ++r)
                    one[r] = T(1);
                if (!precond(Src{nullptr, jj}, one))
                    return false;
                for (long long e = tid; e < nE; e += nt)
                    xp[e] += (double)z[e];
                __syncthreads();
            }
        }
        res.iters += steps;
        res.cycles += cycles;
        res.reorth += reorth_steps;
        if (status != HEC_OK && res.status == HEC_OK)
            res.status = status;
        res.rel_resid = worst > res.rel_resid ? worst : res.rel_resid;
        store_group(g0, [&](long long e) { return xp[e]; });
        __syncthreads();
        return true;
    }

    // The single-operation modes (parity tests): x = A b, x = M^{-1} b.
    __device__ bool op_group(int g0)
    {
        load_group(g0);
        if (a.op == BOP_SPMV64) {
            double part[NR];
            for (int r = 0; r < NR; ++r)
                part[r] = 0.0;
            resid64<double>(nullptr, bp, 0, xp, part);
            __syncthreads();
            store_group(g0, [&](long long e) { return -xp[e]; });
        } else if (a.op == BOP_SPMV_IN) {
            for (long long e = tid; e < Ep; e += nt)
                z[e] = (T)bp[e];
            __syncthreads();
            spmv_in(z, 1);
            __syncthreads();
            store_group(g0, [&](long long e) { return (double)*vel(1, e); });
        } else {
            for (long long e = tid; e < Ep; e += nt)
                *vel(0, e) = (T)bp[e];
            fence_proxy_async_global();
            __syncthreads();
            T one[NR];
            for (int r = 0; r < NR; ++r)
                one[r] = T(1);
            if (!precond(Src{nullptr, 0}, one))
                return false;
            store_group(g0, [&](long long e) { return (double)z[e]; });
        }
        __syncthreads();
        return true;
    }

    __device__ void run()
    {
        if (tid == 0) {
            for (int i = 0; i < a.nstages; ++i)
                mbar_init(&full[i], 1);
            for (int i = 0; i < a.sstages; ++i)
                mbar_init(&full2[i], 1);
            fence_mbar_init();
        }
        // the ring's zero slot (padding dependencies)
        for (int r = tid; r < NR; r += nt)
            ring[(size_t)(a.ring_mask + 1) * NR + r] = T(0);
        __syncthreads();
        const int groups = (a.nrhs + NR - 1) / NR;
        for (;;) {
            if (tid == 0) {
                int sidx = -1;
                if (*reinterpret_cast<volatile int *>(a.err) == 0) {
                    const int q = atomicAdd(a.queue, 1);
                    if (q < a.nsys)
                        sidx = a.order[q];
                }
                misc[MI_SYS] = sidx;
            }
            __syncthreads();
            const int sidx = misc[MI_SYS];
            if (sidx < 0)
                return;
            if (a.only && !a.only[sidx]) {
                __syncthreads();  // every thread has read misc before it is rewritten
                continue;
            }
            s = a.sys[sidx];
            nE = (long long)s.n * NR;
            Ep = ((nE + nt - 1) >> tshift) << tshift;
            ntiles = (int)(Ep >> tshift);
            BatchResult res{0, 0, HEC_OK, 0, 0.0};
            for (int g = 0; g < groups; ++g) {
                const bool ok = a.op == BOP_SOLVE ? solve_group(g, res) : op_group(g);
                if (!ok)
                    return;
            }
            if (tid == 0 && a.op == BOP_SOLVE)
                a.res[sidx] = res;
            __syncthreads();
        }
    }
};

template <class T, int NR>
__global__ void __launch_bounds__(kBatchMaxThreads) k_batch(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Batch<T, NR> b(a, smem);
    b.run();
}

template <class T, int NR> const void *kernel_ptr() { return (const void *)k_batch<T, NR>; }

const void *select_kernel(bool fp32, int NR)
{
    if (fp32)
        return NR == 1 ? kernel_ptr<float, 1>() : NR == 2 ? kernel_ptr<float, 2>() : kernel_ptr<float, 4>();
    return NR == 1 ? kernel_ptr<double, 1>() : NR == 2 ? kernel_ptr<double, 2>() : kernel_ptr<double, 4>();
}

// The dynamic shared memory limit is an attribute of the kernel, shared by
// every thread of the process: it is raised once, to the device's opt-in
// maximum, never lowered per launch (concurrent launches of different sizes
// from several host threads would otherwise race on it).
cudaError_t prepare(const void *k)
{
    static std::mutex mu;
    static std::set<const void *> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(k))
        return cudaSuccess;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess)  // the opt-in limit covers static and dynamic shared memory
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
        done.insert(k);
    return e;
}

} // namespace

int launch_batch(const BatchArgs &a, bool fp32, int NR, int threads, int grid, int smem,
                 cudaStream_t s)
{
    const void *k = select_kernel(fp32, NR);
    cudaError_t e = prepare(k);
    if (e != cudaSuccess)
        return (int)e;
    void *args[] = {(void *)&a};
    return (int)cudaLaunchKernel(k, dim3(grid), dim3(threads), args, (size_t)smem, s);
}

int batch_occupancy(bool fp32, int NR, int threads, int smem)
{
    const void *k = select_kernel(fp32, NR);
    if (prepare(k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, (size_t)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

} // namespace hec
