// k_vec.cu -- vector operations (Section 2.3, Eqs. 3-6) and the fused vector
// updates of the Krylov loops (Algorithm 4 and GMRES), each with its dot
// products reduced in the same launch.
#include "reduce.cuh"

namespace hec {

template <int OP>
__global__ void __launch_bounds__(kThreads) k_vec(VecArgs a)
{
    count_launch(a.st);
    SolverState *st = a.st;
    constexpr int ND = (OP == V_DOT || OP == V_NRM2SQ || OP == V_BICG_S || OP == V_CG_XR) ? 1
                       : (OP == V_BICG_XR)                                                  ? 2
                                                                                            : 0;
    if (OP == V_BICG_S && st->skip)
        return;
    if (OP == V_CG_P && st->done)
        return;
    if (OP == V_ZERO_IF_ST && !st->zero_x)
        return;
    if ((a.guard == 1 && st->cycle_end) || (a.guard == 2 && st->done))
        return;
    const double *x = a.x;
    double *z = a.z;
    if (a.x_from_j)
        x += (int64_t)st->j * a.ldv;
    if (a.z_from_j)
        z += (int64_t)st->j * a.ldv;
    double acc[ND > 0 ? ND : 1];
#pragma unroll
    for (int d = 0; d < (ND > 0 ? ND : 1); ++d)
        acc[d] = 0.0;

    // per-launch scalars
    double c0 = a.a, c1 = a.b;
    int mode = 0;
    if (OP == V_SCALE_ST)
        c0 = st->scale;
    if (OP == V_BICG_P) {
        if (st->iters == 0) {
            mode = 1; // first pass: p = r
        } else {
            c0 = (st->rho / st->rho_prev) * (st->alpha / st->omega); // beta
            c1 = st->omega;
        }
    }
    if (OP == V_BICG_S)
        c0 = st->alpha;
    if (OP == V_CG_XR) {
        c0 = st->alpha;
        mode = st->skip; // breakdown in alpha: no update (the sum still runs)
    }
    if (OP == V_CG_P) {
        mode = st->iters == 0; // first pass: p = z
        c0 = st->cg_beta;
    }
    if (OP == V_BICG_XR) {
        c0 = st->alpha;
        c1 = st->omega;
        mode = st->s_conv ? 1 : (st->skip ? 2 : 0);
    }

    const int stride = gridDim.x * kThreads;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += stride) {
        if (OP == V_AXPBY) {
            z[i] = c0 * x[i] + c1 * z[i];
        } else if (OP == V_WAXPBY) {
            z[i] = c0 * x[i] + c1 * a.y[i];
        } else if (OP == V_DOT) {
            acc[0] = fma(x[i], a.y[i], acc[0]);
        } else if (OP == V_NRM2SQ) {
            double t = x[i];
            acc[0] = fma(t, t, acc[0]);
        } else if (OP == V_COPY) {
            z[i] = x[i];
        } else if (OP == V_SCALE_ST) {
            z[i] = c0 * x[i];
        } else if (OP == V_BICG_P) {
            // x = r, y = v, z = p
            z[i] = mode ? x[i] : fma(c0, z[i] - c1 * a.y[i], x[i]);
        } else if (OP == V_BICG_S) {
            // x = r, y = v, z = s
            double s = fma(-c0, a.y[i], x[i]);
            z[i] = s;
            acc[0] = fma(s, s, acc[0]);
        } else if (OP == V_BICG_XR) {
            // w = x (solution), u = p*, v = s*, q = t, x = s, y = r0, z = r
            if (mode == 0) {
                a.w[i] = fma(c1, a.v[i], fma(c0, a.u[i], a.w[i]));
                double r = fma(-c1, a.q[i], x[i]);
                z[i] = r;
                acc[0] = fma(r, r, acc[0]);
                acc[1] = fma(a.y[i], r, acc[1]);
            } else if (mode == 1) {
                a.w[i] = fma(c0, a.u[i], a.w[i]);
            }
        } else if (OP == V_CG_XR) {
            // w = x (solution), u = p, q = A p, z = r
            if (!mode) {
                a.w[i] = fma(c0, a.u[i], a.w[i]);
                const double r = fma(-c0, a.q[i], z[i]);
                z[i] = r;
                acc[0] = fma(r, r, acc[0]);
            }
        } else if (OP == V_CG_P) {
            // x = z (preconditioned residual), z = p
            z[i] = mode ? x[i] : fma(c0, z[i], x[i]);
        } else if (OP == V_AXPY_ST1) {
            z[i] += x[i];
        } else if (OP == V_ZERO_IF_ST) {
            z[i] = 0.0;
        }
    }
    if constexpr (ND > 0) {
        double v[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d)
            v[d] = acc[d];
        reduce_and_finalize<ND>(v, a.red, a.op, a.result, st);
    }
}

int launch_vec(VecOp vop, const VecArgs &a, int grid, cudaStream_t s)
{
    switch (vop) {
#define HEC_VEC_CASE(OPV)                                                                        \
    case OPV:                                                                                    \
        k_vec<OPV><<<grid, kThreads, 0, s>>>(a);                                                 \
        return 0;
        HEC_VEC_CASE(V_AXPBY)
        HEC_VEC_CASE(V_WAXPBY)
        HEC_VEC_CASE(V_DOT)
        HEC_VEC_CASE(V_NRM2SQ)
        HEC_VEC_CASE(V_COPY)
        HEC_VEC_CASE(V_SCALE_ST)
        HEC_VEC_CASE(V_BICG_P)
        HEC_VEC_CASE(V_BICG_S)
        HEC_VEC_CASE(V_BICG_XR)
        HEC_VEC_CASE(V_AXPY_ST1)
        HEC_VEC_CASE(V_ZERO_IF_ST)
        HEC_VEC_CASE(V_CG_XR)
        HEC_VEC_CASE(V_CG_P)
#undef HEC_VEC_CASE
    }
    return -1;
}

// ------------------------------------------------------------------ typed vector kernels

// V_COPY, V_SCALE_ST, V_AXPY_ST1, V_JACOBI with element types TX (x) and TZ (z).
template <int OP, class TX, class TZ> __global__ void __launch_bounds__(kThreads) k_vec_typed(VecArgs a)
{
    count_launch(a.st);
    SolverState *st = a.st;
    if ((a.guard == 1 && st->cycle_end) || (a.guard == 2 && st->done))
        return;
    if (OP == V_JACOBI && st && st->skip) // as the triangular solves: a skipped apply
        return;
    const TZ *d = reinterpret_cast<const TZ *>(a.dv);
    const TX *x = reinterpret_cast<const TX *>(a.xv);
    TZ *z = reinterpret_cast<TZ *>(a.zv);
    if (a.x_from_j)
        x += (int64_t)st->j * a.ldv;
    if (a.z_from_j)
        z += (int64_t)st->j * a.ldv;
    const double sc = (OP == V_SCALE_ST) ? st->scale : 1.0;
    const int stride = gridDim.x * kThreads;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += stride) {
        if (OP == V_COPY)
            z[i] = TZ(x[i]);
        else if (OP == V_SCALE_ST)
            z[i] = TZ(sc * double(x[i]));
        else if (OP == V_AXPY_ST1)
            z[i] = z[i] + TZ(x[i]);
        else if (OP == V_JACOBI)
            z[i] = d[i] * TZ(x[i]);
    }
}

template <int OP> static int launch_typed_op(const VecArgs &a, bool x32, bool z32, int grid, cudaStream_t s)
{
    if (x32 && z32)
        k_vec_typed<OP, float, float><<<grid, kThreads, 0, s>>>(a);
    else if (x32)
        k_vec_typed<OP, float, double><<<grid, kThreads, 0, s>>>(a);
    else if (z32)
        k_vec_typed<OP, double, float><<<grid, kThreads, 0, s>>>(a);
    else
        k_vec_typed<OP, double, double><<<grid, kThreads, 0, s>>>(a);
    return 0;
}

int launch_vec_typed(VecOp vop, const VecArgs &a, bool x32, bool z32, int grid, cudaStream_t s)
{
    switch (vop) {
    case V_COPY: return launch_typed_op<V_COPY>(a, x32, z32, grid, s);
    case V_SCALE_ST: return launch_typed_op<V_SCALE_ST>(a, x32, z32, grid, s);
    case V_AXPY_ST1: return launch_typed_op<V_AXPY_ST1>(a, x32, z32, grid, s);
    case V_JACOBI: return launch_typed_op<V_JACOBI>(a, x32, z32, grid, s);
    default: return -1;
    }
}

// ------------------------------------------------------------------ GMRES basis kernels
// The basis (m + 1 vectors of n) is streamed by every projection and update
// pass and is larger than L2 for large n; it is read under an evict-first L2
// policy so that w, which every vector group re-reads, stays in L2.
// (Measured on the 128^3 case: the mixed-precision GMRES(30) solve 5% faster,
// the FP64 one unchanged.)
__device__ __forceinline__ uint64_t basis_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ double ld_basis(const double *p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_basis(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
                 : "=f"(v) : "l"(p), "l"(pol));
    return v;
}


constexpr int kGroup = 8; // basis vectors per CTA in a projection

// h[i] = (V_i, w), i < k.  Grid (row blocks, vector groups); every CTA keeps
// kGroup running sums per thread (in T) and reduces them once at the end (in
// FP64, fixed order).
template <class T> __global__ void __launch_bounds__(kThreads) k_multidot(BasisArgs a)
{
    count_launch(a.st);
    int k = a.k;
    if (a.k_from_st == 1)
        k = a.st->j + 1;
    else if (a.k_from_st == 2)
        k = a.st->jend;
    const T *V = reinterpret_cast<const T *>(a.V);
    const T *w = reinterpret_cast<const T *>(a.w);
    const int g0 = blockIdx.y * kGroup;
    T acc[kGroup];
#pragma unroll
    for (int q = 0; q < kGroup; ++q)
        acc[q] = T(0);
    if (g0 < k) {
        const uint64_t pol = basis_policy();
        const int stride = gridDim.x * kThreads;
        for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += stride) {
            const T wi = w[i];
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
                if (g0 + q < k)
                    acc[q] = fma(ld_basis(&V[(int64_t)(g0 + q) * a.ldv + i], pol), wi, acc[q]);
        }
    }
    // block reduction of the kGroup sums
    __shared__ double sh[kGroup][kThreads / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kGroup; ++q) {
        double t = warp_sum(double(acc[q]));
        if (lane == 0)
            sh[q][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < kGroup) {
        double t = 0.0;
        for (int ww = 0; ww < kThreads / 32; ++ww)
            t += sh[threadIdx.x][ww];
        // partials layout: [vector][row block]
        const int q = g0 + threadIdx.x;
        if (q < k)
            a.red.partials[(size_t)q * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned tk = atomicAdd(a.red.ticket, 1u);
        s_last = (tk == gridDim.x * gridDim.y - 1);
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    for (int q = threadIdx.x; q < k; q += kThreads) {
        double t = 0.0;
        for (unsigned c = 0; c < gridDim.x; ++c)
            t += __ldcg(&a.red.partials[(size_t)q * gridDim.x + c]);
        if (a.op == FIN_GMRES_H1)
            a.st->h1[q] = t;
        else if (a.op == FIN_GMRES_H2)
            a.st->h2[q] = t;
        else
            a.result[q] = t;
    }
    if (threadIdx.x == 0)
        *a.red.ticket = 0u;
}

int launch_multidot(const BasisArgs &a, int grid, cudaStream_t s, bool fp32)
{
    // a.k is the number of vectors, or an upper bound of it when k_from_st
    dim3 g(grid, (a.k + kGroup - 1) / kGroup);
    if (fp32)
        k_multidot<float><<<g, kThreads, 0, s>>>(a);
    else
        k_multidot<double><<<g, kThreads, 0, s>>>(a);
    return 0;
}

// wout = w - sum_{i<k} coef[i] V_i, optionally with (wout, wout) reduced.
template <bool NORM, class T> __global__ void __launch_bounds__(kThreads) k_basis_update(BasisArgs a)
{
    count_launch(a.st);
    int k = a.k;
    if (a.k_from_st == 1)
        k = a.st->j + 1;
    else if (a.k_from_st == 2)
        k = a.st->jend;
    const T *V = reinterpret_cast<const T *>(a.V);
    const T *w = reinterpret_cast<const T *>(a.w);
    T *wout = reinterpret_cast<T *>(a.wout);
    __shared__ T sc[kMaxRestart + 1];
    for (int q = threadIdx.x; q < k; q += kThreads)
        sc[q] = T(a.coef[q]);
    __syncthreads();
    T acc = T(0);
    const uint64_t pol = basis_policy();
    const int stride = gridDim.x * kThreads;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += stride) {
        T t = w[i];
        for (int q = 0; q < k; ++q)
            t = fma(-sc[q], ld_basis(&V[(int64_t)q * a.ldv + i], pol), t);
        wout[i] = t;
        if (NORM)
            acc = fma(t, t, acc);
    }
    if (NORM) {
        double v[1] = {double(acc)};
        reduce_and_finalize<1>(v, a.red, a.op, a.result, a.st);
    }
}

int launch_basis_update(const BasisArgs &a, bool with_norm, int grid, cudaStream_t s, bool fp32)
{
    if (with_norm) {
        if (fp32)
            k_basis_update<true, float><<<grid, kThreads, 0, s>>>(a);
        else
            k_basis_update<true, double><<<grid, kThreads, 0, s>>>(a);
    } else {
        if (fp32)
            k_basis_update<false, float><<<grid, kThreads, 0, s>>>(a);
        else
            k_basis_update<false, double><<<grid, kThreads, 0, s>>>(a);
    }
    return 0;
}

// wout = sum_{i<k} coef[i] V_i
template <class T> __global__ void __launch_bounds__(kThreads) k_basis_combine(BasisArgs a)
{
    count_launch(a.st);
    int k = a.k;
    if (a.k_from_st == 1)
        k = a.st->j + 1;
    else if (a.k_from_st == 2)
        k = a.st->jend;
    const T *V = reinterpret_cast<const T *>(a.V);
    T *wout = reinterpret_cast<T *>(a.wout);
    __shared__ T sc[kMaxRestart + 1];
    for (int q = threadIdx.x; q < k; q += kThreads)
        sc[q] = T(a.coef[q]);
    __syncthreads();
    const uint64_t pol = basis_policy();
    const int stride = gridDim.x * kThreads;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += stride) {
        T t = T(0);
        for (int q = 0; q < k; ++q)
            t = fma(sc[q], ld_basis(&V[(int64_t)q * a.ldv + i], pol), t);
        wout[i] = t;
    }
}

int launch_basis_combine(const BasisArgs &a, int grid, cudaStream_t s, bool fp32)
{
    if (fp32)
        k_basis_combine<float><<<grid, kThreads, 0, s>>>(a);
    else
        k_basis_combine<double><<<grid, kThreads, 0, s>>>(a);
    return 0;
}

// ------------------------------------------------------------------ small kernels

// Back substitution R y = g of the Givens-reduced Hessenberg matrix (one thread).
__global__ void k_gmres_lsq(SolverState *st)
{
    count_launch(st);
    if (threadIdx.x != 0)
        return;
    const int je = st->jend, ld = kMaxRestart;
    for (int i = je - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int l = i + 1; l < je; ++l)
            s -= st->H[i * ld + l] * st->y[l];
        st->y[i] = s / st->H[i * ld + i];
    }
}

int launch_gmres_lsq(SolverState *st, cudaStream_t s)
{
    k_gmres_lsq<<<1, 32, 0, s>>>(st);
    return 0;
}

// Loop condition of the solve graph's while node.
__global__ void k_loopcond(SolverState *st)
{
    count_launch(st);
    if (threadIdx.x == 0)
        set_cond(st, st->h_while, !st->done);
}

int launch_loopcond(SolverState *st, cudaStream_t s)
{
    k_loopcond<<<1, 32, 0, s>>>(st);
    return 0;
}

} // namespace hec
