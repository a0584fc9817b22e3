// reduce.cuh -- deterministic two-stage reductions fused into the streaming
// kernels (Eqs. 5-6), and the scalar recurrences of the Krylov solvers that
// the last CTA of a reducing launch evaluates.
#pragma once

#include "../../include/hecgpu.h"
#include "kernels.cuh"

namespace hec {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void count_launch(SolverState *st)
{
    if (st && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
        atomicAdd(&st->launches, 1ull);
}

// Set a conditional node's value -- only inside the solve graph; a solve
// driven from the host reads the flags instead.
__device__ __forceinline__ void set_cond(const SolverState *st, cudaGraphConditionalHandle h, int on)
{
    if (st->graph_mode)
        cudaGraphSetConditional(h, on ? 1u : 0u);
}

// Scalar recurrences (one thread).  s[0..nd) are the reduced values.
__device__ inline void finalize(int op, const double *s, int nd, double *result, SolverState *st)
{
    switch (op) {
    case FIN_STORE:
        for (int d = 0; d < nd; ++d)
            result[d] = s[d];
        break;
    case FIN_STORE_SQRT:
        result[0] = sqrt(s[0]);
        break;
    case FIN_NRM_B:
        st->bnorm = sqrt(s[0]);
        if (st->bnorm == 0.0) {
            st->done = 1;
            st->zero_x = 1;
            st->status = HEC_OK;
        }
        break;
    case FIN_BICG_INIT: {
        // r_0 = b - A x_0 and the shadow residual r_0: rho_0 = (r_0, r_0)
        double rr = s[0];
        st->rho = rr;
        if (st->done)
            break;
        st->est = sqrt(rr) / st->bnorm;
        if (sqrt(rr) <= st->tol * st->bnorm) {
            st->done = 1;
            st->status = HEC_OK;
        } else if (st->maxit <= 0) {
            st->done = 1;
            st->status = HEC_MAXIT;
        }
        break;
    }
    case FIN_BICG_ALPHA: {
        double r0v = s[0];
        if (r0v == 0.0) {
            st->skip = 1;
            st->status = HEC_BREAKDOWN;
        } else {
            st->alpha = st->rho / r0v;
        }
        break;
    }
    case FIN_BICG_S: {
        double sn = sqrt(s[0]);
        if (sn <= st->tol * st->bnorm) {
            st->s_conv = 1;
            st->skip = 1;
            st->est = sn / st->bnorm;
        }
        break;
    }
    case FIN_BICG_OMEGA: {
        double ts = s[0], tt = s[1];
        st->omega = (tt == 0.0) ? 0.0 : ts / tt;
        break;
    }
    case FIN_BICG_XR: {
        st->iters += 1;
        if (st->s_conv) {
            st->done = 1;
            st->status = HEC_OK;
        } else if (st->skip) { // (r0, v) = 0
            st->done = 1;
            st->status = HEC_BREAKDOWN;
        } else {
            double rn = sqrt(s[0]), rho_new = s[1];
            st->est = rn / st->bnorm;
            if (rn <= st->tol * st->bnorm) {
                st->done = 1;
                st->status = HEC_OK;
            } else if (st->omega == 0.0 || rho_new == 0.0 || isnan(rn) || isnan(rho_new)) {
                st->done = 1;
                st->status = HEC_BREAKDOWN;
            } else if (st->iters >= st->maxit) {
                st->done = 1;
                st->status = HEC_MAXIT;
            }
            st->rho_prev = st->rho;
            st->rho = rho_new;
        }
        st->skip = 0;
        st->s_conv = 0;
        set_cond(st, st->h_while, !st->done);
        break;
    }
    case FIN_TRUE_RESID:
        st->rel_resid = (st->bnorm > 0.0) ? sqrt(s[0]) / st->bnorm : 0.0;
        break;
    case FIN_GMRES_CYCLE: {
        double beta = sqrt(s[0]);
        if (st->done)
            break;
        // mixed precision: the previous FP32 cycle promised a residual of
        // est * ||b||; a true FP64 residual far above it, with less than a
        // halving over the cycle, means the FP32 arithmetic, not the Krylov
        // space, limits the refinement
        // -- and eight cycles in a row that each cut the true residual by
        // less than 10% mean the FP32 inner cycles gain too little on this
        // system (measured: an ill-conditioned 2D system of 737,881 unknowns
        // reached 1.6e-5 after 20,000 mixed steps where FP64 converges in
        // 12,801)
        const double promised = st->est * st->bnorm;
        if (st->inner_rtol > 0.0 && st->restarts > 0) {
            st->stag_run = (promised > 0.0 && beta > 10.0 * promised && beta > 0.5 * st->beta_cycle)
                               ? st->stag_run + 1
                               : 0;
            st->slow_run = beta > 0.9 * st->beta_cycle ? st->slow_run + 1 : 0;
        }
        st->est = beta / st->bnorm;
        if (beta <= st->tol * st->bnorm) {
            st->done = 1;
            st->status = HEC_OK;
        } else if (isnan(beta)) {
            st->done = 1;
            st->status = HEC_BREAKDOWN;
        } else if (st->iters >= st->maxit) {
            st->done = 1;
            st->status = HEC_MAXIT;
        } else if (st->stag_run >= 2 || st->slow_run >= 8) {
            // the host continues in FP64
            st->done = 1;
            st->stagnated = 1;
            st->status = HEC_MAXIT;
        } else {
            st->restarts += 1;
            st->j = 0;
            st->cycle_end = 0;
            st->beta_cycle = beta;
            for (int i = 0; i <= st->restart; ++i)
                st->g[i] = 0.0;
            st->g[0] = beta;
            st->scale = 1.0 / beta;
        }
        break;
    }
    case FIN_GMRES_W0:
        st->w0norm = sqrt(s[0]);
        break;
    case FIN_GMRES_STEP: {
        const int j = st->j, m = st->restart;
        const int ld = kMaxRestart;
        double hn = sqrt(s[0]);
        for (int i = 0; i <= j; ++i)
            st->H[i * ld + j] = st->h1[i] + st->h2[i];
        st->H[(j + 1) * ld + j] = hn;
        for (int i = 0; i < j; ++i) {
            double a = st->H[i * ld + j], c = st->H[(i + 1) * ld + j];
            st->H[i * ld + j] = st->cs[i] * a + st->sn[i] * c;
            st->H[(i + 1) * ld + j] = -st->sn[i] * a + st->cs[i] * c;
        }
        double a = st->H[j * ld + j], c = st->H[(j + 1) * ld + j];
        double den = sqrt(a * a + c * c);
        st->cs[j] = (den == 0.0) ? 1.0 : a / den;
        st->sn[j] = (den == 0.0) ? 0.0 : c / den;
        st->H[j * ld + j] = den;
        st->H[(j + 1) * ld + j] = 0.0;
        st->g[j + 1] = -st->sn[j] * st->g[j];
        st->g[j] = st->cs[j] * st->g[j];
        st->iters += 1;
        double est = fabs(st->g[j + 1]);
        st->est = est / st->bnorm;
        int happy = (hn == 0.0) || (hn <= 1e-300 * st->w0norm);
        int end = (est <= st->tol * st->bnorm) || happy || (j + 1 == m) ||
                  (st->iters >= st->maxit) || isnan(est) ||
                  (est <= st->inner_rtol * st->beta_cycle);
        st->cycle_end = end;
        if (end) {
            st->jend = j + 1;
        } else {
            st->scale = 1.0 / hn;
            st->j = j + 1;
        }
        set_cond(st, st->h_if, end);
        break;
    }
    case FIN_CG_INIT: {
        // r_0 = b - A x_0
        if (st->done)
            break;
        const double rn = sqrt(s[0]);
        st->est = rn / st->bnorm;
        if (rn <= st->tol * st->bnorm) {
            st->done = 1;
            st->status = HEC_OK;
        } else if (st->maxit <= 0) {
            st->done = 1;
            st->status = HEC_MAXIT;
        }
        break;
    }
    case FIN_CG_RHO: {
        // (r_{j+1}, z_{j+1}): beta_j and the next rho; the loop goes on
        // unless the residual test, the budget or a breakdown ended it
        if (!st->done) {
            const double rz = s[0];
            if (rz == 0.0 || isnan(rz)) {
                st->done = 1;
                st->status = HEC_BREAKDOWN;
            } else {
                st->cg_beta = (st->iters > 0) ? rz / st->rho : 0.0;
                st->rho = rz;
            }
        }
        st->skip = 0; // the last pass skipped its preconditioner apply; the exit runs
        set_cond(st, st->h_while, !st->done);
        break;
    }
    case FIN_CG_ALPHA: {
        const double pq = s[0];
        if (pq == 0.0 || isnan(pq)) {
            st->skip = 1; // no update of x, r; the pass ends the loop
            st->done = 1;
            st->status = HEC_BREAKDOWN;
        } else {
            st->alpha = st->rho / pq;
        }
        break;
    }
    case FIN_CG_R: {
        if (st->skip)
            break;
        st->iters += 1;
        const double rn = sqrt(s[0]);
        st->est = rn / st->bnorm;
        if (rn <= st->tol * st->bnorm) {
            st->done = 1;
            st->status = HEC_OK;
        } else if (isnan(rn)) {
            st->done = 1;
            st->status = HEC_BREAKDOWN;
        } else if (st->iters >= st->maxit) {
            st->done = 1;
            st->status = HEC_MAXIT;
        }
        st->skip = st->done; // no preconditioner apply after the last pass
        break;
    }
    default:
        break;
    }
}

// Block reduction of ND per-thread values, per-CTA partials, and a
// fixed-order sum plus finalize() by the CTA that arrives last.  All threads
// of the CTA must call it.  The summation order depends only on the grid
// size, never on timing, so results are deterministic.
template <int ND>
__device__ __forceinline__ void reduce_and_finalize(double (&v)[ND], const RedScratch &red, int op,
                                                    double *result, SolverState *st)
{
    __shared__ double sh[ND][kThreads / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        double t = warp_sum(v[d]);
        if (lane == 0)
            sh[d][wid] = t;
    }
    __syncthreads();
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w)
                t += sh[d][w];
            red.partials[(size_t)bid * ND + d] = t;
        }
        __threadfence();
        unsigned tk = atomicAdd(red.ticket, 1u);
        s_last = (tk == nblk - 1);
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        double t = 0.0;
        for (unsigned c = threadIdx.x; c < nblk; c += kThreads)
            t += __ldcg(&red.partials[(size_t)c * ND + d]);
        t = warp_sum(t);
        if (lane == 0)
            sh[d][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            s[d] = 0.0;
            for (int w = 0; w < kThreads / 32; ++w)
                s[d] += sh[d][w];
        }
        *red.ticket = 0u;
        finalize(op, s, ND, result, st);
    }
}

} // namespace hec
