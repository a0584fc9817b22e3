/*
 * hec_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see the
 * header).  Every function restates one passage of Yang, Liu and Chen,
 * "Development of Krylov and AMG linear solvers for large-scale sparse
 * matrices on GPUs", Section 2, in the paper's order and notation.  Where
 * the paper is silent or garbled the reading taken is written next to the
 * code.  Compile with -ffp-contract=off so the results are the same on every
 * host (no fused multiply-add contraction).
 */
#include "hec_oracle.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Section 2.2-2.3: SpMV and vector operations                         */
/* ------------------------------------------------------------------ */

/* Eq. 2 with the row-wise evaluation of Algorithm 1: every row i is the
 * inner product of row i of A with x (Eq. 1 is the same sum seen column by
 * column), taken over the stored entries in ascending column order. */
void orc_spmv(int n, const int *rp, const int *ci, const double *va, double alpha,
              const double *x, double beta, double *y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            s += va[e] * x[ci[e]];
        y[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * y[i];
    }
}

/* The same row loop restricted to rows [lo, hi): the oracle's SpMV split
 * over host threads for the all-cores CPU baseline (each row is summed as in
 * orc_spmv, so the result is identical). */
void orc_spmv_range(int n, const int *rp, const int *ci, const double *va, double alpha,
                    const double *x, double beta, double *y, int lo, int hi)
{
    (void)n;
    for (int i = lo; i < hi; ++i) {
        double s = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            s += va[e] * x[ci[e]];
        y[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * y[i];
    }
}

/* Eq. 5 */
double orc_dot(int n, const double *x, const double *y)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += x[i] * y[i];
    return s;
}

/* Eq. 6 */
double orc_nrm2(int n, const double *x) { return sqrt(orc_dot(n, x, x)); }

/* Eq. 3 */
void orc_axpby(int n, double a, const double *x, double b, double *y)
{
    for (int i = 0; i < n; ++i)
        y[i] = a * x[i] + b * y[i];
}

/* Eq. 4 */
void orc_waxpby(int n, double a, const double *x, double b, const double *y, double *z)
{
    for (int i = 0; i < n; ++i)
        z[i] = a * x[i] + b * y[i];
}

/* ------------------------------------------------------------------ */
/* Section 2.4: ILU(k), Eqs. 9-10 and Algorithm 2                      */
/* ------------------------------------------------------------------ */

void orc_csr_free(orc_csr *m)
{
    if (!m)
        return;
    free(m->rp);
    free(m->ci);
    free(m->va);
    free(m->lev);
    memset(m, 0, sizeof(*m));
}

/* Growable output arrays of the factor. */
typedef struct {
    int cap, len;
    int *ci;
    double *va;
    int *lev;
} grow_t;

static int grow_push(grow_t *g, int c, double v, int l)
{
    if (g->len == g->cap) {
        int nc = g->cap ? 2 * g->cap : 1024;
        int *a = (int *)realloc(g->ci, sizeof(int) * (size_t)nc);
        if (!a)
            return -1;
        g->ci = a;
        double *b = (double *)realloc(g->va, sizeof(double) * (size_t)nc);
        if (!b)
            return -1;
        g->va = b;
        int *d = (int *)realloc(g->lev, sizeof(int) * (size_t)nc);
        if (!d)
            return -1;
        g->lev = d;
        g->cap = nc;
    }
    g->ci[g->len] = c;
    g->va[g->len] = v;
    g->lev[g->len] = l;
    g->len++;
    return 0;
}

#define LEV_INF (INT_MAX / 4)

/*
 * Algorithm 2, row by row.  Row i is held as a sorted linked list of the
 * positions it touches, each with a value A_ij and a level L_ij:
 *   - Eq. 9: positions of the pattern P of A start with level 0; every other
 *     position has level infinity (it simply is not in the list).
 *   - For p = 1 .. i-1 in ascending order with L_ip <= k (positions created
 *     as fill earlier in the same row are visited too, because the list is
 *     walked in order while it grows):
 *         A_ip = A_ip / A_pp
 *         for every j > p:  A_ij = A_ij - A_ip A_pj,
 *                           L_ij = min(L_ij, L_ip + L_pj + 1)     (Eq. 10)
 *     Reading: A_pj and L_pj come from the finished row p, whose dropped
 *     positions are zero with level infinity, so only the positions kept in
 *     row p with j > p change anything; the loop visits exactly those.
 *   - After the p loop, every position of row i with L_ij > k is set to zero
 *     (dropped).  Reading: in Algorithm 2 this test sits after the p loop
 *     with j unbound; it is taken to apply to all j of row i.
 * Row 1 has no p < 1 and is copied unchanged.
 */
int orc_iluk(int n, const int *rp, const int *ci, const double *va, int k, orc_csr *out)
{
    memset(out, 0, sizeof(*out));
    if (n <= 0 || k < 0)
        return ORC_ERR_INVALID;
    for (int i = 0; i < n; ++i) {
        int has_diag = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n)
                return ORC_ERR_INVALID;
            if (e > rp[i] && ci[e] <= ci[e - 1])
                return ORC_ERR_INVALID;
            if (ci[e] == i)
                has_diag = 1;
        }
        if (!has_diag)
            return ORC_ERR_INVALID;
    }

    double *wv = (double *)calloc((size_t)n, sizeof(double));
    int *wl = (int *)malloc(sizeof(int) * (size_t)n);
    int *nxt = (int *)malloc(sizeof(int) * (size_t)n);
    int *stamp = (int *)malloc(sizeof(int) * (size_t)n);
    int *frp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *fdiag = (int *)malloc(sizeof(int) * (size_t)n); /* position of U_pp */
    grow_t g = {0, 0, NULL, NULL, NULL};
    int status = ORC_OK;
    if (!wv || !wl || !nxt || !stamp || !frp || !fdiag) {
        status = ORC_ERR_INVALID;
        goto done;
    }
    for (int i = 0; i < n; ++i)
        stamp[i] = -1;
    frp[0] = 0;

    for (int i = 0; i < n; ++i) {
        /* Eq. 9: load the pattern of row i with level 0. */
        int head = -1, tail = -1;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            wv[j] = va[e];
            wl[j] = 0;
            stamp[j] = i;
            nxt[j] = -1;
            if (tail < 0)
                head = j;
            else
                nxt[tail] = j;
            tail = j;
        }
        /* The p loop of Algorithm 2. */
        for (int p = head; p >= 0 && p < i; p = nxt[p]) {
            if (wl[p] > k)
                continue;
            double upp = g.va[fdiag[p]];
            if (upp == 0.0) {
                status = ORC_ERR_ZERO_PIVOT;
                goto done;
            }
            wv[p] = wv[p] / upp;
            /* for j > p over the kept entries of row p */
            int cursor = p; /* list node after which j is searched */
            for (int e = fdiag[p] + 1; e < frp[p + 1]; ++e) {
                int j = g.ci[e];
                if (stamp[j] != i) {
                    /* position not yet in row i: value 0, level infinity */
                    while (nxt[cursor] >= 0 && nxt[cursor] < j)
                        cursor = nxt[cursor];
                    wv[j] = 0.0;
                    wl[j] = LEV_INF;
                    stamp[j] = i;
                    nxt[j] = nxt[cursor];
                    nxt[cursor] = j;
                    cursor = j;
                } else {
                    cursor = j;
                }
                wv[j] = wv[j] - wv[p] * g.va[e];
                int cand = wl[p] + g.lev[e] + 1;
                if (cand < wl[j])
                    wl[j] = cand;
            }
        }
        /* Drop the positions of row i whose level exceeds k. */
        fdiag[i] = -1;
        for (int j = head; j >= 0; j = nxt[j]) {
            if (wl[j] > k)
                continue;
            if (j == i)
                fdiag[i] = g.len;
            if (grow_push(&g, j, wv[j], wl[j]) != 0) {
                status = ORC_ERR_INVALID;
                goto done;
            }
        }
        frp[i + 1] = g.len;
        if (g.va[fdiag[i]] == 0.0) {
            status = ORC_ERR_ZERO_PIVOT;
            goto done;
        }
    }

done:
    free(wv);
    free(wl);
    free(nxt);
    free(stamp);
    free(fdiag);
    if (status != ORC_OK) {
        free(frp);
        free(g.ci);
        free(g.va);
        free(g.lev);
        return status;
    }
    out->n = n;
    out->rp = frp;
    out->ci = g.ci;
    out->va = g.va;
    out->lev = g.lev;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Section 2.6: level schedule, Eq. 11                                 */
/* ------------------------------------------------------------------ */

/* Eq. 11: l(i) = 1 + max l(j) over the off-diagonal entries j of row i in
 * the triangle being solved, with l initialised to 0 (so the max over no
 * entry is 0 and the first level is 1).  For the upper factor the rows are
 * taken in reverse (Section 2.6 turns an upper system into a lower one). */
int orc_levels(int n, const int *rp, const int *ci, int upper, int *level)
{
    int nlev = 0;
    for (int i = 0; i < n; ++i)
        level[i] = 0;
    for (int t = 0; t < n; ++t) {
        int i = upper ? n - 1 - t : t;
        int m = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            if ((upper && j > i) || (!upper && j < i))
                if (level[j] > m)
                    m = level[j];
        }
        level[i] = 1 + m;
        if (level[i] > nlev)
            nlev = level[i];
    }
    return nlev;
}

/* Solve L y = b with the unit-lower part of a combined factor (Eq. 8). */
void orc_lsolve_unit(int n, const int *rp, const int *ci, const double *va,
                     const double *b, double *y)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int e = rp[i]; e < rp[i + 1] && ci[e] < i; ++e)
            s -= va[e] * y[ci[e]];
        y[i] = s;
    }
}

/* Solve U z = y with the upper part (diagonal included) of a combined factor. */
int orc_usolve(int n, const int *rp, const int *ci, const double *va,
               const double *y, double *z)
{
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        double d = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] == i)
                d = va[e];
            else if (ci[e] > i)
                s -= va[e] * z[ci[e]];
        }
        if (d == 0.0)
            return ORC_ERR_ZERO_PIVOT;
        z[i] = s / d;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Section 2.5: restricted additive Schwarz                            */
/* ------------------------------------------------------------------ */

struct orc_ras {
    int n, nblocks;
    double *dinv;         /* damped Jacobi: omega / a_ii (then nblocks = 0) */
    int *own_lo, *own_hi; /* owned range W_b = [own_lo, own_hi) */
    int *nv;              /* |V_b| */
    int **rows;           /* V_b, ascending global ids */
    orc_csr *fac;         /* ILU(k) of A[V_b, V_b] */
    double *wr, *wy, *wz; /* scratch of max |V_b| */
};

void orc_ras_free(orc_ras *M)
{
    if (!M)
        return;
    for (int b = 0; b < M->nblocks; ++b) {
        if (M->rows)
            free(M->rows[b]);
        if (M->fac)
            orc_csr_free(&M->fac[b]);
    }
    free(M->own_lo);
    free(M->own_hi);
    free(M->nv);
    free(M->rows);
    free(M->fac);
    free(M->wr);
    free(M->wy);
    free(M->wz);
    free(M->dinv);
    free(M);
}

/*
 * Damped Jacobi (Section 2.8 names it among the smoothers built from the
 * SpMV and vector operations): one relaxation step x <- x + omega D^{-1}
 * (b - A x) from x = 0, used as the preconditioner z = omega D^{-1} r, D the
 * diagonal of A.  The factor omega / a_ii is formed once per row.  A zero
 * or missing diagonal entry gives ORC_ERR_ZERO_PIVOT.
 */
orc_ras *orc_jacobi_setup(int n, const int *rp, const int *ci, const double *va, double omega,
                          int *status)
{
    *status = ORC_OK;
    if (n <= 0 || !(omega > 0.0)) {
        *status = ORC_ERR_INVALID;
        return NULL;
    }
    orc_ras *M = (orc_ras *)calloc(1, sizeof(orc_ras));
    M->n = n;
    M->dinv = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i)
                d = va[e];
        if (d == 0.0) {
            *status = ORC_ERR_ZERO_PIVOT;
            orc_ras_free(M);
            return NULL;
        }
        M->dinv[i] = omega / d;
    }
    return M;
}

/*
 * Section 2.5 on one device (only the inner level of the two-level scheme
 * exists there).  Readings:
 *   - Partition: the sequence partition the paper uses for matrices of
 *     regular structure (Section 2.2): block b owns the contiguous rows
 *     W_b = [floor(b n / nb), floor((b+1) n / nb)).
 *   - Overlap: each block takes in "some layers of neighbour entries".  Layer
 *     d+1 is V^{d+1} = V^d plus every column j with a stored A_ij, i in V^d
 *     (row-pattern adjacency), starting from V^0 = W_b.
 *   - Block matrix: A[V_b, V_b], rows and columns in ascending global order;
 *     the entries outside the block are removed.
 *   - Each block is factorised with ILU(k) (Algorithm 2).
 */
orc_ras *orc_ras_setup(int n, const int *rp, const int *ci, const double *va, int k,
                       int nblocks, int overlap, int *status)
{
    *status = ORC_OK;
    if (n <= 0 || nblocks < 1 || nblocks > n || overlap < 0 || k < 0) {
        *status = ORC_ERR_INVALID;
        return NULL;
    }
    orc_ras *M = (orc_ras *)calloc(1, sizeof(orc_ras));
    M->n = n;
    M->nblocks = nblocks;
    M->own_lo = (int *)malloc(sizeof(int) * (size_t)nblocks);
    M->own_hi = (int *)malloc(sizeof(int) * (size_t)nblocks);
    M->nv = (int *)calloc((size_t)nblocks, sizeof(int));
    M->rows = (int **)calloc((size_t)nblocks, sizeof(int *));
    M->fac = (orc_csr *)calloc((size_t)nblocks, sizeof(orc_csr));
    char *in = (char *)malloc((size_t)n);
    int *g2l = (int *)malloc(sizeof(int) * (size_t)n);
    int maxnv = 0;
    for (int b = 0; b < nblocks; ++b) {
        int lo = (int)((long long)b * n / nblocks);
        int hi = (int)((long long)(b + 1) * n / nblocks);
        M->own_lo[b] = lo;
        M->own_hi[b] = hi;
        memset(in, 0, (size_t)n);
        for (int i = lo; i < hi; ++i)
            in[i] = 1;
        for (int d = 0; d < overlap; ++d) {
            /* V^{d+1} = V^d + neighbours of every row of V^d */
            char *next = (char *)malloc((size_t)n);
            memcpy(next, in, (size_t)n);
            for (int i = 0; i < n; ++i)
                if (in[i])
                    for (int e = rp[i]; e < rp[i + 1]; ++e)
                        next[ci[e]] = 1;
            memcpy(in, next, (size_t)n);
            free(next);
        }
        int nv = 0;
        for (int i = 0; i < n; ++i)
            if (in[i])
                nv++;
        M->nv[b] = nv;
        M->rows[b] = (int *)malloc(sizeof(int) * (size_t)nv);
        nv = 0;
        for (int i = 0; i < n; ++i) {
            g2l[i] = in[i] ? nv : -1;
            if (in[i])
                M->rows[b][nv++] = i;
        }
        if (nv > maxnv)
            maxnv = nv;
        /* A_b = A[V_b, V_b] */
        int *brp = (int *)malloc(sizeof(int) * (size_t)(nv + 1));
        size_t cnt = 0;
        for (int t = 0; t < nv; ++t) {
            int i = M->rows[b][t];
            for (int e = rp[i]; e < rp[i + 1]; ++e)
                if (g2l[ci[e]] >= 0)
                    cnt++;
        }
        int *bci = (int *)malloc(sizeof(int) * (cnt ? cnt : 1));
        double *bva = (double *)malloc(sizeof(double) * (cnt ? cnt : 1));
        cnt = 0;
        brp[0] = 0;
        for (int t = 0; t < nv; ++t) {
            int i = M->rows[b][t];
            for (int e = rp[i]; e < rp[i + 1]; ++e)
                if (g2l[ci[e]] >= 0) {
                    bci[cnt] = g2l[ci[e]];
                    bva[cnt] = va[e];
                    cnt++;
                }
            brp[t + 1] = (int)cnt;
        }
        int st = orc_iluk(nv, brp, bci, bva, k, &M->fac[b]);
        free(brp);
        free(bci);
        free(bva);
        if (st != ORC_OK) {
            *status = st;
            free(in);
            free(g2l);
            orc_ras_free(M);
            return NULL;
        }
    }
    free(in);
    free(g2l);
    M->wr = (double *)malloc(sizeof(double) * (size_t)maxnv);
    M->wy = (double *)malloc(sizeof(double) * (size_t)maxnv);
    M->wz = (double *)malloc(sizeof(double) * (size_t)maxnv);
    return M;
}

/* z = M^{-1} r: for every block, restrict r to V_b, solve L_b U_b z_b = r_b
 * (Eq. 7-8 on the block), and write back only the rows the block owns. */
void orc_ras_apply(const orc_ras *M, const double *r, double *z)
{
    if (M->dinv) { /* damped Jacobi */
        for (int i = 0; i < M->n; ++i)
            z[i] = M->dinv[i] * r[i];
        return;
    }
    for (int b = 0; b < M->nblocks; ++b) {
        const orc_csr *F = &M->fac[b];
        int nv = M->nv[b];
        for (int t = 0; t < nv; ++t)
            M->wr[t] = r[M->rows[b][t]];
        orc_lsolve_unit(nv, F->rp, F->ci, F->va, M->wr, M->wy);
        orc_usolve(nv, F->rp, F->ci, F->va, M->wy, M->wz);
        for (int t = 0; t < nv; ++t) {
            int g = M->rows[b][t];
            if (g >= M->own_lo[b] && g < M->own_hi[b])
                z[g] = M->wz[t];
        }
    }
}

int orc_ras_nblocks(const orc_ras *M) { return M->nblocks; }

int orc_ras_block_size(const orc_ras *M, int b, int *own_lo, int *own_hi)
{
    *own_lo = M->own_lo[b];
    *own_hi = M->own_hi[b];
    return M->nv[b];
}

void orc_ras_block_rows(const orc_ras *M, int b, int *rows)
{
    memcpy(rows, M->rows[b], sizeof(int) * (size_t)M->nv[b]);
}

const orc_csr *orc_ras_block_factor(const orc_ras *M, int b) { return &M->fac[b]; }

/* Preconditioner solve M x = y (Eq. 7); M == NULL is the identity. */
static void precond(const orc_ras *M, int n, const double *y, double *x)
{
    if (M)
        orc_ras_apply(M, y, x);
    else
        memcpy(x, y, sizeof(double) * (size_t)n);
}

/* ------------------------------------------------------------------ */
/* Section 2.7: Krylov solvers                                         */
/* ------------------------------------------------------------------ */

static void true_resid(int n, const int *rp, const int *ci, const double *va,
                       const double *b, const double *x, double *r)
{
    memcpy(r, b, sizeof(double) * (size_t)n);
    orc_spmv(n, rp, ci, va, -1.0, x, 1.0, r);
}

/*
 * BiCGSTAB (Section 2.7), written from the standard derivation: van der
 * Vorst, SIAM J. Sci. Stat. Comput. 13 (1992), and Saad, "Iterative Methods
 * for Sparse Linear Systems", 2nd ed., Section 7.4.2, applied to the right-
 * preconditioned operator B = A M^{-1} (Saad, Section 9.3.2).  With u the
 * iterate of B u = b, x = M^{-1} u is tracked directly, so that every
 * direction p and every intermediate residual s pass through the
 * preconditioner once: p^ = M^{-1} p, s^ = M^{-1} s.  One iteration j:
 *   v = A p^,  alpha = (r, r~) / (v, r~),  s = r - alpha v,
 *   t = A s^,  omega = (t, s) / (t, t),
 *   x += alpha p^ + omega s^,  r = s - omega t,
 *   beta = (r_new, r~) / (r_old, r~) * alpha / omega,
 *   p = r + beta (p - omega v).
 * Readings where the paper leaves a choice open:
 *   - the shadow residual r~ is the initial residual r_0;
 *   - convergence means ||.||_2 <= tol * ||b||_2, tested on s (then
 *     x += alpha p^ alone) and on the new r;
 *   - (r, r~) = 0 or (v, r~) = 0 is a breakdown (status BREAKDOWN); so is
 *     omega = 0 ((t, t) = 0 gives omega = 0) unless r already converged;
 *   - one iteration is one j above;
 *   - b = 0 returns x = 0 at once;
 *   - on exit the true residual ||b - A x|| / ||b|| is recomputed.
 */
int orc_bicgstab(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
                 const double *b, double *x, double tol, int maxit, orc_info *info)
{
    memset(info, 0, sizeof(*info));
    size_t sz = sizeof(double) * (size_t)n;
    double *r = (double *)malloc(sz), *rt = (double *)malloc(sz), *p = (double *)malloc(sz);
    double *ph = (double *)malloc(sz), *v = (double *)malloc(sz), *s = (double *)malloc(sz);
    double *sh = (double *)malloc(sz), *t = (double *)malloc(sz);
    double bnorm = orc_nrm2(n, b);
    int status = ORC_MAXIT;
    int k = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sz);
        status = ORC_OK;
        goto finish;
    }
    true_resid(n, rp, ci, va, b, x, r); /* r = b - A x_0 */
    if (orc_nrm2(n, r) <= tol * bnorm) {
        status = ORC_OK;
        goto finish;
    }
    memcpy(rt, r, sz); /* shadow residual */
    memcpy(p, r, sz);  /* first direction */
    double rho = orc_dot(n, r, rt);
    while (k < maxit) {
        ++k;
        precond(M, n, p, ph);
        orc_spmv(n, rp, ci, va, 1.0, ph, 0.0, v);
        double vr = orc_dot(n, v, rt);
        if (vr == 0.0) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rho / vr;
        orc_waxpby(n, 1.0, r, -alpha, v, s);
        if (orc_nrm2(n, s) <= tol * bnorm) {
            orc_axpby(n, alpha, ph, 1.0, x);
            status = ORC_OK;
            break;
        }
        precond(M, n, s, sh);
        orc_spmv(n, rp, ci, va, 1.0, sh, 0.0, t);
        double tt = orc_dot(n, t, t);
        double omega = (tt == 0.0) ? 0.0 : orc_dot(n, t, s) / tt;
        for (int i = 0; i < n; ++i)
            x[i] += alpha * ph[i] + omega * sh[i];
        orc_waxpby(n, 1.0, s, -omega, t, r);
        if (orc_nrm2(n, r) <= tol * bnorm) {
            status = ORC_OK;
            break;
        }
        if (omega == 0.0) {
            status = ORC_BREAKDOWN;
            break;
        }
        double rho_new = orc_dot(n, r, rt);
        if (rho_new == 0.0) {
            status = ORC_BREAKDOWN;
            break;
        }
        double beta = (rho_new / rho) * (alpha / omega);
        for (int i = 0; i < n; ++i)
            p[i] = r[i] + beta * (p[i] - omega * v[i]);
        rho = rho_new;
    }
finish:
    info->iters = k;
    info->status = status;
    if (bnorm > 0.0) {
        true_resid(n, rp, ci, va, b, x, r);
        info->rel_resid = orc_nrm2(n, r) / bnorm;
    }
    free(r); free(rt); free(p); free(ph); free(v); free(s); free(sh); free(t);
    return status;
}

/*
 * Preconditioned conjugate gradients.  The paper lists CG among the Krylov
 * solvers it implements (Section 2.7) and refers to Saad's book and the
 * Templates for the method; this is their textbook preconditioned form:
 *   r_0 = b - A x_0, z_0 = M^{-1} r_0, p_0 = z_0;
 *   for j = 0, 1, ...: alpha_j = (r_j, z_j) / (A p_j, p_j);
 *     x_{j+1} = x_j + alpha_j p_j;  r_{j+1} = r_j - alpha_j A p_j;
 *     stop when ||r_{j+1}|| <= tol ||b||;
 *     z_{j+1} = M^{-1} r_{j+1};  beta_j = (r_{j+1}, z_{j+1}) / (r_j, z_j);
 *     p_{j+1} = z_{j+1} + beta_j p_j.
 * Readings: one pass of the loop is one iteration; (A p, p) = 0 or
 * (r, z) = 0 before convergence is a breakdown (A or M not positive
 * definite); b = 0 returns x = 0; the true residual is recomputed at exit.
 */
int orc_cg(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
           const double *b, double *x, double tol, int maxit, orc_info *info)
{
    memset(info, 0, sizeof(*info));
    size_t sz = sizeof(double) * (size_t)n;
    double *r = (double *)malloc(sz), *z = (double *)malloc(sz), *p = (double *)malloc(sz);
    double *q = (double *)malloc(sz);
    double bnorm = orc_nrm2(n, b);
    int status = ORC_MAXIT;
    int j = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sz);
        status = ORC_OK;
        goto finish;
    }
    true_resid(n, rp, ci, va, b, x, r); /* r_0 = b - A x_0 */
    if (orc_nrm2(n, r) <= tol * bnorm) {
        status = ORC_OK;
        goto finish;
    }
    precond(M, n, r, z); /* z_0 = M^{-1} r_0 */
    memcpy(p, z, sz);    /* p_0 = z_0 */
    double rz = orc_dot(n, r, z);
    if (rz == 0.0) {
        status = ORC_BREAKDOWN;
        goto finish;
    }
    while (j < maxit) {
        orc_spmv(n, rp, ci, va, 1.0, p, 0.0, q); /* q = A p_j */
        double pq = orc_dot(n, p, q);
        if (pq == 0.0) {
            status = ORC_BREAKDOWN;
            break;
        }
        double alpha = rz / pq;
        orc_axpby(n, alpha, p, 1.0, x);  /* x_{j+1} = x_j + alpha p_j */
        orc_axpby(n, -alpha, q, 1.0, r); /* r_{j+1} = r_j - alpha A p_j */
        ++j;
        if (orc_nrm2(n, r) <= tol * bnorm) {
            status = ORC_OK;
            break;
        }
        precond(M, n, r, z); /* z_{j+1} = M^{-1} r_{j+1} */
        double rz_new = orc_dot(n, r, z);
        if (rz_new == 0.0) {
            status = ORC_BREAKDOWN;
            break;
        }
        double beta = rz_new / rz;
        for (int i = 0; i < n; ++i) /* p_{j+1} = z_{j+1} + beta p_j */
            p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
finish:
    info->iters = j;
    info->status = status;
    if (bnorm > 0.0) {
        true_resid(n, rp, ci, va, b, x, r);
        info->rel_resid = orc_nrm2(n, r) / bnorm;
    }
    free(r); free(z); free(p); free(q);
    return status;
}

/*
 * Restarted GMRES(m), right-preconditioned (A M^{-1} u = b, x = M^{-1} u).
 * The paper lists GMRES among its solvers and defers the method to Saad's
 * book; this follows that textbook form:
 *   cycle: r = b - A x, beta = ||r||, v_1 = r / beta, g = beta e_1;
 *   step j: w = A M^{-1} v_j; modified Gram-Schmidt h_ij = (w, v_i),
 *           w -= h_ij v_i; h_{j+1,j} = ||w||; the earlier Givens rotations
 *           are applied to column j, a new rotation zeroes h_{j+1,j}, g is
 *           rotated; |g_{j+1}| is the residual norm of the current iterate;
 *   the cycle ends when |g_{j+1}| <= tol ||b||, when j = m, when h_{j+1,j}
 *   vanishes (happy breakdown, h_{j+1,j} <= 1e-300 ||w|| before
 *   orthogonalisation) or when the total number of steps reaches maxit;
 *   then y solves the triangular R y = g and x += M^{-1} V y.
 * The solve stops when the recomputed true residual is <= tol ||b||
 * (status OK) or the step budget is spent (status MAXIT).
 */
int orc_gmres(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
              const double *b, double *x, double tol, int maxit, int restart, orc_info *info)
{
    memset(info, 0, sizeof(*info));
    if (restart < 1 || maxit < 0)
        return ORC_ERR_INVALID;
    int m = restart;
    size_t sz = sizeof(double) * (size_t)n;
    double *V = (double *)malloc(sz * (size_t)(m + 1));
    double *r = (double *)malloc(sz), *z = (double *)malloc(sz), *w = (double *)malloc(sz);
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m + j] */
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double bnorm = orc_nrm2(n, b);
    int status = ORC_MAXIT, total = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sz);
        status = ORC_OK;
        goto finish;
    }
    true_resid(n, rp, ci, va, b, x, r);
    double beta = orc_nrm2(n, r);
    if (beta <= tol * bnorm) {
        status = ORC_OK;
        goto finish;
    }
    while (total < maxit) {
        info->restarts++;
        for (int i = 0; i < n; ++i)
            V[i] = r[i] / beta;
        for (int i = 0; i <= m; ++i)
            g[i] = 0.0;
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * (size_t)n;
            precond(M, n, vj, z);
            orc_spmv(n, rp, ci, va, 1.0, z, 0.0, w);
            double wnorm0 = orc_nrm2(n, w);
            for (int i = 0; i <= j; ++i) {
                double *vi = V + (size_t)i * (size_t)n;
                double h = orc_dot(n, w, vi);
                H[i * m + j] = h;
                orc_axpby(n, -h, vi, 1.0, w);
            }
            double hn = orc_nrm2(n, w);
            H[(j + 1) * m + j] = hn;
            /* earlier rotations on column j */
            for (int i = 0; i < j; ++i) {
                double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            /* new rotation zeroing H[j+1][j] */
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double den = sqrt(a * a + c * c);
            cs[j] = (den == 0.0) ? 1.0 : a / den;
            sn[j] = (den == 0.0) ? 0.0 : c / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            total++;
            jend = j + 1;
            info->est_resid = fabs(g[j + 1]) / bnorm;
            int happy = (hn <= 1e-300 * wnorm0) || hn == 0.0;
            if (fabs(g[j + 1]) <= tol * bnorm || happy || total >= maxit)
                break;
            double *vn = V + (size_t)(j + 1) * (size_t)n;
            for (int i = 0; i < n; ++i)
                vn[i] = w[i] / hn;
        }
        /* back substitution R y = g */
        for (int i = jend - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < jend; ++l)
                s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        /* x += M^{-1} V y */
        memset(w, 0, sz);
        for (int l = 0; l < jend; ++l)
            orc_axpby(n, y[l], V + (size_t)l * (size_t)n, 1.0, w);
        precond(M, n, w, z);
        orc_axpby(n, 1.0, z, 1.0, x);
        true_resid(n, rp, ci, va, b, x, r);
        beta = orc_nrm2(n, r);
        if (beta <= tol * bnorm) {
            status = ORC_OK;
            break;
        }
    }
finish:
    info->iters = total;
    info->status = status;
    if (bnorm > 0.0) {
        true_resid(n, rp, ci, va, b, x, r);
        info->rel_resid = orc_nrm2(n, r) / bnorm;
    }
    free(V); free(r); free(z); free(w); free(H); free(cs); free(sn); free(g); free(y);
    return status;
}
