/*
 * hec_oracle.h -- plain FP64 CPU oracle for the ILU(k)/RAS-preconditioned
 * Krylov method of Yang, Liu and Chen, "Development of Krylov and AMG linear
 * solvers for large-scale sparse matrices on GPUs" (Section 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the correctness reference that the
 * CUDA library is checked against.  Only the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark may call it.  It shares no
 * code, header, table or constant with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Everything is CSR, 0-based, int indices, double values, single-threaded,
 * written for clarity rather than speed.  Matrices must have strictly
 * ascending column indices within a row and a stored diagonal.
 *
 * Parity status of each function (see the pins in tests/test_oracle_pins.py):
 *   orc_spmv, orc_dot, orc_nrm2, orc_axpby, orc_waxpby  pinned
 *   orc_iluk                                           pinned
 *   orc_levels                                         pinned
 *   orc_lsolve_unit, orc_usolve                        pinned
 *   orc_ras_*                                          pinned
 *   orc_bicgstab, orc_gmres                            pinned
 *   orc_jacobi_setup, orc_cg                           pinned
 */
#ifndef HEC_ORACLE_H
#define HEC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes of the oracle (its own numbering). */
#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_ZERO_PIVOT (-3)
#define ORC_MAXIT 1
#define ORC_BREAKDOWN 2

/* Eq. 2 (computed row by row as in Algorithm 1): y <- alpha*A*x + beta*y. */
void orc_spmv(int n, const int *rp, const int *ci, const double *va, double alpha,
              const double *x, double beta, double *y);
/* Eq. 5 and Eq. 6. */
double orc_dot(int n, const double *x, const double *y);
double orc_nrm2(int n, const double *x);
/* Eq. 3: y <- a*x + b*y.  Eq. 4: z <- a*x + b*y. */
void orc_axpby(int n, double a, const double *x, double b, double *y);
void orc_waxpby(int n, double a, const double *x, double b, const double *y, double *z);

/* A factor in CSR form, malloc-owned.  For orc_iluk the entries j < i of a row
 * hold the unit-lower factor L (multipliers), j >= i hold U (diagonal
 * included); this is the shared storage of L and U described with Eq. 8.
 * lev[] holds the fill level of every kept entry (Eqs. 9-10). */
typedef struct {
    int n;
    int *rp;
    int *ci;
    double *va;
    int *lev;
} orc_csr;

void orc_csr_free(orc_csr *m);

/* Eqs. 9-10, Algorithm 2: ILU(k) of A.  Returns ORC_OK or
 * ORC_ERR_ZERO_PIVOT (a pivot a_pp == 0 met while eliminating). */
int orc_iluk(int n, const int *rp, const int *ci, const double *va, int k, orc_csr *out);

/* Eq. 11: level of every row of a triangular factor.  upper == 0 uses the
 * entries j < i of each row (forward order), upper == 1 the entries j > i
 * (rows taken from n-1 down to 0, the "reversed L" of Section 2.6).
 * Levels start at 1.  Returns the number of levels. */
int orc_levels(int n, const int *rp, const int *ci, int upper, int *level);

/* Forward substitution with the unit-lower part (entries j < i) of a combined
 * factor, and backward substitution with its upper part (entries j >= i). */
void orc_lsolve_unit(int n, const int *rp, const int *ci, const double *va,
                     const double *b, double *y);
int orc_usolve(int n, const int *rp, const int *ci, const double *va,
               const double *y, double *z);

/* Restricted additive Schwarz preconditioner (Section 2.5), inner level on one
 * device: sequence partition into nblocks contiguous owned row ranges, each
 * grown by `overlap` layers of matrix-graph neighbours, local ILU(k) on each
 * block, restricted (owner-only) write-back. */
typedef struct orc_ras orc_ras;
orc_ras *orc_ras_setup(int n, const int *rp, const int *ci, const double *va, int k,
                       int nblocks, int overlap, int *status);
void orc_ras_apply(const orc_ras *M, const double *r, double *z);
int orc_ras_nblocks(const orc_ras *M);
/* Block b: number of rows of V_b and the owned range [own_lo, own_hi). */
int orc_ras_block_size(const orc_ras *M, int b, int *own_lo, int *own_hi);
/* Block b: the global row ids of V_b (ascending), nv entries. */
void orc_ras_block_rows(const orc_ras *M, int b, int *rows);
/* Block b: its factor (local indices), not owned by the caller. */
const orc_csr *orc_ras_block_factor(const orc_ras *M, int b);
void orc_ras_free(orc_ras *M);

/* orc_spmv on rows [lo, hi) only (for running the row loop on several host
 * threads; identical per-row arithmetic). */
void orc_spmv_range(int n, const int *rp, const int *ci, const double *va, double alpha,
                    const double *x, double beta, double *y, int lo, int hi);

/* Solver outcome. */
typedef struct {
    int iters;          /* BiCGSTAB: loop passes; GMRES: Arnoldi steps */
    int restarts;       /* GMRES cycles started */
    int status;         /* ORC_OK, ORC_MAXIT, ORC_BREAKDOWN */
    double rel_resid;   /* true ||b - A x|| / ||b|| recomputed at exit */
    double est_resid;   /* GMRES: last Givens estimate |g_{j+1}| / ||b|| */
} orc_info;

/* Damped Jacobi preconditioner z = omega D^{-1} r (an orc_ras handle with
 * no blocks: orc_ras_apply and the solvers take it like a RAS one).  status:
 * ORC_OK, ORC_ERR_INVALID (n <= 0 or omega <= 0) or ORC_ERR_ZERO_PIVOT. */
orc_ras *orc_jacobi_setup(int n, const int *rp, const int *ci, const double *va, double omega,
                          int *status);

/* Preconditioned conjugate gradients (Saad / Templates); M == NULL means no
 * preconditioner.  x holds x0 on entry and the solution on exit. */
int orc_cg(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
           const double *b, double *x, double tol, int maxit, orc_info *info);

/* Right-preconditioned BiCGSTAB (Section 2.7; van der Vorst 1992, Saad
 * Section 7.4.2 on A M^{-1}).  M == NULL means no
 * preconditioner.  x holds x0 on entry and the solution on exit. */
int orc_bicgstab(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
                 const double *b, double *x, double tol, int maxit, orc_info *info);

/* Restarted, right-preconditioned GMRES(m) with modified Gram-Schmidt
 * Arnoldi and Givens rotations (the method the paper implements and refers
 * to Saad's book for).  M == NULL means no preconditioner. */
int orc_gmres(int n, const int *rp, const int *ci, const double *va, const orc_ras *M,
              const double *b, double *x, double tol, int maxit, int restart, orc_info *info);

#ifdef __cplusplus
}
#endif
#endif
