/*
 * hecgpu.h -- C ABI of the GB300 (sm_103a) ILU(k)/RAS-preconditioned Krylov
 * library.  The operations follow Yang, Liu and Chen, "Development of Krylov
 * and AMG linear solvers for large-scale sparse matrices on GPUs":
 *   hec_build       HEC matrix format (Section 2.1): a column-major ELL slab
 *                   plus a CSR tail for the entries that do not fit.
 *   hec_spmv        SpMV on HEC (Section 2.2, Algorithm 1, Eqs. 1-2).
 *   hec_axpby ...   vector operations (Section 2.3, Eqs. 3-6).
 *   ilu_k_setup     ILU(k) (Section 2.4, Eqs. 8-10, Algorithm 2) on every
 *                   block of a restricted additive Schwarz partition
 *                   (Section 2.5).
 *   level_schedule  level sets of every L_b and U_b (Section 2.6, Eq. 11,
 *                   Algorithm 3) and the device layout the solver streams.
 *   hec_precond_apply  z = M^{-1} r, M the RAS/ILU(k) preconditioner
 *                   (Eq. 7), by level-scheduled triangular solves.
 *   krylov_solve    preconditioned BiCGSTAB (Section 2.7, Algorithm 4) or
 *                   restarted GMRES(m) (Section 2.7).
 *
 * Conventions
 *   - Every call returns int: 0 (HEC_OK), a negative error code, or a
 *     positive solver outcome (HEC_MAXIT, HEC_BREAKDOWN).  No exception
 *     crosses the ABI.  hec_last_error() returns a message for the calling
 *     thread's last failure.
 *   - Indices are 0-based int32.  A CSR matrix must be square, with strictly
 *     ascending column indices in every row (else HEC_ERR_UNSORTED_CSR);
 *     ilu_k_setup also needs every diagonal entry stored.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is ordered on it; calls that return host data
 *     (queries, krylov_solve's info) synchronise it.
 *   - Handles own their device memory.  It comes from the allocator set with
 *     hec_set_allocator (default: the stream-ordered cudaMallocAsync /
 *     cudaFreeAsync on the stream a handle was created with, so destroy a
 *     handle before that stream).  Vectors passed in
 *     (x, y, r, z, b) are owned by the caller and only borrowed for the call.
 *   - Values are FP64.  There is no CPU fallback: a call that needs the
 *     device fails with HEC_ERR_CUDA when no CUDA device is present.
 */
#ifndef HECGPU_H
#define HECGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define HEC_OK 0
#define HEC_ERR_INVALID (-1)      /* bad argument or handle state            */
#define HEC_ERR_OOM (-2)          /* device or host memory exhausted         */
#define HEC_ERR_ZERO_PIVOT (-3)   /* ILU(k) met a pivot equal to zero        */
#define HEC_ERR_UNSORTED_CSR (-4) /* columns not strictly ascending / range  */
#define HEC_ERR_CUDA (-5)         /* a CUDA runtime call failed              */
#define HEC_ERR_TIMEOUT (-6)      /* a bounded device wait ran out           */
#define HEC_ERR_DEBUG (-7)        /* a device-side check of the debug build
                                     (compiled with HEC_DEBUG) failed; see
                                     hec_debug_record                       */
#define HEC_MAXIT 1               /* solver stopped at maxit                 */
#define HEC_BREAKDOWN 2           /* BiCGSTAB rho = 0, (r0,v) = 0, omega = 0  */

/* ---------------------------------------------------------------- types */
typedef struct hec_matrix_s *hec_matrix_t;   /* HEC matrix on the device     */
typedef struct hec_precond_s *hec_precond_t; /* RAS blocks, ILU(k) factors   */

/* A CSR matrix, borrowed for the call (copied). */
typedef struct {
    int32_t n;              /* rows = columns, >= 1                          */
    int32_t nnz;            /* row_ptr[n]                                    */
    const int32_t *row_ptr; /* n + 1 entries                                 */
    const int32_t *col;     /* nnz entries                                   */
    const double *val;      /* nnz entries                                   */
    int32_t on_device;      /* 0: the three arrays are host memory; 1: device */
} hec_csr_t;

/* Options of hec_build.  A zeroed struct (or NULL) selects the defaults. */
typedef struct {
    int32_t ell_width;    /* K, entries per row kept in the ELL slab; 0 = auto
                             (largest K that at least a third of the rows
                             reach); the rest of a longer row goes to the CSR
                             tail                                           */
    int32_t ell_ld_align; /* slab leading dimension = n rounded up to this
                             multiple of 32; 0 = 256 (Section 2.1)           */
    int32_t flags;        /* HEC_HOST_ONLY: keep the host structure only (no
                             device memory; queries work, compute calls
                             return HEC_ERR_INVALID)                        */
    int32_t reserved;
} hec_opts_t;

#define HEC_HOST_ONLY 1

typedef struct {
    int32_t n, nnz;
    int32_t ell_width;  /* K                                                  */
    int32_t ell_ld;     /* slab leading dimension                             */
    int32_t tail_rows;  /* rows with more than K entries                      */
    int32_t tail_nnz;   /* entries stored in the CSR tail                     */
    int64_t device_bytes;
} hec_matrix_info_t;

typedef struct {
    int32_t nblocks, overlap, k;
    int32_t scheduled;       /* level_schedule has run                        */
    int64_t rows_total;      /* sum over blocks of |V_b|                      */
    int64_t factor_nnz;      /* sum over blocks of nnz(L_b) + nnz(U_b)        */
    int32_t max_levels_L;    /* largest level count of an L_b                 */
    int32_t max_levels_U;    /* largest level count of a U_b                  */
    int64_t apply_bytes;     /* algorithmic bytes one hec_precond_apply moves  */
    int64_t device_bytes;
    int32_t ring_slots;      /* shared-memory window of solved values          */
    int32_t global_passes;   /* (block, factor) solves whose dependencies do
                                not fit the window and are read from global
                                memory instead                                */
    int64_t apply_bytes_f32; /* the same for the FP32 layout (0 until built)   */
    int32_t trsv_parts;      /* CTAs per RAS block of the FP64 triangular solve */
    int32_t import_slots;    /* shared-memory window of values received from a
                                neighbouring CTA (0: no block is split)        */
    int32_t split_blocks;    /* RAS blocks solved by more than one CTA         */
    int32_t trsv_resident;   /* 1: the FP64 triangular solves run the resident-
                                vector kernel (hec_precond_set_trsv_kernel)    */
} hec_precond_info_t;

#define HEC_GMRES 0
#define HEC_BICGSTAB 1
/* Preconditioned conjugate gradients (Section 2.7 lists CG among the Krylov
 * methods and refers to Saad's book for it): r_0 = b - A x_0, z = M^{-1} r,
 * p = z; per pass alpha = (r, z) / (A p, p), x += alpha p, r -= alpha A p,
 * stop when ||r|| <= tol ||b||, z = M^{-1} r, beta = (r_new, z_new) /
 * (r, z), p = z + beta p.  For symmetric positive definite A and M (ILU(k)
 * with one block of a symmetric matrix, damped Jacobi, none); (A p, p) = 0
 * or (r, z) = 0 before convergence ends with HEC_BREAKDOWN.  FP64 only. */
#define HEC_CG 2

typedef struct {
    int32_t method;     /* HEC_GMRES, HEC_BICGSTAB or HEC_CG                  */
    int32_t flags;      /* HEC_X0_ZERO: ignore the content of x, start at 0;
                           HEC_SOLVE_EAGER: launch the solve's kernels
                           directly on the stream and drive the loop from the
                           host (one small read per iteration) instead of the
                           device-side graph loop -- same kernels, same
                           results; for profilers that cannot see the kernels
                           of a graph with conditional nodes                */
    int64_t spin_limit; /* polls of a device wait before HEC_ERR_TIMEOUT;
                           0 = default (about a second)                      */
} hec_solve_opts_t;

#define HEC_X0_ZERO 1
#define HEC_SOLVE_EAGER 2
/* Mixed precision (GMRES only): every restart cycle is an inner solve in FP32
 * -- FP32 SpMV, FP32 ILU(k) triangular solves, FP32 Krylov basis, FP32
 * products and accumulation -- and FP64 is kept for the outer residual
 * r = b - A x recomputed at every cycle start, the update of x, and the
 * Hessenberg least-squares / Givens step: FP64 iterative refinement with
 * FP32 GMRES cycles.  Convergence is judged on the FP64 residual.  A cycle
 * also ends when its FP32 estimate has dropped by 1e-5. */
#define HEC_MIXED_FP32 4

typedef struct {
    int32_t iters;          /* BiCGSTAB, CG passes / GMRES Arnoldi steps      */
    int32_t restarts;       /* GMRES cycles started                           */
    int32_t status;         /* HEC_OK, HEC_MAXIT, HEC_BREAKDOWN or an error   */
    int32_t fp64_finish;    /* HEC_MIXED_FP32: the FP32 cycles stopped refining
                               (two cycles in a row left a true FP64 residual
                               above 10x the cycle's own final estimate and
                               above half the cycle's starting residual, or
                               eight cycles in a row each cut it by less than
                               10%) and
                               the solve was finished in FP64 from the current
                               x (iters, restarts count both phases); batched
                               solves: the number of systems finished so    */
    double rel_resid;       /* true ||b - A x|| / ||b|| recomputed at the end */
    double est_resid;       /* GMRES: last Givens estimate / ||b||; BiCGSTAB:
                               last recursive residual / ||b||                */
    int64_t kernel_launches;/* library kernels the solve ran                  */
    int64_t h2d_bytes;      /* host->device bytes copied (host b / x)         */
    int64_t d2h_bytes;      /* device->host bytes copied (host x)             */
} hec_solve_info_t;

/* ---------------------------------------------------------------- misc */
const char *hec_status_string(int status);
/* Message describing the calling thread's last failing call ("" if none). */
const char *hec_last_error(void);
/* Device allocator for every handle and workspace allocation: alloc(bytes,
 * stream, ctx) returns device memory or NULL; free(ptr, stream, ctx).  NULL
 * functions restore cudaMalloc / cudaFree.  Affects later allocations only;
 * memory is always returned through the allocator that produced it. */
int hec_set_allocator(void *(*alloc_fn)(size_t bytes, void *stream, void *ctx),
                      void (*free_fn)(void *ptr, void *stream, void *ctx), void *ctx);

/* ---------------------------------------------------------------- HEC matrix */
/* Section 2.1: convert A to HEC (ELL slab + CSR tail) and upload it.  The
 * slab is column-major, entry k of row i at [k * ell_ld + i]; short rows are
 * padded with value 0 and their own row index as column. */
int hec_build(const hec_csr_t *A, const hec_opts_t *opts, void *stream, hec_matrix_t *out);
int hec_matrix_info(hec_matrix_t A, hec_matrix_info_t *info);
/* Host copies of the HEC arrays (each pointer may be NULL to skip it):
 * ell_col/ell_val: K * ell_ld entries; tail_rows: tail_rows entries;
 * tail_ptr: tail_rows + 1; tail_col/tail_val: tail_nnz. */
int hec_matrix_export(hec_matrix_t A, int32_t *ell_col, double *ell_val, int32_t *tail_rows,
                      int32_t *tail_ptr, int32_t *tail_col, double *tail_val);
void hec_matrix_destroy(hec_matrix_t A);

/* Eq. 2 (Algorithm 1): y_out = alpha * A x + beta * y_in on the device.
 * y_in may equal y_out; it is not read when beta == 0; x must not overlap
 * y_out.  x, y_in, y_out: device arrays of n doubles; y_out must be 16-byte
 * aligned (rows are stored in pairs; HEC_ERR_INVALID otherwise, before any
 * device work).  When dots != NULL (device, 2 doubles) the
 * reductions of the result are fused into the same launch:
 * dots[0] = (w, y_out) (w: device array of n doubles; NULL means y_out) and
 * dots[1] = (y_out, y_out), each summed in a fixed order (deterministic). */
int hec_spmv(hec_matrix_t A, double alpha, const double *x, double beta, const double *y_in,
             double *y_out, const double *w, double *dots, void *stream);

/* The FP32 SpMV of the mixed-precision inner solves, Eq. 2 with FP32 values
 * (the matrix's values rounded once to FP32, kept beside the FP64 ones after
 * the first FP32 call), FP32 products and accumulation.  x, y_in, y_out:
 * device arrays of n floats, y_out 16-byte aligned (rows are stored four at
 * a time; HEC_ERR_INVALID otherwise, before any device work); no fused dots. */
int hec_spmv_f32(hec_matrix_t A, float alpha, const float *x, float beta, const float *y_in,
                 float *y_out, void *stream);

/* ---------------------------------------------------------------- vector ops */
/* Eqs. 3-6 on device arrays of n doubles.  hec_dot / hec_nrm2 write their
 * result to *result (device, 1 double), summed in a fixed order. */
int hec_axpby(int32_t n, double a, const double *x, double b, double *y, void *stream);
int hec_waxpby(int32_t n, double a, const double *x, double b, const double *y, double *z,
               void *stream);
int hec_dot(int32_t n, const double *x, const double *y, double *result, void *stream);
int hec_nrm2(int32_t n, const double *x, double *result, void *stream);
/* Arnoldi projection: h[i] = (V_i, w) for i < k, V column-major with leading
 * dimension ldv (>= n), h: device array of k doubles. */
int hec_multidot(int32_t n, int32_t k, const double *V, int64_t ldv, const double *w, double *h,
                 void *stream);

/* ---------------------------------------------------------------- preconditioner */
/* Damped Jacobi (Section 2.8 builds it, as a smoother, from the SpMV and
 * vector operations): the preconditioner z = omega D^{-1} r, D the diagonal
 * of A, usable wherever an ILU(k)/RAS handle is (apply calls, krylov_solve
 * with any method, the mixed-precision mode).  omega / a_ii is formed once
 * on the host in FP64 and kept on the device (an FP32 copy is made on the
 * first FP32 use).  The handle needs no level_schedule (calling it is a
 * no-op); hec_precond_info reports k = -1, nblocks = 0 and 24 n algorithmic
 * bytes per apply; the block/factor/level queries return HEC_ERR_INVALID.
 * Returns HEC_ERR_INVALID for omega <= 0 or not finite, HEC_ERR_ZERO_PIVOT
 * for a zero or missing diagonal entry. */
int hec_jacobi_setup(hec_matrix_t A, double omega, void *stream, hec_precond_t *out);
/* Sections 2.4-2.5: partition the rows into nblocks contiguous owned ranges
 * W_b = [floor(b n / nblocks), floor((b+1) n / nblocks)), grow each by
 * `overlap` layers of matrix-graph neighbours (V_b), and factorise every
 * A[V_b, V_b] by ILU(k).  Factors are computed on the host and kept there
 * until level_schedule uploads them.  Returns HEC_ERR_ZERO_PIVOT if a pivot
 * is zero, HEC_ERR_INVALID if a diagonal entry is missing. */
int ilu_k_setup(hec_matrix_t A, int32_t k, int32_t nblocks, int32_t overlap, void *stream,
                hec_precond_t *out);
/* Section 2.6 (Eq. 11, Algorithm 3): level of every row of every L_b and
 * U_b, and the level-major device layout of the factors.  Idempotent. */
int level_schedule(hec_precond_t M, void *stream);
int hec_precond_info(hec_precond_t M, hec_precond_info_t *info);
/* Block b: |V_b| (*nv), the owned range, and the global row ids of V_b in
 * ascending order (rows may be NULL). */
int hec_precond_get_block(hec_precond_t M, int32_t b, int32_t *nv, int32_t *own_lo,
                          int32_t *own_hi, int32_t *rows);
/* Block b: the combined ILU(k) factor of A[V_b, V_b] in local indices (L
 * strictly below the diagonal, unit diagonal implied; U on and above),
 * host copies; any array may be NULL, *nnz is always set. */
int hec_precond_get_factor(hec_precond_t M, int32_t b, int32_t *nnz, int32_t *row_ptr,
                           int32_t *col, double *val, int32_t *lev);
#define HEC_FACTOR_L 0
#define HEC_FACTOR_U 1
/* Block b, factor L or U: number of levels (Eq. 11) and the level sets,
 * level_ptr (nlev + 1) and level_rows (local row ids, ascending inside each
 * level); arrays may be NULL. */
int hec_precond_get_levels(hec_precond_t M, int32_t b, int32_t which, int32_t *nlev,
                           int32_t *level_ptr, int32_t *level_rows);
/* The level-major factor layout that the triangular solves stream (Section
 * 2.6, Eq. 11: the rows of every level of L_b, then of U_b), host copies, for
 * inspection and host-side checks.  fp32 = 0: the FP64 layout; fp32 = 1: the
 * FP32 layout of the mixed-precision mode (packed, and on a device handle
 * uploaded, on first request).  *pack_bytes, *nchunks, *ring_slots (R, the
 * shared-memory window of a CTA's own solved values, a power of two),
 * *import_slots (RI, the window of values received from a neighbouring CTA;
 * 0 when no block is split), *parts (P, CTAs per RAS block) and *fixed_width
 * (0, or the one segment width of every warp) are always set; pack
 * (pack_bytes bytes), chunks (2 per chunk: byte offset / 16, byte count) and
 * programs (8 per CTA, nblocks * P of them, block b's part p at b * P + p:
 * first chunk, first U chunk, end chunk, ring_L, ring_U -- 1 when that pass
 * reads dependencies from shared memory, 0 when from the global scratch --
 * the program's y and z scratch offsets, and links: bit 0 when part p - 1 of
 * the block exists, bit 1 when part p + 1 does) may be NULL.
 *
 * A part is a contiguous range of the block's local rows; L_b is lower
 * triangular in that order, so in the L pass part p reads only its own and
 * part p - 1's values, in the U pass its own and part p + 1's.  A block is
 * split only when no dependency reaches further.
 *
 * A chunk holds rows of one level.  It starts with 28 int32: row count,
 * warp count, position (in the part's level-major order) of its first row,
 * flags (bit 0: U pass, bit 1: exports, bit 2: no warp segment wider than
 * 8 entries), the entry width of each of 8 warp
 * segments, each segment's byte offset, the byte offsets of src, dst, dinv
 * and exp, need_prev and need_next (the completed-chunk counts of parts
 * p - 1 and p + 1 this chunk waits for), and two zeros.  Segment w covers
 * rows 32w .. 32w+31 as val[width][stride] (8- or 4-byte values) then
 * dep[width][stride] (int32); stride is 32, or for the last warp its row
 * count rounded up to 4.  In a pass read from shared memory dep is a slot:
 * own values at slot position & (R - 1), values from the neighbouring part
 * at R + (import position & (RI - 1)); otherwise dep is a position of the
 * same pass in the global scratch.  Row t of the L pass computes
 * y[pos] = r[src[t]] - sum_k val[k] y[dep[k]]; of the U pass
 * z[pos] = (y[src[t]] - sum_k val[k] z[dep[k]]) * dinv[t], written to
 * global row dst[t] when dst[t] >= 0 (an owned row).  exp[t] >= 0 is the
 * slot that row's value takes in the neighbour's ring (L: part p + 1, U:
 * part p - 1).  Padding entries have value 0.
 *
 * Layouts of the resident kernel (hec_precond_info_t.trsv_resident; chunk
 * flag bit 5) have one program per block (*parts = 1) whose y scratch offset
 * is the offset of the block's V_b in the kernel's row list and whose z
 * scratch offset is its first group of consecutive chunks (the kernel
 * streams a group of up to 16 KB with one bulk copy; flag bit 6 marks a
 * group's last chunk), and chunks of 8 int32 (row count, warp count, first
 * position, flags, the next chunk's offset in its group's stage and its
 * warp count, FW, 0) followed, for each of the kernel's solving warps (every
 * chunk has the same size; warps past the row count hold padding), by val
 * (ceil(FW / VW) vectors of 32 lanes x 16 bytes, VW = 16 / value bytes: lane
 * l's entries k VW .. k VW + VW - 1 in vector k), idx (ceil((FW + 1) / 8)
 * vectors of 32 lanes x 8 uint16: lane l's FW dependency slots, then its own
 * slot) and dinv[32] (read in the U pass).
 * Slots are the block's local row indices; slot nv (the block's row count)
 * holds 0 and pads short rows and the rows past the chunk's end.  Row t of
 * the L pass computes x[own] -= sum_k val[k] x[dep[k]] with x = r on V_b at
 * the start; of the U pass x[own] = (x[own] - sum_k val[k] x[dep[k]]) *
 * dinv[t]; z on the owned rows is x at the end.  The stream must be NULL or
 * a CUDA stream; a device handle's layout is read back on it
 * (synchronously).  HEC_ERR_INVALID for a damped-Jacobi handle or before
 * level_schedule. */
int hec_precond_get_layout(hec_precond_t M, int32_t fp32, int64_t *pack_bytes, int32_t *nchunks,
                           int32_t *ring_slots, int32_t *import_slots, int32_t *parts,
                           int32_t *fixed_width, void *pack, uint32_t *chunks, int64_t *programs,
                           void *stream);
/* CTAs that solve each RAS block's triangular systems (Section 2.6: the
 * rows of one level are independent, so they may be spread over several
 * SMs): 0 = automatic (split while the widest block's levels hold more than
 * 128 rows per CTA in the FP64 layout, 256 in the FP32 one, and nblocks * P
 * CTAs fit on the device's SMs), or 1, 2, 4 or 8 for both layouts.  The CTAs of one block run as one thread-block cluster.  A block
 * whose dependencies do not allow the split gets fewer parts.  Call it
 * between ilu_k_setup and level_schedule; HEC_ERR_INVALID afterwards, for a
 * damped-Jacobi handle or another value. */
int hec_precond_set_trsv_parts(hec_precond_t M, int32_t parts);
/* Which kernel applies the triangular solves (Section 2.6, Eq. 11: both walk
 * the levels of L_b, then of U_b, and give the same z up to the rounding of
 * the per-row sums, which are taken in the same order):
 *   HEC_TRSV_STREAMED -- the level-major chunks stream through a shared-
 *     memory ring of recent solved values; the right-hand sides are gathered
 *     per chunk from r (L) and from a global y scratch (U); a block may be
 *     split over the CTAs of a cluster (hec_precond_set_trsv_parts).  For
 *     large blocks.
 *   HEC_TRSV_RESIDENT -- one CTA per block keeps the block's whole vector in
 *     shared memory and solves in place: a level's critical path is shared
 *     memory, the row's multiply-adds and one barrier.  For blocks below
 *     65535 rows whose factor rows hold at most 8 entries and whose vector
 *     (rows + 1 values) fits in shared memory beside three chunk stages:
 *     the latency-first form for small systems.
 *   HEC_TRSV_AUTO (default) -- resident when every block fits, no level
 *     holds more than 128 rows and the streamed kernel would not split a
 *     block over several CTAs (measured on GB300: 1.1-1.2x faster there,
 *     slower on wider levels), else streamed.
 * The FP32 layout of the mixed-precision mode follows the same rule.  Call
 * it between ilu_k_setup and level_schedule; HEC_ERR_INVALID afterwards,
 * for a damped-Jacobi handle or another value; level_schedule returns
 * HEC_ERR_INVALID when HEC_TRSV_RESIDENT is asked for and a block does not
 * fit. */
#define HEC_TRSV_AUTO 0
#define HEC_TRSV_STREAMED 1
#define HEC_TRSV_RESIDENT 2
int hec_precond_set_trsv_kernel(hec_precond_t M, int32_t kernel);
/* Debug builds (compiled with HEC_DEBUG; not a counterpart of anything in the
 * paper): the triangular-solve kernel checks every chunk header against the
 * position its program has reached, every gathered index against n, and
 * every dependency slot against the ring, and on a violation skips the
 * access, sets the error word to HEC_ERR_DEBUG and records the first one.
 * record: 8 int32 -- code (1 pass flag, 2 row count, 3 gathered index,
 * 4 chunk position, 5 ring slot, 6 scratch position, 7 destination row;
 * 0 = none), program, chunk, thread, value, bound, 0, 0.  clear != 0 resets
 * it.  HEC_ERR_INVALID in a release build. */
int hec_debug_record(int32_t *record, int32_t clear);
/* z = M^{-1} r (Eq. 7 with M = the RAS combination of L_b U_b): every block
 * gathers r on V_b, solves L_b then U_b level by level, and writes z on its
 * owned rows only.  r, z: device arrays of n doubles, r != z.  Needs
 * level_schedule.  Waits are bounded by spin_limit polls (0 = default); a
 * wait that runs out is reported by hec_precond_status. */
int hec_precond_apply(hec_precond_t M, const double *r, double *z, int64_t spin_limit,
                      void *stream);
/* Synchronise the stream and return (and clear) the device error word of
 * the preconditioner: HEC_OK or HEC_ERR_TIMEOUT. */
int hec_precond_status(hec_precond_t M, void *stream);
/* The same z = M^{-1} r as hec_precond_apply, for callers that must not
 * allocate device memory while they run: for example a time-stepping code
 * whose device memory budget is fixed at start-up and shared with other
 * processes, or a latency-bound loop that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree.  (The paper has no counterpart;
 * it is a property of this library's interface.)  The call allocates
 * nothing: the solve's intermediate vectors live in one static device array
 * of 2^20 doubles (8 MiB) inside the library, which every device that loads
 * the library holds until the process exits.  A preconditioner whose scratch
 * (sum over blocks of the rows solved, plus the rows of blocks that read
 * dependencies from global memory) exceeds 2^20 doubles is rejected with
 * HEC_ERR_INVALID; hec_precond_apply has no such limit.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong results, so serialise them.  Nothing in the
 * array needs to start at zero.  Arguments, ownership and the bounded-wait
 * status word are as for hec_precond_apply. */
int hec_precond_apply_noalloc(hec_precond_t M, const double *r, double *z, int64_t spin_limit,
                              void *stream);
/* The FP32 preconditioner of the mixed-precision inner solves: the same
 * z = M^{-1} r with the ILU(k) factors rounded once to FP32 (a second device
 * layout, built on first use) and FP32 arithmetic.  r, z: device arrays of n
 * floats, r != z.  Status as for hec_precond_apply. */
int hec_precond_apply_f32(hec_precond_t M, const float *r, float *z, int64_t spin_limit,
                          void *stream);
void hec_precond_destroy(hec_precond_t M);
/* Numeric refactorisation on the GPU: A keeps its sparsity pattern and takes
 * the nnz new values `val` (host or device array of doubles, in the CSR
 * order A was built from).  The HEC slab and tail (Section 2.1) are
 * rewritten on the device (and their FP32 copies, if made).  When M is not
 * NULL it must have been built from A: a damped-Jacobi handle recomputes
 * omega / a_ii; an ILU(k)/RAS handle (level_schedule done) recomputes every
 * block's factor on its existing fill pattern -- the pattern of Eqs. 9-10
 * depends on the structure only -- by the elimination of Algorithm 2, one
 * CTA per RAS block, rows of one L level (Eq. 11) in parallel, with the
 * host's operation order and rounding (the factors are bit-identical to a
 * fresh ilu_k_setup of the new matrix), and refills the values of its
 * triangular-solve layouts.  Solve graphs and handles stay valid.  The first
 * call per handle uploads index maps (about 12 bytes per matrix entry and 16
 * per factor entry), later calls only stream values.  The call synchronises
 * the stream.  Returns HEC_OK, HEC_ERR_ZERO_PIVOT (the factors are then
 * unusable until the next successful refactor) or HEC_ERR_INVALID. */
int hec_refactor(hec_matrix_t A, hec_precond_t M, const double *val, void *stream);

/* ---------------------------------------------------------------- Krylov */
/* Section 2.7: solve A x = b with the right-preconditioned BiCGSTAB of
 * Algorithm 4, restarted GMRES(restart) or preconditioned CG (opts->method),
 * M == NULL meaning no preconditioner; M is an ILU(k)/RAS or a damped-Jacobi
 * handle.  Convergence: ||r|| <= tol ||b|| (BiCGSTAB, CG: the recursive
 * residual; GMRES: the true residual checked at every cycle end).  b and x
 * are device or host arrays of n doubles (host arrays are staged through
 * device memory; the byte counts are reported in info);
 * x holds x0 on entry unless HEC_X0_ZERO, and the solution on exit.  The
 * whole iteration runs on the device as one CUDA graph with a device-side
 * loop condition; the call synchronises the stream at the end.  Returns
 * HEC_OK, HEC_MAXIT, HEC_BREAKDOWN or an error; info may be NULL. */
int krylov_solve(hec_matrix_t A, hec_precond_t M, const double *b, double *x, double tol,
                 int32_t maxit, int32_t restart, const hec_solve_opts_t *opts, void *stream,
                 hec_solve_info_t *info);
/* Device bytes that the first krylov_solve(A, M, ..., restart, opts) with
 * these method, restart and precision arguments allocates beyond what the
 * handles already hold (*bytes; 0 once such a solve has run, since the
 * workspace stays cached in the handles):
 *   - the solver's FP64 vectors and Krylov basis (and, for HEC_MIXED_FP32,
 *     its FP32 ones), padded to a multiple of 32 entries;
 *   - its device-resident state and the reduction scratch, which scales with
 *     the device's SM count;
 *   - with HEC_MIXED_FP32, the FP32 copies of A's values and of M's factor
 *     layout (or Jacobi diagonal) that the first mixed solve makes.  The
 *     FP32 layout is packed on the host here to be counted.
 * A mixed solve that finishes in FP64 also allocates what this call
 * reports without HEC_MIXED_FP32.  Host work only; host-only handles
 * work.  HEC_ERR_INVALID for arguments krylov_solve would reject. */
int hec_workspace_bytes(hec_matrix_t A, hec_precond_t M, int32_t restart,
                        const hec_solve_opts_t *opts, int64_t *bytes);

/* ---------------------------------------------------------------- batches */
/* Many independent systems A_s x_s = b_s (s = 0 .. nsys-1), each with nrhs
 * right-hand sides, solved by ONE persistent kernel launch: every system is
 * solved start to finish by one CTA, the costliest systems first, with the
 * same operations as the single-system path -- HEC SpMV (Eq. 2, Algorithm
 * 1), ILU(k) factors (Eqs. 9-10, Algorithm 2) applied by level-scheduled
 * triangular solves (Eq. 11, Algorithm 3), restarted GMRES(m) (Section 2.7)
 * -- and up to 4 right-hand sides of a system advanced in lockstep, so the
 * matrix and factor entries are read once for all of them.  The paper solves
 * one system at a time; batching is this library's extension.
 *
 * A system's arithmetic depends only on the system, nrhs and the batch
 * configuration (threads per CTA), never on the other systems: a system gives
 * bit-identical results alone and in any batch solved with the same
 * configuration. */
typedef struct hec_batch_s *hec_batch_t;

/* The systems as one concatenated CSR (host memory, copied).  System s owns
 * global rows [sys_ptr[s], sys_ptr[s+1]); its column indices are local to it
 * (0 .. n_s - 1), strictly ascending in every row, diagonal stored. */
typedef struct {
    int32_t nsys;            /* >= 1                                          */
    int32_t reserved;
    const int64_t *sys_ptr;  /* nsys + 1 entries, sys_ptr[0] = 0              */
    const int64_t *row_ptr;  /* sys_ptr[nsys] + 1 entries into col / val      */
    const int32_t *col;
    const double *val;
} hec_batch_csr_t;

/* Launch configuration of the batched kernel.  Zero fields take defaults. */
typedef struct {
    int32_t threads;      /* CTA size: 128, 256 or 512; 0 = 256                 */
    int32_t ctas_per_sm;  /* resident CTAs per SM; 0 = as many as fit (<= 4)    */
    int32_t ell_width;    /* 0: per system, the largest K that a third of its
                             rows reach; > 0: this K for every system.  Rows
                             longer than K are stored whole in the CSR tail   */
    int32_t nstages;      /* bulk-copy stages of the triangular solves; 0 = 8   */
} hec_batch_config_t;

typedef struct {
    int32_t nsys;
    int32_t ilu_k;           /* -1 before ilu_k_setup_batched                  */
    int64_t rows, nnz;       /* totals over the systems                         */
    int64_t factor_nnz;      /* sum of nnz(L_s) + nnz(U_s)                      */
    int32_t max_n;           /* largest system                                  */
    int32_t ring_slots;      /* shared-memory window of solved values (positions) */
    int64_t device_bytes;    /* matrices, factors and the last solve's workspace */
    hec_batch_config_t config;
} hec_batch_info_t;

/* Outcome of one system (the worst of its right-hand sides). */
typedef struct {
    int32_t iters;      /* Arnoldi steps, summed over groups of 4 right-hand sides */
    int32_t cycles;     /* restart cycles                                         */
    int32_t status;     /* HEC_OK, HEC_MAXIT, HEC_BREAKDOWN                        */
    int32_t reorth;     /* Arnoldi steps whose classical Gram-Schmidt took a third
                           (re-orthogonalising) pass: the second projection lost
                           more than half of ||w||^2 for one of the right-hand sides */
    double rel_resid;   /* largest true ||b - A x|| / ||b|| over its right-hand sides */
} hec_batch_sys_info_t;

/* Builds the batch: copies and checks every system (HEC_ERR_UNSORTED_CSR,
 * HEC_ERR_INVALID as for hec_build).  cfg may be NULL.  Device memory is laid
 * out on first use. */
int hec_build_batched(const hec_batch_csr_t *A, const hec_batch_config_t *cfg, void *stream,
                      hec_batch_t *out);
/* ILU(k) of every system (Eqs. 9-10, Algorithm 2) and the level sets of its
 * factors (Eq. 11); the unknowns of a system are then stored in the level
 * order of L.  Returns HEC_OK, HEC_ERR_ZERO_PIVOT (system index in
 * hec_last_error) or HEC_ERR_INVALID. */
int ilu_k_setup_batched(hec_batch_t B, int32_t k);
int hec_batch_info(hec_batch_t B, hec_batch_info_t *info);
/* Replaces the launch configuration (the ELL width rebuilds the layout). */
int hec_batch_set_config(hec_batch_t B, const hec_batch_config_t *cfg);
/* Autotuner: times the solve of a sample of the systems (about eight per SM,
 * spread over the size range, one restart cycle each) under candidate
 * configurations -- CTA size, CTAs per SM, bulk-copy stages and ELL width --
 * keeps the fastest in B and returns it in *chosen (may be NULL).  nrhs,
 * restart and opts (HEC_MIXED_FP32) as the solves it tunes for. */
int hec_batch_autotune(hec_batch_t B, int32_t nrhs, int32_t restart,
                       const hec_solve_opts_t *opts, void *stream, hec_batch_config_t *chosen);
/* Solves every system.  b, x: device or host arrays of sys_ptr[nsys] x nrhs
 * doubles, row-major (value of right-hand side r of global row i at
 * i * nrhs + r); x holds x0 unless HEC_X0_ZERO.  tol, maxit (Arnoldi steps
 * per group of <= 4 right-hand sides), restart (<= 31) as for krylov_solve.
 * Without HEC_MIXED_FP32 the inner cycles run in FP64; with it, in FP32
 * inside FP64 refinement (cycles end when their estimate has dropped by
 * 1e-5); a system whose FP32 cycles stop refining (see fp64_finish) is
 * finished in FP64 from its current x by a second launch
 * restricted to such systems (info->fp64_finish counts them).  A right-hand
 * side with b = 0 returns x = 0.  One kernel launch (two with FP64 finishes);
 * the call synchronises the stream.  Returns HEC_OK when every system
 * converged, else the first non-OK system status, or an error.  info (sums
 * over systems, rel_resid the largest) and sys_info (nsys entries, host) may
 * be NULL. */
int krylov_solve_batched(hec_batch_t B, const double *b, double *x, int32_t nrhs, double tol,
                         int32_t maxit, int32_t restart, const hec_solve_opts_t *opts,
                         void *stream, hec_solve_info_t *info, hec_batch_sys_info_t *sys_info);
/* The batched kernel's single operations, for tests: x = A b per system
 * (op 0: FP64 values; op 1: FP32 values and arithmetic) and x = M^{-1} b
 * (op 2: FP32 factors and arithmetic; op 3: FP64).  b, x: device arrays laid
 * out as in krylov_solve_batched. */
int hec_batch_apply(hec_batch_t B, int32_t op, const double *b, double *x, int32_t nrhs,
                    void *stream);
void hec_batch_destroy(hec_batch_t B);

/* ---------------------------------------------------------------- serving */
/* A solve server: requests (a matrix, a right-hand side, the ILU level) are
 * queued, admitted in arrival order when their device memory fits the
 * budget, set up (HEC layout, ILU(k), level schedule) and solved with
 * restarted GMRES(m) to tol -- the paper's per-system method -- by `lanes`
 * host threads, each with its own CUDA stream, so that the solves of
 * different requests overlap on the device and a lane takes the next request
 * as soon as its last one is done (continuous batching).  A request's matrix,
 * factors and Krylov basis stay resident on the device while it runs; with a
 * nonzero key they stay resident afterwards too (least recently used evicted
 * first when the budget needs room), and later requests with the same key
 * reuse them without setup (a key serves one request at a time: a request
 * whose key is in use waits, and later requests may start before it).
 * Systems of at most small_rows unknowns run on
 * the batched kernel as one-CTA launches, larger ones on the single-system
 * path with RAS blocks of about block_rows rows.  A request's result depends
 * only on the request: it is bit-identical alone and in any mix.  The paper
 * has no serving layer; this is the library's extension. */
typedef struct hec_server_s *hec_server_t;

typedef struct {
    int64_t device_budget;  /* bytes for resident requests; 0 = half the free memory */
    int32_t lanes;          /* concurrent solves; 0 = 8                                */
    int32_t restart;        /* GMRES(m), <= 31; 0 = 30                                 */
    int32_t maxit;          /* Arnoldi steps per solve; 0 = 20000                      */
    int32_t flags;          /* HEC_MIXED_FP32: FP32 inner cycles, FP64 refinement     */
    double tol;             /* relative residual; 0 = 1e-8                             */
    int32_t small_rows;     /* 0 = 32768                                               */
    int32_t block_rows;     /* 0 = 16384                                               */
    int32_t keep_solutions; /* 1: keep x for hec_server_solution; 0: discard           */
    int32_t reserved;
} hec_server_opts_t;

typedef struct {
    hec_csr_t A;      /* host arrays, copied at submit; with a key, A.row_ptr may
                         be NULL (A.n still set): solve with the system resident
                         under that key (HEC_ERR_INVALID in the result if none)     */
    const double *b;  /* host, A.n values, copied                                   */
    int32_t ilu_k;    /* >= 0                                                       */
    int32_t reserved;
    uint64_t key;     /* 0: nothing kept; else requests with equal keys reuse the
                         resident set-up form: without a matrix as it is; with a
                         matrix of the same sparsity pattern (row_ptr and col,
                         compared by entry count and a 64-bit FNV-1a hash) and
                         level, refactored
                         on the GPU with the new values (hec_refactor); with
                         another pattern (or for a one-CTA batched system), set
                         up again.  If that refactor or new set-up fails, the
                         key's resident system is dropped (the error is the
                         request's status): the next request with the key
                         must carry a matrix                                       */
    uint64_t tag;     /* returned with the result                                   */
} hec_request_t;

typedef struct {
    uint64_t ticket, tag;
    int32_t status;     /* HEC_OK, HEC_MAXIT, HEC_BREAKDOWN or an error code           */
    int32_t iters;      /* Arnoldi steps                                               */
    double rel_resid;   /* true FP64 ||b - A x|| / ||b||                               */
    double t_submit;    /* seconds on the server clock (hec_server_clock)              */
    double t_start;     /* admitted to a lane                                          */
    double t_setup;     /* set-up done (= t_start when reused)                         */
    double t_done;
    int32_t lane;
    int32_t reused;     /* 1: the matrix and factors were resident already             */
    int32_t fp64_finish;/* 1: the mixed-precision solve was finished in FP64           */
    int32_t refactored; /* 1: a resident system took new values by hec_refactor         */
    int64_t device_bytes;
} hec_result_t;

int hec_server_create(const hec_server_opts_t *opts, hec_server_t *out);
/* Queues a request; *ticket identifies it.  Never blocks on the device. */
int hec_server_submit(hec_server_t S, const hec_request_t *req, uint64_t *ticket);
/* Moves up to max finished results into out (completion order), waiting up
 * to wait_ms for the first; *count = number returned. */
int hec_server_poll(hec_server_t S, hec_result_t *out, int32_t max, int32_t *count,
                    int32_t wait_ms);
/* Copies the solution of a finished request (keep_solutions = 1) and drops it. */
int hec_server_solution(hec_server_t S, uint64_t ticket, double *x, int32_t n);
/* Seconds since the server started (the clock of hec_result_t). */
double hec_server_clock(hec_server_t S);
/* Requests queued, running, finished-but-not-polled; bytes reserved. */
int hec_server_stats(hec_server_t S, int32_t *queued, int32_t *running, int32_t *finished,
                     int64_t *reserved_bytes);
/* Waits for every submitted request to finish, then frees everything. */
void hec_server_destroy(hec_server_t S);

#ifdef __cplusplus
}
#endif
#endif
