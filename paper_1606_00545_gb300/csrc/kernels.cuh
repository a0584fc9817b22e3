// kernels.cuh -- device-side data structures and launch wrappers shared by the
// CUDA translation units of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hec {

constexpr int kThreads = 256;         // threads per CTA of the streaming kernels
constexpr int kSpmvTile = 2 * kThreads; // rows per SpMV tile: 2 adjacent rows per thread
constexpr int kSpmvLongRow = 256;       // tail rows longer than this take a whole CTA
constexpr int kMaxRestart = 128;      // largest GMRES(m) supported
constexpr int kMaxDots = 2;           // fused reductions per launch

// Reduction finalisers: what the last CTA of a reducing launch does with the
// summed values (all of them run on one thread, after a fixed-order sum).
enum FinOp : int {
    FIN_STORE = 0,        // result[d] = sum_d
    FIN_STORE_SQRT,       // result[0] = sqrt(sum_0)
    FIN_NRM_B,            // ||b||: bnorm, b == 0 -> done + zero_x
    FIN_BICG_INIT,        // r = b - A x0: rho = (r, r); converged test
    FIN_BICG_ALPHA,       // v = A p*: alpha = rho / (r0, v)
    FIN_BICG_S,           // s = r - alpha v: ||s|| test
    FIN_BICG_OMEGA,       // t = A s*: omega = (t, s) / (t, t)
    FIN_BICG_XR,          // x, r update: ||r||, rho_new, end-of-pass tests
    FIN_TRUE_RESID,       // r = b - A x at exit: rel_resid
    FIN_GMRES_CYCLE,      // r = b - A x at cycle start: beta, tests
    FIN_GMRES_W0,         // w = A z: ||w|| before orthogonalisation
    FIN_GMRES_H1,         // first projection h1 (k values)
    FIN_GMRES_H2,         // second projection h2 (k values)
    FIN_GMRES_STEP,       // ||w''||: Hessenberg column, Givens, cycle tests
    FIN_CG_INIT,          // r = b - A x0: ||r|| test
    FIN_CG_RHO,           // (r, z): rho, beta = rho_new / rho; loop condition
    FIN_CG_ALPHA,         // q = A p: alpha = rho / (p, q)
    FIN_CG_R,             // x, r update: ||r|| test, iteration count
};

// Device-resident solver state: scalars of Algorithm 4 / GMRES, loop flags,
// and the conditional-node handles of the solve graph.
struct __align__(16) SolverState {
    // per-call inputs
    double tol;
    int maxit, restart, method, flags;
    // scalars
    double bnorm, rho, rho_prev, alpha, omega, scale, w0norm, est, rel_resid;
    double inner_rtol, beta_cycle; // mixed precision: inner cycle tolerance, cycle start ||r||
    double cg_beta;                // CG: (r_{j+1}, z_{j+1}) / (r_j, z_j)
    int stag_run, stagnated;       // mixed precision: cycles in a row whose true FP64
                                   // residual exceeded 10x the FP32 cycle's estimate
    int slow_run, slow_pad;        // mixed precision: cycles in a row that reduced the
                                   // true FP64 residual by less than 10%
    double dots[kMaxDots];
    int iters, restarts, status, done;
    int skip, s_conv, zero_x, j;
    int jend, cycle_end, err, graph_mode; // graph_mode: kernels run inside the solve graph
    unsigned long long launches;
    cudaGraphConditionalHandle h_while, h_if;
    // GMRES small dense part
    double H[(kMaxRestart + 1) * kMaxRestart]; // H[i * kMaxRestart + j]
    double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
    double h1[kMaxRestart + 1], h2[kMaxRestart + 1];
};

// Reduction scratch of one launch stream: per-CTA partials and a ticket.
struct RedScratch {
    double *partials;   // >= grid * width doubles
    unsigned *ticket;   // zero between launches
    int capacity;       // doubles available in partials
};

// ------------------------------------------------------------------ SpMV
// Values and vectors are FP64, or FP32 when launched with fp32 = true (the
// inner solves of the mixed-precision mode); indices are always int32.
struct SpmvArgs {
    int n, ld, K, ntiles;
    const int *ell_col;
    const void *ell_val;
    const int *tail_rows, *tail_ptr, *tail_col, *tile_tail;
    const int *tile_group, *tile_long, *tail_long; // tail schedule (see build_hec)
    const void *tail_val;
    const void *x;
    const void *y_in;
    void *y_out;
    const void *w0, *w1;   // dot partners; nullptr = y_out itself
    double alpha, beta;
    RedScratch red;
    double *result;        // FIN_STORE destination (device)
    int op;
    SolverState *st;       // nullable
};
// mode: 0 y = s, 1 y = alpha s, 2 y = alpha s + beta y_in
int launch_spmv(const SpmvArgs &a, int mode, int ndot, bool has_tail, int grid,
                cudaStream_t s, bool fp32 = false);

// ------------------------------------------------------------------ vector kernels
enum VecOp : int {
    V_AXPBY = 0,   // y = a x + b y
    V_WAXPBY,      // z = a x + b y
    V_DOT,         // (x, y)
    V_NRM2SQ,      // (x, x)
    V_COPY,        // z = x
    V_SCALE_ST,    // z = st->scale * x           (GMRES basis normalisation)
    V_BICG_P,      // p = r + beta (p - omega v)  (Algorithm 4)
    V_BICG_S,      // s = r - alpha v, (s, s)
    V_BICG_XR,     // x += alpha p* + omega s*, r = s - omega t, (r, r), (r0, r)
    V_AXPY_ST1,    // y += x                       (GMRES x update)
    V_ZERO_IF_ST,  // z = 0 if st->zero_x
    V_CG_XR,       // x += alpha p, r -= alpha q, (r, r)          (CG)
    V_CG_P,        // p = z + beta p (first pass: p = z)           (CG)
    V_JACOBI,      // z = d .* x (typed: damped Jacobi, d = omega / a_ii)
};
struct VecArgs {
    int n;
    double a, b;
    const double *x, *y;
    double *z, *w;           // outputs (meaning per op)
    const double *u, *v, *q; // extra inputs (meaning per op)
    RedScratch red;
    double *result;
    int op;                  // FinOp
    SolverState *st;
    int x_from_j;            // x = x + st->j * ldv (GMRES basis column)
    int z_from_j;
    int64_t ldv;
    int guard;               // 1: no-op if st->cycle_end, 2: no-op if st->done
    const void *xv;          // typed operands of launch_vec_typed
    void *zv;
    const void *dv;          // V_JACOBI: the scaled inverse diagonal (z's type)
};
int launch_vec(VecOp vop, const VecArgs &a, int grid, cudaStream_t s);
// V_COPY, V_SCALE_ST, V_AXPY_ST1 and V_JACOBI on a.xv / a.zv with element types chosen
// by x32 / z32 (FP32 if set, else FP64): the FP32 basis of the mixed-precision
// mode, the FP64 -> FP32 start vector and the FP32 -> FP64 correction.
int launch_vec_typed(VecOp vop, const VecArgs &a, bool x32, bool z32, int grid, cudaStream_t s);

// GMRES Arnoldi: projections and basis combinations (column-major basis V,
// leading dimension ldv; k vectors = st->j + 1 when k_from_st).
// V, w, wout: FP64, or FP32 when launched with fp32 = true (coefficients and
// reduced values stay FP64).
struct BasisArgs {
    int n;
    int k;                 // number of basis vectors (if !k_from_st)
    int k_from_st;         // 1: k = st->j + 1; 2: k = st->jend
    const void *V;
    int64_t ldv;
    const void *w;         // vector projected / updated
    void *wout;            // updated vector
    const double *coef;    // coefficients (device), e.g. st->h1
    RedScratch red;
    double *result;
    int op;
    SolverState *st;
};
int launch_multidot(const BasisArgs &a, int grid, cudaStream_t s, bool fp32 = false);
// wout = w - sum_i coef[i] V_i  (with_norm: + fused (wout, wout) -> op)
int launch_basis_update(const BasisArgs &a, bool with_norm, int grid, cudaStream_t s,
                        bool fp32 = false);
// wout = sum_i coef[i] V_i
int launch_basis_combine(const BasisArgs &a, int grid, cudaStream_t s, bool fp32 = false);

// ------------------------------------------------------------------ TRSV (RAS)
struct TrsvBlock {
    int chunk_begin, chunk_end; // chunk ids of this program (L chunks then U chunks)
    int chunk_mid;              // first U chunk
    int links;                  // bit 0: part p - 1 of the same RAS block exists, bit 1: part p + 1
    int ring_L, ring_U;         // 1: dependencies read from the shared-memory ring
    int64_t yoff, zoff;         // offsets of this program in the y / z scratch (resident
                                // kernel: yoff = offset of the block's V_b in vrows, zoff =
                                // its first chunk group)
    int nv;                     // resident kernel: the block's local rows
    int own0, own1;             // resident kernel: its owned local rows [own0, own1)
    int ngroups;                // resident kernel: its chunk groups
};
struct TrsvArgs {
    int nblocks;                // programs: RAS blocks x parts
    int parts;                  // CTAs per RAS block = cluster size (1: no cluster)
    const TrsvBlock *blocks;
    const uint2 *chunks;        // {offset in 16-byte units, bytes}
    const unsigned char *pack;  // packed chunk data
    const void *r;              // FP64, or FP32 for the FP32 layout
    void *z;
    void *ysc, *zsc;            // scratch: y by L position, z by U position
    int ring_mask;              // own ring slots R - 1 (power of two)
    int import_slots;           // import ring slots RI (0 without split blocks)
    int stage_bytes, nstages;
    int fixed_width;            // > 0: fixed-slot layout of this uniform row width (4, 6 or 8)
    int exp_arrays;             // fixed-slot chunks carry export slots
    long long spin_limit;
    int *err;                   // device error word
    SolverState *st;            // nullable: skip / basis column / launch count
    int n;                      // rows of z (bounds checks of the debug build)
    int r_from_j;
    int64_t ldv;
    int resident;               // 1: the resident-vector kernel (fixed_width: its row width)
    int res_slots;              // resident kernel: shared-memory vector slots (largest nv + 1)
    const int *vrows;           // resident kernel: V_b of every block, concatenated
    const uint2 *groups;        // resident kernel: chunk groups {offset / 16, bytes}
    int res_warps;              // resident kernel: solving warps (2, 4 or 8)
    int res_group;              // resident kernel: chunks per group of one bulk copy
};
// Shared memory of one CTA: stages, right-hand-side slots, own and import
// ring, barriers and the two progress counters (vbytes: 8 for FP64, 4 for FP32).
size_t trsv_smem_bytes(int stage_bytes, int nstages, int ring_slots, int vbytes);
// Largest stage count (3..8) that fits the device's shared memory per CTA
// (ring_slots: own + import slots).
int trsv_stages_for(int stage_bytes, int ring_slots, int vbytes);
// The same for the resident-vector kernel: stages and a vector of res_slots values.
size_t trsv_res_smem_bytes(int stage_bytes, int nstages, int res_slots, int vbytes);
// Largest stage count (3..8) that fits, 0 if even 3 stages do not.
int trsv_res_stages_for(int stage_bytes, int res_slots, int vbytes);
int launch_trsv(const TrsvArgs &a, cudaStream_t s, bool fp32 = false);
// The first violation a debug build (HEC_DEBUG) recorded: code, program,
// chunk, thread, value, bound, 0, 0 (all 0: none); clear resets it.
int trsv_debug_read(int *out, bool clear);
bool trsv_debug_build();
// The uniform width (4, 6 or 8) the FP32 layout is padded to for rows of at
// most longest_row entries; 0: longer rows, generic layout.
int trsv_uniform_width(int longest_row);

// ------------------------------------------------------------------ numeric refactorisation
// Factors of all RAS blocks, concatenated: rows by block (row0 of block b at
// blk_row0[b]), entries by row (rp: global entry offsets, ci: block-local
// columns, dg: global entry index of each row's diagonal).
struct RefactorArgs {
    int64_t nent;            // factor entries over all blocks
    const double *val;       // the new CSR values of A
    const int *src;          // per factor entry: its CSR index in A, -1 for fill
    double *f;               // factor values (out)
    const int *rp, *ci, *dg;
    const int *blk_row0;     // nblocks + 1
    const int *blk_lev0;     // nblocks + 1: offsets into lptr (each block: nlev + 1 entries)
    const int *lptr, *lrows; // L level sets per block (local rows, by block row offset)
    int *err;                // device error word (HEC_ERR_ZERO_PIVOT)
};
// Per row of every chunk of a triangular-solve layout: where its values come from.
struct FillArgs {
    unsigned char *pack;
    const uint2 *chunks;     // {offset in 16-byte units, bytes}
    const int64_t *chunk_row0;
    const int *rm_start, *rm_len, *rm_diag; // factor entry of the pass's first value, count, diagonal
    const double *f;
};
int launch_scatter_hec(int64_t nnz, const double *val, const int64_t *slot, double *ell,
                       double *tail, cudaStream_t s);
int launch_cast_f32(int64_t n, const double *x, float *y, cudaStream_t s);
int launch_refactor(const RefactorArgs &a, int nblocks, cudaStream_t s);
int launch_fill_pack(const FillArgs &a, int nchunks, bool fp32, cudaStream_t s);
int launch_jacobi_dinv(int n, const double *val, const int64_t *diag, double omega, double *dinv,
                       float *dinv32, int *err, cudaStream_t s);

// ------------------------------------------------------------------ small solver kernels
int launch_gmres_lsq(SolverState *st, cudaStream_t s);
int launch_loopcond(SolverState *st, cudaStream_t s);

} // namespace hec
