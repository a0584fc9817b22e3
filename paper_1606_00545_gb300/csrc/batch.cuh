// batch.cuh -- device layout and kernel interface of the batched solver: many
// independent systems A_s x_s = b_s, each solved start to finish by one CTA of
// a persistent kernel (restarted GMRES(m), Section 2.7, right-preconditioned
// by ILU(k) of A_s, Sections 2.5-2.6, with FP64 iterative refinement around
// FP32 inner cycles).  Shared by the kernel (k_batch.cu) and the host setup
// (hec_batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hec {

// Rows per triangular-solve chunk: a chunk is consecutive rows of one level.
constexpr int kBatchChunkRows = 128;
// Longest GMRES cycle the batched kernel accepts: the basis passes keep one
// partial dot product per basis vector in registers (31 vectors + ||w||^2).
constexpr int kBatchMaxRestart = 31;
// Largest CTA the batched kernel is compiled for.
constexpr int kBatchMaxThreads = 512;

// One chunk of a triangular pass, as the issuing thread reads it.
struct BChunk {
    int off16;  // byte offset of the chunk's block in the factor arena / 16
    int bytes;  // block bytes (multiple of 16)
    int first;  // position (in the pass's order) of the chunk's first row
    int nrows;
};

// A chunk block in the factor arena (value type T; stride = nrows rounded up
// to 4):
//   int4 header {nrows, width, first, flags (bit 0: U pass)}
//   dst[stride]          int32: L pass -- U-order position of the row (where
//                        y goes); U pass -- vector position (where z goes)
//   dep[width][stride]   int32: ring slot of each dependency (padding: the
//                        zero slot, ring_mask + 1)
//   val[width][stride]   T: L multipliers / U off-diagonal entries
//   dinv[stride]         T: U pass only, 1 / u_ii
// Column k of row i sits at [k * stride + i], so a warp's loads are
// consecutive.

// One system, as every thread of its CTA reads it.  Positions: the system's
// unknowns renumbered in the level order of L (Eq. 11), so that the rows of a
// level are consecutive in every vector.
struct BatchSys {
    int n;           // unknowns
    int K, ld;       // ELL width and leading dimension of the slab
    int ntail;       // rows stored whole in the CSR tail
    int chL, nchL;   // chunks of the L pass
    int chU, nchU;   // chunks of the U pass
    long long row0;  // first row of the system in the caller's vectors
    long long ell;   // offset of the slab (elements) in the ELL arrays
    long long tail;  // offset in tail_rows
    long long tptr;  // offset in tail_ptr (ntail + 1 entries)
    long long perm;  // offset in row_of_pos (n entries)
};

// Per-system outcome, the layout of hec_batch_sys_info_t.
struct BatchResult {
    int iters, cycles, status;
    int reorth; // Arnoldi steps that took the third (re-orthogonalising) pass
    double rel_resid;
};

enum BatchOp : int {
    BOP_SOLVE = 0,
    BOP_SPMV64 = 1,    // x = A b, FP64 values
    BOP_SPMV_IN = 2,   // x = A b in the inner type
    BOP_PRECOND = 3,   // x = M^{-1} b in the inner type
};

struct BatchArgs {
    int nsys, nrhs, m, maxit;
    double tol, inner_rtol;
    int x0_zero, op;
    const BatchSys *sys;
    const int *order;  // queue position -> system index (costliest first)
    const BChunk *chunks;
    const unsigned char *fac;
    const int *ell_col;
    const double *ell_val64;
    const void *ell_val;  // inner type
    const int *tail_rows;
    const long long *tail_ptr;
    const int *tail_col;
    const double *tail_val64;
    const void *tail_val;
    const int *row_of_pos;
    const double *b;
    double *x;
    unsigned char *ws;     // per-CTA workspace, ws_stride bytes each
    long long ws_stride;
    long long E;           // elements of one vector (positions x NR, rounded to the CTA size)
    long long offZ, offY, offX, offB, offR;  // byte offsets in a CTA's workspace
    int ring_mask, nstages, stage_bytes, ent_bytes;
    int sstages, sbytes;   // basis-tile stages: count and bytes (m + 1 slots of a tile)
    long long spin_limit;
    int *queue;
    int *err;
    BatchResult *res;
    const unsigned char *only;  // nullable: solve only the systems marked 1
};

// Dynamic shared memory of one CTA.  The triangular-solve stages and the
// basis-tile stages are used at different times and share one region.
struct BatchSmem {
    int stage, ring, bar, bar2, red, out, coef, dbl, misc, total;
};

// Doubles of per-right-hand-side state: h, h2, cs, sn, g, y, sig, scalars.
__host__ __device__ inline int batch_rhs_doubles(int m) { return 7 * m + 24; }

// Per-system status of a mixed-precision solve whose FP32 cycles stopped
// reducing the FP64 residual; the host finishes such systems in FP64.
constexpr int kBatchStagnated = 100;

__host__ __device__ inline BatchSmem batch_smem(int nstages, int stage_bytes, int sstages,
                                                int sbytes, int ring_slots, int NR, int tsz, int m,
                                                int threads)
{
    auto al = [](int p, int a) { return (p + a - 1) / a * a; };
    BatchSmem o;
    o.stage = 0;
    int p = nstages * stage_bytes > sstages * sbytes ? nstages * stage_bytes : sstages * sbytes;
    o.ring = al(p, 16);
    p = o.ring + (ring_slots + 1) * NR * tsz;
    o.bar = al(p, 16);
    p = o.bar + nstages * 8;
    o.bar2 = al(p, 16);
    p = o.bar2 + sstages * 8;
    o.red = al(p, 16);
    p = o.red + (threads / 32) * 32 * 4 * 8;
    o.out = al(p, 16);
    p = o.out + 32 * 4 * 8;
    o.coef = al(p, 16);
    p = o.coef + (m + 1) * 4 * tsz;
    o.dbl = al(p, 16);
    p = o.dbl + NR * batch_rhs_doubles(m) * 8;
    o.misc = al(p, 16);
    p = o.misc + 64;
    o.total = al(p, 128);
    return o;
}

// Bytes of a stage's right-hand-side area: a chunk's rows plus 16-byte
// alignment slack on both ends.
__host__ __device__ inline int batch_rhs_area(int NR, int tsz)
{
    return kBatchChunkRows * NR * tsz + 32;
}

// Launch of the batched kernel for inner type float (fp32) or double and
// NR right-hand sides per CTA pass (1, 2 or 4).  Returns a cudaError_t.
int launch_batch(const BatchArgs &a, bool fp32, int NR, int threads, int grid, int smem,
                 cudaStream_t s);
// Resident CTAs per SM for this configuration (0: does not fit).
int batch_occupancy(bool fp32, int NR, int threads, int smem);

} // namespace hec
