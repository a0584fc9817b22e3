// hec_setup.h -- host-side setup of the library: HEC conversion, RAS
// partition, ILU(k) factorisation, level schedule, and the level-major chunk
// layout that the triangular-solve kernel streams.  Host C++ only.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace hec {

struct HostCSR {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> va;
};

// Returns HEC_OK, HEC_ERR_INVALID or HEC_ERR_UNSORTED_CSR (msg filled).
int check_csr(int n, const int *rp, const int *ci, int nnz, bool need_diag, std::string &msg);

// --------------------------------------------------------------- HEC (Section 2.1)
struct HecHost {
    int n = 0, K = 0, ld = 0;
    std::vector<int> ell_col;      // K * ld, column-major
    std::vector<double> ell_val;   // K * ld
    std::vector<int> tail_rows;    // rows with more than K entries, ascending
    std::vector<int> tail_ptr;     // tail_rows.size() + 1
    std::vector<int> tail_col;
    std::vector<double> tail_val;
    std::vector<int> tile_tail;    // per SpMV tile: first tail row index (ntiles + 1)
    std::vector<int> tile_group;   // per tile: lanes per short tail row (4, 8, 16 or 32)
    std::vector<int> tile_long;    // per tile: first index into tail_long (ntiles + 1)
    std::vector<int> tail_long;    // tail rows longer than kSpmvLongRow, by tile
};
int ell_width_auto(const HostCSR &A);
void build_hec(const HostCSR &A, int K, int align, HecHost &H);

// --------------------------------------------------------------- RAS + ILU(k)
struct BlockFactor {
    int own_lo = 0, own_hi = 0;  // owned global rows [own_lo, own_hi)
    std::vector<int> rows;       // V_b, ascending global ids
    HostCSR F;                   // A_b, then its ILU(k) factor (local indices)
    std::vector<int> lev;        // fill level of every factor entry
    std::vector<int> diag;       // position of the diagonal of every row in F
    // Eq. 11 on the full factor
    int nlevL = 0, nlevU = 0;
    std::vector<int> levL, levU;            // level of each local row (1-based)
    std::vector<int> lptrL, lrowsL, lptrU, lrowsU;
};

// Sequence partition + overlap growth + extraction of A[V_b, V_b].
void ras_blocks(const HostCSR &A, int nblocks, int overlap, std::vector<BlockFactor> &out);
// In place: B.F becomes the ILU(k) factor.  HEC_OK / HEC_ERR_ZERO_PIVOT / HEC_ERR_INVALID.
int iluk_block(BlockFactor &B, int k, std::string &msg);
// Level sets of L_b and U_b (Eq. 11).
void levels_block(BlockFactor &B);

// --------------------------------------------------------------- device layout
// (trsv_layout.cpp)
struct TrsvPack {
    std::vector<unsigned char> pack;
    std::vector<uint2> chunks;
    std::vector<TrsvBlock> blocks; // one program per (RAS block, part): block b, part p at b * parts + p
    int parts = 1;              // CTAs per RAS block (the cluster size of the launch)
    int stage_bytes = 0;        // shared-memory stage the kernel streams chunks into
    int exp_arrays = 0;         // fixed-slot chunks carry export slots
    int64_t ysz = 0, zsz = 0;   // scratch lengths (values)
    int ring_slots = 0;         // own ring R: power of two (>= 32)
    int import_slots = 0;       // import ring RI: power of two, 0 when no block is split
    int64_t alg_bytes = 0;      // algorithmic bytes of one apply
    int64_t rows_L = 0, rows_U = 0;
    // where every chunk row's values come from, for refilling them from new
    // factor values on the device: factor entries are numbered over all
    // blocks in order (block b's entries start after those of blocks < b)
    std::vector<int64_t> chunk_row0; // per chunk: first index into the row maps
    std::vector<int> rm_start, rm_len, rm_diag; // first value's entry, count, diagonal (U; -1 for L)
    // resident-vector layout (pack_trsv_resident): one CTA per block, the
    // block's vector in shared memory
    int resident = 0;
    int res_slots = 0;          // largest block's rows + 1
    int res_warps = 0;          // solving warps of the kernel (2, 4 or 8): chunks of 32 x that rows
    int res_group = 1;          // chunks per group (one bulk copy; every chunk the same size)
    std::vector<int> vrows;     // V_b of every block, concatenated (TrsvBlock::yoff)
    std::vector<uint2> groups;  // bulk copies of consecutive chunks (TrsvBlock::zoff, ::pad)
};
// vb: bytes per stored value, 8 (FP64 layout) or 4 (FP32 layout).
// uniform_width > 0 (at most 8): every row is padded to this width (value 0)
// and chunks use the fixed-slot format, so the kernel addresses every row's
// data at compile-time offsets; it must be >= the longest row.  stage_bytes
// is raised, if needed, to hold the largest fixed-slot chunk (out.stage_bytes).
// parts (1, 2, 4 or 8): CTAs per RAS block; a block whose dependencies do
// not allow that split gets fewer (its remaining programs are empty).
int pack_trsv(const std::vector<BlockFactor> &B, int n, int stage_bytes, int max_ring, int vb,
              TrsvPack &out, std::string &msg, int uniform_width = 0, int parts = 1);
// The resident-vector layout of k_trsv_res: every block one program, its rows
// padded to `width` (2, 3, 4, 6 or 8: trsv_resident_width of the longest
// row), dependencies as local row slots, every block below 65535 rows.
int pack_trsv_resident(const std::vector<BlockFactor> &B, int width, int vb, TrsvPack &out,
                       std::string &msg);
// The resident width for rows of at most longest_row entries, 0 if none.
int trsv_resident_width(int longest_row);
// The parts per block worth launching: split while the widest block's levels
// hold more than rows_per_part rows per part and the CTAs fit on sm_count SMs.
int trsv_auto_parts(const std::vector<BlockFactor> &B, int sm_count, int rows_per_part);
// The longest off-diagonal row of any L_b (upass false) or U_b.
int max_factor_width(const std::vector<BlockFactor> &B, bool upass);

// Run f(i) for i in [0, count) on the host's cores.
void parallel_for(int count, const std::function<void(int)> &f);

} // namespace hec
