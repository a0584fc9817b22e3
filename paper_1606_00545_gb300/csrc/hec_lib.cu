// hec_lib.cu -- the C ABI declared in include/hecgpu.h: handles, device memory,
// launches, and the CUDA-graph drivers of BiCGSTAB (Algorithm 4) and
// restarted GMRES(m) (Section 2.7).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hecgpu.h"
#include "hec_setup.h"
#include "kernels.cuh"
#include "runtime.h"

using namespace hec;

// ====================================================================== runtime
namespace hec {

namespace {
thread_local std::string g_last_error;
std::mutex g_alloc_mu;
AllocFns g_alloc;
} // namespace

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(HEC_ERR_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return HEC_OK;
}

AllocFns current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

void set_allocator(const AllocFns &f)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = f;
}

int device_sms()
{
    static int sms = -1;
    if (sms < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    return sms;
}

int device_smem_optin()
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        optin = 227 * 1024;
    return optin;
}

void keep_pool_memory()
{
    static std::once_flag once;
    std::call_once(once, []() {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const char *last_error_text() { return g_last_error.c_str(); }

} // namespace hec

namespace {

// Reduction scratch: partials sized for every reducing launch of the library.
struct Reducer {
    DevBuf partials, ticket;
    RedScratch r{};
    static int capacity()
    {
        return std::max(device_sms() * 8 * kMaxDots, device_sms() * 4 * (kMaxRestart + 1));
    }
    int init(cudaStream_t s)
    {
        const int cap = capacity();
        HEC_TRY(partials.alloc((size_t)cap * sizeof(double), s));
        HEC_TRY(ticket.alloc(sizeof(unsigned), s));
        HEC_CK(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s));
        r.partials = partials.as<double>();
        r.ticket = ticket.as<unsigned>();
        r.capacity = cap;
        return HEC_OK;
    }
};

std::atomic<uint64_t> g_next_id(1);

} // namespace

// ====================================================================== handles
struct Solver;

struct hec_matrix_s {
    uint64_t id = 0;
    bool host_only = false;
    HostCSR csr;
    HecHost hec;
    DevBuf ell_col, ell_val, tail_rows, tail_ptr, tail_col, tail_val, tile_tail;
    DevBuf tile_group, tile_long, tail_long;
    DevBuf ell_val32, tail_val32; // FP32 copies of the values, made on first FP32 use
    bool f32_ready = false;
    // hec_refactor: CSR entry -> slab / tail slot, CSR index of each diagonal,
    // staging for host values; the host HEC copy is refreshed on demand
    DevBuf d_slot, d_diagidx, d_newval;
    const double *d_newval_view = nullptr; // the new values of the refactor in progress
    bool hec_host_stale = false;
    Reducer red;
    std::vector<std::unique_ptr<Solver>> solvers; // solves without a preconditioner
    int64_t device_bytes() const
    {
        return (int64_t)(d_slot.bytes + d_diagidx.bytes + d_newval.bytes +
                         ell_col.bytes + ell_val.bytes + tail_rows.bytes + tail_ptr.bytes +
                         tail_col.bytes + tail_val.bytes + tile_tail.bytes + tile_group.bytes +
                         tile_long.bytes + tail_long.bytes + red.partials.bytes +
                         ell_val32.bytes + tail_val32.bytes);
    }
    ~hec_matrix_s();
};

// The device layout of the factors for one value type: the chunk stream the
// triangular-solve kernel reads, and its scratch.
struct TrsvLayout {
    TrsvPack pack;
    DevBuf d_pack, d_chunks, d_blocks, d_ysc, d_zsc, d_vrows, d_groups;
    DevBuf d_row0, d_rms, d_rml, d_rmd; // value maps of hec_refactor (uploaded on first use)
    int nstages = 8;
    int vbytes = 8;
    int fixed_width = 0; // uniform row width of the fixed-slot format (0: per-warp widths)
    bool built = false;
    int64_t device_bytes() const
    {
        return (int64_t)(d_pack.bytes + d_chunks.bytes + d_blocks.bytes + d_ysc.bytes +
                         d_zsc.bytes + d_vrows.bytes + d_groups.bytes + d_row0.bytes +
                         d_rms.bytes + d_rml.bytes + d_rmd.bytes);
    }
};

struct hec_precond_s {
    uint64_t matrix_id = 0;
    int kind = 0; // 0: RAS with ILU(k) blocks, 1: damped Jacobi
    double omega = 1.0;
    DevBuf dinv, dinv32; // damped Jacobi: omega / a_ii (FP64; FP32 copy on first mixed use)
    int n = 0, k = 0, nblocks = 0, overlap = 0;
    bool host_only = false, scheduled = false;
    std::vector<BlockFactor> blocks;
    TrsvLayout lay[2]; // [0] FP64 values (level_schedule), [1] FP32 (built on first use)
    DevBuf d_err;
    int stage_bytes = 24576;
    int trsv_parts = 0; // CTAs per RAS block of the triangular solve (0: automatic)
    int trsv_kernel = HEC_TRSV_AUTO; // triangular-solve kernel (hec_precond_set_trsv_kernel)
    std::vector<std::unique_ptr<Solver>> solvers;
    // hec_refactor: every block's factor on the device (entries numbered over
    // all blocks), its source map into A and the L level sets; the host copy
    // of the factor values is refreshed on demand
    DevBuf rf_rp, rf_ci, rf_dg, rf_f, rf_src, rf_row0, rf_lev0, rf_lptr, rf_lrows;
    int64_t rf_nent = 0;
    bool rf_ready = false, factor_host_stale = false;
    int64_t device_bytes() const
    {
        return lay[0].device_bytes() + lay[1].device_bytes() + (int64_t)d_err.bytes +
               (int64_t)dinv.bytes + (int64_t)dinv32.bytes + (int64_t)rf_rp.bytes +
               (int64_t)rf_ci.bytes + (int64_t)rf_dg.bytes + (int64_t)rf_f.bytes +
               (int64_t)rf_src.bytes + (int64_t)rf_row0.bytes + (int64_t)rf_lev0.bytes +
               (int64_t)rf_lptr.bytes + (int64_t)rf_lrows.bytes;
    }
    ~hec_precond_s();
};

namespace {

constexpr long long kDefaultSpin = 1ll << 24;
constexpr int kJacobi = 1; // hec_precond_s::kind of a damped-Jacobi handle
constexpr int kMaxRing = 8192; // shared-memory ring slots (doubles)

// ---------------------------------------------------------------- launch helpers
SpmvArgs spmv_args(const hec_matrix_s *A)
{
    SpmvArgs a{};
    a.n = A->hec.n;
    a.ld = A->hec.ld;
    a.K = A->hec.K;
    a.ntiles = (A->hec.n + kSpmvTile - 1) / kSpmvTile;
    a.ell_col = A->ell_col.as<int>();
    a.ell_val = A->ell_val.as<double>();
    a.tail_rows = A->tail_rows.as<int>();
    a.tail_ptr = A->tail_ptr.as<int>();
    a.tail_col = A->tail_col.as<int>();
    a.tail_val = A->tail_val.as<double>();
    a.tile_tail = A->tile_tail.as<int>();
    a.tile_group = A->tile_group.as<int>();
    a.tile_long = A->tile_long.as<int>();
    a.tail_long = A->tail_long.as<int>();
    a.alpha = 1.0;
    a.beta = 0.0;
    a.op = FIN_STORE;
    return a;
}

// CTAs of an SpMV launch: one per row block (one 512-row tile in FP64, two
// in FP32, where a thread owns four rows), at most 8 per SM.
int spmv_grid(const hec_matrix_s *A, bool fp32)
{
    const int64_t tiles = (A->hec.n + kSpmvTile - 1) / kSpmvTile;
    return grid_for(fp32 ? (tiles + 1) / 2 : tiles, 1, 8);
}

int run_spmv(const hec_matrix_s *A, SpmvArgs a, int mode, int ndot, cudaStream_t s,
             bool fp32 = false)
{
    if (fp32) {
        a.ell_val = A->ell_val32.p;
        a.tail_val = A->tail_val32.p;
    }
    if (launch_spmv(a, mode, ndot, !A->hec.tail_rows.empty(), spmv_grid(A, fp32), s, fp32) != 0)
        return fail(HEC_ERR_INVALID, "no SpMV variant for mode %d ndot %d", mode, ndot);
    return check_launch("spmv");
}

// FP32 copies of the HEC values (slab and tail), for the FP32 inner solves.
int ensure_f32(hec_matrix_s *A, cudaStream_t s)
{
    if (A->f32_ready)
        return HEC_OK;
    // rounded on the device from the current FP64 values (hec_refactor may
    // have replaced them)
    const int64_t ne = (int64_t)A->hec.ell_val.size(), nt = (int64_t)A->hec.tail_val.size();
    HEC_TRY(A->ell_val32.alloc(ne * sizeof(float), s));
    HEC_TRY(A->tail_val32.alloc(nt * sizeof(float), s));
    launch_cast_f32(ne, A->ell_val.as<double>(), A->ell_val32.as<float>(), s);
    launch_cast_f32(nt, A->tail_val.as<double>(), A->tail_val32.as<float>(), s);
    HEC_TRY(check_launch("cast"));
    HEC_CK(cudaStreamSynchronize(s));
    A->f32_ready = true;
    return HEC_OK;
}

int vec_grid(int64_t n) { return grid_for(n, kThreads, 8); }

int run_vec(VecOp op, const VecArgs &a, cudaStream_t s)
{
    if (launch_vec(op, a, vec_grid(a.n), s) != 0)
        return fail(HEC_ERR_INVALID, "bad vector op");
    return check_launch("vector op");
}

// Arguments of the triangular-solve kernel over layout L of M (L = M->lay[0]
// for FP64 values, M->lay[1] for FP32).
TrsvArgs trsv_args(const hec_precond_s *M, const TrsvLayout &L, long long spin)
{
    TrsvArgs a{};
    a.nblocks = (int)L.pack.blocks.size();
    a.parts = L.pack.parts;
    a.import_slots = L.pack.import_slots;
    a.blocks = L.d_blocks.as<TrsvBlock>();
    a.chunks = L.d_chunks.as<uint2>();
    a.pack = L.d_pack.as<unsigned char>();
    a.ysc = L.d_ysc.p;
    a.zsc = L.pack.zsz ? L.d_zsc.p : nullptr;
    a.ring_mask = L.pack.ring_slots - 1;
    a.stage_bytes = L.pack.stage_bytes;
    a.nstages = L.nstages;
    a.fixed_width = L.fixed_width;
    a.exp_arrays = L.pack.exp_arrays;
    a.spin_limit = spin;
    a.err = M->d_err.as<int>();
    a.n = M->n;
    a.resident = L.pack.resident;
    a.res_slots = L.pack.res_slots;
    a.vrows = L.d_vrows.as<int>();
    a.groups = L.d_groups.as<uint2>();
    a.res_warps = L.pack.res_warps;
    a.res_group = L.pack.res_group;
    return a;
}

int run_trsv(const TrsvArgs &a, cudaStream_t s, bool fp32 = false)
{
    if (launch_trsv(a, s, fp32) != 0)
        return fail(HEC_ERR_CUDA, "cannot configure the triangular-solve kernel");
    return check_launch("trsv");
}

// The host copy of the factor values after hec_refactor replaced them on the
// device (factor queries and a layout packed later read it).
int refresh_host_factors(hec_precond_s *M, cudaStream_t s)
{
    if (!M->factor_host_stale)
        return HEC_OK;
    std::vector<double> f((size_t)M->rf_nent);
    HEC_CK(cudaMemcpyAsync(f.data(), M->rf_f.p, f.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           s));
    HEC_CK(cudaStreamSynchronize(s));
    size_t off = 0;
    for (BlockFactor &B : M->blocks) {
        std::memcpy(B.F.va.data(), f.data() + off, B.F.va.size() * sizeof(double));
        off += B.F.va.size();
    }
    M->factor_host_stale = false;
    return HEC_OK;
}

// CTAs per RAS block: the handle's choice, else split while levels are wide
// and the CTAs fit on the device's SMs (host-only handles: 152, GB300's count).
// FP64 (idx 0): split above 4 warps of rows per level and CTA -- each
// warp's FP64 multiply-add chain occupies its SM sub-partition's FP64 pipe, so
// fewer rows per SM shorten a level.  FP32 (idx 1): split only above one
// chunk (8 warps) per level: an FP32 level costs the same with fewer rows.
int layout_parts(const hec_precond_s *M, int idx)
{
    if (M->trsv_parts > 0)
        return M->trsv_parts;
    return trsv_auto_parts(M->blocks, M->host_only ? 152 : device_sms(), idx == 0 ? 128 : 256);
}

// The triangular-solve layout with (idx 0) FP64 or (idx 1) FP32 values: the
// resident-vector kernel's when asked for, or automatically when every
// block's vector fits in shared memory beside three stages, no level holds
// more than 128 rows and the streamed kernel would not split a block (on
// GB300 the resident kernel is 1.1-1.2x faster there -- 0.104 against 0.122
// ms on the 64 x 64 ILU(0) block -- and slower on wider levels); else the
// streamed kernel's.  Sets the row width of the
// fixed-slot formats (0: generic) and, for the resident layout, the stage
// count (the streamed kernel's is sized at upload).
int pack_layout(const hec_precond_s *M, int idx, TrsvPack &P, int &fixed_width, int &nstages,
                std::string &msg)
{
    const int vb = idx == 0 ? 8 : 4;
    const int longest =
        std::max(max_factor_width(M->blocks, false), max_factor_width(M->blocks, true));
    if (M->trsv_kernel != HEC_TRSV_STREAMED) {
        const int rw = trsv_resident_width(longest);
        int maxnv = 0, widest = 0;
        for (const BlockFactor &B : M->blocks) {
            maxnv = std::max(maxnv, B.F.n);
            for (size_t l = 0; l + 1 < B.lptrL.size(); ++l)
                widest = std::max(widest, B.lptrL[l + 1] - B.lptrL[l]);
            for (size_t l = 0; l + 1 < B.lptrU.size(); ++l)
                widest = std::max(widest, B.lptrU[l + 1] - B.lptrU[l]);
        }
        // automatic: levels of at most 128 rows (4 solving warps) on blocks
        // the streamed kernel would not split
        const bool want = M->trsv_kernel == HEC_TRSV_RESIDENT ||
                          (widest <= 128 && layout_parts(M, idx) == 1);
        if (rw > 0 && maxnv < 65535 && want) {
            const int rc = pack_trsv_resident(M->blocks, rw, vb, P, msg);
            if (rc != HEC_OK)
                return rc;
            // shared memory of the stage count (host-only handles: 3 stages
            // within GB300's 227 KB per block)
            nstages = M->host_only
                          ? (trsv_res_smem_bytes(P.stage_bytes, 3, P.res_slots, vb) <= 226 * 1024
                                 ? 3
                                 : 0)
                          : trsv_res_stages_for(P.stage_bytes, P.res_slots, vb);
            if (nstages > 0) {
                fixed_width = rw;
                return HEC_OK;
            }
        }
        if (M->trsv_kernel == HEC_TRSV_RESIDENT) {
            msg = "the resident triangular-solve kernel needs rows of at most 8 entries, blocks "
                  "below 65535 rows and a block vector that fits in shared memory";
            return HEC_ERR_INVALID;
        }
    }
    // pad every row to one short width when the factors allow it: the
    // fixed-slot chunks that the kernel streams from registers one chunk
    // ahead (the padding costs multiply-adds only where a warp's rows are
    // shorter than the width)
    fixed_width = trsv_uniform_width(longest);
    return pack_trsv(M->blocks, M->n, M->stage_bytes, kMaxRing, vb, P, msg, fixed_width,
                     layout_parts(M, idx));
}

// Pack, upload and size the scratch of the layout with vb-byte values.
int build_layout(hec_precond_s *M, int idx, cudaStream_t s)
{
    TrsvLayout &L = M->lay[idx];
    if (L.built)
        return HEC_OK;
    HEC_TRY(refresh_host_factors(M, s));
    L.vbytes = idx == 0 ? 8 : 4;
    std::string msg;
    const int rc = pack_layout(M, idx, L.pack, L.fixed_width, L.nstages, msg);
    if (rc != HEC_OK)
        return fail(rc, "%s", msg.c_str());
    const bool res = L.pack.resident != 0;
    if (!M->host_only) {
        if (!res)
            L.nstages = trsv_stages_for(L.pack.stage_bytes,
                                        L.pack.ring_slots + L.pack.import_slots, L.vbytes);
        HEC_TRY(upload(L.d_pack, L.pack.pack, s));
        if (res) {
            HEC_TRY(upload(L.d_vrows, L.pack.vrows, s));
            HEC_TRY(upload(L.d_groups, L.pack.groups, s));
        }
        HEC_TRY(upload(L.d_chunks, L.pack.chunks, s));
        HEC_TRY(upload(L.d_blocks, L.pack.blocks, s));
        HEC_TRY(L.d_ysc.alloc(std::max<int64_t>(L.pack.ysz, 1) * L.vbytes, s));
        HEC_TRY(L.d_zsc.alloc(std::max<int64_t>(L.pack.zsz, 1) * L.vbytes, s));
        HEC_CK(cudaStreamSynchronize(s));
        L.pack.pack.clear();
        L.pack.pack.shrink_to_fit();
    }
    L.built = true;
    return HEC_OK;
}

// The FP32 form of a preconditioner for the mixed-precision inner solves:
// the FP32 factor layout, or the FP32 copy of a Jacobi diagonal.
int ensure_precond_f32(hec_precond_s *M, cudaStream_t s)
{
    if (M->kind != kJacobi)
        return build_layout(M, 1, s);
    if (M->dinv32.p)
        return HEC_OK;
    std::vector<double> d(M->n);
    HEC_CK(cudaMemcpyAsync(d.data(), M->dinv.p, sizeof(double) * d.size(), cudaMemcpyDeviceToHost,
                           s));
    HEC_CK(cudaStreamSynchronize(s));
    std::vector<float> f(d.begin(), d.end());
    HEC_TRY(upload(M->dinv32, f, s));
    HEC_CK(cudaStreamSynchronize(s));
    return HEC_OK;
}

// z = omega D^{-1} r on the caller's stream (FP64 or FP32 operands).
int run_jacobi(const hec_precond_s *M, const void *r, void *z, bool fp32, cudaStream_t s)
{
    VecArgs va{};
    va.n = M->n;
    va.xv = r;
    va.zv = z;
    va.dv = fp32 ? M->dinv32.p : M->dinv.p;
    if (launch_vec_typed(V_JACOBI, va, fp32, fp32, vec_grid(M->n), s) != 0)
        return fail(HEC_ERR_INVALID, "bad typed vector op");
    return check_launch("jacobi");
}

// Global reducer for the stand-alone vector calls (one per process).
std::mutex g_red_mu;
std::unique_ptr<Reducer> g_red;
int global_reducer(cudaStream_t s, RedScratch &out)
{
    std::lock_guard<std::mutex> lk(g_red_mu);
    if (!g_red) {
        std::unique_ptr<Reducer> r(new Reducer());
        HEC_TRY(r->init(s));
        g_red = std::move(r);
    }
    out = g_red->r;
    return HEC_OK;
}

} // namespace

// ====================================================================== solver (graphs)
struct Solver {
    uint64_t matrix_id = 0;
    int method = 0, restart = 0;
    bool mixed = false; // GMRES with FP32 inner cycles and FP64 refinement
    int n = 0;
    int64_t ldv = 0;
    DevBuf ws, ws32, st_buf;
    Reducer red;
    SolverState *st = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *r0 = nullptr, *p = nullptr, *ps = nullptr;
    double *v = nullptr, *s = nullptr, *ss = nullptr, *t = nullptr;
    double *q = nullptr; // CG: A p
    // GMRES basis and step vectors: FP64, or FP32 when mixed
    void *V = nullptr, *z = nullptr, *w = nullptr, *u = nullptr, *zu = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle h_while = 0, h_if = 0;
    int64_t init_launches = 0;
    ~Solver()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (graph)
            cudaGraphDestroy(graph);
    }
};

hec_matrix_s::~hec_matrix_s() { solvers.clear(); }
hec_precond_s::~hec_precond_s() { solvers.clear(); }

namespace {

// Address of a member of the device-resident solver state.
template <class T>
T *dev_field(SolverState *st, size_t off)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(st) + off);
}

// Capture helper: begin capturing launches into `g` after `deps`.
int begin_capture(cudaStream_t cs, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps)
{
    HEC_CK(cudaStreamBeginCaptureToGraph(cs, g, deps, nullptr, ndeps,
                                         cudaStreamCaptureModeRelaxed));
    return HEC_OK;
}

// End the capture and return the node(s) the next node must follow.
int end_capture(cudaStream_t cs, std::vector<cudaGraphNode_t> &tail)
{
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    HEC_CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, nullptr, &nd));
    tail.assign(deps, deps + nd);
    cudaGraph_t g = nullptr;
    HEC_CK(cudaStreamEndCapture(cs, &g));
    return HEC_OK;
}

int add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps,
                    cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraphNode_t &node, cudaGraph_t &body)
{
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    HEC_CK(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                            &np));
    body = np.conditional.phGraph_out[0];
    return HEC_OK;
}

// --- launch sequences ----------------------------------------------------------
// The same sequences run inside the solve graph (captured once) or, for
// profilers that cannot see the kernels of a graph with conditional nodes,
// directly on a stream with one host check per iteration (HEC_SOLVE_EAGER).

// z = M^{-1} r inside a solve: FP64 layout, or the FP32 one for the inner
// solves of the mixed-precision mode (in, out are then FP32 vectors).
int seq_precond(const hec_precond_s *M, Solver &S, const void *in, void *out, int from_j,
                cudaStream_t cs)
{
    if (M->kind == kJacobi) {
        VecArgs va{};
        va.n = S.n;
        va.st = S.st;
        va.xv = in;
        va.x_from_j = from_j;
        va.ldv = S.ldv;
        va.zv = out;
        va.dv = S.mixed ? M->dinv32.p : M->dinv.p;
        if (launch_vec_typed(V_JACOBI, va, S.mixed, S.mixed, vec_grid(S.n), cs) != 0)
            return fail(HEC_ERR_INVALID, "bad typed vector op");
        return check_launch("jacobi");
    }
    TrsvArgs a = trsv_args(M, M->lay[S.mixed ? 1 : 0], kDefaultSpin);
    a.r = in;
    a.z = out;
    a.st = S.st;
    a.r_from_j = from_j;
    a.ldv = S.ldv;
    return run_trsv(a, cs, S.mixed);
}

int seq_norm_b(Solver &S, cudaStream_t cs)
{
    VecArgs va{};
    va.n = S.n;
    va.st = S.st;
    va.red = S.red.r;
    va.x = S.b;
    va.op = FIN_NRM_B;
    return run_vec(V_NRM2SQ, va, cs);
}

// BiCGSTAB start (Section 2.7): ||b||, the residual r0 = b - A x0 and
// rho_0 = (r0, r0); r0 is kept as the shadow residual.
int seq_bicg_init(hec_matrix_s *A, Solver &S, cudaStream_t cs)
{
    HEC_TRY(seq_norm_b(S, cs));
    SpmvArgs sa = spmv_args(A);
    sa.st = S.st;
    sa.red = S.red.r;
    sa.x = S.x;
    sa.alpha = -1.0;
    sa.beta = 1.0;
    sa.y_in = S.b;
    sa.y_out = S.r;
    sa.w0 = nullptr;
    sa.op = FIN_BICG_INIT;
    HEC_TRY(run_spmv(A, sa, 2, 1, cs));
    VecArgs cp{};
    cp.n = S.n;
    cp.st = S.st;
    cp.x = S.r;
    cp.z = S.r0;
    return run_vec(V_COPY, cp, cs);
}

// One BiCGSTAB iteration (Section 2.7): direction update, two preconditioner
// applies and SpMVs with the alpha and omega reductions fused into the SpMV
// epilogues, then the x and r updates with the convergence tests.
int seq_bicg_body(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    const int n = S.n;
    VecArgs pa{};
    pa.n = n;
    pa.st = S.st;
    pa.x = S.r;
    pa.y = S.v;
    pa.z = S.p;
    HEC_TRY(run_vec(V_BICG_P, pa, cs)); // p = r + beta (p - omega v)
    if (M)
        HEC_TRY(seq_precond(M, S, S.p, S.ps, 0, cs)); // M p* = p
    SpmvArgs v = spmv_args(A);
    v.st = S.st;
    v.red = S.red.r;
    v.x = M ? S.ps : S.p;
    v.y_out = S.v;
    v.w0 = S.r0;
    v.op = FIN_BICG_ALPHA;
    HEC_TRY(run_spmv(A, v, 0, 1, cs)); // v = A p*, (r0, v) -> alpha
    VecArgs sv{};
    sv.n = n;
    sv.st = S.st;
    sv.red = S.red.r;
    sv.x = S.r;
    sv.y = S.v;
    sv.z = S.s;
    sv.op = FIN_BICG_S;
    HEC_TRY(run_vec(V_BICG_S, sv, cs)); // s = r - alpha v, ||s||
    if (M)
        HEC_TRY(seq_precond(M, S, S.s, S.ss, 0, cs)); // M s* = s
    SpmvArgs t = spmv_args(A);
    t.st = S.st;
    t.red = S.red.r;
    t.x = M ? S.ss : S.s;
    t.y_out = S.t;
    t.w0 = S.s;
    t.w1 = nullptr;
    t.op = FIN_BICG_OMEGA;
    HEC_TRY(run_spmv(A, t, 0, 2, cs)); // t = A s*, (t, s), (t, t) -> omega
    VecArgs xr{};
    xr.n = n;
    xr.st = S.st;
    xr.red = S.red.r;
    xr.w = S.x;
    xr.u = M ? S.ps : S.p;
    xr.v = M ? S.ss : S.s;
    xr.q = S.t;
    xr.x = S.s;
    xr.y = S.r0;
    xr.z = S.r;
    xr.op = FIN_BICG_XR;
    return run_vec(V_BICG_XR, xr, cs); // x, r updates; tests; loop condition
}

// Preconditioned CG, start: ||b||, r = b - A x0 (||r|| test), z = M^{-1} r,
// rho = (r, z), p = z.
int seq_cg_rz_p(hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    double *z = S.r;
    if (M) {
        HEC_TRY(seq_precond(M, S, S.r, S.s, 0, cs)); // z = M^{-1} r
        z = S.s;
    }
    VecArgs d{};
    d.n = S.n;
    d.st = S.st;
    d.red = S.red.r;
    d.x = S.r;
    d.y = z;
    d.op = FIN_CG_RHO;
    HEC_TRY(run_vec(V_DOT, d, cs)); // (r, z): beta, rho, loop condition
    VecArgs pp{};
    pp.n = S.n;
    pp.st = S.st;
    pp.x = z;
    pp.z = S.p;
    return run_vec(V_CG_P, pp, cs); // p = z + beta p
}

int seq_cg_init(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    HEC_TRY(seq_norm_b(S, cs));
    SpmvArgs sa = spmv_args(A);
    sa.st = S.st;
    sa.red = S.red.r;
    sa.x = S.x;
    sa.alpha = -1.0;
    sa.beta = 1.0;
    sa.y_in = S.b;
    sa.y_out = S.r;
    sa.op = FIN_CG_INIT;
    HEC_TRY(run_spmv(A, sa, 2, 1, cs)); // r = b - A x0, ||r||
    return seq_cg_rz_p(M, S, cs);
}

// One pass: q = A p with (p, q) -> alpha; x += alpha p, r -= alpha q with
// ||r|| -> tests; z = M^{-1} r; (r, z) -> beta; p = z + beta p.
int seq_cg_body(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    SpmvArgs q = spmv_args(A);
    q.st = S.st;
    q.red = S.red.r;
    q.x = S.p;
    q.y_out = S.q;
    q.w0 = S.p;
    q.op = FIN_CG_ALPHA;
    HEC_TRY(run_spmv(A, q, 0, 1, cs)); // q = A p, (p, q)
    VecArgs xr{};
    xr.n = S.n;
    xr.st = S.st;
    xr.red = S.red.r;
    xr.w = S.x;
    xr.u = S.p;
    xr.q = S.q;
    xr.z = S.r;
    xr.op = FIN_CG_R;
    HEC_TRY(run_vec(V_CG_XR, xr, cs)); // x, r updates, ||r||
    return seq_cg_rz_p(M, S, cs);
}

// Exit: x = 0 if b = 0; the true residual ||b - A x|| / ||b||.
int seq_exit(hec_matrix_s *A, Solver &S, cudaStream_t cs)
{
    VecArgs zx{};
    zx.n = S.n;
    zx.st = S.st;
    zx.z = S.x;
    HEC_TRY(run_vec(V_ZERO_IF_ST, zx, cs));
    SpmvArgs fr = spmv_args(A);
    fr.st = S.st;
    fr.red = S.red.r;
    fr.x = S.x;
    fr.alpha = -1.0;
    fr.beta = 1.0;
    fr.y_in = S.b;
    fr.y_out = S.r;
    fr.op = FIN_TRUE_RESID;
    return run_spmv(A, fr, 2, 1, cs);
}

// GMRES cycle start: r = b - A x, beta = ||r||, v_1 = r / beta.
int seq_gmres_cycle(hec_matrix_s *A, Solver &S, cudaStream_t cs)
{
    SpmvArgs sa = spmv_args(A);
    sa.st = S.st;
    sa.red = S.red.r;
    sa.x = S.x;
    sa.alpha = -1.0;
    sa.beta = 1.0;
    sa.y_in = S.b;
    sa.y_out = S.r;
    sa.op = FIN_GMRES_CYCLE;
    HEC_TRY(run_spmv(A, sa, 2, 1, cs));
    VecArgs sc{};
    sc.n = S.n;
    sc.st = S.st;
    sc.xv = S.r;
    sc.zv = S.V; // column 0 (FP32 in the mixed mode: the inner solve's start vector)
    sc.guard = 2;
    if (launch_vec_typed(V_SCALE_ST, sc, false, S.mixed, vec_grid(S.n), cs) != 0)
        return fail(HEC_ERR_INVALID, "bad typed vector op");
    return check_launch("scale");
}

// One Arnoldi step: z = M^{-1} v_j, w = A z, two classical Gram-Schmidt
// passes, h_{j+1,j} = ||w||, Givens update, v_{j+1} = w / h_{j+1,j}.  In the
// mixed mode every vector of the step is FP32 (the Hessenberg column and the
// Givens rotations stay FP64 in the solver state).
int seq_gmres_step(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    const int n = S.n, m = S.restart;
    const bool f = S.mixed;
    if (M) {
        HEC_TRY(seq_precond(M, S, S.V, S.z, 1, cs)); // z = M^{-1} v_j
    } else {
        VecArgs c{};
        c.n = n;
        c.st = S.st;
        c.xv = S.V;
        c.x_from_j = 1;
        c.ldv = S.ldv;
        c.zv = S.z;
        if (launch_vec_typed(V_COPY, c, f, f, vec_grid(n), cs) != 0)
            return fail(HEC_ERR_INVALID, "bad typed vector op");
        HEC_TRY(check_launch("copy"));
    }
    SpmvArgs w = spmv_args(A);
    w.st = S.st;
    w.red = S.red.r;
    w.x = S.z;
    w.y_out = S.w;
    w.op = FIN_GMRES_W0;
    HEC_TRY(run_spmv(A, w, 0, 1, cs, f)); // w = A z, ||w||
    const int mdgrid = grid_for(n, kThreads, 2);
    BasisArgs h{};
    h.n = n;
    h.k = m + 1;
    h.k_from_st = 1;
    h.V = S.V;
    h.ldv = S.ldv;
    h.w = S.w;
    h.red = S.red.r;
    h.st = S.st;
    h.op = FIN_GMRES_H1;
    launch_multidot(h, mdgrid, cs, f); // h1 = V^T w
    HEC_TRY(check_launch("multidot"));
    BasisArgs up = h;
    up.coef = dev_field<double>(S.st, offsetof(SolverState, h1));
    up.wout = S.w;
    launch_basis_update(up, false, vec_grid(n), cs, f); // w -= V h1
    HEC_TRY(check_launch("basis update"));
    BasisArgs h2 = h;
    h2.op = FIN_GMRES_H2;
    launch_multidot(h2, mdgrid, cs, f); // h2 = V^T w
    HEC_TRY(check_launch("multidot"));
    BasisArgs up2 = h;
    up2.coef = dev_field<double>(S.st, offsetof(SolverState, h2));
    up2.wout = S.w;
    up2.op = FIN_GMRES_STEP;
    launch_basis_update(up2, true, vec_grid(n), cs, f); // w -= V h2, ||w||, Givens
    HEC_TRY(check_launch("basis update"));
    VecArgs sc{};
    sc.n = n;
    sc.st = S.st;
    sc.xv = S.w;
    sc.zv = S.V;
    sc.z_from_j = 1; // j already advanced when the cycle goes on
    sc.ldv = S.ldv;
    sc.guard = 1;
    if (launch_vec_typed(V_SCALE_ST, sc, f, f, vec_grid(n), cs) != 0) // v_{j+1} = w / h_{j+1,j}
        return fail(HEC_ERR_INVALID, "bad typed vector op");
    return check_launch("scale");
}

// Cycle end: y = R^{-1} g, x += M^{-1} V y, next cycle start.  In the mixed
// mode the correction M^{-1} V y is FP32 and is added to the FP64 x; the
// next cycle start recomputes the residual in FP64 (iterative refinement).
int seq_gmres_cycle_end(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    const bool f = S.mixed;
    if (launch_gmres_lsq(S.st, cs) != 0)
        return fail(HEC_ERR_CUDA, "lsq");
    HEC_TRY(check_launch("lsq"));
    BasisArgs cb{};
    cb.n = S.n;
    cb.k = S.restart;
    cb.k_from_st = 2;
    cb.V = S.V;
    cb.ldv = S.ldv;
    cb.coef = dev_field<double>(S.st, offsetof(SolverState, y));
    cb.wout = S.u;
    cb.st = S.st;
    launch_basis_combine(cb, vec_grid(S.n), cs, f); // u = V y
    HEC_TRY(check_launch("basis combine"));
    if (M)
        HEC_TRY(seq_precond(M, S, S.u, S.zu, 0, cs)); // zu = M^{-1} u
    VecArgs ax{};
    ax.n = S.n;
    ax.st = S.st;
    ax.xv = M ? S.zu : S.u;
    ax.zv = S.x;
    if (launch_vec_typed(V_AXPY_ST1, ax, f, false, vec_grid(S.n), cs) != 0) // x += zu
        return fail(HEC_ERR_INVALID, "bad typed vector op");
    HEC_TRY(check_launch("x update"));
    return seq_gmres_cycle(A, S, cs);
}

int seq_loopcond(Solver &S, cudaStream_t cs)
{
    if (launch_loopcond(S.st, cs) != 0)
        return fail(HEC_ERR_CUDA, "loopcond");
    return check_launch("loopcond");
}

// --- solve graphs -------------------------------------------------------------

int build_bicgstab(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    HEC_CK(cudaGraphCreate(&S.graph, 0));
    HEC_CK(cudaGraphConditionalHandleCreate(&S.h_while, S.graph, 1, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> tail;
    HEC_TRY(begin_capture(cs, S.graph, nullptr, 0));
    HEC_TRY(seq_bicg_init(A, S, cs));
    HEC_TRY(seq_loopcond(S, cs));
    HEC_TRY(end_capture(cs, tail));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    HEC_TRY(add_conditional(S.graph, tail, S.h_while, cudaGraphCondTypeWhile, wnode, body));
    HEC_TRY(begin_capture(cs, body, nullptr, 0));
    HEC_TRY(seq_bicg_body(A, M, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_TRY(begin_capture(cs, S.graph, &wnode, 1));
    HEC_TRY(seq_exit(A, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_CK(cudaGraphInstantiate(&S.exec, S.graph, 0));
    return HEC_OK;
}

int build_cg(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    HEC_CK(cudaGraphCreate(&S.graph, 0));
    HEC_CK(cudaGraphConditionalHandleCreate(&S.h_while, S.graph, 1, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> tail;
    HEC_TRY(begin_capture(cs, S.graph, nullptr, 0));
    HEC_TRY(seq_cg_init(A, M, S, cs));
    HEC_TRY(seq_loopcond(S, cs));
    HEC_TRY(end_capture(cs, tail));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    HEC_TRY(add_conditional(S.graph, tail, S.h_while, cudaGraphCondTypeWhile, wnode, body));
    HEC_TRY(begin_capture(cs, body, nullptr, 0));
    HEC_TRY(seq_cg_body(A, M, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_TRY(begin_capture(cs, S.graph, &wnode, 1));
    HEC_TRY(seq_exit(A, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_CK(cudaGraphInstantiate(&S.exec, S.graph, 0));
    return HEC_OK;
}

int build_gmres(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t cs)
{
    HEC_CK(cudaGraphCreate(&S.graph, 0));
    HEC_CK(cudaGraphConditionalHandleCreate(&S.h_while, S.graph, 1, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> tail;
    HEC_TRY(begin_capture(cs, S.graph, nullptr, 0));
    HEC_TRY(seq_norm_b(S, cs));
    HEC_TRY(seq_gmres_cycle(A, S, cs));
    HEC_TRY(seq_loopcond(S, cs));
    HEC_TRY(end_capture(cs, tail));
    cudaGraphNode_t wnode;
    cudaGraph_t body;
    HEC_TRY(add_conditional(S.graph, tail, S.h_while, cudaGraphCondTypeWhile, wnode, body));
    HEC_CK(cudaGraphConditionalHandleCreate(&S.h_if, body, 0, cudaGraphCondAssignDefault));
    HEC_TRY(begin_capture(cs, body, nullptr, 0));
    HEC_TRY(seq_gmres_step(A, M, S, cs));
    HEC_TRY(end_capture(cs, tail));
    cudaGraphNode_t ifnode;
    cudaGraph_t ifbody;
    HEC_TRY(add_conditional(body, tail, S.h_if, cudaGraphCondTypeIf, ifnode, ifbody));
    HEC_TRY(begin_capture(cs, ifbody, nullptr, 0));
    HEC_TRY(seq_gmres_cycle_end(A, M, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_TRY(begin_capture(cs, body, &ifnode, 1));
    HEC_TRY(seq_loopcond(S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_TRY(begin_capture(cs, S.graph, &wnode, 1));
    HEC_TRY(seq_exit(A, S, cs));
    HEC_TRY(end_capture(cs, tail));
    HEC_CK(cudaGraphInstantiate(&S.exec, S.graph, 0));
    return HEC_OK;
}

// The solve without graphs: the same launch sequences, the loop driven from
// the host (one small device-to-host read per iteration).
int run_eager(hec_matrix_s *A, hec_precond_s *M, Solver &S, cudaStream_t s)
{
    int flags[2] = {0, 0}; // done, cycle_end
    auto read_flags = [&]() -> int {
        HEC_CK(cudaMemcpyAsync(&flags[0], dev_field<int>(S.st, offsetof(SolverState, done)),
                               sizeof(int), cudaMemcpyDeviceToHost, s));
        HEC_CK(cudaMemcpyAsync(&flags[1], dev_field<int>(S.st, offsetof(SolverState, cycle_end)),
                               sizeof(int), cudaMemcpyDeviceToHost, s));
        HEC_CK(cudaStreamSynchronize(s));
        return HEC_OK;
    };
    if (S.method == HEC_BICGSTAB) {
        HEC_TRY(seq_bicg_init(A, S, s));
        HEC_TRY(read_flags());
        while (!flags[0]) {
            HEC_TRY(seq_bicg_body(A, M, S, s));
            HEC_TRY(read_flags());
        }
    } else if (S.method == HEC_CG) {
        HEC_TRY(seq_cg_init(A, M, S, s));
        HEC_TRY(read_flags());
        while (!flags[0]) {
            HEC_TRY(seq_cg_body(A, M, S, s));
            HEC_TRY(read_flags());
        }
    } else {
        HEC_TRY(seq_norm_b(S, s));
        HEC_TRY(seq_gmres_cycle(A, S, s));
        HEC_TRY(read_flags());
        while (!flags[0]) {
            HEC_TRY(seq_gmres_step(A, M, S, s));
            HEC_TRY(read_flags());
            if (flags[1]) {
                HEC_TRY(seq_gmres_cycle_end(A, M, S, s));
                HEC_TRY(read_flags());
            }
        }
    }
    return seq_exit(A, S, s);
}

// FP64 and FP32 vectors (of the padded length) of a solver's workspace.
int solver_vecs64(int method, int restart, bool mixed)
{
    return method == HEC_BICGSTAB ? 10 : method == HEC_CG ? 6 : (mixed ? 3 : (restart + 1) + 7);
}
int solver_vecs32(int restart, bool mixed) { return mixed ? (restart + 1) + 4 : 0; }

// The solver (workspace, graph) cached in the handles for these arguments.
Solver *cached_solver(hec_matrix_s *A, hec_precond_s *M, int method, int restart, bool mixed)
{
    auto &cache = M ? M->solvers : A->solvers;
    for (auto &p : cache)
        if (p->matrix_id == A->id && p->method == method && p->mixed == mixed &&
            (method != HEC_GMRES || p->restart == restart))
            return p.get();
    return nullptr;
}

int make_solver(hec_matrix_s *A, hec_precond_s *M, int method, int restart, bool mixed,
                cudaStream_t s, Solver *&out)
{
    auto &cache = M ? M->solvers : A->solvers;
    if (Solver *c = cached_solver(A, M, method, restart, mixed)) {
        out = c;
        return HEC_OK;
    }
    std::unique_ptr<Solver> S(new Solver());
    S->matrix_id = A->id;
    S->method = method;
    S->restart = restart;
    S->mixed = mixed;
    S->n = A->hec.n;
    S->ldv = ((int64_t)S->n + 31) / 32 * 32;
    const int64_t nv = S->ldv;
    const int nvec = solver_vecs64(method, restart, mixed);
    HEC_TRY(S->ws.alloc((size_t)nvec * nv * sizeof(double), s));
    HEC_CK(cudaMemsetAsync(S->ws.p, 0, S->ws.bytes, s));
    if (mixed) {
        // FP32 basis and step vectors of the inner cycles
        HEC_TRY(S->ws32.alloc((size_t)solver_vecs32(restart, mixed) * nv * sizeof(float), s));
        HEC_CK(cudaMemsetAsync(S->ws32.p, 0, S->ws32.bytes, s));
    }
    HEC_TRY(S->st_buf.alloc(sizeof(SolverState), s));
    HEC_CK(cudaMemsetAsync(S->st_buf.p, 0, sizeof(SolverState), s));
    HEC_TRY(S->red.init(s));
    S->st = S->st_buf.as<SolverState>();
    double *base = S->ws.as<double>();
    auto vec = [&](int i) { return base + (int64_t)i * nv; };
    if (method == HEC_BICGSTAB) {
        S->b = vec(0);
        S->x = vec(1);
        S->r = vec(2);
        S->r0 = vec(3);
        S->p = vec(4);
        S->ps = vec(5);
        S->v = vec(6);
        S->s = vec(7);
        S->ss = vec(8);
        S->t = vec(9);
    } else if (method == HEC_CG) {
        S->b = vec(0);
        S->x = vec(1);
        S->r = vec(2);
        S->s = vec(3); // z = M^{-1} r
        S->p = vec(4);
        S->q = vec(5);
    } else if (!mixed) {
        S->b = vec(0);
        S->x = vec(1);
        S->r = vec(2);
        S->z = vec(3);
        S->w = vec(4);
        S->u = vec(5);
        S->zu = vec(6);
        S->V = vec(7);
    } else {
        S->b = vec(0);
        S->x = vec(1);
        S->r = vec(2);
        float *b32 = S->ws32.as<float>();
        auto vec32 = [&](int i) { return b32 + (int64_t)i * nv; };
        S->z = vec32(0);
        S->w = vec32(1);
        S->u = vec32(2);
        S->zu = vec32(3);
        S->V = vec32(4);
    }
    HEC_CK(cudaStreamSynchronize(s));
    cudaStream_t cs;
    HEC_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int rc = method == HEC_BICGSTAB ? build_bicgstab(A, M, *S, cs)
             : method == HEC_CG     ? build_cg(A, M, *S, cs)
                                    : build_gmres(A, M, *S, cs);
    cudaStreamDestroy(cs);
    if (rc != HEC_OK)
        return rc;
    out = S.get();
    cache.push_back(std::move(S));
    return HEC_OK;
}

int upload_matrix(hec_matrix_s *A, cudaStream_t s)
{
    const HecHost &H = A->hec;
    HEC_TRY(upload(A->ell_col, H.ell_col, s));
    HEC_TRY(upload(A->ell_val, H.ell_val, s));
    HEC_TRY(upload(A->tail_rows, H.tail_rows, s));
    HEC_TRY(upload(A->tail_ptr, H.tail_ptr, s));
    HEC_TRY(upload(A->tail_col, H.tail_col, s));
    HEC_TRY(upload(A->tail_val, H.tail_val, s));
    HEC_TRY(upload(A->tile_tail, H.tile_tail, s));
    HEC_TRY(upload(A->tile_group, H.tile_group, s));
    HEC_TRY(upload(A->tile_long, H.tile_long, s));
    HEC_TRY(upload(A->tail_long, H.tail_long, s));
    HEC_TRY(A->red.init(s));
    HEC_CK(cudaStreamSynchronize(s));
    return HEC_OK;
}

} // namespace

// ====================================================================== numeric refactorisation
namespace {

// A's new values (same pattern, CSR order of hec_build): the device slab and
// tail, their FP32 copies if made, and the host CSR copy.  Stream-ordered.
int refactor_matrix(hec_matrix_s *A, const double *val, cudaStream_t s)
{
    const int n = A->hec.n;
    const int64_t nnz = (int64_t)A->csr.ci.size();
    const HostCSR &C = A->csr;
    const HecHost &H = A->hec;
    if (!A->d_slot.p) {
        // CSR entry -> ELL slot k * ld + i, or tail entry (encoded -t - 1)
        std::vector<int64_t> slot(nnz);
        int64_t t = 0;
        for (int i = 0; i < n; ++i)
            for (int e = C.rp[i]; e < C.rp[i + 1]; ++e) {
                const int k = e - C.rp[i];
                slot[e] = k < H.K ? (int64_t)k * H.ld + i : -(t++) - 1;
            }
        HEC_TRY(upload(A->d_slot, slot, s));
    }
    const double *dval = val;
    const bool dev = is_device_ptr(val);
    if (!dev) {
        if (!A->d_newval.p)
            HEC_TRY(A->d_newval.alloc(nnz * sizeof(double), s));
        HEC_CK(cudaMemcpyAsync(A->d_newval.p, val, nnz * sizeof(double), cudaMemcpyHostToDevice, s));
        dval = A->d_newval.as<double>();
    }
    launch_scatter_hec(nnz, dval, A->d_slot.as<int64_t>(), A->ell_val.as<double>(),
                       A->tail_val.as<double>(), s);
    HEC_TRY(check_launch("scatter"));
    if (A->f32_ready) {
        launch_cast_f32((int64_t)H.ell_val.size(), A->ell_val.as<double>(),
                        A->ell_val32.as<float>(), s);
        launch_cast_f32((int64_t)H.tail_val.size(), A->tail_val.as<double>(),
                        A->tail_val32.as<float>(), s);
        HEC_TRY(check_launch("cast"));
    }
    // the host CSR copy: later host-side setups read it
    HEC_CK(cudaMemcpyAsync(A->csr.va.data(), val, nnz * sizeof(double),
                           dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    A->hec_host_stale = true;
    // the values the preconditioner step reads
    A->d_newval_view = dval;
    return HEC_OK;
}

// The factor data of every block on the device, built on the first refactor.
int upload_refactor_data(const hec_matrix_s *A, hec_precond_s *M, cudaStream_t s)
{
    if (M->rf_ready)
        return HEC_OK;
    const int nb = M->nblocks;
    std::vector<int> row0(nb + 1, 0), lev0(nb + 1, 0);
    int64_t nent = 0;
    for (int b = 0; b < nb; ++b) {
        row0[b + 1] = row0[b] + M->blocks[b].F.n;
        lev0[b + 1] = lev0[b] + (int)M->blocks[b].lptrL.size();
        nent += (int64_t)M->blocks[b].F.ci.size();
    }
    if (nent >= INT32_MAX)
        return fail(HEC_ERR_INVALID, "factors of %lld entries exceed the refactor index range",
                    (long long)nent);
    std::vector<int> rp((size_t)row0[nb] + 1), ci((size_t)nent), dg((size_t)row0[nb]),
        src((size_t)nent), lptr((size_t)lev0[nb]), lrows((size_t)row0[nb]);
    const HostCSR &C = A->csr;
    parallel_for(nb, [&](int b) {
        const BlockFactor &B = M->blocks[b];
        const HostCSR &F = B.F;
        int64_t e0 = 0;
        for (int q = 0; q < b; ++q)
            e0 += (int64_t)M->blocks[q].F.ci.size();
        for (int i = 0; i < F.n; ++i) {
            const int r = row0[b] + i;
            rp[r] = (int)(e0 + F.rp[i]);
            dg[r] = (int)(e0 + B.diag[i]);
            lrows[r] = B.lrowsL[i];
            const int g = B.rows[i];
            for (int e = F.rp[i]; e < F.rp[i + 1]; ++e) {
                ci[e0 + e] = F.ci[e];
                int sidx = -1;
                if (B.lev[e] == 0) { // an entry of A[V_b, V_b]
                    const int gc = B.rows[F.ci[e]];
                    const int *lo = C.ci.data() + C.rp[g], *hi = C.ci.data() + C.rp[g + 1];
                    const int *it = std::lower_bound(lo, hi, gc);
                    if (it != hi && *it == gc)
                        sidx = (int)(it - C.ci.data());
                }
                src[e0 + e] = sidx;
            }
        }
        for (size_t l = 0; l < B.lptrL.size(); ++l)
            lptr[lev0[b] + l] = B.lptrL[l];
    });
    rp[row0[nb]] = (int)nent;
    HEC_TRY(upload(M->rf_rp, rp, s));
    HEC_TRY(upload(M->rf_ci, ci, s));
    HEC_TRY(upload(M->rf_dg, dg, s));
    HEC_TRY(upload(M->rf_src, src, s));
    HEC_TRY(upload(M->rf_row0, row0, s));
    HEC_TRY(upload(M->rf_lev0, lev0, s));
    HEC_TRY(upload(M->rf_lptr, lptr, s));
    HEC_TRY(upload(M->rf_lrows, lrows, s));
    HEC_TRY(M->rf_f.alloc(nent * sizeof(double), s));
    HEC_CK(cudaStreamSynchronize(s));
    M->rf_nent = nent;
    M->rf_ready = true;
    return HEC_OK;
}

int refactor_precond(hec_matrix_s *A, hec_precond_s *M, cudaStream_t s)
{
    const double *dval = A->d_newval_view;
    if (M->kind == kJacobi) {
        if (!A->d_diagidx.p) {
            std::vector<int64_t> d(M->n, -1);
            const HostCSR &C = A->csr;
            for (int i = 0; i < M->n; ++i)
                for (int e = C.rp[i]; e < C.rp[i + 1]; ++e)
                    if (C.ci[e] == i)
                        d[i] = e;
            HEC_TRY(upload(A->d_diagidx, d, s));
        }
        launch_jacobi_dinv(M->n, dval, A->d_diagidx.as<int64_t>(), M->omega, M->dinv.as<double>(),
                           M->dinv32.p ? M->dinv32.as<float>() : nullptr, M->d_err.as<int>(), s);
        return check_launch("jacobi dinv");
    }
    HEC_TRY(upload_refactor_data(A, M, s));
    RefactorArgs ra{};
    ra.nent = M->rf_nent;
    ra.val = dval;
    ra.src = M->rf_src.as<int>();
    ra.f = M->rf_f.as<double>();
    ra.rp = M->rf_rp.as<int>();
    ra.ci = M->rf_ci.as<int>();
    ra.dg = M->rf_dg.as<int>();
    ra.blk_row0 = M->rf_row0.as<int>();
    ra.blk_lev0 = M->rf_lev0.as<int>();
    ra.lptr = M->rf_lptr.as<int>();
    ra.lrows = M->rf_lrows.as<int>();
    ra.err = M->d_err.as<int>();
    launch_refactor(ra, M->nblocks, s);
    HEC_TRY(check_launch("refactor"));
    for (int idx = 0; idx < 2; ++idx) {
        TrsvLayout &L = M->lay[idx];
        if (!L.built)
            continue;
        if (!L.d_row0.p) {
            HEC_TRY(upload(L.d_row0, L.pack.chunk_row0, s));
            HEC_TRY(upload(L.d_rms, L.pack.rm_start, s));
            HEC_TRY(upload(L.d_rml, L.pack.rm_len, s));
            HEC_TRY(upload(L.d_rmd, L.pack.rm_diag, s));
        }
        FillArgs fa{};
        fa.pack = L.d_pack.as<unsigned char>();
        fa.chunks = L.d_chunks.as<uint2>();
        fa.chunk_row0 = L.d_row0.as<int64_t>();
        fa.rm_start = L.d_rms.as<int>();
        fa.rm_len = L.d_rml.as<int>();
        fa.rm_diag = L.d_rmd.as<int>();
        fa.f = M->rf_f.as<double>();
        launch_fill_pack(fa, (int)L.pack.chunks.size(), idx == 1, s);
        HEC_TRY(check_launch("fill"));
    }
    M->factor_host_stale = true;
    return HEC_OK;
}

} // namespace

// ====================================================================== C ABI
extern "C" {

const char *hec_status_string(int status)
{
    switch (status) {
    case HEC_OK: return "ok";
    case HEC_ERR_INVALID: return "invalid argument";
    case HEC_ERR_OOM: return "out of device memory";
    case HEC_ERR_ZERO_PIVOT: return "zero pivot in ILU(k)";
    case HEC_ERR_UNSORTED_CSR: return "CSR columns not strictly ascending or out of range";
    case HEC_ERR_CUDA: return "CUDA error";
    case HEC_ERR_TIMEOUT: return "bounded device wait ran out";
    case HEC_MAXIT: return "iteration limit reached";
    case HEC_BREAKDOWN: return "solver breakdown";
    default: return "unknown status";
    }
}

const char *hec_last_error(void) { return hec::last_error_text(); }

int hec_set_allocator(void *(*alloc_fn)(size_t, void *, void *), void (*free_fn)(void *, void *, void *),
                      void *ctx)
{
    return abi_guard(__func__, [&]() -> int {
        if ((alloc_fn == nullptr) != (free_fn == nullptr))
            return fail(HEC_ERR_INVALID, "allocator needs both functions or neither");
        AllocFns f;
        f.alloc = alloc_fn;
        f.free_ = free_fn;
        f.ctx = ctx;
        set_allocator(f);
        return HEC_OK;
    });
}

int hec_build(const hec_csr_t *Ain, const hec_opts_t *opts, void *stream, hec_matrix_t *out)
{
    return abi_guard(__func__, [&]() -> int {
        if (!Ain || !out)
            return fail(HEC_ERR_INVALID, "null argument");
        *out = nullptr;
        hec_opts_t o{};
        if (opts)
            o = *opts;
        const int align = o.ell_ld_align ? o.ell_ld_align : 256;
        if (align < 32 || align % 32 != 0)
            return fail(HEC_ERR_INVALID, "ell_ld_align must be a positive multiple of 32");
        if (o.ell_width < 0)
            return fail(HEC_ERR_INVALID, "ell_width must be >= 0");
        const int n = Ain->n, nnz = Ain->nnz;
        if (n < 1 || nnz < 0)
            return fail(HEC_ERR_INVALID, "bad sizes n=%d nnz=%d", n, nnz);
        cudaStream_t s = (cudaStream_t)stream;
        std::unique_ptr<hec_matrix_s> A(new hec_matrix_s());
        A->id = g_next_id++;
        A->host_only = (o.flags & HEC_HOST_ONLY) != 0;
        HostCSR &C = A->csr;
        C.n = n;
        C.rp.resize(n + 1);
        C.ci.resize(nnz);
        C.va.resize(nnz);
        if (Ain->on_device) {
            HEC_CK(cudaMemcpy(C.rp.data(), Ain->row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
            if (nnz) {
                HEC_CK(cudaMemcpy(C.ci.data(), Ain->col, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
                HEC_CK(cudaMemcpy(C.va.data(), Ain->val, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
            }
        } else {
            if (!Ain->row_ptr || (nnz && (!Ain->col || !Ain->val)))
                return fail(HEC_ERR_INVALID, "null CSR array");
            std::memcpy(C.rp.data(), Ain->row_ptr, sizeof(int) * (n + 1));
            if (nnz) {
                std::memcpy(C.ci.data(), Ain->col, sizeof(int) * nnz);
                std::memcpy(C.va.data(), Ain->val, sizeof(double) * nnz);
            }
        }
        std::string msg;
        int rc = check_csr(n, C.rp.data(), C.ci.data(), nnz, false, msg);
        if (rc != HEC_OK)
            return fail(rc, "%s", msg.c_str());
        const int K = o.ell_width ? o.ell_width : ell_width_auto(C);
        build_hec(C, K, align, A->hec);
        if (!A->host_only)
            HEC_TRY(upload_matrix(A.get(), s));
        *out = A.release();
        return HEC_OK;
    });
}

int hec_matrix_info(hec_matrix_t A, hec_matrix_info_t *info)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !info)
            return fail(HEC_ERR_INVALID, "null argument");
        info->n = A->hec.n;
        info->nnz = (int32_t)A->csr.ci.size();
        info->ell_width = A->hec.K;
        info->ell_ld = A->hec.ld;
        info->tail_rows = (int32_t)A->hec.tail_rows.size();
        info->tail_nnz = (int32_t)A->hec.tail_col.size();
        info->device_bytes = A->device_bytes();
        return HEC_OK;
    });
}

int hec_matrix_export(hec_matrix_t A, int32_t *ell_col, double *ell_val, int32_t *tail_rows,
                      int32_t *tail_ptr, int32_t *tail_col, double *tail_val)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A)
            return fail(HEC_ERR_INVALID, "null matrix");
        if (A->hec_host_stale) { // hec_refactor replaced the values on the device
            HEC_CK(cudaMemcpy(A->hec.ell_val.data(), A->ell_val.p,
                              A->hec.ell_val.size() * sizeof(double), cudaMemcpyDeviceToHost));
            HEC_CK(cudaMemcpy(A->hec.tail_val.data(), A->tail_val.p,
                              A->hec.tail_val.size() * sizeof(double), cudaMemcpyDeviceToHost));
            A->hec_host_stale = false;
        }
        const HecHost &H = A->hec;
        auto cp = [](void *dst, const void *src, size_t bytes) {
            if (dst && bytes)
                std::memcpy(dst, src, bytes);
        };
        cp(ell_col, H.ell_col.data(), H.ell_col.size() * sizeof(int));
        cp(ell_val, H.ell_val.data(), H.ell_val.size() * sizeof(double));
        cp(tail_rows, H.tail_rows.data(), H.tail_rows.size() * sizeof(int));
        cp(tail_ptr, H.tail_ptr.data(), H.tail_ptr.size() * sizeof(int));
        cp(tail_col, H.tail_col.data(), H.tail_col.size() * sizeof(int));
        cp(tail_val, H.tail_val.data(), H.tail_val.size() * sizeof(double));
        return HEC_OK;
    });
}

void hec_matrix_destroy(hec_matrix_t A) { delete A; }

int hec_spmv(hec_matrix_t A, double alpha, const double *x, double beta, const double *y_in,
             double *y_out, const double *w, double *dots, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !x || !y_out)
            return fail(HEC_ERR_INVALID, "null argument");
        // a thread stores its two adjacent rows with one 16-byte store
        if (reinterpret_cast<uintptr_t>(y_out) % (2 * sizeof(double)) != 0)
            return fail(HEC_ERR_INVALID, "y_out must be 16-byte aligned");
        if (A->host_only)
            return fail(HEC_ERR_INVALID, "host-only matrix has no device data");
        if (beta != 0.0 && !y_in)
            return fail(HEC_ERR_INVALID, "y_in is needed when beta != 0");
        if (x == y_out)
            return fail(HEC_ERR_INVALID, "x and y_out must not alias");
        SpmvArgs a = spmv_args(A);
        a.x = x;
        a.alpha = alpha;
        a.beta = beta;
        a.y_in = y_in;
        a.y_out = y_out;
        a.red = A->red.r;
        a.w0 = w;
        a.w1 = nullptr;
        a.result = dots;
        a.op = FIN_STORE;
        const int mode = (beta != 0.0) ? 2 : (alpha != 1.0 ? 1 : 0);
        return run_spmv(A, a, mode, dots ? 2 : 0, (cudaStream_t)stream);
    });
}

int hec_spmv_f32(hec_matrix_t A, float alpha, const float *x, float beta, const float *y_in,
                 float *y_out, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !x || !y_out)
            return fail(HEC_ERR_INVALID, "null argument");
        // a thread stores its four adjacent rows with one 16-byte store
        if (reinterpret_cast<uintptr_t>(y_out) % (4 * sizeof(float)) != 0)
            return fail(HEC_ERR_INVALID, "y_out must be 16-byte aligned");
        if (A->host_only)
            return fail(HEC_ERR_INVALID, "host-only matrix has no device data");
        if (beta != 0.0f && !y_in)
            return fail(HEC_ERR_INVALID, "y_in is needed when beta != 0");
        if ((const void *)x == (const void *)y_out)
            return fail(HEC_ERR_INVALID, "x and y_out must not alias");
        cudaStream_t s = (cudaStream_t)stream;
        HEC_TRY(ensure_f32(A, s));
        SpmvArgs a = spmv_args(A);
        a.x = x;
        a.alpha = alpha;
        a.beta = beta;
        a.y_in = y_in;
        a.y_out = y_out;
        const int mode = (beta != 0.0f) ? 2 : (alpha != 1.0f ? 1 : 0);
        return run_spmv(A, a, mode, 0, s, true);
    });
}

int hec_axpby(int32_t n, double a, const double *x, double b, double *y, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (n < 0 || (n > 0 && (!x || !y)))
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (n == 0)
            return HEC_OK;
        VecArgs v{};
        v.n = n;
        v.a = a;
        v.b = b;
        v.x = x;
        v.z = y;
        return run_vec(V_AXPBY, v, (cudaStream_t)stream);
    });
}

int hec_waxpby(int32_t n, double a, const double *x, double b, const double *y, double *z,
               void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (n < 0 || (n > 0 && (!x || !y || !z)))
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (n == 0)
            return HEC_OK;
        VecArgs v{};
        v.n = n;
        v.a = a;
        v.b = b;
        v.x = x;
        v.y = y;
        v.z = z;
        return run_vec(V_WAXPBY, v, (cudaStream_t)stream);
    });
}

int hec_dot(int32_t n, const double *x, const double *y, double *result, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (n < 0 || !result || (n > 0 && (!x || !y)))
            return fail(HEC_ERR_INVALID, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        if (n == 0) {
            HEC_CK(cudaMemsetAsync(result, 0, sizeof(double), s));
            return HEC_OK;
        }
        VecArgs v{};
        v.n = n;
        v.x = x;
        v.y = y;
        v.result = result;
        v.op = FIN_STORE;
        HEC_TRY(global_reducer(s, v.red));
        return run_vec(V_DOT, v, s);
    });
}

int hec_nrm2(int32_t n, const double *x, double *result, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (n < 0 || !result || (n > 0 && !x))
            return fail(HEC_ERR_INVALID, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        if (n == 0) {
            HEC_CK(cudaMemsetAsync(result, 0, sizeof(double), s));
            return HEC_OK;
        }
        VecArgs v{};
        v.n = n;
        v.x = x;
        v.result = result;
        v.op = FIN_STORE;
        HEC_TRY(global_reducer(s, v.red));
        v.op = FIN_STORE_SQRT;
        return run_vec(V_NRM2SQ, v, s);
    });
}

int hec_multidot(int32_t n, int32_t k, const double *V, int64_t ldv, const double *w, double *h,
                 void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (n < 1 || k < 1 || k > kMaxRestart + 1 || ldv < n || !V || !w || !h)
            return fail(HEC_ERR_INVALID, "bad arguments (k must be in 1..%d)", kMaxRestart + 1);
        cudaStream_t s = (cudaStream_t)stream;
        BasisArgs a{};
        a.n = n;
        a.k = k;
        a.V = V;
        a.ldv = ldv;
        a.w = w;
        a.result = h;
        a.op = FIN_STORE;
        HEC_TRY(global_reducer(s, a.red));
        launch_multidot(a, grid_for(n, kThreads, 2), s);
        return check_launch("multidot");
    });
}

int ilu_k_setup(hec_matrix_t A, int32_t k, int32_t nblocks, int32_t overlap, void *stream,
                hec_precond_t *out)
{
    return abi_guard(__func__, [&]() -> int {
        (void)stream;
        if (!A || !out)
            return fail(HEC_ERR_INVALID, "null argument");
        *out = nullptr;
        const int n = A->hec.n;
        if (k < 0 || overlap < 0 || nblocks < 1 || nblocks > n)
            return fail(HEC_ERR_INVALID, "need k >= 0, overlap >= 0, 1 <= nblocks <= n");
        std::string msg;
        int rc = check_csr(n, A->csr.rp.data(), A->csr.ci.data(), (int)A->csr.ci.size(), true, msg);
        if (rc != HEC_OK)
            return fail(rc, "%s", msg.c_str());
        std::unique_ptr<hec_precond_s> M(new hec_precond_s());
        M->matrix_id = A->id;
        M->n = n;
        M->k = k;
        M->nblocks = nblocks;
        M->overlap = overlap;
        M->host_only = A->host_only;
        ras_blocks(A->csr, nblocks, overlap, M->blocks);
        std::vector<int> rcs(nblocks, HEC_OK);
        std::vector<std::string> msgs(nblocks);
        parallel_for(nblocks, [&](int b) { rcs[b] = iluk_block(M->blocks[b], k, msgs[b]); });
        for (int b = 0; b < nblocks; ++b)
            if (rcs[b] != HEC_OK)
                return fail(rcs[b], "block %d: %s", b, msgs[b].c_str());
        *out = M.release();
        return HEC_OK;
    });
}

int hec_jacobi_setup(hec_matrix_t A, double omega, void *stream, hec_precond_t *out)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !out)
            return fail(HEC_ERR_INVALID, "null argument");
        *out = nullptr;
        if (!(omega > 0.0) || !std::isfinite(omega))
            return fail(HEC_ERR_INVALID, "omega must be a finite positive number");
        const int n = A->hec.n;
        const HostCSR &C = A->csr;
        std::vector<double> d(n);
        for (int i = 0; i < n; ++i) {
            double a = 0.0;
            for (int e = C.rp[i]; e < C.rp[i + 1]; ++e)
                if (C.ci[e] == i)
                    a = C.va[e];
            if (a == 0.0)
                return fail(HEC_ERR_ZERO_PIVOT, "row %d has a zero or missing diagonal entry", i);
            d[i] = omega / a;
        }
        std::unique_ptr<hec_precond_s> M(new hec_precond_s());
        M->matrix_id = A->id;
        M->kind = kJacobi;
        M->omega = omega;
        M->n = n;
        M->host_only = A->host_only;
        cudaStream_t s = (cudaStream_t)stream;
        if (!M->host_only) {
            HEC_TRY(upload(M->dinv, d, s));
            HEC_TRY(M->d_err.alloc(sizeof(int), s));
            HEC_CK(cudaMemsetAsync(M->d_err.p, 0, sizeof(int), s));
            HEC_CK(cudaStreamSynchronize(s));
        }
        M->scheduled = true;
        *out = M.release();
        return HEC_OK;
    });
}

int level_schedule(hec_precond_t M, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M)
            return fail(HEC_ERR_INVALID, "null preconditioner");
        if (M->scheduled)
            return HEC_OK; // also every damped-Jacobi handle: nothing to schedule
        cudaStream_t s = (cudaStream_t)stream;
        parallel_for(M->nblocks, [&](int b) { levels_block(M->blocks[b]); });
        HEC_TRY(build_layout(M, 0, s));
        if (!M->host_only) {
            HEC_TRY(M->d_err.alloc(sizeof(int), s));
            HEC_CK(cudaMemsetAsync(M->d_err.p, 0, sizeof(int), s));
            HEC_CK(cudaStreamSynchronize(s));
        }
        M->scheduled = true;
        return HEC_OK;
    });
}

int hec_precond_info(hec_precond_t M, hec_precond_info_t *info)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || !info)
            return fail(HEC_ERR_INVALID, "null argument");
        std::memset(info, 0, sizeof(*info));
        info->nblocks = M->nblocks;
        info->overlap = M->overlap;
        info->k = M->kind == kJacobi ? -1 : M->k;
        info->scheduled = M->scheduled ? 1 : 0;
        for (const BlockFactor &B : M->blocks) {
            info->rows_total += B.F.n;
            info->factor_nnz += (int64_t)B.F.ci.size();
            info->max_levels_L = std::max(info->max_levels_L, B.nlevL);
            info->max_levels_U = std::max(info->max_levels_U, B.nlevU);
        }
        info->apply_bytes = M->kind == kJacobi ? (int64_t)M->n * 24 // r, d read; z written
                            : M->scheduled          ? M->lay[0].pack.alg_bytes
                                                    : 0;
        info->device_bytes = M->device_bytes();
        info->ring_slots = M->scheduled ? M->lay[0].pack.ring_slots : 0;
        info->apply_bytes_f32 = M->lay[1].built ? M->lay[1].pack.alg_bytes : 0;
        for (const TrsvBlock &T : M->lay[0].pack.blocks)
            info->global_passes += (T.ring_L ? 0 : 1) + (T.ring_U ? 0 : 1);
        info->trsv_parts = M->scheduled && M->kind != kJacobi ? M->lay[0].pack.parts : 0;
        info->trsv_resident = M->scheduled && M->kind != kJacobi ? M->lay[0].pack.resident : 0;
        info->import_slots = M->scheduled && M->kind != kJacobi ? M->lay[0].pack.import_slots : 0;
        {
            const TrsvPack &P = M->lay[0].pack;
            for (size_t q = 0; q < P.blocks.size(); q += (size_t)std::max(P.parts, 1))
                info->split_blocks += (P.blocks[q].links & 2) ? 1 : 0;
        }
        return HEC_OK;
    });
}

int hec_precond_get_block(hec_precond_t M, int32_t b, int32_t *nv, int32_t *own_lo,
                          int32_t *own_hi, int32_t *rows)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || b < 0 || b >= M->nblocks)
            return fail(HEC_ERR_INVALID, "bad block");
        const BlockFactor &B = M->blocks[b];
        if (nv)
            *nv = (int32_t)B.rows.size();
        if (own_lo)
            *own_lo = B.own_lo;
        if (own_hi)
            *own_hi = B.own_hi;
        if (rows)
            std::memcpy(rows, B.rows.data(), B.rows.size() * sizeof(int));
        return HEC_OK;
    });
}

int hec_precond_get_factor(hec_precond_t M, int32_t b, int32_t *nnz, int32_t *row_ptr,
                           int32_t *col, double *val, int32_t *lev)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || b < 0 || b >= M->nblocks || !nnz)
            return fail(HEC_ERR_INVALID, "bad arguments");
        HEC_TRY(refresh_host_factors(M, nullptr));
        const BlockFactor &B = M->blocks[b];
        *nnz = (int32_t)B.F.ci.size();
        if (row_ptr)
            std::memcpy(row_ptr, B.F.rp.data(), B.F.rp.size() * sizeof(int));
        if (col)
            std::memcpy(col, B.F.ci.data(), B.F.ci.size() * sizeof(int));
        if (val)
            std::memcpy(val, B.F.va.data(), B.F.va.size() * sizeof(double));
        if (lev)
            std::memcpy(lev, B.lev.data(), B.lev.size() * sizeof(int));
        return HEC_OK;
    });
}

int hec_precond_get_levels(hec_precond_t M, int32_t b, int32_t which, int32_t *nlev,
                           int32_t *level_ptr, int32_t *level_rows)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || b < 0 || b >= M->nblocks || (which != HEC_FACTOR_L && which != HEC_FACTOR_U))
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (!M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        const BlockFactor &B = M->blocks[b];
        const bool u = which == HEC_FACTOR_U;
        if (nlev)
            *nlev = u ? B.nlevU : B.nlevL;
        const std::vector<int> &p = u ? B.lptrU : B.lptrL;
        const std::vector<int> &r = u ? B.lrowsU : B.lrowsL;
        if (level_ptr)
            std::memcpy(level_ptr, p.data(), p.size() * sizeof(int));
        if (level_rows)
            std::memcpy(level_rows, r.data(), r.size() * sizeof(int));
        return HEC_OK;
    });
}

int hec_precond_get_layout(hec_precond_t M, int32_t fp32, int64_t *pack_bytes, int32_t *nchunks,
                           int32_t *ring_slots, int32_t *import_slots, int32_t *parts,
                           int32_t *fixed_width, void *pack, uint32_t *chunks, int64_t *programs,
                           void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || (fp32 != 0 && fp32 != 1) || !pack_bytes || !nchunks || !ring_slots ||
            !import_slots || !parts || !fixed_width)
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (M->kind == kJacobi)
            return fail(HEC_ERR_INVALID, "a damped-Jacobi preconditioner has no factor layout");
        if (!M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        HEC_TRY(build_layout(M, fp32, s));
        const TrsvLayout &L = M->lay[fp32];
        int64_t total = 0;
        for (const uint2 &c : L.pack.chunks)
            total = std::max<int64_t>(total, (int64_t)c.x * 16 + c.y);
        *pack_bytes = total;
        *nchunks = (int32_t)L.pack.chunks.size();
        *ring_slots = L.pack.ring_slots;
        *import_slots = L.pack.import_slots;
        *parts = L.pack.parts;
        *fixed_width = L.fixed_width;
        if (pack && total > 0) {
            if (!L.pack.pack.empty()) {
                std::memcpy(pack, L.pack.pack.data(), (size_t)total);
            } else { // uploaded (and possibly refilled by hec_refactor): the device copy
                HEC_CK(cudaMemcpyAsync(pack, L.d_pack.p, (size_t)total, cudaMemcpyDeviceToHost, s));
                HEC_CK(cudaStreamSynchronize(s));
            }
        }
        if (chunks)
            for (size_t c = 0; c < L.pack.chunks.size(); ++c) {
                chunks[2 * c] = L.pack.chunks[c].x;
                chunks[2 * c + 1] = L.pack.chunks[c].y;
            }
        if (programs)
            for (size_t b = 0; b < L.pack.blocks.size(); ++b) {
                const TrsvBlock &T = L.pack.blocks[b];
                int64_t *o = programs + 8 * b;
                o[0] = T.chunk_begin;
                o[1] = T.chunk_mid;
                o[2] = T.chunk_end;
                o[3] = T.ring_L;
                o[4] = T.ring_U;
                o[5] = T.yoff;
                o[6] = T.zoff;
                o[7] = T.links;
            }
        return HEC_OK;
    });
}

int hec_debug_record(int32_t *record, int32_t clear)
{
    return abi_guard(__func__, [&]() -> int {
        if (!record)
            return fail(HEC_ERR_INVALID, "null record");
        if (!trsv_debug_build())
            return fail(HEC_ERR_INVALID, "not a debug build (compile with HEC_DEBUG)");
        int r[8];
        if (trsv_debug_read(r, clear != 0) != 0)
            return fail(HEC_ERR_CUDA, "cannot read the debug record");
        std::memcpy(record, r, sizeof(r));
        return HEC_OK;
    });
}

int hec_precond_set_trsv_parts(hec_precond_t M, int32_t parts)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || (parts != 0 && parts != 1 && parts != 2 && parts != 4 && parts != 8))
            return fail(HEC_ERR_INVALID, "parts must be 0 (automatic), 1, 2, 4 or 8");
        if (M->kind == kJacobi)
            return fail(HEC_ERR_INVALID, "a damped-Jacobi preconditioner has no triangular solve");
        if (M->scheduled)
            return fail(HEC_ERR_INVALID, "set the parts before level_schedule");
        M->trsv_parts = parts;
        return HEC_OK;
    });
}

int hec_precond_set_trsv_kernel(hec_precond_t M, int32_t kernel)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || (kernel != HEC_TRSV_AUTO && kernel != HEC_TRSV_STREAMED &&
                   kernel != HEC_TRSV_RESIDENT))
            return fail(HEC_ERR_INVALID,
                        "kernel must be HEC_TRSV_AUTO, HEC_TRSV_STREAMED or HEC_TRSV_RESIDENT");
        if (M->kind == kJacobi)
            return fail(HEC_ERR_INVALID, "a damped-Jacobi preconditioner has no triangular solve");
        if (M->scheduled)
            return fail(HEC_ERR_INVALID, "choose the kernel before level_schedule");
        M->trsv_kernel = kernel;
        return HEC_OK;
    });
}

int hec_precond_apply(hec_precond_t M, const double *r, double *z, int64_t spin_limit, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || !r || !z || r == z)
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (M->host_only)
            return fail(HEC_ERR_INVALID, "host-only preconditioner has no device data");
        if (!M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        if (M->kind == kJacobi)
            return run_jacobi(M, r, z, false, (cudaStream_t)stream);
        TrsvArgs a = trsv_args(M, M->lay[0], spin_limit ? spin_limit : kDefaultSpin);
        a.r = r;
        a.z = z;
        return run_trsv(a, (cudaStream_t)stream);
    });
}

int hec_precond_apply_f32(hec_precond_t M, const float *r, float *z, int64_t spin_limit,
                          void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || !r || !z || (const void *)r == (const void *)z)
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (M->host_only)
            return fail(HEC_ERR_INVALID, "host-only preconditioner has no device data");
        if (!M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        cudaStream_t s = (cudaStream_t)stream;
        HEC_TRY(ensure_precond_f32(M, s));
        if (M->kind == kJacobi)
            return run_jacobi(M, r, z, true, s);
        TrsvArgs a = trsv_args(M, M->lay[1], spin_limit ? spin_limit : kDefaultSpin);
        a.r = r;
        a.z = z;
        return run_trsv(a, s, true);
    });
}

int hec_precond_status(hec_precond_t M, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || M->host_only || !M->scheduled)
            return fail(HEC_ERR_INVALID, "bad preconditioner");
        cudaStream_t s = (cudaStream_t)stream;
        int err = 0;
        HEC_CK(cudaMemcpyAsync(&err, M->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        HEC_CK(cudaStreamSynchronize(s));
        if (err) {
            HEC_CK(cudaMemsetAsync(M->d_err.p, 0, sizeof(int), s));
            HEC_CK(cudaStreamSynchronize(s));
            return fail(err, "a bounded device wait ran out");
        }
        return HEC_OK;
    });
}

void hec_precond_destroy(hec_precond_t M) { delete M; }

int hec_refactor(hec_matrix_t A, hec_precond_t M, const double *val, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !val)
            return fail(HEC_ERR_INVALID, "null argument");
        if (A->host_only || (M && M->host_only))
            return fail(HEC_ERR_INVALID, "host-only handle");
        if (M && M->matrix_id != A->id)
            return fail(HEC_ERR_INVALID, "preconditioner was built from another matrix");
        if (M && M->kind != kJacobi && !M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        cudaStream_t s = (cudaStream_t)stream;
        HEC_TRY(refactor_matrix(A, val, s));
        if (M)
            HEC_TRY(refactor_precond(A, M, s));
        HEC_CK(cudaStreamSynchronize(s));
        if (M) {
            int err = 0;
            HEC_CK(cudaMemcpy(&err, M->d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
            if (err) {
                HEC_CK(cudaMemset(M->d_err.p, 0, sizeof(int)));
                return fail(err, "numeric refactorisation: a pivot is zero");
            }
        }
        return HEC_OK;
    });
}

int hec_workspace_bytes(hec_matrix_t A, hec_precond_t M, int32_t restart,
                        const hec_solve_opts_t *opts, int64_t *bytes)
{
    return abi_guard(__func__, [&]() -> int {
        if (!A || !bytes)
            return fail(HEC_ERR_INVALID, "null argument");
        *bytes = 0;
        if (M && (M->matrix_id != A->id))
            return fail(HEC_ERR_INVALID, "preconditioner was built from another matrix");
        if (M && !M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        hec_solve_opts_t o{};
        if (opts)
            o = *opts;
        if (o.method != HEC_GMRES && o.method != HEC_BICGSTAB && o.method != HEC_CG)
            return fail(HEC_ERR_INVALID, "unknown method");
        if (o.method == HEC_GMRES && (restart < 1 || restart > kMaxRestart))
            return fail(HEC_ERR_INVALID, "restart must be in 1..%d", kMaxRestart);
        if (o.method != HEC_GMRES)
            restart = 0;
        const bool mixed = (o.flags & HEC_MIXED_FP32) != 0;
        if (mixed && o.method != HEC_GMRES)
            return fail(HEC_ERR_INVALID, "HEC_MIXED_FP32 needs method HEC_GMRES");
        // a device allocation of 0 bytes takes 16 (DevBuf)
        auto dev = [](int64_t b) { return b > 0 ? b : (int64_t)16; };
        int64_t total = 0;
        if (!cached_solver(A, M, o.method, restart, mixed)) {
            const int64_t nv = ((int64_t)A->hec.n + 31) / 32 * 32;
            total += dev(solver_vecs64(o.method, restart, mixed) * nv * (int64_t)sizeof(double));
            if (mixed)
                total += dev(solver_vecs32(restart, mixed) * nv * (int64_t)sizeof(float));
            total += (int64_t)sizeof(SolverState) + (int64_t)Reducer::capacity() * 8 +
                     (int64_t)sizeof(unsigned);
        }
        if (mixed && !A->f32_ready)
            total += dev((int64_t)A->hec.ell_val.size() * 4) + dev((int64_t)A->hec.tail_val.size() * 4);
        if (mixed && M && M->kind == kJacobi && !M->dinv32.p)
            total += dev((int64_t)M->n * 4);
        if (mixed && M && M->kind != kJacobi && !M->lay[1].built) {
            // the FP32 layout the first mixed solve packs and uploads, packed
            // here on the host to be counted
            TrsvPack P;
            std::string msg;
            int fw = 0, ns = 0;
            const int rc = pack_layout(M, 1, P, fw, ns, msg);
            if (rc != HEC_OK)
                return fail(rc, "%s", msg.c_str());
            total += dev((int64_t)P.pack.size()) + dev((int64_t)(P.chunks.size() * sizeof(uint2))) +
                     dev((int64_t)(P.blocks.size() * sizeof(TrsvBlock))) +
                     std::max<int64_t>(P.ysz, 1) * 4 + std::max<int64_t>(P.zsz, 1) * 4 +
                     (P.resident ? dev((int64_t)(P.vrows.size() * sizeof(int))) +
                                       dev((int64_t)(P.groups.size() * sizeof(uint2)))
                                 : 0);
        }
        *bytes = total;
        return HEC_OK;
    });
}

int krylov_solve(hec_matrix_t A, hec_precond_t M, const double *b, double *x, double tol,
                 int32_t maxit, int32_t restart, const hec_solve_opts_t *opts, void *stream,
                 hec_solve_info_t *info)
{
    return abi_guard(__func__, [&]() -> int {
        if (info)
            std::memset(info, 0, sizeof(*info));
        if (!A || !b || !x)
            return fail(HEC_ERR_INVALID, "null argument");
        if (A->host_only || (M && M->host_only))
            return fail(HEC_ERR_INVALID, "host-only handle");
        if (M && (M->matrix_id != A->id))
            return fail(HEC_ERR_INVALID, "preconditioner was built from another matrix");
        if (M && !M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        hec_solve_opts_t o{};
        if (opts)
            o = *opts;
        if (o.method != HEC_GMRES && o.method != HEC_BICGSTAB && o.method != HEC_CG)
            return fail(HEC_ERR_INVALID, "unknown method");
        if (!(tol >= 0.0) || maxit < 0)
            return fail(HEC_ERR_INVALID, "tol >= 0 and maxit >= 0 required");
        if (o.method == HEC_GMRES && (restart < 1 || restart > kMaxRestart))
            return fail(HEC_ERR_INVALID, "restart must be in 1..%d", kMaxRestart);
        if (o.method != HEC_GMRES)
            restart = 0;
        const bool mixed = (o.flags & HEC_MIXED_FP32) != 0;
        if (mixed && o.method != HEC_GMRES)
            return fail(HEC_ERR_INVALID, "HEC_MIXED_FP32 needs method HEC_GMRES");
        cudaStream_t s = (cudaStream_t)stream;
        if (mixed) {
            HEC_TRY(ensure_f32(A, s));
            if (M)
                HEC_TRY(ensure_precond_f32(M, s));
        }
        Solver *S = nullptr;
        HEC_TRY(make_solver(A, M, o.method, restart, mixed, s, S));
        const int n = S->n;
        const size_t vb = sizeof(double) * (size_t)n;
        // state header
        std::unique_ptr<SolverState> hp(new SolverState());
        SolverState &h = *hp;
        std::memset(&h, 0, offsetof(SolverState, H));
        h.tol = tol;
        h.maxit = maxit;
        h.restart = restart;
        h.method = o.method;
        h.flags = o.flags;
        h.h_while = S->h_while;
        h.h_if = S->h_if;
        const bool eager = (o.flags & HEC_SOLVE_EAGER) != 0;
        h.graph_mode = eager ? 0 : 1;
        // an FP32 inner cycle also ends once it has reduced its FP32 residual by
        // this factor: below it the FP32 arithmetic cannot be trusted, the FP64
        // refinement (next cycle start) takes over
        h.inner_rtol = mixed ? 1e-5 : 0.0;
        HEC_CK(cudaMemcpyAsync(S->st, &h, offsetof(SolverState, H), cudaMemcpyHostToDevice, s));
        int64_t h2d = 0, d2h = 0;
        const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
        HEC_CK(cudaMemcpyAsync(S->b, b, vb, bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        if (!bdev)
            h2d += vb;
        if (o.flags & HEC_X0_ZERO) {
            HEC_CK(cudaMemsetAsync(S->x, 0, vb, s));
        } else {
            HEC_CK(cudaMemcpyAsync(S->x, x, vb, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
            if (!xdev)
                h2d += vb;
        }
        if (eager)
            HEC_TRY(run_eager(A, M, *S, s));
        else
            HEC_CK(cudaGraphLaunch(S->exec, s));
        HEC_CK(cudaMemcpyAsync(x, S->x, vb, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        if (!xdev)
            d2h += vb;
        HEC_CK(cudaMemcpyAsync(&h, S->st, offsetof(SolverState, H), cudaMemcpyDeviceToHost, s));
        HEC_CK(cudaStreamSynchronize(s));
        int status = h.err ? h.err : h.status;
        if (info) {
            info->iters = h.iters;
            info->restarts = h.restarts;
            info->status = status;
            info->rel_resid = h.rel_resid;
            info->est_resid = h.est;
            info->kernel_launches = (int64_t)h.launches;
            info->h2d_bytes = h2d;
            info->d2h_bytes = d2h;
        }
        if (h.err)
            return fail(h.err, "a bounded device wait ran out during the solve");
        if (mixed && h.stagnated && !h.err) {
            // the FP32 cycles stopped refining: finish in FP64 from the current x
            hec_solve_opts_t o64 = o;
            o64.flags &= ~(HEC_MIXED_FP32 | HEC_X0_ZERO);
            hec_solve_info_t i64{};
            status = krylov_solve(A, M, b, x, tol, std::max(0, maxit - h.iters), restart, &o64, stream,
                                  &i64);
            if (info) {
                info->iters += i64.iters;
                info->restarts += i64.restarts;
                info->status = i64.status;
                info->rel_resid = i64.rel_resid;
                info->est_resid = i64.est_resid;
                info->kernel_launches += i64.kernel_launches;
                info->h2d_bytes += i64.h2d_bytes;
                info->d2h_bytes += i64.d2h_bytes;
                info->fp64_finish = 1;
            }
        }
        return status;
    });
}

} // extern "C"

// ====================================================================== apply without allocation
// The triangular-solve kernel needs scratch for the intermediate y = L^{-1} r
// (and, for blocks whose dependency window is too wide for shared memory, for
// z by position).  hec_precond_apply uses the scratch that level_schedule
// allocated in the handle; hec_precond_apply_noalloc uses this file-scope
// device array instead, so the call itself never allocates.  The array is
// part of the library image: every device that loads the library holds it
// until the process exits.
namespace {

constexpr long long kNoallocScratchDoubles = 1ll << 20; // 8 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so the
// address must come from cudaGetSymbolAddress with the device current.
int noalloc_scratch(double **out)
{
    int dev = 0;
    HEC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(HEC_ERR_INVALID, "device %d beyond the %d devices supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        HEC_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return HEC_OK;
}

} // namespace

extern "C" int hec_precond_apply_noalloc(hec_precond_t M, const double *r, double *z,
                                         int64_t spin_limit, void *stream)
{
    return abi_guard(__func__, [&]() -> int {
        if (!M || !r || !z || r == z)
            return fail(HEC_ERR_INVALID, "bad arguments");
        if (M->host_only)
            return fail(HEC_ERR_INVALID, "host-only preconditioner has no device data");
        if (!M->scheduled)
            return fail(HEC_ERR_INVALID, "level_schedule has not run");
        if (M->kind == kJacobi) // no scratch at all
            return run_jacobi(M, r, z, false, (cudaStream_t)stream);
        const TrsvPack &P = M->lay[0].pack;
        const long long need = (long long)P.ysz + (long long)P.zsz;
        if (need > kNoallocScratchDoubles)
            return fail(HEC_ERR_INVALID,
                        "preconditioner needs %lld scratch doubles; the static array of "
                        "hec_precond_apply_noalloc holds %lld (use hec_precond_apply)",
                        need, kNoallocScratchDoubles);
        double *scratch = nullptr;
        HEC_TRY(noalloc_scratch(&scratch));
        // y and z scratch are written before they are read inside one launch, so
        // nothing in the shared array has to start at zero.
        TrsvArgs a = trsv_args(M, M->lay[0], spin_limit ? spin_limit : kDefaultSpin);
        a.r = r;
        a.z = z;
        a.ysc = scratch;
        a.zsc = P.zsz ? scratch + P.ysz : nullptr;
        return run_trsv(a, (cudaStream_t)stream);
    });
}
