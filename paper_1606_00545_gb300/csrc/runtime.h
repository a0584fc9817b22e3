// runtime.h -- host runtime shared by the library's translation units: error
// reporting, the pluggable device allocator, owned device buffers, and device
// queries.  Host C++ only; the definitions of the non-inline functions live in
// hec_lib.cu.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <exception>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/hecgpu.h"

namespace hec {

// Records a printf-style message for hec_last_error() and returns `code`.
int fail(int code, const char *fmt, ...);
// HEC_OK, or HEC_ERR_CUDA with the pending launch error recorded.
int check_launch(const char *what);

#define HEC_CK(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return ::hec::fail(HEC_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                               __FILE__, __LINE__);                                               \
    } while (0)

#define HEC_TRY(expr)                                                                             \
    do {                                                                                          \
        int r_ = (expr);                                                                          \
        if (r_ != HEC_OK)                                                                         \
            return r_;                                                                            \
    } while (0)

// Runs the body of a C ABI entry point.  A C++ exception (a host allocation
// that failed, a vector larger than it can be, a thread that could not start)
// becomes an error code and a message instead of crossing the ABI.
template <class F> int abi_guard(const char *where, F &&body) noexcept
{
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return fail(HEC_ERR_OOM, "%s: host memory exhausted", where);
    } catch (const std::exception &e) {
        return fail(HEC_ERR_INVALID, "%s: %s", where, e.what());
    } catch (...) {
        return fail(HEC_ERR_INVALID, "%s: unknown exception", where);
    }
}

// The allocator registered with hec_set_allocator (both null: cudaMalloc).
struct AllocFns {
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*free_)(void *, void *, void *) = nullptr;
    void *ctx = nullptr;
};
AllocFns current_allocator();
void set_allocator(const AllocFns &f);

// Keeps freed memory of the device's default stream-ordered pool cached
// instead of returning it at every synchronisation.
void keep_pool_memory();

// One device allocation, returned through the allocator that made it.  The
// default allocator is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// stream of the allocation), so a handle's allocations and frees never
// synchronise the device while other streams run; a handle must therefore be
// destroyed before the stream it was created on.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    AllocFns fns;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (!p)
            return;
        if (fns.free_)
            fns.free_(p, (void *)st, fns.ctx);
        else
            cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t nbytes, cudaStream_t s)
    {
        release();
        if (nbytes == 0)
            nbytes = 16;
        fns = current_allocator();
        st = s;
        if (fns.alloc) {
            p = fns.alloc(nbytes, (void *)s, fns.ctx);
            if (!p)
                return fail(HEC_ERR_OOM, "allocator returned NULL for %zu bytes", nbytes);
        } else {
            keep_pool_memory();
            cudaError_t e = cudaMallocAsync(&p, nbytes, s);
            if (e != cudaSuccess) {
                p = nullptr;
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? HEC_ERR_OOM : HEC_ERR_CUDA,
                            "cudaMallocAsync(%zu): %s", nbytes, cudaGetErrorString(e));
            }
        }
        bytes = nbytes;
        return HEC_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

template <class T> int upload(DevBuf &d, const std::vector<T> &h, cudaStream_t s)
{
    HEC_TRY(d.alloc(h.size() * sizeof(T), s));
    if (!h.empty())
        HEC_CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return HEC_OK;
}

int device_sms();
// Dynamic shared memory a CTA may opt in to.
int device_smem_optin();

inline int grid_for(int64_t items, int per_cta, int ctas_per_sm)
{
    int64_t need = (items + per_cta - 1) / per_cta;
    int64_t cap = (int64_t)device_sms() * ctas_per_sm;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

bool is_device_ptr(const void *p);
const char *last_error_text();

} // namespace hec
