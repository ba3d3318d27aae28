// Internal helpers shared by the library's .cu files: status plumbing,
// device properties, launch sizing.  Not part of the public ABI.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

#include "orand.h"

namespace orand_impl {

// Last CUDA error seen on this host thread (reported by orand_last_cuda_error).
void set_last_cuda_error(cudaError_t e);

// Map a CUDA error to a status, remembering it for orand_last_cuda_error().
inline orand_status_t cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return ORAND_OK;
    set_last_cuda_error(e);
    return ORAND_ERR_CUDA;
}

// Status of the launch just issued (configuration errors only; the launch
// itself is asynchronous).
inline orand_status_t launch_status() { return cuda_status(cudaGetLastError()); }

// With ORAND_LOG=1 in the environment, failing CUDA calls made through
// ORAND_CUDA_TRY are reported on stderr with their call site.
bool log_enabled();
void log_cuda_failure(const char *what, const char *file, int line, cudaError_t e);

#define ORAND_CUDA_TRY(call)                                                            \
    do {                                                                                \
        cudaError_t orand_e_ = (call);                                                  \
        if (orand_e_ != cudaSuccess) {                                                  \
            ::orand_impl::log_cuda_failure(#call, __FILE__, __LINE__, orand_e_);        \
            return ::orand_impl::cuda_status(orand_e_);                                 \
        }                                                                               \
    } while (0)

// Allocation-failure injection for tests: while ORAND_FAIL_ALLOC=1 is set
// in the environment, every allocation the library would make (contexts,
// context scratch, the ragged batcher's state, tables and pinned staging)
// is refused before the allocator is called, and the call returns
// ORAND_ERR_ALLOC.  Read at each allocation (they are rare), so a test can
// switch it on and off inside one process.
bool alloc_blocked();

// NVTX ranges named after the C-ABI call, around each call that launches
// work, for profilers; off unless ORAND_NVTX=1 at the first call.
bool nvtx_enabled();
void nvtx_push(const char *name);
void nvtx_pop();
struct NvtxRange {
    bool on;
    explicit NvtxRange(const char *name) : on(nvtx_enabled())
    {
        if (on) nvtx_push(name);
    }
    ~NvtxRange()
    {
        if (on) nvtx_pop();
    }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define ORAND_NVTX_RANGE(name) ::orand_impl::NvtxRange orand_nvtx_range_(name)

struct DeviceInfo {
    int device;
    int sm_count;
    int cc_major, cc_minor;
    int max_threads_per_sm;
};

// Properties of the current device, cached per device ordinal.  Returns
// ORAND_ERR_UNSUPPORTED when the device is not compute capability 10.3,
// the only target this library is compiled for.
orand_status_t current_device(DeviceInfo *info);

// Overflow-checked helpers.
inline bool mul_overflows(uint64_t a, uint64_t b, uint64_t *out)
{
    if (a != 0 && b > UINT64_MAX / a) return true;
    *out = a * b;
    return false;
}

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Grid size for a grid-stride kernel: enough resident blocks to fill the
// GPU (sm_count * blocks_per_sm), never more than the work needs.
inline unsigned grid_for(uint64_t work_items, unsigned block, int sm_count, int blocks_per_sm)
{
    uint64_t need = ceil_div(work_items, block);
    uint64_t full = (uint64_t)sm_count * (uint64_t)blocks_per_sm;
    if (need > full) need = full;
    if (need == 0) need = 1;
    return (unsigned)need;
}

}  // namespace orand_impl
