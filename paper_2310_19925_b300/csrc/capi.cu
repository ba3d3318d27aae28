// Library-wide C ABI pieces: status strings, version, per-thread last CUDA
// error, cached device properties.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "ctx.cuh"

namespace orand_impl {

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

void set_last_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

bool log_enabled()
{
    static const bool on = [] {
        const char *v = getenv("ORAND_LOG");
        return v && v[0] && v[0] != '0';
    }();
    return on;
}

void log_cuda_failure(const char *what, const char *file, int line, cudaError_t e)
{
    if (log_enabled()) fprintf(stderr, "orand: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

bool alloc_blocked()
{
    const char *v = getenv("ORAND_FAIL_ALLOC");
    return v && v[0] == '1';
}

bool nvtx_enabled()
{
    static const bool on = [] {
        const char *v = getenv("ORAND_NVTX");
        return v && v[0] == '1';
    }();
    return on;
}

void nvtx_push(const char *name) { nvtxRangePushA(name); }
void nvtx_pop() { nvtxRangePop(); }

namespace {
constexpr int kMaxDevices = 64;
struct DeviceCache {
    std::once_flag once[kMaxDevices];
    DeviceInfo info[kMaxDevices];
    orand_status_t status[kMaxDevices];
};
DeviceCache &device_cache()
{
    static DeviceCache c;
    return c;
}
}  // namespace

orand_status_t current_device(DeviceInfo *info)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return ORAND_ERR_UNSUPPORTED;
    DeviceCache &c = device_cache();
    std::call_once(c.once[dev], [&]() {
        DeviceInfo d{};
        d.device = dev;
        orand_status_t st = ORAND_OK;
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) !=
                cudaSuccess) {
            set_last_cuda_error(cudaGetLastError());
            st = ORAND_ERR_CUDA;
        } else if (d.cc_major != 10 || d.cc_minor != 3) {
            st = ORAND_ERR_UNSUPPORTED;
        }
        c.info[dev] = d;
        c.status[dev] = st;
    });
    *info = c.info[dev];
    return c.status[dev];
}

orand_status_t ctx_check(orand_ctx_t ctx)
{
    if (ctx == nullptr) return ORAND_ERR_INVALID_ARG;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    return dev == ctx->device ? ORAND_OK : ORAND_ERR_INVALID_ARG;
}

orand_status_t ctx_scratch(orand_ctx_t ctx, size_t bytes, void **ptr)
{
    orand_status_t st = ctx_check(ctx);
    if (st != ORAND_OK) return st;
    if (bytes > ctx->scratch_bytes) {
        const size_t want = (bytes + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
        if (ctx->scratch) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_status(e);
            cudaFree(ctx->scratch);
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
        }
        void *p = nullptr;
        if (alloc_blocked()) return ORAND_ERR_ALLOC;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            set_last_cuda_error(cudaGetLastError());
            return ORAND_ERR_ALLOC;
        }
        ctx->scratch = p;
        ctx->scratch_bytes = want;
    }
    *ptr = ctx->scratch;
    return ORAND_OK;
}

void ragged_state_free(orand_ctx_t ctx);

}  // namespace orand_impl

extern "C" {

orand_status_t orand_ctx_create(orand_ctx_t *ctx)
{
    if (ctx == nullptr) return ORAND_ERR_INVALID_ARG;
    *ctx = nullptr;
    // The host object first, so an allocation failure is reported as such
    // whatever the device's state.
    orand_ctx_s *c = orand_impl::alloc_blocked() ? nullptr : new (std::nothrow) orand_ctx_s();
    if (c == nullptr) return ORAND_ERR_ALLOC;
    orand_impl::DeviceInfo info;
    orand_status_t st = orand_impl::current_device(&info);
    if (st != ORAND_OK) {
        delete c;
        return st;
    }
    c->device = info.device;
    *ctx = c;
    return ORAND_OK;
}

orand_status_t orand_ctx_destroy(orand_ctx_t ctx)
{
    if (ctx == nullptr) return ORAND_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    orand_impl::ragged_state_free(ctx);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (prev >= 0) cudaSetDevice(prev);
    delete ctx;
    return orand_impl::cuda_status(e);
}

const char *orand_status_string(orand_status_t status)
{
    switch (status) {
    case ORAND_OK: return "ORAND_OK";
    case ORAND_ERR_INVALID_ARG: return "ORAND_ERR_INVALID_ARG: null pointer, unknown enum or bad field";
    case ORAND_ERR_OVERFLOW: return "ORAND_ERR_OVERFLOW: size overflows, or a stream needs more than 2^32 words";
    case ORAND_ERR_ALIGNMENT: return "ORAND_ERR_ALIGNMENT: pointer or offset not aligned to its element size";
    case ORAND_ERR_ALLOC: return "ORAND_ERR_ALLOC: a library allocation (context, scratch, batch tables) failed";
    case ORAND_ERR_CUDA: return "ORAND_ERR_CUDA: CUDA runtime call or launch failed";
    case ORAND_ERR_DEVICE_TIMEOUT: return "ORAND_ERR_DEVICE_TIMEOUT: a device-side wait gave up";
    case ORAND_ERR_UNSUPPORTED: return "ORAND_ERR_UNSUPPORTED: device is not compute capability 10.3 (sm_103a)";
    case ORAND_ERR_SCRATCH_LIMIT:
        return "ORAND_ERR_SCRATCH_LIMIT: request exceeds the fixed scratch of the allocation-free entry point";
    }
    return "ORAND: unknown status";
}

int orand_version(void) { return 100; }

cudaError_t orand_last_cuda_error(void) { return orand_impl::g_last_cuda_error; }

}  // extern "C"
