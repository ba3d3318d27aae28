// cuRAND comparison for the fused 2D walk (the same workload as
// orand_brownian_walk), through cuRAND's device API with its Philox
// generator, as the paper's comparison system uses it (Fig. 2):
//
//   walk2d_curand_setup_kernel  curand_init(seed, particle, 0) per particle,
//                               then the start position from two uniforms;
//                               the state goes to HBM.
//   walk2d_curand_step_kernel   Fig. 2's pattern: one launch per step; the
//                               state and the position are loaded from and
//                               stored to HBM every step.
//   walk2d_curand_fused_kernel  cuRAND at its best: one launch, the state in
//                               registers for the whole walk, the same
//                               block-compensated sums as walk2d_kernel.
//
// Only the generator differs from the library's walk, so the timings
// compare stateless counter-based draws with cuRAND's stateful ones.
#include <curand_kernel.h>

#include "common.cuh"

namespace orand_impl {

constexpr int kCurandWalkBlock = 128;
constexpr uint32_t kCurandSumBlock = 16;

__device__ __forceinline__ void kahan_add_cw(float &x, float &c, float inc)
{
    const float y = inc - c;
    const float t = x + y;
    c = (t - x) - y;
    x = t;
}

__global__ void __launch_bounds__(kCurandWalkBlock) walk2d_curand_setup_kernel(uint64_t n, uint64_t p_first,
                                                                              uint64_t seed,
                                                                              curandStatePhilox4_32_10_t *states,
                                                                              float2 *__restrict__ pos)
{
    const uint64_t i = (uint64_t)blockIdx.x * kCurandWalkBlock + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, p_first + i, 0, &st);
    const float x = curand_uniform(&st), y = curand_uniform(&st);
    states[i] = st;
    pos[i] = make_float2(x, y);
}

__global__ void __launch_bounds__(kCurandWalkBlock) walk2d_curand_step_kernel(uint64_t n, float s,
                                                                             curandStatePhilox4_32_10_t *states,
                                                                             float2 *__restrict__ pos)
{
    const uint64_t i = (uint64_t)blockIdx.x * kCurandWalkBlock + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st = states[i];
    const float2 z = curand_normal2(&st);
    float2 p = pos[i];
    p.x = fmaf(s, z.x, p.x);
    p.y = fmaf(s, z.y, p.y);
    pos[i] = p;
    states[i] = st;
}

__global__ void __launch_bounds__(kCurandWalkBlock, 1) walk2d_curand_fused_kernel(uint64_t n, uint64_t p_first,
                                                                              uint64_t seed, uint32_t steps, float s,
                                                                              float2 *__restrict__ pos)
{
    const uint64_t i = (uint64_t)blockIdx.x * kCurandWalkBlock + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, p_first + i, 0, &st);
    float x = curand_uniform(&st), y = curand_uniform(&st), cx = 0.f, cy = 0.f;
    for (uint32_t done = 0; done < steps;) {
        const uint32_t len = min(kCurandSumBlock, steps - done);
        float sx = 0.f, sy = 0.f;
        auto step = [&]() {
            const float2 z = curand_normal2(&st);
            sx = fmaf(s, z.x, sx);
            sy = fmaf(s, z.y, sy);
        };
        if (len == kCurandSumBlock) {
            // The same full-block unrolling and launch bounds as walk2d_kernel.
#pragma unroll 4
            for (uint32_t k = 0; k < kCurandSumBlock; ++k) step();
        } else {
            for (uint32_t k = 0; k < len; ++k) step();
        }
        kahan_add_cw(x, cx, sx);
        kahan_add_cw(y, cy, sy);
        done += len;
    }
    pos[i] = make_float2(x, y);
}

static orand_status_t walk2d_curand_args(const orand_walk2d_t *p, const void *pos, unsigned *grid, float *s)
{
    if (p == nullptr) return ORAND_ERR_INVALID_ARG;
    if (!(p->dt >= 0.0f) || !(p->D >= 0.0f) || !isfinite(p->dt) || !isfinite(p->D)) return ORAND_ERR_INVALID_ARG;
    if (p->p_first + p->n_particles < p->p_first) return ORAND_ERR_OVERFLOW;
    if (p->steps == UINT32_MAX) return ORAND_ERR_OVERFLOW;
    const uint64_t g = ceil_div(p->n_particles, kCurandWalkBlock);
    if (g > 0x7FFFFFFFull) return ORAND_ERR_OVERFLOW;
    if (p->n_particles && pos == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)pos % 8) return ORAND_ERR_ALIGNMENT;
    *grid = (unsigned)g;
    *s = (float)sqrt(2.0 * (double)p->D * (double)p->dt);
    return ORAND_OK;
}

}  // namespace orand_impl

using namespace orand_impl;

extern "C" {

size_t orand_walk2d_curand_state_bytes(void) { return sizeof(curandStatePhilox4_32_10_t); }

orand_status_t orand_walk2d_curand_setup(const orand_walk2d_t *p, void *states, float *pos_out, uint64_t curand_seed,
                                         cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk2d_curand_setup");
    unsigned grid;
    float s;
    orand_status_t st = walk2d_curand_args(p, pos_out, &grid, &s);
    if (st != ORAND_OK || p->n_particles == 0) return st;
    if (states == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)states % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    walk2d_curand_setup_kernel<<<grid, kCurandWalkBlock, 0, stream>>>(
        p->n_particles, p->p_first, curand_seed, (curandStatePhilox4_32_10_t *)states, (float2 *)pos_out);
    return launch_status();
}

orand_status_t orand_walk2d_curand_run(const orand_walk2d_t *p, void *states, float *pos, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk2d_curand_run");
    unsigned grid;
    float s;
    orand_status_t st = walk2d_curand_args(p, pos, &grid, &s);
    if (st != ORAND_OK || p->n_particles == 0) return st;
    if (states == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)states % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    // Fig. 2's host loop: one launch per step.
    for (uint32_t t = 0; t < p->steps; ++t)
        walk2d_curand_step_kernel<<<grid, kCurandWalkBlock, 0, stream>>>(
            p->n_particles, s, (curandStatePhilox4_32_10_t *)states, (float2 *)pos);
    return launch_status();
}

orand_status_t orand_walk2d_curand_fused(const orand_walk2d_t *p, float *pos_out, uint64_t curand_seed,
                                         cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk2d_curand_fused");
    unsigned grid;
    float s;
    orand_status_t st = walk2d_curand_args(p, pos_out, &grid, &s);
    if (st != ORAND_OK || p->n_particles == 0) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    walk2d_curand_fused_kernel<<<grid, kCurandWalkBlock, 0, stream>>>(p->n_particles, p->p_first, curand_seed,
                                                                     p->steps, s, (float2 *)pos_out);
    return launch_status();
}

}  // extern "C"
