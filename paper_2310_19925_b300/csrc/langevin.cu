// The paper's Brownian-dynamics macro-benchmark (Fig. 1 and §5): 2D particles
// with velocity drag and a uniform FP64 random kick per step, on B300.
//
// Three forms of the same simulation:
//   * langevin_step_kernel: the paper's OpenRAND pattern (Fig. 1).  One launch
//     per step; the particle struct is read and written in global memory
//     every step; the generator is constructed in-thread from (pid, iter)
//     with no stored state.
//   * langevin_fused_kernel: this library's design.  All steps in one launch,
//     with position, velocity and round keys in registers.  It gives the same
//     bits as the per-step form.
//   * langevin_curand_*: the paper's cuRAND pattern (Fig. 2).  A Philox state
//     per particle is set up by curand_init(1984, i, 0), then loaded and
//     stored every step.  This is the comparison system of §5.
// The FP64 updates use explicit round-to-nearest operations in the paper's
// order (no fused multiply-add), so the per-step and fused kernels match the
// plain-C oracle bit for bit.
#include <curand_kernel.h>

#include "common.cuh"
#include "orand_device.cuh"

namespace orand_impl {

constexpr int kLangevinBlock = 256;

struct LangevinArgs {
    uint64_t n, p_first, seed;
    double dt, g_over_m, sqrt_dt;
};

// draw_double2 of Fig. 1: the two FP64 uniforms of one Philox block (words
// 0-1 and 2-3, first word high, as in Fig. 3).
__device__ __forceinline__ double2 draw_double2(const orand::PhiloxKeys &keys, uint32_t counter)
{
    const uint4 w = keys.block(0u, counter);
    return make_double2(orand::u01_f64(w.x, w.y), orand::u01_f64(w.z, w.w));
}

// 2r - 1 for the FP64 uniform r = u01_f64(hi, lo), built from integer bits.
// With m = (hi:lo) >> 11 (53 bits), r = m 2^-53 and 2r - 1 = (m - 2^52) 2^-52,
// which is exactly representable; Fig. 1's (r * 2 - 1) rounds to the same
// value (both of its steps are exact), so this costs no FP64 operation and
// changes no bit.
__device__ __forceinline__ double u11_f64(uint32_t hi, uint32_t lo)
{
    const uint64_t m = (((uint64_t)hi << 32) | lo) >> 11;
    const bool pos = (m >> 52) != 0;
    const uint64_t a = pos ? (m & ((1ull << 52) - 1)) : (1ull << 52) - m;  // |m - 2^52| <= 2^52
    if (a == 0) return 0.0;                                                 // 1.0 - 1.0 = +0
    const int lz = __clzll((long long)a);                                   // 11..63
    const uint64_t mant = (a << (lz - 11)) & ((1ull << 52) - 1);            // leading bit dropped
    const uint64_t bits = ((uint64_t)!pos << 63) | ((uint64_t)(1034 - lz) << 52) | mant;  // 2^(11 - lz)
    return __longlong_as_double((long long)bits);
}

// One step of Fig. 1 (drag, kick, then the position update) with the kicks'
// 2r - 1 taken from the block's words by u11_f64: 14 FP64 operations instead
// of Fig. 1's 18, the same bits.  The FP64 pipe
// bounds this simulation on B300, so the fused kernel uses this form; the
// per-step kernel keeps Fig. 1's arithmetic.
__device__ __forceinline__ void langevin_update_words(const LangevinArgs &a, uint4 w, double &x, double &y,
                                                      double &vx, double &vy)
{
    vx = __dsub_rn(vx, __dmul_rn(__dmul_rn(a.g_over_m, vx), a.dt));
    vy = __dsub_rn(vy, __dmul_rn(__dmul_rn(a.g_over_m, vy), a.dt));
    vx = __dadd_rn(vx, __dmul_rn(u11_f64(w.x, w.y), a.sqrt_dt));
    vy = __dadd_rn(vy, __dmul_rn(u11_f64(w.z, w.w), a.sqrt_dt));
    x = __dadd_rn(x, __dmul_rn(vx, a.dt));
    y = __dadd_rn(y, __dmul_rn(vy, a.dt));
}

__global__ void __launch_bounds__(kLangevinBlock) langevin_init_kernel(LangevinArgs a,
                                                                      orand_particle_t *__restrict__ ps)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t pid = a.p_first + i;
    const orand::PhiloxKeys keys(a.seed ^ pid);
    const double2 r = draw_double2(keys, 0u);
    orand_particle_t p;
    p.x = r.x;
    p.y = r.y;
    p.vx = 0.0;
    p.vy = 0.0;
    p.pid = pid;
    ps[i] = p;
}

__global__ void __launch_bounds__(kLangevinBlock) langevin_step_kernel(LangevinArgs a,
                                                                      orand_particle_t *__restrict__ ps,
                                                                      uint32_t counter)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    orand_particle_t p = ps[i];
    const orand::PhiloxKeys keys(a.seed ^ p.pid);
    // Fig. 1 order: drag first, then the draw and the kick.
    p.vx = __dsub_rn(p.vx, __dmul_rn(__dmul_rn(a.g_over_m, p.vx), a.dt));
    p.vy = __dsub_rn(p.vy, __dmul_rn(__dmul_rn(a.g_over_m, p.vy), a.dt));
    const double2 r = draw_double2(keys, counter);
    p.vx = __dadd_rn(p.vx, __dmul_rn(__dsub_rn(__dmul_rn(r.x, 2.0), 1.0), a.sqrt_dt));
    p.vy = __dadd_rn(p.vy, __dmul_rn(__dsub_rn(__dmul_rn(r.y, 2.0), 1.0), a.sqrt_dt));
    p.x = __dadd_rn(p.x, __dmul_rn(p.vx, a.dt));
    p.y = __dadd_rn(p.y, __dmul_rn(p.vy, a.dt));
    ps[i] = p;
}

__global__ void __launch_bounds__(kLangevinBlock) langevin_fused_kernel(LangevinArgs a,
                                                                       orand_particle_t *__restrict__ ps,
                                                                       uint32_t first_counter, uint32_t steps)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    orand_particle_t p = ps[i];
    const orand::PhiloxKeys keys(a.seed ^ p.pid);
    double x = p.x, y = p.y, vx = p.vx, vy = p.vy;
    for (uint32_t k = 0; k < steps; ++k) langevin_update_words(a, keys.block(0u, first_counter + k), x, y, vx, vy);
    p.x = x;
    p.y = y;
    p.vx = vx;
    p.vy = vy;
    ps[i] = p;
}

// ------------------------------------------------- cuRAND pattern (Fig. 2)

__global__ void __launch_bounds__(kLangevinBlock) curand_setup_kernel(LangevinArgs a, uint64_t curand_seed,
                                                                     curandStatePhilox4_32_10_t *states)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    curand_init(curand_seed, a.p_first + i, 0, &states[i]);
}

__global__ void __launch_bounds__(kLangevinBlock) curand_init_particles_kernel(LangevinArgs a,
                                                                              orand_particle_t *__restrict__ ps,
                                                                              curandStatePhilox4_32_10_t *states)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    curandStatePhilox4_32_10_t st = states[i];
    const double2 r = curand_uniform2_double(&st);
    orand_particle_t p;
    p.x = r.x;
    p.y = r.y;
    p.vx = 0.0;
    p.vy = 0.0;
    p.pid = a.p_first + i;
    states[i] = st;
    ps[i] = p;
}

__global__ void __launch_bounds__(kLangevinBlock) curand_step_kernel(LangevinArgs a, orand_particle_t *__restrict__ ps,
                                                                    curandStatePhilox4_32_10_t *states)
{
    const uint64_t i = (uint64_t)blockIdx.x * kLangevinBlock + threadIdx.x;
    if (i >= a.n) return;
    orand_particle_t p = ps[i];
    p.vx = __dsub_rn(p.vx, __dmul_rn(__dmul_rn(a.g_over_m, p.vx), a.dt));
    p.vy = __dsub_rn(p.vy, __dmul_rn(__dmul_rn(a.g_over_m, p.vy), a.dt));
    curandStatePhilox4_32_10_t st = states[i];
    const double2 r = curand_uniform2_double(&st);
    p.vx = __dadd_rn(p.vx, __dmul_rn(__dsub_rn(__dmul_rn(r.x, 2.0), 1.0), a.sqrt_dt));
    p.vy = __dadd_rn(p.vy, __dmul_rn(__dsub_rn(__dmul_rn(r.y, 2.0), 1.0), a.sqrt_dt));
    p.x = __dadd_rn(p.x, __dmul_rn(p.vx, a.dt));
    p.y = __dadd_rn(p.y, __dmul_rn(p.vy, a.dt));
    states[i] = st;
    ps[i] = p;
}

// ------------------------------------------------------------------ host

static orand_status_t langevin_args(const orand_langevin2d_t *p, LangevinArgs *a)
{
    if (p == nullptr) return ORAND_ERR_INVALID_ARG;
    if (!(p->dt >= 0.0) || !(p->mass > 0.0) || !(p->gamma >= 0.0) || p->dt > 1e300 || p->gamma > 1e300)
        return ORAND_ERR_INVALID_ARG;
    if (p->p_first + p->n_particles < p->p_first) return ORAND_ERR_OVERFLOW;
    if (ceil_div(p->n_particles, kLangevinBlock) > 0x7FFFFFFFull) return ORAND_ERR_OVERFLOW;
    a->n = p->n_particles;
    a->p_first = p->p_first;
    a->seed = p->seed;
    a->dt = p->dt;
    a->g_over_m = p->gamma / p->mass;
    a->sqrt_dt = sqrt(p->dt);
    return ORAND_OK;
}

static orand_status_t check_particles(const void *ps)
{
    if (ps == nullptr) return ORAND_ERR_INVALID_ARG;
    return ((uintptr_t)ps % 8) ? ORAND_ERR_ALIGNMENT : ORAND_OK;
}

static unsigned lgrid(uint64_t n) { return (unsigned)ceil_div(n, kLangevinBlock); }

}  // namespace orand_impl

using namespace orand_impl;

extern "C" {

orand_status_t orand_langevin2d_init(const orand_langevin2d_t *p, orand_particle_t *particles, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_init");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    langevin_init_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles);
    return launch_status();
}

orand_status_t orand_langevin2d_step(const orand_langevin2d_t *p, orand_particle_t *particles, uint32_t counter,
                                     cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_step");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    langevin_step_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles, counter);
    return launch_status();
}

orand_status_t orand_langevin2d_fused(const orand_langevin2d_t *p, orand_particle_t *particles,
                                      uint32_t first_counter, uint32_t steps, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_fused");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    if ((uint64_t)first_counter + steps > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    langevin_fused_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles, first_counter, steps);
    return launch_status();
}

orand_status_t orand_langevin2d_run_per_step(const orand_langevin2d_t *p, orand_particle_t *particles,
                                             uint32_t first_counter, uint32_t steps, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_run_per_step");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    if ((uint64_t)first_counter + steps > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    // The paper's host loop (Fig. 1): one launch per step.
    for (uint32_t k = 0; k < steps; ++k)
        langevin_step_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles, first_counter + k);
    return launch_status();
}

size_t orand_langevin2d_curand_state_bytes(void) { return sizeof(curandStatePhilox4_32_10_t); }

orand_status_t orand_langevin2d_curand_setup(const orand_langevin2d_t *p, orand_particle_t *particles, void *states,
                                             uint64_t curand_seed, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_curand_setup");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    if (states == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)states % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    curandStatePhilox4_32_10_t *s = (curandStatePhilox4_32_10_t *)states;
    curand_setup_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, curand_seed, s);
    curand_init_particles_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles, s);
    return launch_status();
}

orand_status_t orand_langevin2d_curand_step(const orand_langevin2d_t *p, orand_particle_t *particles, void *states,
                                            cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_curand_step");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    if (states == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)states % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    curand_step_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles,
                                                                   (curandStatePhilox4_32_10_t *)states);
    return launch_status();
}

}  // extern "C"

extern "C" orand_status_t orand_langevin2d_curand_run(const orand_langevin2d_t *p, orand_particle_t *particles,
                                                      void *states, uint32_t steps, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_langevin2d_curand_run");
    LangevinArgs a;
    orand_status_t st = langevin_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_particles(particles)) != ORAND_OK) return st;
    if (states == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)states % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    // The paper's cuRAND host loop (Fig. 2): one launch per step.
    for (uint32_t k = 0; k < steps; ++k)
        curand_step_kernel<<<lgrid(a.n), kLangevinBlock, 0, stream>>>(a, particles,
                                                                       (curandStatePhilox4_32_10_t *)states);
    return launch_status();
}
