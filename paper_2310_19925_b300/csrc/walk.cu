// Brownian-walk kernels: the fused 2D walk (the paper's macro-benchmark,
// Fig. 1 and §5, pure-diffusion FP32 form), the differentiable 3D drift walk
// (forward with checkpoints, noise-regenerating adjoint) and the plain
// noise-storing one-launch-per-step baseline of the same 3D walk.
//
// Fused kernels keep each particle's position and its Philox round keys in
// registers for the whole walk.  A step is one Philox block, keyed by the
// particle id with counter (0, t, 0, 0), followed by Box-Muller in FP32 and
// a compensated position update.  Only the start and end touch HBM.  The cost is
// integer- and FP-pipe work per step, not bytes.
#include <math.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ctx.cuh"
#include "orand_device.cuh"

namespace orand_impl {

constexpr int kWalkBlock = 256;
constexpr int kRedWidth = 5;  // FP64 partial sums per block: loss, or (dmu0..2, dsigma, dkappa)

// Kahan-compensated x += inc.
__device__ __forceinline__ void kahan_add(float &x, float &c, float inc)
{
    const float y = inc - c;
    const float t = x + y;
    c = (t - x) - y;
    x = t;
}

// Deterministic block sum of `W` doubles per thread into partials[blockIdx.x * W + j].
template <int W>
__device__ __forceinline__ void block_reduce_store(double (&v)[W], double *partials)
{
    __shared__ double red[kWalkBlock / 32][W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        double x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) red[warp][j] = x;
    }
    __syncthreads();
    if (threadIdx.x < W) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWalkBlock / 32; ++w) s += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * W + threadIdx.x] = s;
    }
}

// Sum the `n` per-block partials of each of W columns in a fixed order,
// scale by `scale` (and by *gscale if given) and write out[0..W).
template <int W>
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double *__restrict__ partials, uint32_t n,
                                                              double scale, const double *__restrict__ gscale,
                                                              double *__restrict__ out, int n_out)
{
    __shared__ double sh[256];
    for (int j = 0; j < n_out; ++j) {
        double s = 0.0;
        for (uint32_t i = threadIdx.x; i < n; i += 256) s += partials[(size_t)i * W + j];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[j] = sh[0] * scale * (gscale ? *gscale : 1.0);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 2D walk

// The 2D kernel is bound by instruction issue (58 instructions per
// particle-step, nearly all of them the Philox rounds and Box-Muller).  One
// particle per thread; the position sum is compensated per block of
// kSumBlock steps (plain FMA sums inside a block, a Kahan add of each block
// sum), which saves the per-step compensation while keeping the rounding
// error of the whole walk at the level of one FP32 rounding per block sum.
// A full block takes its steps in pairs: the two steps' Philox blocks are
// independent chains, and the FP32 parts of their Box-Muller maps and sums
// run as packed pairs (one f32x2 instruction for both steps; each lane is
// rounded as the scalar operation, so every normal has the same bits; only
// the block sum is split into an even-step and an odd-step half).  The loop
// over the 16 pairs is unrolled by 2, and with the launch bound of one block
// per SM ptxas keeps the round keys in registers (72 registers).  Measured on
// B300 (full walk, 2^24 x 10^4, 16-step blocks): 425.5 ms against 433.8 with
// scalar steps unrolled by 4; pairs unrolled by 1 or 4 took 436.3 and 427.3
// ms.  Earlier, with scalar steps: two particles per thread 437.9 ms, three
// or four slower still, and launch bounds that fit 32 or 40 warps per SM
// 436.6-446.1 ms.  With the half-turn angle split: 404.3 ms; the map's
// packed constants read from constant memory (below) 400.1 ms; and block
// sums of 32 steps instead of 16 (half the Kahan adds and loop control per
// step; each half of a block sum then adds 16 terms instead of 8) 396.3 ms.
constexpr int kWalk2dBlock = 256;
// Steps per block sum, every walk.  3D (2^22 x 4096, forward + adjoint):
// 116.5 ms with 16-step blocks, 115.4 with 32 (OU 133.2 and 132.6).
constexpr uint32_t kSumBlock = 32;

// The walks' map's FP32 constants as packed pairs (both lanes the same).
// The 2D kernel reads them from constant memory once, before its step loop;
// written as immediates, ptxas re-creates some of them inside the loop
// (ncu, 2^20 x 1000: 60.2 against 59.1 instructions per particle-step).
// The 3D kernels measured slower that way (117.1 against 116.6 ms) and keep
// the immediates.
struct WalkMapConsts {
    unsigned long long u1_scale, minus_one, one, c3, c4, c5, c6, two, log_scale, angle_scale;
};
__device__ __forceinline__ WalkMapConsts walk_map_consts_imm()
{
    using namespace orand::x2;
    return {splat(0x1p-24f), splat(-1.0f), splat(1.0f), splat(2.0f / 6.0f), splat(0.4f), splat(0.5f),
            splat(2.0f / 3.0f), splat(2.0f), splat(-1.3862943611198906f), splat(0x1p-31f * 3.14159265358979324f)};
}
static __constant__ float2 kWalkMapConsts[10] = {
    {0x1p-24f, 0x1p-24f}, {-1.0f, -1.0f}, {1.0f, 1.0f}, {2.0f / 6.0f, 2.0f / 6.0f}, {0.4f, 0.4f}, {0.5f, 0.5f},
    {2.0f / 3.0f, 2.0f / 3.0f}, {2.0f, 2.0f}, {-1.3862943611198906f, -1.3862943611198906f},
    {0x1p-31f * 3.14159265358979324f, 0x1p-31f * 3.14159265358979324f}};
__device__ __forceinline__ WalkMapConsts walk_map_consts_loaded()
{
    const unsigned long long *p = reinterpret_cast<const unsigned long long *>(kWalkMapConsts);
    return {p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8], p[9]};
}

// The walks' Box-Muller map (bm_radius_walk, bm_cos_sin_walk) for two
// pairs at once, (radius word, angle word) = (u_a, t_a) in lane 0 and
// (u_b, t_b) in lane 1, with its FP32 arithmetic on packed pairs (each lane
// rounded as the scalar map, so the same bits): the radii as a packed pair,
// each carrying its angle's half-turn sign, and each angle's cosine and sine
// at phi in [0, pi).  radius * cosine and radius * sine are then the
// products of bm_radius_walk and bm_cos_sin_walk bit for bit (a sign flip is
// exact).
__device__ __forceinline__ unsigned long long walk_map_x2(uint32_t u_a, uint32_t t_a, uint32_t u_b, uint32_t t_b,
                                                          float &ca, float &sa, float &cb, float &sb,
                                                          const WalkMapConsts &k = walk_map_consts_imm())
{
    using namespace orand::x2;
    const unsigned long long u1 = mul(pack(__uint2float_rn((u_a >> 8) + 1u), __uint2float_rn((u_b >> 8) + 1u)),
                                      k.u1_scale);
    const unsigned long long v = fma(u1, k.minus_one, k.one);                   /* 1 - u1 */
    unsigned long long p2 = fma(v, k.c3, k.c4);
    p2 = fma(p2, v, k.c5);
    p2 = fma(p2, v, k.c6);
    p2 = fma(p2, v, k.one);
    p2 = fma(p2, v, k.two);
    const float2 x_series = unpack(mul(v, p2));
    const float2 uu = unpack(u1);
    const float2 x_log = unpack(mul(k.log_scale, pack(orand::sfu_lg2(uu.x), orand::sfu_lg2(uu.y))));
    const float2 vv = unpack(v);
    const float xa = vv.x < 0.0625f ? x_series.x : x_log.x, xb = vv.y < 0.0625f ? x_series.y : x_log.y;
    const float2 ph = unpack(mul(pack((float)(t_a & 0x7FFFFF00u), (float)(t_b & 0x7FFFFF00u)), k.angle_scale));
    ca = orand::sfu_cos(ph.x);
    sa = orand::sfu_sin(ph.x);
    cb = orand::sfu_cos(ph.y);
    sb = orand::sfu_sin(ph.y);
    // The half-turn sign (bit 31 of the angle word) on the radius: the same
    // products as bm_cos_sin_walk's signed cosine and sine, one xor per pair.
    return pack(__uint_as_float(__float_as_uint(orand::sfu_sqrt(xa)) ^ (t_a & 0x80000000u)),
                __uint_as_float(__float_as_uint(orand::sfu_sqrt(xb)) ^ (t_b & 0x80000000u)));
}

// Steps t (lane 0) and t + 1 (lane 1) of a 2D walk from their Philox blocks
// wa, wb, accumulated into the packed block sums.
__device__ __forceinline__ void walk2d_step_pair(uint4 wa, uint4 wb, unsigned long long &sxx,
                                                 unsigned long long &syy, const WalkMapConsts &k)
{
    using namespace orand::x2;
    float ca, sa, cb, sb;
    const unsigned long long r = walk_map_x2(wa.x, wa.y, wb.x, wb.y, ca, sa, cb, sb, k);
    sxx = fma(r, pack(ca, cb), sxx);
    syy = fma(r, pack(sa, sb), syy);
}

__global__ void __launch_bounds__(kWalk2dBlock, 1) walk2d_kernel(uint64_t n, uint64_t p_first, uint64_t seed,
                                                                uint32_t steps, float s, float2 *__restrict__ out)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalk2dBlock + threadIdx.x;
    if (i >= n) return;
    const orand::PhiloxKeys keys(seed ^ (p_first + i));
    const WalkMapConsts mk = walk_map_consts_loaded();
    const uint4 w0 = keys.block(0u, 0u);
    float x = orand::u01_f32(w0.x), y = orand::u01_f32(w0.y), cx = 0.f, cy = 0.f;
    // t runs 1..steps in blocks of kSumBlock; `done` counts steps taken so
    // the loop cannot wrap when steps is near 2^32.
    for (uint32_t done = 0; done < steps;) {
        const uint32_t len = min(kSumBlock, steps - done);
        float sx = 0.f, sy = 0.f;
        if (len == kSumBlock) {
            unsigned long long sxx = orand::x2::splat(0.0f), syy = orand::x2::splat(0.0f);
#pragma unroll 2
            for (uint32_t k = 1; k <= kSumBlock; k += 2)
                walk2d_step_pair(keys.block(0u, done + k), keys.block(0u, done + k + 1), sxx, syy, mk);
            const float2 a = orand::x2::unpack(sxx), b = orand::x2::unpack(syy);
            sx = a.x + a.y;
            sy = b.x + b.y;
        } else {
            for (uint32_t k = 1; k <= len; ++k) {
                // (r cos, r sin); the block sum is scaled by s once, at the flush.
                const uint4 w = keys.block(0u, done + k);
                const float r = orand::bm_radius_walk(w.x);
                float c, sn;
                orand::bm_cos_sin_walk(w.y, &c, &sn);
                sx = fmaf(r, c, sx);
                sy = fmaf(r, sn, sy);
            }
        }
        kahan_add(x, cx, s * sx);
        kahan_add(y, cy, s * sy);
        done += len;
    }
    out[i] = make_float2(x, y);
}

// ------------------------------------------------------------------ 3D walk

struct Walk3dArgs {
    uint64_t n, p_first, seed;
    uint32_t steps, K;
    float mu_dt[3];     // fl32(mu_c * dt)
    float sig_sqdt;     // fl32(sigma * sqrt(dt))
    float kappa_dt;     // fl32(kappa * dt)
    float decay_f;      // fl32(1 - kappa dt): lambda_t = lambda_{t+1} * decay
    float inv_decay_f;  // fl32(1 / (1 - kappa dt)): reverse-time position recompute
    double k_over_p;    // k / p_total
    double t_dt;        // steps * dt (FP64, exact product of the FP32 dt)
    double sqdt;        // sqrt(dt) in FP64
    double dt;          // dt in FP64
    double decay_K;     // (1 - kappa dt)^K: lambda across one full checkpoint segment
    double decay_last;  // (1 - kappa dt)^(steps - (nseg - 1) K): the last, possibly short, segment
};

// z_t: the pair (w.x, w.y) gives z0 = r cos, z1 = r sin, the pair (w.z, w.w)
// the cosine z2 = r' cos'; both pairs' maps run on packed FP32 pairs.
__device__ __forceinline__ void walk3d_normals(const orand::PhiloxKeys &keys, uint32_t t_counter, float z[3])
{
    const uint4 w = keys.block(0u, t_counter);
    float ca, sa, cb, sb;
    const unsigned long long r = walk_map_x2(w.x, w.y, w.z, w.w, ca, sa, cb, sb);
    const float2 zz = orand::x2::unpack(orand::x2::mul(r, orand::x2::pack(ca, cb)));
    z[0] = zz.x;
    z[1] = orand::x2::unpack(r).x * sa;
    z[2] = zz.y;
}

// sigma sqrt(dt) * (z0, z1, z2) with the scale folded into the two radii.
__device__ __forceinline__ void walk3d_scaled_normals(const orand::PhiloxKeys &keys, uint32_t t_counter,
                                                      float scale, float z[3])
{
    const uint4 w = keys.block(0u, t_counter);
    float ca, sa, cb, sb;
    const unsigned long long r =
        orand::x2::mul(orand::x2::splat(scale), walk_map_x2(w.x, w.y, w.z, w.w, ca, sa, cb, sb));
    const float2 zz = orand::x2::unpack(orand::x2::mul(r, orand::x2::pack(ca, cb)));
    z[0] = zz.x;
    z[1] = orand::x2::unpack(r).x * sa;
    z[2] = zz.y;
}

__device__ __forceinline__ void walk3d_x0(const orand::PhiloxKeys &keys, float x[3])
{
    const uint4 w = keys.block(0u, 0u);
    x[0] = 2.0f * orand::u01_f32(w.x) - 1.0f;
    x[1] = 2.0f * orand::u01_f32(w.y) - 1.0f;
    x[2] = 2.0f * orand::u01_f32(w.z) - 1.0f;
}

__global__ void __launch_bounds__(kWalkBlock) walk3d_init_kernel(Walk3dArgs a, float *__restrict__ x0)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    if (i >= a.n) return;
    const orand::PhiloxKeys keys(a.seed ^ (a.p_first + i));
    float x[3];
    walk3d_x0(keys, x);
    x0[3 * i] = x[0];
    x0[3 * i + 1] = x[1];
    x0[3 * i + 2] = x[2];
}

// Forward walk.  Increments are summed in FP32 over blocks of at most
// kSumBlock steps (a block also ends at each checkpoint) and each block sum
// is Kahan-added to the position, as in the 2D kernel.  OU: the drift
// mu - kappa x is evaluated at the current position x + s (s the block's
// partial sum); without it the constant drift mu dt is added once per block.
// Launch bounds (measured on B300, forward + adjoint of 2^22 x 4096, with
// the walks' earlier map): one block per SM for the constant drift (86 and
// 83 registers, 142.4 ms; three blocks: 143.7 ms), three for OU (78 and 80
// registers, 158.3 ms; one block: 159.9 ms).
template <bool OU>
__global__ void __launch_bounds__(kWalkBlock, OU ? 3 : 1) walk3d_fwd_kernel(Walk3dArgs a, const float *__restrict__ x0_in,
                                                               float *__restrict__ xT, float *__restrict__ ckpt,
                                                               double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double loss[kRedWidth] = {};
    if (i < a.n) {
        const orand::PhiloxKeys keys(a.seed ^ (a.p_first + i));
        float x[3], c[3] = {0.f, 0.f, 0.f};
        if (x0_in) {
            x[0] = x0_in[3 * i];
            x[1] = x0_in[3 * i + 1];
            x[2] = x0_in[3 * i + 2];
        } else {
            walk3d_x0(keys, x);
        }
        const bool want_ck = ckpt != nullptr && a.K != 0;  // every block must advance t
        uint32_t next_ck = 0, j = 0;
        for (uint32_t t = 0; t < a.steps;) {
            if (want_ck && t == next_ck) {
                float *dst = ckpt + ((size_t)j * a.n + i) * 3;
                dst[0] = x[0];
                dst[1] = x[1];
                dst[2] = x[2];
                ++j;
                next_ck += a.K;
            }
            uint32_t len = min(kSumBlock, a.steps - t);
            if (want_ck) len = min(len, next_ck - t);
            float sum[3] = {0.f, 0.f, 0.f};
            // OU: the drift needs each scaled step.  Constant drift: the block
            // sums the unit normals and scales the sum once at the flush.
            auto step = [&](uint32_t tc) {
                float z[3];
                if (OU) walk3d_scaled_normals(keys, tc, a.sig_sqdt, z);
                else walk3d_normals(keys, tc, z);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (OU) sum[q] += fmaf(-a.kappa_dt, x[q] + sum[q], z[q] + a.mu_dt[q]);
                    else sum[q] += z[q];
                }
            };
            if (len == kSumBlock) {
                // A full block: constant trip count, unrolled (as in the 2D walk).
#pragma unroll 4
                for (uint32_t k = 0; k < kSumBlock; ++k) step(t + k + 1u);
            } else {
                for (uint32_t k = 0; k < len; ++k) step(t + k + 1u);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
                kahan_add(x[q], c[q], OU ? sum[q] : fmaf((float)len, a.mu_dt[q], a.sig_sqdt * sum[q]));
            t += len;
        }
        xT[3 * i] = x[0];
        xT[3 * i + 1] = x[1];
        xT[3 * i + 2] = x[2];
        const double r2 = (double)x[0] * x[0] + (double)x[1] * x[1] + (double)x[2] * x[2];
        loss[0] = 0.5 * r2;
    }
    if (partials) block_reduce_store<kRedWidth>(loss, partials);
}

// Adjoint of the walk and the loss, regenerating every z_t from its key and
// walking time backwards.  lambda_T = k x_T / p_total * g.
//   OU = false (kappa = 0, dL/dkappa not wanted): lambda is constant, so
//     dL/dmu_c = lambda_c T dt and dL/dsigma = sum_c lambda_c sqrt(dt) sum_t z_t,c.
//   OU = true: per checkpoint segment, newest first, starting from the
//     segment's end position (the next checkpoint, or x_T), each step t-1 -> t
//     (noise counter t) adds lambda_t dt to dL/dmu, lambda_t . sqrt(dt) z_{t-1}
//     to dL/dsigma and lambda_t . (-x_{t-1} dt) to dL/dkappa.  Then it
//     recomputes x_{t-1} = (x_t - mu dt - sigma sqrt(dt) z_{t-1}) / (1 - kappa dt)
//     and sets lambda_{t-1} = lambda_t (1 - kappa dt).  lambda and the sums run
//     in FP32 within a segment (at most K steps) and are re-anchored in FP64
//     between segments.
template <bool OU>
__global__ void __launch_bounds__(kWalkBlock, OU ? 3 : 1) walk3d_bwd_kernel(Walk3dArgs a, const float *__restrict__ xT,
                                                               const float *__restrict__ ckpt,
                                                               const double *__restrict__ grad_loss,
                                                               float *__restrict__ dx0,
                                                               double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double g[kRedWidth] = {};
    if (i < a.n) {
        const double gl = grad_loss ? *grad_loss : 1.0;
        const orand::PhiloxKeys keys(a.seed ^ (a.p_first + i));
        double lam[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) lam[q] = a.k_over_p * (double)xT[3 * i + q] * gl;
        if constexpr (!OU) {
            // S = sum of z_t, in blocks of kSumBlock steps Kahan-added to S.
            float S[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
            for (uint32_t tt = a.steps; tt > 0;) {
                const uint32_t len = min(kSumBlock, tt);
                float sum[3] = {0.f, 0.f, 0.f};
                auto step = [&](uint32_t tc) {
                    float z[3];
                    walk3d_normals(keys, tc, z);   // z_{t-1} uses counter t
#pragma unroll
                    for (int q = 0; q < 3; ++q) sum[q] += z[q];
                };
                if (len == kSumBlock) {
                    // A full block: constant trip count, unrolled (measured on
                    // B300: 15 % faster than the variable-length loop).
#pragma unroll 4
                    for (uint32_t k = 0; k < kSumBlock; ++k) step(tt - k);
                } else {
                    for (uint32_t k = 0; k < len; ++k) step(tt - k);
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) kahan_add(S[q], c[q], sum[q]);
                tt -= len;
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                g[q] = lam[q] * a.t_dt;
                g[3] += lam[q] * a.sqdt * (double)S[q];
            }
        } else {
            float x[3] = {xT[3 * i], xT[3 * i + 1], xT[3 * i + 2]};
            const uint32_t nseg = (a.steps + a.K - 1) / a.K;
            for (uint32_t jj = nseg; jj > 0; --jj) {
                const uint32_t t0 = (jj - 1) * a.K;
                const uint32_t t1 = min(a.steps, t0 + a.K);
                if (jj < nseg) {   // segment end x_{jj K} is checkpoint jj
                    const float *ck = ckpt + ((size_t)jj * a.n + i) * 3;
                    x[0] = ck[0];
                    x[1] = ck[1];
                    x[2] = ck[2];
                }
                float lf[3] = {(float)lam[0], (float)lam[1], (float)lam[2]};
                float amu[3] = {0.f, 0.f, 0.f}, asig = 0.f, akap = 0.f;
                auto step = [&](uint32_t t) {
                    float z[3];
                    walk3d_normals(keys, t, z);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        amu[q] += lf[q];
                        asig = fmaf(lf[q], z[q], asig);
                        const float xp = (x[q] - fmaf(a.sig_sqdt, z[q], a.mu_dt[q])) * a.inv_decay_f;
                        akap = fmaf(lf[q], xp, akap);
                        x[q] = xp;
                        lf[q] *= a.decay_f;
                    }
                };
                // Steps t1, t1 - 1, ..., t0 + 1 in runs of kSumBlock with a
                // constant trip count, then the rest.
                uint32_t t = t1;
                for (; t - t0 >= kSumBlock; t -= kSumBlock) {
#pragma unroll 4
                    for (uint32_t k = 0; k < kSumBlock; ++k) step(t - k);
                }
                for (; t > t0; --t) step(t);
                const double seg_decay = (jj == nseg) ? a.decay_last : a.decay_K;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    g[q] += (double)amu[q] * a.dt;
                    lam[q] *= seg_decay;
                }
                g[3] += (double)asig * a.sqdt;
                g[4] -= (double)akap * a.dt;
            }
        }
        if (dx0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) dx0[3 * i + q] = (float)lam[q];
        }
    }
    block_reduce_store<kRedWidth>(g, partials);
}

// The walks' Box-Muller map on word pairs, for inspection and testing.
__global__ void __launch_bounds__(256) walk_normals_kernel(const uint32_t *__restrict__ words, uint64_t n_pairs,
                                                          float *__restrict__ out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float2 z = orand::box_muller_walk_f32(words[2 * i], words[2 * i + 1]);
        out[2 * i] = z.x;
        out[2 * i + 1] = z.y;
    }
}

// ------------------------------------------- fused noise-storing baseline
//
// The other side of the regeneration trade-off: the same fused forward
// (constant drift, block sums) also writes every standard normal z_t to
// z_store[t][i][3], and the backward reads z back instead of regenerating
// it.  This costs 12 bytes of HBM per particle-step (written once, read
// once) in exchange for the backward's random-number work.

__global__ void __launch_bounds__(kWalkBlock) stored_fwd_kernel(Walk3dArgs a, const float *__restrict__ x0_in,
                                                               float *__restrict__ xT, float *__restrict__ z_store,
                                                               double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double loss[kRedWidth] = {};
    if (i < a.n) {
        const orand::PhiloxKeys keys(a.seed ^ (a.p_first + i));
        float x[3], c[3] = {0.f, 0.f, 0.f};
        if (x0_in) {
            x[0] = x0_in[3 * i];
            x[1] = x0_in[3 * i + 1];
            x[2] = x0_in[3 * i + 2];
        } else {
            walk3d_x0(keys, x);
        }
        for (uint32_t t = 0; t < a.steps;) {
            const uint32_t len = min(kSumBlock, a.steps - t);
            float sum[3] = {0.f, 0.f, 0.f};
            auto step = [&](uint32_t k) {
                float z[3];
                walk3d_normals(keys, t + k + 1u, z);
                float *dst = z_store + ((size_t)(t + k) * a.n + i) * 3;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    dst[q] = z[q];
                    sum[q] = fmaf(a.sig_sqdt, z[q], sum[q]);
                }
            };
            if (len == kSumBlock) {
                // The same full-block unrolling as the regenerating forward.
#pragma unroll 4
                for (uint32_t k = 0; k < kSumBlock; ++k) step(k);
            } else {
                for (uint32_t k = 0; k < len; ++k) step(k);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) kahan_add(x[q], c[q], fmaf((float)len, a.mu_dt[q], sum[q]));
            t += len;
        }
        xT[3 * i] = x[0];
        xT[3 * i + 1] = x[1];
        xT[3 * i + 2] = x[2];
        loss[0] = 0.5 * ((double)x[0] * x[0] + (double)x[1] * x[1] + (double)x[2] * x[2]);
    }
    if (partials) block_reduce_store<kRedWidth>(loss, partials);
}

__global__ void __launch_bounds__(kWalkBlock) stored_bwd_kernel(Walk3dArgs a, const float *__restrict__ xT,
                                                               const float *__restrict__ z_store,
                                                               const double *__restrict__ grad_loss,
                                                               float *__restrict__ dx0, double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double g[kRedWidth] = {};
    if (i < a.n) {
        const double gl = grad_loss ? *grad_loss : 1.0;
        float S[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
        for (uint32_t t = 0; t < a.steps;) {
            const uint32_t len = min(kSumBlock, a.steps - t);
            float sum[3] = {0.f, 0.f, 0.f};
#pragma unroll 8
            for (uint32_t k = 0; k < len; ++k) {
                const float *src = z_store + ((size_t)(t + k) * a.n + i) * 3;
#pragma unroll
                for (int q = 0; q < 3; ++q) sum[q] += __ldg(src + q);
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) kahan_add(S[q], c[q], sum[q]);
            t += len;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double lam = a.k_over_p * (double)xT[3 * i + q] * gl;
            g[q] = lam * a.t_dt;
            g[3] += lam * a.sqdt * (double)S[q];
            if (dx0) dx0[3 * i + q] = (float)lam;
        }
    }
    block_reduce_store<kRedWidth>(g, partials);
}

// ------------------------------------------- plain noise-storing baseline

__global__ void __launch_bounds__(kWalkBlock) plain_init_kernel(Walk3dArgs a, const float *__restrict__ x0_in,
                                                               float *__restrict__ x)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    if (i >= a.n) return;
    if (x0_in) {
        for (int q = 0; q < 3; ++q) x[3 * i + q] = x0_in[3 * i + q];
    } else {
        const orand::PhiloxKeys keys(a.seed ^ (a.p_first + i));
        float v[3];
        walk3d_x0(keys, v);
        for (int q = 0; q < 3; ++q) x[3 * i + q] = v[q];
    }
}

// One step of the walk for all particles: regenerate the key (state
// construction per launch, as in the paper's listing), draw z_t, store it,
// update x in HBM.
__global__ void __launch_bounds__(kWalkBlock) plain_step_kernel(Walk3dArgs a, uint32_t t, float *__restrict__ x,
                                                               float *__restrict__ z_t)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    if (i >= a.n) return;
    const uint64_t key64 = a.seed ^ (a.p_first + i);
    const uint4 w = orand::philox_block(key64, t + 1u, 0u);
    const float2 p = orand::box_muller_walk_f32(w.x, w.y);
    const float z[3] = {p.x, p.y, orand::box_muller_cos_walk_f32(w.z, w.w)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        z_t[3 * i + q] = z[q];
        x[3 * i + q] = x[3 * i + q] + fmaf(-a.kappa_dt, x[3 * i + q], fmaf(a.sig_sqdt, z[q], a.mu_dt[q]));
    }
}

__global__ void __launch_bounds__(kWalkBlock) plain_loss_kernel(Walk3dArgs a, const float *__restrict__ x,
                                                               double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double v[kRedWidth] = {};
    if (i < a.n) {
        const double r2 = (double)x[3 * i] * x[3 * i] + (double)x[3 * i + 1] * x[3 * i + 1] +
                          (double)x[3 * i + 2] * x[3 * i + 2];
        v[0] = 0.5 * r2;
    }
    block_reduce_store<kRedWidth>(v, partials);
}

// Backward, one launch per step: S += z_t read back from HBM.
__global__ void __launch_bounds__(kWalkBlock) plain_bwd_step_kernel(uint64_t n3, const float *__restrict__ z_t,
                                                                   float *__restrict__ S)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    if (i < n3) S[i] += z_t[i];
}

__global__ void __launch_bounds__(kWalkBlock) plain_bwd_final_kernel(Walk3dArgs a, const float *__restrict__ xT,
                                                                    const float *__restrict__ S,
                                                                    const double *__restrict__ grad_loss,
                                                                    float *__restrict__ dx0,
                                                                    double *__restrict__ partials)
{
    const uint64_t i = (uint64_t)blockIdx.x * kWalkBlock + threadIdx.x;
    double g[kRedWidth] = {};
    if (i < a.n) {
        const double gl = grad_loss ? *grad_loss : 1.0;
        for (int q = 0; q < 3; ++q) {
            const double lam = a.k_over_p * (double)xT[3 * i + q] * gl;
            g[q] = lam * a.t_dt;
            g[3] += lam * a.sqdt * (double)S[3 * i + q];
            if (dx0) dx0[3 * i + q] = (float)lam;
        }
    }
    block_reduce_store<kRedWidth>(g, partials);
}

// ------------------------------------------------------------ host side

static unsigned walk_grid(uint64_t n) { return (unsigned)ceil_div(n, kWalkBlock); }

// One particle per thread: the grid must fit the 2^31 - 1 block limit.
static bool walk_grid_ok(uint64_t n) { return ceil_div(n, kWalkBlock) <= 0x7FFFFFFFull; }

static bool finite_nonneg(float v) { return isfinite(v) && v >= 0.0f; }

static orand_status_t walk3d_args(const orand_walk3d_t *p, Walk3dArgs *a)
{
    if (p == nullptr) return ORAND_ERR_INVALID_ARG;
    if (!finite_nonneg(p->dt) || !finite_nonneg(p->sigma) || !isfinite(p->k) || !isfinite(p->mu[0]) ||
        !isfinite(p->mu[1]) || !isfinite(p->mu[2]) || !isfinite(p->kappa) || p->reserved != 0)
        return ORAND_ERR_INVALID_ARG;
    if (!(1.0 - (double)p->kappa * (double)p->dt > 0.0)) return ORAND_ERR_INVALID_ARG;  // decay must stay positive
    if (p->p_first + p->n_particles < p->p_first) return ORAND_ERR_OVERFLOW;
    if (!walk_grid_ok(p->n_particles)) return ORAND_ERR_OVERFLOW;
    if (p->steps == UINT32_MAX) return ORAND_ERR_OVERFLOW;  // counters t + 1 must fit 32 bits
    a->n = p->n_particles;
    a->p_first = p->p_first;
    a->seed = p->seed;
    a->steps = p->steps;
    a->K = p->ckpt_every;
    const double dt = (double)p->dt;
    for (int q = 0; q < 3; ++q) a->mu_dt[q] = (float)((double)p->mu[q] * dt);
    a->sig_sqdt = (float)((double)p->sigma * sqrt(dt));
    const double P = (double)(p->p_total ? p->p_total : p->n_particles);
    a->k_over_p = P > 0 ? (double)p->k / P : 0.0;
    a->t_dt = (double)p->steps * dt;
    a->sqdt = sqrt(dt);
    a->dt = dt;
    const double decay = 1.0 - (double)p->kappa * dt;
    a->kappa_dt = (float)((double)p->kappa * dt);
    a->decay_f = (float)decay;
    a->inv_decay_f = (float)(1.0 / decay);
    const uint32_t nseg = a->K ? (a->steps + a->K - 1) / a->K : 0;
    a->decay_K = a->K ? pow(decay, (double)a->K) : 1.0;
    a->decay_last = nseg ? pow(decay, (double)(a->steps - (nseg - 1) * a->K)) : 1.0;
    return ORAND_OK;
}



static orand_status_t check_ptr(const void *ptr, size_t align)
{
    if (ptr == nullptr) return ORAND_ERR_INVALID_ARG;
    return ((uintptr_t)ptr % align) ? ORAND_ERR_ALIGNMENT : ORAND_OK;
}

// Argument checks of the adjoint shared by both entry points.  With
// kappa != 0 or dL/dkappa wanted, the checkpoints are needed (ckpt_every > 0).
static orand_status_t bwd_validate(const Walk3dArgs &a, const orand_walk3d_t *p, const float *xT,
                                   const float *ckpt, const double *grad_loss, double *dmu, double *dsigma,
                                   double *dkappa, float *dx0)
{
    orand_status_t st;
    if ((st = check_ptr(dmu, 8)) != ORAND_OK || (st = check_ptr(dsigma, 8)) != ORAND_OK) return st;
    if (dkappa && ((uintptr_t)dkappa % 8)) return ORAND_ERR_ALIGNMENT;
    if (a.n == 0) return ORAND_OK;
    if ((st = check_ptr(xT, 4)) != ORAND_OK) return st;
    if (dx0 && ((uintptr_t)dx0 % 4)) return ORAND_ERR_ALIGNMENT;
    if (grad_loss && ((uintptr_t)grad_loss % 8)) return ORAND_ERR_ALIGNMENT;
    const bool ou = p->kappa != 0.0f || dkappa != nullptr;
    if (ou && a.steps > 0) {
        if (a.K == 0) return ORAND_ERR_INVALID_ARG;
        if (a.steps > a.K && (st = check_ptr(ckpt, 4)) != ORAND_OK) return st;
    }
    return ORAND_OK;
}

static orand_status_t bwd_zero(double *dmu, double *dsigma, double *dkappa, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(dmu, 0, 3 * sizeof(double), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsigma, 0, sizeof(double), stream);
    if (e == cudaSuccess && dkappa) e = cudaMemsetAsync(dkappa, 0, sizeof(double), stream);
    return cuda_status(e);
}

// Adjoint kernel plus the fixed-order reductions of its FP64 partials.
static orand_status_t bwd_launch(const Walk3dArgs &a, const orand_walk3d_t *p, const float *xT, const float *ckpt,
                                 const double *grad_loss, double *dmu, double *dsigma, double *dkappa, float *dx0,
                                 double *partials, cudaStream_t stream)
{
    const bool ou = p->kappa != 0.0f || dkappa != nullptr;
    const unsigned grid = walk_grid(a.n);
    if (ou) walk3d_bwd_kernel<true><<<grid, kWalkBlock, 0, stream>>>(a, xT, ckpt, grad_loss, dx0, partials);
    else walk3d_bwd_kernel<false><<<grid, kWalkBlock, 0, stream>>>(a, xT, ckpt, grad_loss, dx0, partials);
    orand_status_t st = launch_status();
    if (st != ORAND_OK) return st;
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials, grid, 1.0, nullptr, dmu, 3);
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials + 3, grid, 1.0, nullptr, dsigma, 1);
    if (dkappa) reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials + 4, grid, 1.0, nullptr, dkappa, 1);
    return launch_status();
}

}  // namespace orand_impl

using namespace orand_impl;

extern "C" {

orand_status_t orand_brownian_walk(const orand_walk2d_t *p, float *pos_out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_brownian_walk");
    if (p == nullptr) return ORAND_ERR_INVALID_ARG;
    if (!finite_nonneg(p->dt) || !finite_nonneg(p->D)) return ORAND_ERR_INVALID_ARG;
    if (p->p_first + p->n_particles < p->p_first) return ORAND_ERR_OVERFLOW;
    if (p->n_particles > UINT64_MAX / 8) return ORAND_ERR_OVERFLOW;
    if (p->n_particles == 0) return ORAND_OK;
    orand_status_t st = check_ptr(pos_out, 8);
    if (st != ORAND_OK) return st;
    if (p->steps == UINT32_MAX) return ORAND_ERR_OVERFLOW;  // counters 1..steps, same limit as the 3D walk
    const uint64_t grid = ceil_div(p->n_particles, (uint64_t)kWalk2dBlock);
    if (grid > 0x7FFFFFFFull) return ORAND_ERR_OVERFLOW;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    const float s = (float)sqrt(2.0 * (double)p->D * (double)p->dt);
    walk2d_kernel<<<(unsigned)grid, kWalk2dBlock, 0, stream>>>(p->n_particles, p->p_first, p->seed, p->steps, s,
                                                              (float2 *)pos_out);
    return launch_status();
}

orand_status_t orand_walk3d_init(const orand_walk3d_t *p, float *x0, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_init");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK || a.n == 0) return st;
    if ((st = check_ptr(x0, 4)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    walk3d_init_kernel<<<walk_grid(a.n), kWalkBlock, 0, stream>>>(a, x0);
    return launch_status();
}

orand_status_t orand_walk3d_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *xT,
                                float *ckpt, double *loss, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_fwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if (a.n == 0) {
        if (loss) return cuda_status(cudaMemsetAsync(loss, 0, sizeof(double), stream));
        return ORAND_OK;
    }
    if ((st = check_ptr(xT, 4)) != ORAND_OK) return st;
    if (x0 && ((uintptr_t)x0 % 4)) return ORAND_ERR_ALIGNMENT;
    if (ckpt && ((uintptr_t)ckpt % 4)) return ORAND_ERR_ALIGNMENT;
    if (loss && ((uintptr_t)loss % 8)) return ORAND_ERR_ALIGNMENT;
    if (a.K == 0) ckpt = nullptr;
    const unsigned grid = walk_grid(a.n);
    double *partials = nullptr;
    if (loss) {
        void *scr = nullptr;
        if ((st = ctx_scratch(ctx, (size_t)grid * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
        partials = (double *)scr;
    }
    if (p->kappa != 0.0f) walk3d_fwd_kernel<true><<<grid, kWalkBlock, 0, stream>>>(a, x0, xT, ckpt, partials);
    else walk3d_fwd_kernel<false><<<grid, kWalkBlock, 0, stream>>>(a, x0, xT, ckpt, partials);
    if ((st = launch_status()) != ORAND_OK || !loss) return st;
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials, grid, a.k_over_p, nullptr, loss, 1);
    return launch_status();
}

orand_status_t orand_walk3d_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT, const float *ckpt,
                                const double *grad_loss, double *dmu, double *dsigma, double *dkappa, float *dx0,
                                cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_bwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if ((st = bwd_validate(a, p, xT, ckpt, grad_loss, dmu, dsigma, dkappa, dx0)) != ORAND_OK) return st;
    if (a.n == 0) return bwd_zero(dmu, dsigma, dkappa, stream);
    void *scr = nullptr;
    if ((st = ctx_scratch(ctx, (size_t)walk_grid(a.n) * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
    return bwd_launch(a, p, xT, ckpt, grad_loss, dmu, dsigma, dkappa, dx0, (double *)scr, stream);
}

orand_status_t orand_walk3d_plain_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *x,
                                      float *z_store, double *loss, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_plain_fwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if (p->kappa != 0.0f) return ORAND_ERR_INVALID_ARG;  // the baseline is the constant-drift walk
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if (a.n == 0) return ORAND_OK;
    if ((st = check_ptr(x, 4)) != ORAND_OK) return st;
    if (a.steps && (st = check_ptr(z_store, 4)) != ORAND_OK) return st;
    if (x0 && ((uintptr_t)x0 % 4)) return ORAND_ERR_ALIGNMENT;
    if (loss && ((uintptr_t)loss % 8)) return ORAND_ERR_ALIGNMENT;
    const unsigned grid = walk_grid(a.n);
    plain_init_kernel<<<grid, kWalkBlock, 0, stream>>>(a, x0, x);
    for (uint32_t t = 0; t < a.steps; ++t)
        plain_step_kernel<<<grid, kWalkBlock, 0, stream>>>(a, t, x, z_store + (size_t)t * a.n * 3);
    if ((st = launch_status()) != ORAND_OK || !loss) return st;
    void *scr = nullptr;
    if ((st = ctx_scratch(ctx, (size_t)grid * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
    plain_loss_kernel<<<grid, kWalkBlock, 0, stream>>>(a, x, (double *)scr);
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>((double *)scr, grid, a.k_over_p, nullptr, loss, 1);
    return launch_status();
}

orand_status_t orand_walk3d_plain_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT,
                                      const float *z_store, const double *grad_loss, double *dmu,
                                      double *dsigma, float *dx0, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_plain_bwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if (p->kappa != 0.0f) return ORAND_ERR_INVALID_ARG;
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if ((st = check_ptr(dmu, 8)) != ORAND_OK || (st = check_ptr(dsigma, 8)) != ORAND_OK) return st;
    if (a.n == 0) {
        cudaError_t e = cudaMemsetAsync(dmu, 0, 3 * sizeof(double), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(dsigma, 0, sizeof(double), stream);
        return cuda_status(e);
    }
    if ((st = check_ptr(xT, 4)) != ORAND_OK) return st;
    if (a.steps && (st = check_ptr(z_store, 4)) != ORAND_OK) return st;
    const unsigned grid = walk_grid(a.n);
    const size_t s_bytes = (a.n * 3 * sizeof(float) + 255) & ~(size_t)255;
    void *scr = nullptr;
    if ((st = ctx_scratch(ctx, s_bytes + (size_t)grid * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
    float *S = (float *)scr;
    double *partials = (double *)((char *)scr + s_bytes);
    cudaError_t e = cudaMemsetAsync(S, 0, a.n * 3 * sizeof(float), stream);
    if (e != cudaSuccess) return cuda_status(e);
    const uint64_t n3 = a.n * 3;
    const unsigned g3 = (unsigned)ceil_div(n3, kWalkBlock);
    for (uint32_t tt = a.steps; tt > 0; --tt)
        plain_bwd_step_kernel<<<g3, kWalkBlock, 0, stream>>>(n3, z_store + (size_t)(tt - 1) * n3, S);
    plain_bwd_final_kernel<<<grid, kWalkBlock, 0, stream>>>(a, xT, S, grad_loss, dx0, partials);
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials, grid, 1.0, nullptr, dmu, 3);
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials + 3, grid, 1.0, nullptr, dsigma, 1);
    return launch_status();
}

orand_status_t orand_walk3d_stored_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *xT,
                                       float *z_store, double *loss, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_stored_fwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if (p->kappa != 0.0f) return ORAND_ERR_INVALID_ARG;  // the baseline is the constant-drift walk
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if (a.n == 0) {
        if (loss) return cuda_status(cudaMemsetAsync(loss, 0, sizeof(double), stream));
        return ORAND_OK;
    }
    if ((st = check_ptr(xT, 4)) != ORAND_OK) return st;
    if (a.steps && (st = check_ptr(z_store, 4)) != ORAND_OK) return st;
    if (x0 && ((uintptr_t)x0 % 4)) return ORAND_ERR_ALIGNMENT;
    if (loss && ((uintptr_t)loss % 8)) return ORAND_ERR_ALIGNMENT;
    const unsigned grid = walk_grid(a.n);
    double *partials = nullptr;
    if (loss) {
        void *scr = nullptr;
        if ((st = ctx_scratch(ctx, (size_t)grid * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
        partials = (double *)scr;
    }
    stored_fwd_kernel<<<grid, kWalkBlock, 0, stream>>>(a, x0, xT, z_store, partials);
    if ((st = launch_status()) != ORAND_OK || !loss) return st;
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials, grid, a.k_over_p, nullptr, loss, 1);
    return launch_status();
}

orand_status_t orand_walk3d_stored_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT,
                                       const float *z_store, const double *grad_loss, double *dmu, double *dsigma,
                                       float *dx0, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk3d_stored_bwd");
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if (p->kappa != 0.0f) return ORAND_ERR_INVALID_ARG;
    if ((st = ctx_check(ctx)) != ORAND_OK) return st;
    if ((st = check_ptr(dmu, 8)) != ORAND_OK || (st = check_ptr(dsigma, 8)) != ORAND_OK) return st;
    if (a.n == 0) return bwd_zero(dmu, dsigma, nullptr, stream);
    if ((st = check_ptr(xT, 4)) != ORAND_OK) return st;
    if (a.steps && (st = check_ptr(z_store, 4)) != ORAND_OK) return st;
    if (dx0 && ((uintptr_t)dx0 % 4)) return ORAND_ERR_ALIGNMENT;
    if (grad_loss && ((uintptr_t)grad_loss % 8)) return ORAND_ERR_ALIGNMENT;
    const unsigned grid = walk_grid(a.n);
    void *scr = nullptr;
    if ((st = ctx_scratch(ctx, (size_t)grid * kRedWidth * sizeof(double), &scr)) != ORAND_OK) return st;
    double *partials = (double *)scr;
    stored_bwd_kernel<<<grid, kWalkBlock, 0, stream>>>(a, xT, z_store, grad_loss, dx0, partials);
    if ((st = launch_status()) != ORAND_OK) return st;
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials, grid, 1.0, nullptr, dmu, 3);
    reduce_partials_kernel<kRedWidth><<<1, 256, 0, stream>>>(partials + 3, grid, 1.0, nullptr, dsigma, 1);
    return launch_status();
}

orand_status_t orand_walk_normals(const uint32_t *words, uint64_t n_pairs, float *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_walk_normals");
    if (n_pairs == 0) return ORAND_OK;
    if (n_pairs > (UINT64_MAX >> 3)) return ORAND_ERR_OVERFLOW;
    orand_status_t st;
    if ((st = check_ptr(words, 4)) != ORAND_OK || (st = check_ptr(out, 4)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    walk_normals_kernel<<<grid_for(n_pairs, 256, info.sm_count, 8), 256, 0, stream>>>(words, n_pairs, out);
    return launch_status();
}

}  // extern "C"

// ------------------------------------------------ allocation-free adjoint
//
// orand_walk3d_bwd_noalloc: the adjoint with its reduction partials in a
// fixed device array instead of context scratch, so no call ever allocates.

namespace orand_impl {

constexpr uint64_t kNoAllocMaxParticles = 1ull << 22;
constexpr unsigned kNoAllocMaxBlocks = (unsigned)(kNoAllocMaxParticles / kWalkBlock);  // 16384

// 16384 blocks x 5 FP64 partials = 640 KiB, resident on every device that
// loads the library.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kRedWidth];

constexpr int kNoAllocDevices = 64;
static std::mutex g_noalloc_mutex[kNoAllocDevices];
static std::atomic<double *> g_noalloc_ptr[kNoAllocDevices];

// Device address of g_noalloc_partials on the current device (the host-side
// name is only a stand-in for that address).  Only a successful lookup is
// kept: after a failure (for example a first call made inside a stream
// capture) the next call on that device tries again.
static orand_status_t noalloc_partials(double **out)
{
    int dev = -1;
    ORAND_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocDevices) return ORAND_ERR_UNSUPPORTED;
    double *ptr = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (ptr == nullptr) {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex[dev]);
        ptr = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
        if (ptr == nullptr) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || p == nullptr) {
                log_cuda_failure("cudaGetSymbolAddress(g_noalloc_partials)", __FILE__, __LINE__, e);
                return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            }
            ptr = (double *)p;
            g_noalloc_ptr[dev].store(ptr, std::memory_order_release);
        }
    }
    *out = ptr;
    return ORAND_OK;
}

}  // namespace orand_impl

extern "C" orand_status_t orand_walk3d_bwd_noalloc(const orand_walk3d_t *p, const float *xT, const float *ckpt,
                                                   const double *grad_loss, double *dmu, double *dsigma,
                                                   double *dkappa, float *dx0, cudaStream_t stream)
{
    Walk3dArgs a;
    orand_status_t st = walk3d_args(p, &a);
    if (st != ORAND_OK) return st;
    if (a.n > kNoAllocMaxParticles) return ORAND_ERR_SCRATCH_LIMIT;
    if ((st = bwd_validate(a, p, xT, ckpt, grad_loss, dmu, dsigma, dkappa, dx0)) != ORAND_OK) return st;
    if (a.n == 0) return bwd_zero(dmu, dsigma, dkappa, stream);
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    double *partials = nullptr;
    if ((st = noalloc_partials(&partials)) != ORAND_OK) return st;
    // Every partial the reductions read (blocks 0 .. grid-1) is written by
    // this call's adjoint kernel first: no clearing needed.
    return bwd_launch(a, p, xT, ckpt, grad_loss, dmu, dsigma, dkappa, dx0, partials, stream);
}
