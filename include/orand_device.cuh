/*
 * orand_device.cuh -- in-thread counter-based generation for CUDA kernels
 * (sm_103a).  Header-only; include it from any .cu file to draw random
 * numbers inside your own kernels with no generator state in memory.
 *
 * This is the device half of the OpenRAND method (arXiv 2310.19925): a
 * generator is built from a 64-bit seed and a 32-bit counter (§3), its state
 * fits in registers (§2: 96 bits of user state), and the same (seed,
 * counter) gives the same stream on every thread count and launch shape.
 * The paper's usage pattern (Fig. 1) reads, with this header:
 *
 *     orand::Philox rng(p.pid, counter);
 *     float2 r = rng.uniform2_f32();
 *
 * Generator definitions follow the publications the paper cites for them
 * (§3): Philox4x32-10 and Threefry4x32-20 (Salmon et al., SC'11), Squares
 * (Widynski 2020), Tyche (Neves & Araujo 2011).  Stream layout, shared by
 * every kernel of the library so that all delivery paths emit identical bits:
 *
 *   Philox    key = (lo32(key64), hi32(key64)), counter block
 *             (b, counter, 0, 0); words 4b..4b+3 are its lanes 0..3.
 *   Threefry  key = (lo32, hi32, 0, 0); same counter block layout.
 *   Squares   word w = squares32((counter << 32) | w, fmix64(key64) | 1).
 *   Tyche     a = hi32(key64), b = lo32(key64), c = 2654435769,
 *             d = 1367130551 ^ counter, 20 MIX; word w = b after MIX w+1.
 *
 * Maps: FP32 uniform (w >> 8) * 2^-24; FP64 uniform from two words, first
 * one high (Fig. 3), ((hi:lo) >> 11) * 2^-53, built with integer ops and
 * one FP32 conversion (no FP64 arithmetic);
 * Box-Muller with u1 = ((w0>>8)+1) * 2^-24, u2 = (w1>>8) * 2^-24,
 * r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2), using the library's own
 * reduced-range log and sincospi and the SFU's square root (within 3 ulp of
 * the FP64 values).  The walk kernels use a cheaper map of the same form
 * (bm_radius_walk, bm_cos_sin_walk: SFU log2, sin and cos, a half-turn
 * split of the angle), accurate to about 1e-6.
 */
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

/* The generator cores (round functions, key schedules, the engines' word
 * draws) compile for the host too, so a CPU program gets the same streams
 * from the same source; the value maps are device-only. */
#define ORAND_HD __host__ __device__ __forceinline__

namespace orand {

/* ---------------------------------------------------------------- Philox */

constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;  /* floor(2^32 / golden ratio) */
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;  /* floor(2^32 (sqrt(3) - 1)) */

/* One Philox round on (c0..c3) with round key (k0, k1).  The 64-bit
 * products map to one wide integer multiply-add each. */
ORAND_HD void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                             uint32_t &c3, uint32_t k0, uint32_t k1)
{
    const uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    const uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
}

/* Stateless Philox4x32-10 block function. */
ORAND_HD uint4 philox4x32_10(uint4 ctr, uint2 key)
{
    uint32_t c0 = ctr.x, c1 = ctr.y, c2 = ctr.z, c3 = ctr.w;
    uint32_t k0 = key.x, k1 = key.y;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        philox_round(c0, c1, c2, c3, k0, k1);
    }
    return make_uint4(c0, c1, c2, c3);
}

/* Philox with the ten round keys precomputed once per stream (a fill
 * thread reuses them for every block of the same key). */
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
    ORAND_HD explicit PhiloxKeys(uint64_t key64)
    {
        uint32_t a = (uint32_t)key64, b = (uint32_t)(key64 >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            k0[r] = a; k1[r] = b;
            a += PHILOX_W0; b += PHILOX_W1;
        }
    }
    ORAND_HD uint4 block(uint32_t b_idx, uint32_t counter) const
    {
        uint32_t c0 = b_idx, c1 = counter, c2 = 0u, c3 = 0u;
#pragma unroll
        for (int r = 0; r < 10; ++r) philox_round(c0, c1, c2, c3, k0[r], k1[r]);
        return make_uint4(c0, c1, c2, c3);
    }
};

ORAND_HD uint4 philox_block(uint64_t key64, uint32_t counter, uint32_t b_idx)
{
    return philox4x32_10(make_uint4(b_idx, counter, 0u, 0u),
                         make_uint2((uint32_t)key64, (uint32_t)(key64 >> 32)));
}

/* -------------------------------------------------------------- Threefry */

ORAND_HD uint32_t rotl32(uint32_t x, int r)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_l(x, x, r);
#else
    return (x << r) | (x >> ((32 - r) & 31));
#endif
}

template <int RA, int RB, bool EVEN>
ORAND_HD void threefry_round(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3)
{
    if (EVEN) {
        x0 += x1; x1 = rotl32(x1, RA) ^ x0;
        x2 += x3; x3 = rotl32(x3, RB) ^ x2;
    } else {
        x0 += x3; x3 = rotl32(x3, RA) ^ x0;
        x2 += x1; x1 = rotl32(x1, RB) ^ x2;
    }
}

/* Four rounds starting at row R0 of the rotation table, then injection I. */
template <int R0, int I>
ORAND_HD void threefry_quad(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                                              const uint32_t ks[5])
{
    constexpr int ROT[8][2] = {{10, 26}, {11, 21}, {13, 27}, {23, 5},
                               {6, 20},  {17, 11}, {25, 10}, {18, 20}};
    threefry_round<ROT[R0 + 0][0], ROT[R0 + 0][1], true>(x0, x1, x2, x3);
    threefry_round<ROT[R0 + 1][0], ROT[R0 + 1][1], false>(x0, x1, x2, x3);
    threefry_round<ROT[R0 + 2][0], ROT[R0 + 2][1], true>(x0, x1, x2, x3);
    threefry_round<ROT[R0 + 3][0], ROT[R0 + 3][1], false>(x0, x1, x2, x3);
    x0 += ks[(I + 0) % 5];
    x1 += ks[(I + 1) % 5];
    x2 += ks[(I + 2) % 5];
    x3 += ks[(I + 3) % 5] + (uint32_t)I;
}

/* Stateless Threefry4x32-20 block function. */
ORAND_HD uint4 threefry4x32_20(uint4 ctr, uint4 key)
{
    uint32_t ks[5];
    ks[0] = key.x; ks[1] = key.y; ks[2] = key.z; ks[3] = key.w;
    ks[4] = 0x1BD11BDAu ^ key.x ^ key.y ^ key.z ^ key.w;
    uint32_t x0 = ctr.x + ks[0], x1 = ctr.y + ks[1], x2 = ctr.z + ks[2], x3 = ctr.w + ks[3];
    threefry_quad<0, 1>(x0, x1, x2, x3, ks);
    threefry_quad<4, 2>(x0, x1, x2, x3, ks);
    threefry_quad<0, 3>(x0, x1, x2, x3, ks);
    threefry_quad<4, 4>(x0, x1, x2, x3, ks);
    threefry_quad<0, 5>(x0, x1, x2, x3, ks);
    return make_uint4(x0, x1, x2, x3);
}

ORAND_HD uint4 threefry_block(uint64_t key64, uint32_t counter, uint32_t b_idx)
{
    return threefry4x32_20(make_uint4(b_idx, counter, 0u, 0u),
                           make_uint4((uint32_t)key64, (uint32_t)(key64 >> 32), 0u, 0u));
}

/* --------------------------------------------------------------- Squares */

/* x*x + y modulo 2^64.  On the GPU from 32-bit halves: one wide
 * multiply-add for the low product plus y, one multiply-add for the cross
 * term 2*xl*xh (xh^2 only reaches bit 64 and above). */
ORAND_HD uint64_t sq_add(uint64_t x, uint64_t y)
{
#ifdef __CUDA_ARCH__
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint64_t p = (uint64_t)xl * xl + y;
    const uint32_t hi = (uint32_t)(p >> 32) + xl * (xh << 1);
    return ((uint64_t)hi << 32) | (uint32_t)p;
#else
    return x * x + y;  /* the same value: a CPU multiplies 64 bits at once */
#endif
}

ORAND_HD uint64_t swap_halves(uint64_t v) { return (v >> 32) | (v << 32); }

ORAND_HD uint32_t squares32(uint64_t ctr, uint64_t key)
{
    uint64_t x = ctr * key;
    const uint64_t y = x, z = y + key;
    x = swap_halves(sq_add(x, y));
    x = swap_halves(sq_add(x, z));
    x = swap_halves(sq_add(x, y));
    return (uint32_t)(sq_add(x, z) >> 32);
}

/* Per-stream Squares key: MurmurHash3's 64-bit finaliser, forced odd. */
ORAND_HD uint64_t squares_key(uint64_t key64)
{
    uint64_t h = key64;
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    h *= 0xC4CEB9FE1A85EC53ull;
    h ^= h >> 33;
    return h | 1ull;
}

/* 32-bit addition issued as the integer multiply-add a * one + b, where
 * `one` is 1 but held in a register whose value the compiler cannot see (a
 * kernel argument), so it stays a multiply-add and runs on the FMA pipe
 * rather than the ALU pipe.  Squares' fills use it (their shifts and adds
 * otherwise load the ALU pipe); the compiler already splits plain adds
 * between the two pipes where it can, so code that needs no steering keeps
 * plain adds. */
struct FmaAdd {
    uint32_t one;
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const
    {
        uint32_t d;
        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(one), "r"(b));
        return d;
    }
};

/* The Squares word for x = ctr * key (y = x) and z = (ctr + 1) * key, the
 * same value as squares32(ctr, key), with every step on the FMA pipe: the
 * cross term 2 xl xh as xl * (xh + xh) with the doubling an FmaAdd, and the
 * low product's 64-bit sum a wide multiply-add. */
__device__ __forceinline__ uint64_t sq_add_fma(uint64_t x, uint64_t y, const FmaAdd &add)
{
    const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
    const uint64_t p = (uint64_t)xl * xl + y;
    uint32_t hi;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(xl), "r"(add(xh, xh)), "r"((uint32_t)(p >> 32)));
    return ((uint64_t)hi << 32) | (uint32_t)p;
}
__device__ __forceinline__ uint32_t squares32_yz(uint64_t y, uint64_t z, const FmaAdd &add)
{
    uint64_t x = swap_halves(sq_add_fma(y, y, add));
    x = swap_halves(sq_add_fma(x, z, add));
    x = swap_halves(sq_add_fma(x, y, add));
    return (uint32_t)(sq_add_fma(x, z, add) >> 32);
}
/* y + key modulo 2^64 on the FMA pipe: a wide multiply-add of the key's low
 * word by one, then the high words. */
__device__ __forceinline__ uint64_t add64_fma(uint64_t y, uint64_t key, const FmaAdd &add)
{
    uint64_t r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"((uint32_t)key), "r"(add.one), "l"(y));
    return ((uint64_t)add((uint32_t)(r >> 32), (uint32_t)(key >> 32)) << 32) | (uint32_t)r;
}
/* Words 4b..4b+3: consecutive counters ctr, ctr + 1, ... share their products,
 * (ctr + 1) key = ctr key + key, so one 64-bit multiply and four additions
 * give every x and z. */
__device__ __forceinline__ uint4 squares_block_fma(uint64_t sq_key, uint32_t counter, uint32_t b_idx,
                                                   const FmaAdd &add)
{
    const uint64_t base = ((uint64_t)counter << 32) | ((uint64_t)b_idx << 2);
    const uint64_t y0 = base * sq_key;
    const uint64_t y1 = add64_fma(y0, sq_key, add), y2 = add64_fma(y1, sq_key, add);
    const uint64_t y3 = add64_fma(y2, sq_key, add), y4 = add64_fma(y3, sq_key, add);
    return make_uint4(squares32_yz(y0, y1, add), squares32_yz(y1, y2, add), squares32_yz(y2, y3, add),
                      squares32_yz(y3, y4, add));
}

/* Four consecutive Squares words 4b..4b+3 of stream (key, counter). */
ORAND_HD uint4 squares_block(uint64_t sq_key, uint32_t counter, uint32_t b_idx)
{
    const uint64_t base = ((uint64_t)counter << 32) | ((uint64_t)b_idx << 2);
    return make_uint4(squares32(base, sq_key), squares32(base + 1, sq_key),
                      squares32(base + 2, sq_key), squares32(base + 3, sq_key));
}

/* ----------------------------------------------------------------- Tyche */

struct TycheState {
    uint32_t a, b, c, d;
};

ORAND_HD void tyche_mix(TycheState &s)
{
#ifdef __CUDA_ARCH__
    s.a += s.b; s.d = __byte_perm(s.d ^ s.a, 0, 0x1032);   /* rotl 16 */
    s.c += s.d; s.b = rotl32(s.b ^ s.c, 12);
    s.a += s.b; s.d = __byte_perm(s.d ^ s.a, 0, 0x2103);   /* rotl 8 */
    s.c += s.d; s.b = rotl32(s.b ^ s.c, 7);
#else
    s.a += s.b; s.d = rotl32(s.d ^ s.a, 16);
    s.c += s.d; s.b = rotl32(s.b ^ s.c, 12);
    s.a += s.b; s.d = rotl32(s.d ^ s.a, 8);
    s.c += s.d; s.b = rotl32(s.b ^ s.c, 7);
#endif
}

ORAND_HD TycheState tyche_init(uint64_t key64, uint32_t counter)
{
    TycheState s;
    s.a = (uint32_t)(key64 >> 32);
    s.b = (uint32_t)key64;
    s.c = 2654435769u;                 /* floor(2^32 / golden ratio) */
    s.d = 1367130551u ^ counter;       /* floor(2^32 / pi) */
#pragma unroll 4
    for (int i = 0; i < 20; ++i) tyche_mix(s);
    return s;
}

ORAND_HD uint32_t tyche_next(TycheState &s)
{
    tyche_mix(s);
    return s.b;
}

/* ------------------------------------------------------------------ maps */

/* (w >> 8) * 2^-24: exact, in [0, 1 - 2^-24]. */
__device__ __forceinline__ float u01_f32(uint32_t w)
{
    return __uint2float_rn(w >> 8) * 0x1p-24f;
}

/* ((hi:lo) >> 11) * 2^-53, exact, in [0, 1), for every (hi, lo).  Built from
 * 32-bit integer ops (leading-zero count, funnel shifts, exponent insert)
 * rather than an integer-to-FP64 conversion, which would run on the narrow
 * FP64 pipe.  The branch on mh == 0 (probability 2^-21) is almost never
 * taken.  u01_f64 below uses a shorter form for the common case. */
__device__ __forceinline__ double u01_f64_general(uint32_t hi, uint32_t lo)
{
    const uint32_t mh = hi >> 11;                        /* m = mh:ml, 53 bits */
    const uint32_t ml = (hi << 21) | (lo >> 11);
    uint32_t rh, rl;
    if (mh != 0) {
        /* top bit of m at 52 - lz: shift m left by lz so it lands on bit 52,
         * drop it (mask), insert the biased exponent 1022 - lz. */
        const uint32_t lz = (uint32_t)__clz((int)mh) - 11u;    /* 0..20 */
        rh = (__funnelshift_l(ml, mh, lz) & 0x000FFFFFu) | ((1022u - lz) << 20);
        rl = ml << lz;
    } else if (ml != 0) {
        const uint32_t lz = (uint32_t)__clz((int)ml);           /* top bit at 31 - lz */
        const uint32_t sh = lz + 21u;                           /* 21..52: to bit 52 */
        const uint64_t v = ((uint64_t)ml << sh) & 0x000FFFFFFFFFFFFFull;
        rh = (uint32_t)(v >> 32) | ((1001u - lz) << 20);
        rl = (uint32_t)v;
    } else {
        rh = 0u;
        rl = 0u;
    }
    return __hiloint2double((int)rh, (int)rl);
}

/* The FP64 bits (high word, low word) of ((hi:lo) >> 11) * 2^-53 when
 * hi >= 2^20 (all but 2^-12 of the words).  Let p >= 20 be the position of
 * hi's leading bit.  hi converted to FP32 with truncation (exact in its top
 * 24 bits) has the bit pattern ((127 + p) << 23) | (hi's 23 bits below the
 * leading one).  The value's leading bit is 2^(p - 32), so its FP64 high word
 * is ((991 + p) << 20) | (hi's 20 bits below the leading one): the FP32
 * pattern shifted right by 3, plus 864 << 20.  The low word holds the next
 * 32 bits of the 53-bit value: (hi:lo) with lo's low 11 bits (the ones the
 * >> 11 drops) cleared, shifted right by p - 20 (0 .. 11), whose low word
 * is one funnel shift.  Four integer operations and one conversion, against
 * about twice that for the general form. */
__device__ __forceinline__ uint2 u01_f64_bits_hi20(uint32_t hi, uint32_t lo)
{
    const uint32_t f = __float_as_uint(__uint2float_rz(hi));
    const uint32_t sh = (f >> 23) - 147u;                       /* p - 20 */
    return make_uint2((f >> 3) + (864u << 20), __funnelshift_r(lo & 0xFFFFF800u, hi, sh));
}

/* ((hi:lo) >> 11) * 2^-53, exact, in [0, 1), for every (hi, lo): the short
 * form above for hi >= 2^20, the general one otherwise. */
__device__ __forceinline__ double u01_f64(uint32_t hi, uint32_t lo)
{
    if (__builtin_expect(hi >= (1u << 20), 1)) {
        const uint2 b = u01_f64_bits_hi20(hi, lo);
        return __hiloint2double((int)b.x, (int)b.y);
    }
    return u01_f64_general(hi, lo);
}

/* The same map without branches (selects only), for latency-bound code
 * where a branch would stop the scheduler from overlapping it with an
 * independent dependency chain.  Identical results. */
__device__ __forceinline__ double u01_f64_nb(uint32_t hi, uint32_t lo)
{
    const uint32_t mh = hi >> 11;
    const uint32_t ml = (hi << 21) | (lo >> 11);
    /* leading zeros of m as a 64-bit value (64 when m = 0) */
    const uint32_t lz64 = mh ? (uint32_t)__clz((int)mh) : 32u + (uint32_t)__clz((int)ml);
    /* shift m left so its top bit lands on bit 52: sh = lz64 - 11 in 0..52 */
    const uint32_t sh = lz64 - 11u;
    const bool big = sh >= 32u;
    const uint32_t s1 = sh & 31u;
    const uint32_t th = big ? (ml << s1) : __funnelshift_l(ml, mh, s1);
    const uint32_t tl = big ? 0u : (ml << s1);
    /* drop the leading bit, insert the biased exponent 1022 - sh */
    const uint32_t rh = (th & 0x000FFFFFu) | ((1022u - sh) << 20);
    const bool zero = (mh | ml) == 0u;
    return __hiloint2double(zero ? 0 : (int)rh, zero ? 0 : (int)tl);
}

/* The SFU's estimates as PTX instructions (lg2.approx, sin.approx, cos.approx,
 * sqrt.approx), used by both Box-Muller maps below. */
__device__ __forceinline__ float sfu_lg2(float x) { float y; asm("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_sin(float x) { float y; asm("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_cos(float x) { float y; asm("cos.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_sqrt(float x) { float y; asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

/* ---------------------------------------------------------- Box-Muller */
/*
 * r = sqrt(-2 ln u1) and (cos, sin)(2 pi u2), specialised to this library's
 * inputs: u1 = k 2^-24 with integer k in [1, 2^24], and 4 u2 = m 2^-22 with
 * integer m in [0, 2^24).  Method: argument reduction plus polynomials
 * (Cody & Waite 1980; Muller, "Elementary Functions", 2016).  The
 * coefficients are this library's own near-minimax fits
 * (paper_2310_19925_b300/csrc/fit_boxmuller.py); the square root is the SFU's
 * estimate.  Measured on every input against FP64: r within 1 ulp, sin and
 * cos within 1.02 ulp, exact zeros exact.  Each normal is within 3 ulp of the
 * correctly rounded FP64 value (2^24 random pairs).
 */
namespace bm {
constexpr float LN2_HI = 0x1.62e400p-1f;     /* ln 2, 16 significant bits: E * LN2_HI is exact */
constexpr float LN2_LO = 0x1.7f7d1cp-20f;    /* ln 2 - LN2_HI */
constexpr float PI_HI = 0x1.921fb6p+1f;      /* float32(pi) */
constexpr float PI_LO = -0x1.777a5cp-24f;    /* float32(pi - PI_HI) */
/* PL: (ln(1+g) - g) / g^2 on g in [sqrt(2)/2 - 1, sqrt(2) - 1], PLi the degree-i coefficient. */
constexpr float PL0 = -0x1.fffffep-2f, PL1 = 0x1.555550p-2f, PL2 = -0x1.00020ap-2f, PL3 = 0x1.99a22ep-3f,
                PL4 = -0x1.5485dcp-3f, PL5 = 0x1.22bcb0p-3f, PL6 = -0x1.0c9354p-3f, PL7 = 0x1.05ae04p-3f,
                PL8 = -0x1.3e9698p-4f;
/* QS: (sin(pi r)/r - pi) / r^2, QC: (cos(pi r) - 1) / r^2, in t = r^2 on [0, 1/16]. */
constexpr float QS0 = -0x1.4abbcep+2f, QS1 = 0x1.466bb4p+1f, QS2 = -0x1.32c258p-1f, QS3 = 0x1.489230p-4f;
constexpr float QC0 = -0x1.3bd3ccp+2f, QC1 = 0x1.03c1f6p+2f, QC2 = -0x1.55dad4p+0f, QC3 = 0x1.e78ce2p-3f,
                QC4 = -0x1.845be8p-5f;
}  // namespace bm

/* sqrt(-2 ln u1), u1 = ((w0 >> 8) + 1) * 2^-24 in (0, 1]. */
__device__ __forceinline__ float bm_radius(uint32_t w0)
{
    const uint32_t k = (w0 >> 8) + 1u;                         /* 1 .. 2^24 */
    const uint32_t bits = __float_as_uint(__uint2float_rn(k)); /* exact */
    /* k = 2^e f with f in [sqrt(2)/2, sqrt(2)): subtracting the bit pattern of
     * sqrt(2)/2 (0x3F3504F3) carries into the exponent field exactly when the
     * significand is >= sqrt(2), so the exponent field is e and the low 23
     * bits, added back to the pattern, are f's.  The extra 24 << 23 gives
     * e - 24 directly (u1 = k 2^-24); the shift is arithmetic. */
    const uint32_t t = bits - 0x4B3504F3u;
    const float E = (float)((int)t >> 23);                     /* ln u1 = E ln 2 + ln f */
    const float g = __uint_as_float((t & 0x007FFFFFu) + 0x3F3504F3u) - 1.0f; /* f - 1, exact */
    float p = fmaf(bm::PL8, g, bm::PL7);
    p = fmaf(p, g, bm::PL6);
    p = fmaf(p, g, bm::PL5);
    p = fmaf(p, g, bm::PL4);
    p = fmaf(p, g, bm::PL3);
    p = fmaf(p, g, bm::PL2);
    p = fmaf(p, g, bm::PL1);
    p = fmaf(p, g, bm::PL0);
    const float lnf = fmaf(g * g, p, g);
    const float lnu = fmaf(E, bm::LN2_HI, fmaf(E, bm::LN2_LO, lnf));
    const float x = fmaf(-2.0f, lnu, 0.0f);                    /* -2 ln u1 >= +0 */
    /* x is +0 or a normal number in [2^-23, 34].  The SFU's square-root
     * estimate keeps r within 1 ulp over all 2^24 inputs (against 0.97 ulp
     * for a reciprocal-square-root estimate plus one Newton step, in five
     * instructions more) and gives +0 at x = +0. */
    return sfu_sqrt(x);
}

/* (cos, sin)(2 pi u2), u2 = (w1 >> 8) * 2^-24: quadrant q = round(4 u2),
 * r = 2 u2 - q/2 in [-1/4, 1/4] exactly, then a signed swap by q mod 4.
 * With a = w1 + 2^29 (mod 2^32; adding half a quadrant at bit 29 leaves the
 * low 8 bits alone), q mod 4 is a's top two bits and r = (bits 8..29 of a)
 * 2^-23 - 1/4: one masked conversion (22 significant bits, exact) and one
 * FMA whose exact result is representable.  Sine is negated for q = 2, 3
 * (a's bit 31), cosine for q = 1, 2: bit 31 of a + 2^30, which is a's bit 31
 * xor its bit 30. */
__device__ __forceinline__ float bm_angle_r(uint32_t a)
{
    return fmaf(__uint2float_rn(a & 0x3FFFFF00u), 0x1p-31f, -0.25f);
}
__device__ __forceinline__ void bm_cos_sin_poly(float r, float *sn, float *cs)
{
    const float t = r * r;
    float qs = fmaf(bm::QS3, t, bm::QS2);
    qs = fmaf(qs, t, bm::QS1);
    qs = fmaf(qs, t, bm::QS0);
    *sn = fmaf(r, bm::PI_HI, r * fmaf(t, qs, bm::PI_LO));
    float qc = fmaf(bm::QC4, t, bm::QC3);
    qc = fmaf(qc, t, bm::QC2);
    qc = fmaf(qc, t, bm::QC1);
    qc = fmaf(qc, t, bm::QC0);
    *cs = fmaf(t, qc, 1.0f);
}
/* The quadrant's swap and signs applied to (sin, cos)(pi r) for the word w1. */
__device__ __forceinline__ void bm_quadrant(uint32_t w1, float sn, float cs, float *c, float *s)
{
    const uint32_t a = w1 + (1u << 29), b = w1 + (3u << 29);
    const bool swap = (a >> 30) & 1u;
    const uint32_t vs = __float_as_uint(swap ? cs : sn), vc = __float_as_uint(swap ? sn : cs);
    *s = __uint_as_float(vs ^ (a & 0x80000000u));
    *c = __uint_as_float(vc ^ (b & 0x80000000u));
}
__device__ __forceinline__ void bm_cos_sin(uint32_t w1, float *c, float *s)
{
    float sn, cs;
    bm_cos_sin_poly(bm_angle_r(w1 + (1u << 29)), &sn, &cs);
    bm_quadrant(w1, sn, cs, c, s);
}

/* Box-Muller pair (r cos 2 pi u2, r sin 2 pi u2) from two words. */
__device__ __forceinline__ float2 box_muller_f32(uint32_t w0, uint32_t w1)
{
    const float r = bm_radius(w0);
    float c, s;
    bm_cos_sin(w1, &c, &s);
    return make_float2(r * c, r * s);
}

/* -------------------------------------------------- packed FP32 pairs
 * Blackwell executes FP32 add, multiply and FMA on register pairs
 * (add/mul/fma.rn.f32x2): one instruction, two lanes, each rounded exactly
 * as the scalar operation would be.  The helpers below keep a pair in one
 * 64-bit value (low half lane 0). */
namespace x2 {
__device__ __forceinline__ unsigned long long pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack(unsigned long long v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long splat(float c) { return pack(c, c); }
__device__ __forceinline__ unsigned long long fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
}  // namespace x2

/* Both Box-Muller pairs of a group of four words, (w.x, w.y) and (w.z, w.w),
 * as (z0, z1, z2, z3) bit patterns: the operations of bm_radius and
 * bm_cos_sin done on packed pairs (lane 0 the first pair, lane 1 the
 * second), so the same bits as two box_muller_f32 calls in about two thirds
 * of the instructions. */
__device__ __forceinline__ uint4 box_muller2_f32(uint4 w)
{
    using namespace x2;
    const uint32_t b0 = __float_as_uint(__uint2float_rn((w.x >> 8) + 1u));
    const uint32_t b1 = __float_as_uint(__uint2float_rn((w.z >> 8) + 1u));
    const uint32_t t0 = b0 - 0x4B3504F3u, t1 = b1 - 0x4B3504F3u;          /* see bm_radius */
    const unsigned long long E = pack((float)((int)t0 >> 23), (float)((int)t1 >> 23));
    const unsigned long long g = add(pack(__uint_as_float((t0 & 0x007FFFFFu) + 0x3F3504F3u),
                                          __uint_as_float((t1 & 0x007FFFFFu) + 0x3F3504F3u)),
                                     splat(-1.0f));
    unsigned long long p = fma(splat(bm::PL8), g, splat(bm::PL7));
    p = fma(p, g, splat(bm::PL6));
    p = fma(p, g, splat(bm::PL5));
    p = fma(p, g, splat(bm::PL4));
    p = fma(p, g, splat(bm::PL3));
    p = fma(p, g, splat(bm::PL2));
    p = fma(p, g, splat(bm::PL1));
    p = fma(p, g, splat(bm::PL0));
    const unsigned long long lnf = fma(mul(g, g), p, g);
    const unsigned long long lnu = fma(E, splat(bm::LN2_HI), fma(E, splat(bm::LN2_LO), lnf));
    const float2 xs = unpack(fma(splat(-2.0f), lnu, splat(0.0f)));        /* -2 ln u1 >= +0 */
    const float ra = sfu_sqrt(xs.x), rb = sfu_sqrt(xs.y);
    const unsigned long long r = fma(pack(__uint2float_rn((w.y + (1u << 29)) & 0x3FFFFF00u),
                                          __uint2float_rn((w.w + (1u << 29)) & 0x3FFFFF00u)),
                                     splat(0x1p-31f), splat(-0.25f));
    const unsigned long long t = mul(r, r);
    unsigned long long qs = fma(splat(bm::QS3), t, splat(bm::QS2));
    qs = fma(qs, t, splat(bm::QS1));
    qs = fma(qs, t, splat(bm::QS0));
    const float2 sn = unpack(fma(r, splat(bm::PI_HI), mul(r, fma(t, qs, splat(bm::PI_LO)))));
    unsigned long long qc = fma(splat(bm::QC4), t, splat(bm::QC3));
    qc = fma(qc, t, splat(bm::QC2));
    qc = fma(qc, t, splat(bm::QC1));
    qc = fma(qc, t, splat(bm::QC0));
    const float2 cs = unpack(fma(t, qc, splat(1.0f)));
    float c0, s0, c1, s1;
    bm_quadrant(w.y, sn.x, cs.x, &c0, &s0);
    bm_quadrant(w.w, sn.y, cs.y, &c1, &s1);
    const float2 z01 = unpack(mul(splat(ra), pack(c0, s0)));
    const float2 z23 = unpack(mul(splat(rb), pack(c1, s1)));
    return make_uint4(__float_as_uint(z01.x), __float_as_uint(z01.y), __float_as_uint(z23.x), __float_as_uint(z23.y));
}

/* Cosine half of a Box-Muller pair: r cos(2 pi u2), the first normal. */
__device__ __forceinline__ float box_muller_cos_f32(uint32_t w0, uint32_t w1)
{
    float c, s;
    bm_cos_sin(w1, &c, &s);
    return bm_radius(w0) * c;
}

/* ---------------------------------------------- the walks' Box-Muller map
 *
 * The walk kernels only need their normals to about 1e-6 (positions are
 * checked to 1e-5 after 10^4 steps), so they use a cheaper map from the
 * same words, built on the SFU's estimates (lg2.approx, sqrt.approx,
 * sin.approx, cos.approx, used as PTX instructions).  Measured over every
 * input: the radius is within 5.5e-7 relative of sqrt(-2 ln u1), and the
 * cosine and sine within 3.4e-7 absolute of cos and sin(2 pi u2).  The fills
 * keep the map above (within 3 ulp). */


/* sqrt(-2 ln u1), u1 = ((w0 >> 8) + 1) 2^-24.  With v = 1 - u1 (exact):
 * for v < 1/16, -2 ln(1 - v) = 2 v (1 + v/2 + v^2/3 + v^3/4 + v^4/5 + v^5/6)
 * (the first omitted term is below 1e-8 relative); elsewhere the SFU's
 * log2 estimate, whose absolute error (about 7e-8) would be a large
 * relative error next to u1 = 1.  Both are evaluated and one is selected,
 * so the lanes of a warp never diverge. */
__device__ __forceinline__ float bm_radius_walk(uint32_t w0)
{
    const float u1 = __uint2float_rn((w0 >> 8) + 1u) * 0x1p-24f;
    const float v = 1.0f - u1;
    /* 2 p(v) with the 2 in the coefficients: each FMA of the doubled chain
     * is exactly twice the plain one, so v * p2 = (2 v) p bit for bit, one
     * multiply fewer. */
    float p2 = fmaf(v, 2.0f / 6.0f, 0.4f);
    p2 = fmaf(p2, v, 0.5f);
    p2 = fmaf(p2, v, 2.0f / 3.0f);
    p2 = fmaf(p2, v, 1.0f);
    p2 = fmaf(p2, v, 2.0f);
    const float x_series = v * p2;
    const float x_log = -1.3862943611198906f * sfu_lg2(u1);   /* -2 ln 2 log2(u1) */
    const float x = v < 0.0625f ? x_series : x_log;
    /* The SFU's square-root estimate (sqrt(+0) = +0 at u1 = 1): one
     * instruction, and over all 2^24 inputs the radius stays within 5.5e-7
     * relative (5.8e-7 with x * rsqrt(x)). */
    return sfu_sqrt(x);
}

/* (cos, sin)(2 pi u2), u2 = (w1 >> 8) 2^-24, by an exact half-turn split:
 * 2 pi u2 = h pi + phi, with h = bit 31 of w1 and phi = pi times the next 23
 * bits' fraction, in [0, pi).  Then (cos, sin)(2 pi u2) = (-1)^h (cos, sin)
 * (phi): the SFU's estimates at phi, both negated for h = 1 (one sign bit,
 * so a caller that multiplies by a radius can flip the radius instead).
 * phi's 23 bits stay in place, w1 & 0x7FFFFF00 (exact in FP32), with the
 * 2^-8 folded into the scale.  The split matters for more than range: the
 * estimates have small mean errors, and each enters c and s with opposite
 * signs for h = 0 and h = 1 at the same phi, so the walk's sum of normals
 * carries no drift from them (a walk of 10^4 steps would otherwise move by
 * about 1e-5).  Measured over all 2^24 inputs: 3.6e-7 absolute error, the
 * same as with a quarter-turn (quadrant) split, and no mean error. */
__device__ __forceinline__ void bm_cos_sin_walk(uint32_t w1, float *c, float *s)
{
    const float ph = (float)(w1 & 0x7FFFFF00u) * (0x1p-31f * 3.14159265358979324f);
    const uint32_t flip = w1 & 0x80000000u;
    *c = __uint_as_float(__float_as_uint(sfu_cos(ph)) ^ flip);
    *s = __uint_as_float(__float_as_uint(sfu_sin(ph)) ^ flip);
}

__device__ __forceinline__ float2 box_muller_walk_f32(uint32_t w0, uint32_t w1)
{
    const float r = bm_radius_walk(w0);
    float c, s;
    bm_cos_sin_walk(w1, &c, &s);
    return make_float2(r * c, r * s);
}

__device__ __forceinline__ float box_muller_cos_walk_f32(uint32_t w0, uint32_t w1)
{
    float c, s;
    bm_cos_sin_walk(w1, &c, &s);
    return bm_radius_walk(w0) * c;
}

/* ------------------------------------------------ engine-style generators */

/* Sequential draw interface of the paper's API (§3; Fig. 1 builds
 * `RNG rng(p.pid, counter)` in the thread and calls `draw_double2()`):
 * construct from (seed, counter), then draw words and values in order.
 *
 * Every class has the same draws, each taking its words from the front of
 * the stream: operator() one word; uniform_f32 one word; uniform_f64 two
 * words (first one high); normal2_f32 two words (one Box-Muller pair, the
 * fills' map); uniform2_f32 and uniform2_f64 two draws of the single form.
 * So a thread's values are those a bulk fill of the same stream writes, in
 * the order drawn.
 *
 * Period: a stream holds 2^32 words (§3).  The random-access engines count
 * words in 32 bits, so past word 2^32 - 1 they wrap to word 0 of the same
 * stream; they also start at any word (`first_word`, a skip-ahead).  Tyche
 * is sequential: it starts at word 0 and does not wrap (past 2^32 words its
 * state simply runs on); drawing that many from one stream is outside the
 * paper's contract. */
template <class G>
class EngineDraws {
  public:
    __device__ __forceinline__ float uniform_f32() { return u01_f32(self()()); }
    __device__ __forceinline__ double uniform_f64()
    {
        const uint32_t h = self()();
        return u01_f64(h, self()());
    }
    __device__ __forceinline__ float2 uniform2_f32()
    {
        const float a = uniform_f32();
        return make_float2(a, uniform_f32());
    }
    __device__ __forceinline__ double2 uniform2_f64()
    {
        const double a = uniform_f64();
        return make_double2(a, uniform_f64());
    }
    __device__ __forceinline__ float2 normal2_f32()
    {
        const uint32_t a = self()();
        return box_muller_f32(a, self()());
    }

  private:
    ORAND_HD G &self() { return *static_cast<G *>(this); }
};

/* Philox and Threefry: word w of the stream is lane w mod 4 of the block
 * with counter (w div 4, counter, 0, 0); a 4-word buffer holds the current
 * block. */
template <class BlockFn>
class BlockEngine : public EngineDraws<BlockEngine<BlockFn>> {
  public:
    ORAND_HD BlockEngine(uint64_t seed, uint32_t counter, uint32_t first_word = 0)
        : key_(seed), counter_(counter), pos_(first_word)
    {
        if (pos_ & 3u) buf_ = BlockFn::block(key_, counter_, pos_ >> 2);
    }
    ORAND_HD uint32_t operator()()
    {
        const uint32_t lane = pos_ & 3u;
        if (lane == 0u) buf_ = BlockFn::block(key_, counter_, pos_ >> 2);
        ++pos_;
        return lane == 0u ? buf_.x : lane == 1u ? buf_.y : lane == 2u ? buf_.z : buf_.w;
    }
    /* Index of the next word within the stream. */
    ORAND_HD uint32_t position() const { return pos_; }

  private:
    uint64_t key_;
    uint32_t counter_, pos_;
    uint4 buf_ = {0u, 0u, 0u, 0u};
};

struct PhiloxBlockFn {
    ORAND_HD static uint4 block(uint64_t key64, uint32_t counter, uint32_t b) { return philox_block(key64, counter, b); }
};
struct ThreefryBlockFn {
    ORAND_HD static uint4 block(uint64_t key64, uint32_t counter, uint32_t b)
    {
        return threefry_block(key64, counter, b);
    }
};

using Philox = BlockEngine<PhiloxBlockFn>;
using Threefry = BlockEngine<ThreefryBlockFn>;

/* Squares: word w = squares32((counter << 32) | w, fmix64(seed) | 1). */
class Squares : public EngineDraws<Squares> {
  public:
    ORAND_HD Squares(uint64_t seed, uint32_t counter, uint32_t first_word = 0)
        : key_(squares_key(seed)), counter_(counter), pos_(first_word) {}
    ORAND_HD uint32_t operator()() { return squares32(((uint64_t)counter_ << 32) | pos_++, key_); }
    ORAND_HD uint32_t position() const { return pos_; }

  private:
    uint64_t key_;
    uint32_t counter_, pos_;
};

/* Tyche: 20 MIX from (seed, counter), then word w = b after MIX w + 1. */
class Tyche : public EngineDraws<Tyche> {
  public:
    ORAND_HD Tyche(uint64_t seed, uint32_t counter) : s_(tyche_init(seed, counter)) {}
    ORAND_HD uint32_t operator()() { return tyche_next(s_); }

  private:
    TycheState s_;
};

}  // namespace orand
