// Group -> values: the word-to-value maps and the stores shared by the bulk
// fill and the ragged batcher, so both paths emit identical bits.  A group is
// four consecutive generator words 4b..4b+3 of one stream; it becomes 4
// values (u32, FP32 uniform, FP32 normal as two Box-Muller pairs) or 2
// values (FP64 uniform, high word first).
#pragma once

#include "orand.h"
#include "orand_device.cuh"

namespace orand_impl {

// Four words 4b..4b+3 of the stream (key64, counter) for the random-access
// generators.
template <int GEN>
__device__ __forceinline__ uint4 group_words(uint64_t key64, uint32_t counter, uint32_t b)
{
    if (GEN == ORAND_PHILOX4x32_10) return orand::philox_block(key64, counter, b);
    if (GEN == ORAND_THREEFRY4x32_20) return orand::threefry_block(key64, counter, b);
    return orand::squares_block(orand::squares_key(key64), counter, b);
}

// Values per group for a dtype.
template <int DT>
struct Vals {
    static constexpr uint32_t V = (DT == ORAND_F64_UNIFORM) ? 2u : 4u;
};

// The group's values as a 16-byte bit pattern, in memory order: 4 x u32,
// 4 x f32 (uniform, or normals z0 z1 of pair (w.x, w.y) then of (w.z, w.w),
// both pairs evaluated on packed FP32 pairs),
// or 2 x f64 (from (w.x, w.y) and (w.z, w.w)).  BRANCH_FREE selects the
// branch-free FP64 map (same bits) for latency-bound callers.
template <int DT, bool BRANCH_FREE = false>
__device__ __forceinline__ uint4 group_bits(uint4 w)
{
    if (DT == ORAND_U32) return w;
    if (DT == ORAND_F32_UNIFORM) {
        // u01_f32 on each word, the exact scaling by 2^-24 done on packed pairs.
        using namespace orand::x2;
        const float2 a = unpack(mul(pack(__uint2float_rn(w.x >> 8), __uint2float_rn(w.y >> 8)), splat(0x1p-24f)));
        const float2 b = unpack(mul(pack(__uint2float_rn(w.z >> 8), __uint2float_rn(w.w >> 8)), splat(0x1p-24f)));
        return make_uint4(__float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(b.x), __float_as_uint(b.y));
    }
    if (DT == ORAND_F64_UNIFORM) {
        if (!BRANCH_FREE && __builtin_expect(min(w.x, w.z) >= (1u << 20), 1)) {
            // Both high words >= 2^20 (all but about 2^-11 of the groups):
            // the short exact form for both values, one test for the pair.
            const uint2 a = orand::u01_f64_bits_hi20(w.x, w.y), b = orand::u01_f64_bits_hi20(w.z, w.w);
            return make_uint4(a.y, a.x, b.y, b.x);
        }
        const double da = BRANCH_FREE ? orand::u01_f64_nb(w.x, w.y) : orand::u01_f64_general(w.x, w.y);
        const double db = BRANCH_FREE ? orand::u01_f64_nb(w.z, w.w) : orand::u01_f64_general(w.z, w.w);
        const unsigned long long a = __double_as_longlong(da);
        const unsigned long long b = __double_as_longlong(db);
        return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    }
    return orand::box_muller2_f32(w);
}

// Masked element stores of a group's bits: values j0 + i for i < V and
// j0 + i < limit, at dst (the address of value j0).
template <int DT>
__device__ __forceinline__ void store_bits_masked(char *dst, uint64_t j0, uint64_t limit, uint4 v)
{
    if (DT == ORAND_F64_UNIFORM) {
        unsigned long long *o = (unsigned long long *)dst;
        if (j0 < limit) o[0] = ((unsigned long long)v.y << 32) | v.x;
        if (j0 + 1 < limit) o[1] = ((unsigned long long)v.w << 32) | v.z;
    } else {
        uint32_t *o = (uint32_t *)dst;
        const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (j0 + i < limit) o[i] = e[i];
    }
}

// Write the values of group b of stream s.  VEC: one 16-byte store at the
// group's contiguous slot g.  Otherwise: element stores masked to j < dps.
template <int DT, bool VEC>
__device__ __forceinline__ void store_group(void *out, uint64_t g, uint64_t s, uint32_t b, uint64_t dps,
                                            uint4 w)
{
    const uint4 v = group_bits<DT>(w);
    if (VEC) {
        reinterpret_cast<uint4 *>(out)[g] = v;
    } else {
        constexpr uint32_t V = Vals<DT>::V;
        constexpr uint32_t E = DT == ORAND_F64_UNIFORM ? 8u : 4u;
        const uint64_t j0 = (uint64_t)b * V;
        store_bits_masked<DT>((char *)out + (s * dps + j0) * E, j0, dps, v);
    }
}

}  // namespace orand_impl
