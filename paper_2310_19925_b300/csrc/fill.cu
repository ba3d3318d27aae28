// Bulk fill kernels: n_streams x draws_per_stream values, stream-major,
// stream s keyed by seed ^ s (one stream per processing element, §3 of the
// paper).  Write-only and HBM-bound for Philox; integer-pipe-bound for the
// longer round functions.
//
// Work unit: a "group" of four consecutive generator words of one stream
// (one Philox/Threefry block, four Squares evaluations, four Tyche steps),
// which becomes 16 bytes of output (4 x u32/f32/normal or 2 x f64).  In
// the vectorised path consecutive threads own consecutive groups, so every
// warp store is one fully coalesced 512-byte row; the grid is sized to the
// resident capacity of the 148 SMs and strides over the groups.
#include "common.cuh"
#include "orand_device.cuh"
#include "values.cuh"

namespace orand_impl {

struct FillArgs {
    uint64_t seed;
    uint64_t n_streams;
    uint64_t dps;         // values per stream
    uint64_t n_groups;    // n_streams * G
    uint64_t stride_div;  // grid threads / G
    uint32_t stride_mod;  // grid threads % G
    uint32_t G;           // groups per stream
    uint32_t counter;
    void *out;
};

// Random-access generators: grid-stride over groups; (s, b) advance
// incrementally so the loop needs no 64-bit division.
template <int GEN, int DT, bool VEC>
__global__ void __launch_bounds__(256) fill_random_access_kernel(FillArgs a)
{
    uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_groups) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t s = g / a.G;
    uint32_t b = (uint32_t)(g - s * a.G);
    for (;;) {
        const uint4 w = group_words<GEN>(a.seed ^ s, a.counter, b);
        store_group<DT, VEC>(a.out, g, s, b, a.dps, w);
        g += stride;
        if (g >= a.n_groups) break;
        s += a.stride_div;
        b += a.stride_mod;
        if (b >= a.G) { b -= a.G; ++s; }
    }
}

// Tyche is sequential within a stream: one thread walks one whole stream.
template <int DT, bool VEC>
__global__ void __launch_bounds__(256) fill_tyche_kernel(FillArgs a)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_streams; s += stride) {
        orand::TycheState st = orand::tyche_init(a.seed ^ s, a.counter);
        for (uint32_t b = 0; b < a.G; ++b) {
            uint4 w;
            w.x = orand::tyche_next(st);
            w.y = orand::tyche_next(st);
            w.z = orand::tyche_next(st);
            w.w = orand::tyche_next(st);
            store_group<DT, VEC>(a.out, s * a.G + b, s, b, a.dps, w);
        }
    }
}

template <int GEN, int DT, bool VEC>
static void launch_one(const FillArgs &a, unsigned grid, cudaStream_t stream)
{
    if (GEN == ORAND_TYCHE)
        fill_tyche_kernel<DT, VEC><<<grid, 256, 0, stream>>>(a);
    else
        fill_random_access_kernel<GEN, DT, VEC><<<grid, 256, 0, stream>>>(a);
}

template <int GEN, int DT>
static void launch_dt(const FillArgs &a, bool vec, unsigned grid, cudaStream_t stream)
{
    if (vec) launch_one<GEN, DT, true>(a, grid, stream);
    else launch_one<GEN, DT, false>(a, grid, stream);
}

template <int GEN>
static void launch_gen(int dt, const FillArgs &a, bool vec, unsigned grid, cudaStream_t stream)
{
    switch (dt) {
    case ORAND_U32: launch_dt<GEN, ORAND_U32>(a, vec, grid, stream); break;
    case ORAND_F32_UNIFORM: launch_dt<GEN, ORAND_F32_UNIFORM>(a, vec, grid, stream); break;
    case ORAND_F64_UNIFORM: launch_dt<GEN, ORAND_F64_UNIFORM>(a, vec, grid, stream); break;
    default: launch_dt<GEN, ORAND_F32_NORMAL>(a, vec, grid, stream); break;
    }
}

// Generator words a stream of dps values of dtype dt consumes.
static bool stream_words(int dt, uint64_t dps, uint64_t *words)
{
    if (dt == ORAND_F64_UNIFORM) return !mul_overflows(dps, 2, words);
    if (dt == ORAND_F32_NORMAL) { *words = (dps / 2 + (dps & 1)) * 2; return true; }
    *words = dps;
    return true;
}

orand_status_t fill_validate(int gen, int dt, uint64_t n_streams, uint64_t dps, const void *out,
                             uint64_t *n_values)
{
    if (gen < 0 || gen > 3 || dt < 0 || dt > 3) return ORAND_ERR_INVALID_ARG;
    uint64_t n, bytes, words;
    if (mul_overflows(n_streams, dps, &n)) return ORAND_ERR_OVERFLOW;
    const uint64_t elem = dt == ORAND_F64_UNIFORM ? 8 : 4;
    if (mul_overflows(n, elem, &bytes)) return ORAND_ERR_OVERFLOW;
    if (!stream_words(dt, dps, &words) || words > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    *n_values = n;
    if (n == 0) return ORAND_OK;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)out % elem) return ORAND_ERR_ALIGNMENT;
    return ORAND_OK;
}

orand_status_t fill_launch(int gen, int dt, uint64_t seed, uint32_t counter, uint64_t n_streams, uint64_t dps,
                           void *out, cudaStream_t stream)
{
    uint64_t n = 0;
    orand_status_t st = fill_validate(gen, dt, n_streams, dps, out, &n);
    if (st != ORAND_OK || n == 0) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;

    const uint32_t V = dt == ORAND_F64_UNIFORM ? 2u : 4u;
    FillArgs a;
    a.seed = seed;
    a.counter = counter;
    a.n_streams = n_streams;
    a.dps = dps;
    a.G = (uint32_t)ceil_div(dps, V);
    a.n_groups = n_streams * a.G;
    a.out = out;
    const bool vec = (dps % V == 0) && ((uintptr_t)out % 16 == 0);
    const uint64_t items = gen == ORAND_TYCHE ? n_streams : a.n_groups;
    const unsigned grid = grid_for(items, 256, info.sm_count, info.max_threads_per_sm / 256);
    const uint64_t threads = (uint64_t)grid * 256u;
    a.stride_div = threads / a.G;
    a.stride_mod = (uint32_t)(threads % a.G);

    switch (gen) {
    case ORAND_PHILOX4x32_10: launch_gen<ORAND_PHILOX4x32_10>(dt, a, vec, grid, stream); break;
    case ORAND_THREEFRY4x32_20: launch_gen<ORAND_THREEFRY4x32_20>(dt, a, vec, grid, stream); break;
    case ORAND_SQUARES32: launch_gen<ORAND_SQUARES32>(dt, a, vec, grid, stream); break;
    default: launch_gen<ORAND_TYCHE>(dt, a, vec, grid, stream); break;
    }
    return launch_status();
}

}  // namespace orand_impl

extern "C" {

orand_status_t orand_fill(orand_gen_t gen, orand_dtype_t dtype, uint64_t seed, uint32_t counter,
                          uint64_t n_streams, uint64_t draws_per_stream, void *out, cudaStream_t stream)
{
    return orand_impl::fill_launch((int)gen, (int)dtype, seed, counter, n_streams, draws_per_stream, out,
                                   stream);
}

orand_status_t orand_fill_u32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                              uint64_t draws_per_stream, uint32_t *out, cudaStream_t stream)
{
    return orand_impl::fill_launch((int)gen, ORAND_U32, seed, counter, n_streams, draws_per_stream, out, stream);
}

orand_status_t orand_fill_uniform_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, float *out, cudaStream_t stream)
{
    return orand_impl::fill_launch((int)gen, ORAND_F32_UNIFORM, seed, counter, n_streams, draws_per_stream,
                                   out, stream);
}

orand_status_t orand_fill_uniform_f64(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, double *out, cudaStream_t stream)
{
    return orand_impl::fill_launch((int)gen, ORAND_F64_UNIFORM, seed, counter, n_streams, draws_per_stream,
                                   out, stream);
}

orand_status_t orand_fill_normal_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                     uint64_t draws_per_stream, float *out, cudaStream_t stream)
{
    return orand_impl::fill_launch((int)gen, ORAND_F32_NORMAL, seed, counter, n_streams, draws_per_stream,
                                   out, stream);
}

}  // extern "C"
