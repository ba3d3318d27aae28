// orand_engine_draws: the device header's engine classes run on the GPU.
// Each thread builds its generator in registers from (its key, counter), as
// the paper's Fig. 1 kernel does with `RNG rng(p.pid, counter)`, and draws
// a fixed interleaving of every value type the classes offer (§3), so that
// the whole per-thread interface is compiled for sm_103a and can be checked
// against an independent implementation.
#include "common.cuh"
#include "orand_device.cuh"

namespace orand_impl {

struct EngineRecord {  // one round of draws, 48 bytes (see orand.h)
    double2 d2;
    double d1;
    float2 n;
    float2 u2;
    uint32_t w;
    float u;
};
static_assert(sizeof(EngineRecord) == 48, "record layout");

template <class E>
__device__ __forceinline__ E make_engine(uint64_t key, uint32_t counter, uint32_t first_word)
{
    if constexpr (__is_same(E, orand::Tyche)) return E(key, counter);
    else return E(key, counter, first_word);
}

template <class E>
__global__ void __launch_bounds__(256) engine_draws_kernel(uint64_t seed, uint32_t counter, uint32_t first_word,
                                                           uint64_t n_threads, uint32_t n_rounds,
                                                           EngineRecord *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_threads; t += stride) {
        E g = make_engine<E>(seed ^ t, counter, first_word);
        EngineRecord *o = out + t * n_rounds;
        for (uint32_t r = 0; r < n_rounds; ++r) {
            EngineRecord rec;
            rec.w = g();
            rec.d1 = g.uniform_f64();
            rec.n = g.normal2_f32();
            rec.u = g.uniform_f32();
            rec.d2 = g.uniform2_f64();
            rec.u2 = g.uniform2_f32();
            o[r] = rec;
        }
    }
}

}  // namespace orand_impl

extern "C" orand_status_t orand_engine_draws(orand_gen_t gen, uint64_t seed, uint32_t counter, uint32_t first_word,
                                             uint64_t n_threads, uint32_t n_rounds, void *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_engine_draws");
    using namespace orand_impl;
    if ((unsigned)gen > ORAND_TYCHE) return ORAND_ERR_INVALID_ARG;
    if (gen == ORAND_TYCHE && first_word != 0) return ORAND_ERR_INVALID_ARG;
    if (gen == ORAND_TYCHE && (uint64_t)n_rounds * 12 > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    uint64_t records, bytes;
    if (mul_overflows(n_threads, n_rounds, &records) || mul_overflows(records, sizeof(EngineRecord), &bytes))
        return ORAND_ERR_OVERFLOW;
    if (records == 0) return ORAND_OK;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)out % 16) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    orand_status_t st = current_device(&info);
    if (st != ORAND_OK) return st;
    const unsigned grid = grid_for(n_threads, 256, info.sm_count, info.max_threads_per_sm / 256);
    EngineRecord *o = (EngineRecord *)out;
    switch (gen) {
    case ORAND_PHILOX4x32_10:
        engine_draws_kernel<orand::Philox><<<grid, 256, 0, stream>>>(seed, counter, first_word, n_threads, n_rounds, o);
        break;
    case ORAND_THREEFRY4x32_20:
        engine_draws_kernel<orand::Threefry><<<grid, 256, 0, stream>>>(seed, counter, first_word, n_threads, n_rounds,
                                                                       o);
        break;
    case ORAND_SQUARES32:
        engine_draws_kernel<orand::Squares><<<grid, 256, 0, stream>>>(seed, counter, first_word, n_threads, n_rounds, o);
        break;
    default:
        engine_draws_kernel<orand::Tyche><<<grid, 256, 0, stream>>>(seed, counter, first_word, n_threads, n_rounds, o);
        break;
    }
    return launch_status();
}
