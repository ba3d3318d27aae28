// Host-side generation and the paper's host micro-benchmark (§5: single-
// threaded generation speed for streams of varying length, against
// std::mt19937).  The generator cores are the same source as the device
// path (orand_device.cuh, compiled here for the CPU), so a host stream has
// the bits of the device fill of the same (seed, counter).  These entry
// points serve host programs and the micro-benchmark; no device entry point
// calls them.
#include <chrono>
#include <random>

#include "orand.h"
#include "orand_device.cuh"
#include "orand_host.h"

namespace {

template <class Engine>
void host_fill(uint64_t seed, uint32_t counter, uint64_t n_streams, uint64_t dps, uint32_t *out)
{
    for (uint64_t s = 0; s < n_streams; ++s) {
        Engine e(seed ^ s, counter);
        uint32_t *o = out + s * dps;
        for (uint64_t j = 0; j < dps; ++j) o[j] = e();
    }
}

// Time `reps` fresh streams of `len` words each; returns ns per stream and
// folds every word into *acc so no draw can be elided.
template <class Make>
double time_streams(Make make, uint64_t len, uint64_t reps, uint32_t *acc)
{
    uint32_t x = 0;
    const auto t0 = std::chrono::steady_clock::now();
    for (uint64_t r = 0; r < reps; ++r) {
        auto e = make(r);
        for (uint64_t i = 0; i < len; ++i) x ^= e();
    }
    const auto t1 = std::chrono::steady_clock::now();
    *acc ^= x;
    return std::chrono::duration<double, std::nano>(t1 - t0).count() / (double)reps;
}

}  // namespace

extern "C" {

orand_status_t orand_host_engine_words(orand_gen_t gen, uint64_t seed, uint32_t counter, uint32_t first_word,
                                       uint64_t n, uint32_t *out)
{
    if ((unsigned)gen > ORAND_TYCHE) return ORAND_ERR_INVALID_ARG;
    if (gen == ORAND_TYCHE && first_word != 0) return ORAND_ERR_INVALID_ARG;
    if (gen == ORAND_TYCHE && n > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    if (n == 0) return ORAND_OK;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)out % 4) return ORAND_ERR_ALIGNMENT;
    switch (gen) {
    case ORAND_PHILOX4x32_10: {
        orand::Philox e(seed, counter, first_word);
        for (uint64_t i = 0; i < n; ++i) out[i] = e();
        break;
    }
    case ORAND_THREEFRY4x32_20: {
        orand::Threefry e(seed, counter, first_word);
        for (uint64_t i = 0; i < n; ++i) out[i] = e();
        break;
    }
    case ORAND_SQUARES32: {
        orand::Squares e(seed, counter, first_word);
        for (uint64_t i = 0; i < n; ++i) out[i] = e();
        break;
    }
    default: {
        orand::Tyche e(seed, counter);
        for (uint64_t i = 0; i < n; ++i) out[i] = e();
        break;
    }
    }
    return ORAND_OK;
}

orand_status_t orand_host_fill_u32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                   uint64_t draws_per_stream, uint32_t *out)
{
    if ((unsigned)gen > ORAND_TYCHE) return ORAND_ERR_INVALID_ARG;
    if (draws_per_stream > (1ull << 32)) return ORAND_ERR_OVERFLOW;  // a stream has 2^32 words
    if (n_streams != 0 && draws_per_stream > UINT64_MAX / n_streams) return ORAND_ERR_OVERFLOW;
    if (n_streams == 0 || draws_per_stream == 0) return ORAND_OK;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)out % 4) return ORAND_ERR_ALIGNMENT;
    switch (gen) {
    case ORAND_PHILOX4x32_10: host_fill<orand::Philox>(seed, counter, n_streams, draws_per_stream, out); break;
    case ORAND_THREEFRY4x32_20: host_fill<orand::Threefry>(seed, counter, n_streams, draws_per_stream, out); break;
    case ORAND_SQUARES32: host_fill<orand::Squares>(seed, counter, n_streams, draws_per_stream, out); break;
    default: host_fill<orand::Tyche>(seed, counter, n_streams, draws_per_stream, out); break;
    }
    return ORAND_OK;
}

orand_status_t orand_host_microbench(int gen, const uint64_t *lengths, uint32_t n_lengths, uint64_t words_per_length,
                                     double *ns_per_stream, uint32_t *sink)
{
    if (!((gen >= ORAND_PHILOX4x32_10 && gen <= ORAND_TYCHE) || gen == ORAND_HOST_MT19937))
        return ORAND_ERR_INVALID_ARG;
    if (n_lengths == 0) return ORAND_OK;
    if (lengths == nullptr || ns_per_stream == nullptr || sink == nullptr) return ORAND_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < n_lengths; ++k)
        if (lengths[k] == 0 || lengths[k] > (1ull << 32)) return ORAND_ERR_INVALID_ARG;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < n_lengths; ++k) {
        const uint64_t len = lengths[k];
        const uint64_t reps = words_per_length / len > 0 ? words_per_length / len : 1;
        double ns;
        switch (gen) {
        case ORAND_PHILOX4x32_10:
            ns = time_streams([](uint64_t r) { return orand::Philox(r, 0u); }, len, reps, &acc);
            break;
        case ORAND_THREEFRY4x32_20:
            ns = time_streams([](uint64_t r) { return orand::Threefry(r, 0u); }, len, reps, &acc);
            break;
        case ORAND_SQUARES32:
            ns = time_streams([](uint64_t r) { return orand::Squares(r, 0u); }, len, reps, &acc);
            break;
        case ORAND_TYCHE:
            ns = time_streams([](uint64_t r) { return orand::Tyche(r, 0u); }, len, reps, &acc);
            break;
        default:
            ns = time_streams([](uint64_t r) { return std::mt19937((uint32_t)r); }, len, reps, &acc);
            break;
        }
        ns_per_stream[k] = ns;
    }
    *sink = acc;
    return ORAND_OK;
}

}  // extern "C"
