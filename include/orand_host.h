/* orand_host.h -- the generators on the host, and the paper's host
 * micro-benchmark (§5, Performance Benchmarks: single-threaded generation
 * time for streams of varying length on the CPU, against std::mt19937).
 *
 * The host streams come from the same generator source as the device path,
 * so orand_host_fill_u32 gives the bits orand_fill_u32 writes on the GPU for
 * the same arguments.  Host memory only, single-threaded, synchronous.
 * These calls are for host programs and the micro-benchmark; the device
 * entry points never use them.
 */
#ifndef ORAND_HOST_H
#define ORAND_HOST_H

#include "orand.h"

#ifdef __cplusplus
extern "C" {
#endif

/* std::mt19937 as the micro-benchmark's baseline generator id. */
#define ORAND_HOST_MT19937 100

/* out[s * draws_per_stream + j] = word j of the stream with key seed ^ s and
 * counter `counter` (the layout of orand_fill_u32), computed on the host.
 * out: host memory, 4-byte aligned.
 * Errors: INVALID_ARG (unknown gen, NULL out with work), OVERFLOW (a stream
 * longer than 2^32 words, or the size product overflows), ALIGNMENT. */
orand_status_t orand_host_fill_u32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                   uint64_t draws_per_stream, uint32_t *out);

/* n words of one stream (key seed, counter `counter`) drawn on the host
 * through the device header's engine classes, starting at word first_word:
 * out[i] = word (first_word + i) mod 2^32 for the random-access generators,
 * which wrap at their 2^32-word period (§3).  Tyche is sequential:
 * first_word must be 0 and n at most 2^32.  out: host memory, 4-byte
 * aligned.
 * Errors: INVALID_ARG (unknown gen, NULL out with n > 0, first_word != 0
 * for Tyche), OVERFLOW (Tyche past 2^32 words), ALIGNMENT. */
orand_status_t orand_host_engine_words(orand_gen_t gen, uint64_t seed, uint32_t counter, uint32_t first_word,
                                       uint64_t n, uint32_t *out);

/* The micro-benchmark.  For each lengths[k] (1..2^32), construct fresh
 * generators (seed r = 0, 1, 2, ..., counter 0; std::mt19937 seeded with r
 * for gen = ORAND_HOST_MT19937) and draw lengths[k] words from each, about
 * words_per_length words in all (at least one stream); ns_per_stream[k] is
 * the mean wall time per stream, construction included, as the paper
 * measures it.  Every word is XOR-folded into *sink so no draw can be
 * skipped.  Runs on the calling thread.
 * Errors: INVALID_ARG (unknown gen, a length of 0 or above 2^32, NULL
 * pointers with n_lengths > 0). */
orand_status_t orand_host_microbench(int gen, const uint64_t *lengths, uint32_t n_lengths, uint64_t words_per_length,
                                     double *ns_per_stream, uint32_t *sink);

#ifdef __cplusplus
}
#endif

#endif /* ORAND_HOST_H */
