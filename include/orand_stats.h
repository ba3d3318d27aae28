/* orand_stats.h -- the parallel-stream correlation harness of the paper's
 * statistical evaluation (§5, Statistical Evaluation), on the GPU.
 *
 * Following the procedure §5 adopts (Anderson et al., HOOMD-blue 2020):
 * many particles each draw a short micro-stream per iteration, the
 * micro-streams are concatenated particle after particle, and the
 * concatenated stream grows iteration after iteration; the whole stream is
 * then checked for correlations between the particles' streams.  The paper
 * feeds it to TestU01 and PractRand.  This library counts three classical
 * statistics on the GPU instead (Knuth, TAOCP vol. 2, §3.3.2): tuple
 * frequencies, the gap test and birthday spacings.  Only integer counts are
 * produced; p-values come from the counts on the host.
 *
 * Conventions as in orand.h: device pointers, asynchronous on `stream`,
 * arguments validated before any launch, ORAND_OK or a negative status.
 * Count arrays are ACCUMULATED into (+=), so a long stream can be fed in
 * pieces; the caller zeroes them first.
 */
#ifndef ORAND_STATS_H
#define ORAND_STATS_H

#include "orand.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The concatenated micro-stream (§5, parallel-stream tests).  For
 * iteration j < n_counters and particle s < n_streams, the `draws` words of
 * the stream with key seed ^ s and counter counter_first + j (the same words
 * orand_fill_u32 gives that stream) land at
 *     out[(j * n_streams + s) * draws + k],  k < draws.
 * draws: 1..64.  counter_first + n_counters - 1 must not pass 2^32 - 1.
 * out: n_counters * n_streams * draws u32, 4-byte aligned.
 * Errors: INVALID_ARG (unknown gen, draws out of range, NULL out with work),
 * OVERFLOW (counter range wraps, size product overflows 2^62 words),
 * ALIGNMENT, CUDA. */
orand_status_t orand_fill_micro_streams(orand_gen_t gen, uint64_t seed, uint64_t n_streams, uint32_t draws,
                                        uint32_t counter_first, uint32_t n_counters, uint32_t *out,
                                        cudaStream_t stream);

/* Tuple frequencies (the serial test).  Tuple m is words[m*stride + i],
 * i < t, for every m with m*stride + t <= n_words; its cell is the fields
 * (w >> shift) & (2^bits - 1) of its words, the first word in the highest
 * position.  counts[cell] += 1 for each tuple.
 * t: 1..4, bits >= 1, t * bits <= 14 (2^14 cells), shift + bits <= 32,
 * stride >= 1.  counts: 2^(t*bits) uint64, 8-byte aligned.
 * Errors: INVALID_ARG, ALIGNMENT, CUDA. */
orand_status_t orand_stat_tuples(const uint32_t *words, uint64_t n_words, uint32_t t, uint32_t bits,
                                 uint32_t shift, uint32_t stride, uint64_t *counts, cudaStream_t stream);

/* The "no hit yet" value of the gap test's carry. */
#define ORAND_GAP_NO_HIT UINT64_MAX

/* Gap test.  Word w is a hit when lo <= w < hi (hi <= 2^32).  Every hit
 * after the first closes a gap, the number of non-hit words since the
 * previous hit: counts[min(gap, t_max)] += 1.  *carry (device memory) holds
 * the number of non-hit words after the last hit of the stream's earlier
 * pieces, or ORAND_GAP_NO_HIT before the first hit; the call reads it and
 * leaves the value for the next piece, so pieces fed in order give the
 * counts of the whole stream.  Initialise it to ORAND_GAP_NO_HIT.
 * t_max: 1..4096.  counts: t_max + 1 uint64; counts and carry 8-byte
 * aligned.  ctx supplies scratch of 16 bytes per 8192 words.
 * Errors: INVALID_ARG (lo >= hi, hi > 2^32, t_max out of range, NULL
 * pointers), ALIGNMENT, ALLOC, CUDA. */
orand_status_t orand_stat_gaps(orand_ctx_t ctx, const uint32_t *words, uint64_t n_words, uint64_t lo, uint64_t hi,
                               uint32_t t_max, uint64_t *counts, uint64_t *carry, cudaStream_t stream);

/* Birthday spacings (Marsaglia; Knuth's form).  Sample q takes the
 * n = 2^log2_n words words[q*n .. q*n + n - 1] (only whole samples); each
 * word's birthday is (w >> shift) & (2^bits - 1) in a year of m = 2^bits
 * days.  With the birthdays sorted, Y(1) <= ... <= Y(n), the n spacings are
 * Y(i+1) - Y(i) and Y(1) + m - Y(n); sorted, R = the number of j with
 * S(j) == S(j-1).  counts[min(R, r_max)] += 1 per sample.  For a good
 * generator R has mean n(n-1)^2/(4m) - n(n-1)^2(n-2)^2/(18m^2) (equal pairs
 * minus triples; Knuth's n^3/(4m) to first order) and is close to Poisson.
 * log2_n: 2..12, bits: 1..32, shift + bits <= 32, r_max: 1..4096.
 * counts: r_max + 1 uint64, 8-byte aligned.
 * Errors: INVALID_ARG, ALIGNMENT, CUDA. */
orand_status_t orand_stat_birthday(const uint32_t *words, uint64_t n_words, uint32_t log2_n, uint32_t bits,
                                   uint32_t shift, uint32_t r_max, uint64_t *counts, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* ORAND_STATS_H */
