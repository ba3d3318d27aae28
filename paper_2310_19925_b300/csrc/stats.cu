// The parallel-stream correlation harness (§5, Statistical Evaluation) on
// the GPU: the concatenated micro-stream generator and three counting
// kernels (tuple frequencies, gap test, birthday spacings; Knuth, TAOCP
// vol. 2, §3.3.2).  All outputs are integer counts accumulated with atomics,
// so every launch shape gives the same counts.
//
//   micro_stream_kernel  one thread per (iteration, particle) micro-stream;
//                        a warp writes 32 * draws consecutive words.
//   tuple_vec_kernel     non-overlapping tuples of 16-byte-aligned words,
//                        four tuples per thread as t 16-byte loads;
//                        tuple_kernel grid-strides over single tuples
//                        otherwise.  Both keep a per-CTA shared-memory
//                        histogram (a column per lane for up to 256 cells),
//                        flushed once per CTA.
//   gap_span_vec_kernel  one warp per span of 8192 words, read 128 words at a
//                        time (a 16-byte load per lane); a ballot of the
//                        lanes with hits and one shuffle give each hit's
//                        distance to the previous one.  gap_span_kernel
//                        reads 32 words at a time, for words that are not
//                        16-byte aligned.  The span's first and last hit go
//                        to scratch.
//   gap_stitch_kernel    the gap before each span's first hit, from the
//                        previous non-empty span or the carried run.
//   gap_carry_kernel     the run of non-hits after the piece's last hit.
//   birthday_kernel      one CTA per sample: counting sort of the birthdays
//                        in shared memory, distinct spacings counted in
//                        rounds of stores into hash slots and read-backs.
#include "common.cuh"
#include "ctx.cuh"
#include "orand_device.cuh"
#include "orand_stats.h"
#include "values.cuh"

namespace orand_impl {

// ------------------------------------------------------- micro-streams

struct MicroArgs {
    uint64_t seed, n_streams, n_micro;  // n_micro = n_counters * n_streams
    uint64_t stride_div, stride_mod;    // grid stride split into (iterations, particles)
    uint32_t draws, counter_first;
    uint32_t *out;
};

template <int GEN>
__global__ void __launch_bounds__(256) micro_stream_kernel(MicroArgs a)
{
    uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.n_micro) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t j = m / a.n_streams, s = m - j * a.n_streams;
    for (;;) {
        uint32_t *o = a.out + m * a.draws;
        const uint64_t key = a.seed ^ s;
        const uint32_t ctr = a.counter_first + (uint32_t)j;
        if (GEN == ORAND_TYCHE) {
            orand::TycheState st = orand::tyche_init(key, ctr);
            for (uint32_t k = 0; k < a.draws; ++k) o[k] = orand::tyche_next(st);
        } else {
            for (uint32_t b = 0; 4 * b < a.draws; ++b) {
                const uint4 w = group_words<GEN>(key, ctr, b);
                const uint32_t k = 4 * b, left = a.draws - k;
                o[k] = w.x;
                if (left > 1) o[k + 1] = w.y;
                if (left > 2) o[k + 2] = w.z;
                if (left > 3) o[k + 3] = w.w;
            }
        }
        m += stride;
        if (m >= a.n_micro) break;
        j += a.stride_div;
        s += a.stride_mod;
        if (s >= a.n_streams) {
            s -= a.n_streams;
            ++j;
        }
    }
}

// --------------------------------------------------------------- tuples

constexpr int kTupleUnroll = 8;  // tuples per thread per pass, all loads issued before the atomics

// LANES = 32: cells of at most 256, each lane counting in its own column
// (hist[cell * 32 + lane]), so a warp's atomics never share a bank or an
// address.  LANES = 1: one column, for up to 2^14 cells.
template <int LANES>
__global__ void __launch_bounds__(256) tuple_kernel(const uint32_t *__restrict__ w, uint64_t n_tuples, uint32_t t,
                                                    uint32_t bits, uint32_t shift, uint32_t stride, uint32_t cells,
                                                    unsigned long long *__restrict__ counts)
{
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i < cells * LANES; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t mask = (1u << bits) - 1u;  // bits <= 14
    const uint32_t col = LANES == 1 ? 0u : (threadIdx.x & 31u);
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t m0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m0 < n_tuples; m0 += kTupleUnroll * gstride) {
        uint32_t cell[kTupleUnroll];
#pragma unroll
        for (int j = 0; j < kTupleUnroll; ++j) cell[j] = 0u;
        for (uint32_t i = 0; i < t; ++i) {
#pragma unroll
            for (int j = 0; j < kTupleUnroll; ++j) {
                const uint64_t m = m0 + j * gstride;
                const uint32_t x = m < n_tuples ? __ldg(w + m * stride + i) : 0u;
                cell[j] = (cell[j] << bits) | ((x >> shift) & mask);
            }
        }
#pragma unroll
        for (int j = 0; j < kTupleUnroll; ++j)
            if (m0 + j * gstride < n_tuples) atomicAdd(&hist[cell[j] * LANES + col], 1u);
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) {
        unsigned long long v = 0;
        for (uint32_t l = 0; l < (uint32_t)LANES; ++l) v += hist[c * LANES + l];
        if (v) atomicAdd(&counts[c], v);
    }
}

// Non-overlapping tuples (stride = t) of 16-byte-aligned words: four tuples
// (4t words) per thread per pass as t 16-byte loads, two passes' loads in
// flight; the tuples after the last whole group of four go to the first
// threads of block 0.
template <int LANES, int T>
__global__ void __launch_bounds__(256) tuple_vec_kernel(const uint32_t *__restrict__ w, uint64_t n_tuples,
                                                        uint32_t bits, uint32_t shift, uint32_t cells,
                                                        unsigned long long *__restrict__ counts)
{
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i < cells * LANES; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t mask = (1u << bits) - 1u;
    const uint32_t col = LANES == 1 ? 0u : (threadIdx.x & 31u);
    const uint64_t n4 = n_tuples / 4;  // groups of four tuples = T quads of words
    const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
    const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
    auto field = [&](uint32_t x) { return (x >> shift) & mask; };
    auto count_group = [&](const uint4 (&v)[T]) {
        const uint32_t *x = reinterpret_cast<const uint32_t *>(v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t cell = 0;
#pragma unroll
            for (int i = 0; i < T; ++i) cell = (cell << bits) | field(x[k * T + i]);
            atomicAdd(&hist[cell * LANES + col], 1u);
        }
    };
    for (uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < n4; g0 += 2 * gstride) {
        uint4 v0[T], v1[T];
        const bool ok1 = g0 + gstride < n4;
#pragma unroll
        for (int i = 0; i < T; ++i) v0[i] = __ldg(w4 + g0 * T + i);
        if (ok1) {
#pragma unroll
            for (int i = 0; i < T; ++i) v1[i] = __ldg(w4 + (g0 + gstride) * T + i);
        }
        count_group(v0);
        if (ok1) count_group(v1);
    }
    if (blockIdx.x == 0 && threadIdx.x < n_tuples - n4 * 4) {
        const uint64_t m = n4 * 4 + threadIdx.x;
        uint32_t cell = 0;
#pragma unroll
        for (int i = 0; i < T; ++i) cell = (cell << bits) | field(__ldg(w + m * T + i));
        atomicAdd(&hist[cell * LANES + col], 1u);
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < cells; c += blockDim.x) {
        unsigned long long v = 0;
        for (uint32_t l = 0; l < (uint32_t)LANES; ++l) v += hist[c * LANES + l];
        if (v) atomicAdd(&counts[c], v);
    }
}

template <int LANES>
static void launch_tuple_vec(uint32_t t, unsigned grid, size_t smem, cudaStream_t stream, const uint32_t *wp,
                             uint64_t nt, uint32_t bits, uint32_t shift, uint32_t cells, unsigned long long *counts)
{
    switch (t) {
    case 1: tuple_vec_kernel<LANES, 1><<<grid, 256, smem, stream>>>(wp, nt, bits, shift, cells, counts); break;
    case 2: tuple_vec_kernel<LANES, 2><<<grid, 256, smem, stream>>>(wp, nt, bits, shift, cells, counts); break;
    case 3: tuple_vec_kernel<LANES, 3><<<grid, 256, smem, stream>>>(wp, nt, bits, shift, cells, counts); break;
    default: tuple_vec_kernel<LANES, 4><<<grid, 256, smem, stream>>>(wp, nt, bits, shift, cells, counts); break;
    }
}

template <int LANES>
static orand_status_t tuple_smem_opt_in(size_t smem)
{
    ORAND_CUDA_TRY(cudaFuncSetAttribute(tuple_kernel<LANES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ORAND_CUDA_TRY(cudaFuncSetAttribute(tuple_vec_kernel<LANES, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    ORAND_CUDA_TRY(cudaFuncSetAttribute(tuple_vec_kernel<LANES, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    ORAND_CUDA_TRY(cudaFuncSetAttribute(tuple_vec_kernel<LANES, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    ORAND_CUDA_TRY(cudaFuncSetAttribute(tuple_vec_kernel<LANES, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    return ORAND_OK;
}

// ----------------------------------------------------------------- gaps

constexpr uint32_t kGapSpan = 8192;  // words per warp span (256 steps of 32)
constexpr int kGapUnroll = 4;        // steps whose loads are issued together
constexpr uint32_t kNone = 0xFFFFFFFFu;

__device__ __forceinline__ bool gap_hit(uint32_t x, uint64_t lo, uint64_t hi)
{
    return (uint64_t)x >= lo && (uint64_t)x < hi;
}

// The same per span with each lane reading four consecutive words as one
// 16-byte load (the words must be 16-byte aligned): a step covers 128 words;
// a hit's previous hit is in its own lane (a lower word), else in the
// nearest lower lane with a hit (its last hit, by a shuffle), else the
// span's running last hit.
__global__ void __launch_bounds__(256) gap_span_vec_kernel(const uint32_t *__restrict__ w, uint64_t n, uint64_t lo,
                                                           uint64_t hi, uint32_t t_max,
                                                           unsigned long long *__restrict__ counts,
                                                           uint32_t *__restrict__ span_first,
                                                           uint32_t *__restrict__ span_last, uint64_t n_spans)
{
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i <= t_max; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    constexpr uint32_t kSteps = kGapSpan / 128;
    for (uint64_t sp = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); sp < n_spans; sp += warps) {
        const uint64_t start = sp * kGapSpan;
        uint32_t first = kNone, last = kNone;  // span-local offsets, warp-uniform
        for (uint32_t it0 = 0; it0 < kSteps; it0 += 2) {
            if (start + (uint64_t)it0 * 128 >= n) break;
            uint32_t hm[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {  // both steps' loads first
                const uint64_t idx = start + (uint64_t)(it0 + u) * 128 + lane * 4u;
                uint32_t v[4];
                if (idx + 3 < n) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(w + idx));
                    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) v[j] = idx + j < n ? __ldg(w + idx + j) : 0u;
                }
                uint32_t h = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) h |= (idx + j < n && gap_hit(v[j], lo, hi)) ? 1u << j : 0u;
                hm[u] = h;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const uint32_t it = it0 + u;
                const uint32_t h = hm[u];
                const uint32_t mask = __ballot_sync(0xFFFFFFFFu, h != 0u);
                if (mask == 0u) continue;
                // the last hit of the nearest lower lane that has one
                const uint32_t below = mask & ((1u << lane) - 1u);
                const uint32_t src = below ? 31u - __clz(below) : lane;
                const uint32_t hs = __shfl_sync(0xFFFFFFFFu, h, src);
                if (h) {
                    uint32_t prev = below ? it * 128 + src * 4 + (31u - __clz(hs)) : last;
                    for (uint32_t b = h; b; b &= b - 1) {
                        const uint32_t pos = it * 128 + lane * 4 + (__ffs(b) - 1);
                        if (prev != kNone) atomicAdd(&hist[min(pos - prev - 1u, t_max)], 1u);
                        prev = pos;
                    }
                }
                const uint32_t fl = __ffs(mask) - 1, ll = 31u - __clz(mask);
                const uint32_t hf = __shfl_sync(0xFFFFFFFFu, h, fl), hl = __shfl_sync(0xFFFFFFFFu, h, ll);
                if (first == kNone) first = it * 128 + fl * 4 + (__ffs(hf) - 1);
                last = it * 128 + ll * 4 + (31u - __clz(hl));
            }
        }
        if (lane == 0) {
            span_first[sp] = first;
            span_last[sp] = last;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= t_max; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], (unsigned long long)hist[i]);
}

// Per span: gaps between hits inside the span into the histogram, and the
// span-local offsets of its first and last hit (kNone when it has none).
__global__ void __launch_bounds__(256) gap_span_kernel(const uint32_t *__restrict__ w, uint64_t n, uint64_t lo,
                                                       uint64_t hi, uint32_t t_max,
                                                       unsigned long long *__restrict__ counts,
                                                       uint32_t *__restrict__ span_first,
                                                       uint32_t *__restrict__ span_last, uint64_t n_spans)
{
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i <= t_max; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t sp = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); sp < n_spans; sp += warps) {
        const uint64_t start = sp * kGapSpan;
        uint32_t first = kNone, last = kNone;  // span-local offsets, warp-uniform
        for (uint32_t it0 = 0; it0 < kGapSpan / 32; it0 += kGapUnroll) {
            if (start + (uint64_t)it0 * 32 >= n) break;
            bool hits[kGapUnroll];
#pragma unroll
            for (int u = 0; u < kGapUnroll; ++u) {  // loads for the next kGapUnroll steps first
                const uint64_t idx = start + (uint64_t)(it0 + u) * 32 + lane;
                hits[u] = idx < n && gap_hit(__ldg(w + idx), lo, hi);
            }
#pragma unroll
            for (int u = 0; u < kGapUnroll; ++u) {
                const uint32_t it = it0 + u;
                const uint32_t mask = __ballot_sync(0xFFFFFFFFu, hits[u]);
                if (hits[u]) {
                    const uint32_t below = mask & ((1u << lane) - 1u);
                    uint32_t gap = kNone;
                    if (below) gap = lane - (31u - __clz(below)) - 1u;
                    else if (last != kNone) gap = it * 32 + lane - last - 1u;
                    if (gap != kNone) atomicAdd(&hist[min(gap, t_max)], 1u);
                }
                if (mask) {
                    if (first == kNone) first = it * 32 + (__ffs(mask) - 1);
                    last = it * 32 + (31u - __clz(mask));
                }
            }
        }
        if (lane == 0) {
            span_first[sp] = first;
            span_last[sp] = last;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= t_max; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], (unsigned long long)hist[i]);
}

// The gap that ends at each non-empty span's first hit.
__global__ void __launch_bounds__(256) gap_stitch_kernel(const uint32_t *__restrict__ span_first,
                                                         const uint32_t *__restrict__ span_last, uint64_t n_spans,
                                                         const unsigned long long *__restrict__ carry, uint32_t t_max,
                                                         unsigned long long *__restrict__ counts)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_spans || span_first[i] == kNone) return;
    const uint64_t pos = i * kGapSpan + span_first[i];
    uint64_t gap = ORAND_GAP_NO_HIT;
    uint64_t k = i;
    while (k > 0) {  // nearest earlier span with a hit
        --k;
        if (span_last[k] != kNone) {
            gap = pos - (k * kGapSpan + span_last[k]) - 1;
            break;
        }
    }
    if (gap == ORAND_GAP_NO_HIT && *carry != ORAND_GAP_NO_HIT) gap = *carry + pos;
    if (gap != ORAND_GAP_NO_HIT) atomicAdd(&counts[gap < t_max ? gap : t_max], 1ull);
}

// The carry after this piece: non-hits after its last hit, or the old
// carry grown by n when the piece has no hit.  One warp.
__global__ void gap_carry_kernel(const uint32_t *__restrict__ span_last, uint64_t n_spans, uint64_t n,
                                 unsigned long long *__restrict__ carry)
{
    const uint32_t lane = threadIdx.x;
    for (uint64_t end = n_spans; end > 0; end = end > 32 ? end - 32 : 0) {
        const bool ok = lane < end && span_last[end - 1 - lane] != kNone;
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, ok);
        if (mask) {
            const uint64_t k = end - 1 - (uint64_t)(__ffs(mask) - 1);  // the last non-empty span
            if (lane == 0) *carry = n - 1 - (k * kGapSpan + span_last[k]);
            return;
        }
    }
    if (lane == 0 && *carry != ORAND_GAP_NO_HIT) *carry += n;
}

// ------------------------------------------------------------- birthday
//
// Per sample (one CTA): the n birthdays are sorted by a counting sort on
// their top log2(n) bits (one shared-memory atomic per key gives both the
// bucket count and the key's rank inside its bucket), a block scan of the
// bucket counts, a scatter, and insertion sorts inside the buckets, which
// hold about one key each.  A sample with a bucket of more than
// kMaxBucket keys (a very non-uniform stream) is sorted by a bitonic
// network instead, so the work stays bounded.  R is then n minus the number
// of distinct spacings, counted without a second sort and without atomics:
// in rounds, every unresolved spacing stores its index into its hash slot
// (4n 16-bit slots) and, after a barrier, reads the slot back.  The spacing
// whose index stayed represents its value (one distinct value); one that
// finds a representative of its own value is a repeat; one that finds
// another value tries again in the next round.  Each round resolves at
// least the last writer of every slot, so the rounds end (about three for
// random spacings).  Measured on B300 (11,994 samples of 4096 keys): 0.44 ms
// per launch, against 0.60 with a linear-probing hash set built by
// compare-and-swap, 0.53 with 2n slots, 0.49 with every round visiting all
// of a thread's spacings, and 0.45 with every thread scanning its share of
// the buckets for ones to sort.

constexpr int kBirthdayBlock = 512;
constexpr uint32_t kMaxBucket = 64;

// Ascending bitonic sort of y[0..n) (n a power of two) by the whole block.
__device__ __forceinline__ void block_bitonic_sort(uint32_t *y, uint32_t n)
{
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t p = threadIdx.x; p < n / 2; p += blockDim.x) {
                const uint32_t lo = ((p & ~(j - 1)) << 1) | (p & (j - 1));
                const uint32_t hi = lo + j;
                const uint32_t a = y[lo], b = y[hi];
                if ((a > b) == ((lo & k) == 0)) {
                    y[lo] = b;
                    y[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Exclusive prefix sum of c[0..nb) in place (nb a power of two <= 4096), by
// the whole block; each thread scans a run of nb / blockDim entries (read
// and written as 16-byte vectors when the run allows).
__device__ __forceinline__ void block_exclusive_scan(uint32_t *c, uint32_t nb, uint32_t *warp_tot)
{
    const uint32_t T = blockDim.x;
    const uint32_t per = (nb + T - 1) / T;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t v[8];  // per <= 8 (nb <= 4096, blockDim >= 512 when nb > 2048)
    if (per == 8) {
        const uint4 a = *reinterpret_cast<const uint4 *>(c + b0), b = *reinterpret_cast<const uint4 *>(c + b0 + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
        for (uint32_t i = 0; i < 8; ++i) v[i] = (i < per && b0 + i < nb) ? c[b0 + i] : 0u;
    }
    uint32_t run = 0;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) run += v[i];
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += x;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t acc = incl - run;
    for (uint32_t w = 0; w < warp; ++w) acc += warp_tot[w];
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
        const uint32_t x = v[i];
        v[i] = acc;
        acc += x;
    }
    if (per == 8) {
        *reinterpret_cast<uint4 *>(c + b0) = make_uint4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<uint4 *>(c + b0 + 4) = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
        for (uint32_t i = 0; i < 8; ++i)
            if (i < per && b0 + i < nb) c[b0 + i] = v[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBirthdayBlock, 3) birthday_kernel(const uint32_t *__restrict__ w, uint64_t n_samples,
                                                                  uint32_t log2_n, uint32_t bits, uint32_t shift,
                                                                  uint32_t r_max,
                                                                  unsigned long long *__restrict__ counts)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t warp_tot[kBirthdayBlock / 32];
    __shared__ uint32_t flags;  // 1: a spacing of 2^32 (all keys equal, 32-bit birthdays)
    const uint32_t n = 1u << log2_n;
    const uint32_t lb = log2_n < bits ? log2_n : bits;  // bucket bits
    const uint32_t nb = 1u << lb;
    const uint32_t tbits = log2_n + 2;                  // 4n hash slots
    uint32_t *keys = smem;                              // n
    uint32_t *cnt = keys + n;                           // nb <= n; dead once the keys are sorted,
    uint32_t *sp = cnt;                                 // then n words hold the n spacings
    uint16_t *slot = reinterpret_cast<uint16_t *>(cnt + n);  // and 2n words the 4n slots
    const uint32_t mask = bits == 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
    const uint64_t m = 1ull << bits;
    constexpr uint32_t kMaxPer = 4096 / kBirthdayBlock;
    for (uint64_t q = blockIdx.x; q < n_samples; q += gridDim.x) {
        uint32_t y[kMaxPer], rank[kMaxPer];
#pragma unroll
        for (uint32_t k = 0; k < kMaxPer; ++k) {
            const uint32_t i = threadIdx.x + k * blockDim.x;
            if (i < n) y[k] = (__ldg(w + q * n + i) >> shift) & mask;
        }
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0u;
        if (threadIdx.x == 0) flags = 0u;
        __syncthreads();
        bool big = false;
#pragma unroll
        for (uint32_t k = 0; k < kMaxPer; ++k) {
            const uint32_t i = threadIdx.x + k * blockDim.x;
            if (i < n) {
                rank[k] = atomicAdd(&cnt[y[k] >> (bits - lb)], 1u);
                big |= rank[k] >= kMaxBucket;
            }
        }
        if (__syncthreads_or(big)) {
#pragma unroll
            for (uint32_t k = 0; k < kMaxPer; ++k) {
                const uint32_t i = threadIdx.x + k * blockDim.x;
                if (i < n) keys[i] = y[k];
            }
            __syncthreads();
            block_bitonic_sort(keys, n);
        } else {
            block_exclusive_scan(cnt, nb, warp_tot);
#pragma unroll
            for (uint32_t k = 0; k < kMaxPer; ++k) {
                const uint32_t i = threadIdx.x + k * blockDim.x;
                if (i < n) keys[cnt[y[k] >> (bits - lb)] + rank[k]] = y[k];
            }
            __syncthreads();
            // Buckets of two or more keys are sorted by the thread that holds
            // the bucket's second key (rank 1), so each is sorted once and a
            // thread visits only such buckets (about a quarter of them).
#pragma unroll
            for (uint32_t k = 0; k < kMaxPer; ++k) {
                const uint32_t i0 = threadIdx.x + k * blockDim.x;
                if (i0 < n && rank[k] == 1u) {
                    const uint32_t b = y[k] >> (bits - lb);
                    const uint32_t s0 = cnt[b], s1 = b + 1 < nb ? cnt[b + 1] : n;
                    for (uint32_t i = s0 + 1; i < s1; ++i) {  // insertion sort, <= kMaxBucket keys
                        const uint32_t v = keys[i];
                        uint32_t j = i;
                        while (j > s0 && keys[j - 1] > v) {
                            keys[j] = keys[j - 1];
                            --j;
                        }
                        keys[j] = v;
                    }
                }
            }
            __syncthreads();
        }
        // Spacings (the last one wraps around); a spacing of 2^32 can only
        // be the wrap of n equal 32-bit keys, so it is the one value kept
        // out of the slots.
        // A thread's spacings are re-read from shared memory in each round
        // (keeping them in registers spills under the launch bound).
        uint32_t pending = 0u, distinct = 0u;
#pragma unroll
        for (uint32_t k = 0; k < kMaxPer; ++k) {
            const uint32_t i = threadIdx.x + k * blockDim.x;
            if (i < n) {
                const uint64_t d = i + 1 < n ? (uint64_t)keys[i + 1] - keys[i] : (uint64_t)keys[0] + m - keys[n - 1];
                if (d == (1ull << 32)) {
                    flags = 1u;
                } else {
                    const uint32_t v = (uint32_t)d;
                    sp[i] = v;
                    slot[(v * 0x9E3779B1u) >> (32 - tbits)] = (uint16_t)i;   // round 1's store
                    pending |= 1u << k;
                }
            }
        }
        // Round 1 reads back every spacing (unrolled); later rounds visit
        // only a thread's unresolved spacings, usually none or one.
        __syncthreads();
#pragma unroll
        for (uint32_t k = 0; k < kMaxPer; ++k) {
            if ((pending >> k) & 1u) {
                const uint32_t i = threadIdx.x + k * blockDim.x;
                const uint32_t v = sp[i];
                const uint32_t j = slot[(v * 0x9E3779B1u) >> (32 - tbits)];
                if (j == i) {
                    ++distinct;                  // the representative of its value
                    pending &= ~(1u << k);
                } else if (sp[j] == v) {
                    pending &= ~(1u << k);       // a repeat of a represented value
                }
            }
        }
        while (__syncthreads_or(pending != 0u)) {
            for (uint32_t q = pending; q != 0u; q &= q - 1u) {
                const uint32_t i = threadIdx.x + (uint32_t)(__ffs(q) - 1) * blockDim.x;
                slot[(sp[i] * 0x9E3779B1u) >> (32 - tbits)] = (uint16_t)i;
            }
            __syncthreads();
            uint32_t left = 0u;
            for (uint32_t q = pending; q != 0u; q &= q - 1u) {
                const uint32_t k = (uint32_t)(__ffs(q) - 1);
                const uint32_t i = threadIdx.x + k * blockDim.x;
                const uint32_t v = sp[i];
                const uint32_t j = slot[(v * 0x9E3779B1u) >> (32 - tbits)];
                if (j == i) ++distinct;
                else if (sp[j] != v) left |= 1u << k;
            }
            pending = left;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) distinct += __shfl_down_sync(0xFFFFFFFFu, distinct, o);
        if ((threadIdx.x & 31u) == 0) warp_tot[threadIdx.x >> 5] = distinct;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t d = flags;
            for (uint32_t i = 0; i < blockDim.x / 32; ++i) d += warp_tot[i];
            const uint32_t R = n - d;
            atomicAdd(&counts[R < r_max ? R : r_max], 1ull);
        }
        __syncthreads();
    }
}

static orand_status_t check_buf(const void *ptr, size_t align)
{
    if (ptr == nullptr) return ORAND_ERR_INVALID_ARG;
    return ((uintptr_t)ptr % align) ? ORAND_ERR_ALIGNMENT : ORAND_OK;
}

}  // namespace orand_impl

using namespace orand_impl;

extern "C" {

orand_status_t orand_fill_micro_streams(orand_gen_t gen, uint64_t seed, uint64_t n_streams, uint32_t draws,
                                        uint32_t counter_first, uint32_t n_counters, uint32_t *out,
                                        cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_micro_streams");
    if ((unsigned)gen > ORAND_TYCHE || draws == 0 || draws > 64) return ORAND_ERR_INVALID_ARG;
    if (n_counters > 0 && (uint64_t)counter_first + n_counters - 1 > UINT32_MAX) return ORAND_ERR_OVERFLOW;
    uint64_t n_micro, n_words;
    if (mul_overflows(n_streams, n_counters, &n_micro) || mul_overflows(n_micro, draws, &n_words) ||
        n_words > (1ull << 62))
        return ORAND_ERR_OVERFLOW;
    if (n_words == 0) return ORAND_OK;
    orand_status_t st = check_buf(out, 4);
    if (st != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    MicroArgs a;
    a.seed = seed;
    a.n_streams = n_streams;
    a.n_micro = n_micro;
    a.draws = draws;
    a.counter_first = counter_first;
    a.out = out;
    const unsigned grid = grid_for(n_micro, 256, info.sm_count, 8);
    const uint64_t stride = (uint64_t)grid * 256;
    a.stride_div = stride / n_streams;
    a.stride_mod = stride % n_streams;
    switch (gen) {
    case ORAND_PHILOX4x32_10: micro_stream_kernel<ORAND_PHILOX4x32_10><<<grid, 256, 0, stream>>>(a); break;
    case ORAND_THREEFRY4x32_20: micro_stream_kernel<ORAND_THREEFRY4x32_20><<<grid, 256, 0, stream>>>(a); break;
    case ORAND_SQUARES32: micro_stream_kernel<ORAND_SQUARES32><<<grid, 256, 0, stream>>>(a); break;
    default: micro_stream_kernel<ORAND_TYCHE><<<grid, 256, 0, stream>>>(a); break;
    }
    return launch_status();
}

orand_status_t orand_stat_tuples(const uint32_t *words, uint64_t n_words, uint32_t t, uint32_t bits,
                                 uint32_t shift, uint32_t stride, uint64_t *counts, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_stat_tuples");
    if (t < 1 || t > 4 || bits < 1 || t * bits > 14 || shift + bits > 32 || stride < 1) return ORAND_ERR_INVALID_ARG;
    orand_status_t st = check_buf(counts, 8);
    if (st != ORAND_OK) return st;
    const uint64_t n_tuples = n_words < t ? 0 : (n_words - t) / stride + 1;
    if (n_tuples == 0) return ORAND_OK;
    if ((st = check_buf(words, 4)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    const uint32_t cells = 1u << (t * bits);
    const bool lanes = cells <= 256;
    const size_t smem = (size_t)cells * (lanes ? 32 : 1) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        if ((st = lanes ? tuple_smem_opt_in<32>(smem) : tuple_smem_opt_in<1>(smem)) != ORAND_OK) return st;
    }
    // Per-CTA u32 counters: launch pieces small enough that no CTA passes 2^31.
    const uint64_t piece = 1ull << 36;
    for (uint64_t m0 = 0; m0 < n_tuples; m0 += piece) {
        const uint64_t nt = n_tuples - m0 < piece ? n_tuples - m0 : piece;
        const unsigned grid = grid_for(nt, 256, info.sm_count, 4);
        const uint32_t *wp = words + m0 * stride;
        if (stride == t && (uintptr_t)wp % 16 == 0) {
            if (lanes) launch_tuple_vec<32>(t, grid, smem, stream, wp, nt, bits, shift, cells, (unsigned long long *)counts);
            else launch_tuple_vec<1>(t, grid, smem, stream, wp, nt, bits, shift, cells, (unsigned long long *)counts);
        } else if (lanes)
            tuple_kernel<32><<<grid, 256, smem, stream>>>(words + m0 * stride, nt, t, bits, shift, stride, cells,
                                                         (unsigned long long *)counts);
        else
            tuple_kernel<1><<<grid, 256, smem, stream>>>(words + m0 * stride, nt, t, bits, shift, stride, cells,
                                                        (unsigned long long *)counts);
        if ((st = launch_status()) != ORAND_OK) return st;
    }
    return ORAND_OK;
}

orand_status_t orand_stat_gaps(orand_ctx_t ctx, const uint32_t *words, uint64_t n_words, uint64_t lo, uint64_t hi,
                               uint32_t t_max, uint64_t *counts, uint64_t *carry, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_stat_gaps");
    if (lo >= hi || hi > (1ull << 32) || t_max < 1 || t_max > 4096) return ORAND_ERR_INVALID_ARG;
    orand_status_t st;
    if ((st = check_buf(counts, 8)) != ORAND_OK || (st = check_buf(carry, 8)) != ORAND_OK) return st;
    if (n_words == 0) return ORAND_OK;
    if ((st = check_buf(words, 4)) != ORAND_OK) return st;
    if (n_words > (1ull << 50)) return ORAND_ERR_OVERFLOW;
    const uint64_t n_spans = ceil_div(n_words, kGapSpan);
    void *scr;
    if ((st = ctx_scratch(ctx, n_spans * 2 * sizeof(uint32_t), &scr)) != ORAND_OK) return st;
    uint32_t *span_first = (uint32_t *)scr, *span_last = span_first + n_spans;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    const size_t smem = (size_t)(t_max + 1) * sizeof(uint32_t);
    const unsigned grid = grid_for(n_spans * 32, 256, info.sm_count, 8);
    if ((uintptr_t)words % 16 == 0)
        gap_span_vec_kernel<<<grid, 256, smem, stream>>>(words, n_words, lo, hi, t_max,
                                                         (unsigned long long *)counts, span_first, span_last, n_spans);
    else
        gap_span_kernel<<<grid, 256, smem, stream>>>(words, n_words, lo, hi, t_max, (unsigned long long *)counts,
                                                     span_first, span_last, n_spans);
    if ((st = launch_status()) != ORAND_OK) return st;
    gap_stitch_kernel<<<(unsigned)ceil_div(n_spans, 256), 256, 0, stream>>>(
        span_first, span_last, n_spans, (const unsigned long long *)carry, t_max, (unsigned long long *)counts);
    if ((st = launch_status()) != ORAND_OK) return st;
    gap_carry_kernel<<<1, 32, 0, stream>>>(span_last, n_spans, n_words, (unsigned long long *)carry);
    return launch_status();
}

orand_status_t orand_stat_birthday(const uint32_t *words, uint64_t n_words, uint32_t log2_n, uint32_t bits,
                                   uint32_t shift, uint32_t r_max, uint64_t *counts, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_stat_birthday");
    if (log2_n < 2 || log2_n > 12 || bits < 1 || bits > 32 || shift + bits > 32 || r_max < 1 || r_max > 4096)
        return ORAND_ERR_INVALID_ARG;
    orand_status_t st = check_buf(counts, 8);
    if (st != ORAND_OK) return st;
    const uint64_t n_samples = n_words >> log2_n;
    if (n_samples == 0) return ORAND_OK;
    if ((st = check_buf(words, 4)) != ORAND_OK) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;
    const uint32_t n = 1u << log2_n;
    const unsigned block = n / 2 < (uint32_t)kBirthdayBlock ? (n / 2 < 32 ? 32 : n / 2) : kBirthdayBlock;
    const size_t smem = (size_t)4 * n * sizeof(uint32_t);  // keys (n); bucket counts, then spacings (n) and slots (2n)
    // The kernel's static shared memory comes on top: opt in whenever the
    // dynamic part reaches the 48 KB default.
    if (smem >= 48 * 1024)
        ORAND_CUDA_TRY(cudaFuncSetAttribute(birthday_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;  // one wave: as many CTAs as fit at once
    ORAND_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, birthday_kernel, (int)block, smem));
    const uint64_t wave = (uint64_t)info.sm_count * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(n_samples < wave ? n_samples : wave);
    birthday_kernel<<<grid, block, smem, stream>>>(words, n_samples, log2_n, bits, shift, r_max,
                                                   (unsigned long long *)counts);
    return launch_status();
}

}  // extern "C"
