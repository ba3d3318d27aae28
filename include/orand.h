/*
 * orand.h -- C ABI of the B300 counter-based random number library
 * (the hot path of OpenRAND, arXiv 2310.19925).
 *
 * Every entry point takes plain pointers, sizes and a cudaStream_t.  Calls
 * are asynchronous on that stream and do not synchronise it.  Device
 * buffers passed in are owned by the caller.  The library never allocates
 * an output; the only memory it owns lives in an orand_ctx_t.  No C++
 * exception crosses this boundary.  Every call validates its arguments
 * before launching anything, and returns ORAND_OK or a negative status.
 *
 * Stream identity (§2, §3 of the paper): a stream is a 64-bit key and a
 * 32-bit counter.  The fills give stream s (0-based within the call) the
 * key seed ^ s and the caller's counter.  Each stream has a period of 2^32
 * generator words.  Value j of stream s is a fixed function of
 * (generator, seed ^ s, counter, j).  It does not depend on the launch
 * shape, the call or the tuning.
 *
 * Generators (§3): Philox4x32-10 and Threefry4x32-20 (Salmon et al. 2011),
 * Squares32 (Widynski 2020), Tyche (Neves & Araujo 2011).  The word layout
 * of each is stated in orand_device.cuh, the in-kernel draw API.
 */
#ifndef ORAND_H_
#define ORAND_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  ORAND_OK = 0; failures are negative. */
typedef enum orand_status_t {
    ORAND_OK = 0,
    ORAND_ERR_INVALID_ARG = -1,     /* null pointer, unknown enum, bad field */
    ORAND_ERR_OVERFLOW = -2,        /* size product overflows, or a stream needs > 2^32 words */
    ORAND_ERR_ALIGNMENT = -3,       /* pointer/offset not aligned to its element size */
    ORAND_ERR_ALLOC = -4,           /* a context-owned allocation failed */
    ORAND_ERR_CUDA = -5,            /* a CUDA runtime call or launch failed */
    ORAND_ERR_DEVICE_TIMEOUT = -6,  /* a device-side wait gave up and set its error word */
    ORAND_ERR_UNSUPPORTED = -7,     /* current device is not the compiled target */
    ORAND_ERR_SCRATCH_LIMIT = -8    /* request larger than a fixed, preallocated scratch area allows */
} orand_status_t;

typedef enum orand_gen_t {
    ORAND_PHILOX4x32_10 = 0,
    ORAND_THREEFRY4x32_20 = 1,
    ORAND_SQUARES32 = 2,
    ORAND_TYCHE = 3
} orand_gen_t;

typedef enum orand_dtype_t {
    ORAND_U32 = 0,          /* raw 32-bit words */
    ORAND_F32_UNIFORM = 1,  /* (w >> 8) * 2^-24, in [0, 1 - 2^-24] */
    ORAND_F64_UNIFORM = 2,  /* two words, first high: ((hi:lo) >> 11) * 2^-53, in [0, 1) */
    ORAND_F32_NORMAL = 3    /* Box-Muller on word pairs (2i, 2i+1); odd counts drop the last sine */
} orand_dtype_t;

/* Human-readable name of a status code (static storage, never NULL). */
const char *orand_status_string(orand_status_t status);

/* Library version as major*10000 + minor*100 + patch. */
int orand_version(void);

/* The CUDA error behind the most recent ORAND_ERR_CUDA returned on the
 * calling host thread (cudaSuccess if none). */
cudaError_t orand_last_cuda_error(void);

/* ------------------------------------------------------------------------
 * Bulk fills (§3: one stream per processing element).
 *
 * out receives n_streams * draws_per_stream values, stream-major:
 * out[s * draws_per_stream + j] = value j of stream s, with key64 = seed ^ s.
 * out is a device pointer aligned to its element size; 16-byte alignment
 * with draws_per_stream a multiple of 4 (2 for FP64) takes the vectorised
 * path, and every other case takes a scalar path with the same bits.
 * n_streams * draws_per_stream == 0 is a no-op (out may then be NULL).
 * Errors: ORAND_ERR_INVALID_ARG (gen/dtype out of range, out NULL),
 * ORAND_ERR_OVERFLOW (element count or byte count overflows 64 bits, or a
 * stream would need more than 2^32 generator words), ORAND_ERR_ALIGNMENT,
 * ORAND_ERR_CUDA (launch failure; see orand_last_cuda_error).
 * ---------------------------------------------------------------------- */
orand_status_t orand_fill_u32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                              uint64_t draws_per_stream, uint32_t *out, cudaStream_t stream);
orand_status_t orand_fill_uniform_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, float *out, cudaStream_t stream);
orand_status_t orand_fill_uniform_f64(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, double *out, cudaStream_t stream);
orand_status_t orand_fill_normal_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                     uint64_t draws_per_stream, float *out, cudaStream_t stream);
/* The same four fills selected by dtype; out is typed by dtype. */
orand_status_t orand_fill(orand_gen_t gen, orand_dtype_t dtype, uint64_t seed, uint32_t counter,
                          uint64_t n_streams, uint64_t draws_per_stream, void *out, cudaStream_t stream);
/* A range of a larger fill: streams first_stream .. first_stream + n_streams
 * - 1 of the problem keyed by seed (stream g has key64 = seed ^ g), written
 * to out[(g - first_stream) * draws_per_stream + j].  orand_fill is this
 * call with first_stream = 0.  Disjoint ranges, on one GPU or one per rank
 * (§3: every stream is independent), concatenate to the whole fill.
 * Errors: as orand_fill, plus ORAND_ERR_OVERFLOW when first_stream +
 * n_streams (or that times draws_per_stream) passes 2^64. */
orand_status_t orand_fill_streams(orand_gen_t gen, orand_dtype_t dtype, uint64_t seed, uint32_t counter,
                                  uint64_t first_stream, uint64_t n_streams, uint64_t draws_per_stream, void *out,
                                  cudaStream_t stream);

/* The word -> value maps alone, applied to caller-provided generator words
 * (Fig. 1's draw helpers and the Box-Muller normal map): value j of `dtype` from
 * words[j] (u32, FP32 uniform), words[2j], words[2j+1] (FP64 uniform, first
 * high) or the pair words[2(j/2)], words[2(j/2)+1] (FP32 normal, j even the
 * cosine, j odd the sine).  words holds 2*n_values words for FP64,
 * 2*ceil(n_values/2) for normals, n_values otherwise; device memory, 4-byte
 * aligned.  out: n_values elements, aligned to the element size.  Same bits
 * as the fills produce from the same words.
 * Errors: INVALID_ARG, OVERFLOW, ALIGNMENT, CUDA. */
orand_status_t orand_map_words(orand_dtype_t dtype, const uint32_t *words, uint64_t n_values, void *out,
                               cudaStream_t stream);

/* The device header's per-thread draw interface (include/orand_device.cuh,
 * the engine classes orand::Philox, Threefry, Squares, Tyche), run on the
 * GPU.  It follows Fig. 1 of the paper: each thread builds its generator in
 * registers from (its key, counter) and draws in order (§3).  Thread t
 * builds the engine for key seed ^ t and `counter`, starting at word
 * first_word of the stream (first_word must be 0 for Tyche, which is
 * sequential), and runs n_rounds rounds of six draws in this order:
 *     w  = g();               d1 = g.uniform_f64();   n  = g.normal2_f32();
 *     u  = g.uniform_f32();   d2 = g.uniform2_f64();  u2 = g.uniform2_f32();
 * which take 12 words per round, so draws straddle the 4-word blocks of
 * Philox and Threefry.  Round r of thread t is a 48-byte record at
 * out + 48 (t n_rounds + r):
 *     double2 d2; double d1; float2 n; float2 u2; uint32_t w; float u;
 * out: device memory, 16-byte aligned, caller-owned.  The random-access
 * engines count words modulo 2^32 (a stream's period, §3); Tyche's draws
 * must stay within 2^32 words.
 * Errors: INVALID_ARG (unknown gen, NULL out with work, first_word != 0 for
 * Tyche), OVERFLOW (size product, or more than 2^32 Tyche words per thread),
 * ALIGNMENT, CUDA. */
orand_status_t orand_engine_draws(orand_gen_t gen, uint64_t seed, uint32_t counter, uint32_t first_word,
                                  uint64_t n_threads, uint32_t n_rounds, void *out, cudaStream_t stream);


/* ------------------------------------------------------------------------
 * Context: owns the library's device scratch (reduction partials, ragged
 * work tables, per-particle accumulators of the baseline walk), the ragged
 * batcher's tuning table and its CUDA-graph cache.  A context belongs to the
 * device that was current at creation; use it from one host thread at a
 * time.  orand_ctx_destroy synchronises that device before freeing.
 * Errors: ORAND_ERR_INVALID_ARG (NULL), ORAND_ERR_ALLOC, ORAND_ERR_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct orand_ctx_s *orand_ctx_t;
orand_status_t orand_ctx_create(orand_ctx_t *ctx);
orand_status_t orand_ctx_destroy(orand_ctx_t ctx);

/* ------------------------------------------------------------------------
 * Fused 2D Brownian walk: the paper's macro-benchmark (Fig. 1, §5) in its
 * pure-diffusion FP32 form, all state in registers, one store per particle.
 * Particle i (0-based in the call) has global id g = p_first + i and key
 * seed ^ g.  Its start position is (u(w0), u(w1)) from the Philox block
 * with counter (0, 0, 0, 0).  Step t = 1..steps adds s * (z0, z1), where
 * (z0, z1) is Box-Muller of words 0 and 1 of the block with counter
 * (0, t, 0, 0) and s = sqrt(2 D dt) (rounded once to FP32).  The sum is
 * compensated per block of 32 steps: the block's increments are summed with
 * FMAs (odd and even steps apart) and each block sum is added to the
 * position with Kahan compensation.
 * pos_out: 2 * n_particles floats (x, y interleaved), 8-byte aligned.
 * Errors: INVALID_ARG (NULL p or pos_out with n > 0, dt or D negative or
 * not finite), OVERFLOW (p_first + n wraps, steps = 2^32 - 1), ALIGNMENT,
 * CUDA.
 * ---------------------------------------------------------------------- */
typedef struct orand_walk2d_t {
    uint64_t n_particles;
    uint64_t p_first;
    uint64_t seed;
    uint32_t steps;
    float dt;
    float D;
    uint32_t reserved;
} orand_walk2d_t;
orand_status_t orand_brownian_walk(const orand_walk2d_t *p, float *pos_out, cudaStream_t stream);

/* cuRAND comparison for the same walk (the paper's comparison system,
 * Fig. 2), with cuRAND's Philox device generator: particle i's state comes
 * from curand_init(curand_seed, p_first + i, 0), its start position from
 * two curand_uniform draws, and each step adds s * curand_normal2.  These
 * are different streams from orand_brownian_walk's; only the cost model is
 * compared.  p->seed is not used.
 *   orand_walk2d_curand_setup: initialise n_particles states (caller-owned,
 *     orand_walk2d_curand_state_bytes() each, 16-byte aligned) and write the
 *     start positions to pos_out.
 *   orand_walk2d_curand_run: Fig. 2's pattern, p->steps launches, each
 *     loading every state and position from HBM and storing them back.
 *   orand_walk2d_curand_fused: one launch, the state in registers for all
 *     steps, the same block-compensated sums as orand_brownian_walk.
 * pos: 2 * n_particles floats, 8-byte aligned.  Errors: as
 * orand_brownian_walk, plus INVALID_ARG / ALIGNMENT for the states. */
size_t orand_walk2d_curand_state_bytes(void);
orand_status_t orand_walk2d_curand_setup(const orand_walk2d_t *p, void *states, float *pos_out, uint64_t curand_seed,
                                         cudaStream_t stream);
orand_status_t orand_walk2d_curand_run(const orand_walk2d_t *p, void *states, float *pos, cudaStream_t stream);
orand_status_t orand_walk2d_curand_fused(const orand_walk2d_t *p, float *pos_out, uint64_t curand_seed,
                                         cudaStream_t stream);

/* The walks' Box-Muller map (the normals every walk kernel draws): for
 * each pair i, out[2i] = r cos(2 pi u2), out[2i+1] = r sin(2 pi u2) with
 * u1 = ((words[2i] >> 8) + 1) 2^-24 and u2 = (words[2i+1] >> 8) 2^-24, from
 * the SFU's estimates: r within 5.8e-7 relative of sqrt(-2 ln u1), cos and
 * sin within 3.4e-7 absolute (measured over every input).  The fills use
 * the exact-to-3-ulp map (orand_map_words with ORAND_F32_NORMAL).
 * words: 2 n_pairs u32, out: 2 n_pairs floats, device memory, 4-byte aligned.
 * Errors: INVALID_ARG, OVERFLOW, ALIGNMENT, CUDA. */
orand_status_t orand_walk_normals(const uint32_t *words, uint64_t n_pairs, float *out, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Differentiable 3D Brownian walk with drift mu - kappa x (kappa = 0: the
 * constant-drift walk; kappa > 0: Ornstein-Uhlenbeck).
 * x_{t+1} = x_t + (mu - kappa x_t) dt + sigma sqrt(dt) z_t, t = 0..steps-1, where z_t are
 * the first three Box-Muller normals of the Philox block with counter
 * (0, t+1, 0, 0) and key seed ^ (p_first + i): (z0, z1) from words 0-1,
 * z2 the cosine normal of words 2-3.  x_0 is given, or else
 * 2 u(w_c) - 1, c = 0..2, from the block with counter (0, 0, 0, 0).
 * The loss is L = (1 / p_total) * sum_i 0.5 k |x_T,i|^2, where p_total
 * is the whole problem's particle count (0 means n_particles).  With this
 * normaliser, calls over particle ranges add up.
 * Layouts: x0, xT, dx0 are n_particles x 3 floats (xyz per particle).  ckpt
 * is ceil(steps / ckpt_every) x n_particles x 3 floats, with checkpoint
 * j = x_{j * ckpt_every}.  The scalar reductions (loss, dmu[3], dsigma)
 * are FP64 device values, summed in a fixed order: results are
 * bit-reproducible.
 * ---------------------------------------------------------------------- */
typedef struct orand_walk3d_t {
    uint64_t n_particles;
    uint64_t p_first;
    uint64_t p_total;
    uint64_t seed;
    uint32_t steps;
    uint32_t ckpt_every;  /* checkpoint interval K in steps; 0 = none */
    float dt;
    float mu[3];
    float sigma;
    float k;
    float kappa;          /* mean reversion; 0 = constant drift */
    uint32_t reserved;    /* must be 0 */
} orand_walk3d_t;

/* x0 = 2u - 1 from counter 0, as the forward uses when x0 is NULL. */
orand_status_t orand_walk3d_init(const orand_walk3d_t *p, float *x0, cudaStream_t stream);

/* Forward: writes xT, the checkpoints (if ckpt is not NULL and ckpt_every > 0)
 * and the loss (if loss is not NULL).  Uses ctx scratch for the loss
 * reduction. */
orand_status_t orand_walk3d_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *xT,
                                float *ckpt, double *loss, cudaStream_t stream);

/* Adjoint: regenerates every z_t from its (particle, t+1) key instead of
 * reading stored noise.  Writes dL/dmu (3 doubles), dL/dsigma (1 double),
 * dL/dkappa (1 double, may be NULL) and dL/dx0 (n x 3 floats, may be NULL),
 * each scaled by *grad_loss (a device double; NULL means 1).
 * With kappa = 0 and dkappa NULL, dx_{t+1}/dx_t = I: the adjoint needs only
 * x_T, and ckpt may be NULL.  Otherwise the adjoint lambda_t decays by
 * (1 - kappa dt) per step, and dL/dkappa = -dt sum_t lambda_{t+1} . x_t needs
 * every position.  The kernel recomputes x_t backwards in time from the end
 * of each checkpoint segment:
 *     x_t = (x_{t+1} - mu dt - sigma sqrt(dt) z_t) / (1 - kappa dt),
 * so ckpt (from orand_walk3d_fwd, same p) is required and ckpt_every must be
 * > 0.  A segment of at most ckpt_every steps bounds the growth of rounding
 * error.  Errors: as the forward, plus INVALID_ARG if a needed ckpt is
 * missing. */
orand_status_t orand_walk3d_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT, const float *ckpt,
                                const double *grad_loss, double *dmu, double *dsigma, double *dkappa, float *dx0,
                                cudaStream_t stream);

/* The adjoint above without a context and without any memory allocation.
 * There is no counterpart in the paper; this entry point exists for callers
 * that must not allocate device memory: code running under a host
 * framework that owns the whole device memory budget, code whose device
 * memory is capped so a new allocation could fail mid-run, and
 * latency-sensitive code that cannot take the device-wide synchronisation
 * cudaMalloc/cudaFree imply.
 * Inputs and outputs are exactly those of orand_walk3d_bwd, with the same
 * bits.  The per-block reduction partials live in a fixed 640 KiB array in
 * the library's device memory, reserved when the library is loaded and held
 * by every device that loads it until the process exits.  That bounds
 * n_particles to at most 4,194,304 (2^22, one 256-thread block per 256
 * particles).  Larger requests return ORAND_ERR_SCRATCH_LIMIT before
 * anything is launched.
 * The first call on a device looks up that array's device address (once
 * per device, with that device current).  Make that first call before any
 * stream capture on the device.  A failed lookup is not remembered: the
 * call returns ORAND_ERR_CUDA and the next call on that device tries again.
 * All calls share the one array.  Every slot a call reads is written
 * earlier in the same call, so nothing needs clearing between calls.  But
 * calls that run at the same time on the GPU (other streams or threads)
 * race on it: order them, for example on one stream.
 * Errors: as orand_walk3d_bwd, plus ORAND_ERR_SCRATCH_LIMIT. */
orand_status_t orand_walk3d_bwd_noalloc(const orand_walk3d_t *p, const float *xT, const float *ckpt,
                                        const double *grad_loss, double *dmu, double *dsigma, double *dkappa,
                                        float *dx0, cudaStream_t stream);

/* Plain baseline of the same walk (kappa must be 0), in the paper's
 * one-launch-per-step pattern (Fig. 1 host loop).  It stores every noise draw: z_store is
 * steps x n_particles x 3 floats.  It works on x in place, starting from
 * x0 (or the counter-0 init), and accumulates without compensation.  The
 * backward reads z_store back, one launch per step, and keeps its
 * per-particle accumulators in ctx scratch.  The outputs are those of
 * orand_walk3d_fwd / orand_walk3d_bwd, up to FP32 summation order. */
orand_status_t orand_walk3d_plain_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *x,
                                      float *z_store, double *loss, cudaStream_t stream);
orand_status_t orand_walk3d_plain_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT,
                                      const float *z_store, const double *grad_loss, double *dmu,
                                      double *dsigma, float *dx0, cudaStream_t stream);

/* Fused noise-storing variant of the same walk (kappa must be 0): the
 * other side of the adjoint's regeneration trade-off.  The forward is the
 * fused, register-resident walk of orand_walk3d_fwd that also writes every
 * standard normal z_t to z_store[t][i][3] (steps x n_particles x 3 floats,
 * 12 bytes per particle-step) and no checkpoints; the backward reads z back
 * from z_store instead of regenerating it.  Same outputs as
 * orand_walk3d_fwd / orand_walk3d_bwd up to FP32 rounding order; z_store
 * holds the same values the plain baseline stores.  Errors: as the plain
 * baseline. */
orand_status_t orand_walk3d_stored_fwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *x0, float *xT,
                                       float *z_store, double *loss, cudaStream_t stream);
orand_status_t orand_walk3d_stored_bwd(orand_ctx_t ctx, const orand_walk3d_t *p, const float *xT,
                                       const float *z_store, const double *grad_loss, double *dmu, double *dsigma,
                                       float *dx0, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Ragged batched generation.  Request i asks for `length` values of
 * `dtype` from the single stream (gen, key64 = seed, counter): exactly the
 * values orand_fill would write for n_streams = 1 with that seed.  They go
 * to (char *)out_base + out_offset_bytes.  reqs is a HOST array; the
 * library copies it before returning, so the caller may reuse it at once.
 * One persistent kernel serves the whole batch from a cached CUDA graph
 * (host-to-device table copy + kernel).  Its block size, chunk size and
 * store width come from an autotuner: the first call for a new size class
 * (log2 of total values, log2 of request count, any Tyche) times candidate
 * configurations on the caller's batch, synchronising the stream.  Every
 * configuration writes identical bits.  Set ORAND_AUTOTUNE=0 to use the
 * default configuration, or pin one with orand_ragged_set_config.
 * Requirements: each output range lies inside [0, out_bytes) and is
 * aligned to its element size (4 or 8 bytes).  A start on a 16-byte
 * boundary takes 16-byte stores.  Ranges must not overlap; they are
 * checked only when ORAND_CHECK_OVERLAP=1.  reserved must be 0.  A stream
 * needs at most 2^32 generator words.  Calls sharing one ctx are ordered:
 * each call waits for the previous batch of that ctx, whatever its stream.
 * Errors: INVALID_ARG, OVERFLOW (range past out_bytes, too many words),
 * ALIGNMENT, ALLOC, CUDA.
 * ---------------------------------------------------------------------- */
typedef struct orand_request_t {
    uint32_t gen;              /* orand_gen_t */
    uint32_t dtype;            /* orand_dtype_t */
    uint64_t seed;             /* the stream's 64-bit key */
    uint32_t counter;          /* the stream's 32-bit counter */
    uint32_t reserved;         /* must be 0 */
    uint64_t length;           /* values */
    uint64_t out_offset_bytes; /* from out_base */
} orand_request_t;

orand_status_t orand_fill_ragged(orand_ctx_t ctx, const orand_request_t *reqs, size_t n, void *out_base,
                                 uint64_t out_bytes, cudaStream_t stream);

/* The same batch as one bulk-fill launch per request, in request order, on
 * one stream: the plain baseline the batcher is measured against. */
orand_status_t orand_fill_ragged_serial(const orand_request_t *reqs, size_t n, void *out_base,
                                        uint64_t out_bytes, cudaStream_t stream);

/* Batcher configuration: block in {64,128,256,512,1024}; chunk_values a
 * multiple of 4 in [128, 2^24]; store_bytes in {4, 8, 16}; ctas_per_sm
 * 0 (as many as fit) or a cap.  set(NULL) returns to autotuning; get
 * reports the configuration of the last call. */
typedef struct orand_ragged_config_t {
    uint32_t block;
    uint32_t chunk_values;
    uint32_t store_bytes;
    uint32_t ctas_per_sm;
} orand_ragged_config_t;
orand_status_t orand_ragged_set_config(orand_ctx_t ctx, const orand_ragged_config_t *cfg);
orand_status_t orand_ragged_get_config(orand_ctx_t ctx, orand_ragged_config_t *cfg);

/* Counters of the batcher on this ctx: graph launches and (re)builds,
 * autotuning runs, size classes tuned. */
typedef struct orand_ragged_stats_t {
    uint64_t graph_launches;
    uint64_t graph_builds;
    uint64_t tune_runs;
    uint64_t tuned_classes;
} orand_ragged_stats_t;
orand_status_t orand_ragged_stats(orand_ctx_t ctx, orand_ragged_stats_t *stats);

/* ------------------------------------------------------------------------
 * The paper's Brownian-dynamics macro-benchmark (Fig. 1, §5): 2D particles
 * with velocity drag and a uniform FP64 kick per step.  Particle i has
 * pid = p_first + i and key seed ^ pid.  Counter 0 sets (x, y) =
 * draw_double2 (the two FP64 uniforms of one Philox block, first word
 * high) and v = 0.  Step `iter` does, in FP64 with round-to-nearest and no
 * fused multiply-add:
 *     v -= gamma / mass * v * dt;  r = draw_double2(pid, iter);
 *     v += (r * 2 - 1) * sqrt(dt);  x += v * dt
 * (the position update is this library's reading; Fig. 1 elides it).
 * particles: n_particles orand_particle_t (array of structures, 8-byte
 * aligned).
 * ---------------------------------------------------------------------- */
typedef struct orand_particle_t {
    double x, y, vx, vy;
    uint64_t pid;
} orand_particle_t;

typedef struct orand_langevin2d_t {
    uint64_t n_particles;
    uint64_t p_first;
    uint64_t seed;
    double dt;
    double gamma;
    double mass;
} orand_langevin2d_t;

/* Counter-0 initialisation (the paper's init_particles). */
orand_status_t orand_langevin2d_init(const orand_langevin2d_t *p, orand_particle_t *particles, cudaStream_t stream);
/* One step with counter `counter`, one launch: the paper's Fig. 1 host loop
 * calls this for counter = 1..STEPS. */
orand_status_t orand_langevin2d_step(const orand_langevin2d_t *p, orand_particle_t *particles, uint32_t counter,
                                     cudaStream_t stream);
/* The Fig. 1 host loop: orand_langevin2d_step for counters first_counter ..
 * first_counter + steps - 1, one launch each. */
orand_status_t orand_langevin2d_run_per_step(const orand_langevin2d_t *p, orand_particle_t *particles,
                                             uint32_t first_counter, uint32_t steps, cudaStream_t stream);
/* Steps with counters first_counter .. first_counter + steps - 1 in one
 * launch, with the state in registers.  Same bits as the same sequence of
 * orand_langevin2d_step calls.  ORAND_ERR_OVERFLOW if the counters pass
 * 2^32. */
orand_status_t orand_langevin2d_fused(const orand_langevin2d_t *p, orand_particle_t *particles,
                                      uint32_t first_counter, uint32_t steps, cudaStream_t stream);
/* The comparison system of §5, in the cuRAND pattern of Fig. 2: one
 * curandStatePhilox4_32_10_t per particle, set up by
 * curand_init(curand_seed, pid, 0), and initial positions drawn from it.
 * Each step then loads and stores the state.  states: n_particles states of
 * orand_langevin2d_curand_state_bytes() each, 16-byte aligned, caller-owned. */
size_t orand_langevin2d_curand_state_bytes(void);
orand_status_t orand_langevin2d_curand_setup(const orand_langevin2d_t *p, orand_particle_t *particles, void *states,
                                             uint64_t curand_seed, cudaStream_t stream);
orand_status_t orand_langevin2d_curand_step(const orand_langevin2d_t *p, orand_particle_t *particles, void *states,
                                            cudaStream_t stream);
/* The Fig. 2 host loop: `steps` calls of orand_langevin2d_curand_step. */
orand_status_t orand_langevin2d_curand_run(const orand_langevin2d_t *p, orand_particle_t *particles, void *states,
                                           uint32_t steps, cudaStream_t stream);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* ORAND_H_ */
