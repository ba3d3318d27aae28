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
    ORAND_ERR_UNSUPPORTED = -7      /* current device is not the compiled target */
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

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* ORAND_H_ */
