// Bulk fill kernels: n_streams x draws_per_stream values, stream-major,
// stream s keyed by seed ^ s (one stream per processing element, §3 of the
// paper); a call may start at any global stream (first_stream), so ranks or
// chunks of one problem fill disjoint stream ranges of it.  Write-only and HBM-bound for Philox; integer-pipe-bound for the
// longer round functions.
//
// Work unit: a "group" of four consecutive generator words of one stream
// (one Philox/Threefry block, four Squares evaluations, four Tyche steps),
// which becomes 16 bytes of output (4 x u32/f32/normal or 2 x f64).  In
// the vectorised path consecutive threads own consecutive groups, so every
// warp store is one fully coalesced 512-byte row; the grid is sized to the
// resident capacity of the 148 SMs and strides over the groups.
#include <atomic>
#include <cstdlib>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "orand_device.cuh"
#include "values.cuh"

namespace orand_impl {

struct FillArgs {
    uint64_t seed;
    uint64_t s_first;     // global index of stream 0 of this call
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
        const uint4 w = group_words<GEN>(a.seed ^ (a.s_first + s), a.counter, b);
        store_group<DT, VEC>(a.out, g, s, b, a.dps, w);
        g += stride;
        if (g >= a.n_groups) break;
        s += a.stride_div;
        b += a.stride_mod;
        if (b >= a.G) { b -= a.G; ++s; }
    }
}

// ------------------------------------------------ tiled TMA-store variant
//
// Each thread owns "runs" of R consecutive groups of one stream (R a power of
// two <= 8 dividing the groups per stream G), so per-stream setup (the ten
// Philox round keys, the Threefry key schedule, the Squares key hash) is paid
// once per R groups.  Runs are consecutive in memory.  A CTA of T threads
// fills one contiguous tile of T * TR runs (TR runs per thread) in shared
// memory, and one thread writes it to HBM with a TMA tensor store
// (cp.async.bulk.tensor).  The copy is double-buffered, so the next tile is
// generated while the previous one drains.
//
// The output is viewed as a 2D tensor of 128-byte rows, and the tensor map
// uses the 128-byte swizzle: 16-byte chunk c of tile row y sits at shared
// offset y * 128 + ((c ^ (y % 8)) * 16).  A run is R chunks of one row
// (R <= 8, runs aligned to R chunks), so a thread's chunk i lands at
// a0 ^ (i * 16) for one base a0, and the eight threads of each 128-byte
// shared-store phase hit eight distinct bank groups for every R.  So the
// group index stays the unrolled loop's constant i, and when each stream is a
// single run, Philox's first two rounds fold across the R blocks of a stream
// at compile time (measured on B300: 7 % faster than rotating the group order
// per thread to avoid the bank conflicts of an unswizzled tile).  Rows past
// the last full row are clipped by the tensor store; the chunks of a final
// partial row (fewer than 8) are stored directly by the threads that make
// them.
//
// Each (generator, dtype, R, shape) has two kernels: the general one, and
// one for launches where every stream is a single run and the output is
// whole rows (the usual case, e.g. 16 words per stream), which skips the
// stream split and the partial-row stores.
//
// Launch shape per row (measured on B300): the light, HBM-bound Philox u32 and
// FP32-uniform fills use T = 128 and TR = 8 / R, which halves the per-tile
// barrier and bookkeeping cost per group.  Every other fill is bound by the
// integer or FMA pipes and keeps T = 256, TR = 1, for more warps per SM.

__device__ __forceinline__ void tensor_store_2d(const CUtensorMap *map, uint32_t smem, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
                 "r"(smem), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v)
{
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

struct TileArgs {
    uint64_t seed;
    uint64_t r_first;      // global index of this launch's first run (the call's first stream x runs per stream, plus the runs of earlier launches)
    uint64_t n_runs;       // runs of this launch
    uint64_t n_tiles;      // ceil(n_runs / (T * TR))
    uint64_t full_chunks;  // 16-byte chunks in the full 128-byte rows of this launch's output
    uint64_t rps;          // runs per stream = G / R
    int rps_shift;         // log2(rps) when rps is a power of two, else -1
    uint32_t counter;
    uint32_t one;          // 1, held where the compiler cannot see it (orand::FmaAdd)
    uint4 *out;            // run r_first's first chunk; 16-byte aligned
};

// Per-stream state of a random-access generator, set up once per run.
template <int GEN>
struct StreamGen;

// Squares is bound by the ALU pipe in its plain form (ncu: 66-72 % ALU), so
// its fills do the cross-term doubling and the 64-bit key steps as integer
// multiply-adds on the FMA pipe (orand::FmaAdd), with one 64-bit multiply
// per four words; measured on B300 (2^24 x 16): u32 0.339 -> 0.311 ms, FP32
// uniform 0.362 -> 0.315 ms, same bits.  Threefry (92-94 % ALU) and Tyche
// (85 %) stay in their plain form: steering their adds to the FMA pipe
// (the compiler already sends about half there) or their rotations to wide
// multiplies whose halves fold into the round's xor measured slower
// (Threefry u32 0.321 -> 0.331 and 0.408 ms).  Philox already splits its
// work between the two pipes.
template <>
struct StreamGen<ORAND_PHILOX4x32_10> {
    orand::PhiloxKeys keys;
    uint32_t counter;
    __device__ __forceinline__ StreamGen(uint64_t key64, uint32_t c, uint32_t) : keys(key64), counter(c) {}
    __device__ __forceinline__ uint4 group(uint32_t b) const { return keys.block(b, counter); }
    // Blocks b0 .. b0 + N - 1 with their rounds interleaved, round by round:
    // N independent multiply chains in flight instead of one block's chain
    // at a time.  The same words as N calls of group().
    template <int N>
    __device__ __forceinline__ void groups(uint32_t b0, uint4 (&w)[N]) const
    {
        uint32_t c0[N], c1[N], c2[N], c3[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            c0[i] = b0 + (uint32_t)i;
            c1[i] = counter;
            c2[i] = 0u;
            c3[i] = 0u;
        }
#pragma unroll
        for (int r = 0; r < 10; ++r) {
#pragma unroll
            for (int i = 0; i < N; ++i) orand::philox_round(c0[i], c1[i], c2[i], c3[i], keys.k0[r], keys.k1[r]);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) w[i] = make_uint4(c0[i], c1[i], c2[i], c3[i]);
    }
};

// The Philox FP64 fill computes a run's blocks in lockstep (StreamGen::groups):
// its runs are 8 blocks long and its kernel is latency-bound (ncu: 51 % issue,
// `wait` the top stall).  Measured on B300, 2^24 x 16: 0.429 -> 0.401 ms, same
// bits.  The FP32-uniform fill measured the same either way and the normal
// fill slower (0.369 -> 0.377 ms), so they keep one block at a time.
template <int GEN, int DT>
constexpr bool kLockstep = GEN == ORAND_PHILOX4x32_10 && DT == ORAND_F64_UNIFORM;

template <>
struct StreamGen<ORAND_THREEFRY4x32_20> {
    uint4 key;
    uint32_t counter;
    __device__ __forceinline__ StreamGen(uint64_t key64, uint32_t c, uint32_t)
        : key(make_uint4((uint32_t)key64, (uint32_t)(key64 >> 32), 0u, 0u)), counter(c) {}
    __device__ __forceinline__ uint4 group(uint32_t b) const
    {
        return orand::threefry4x32_20(make_uint4(b, counter, 0u, 0u), key);
    }
};

template <>
struct StreamGen<ORAND_SQUARES32> {
    uint64_t key;
    uint32_t counter;
    orand::FmaAdd add;
    __device__ __forceinline__ StreamGen(uint64_t key64, uint32_t c, uint32_t one)
        : key(orand::squares_key(key64)), counter(c), add{one} {}
    __device__ __forceinline__ uint4 group(uint32_t b) const { return orand::squares_block_fma(key, counter, b, add); }
};

// Run lr of this launch (global run r = r_first + lr): groups [q*R, q*R + R)
// of stream s.  Chunk i goes to the shared address a0 ^ (i * 16) and, when
// the run lies in a final partial row, straight to HBM as well.  WHOLE: every
// stream is one run (run r is stream r) and the launch's output is whole
// rows, so neither the stream split nor the partial-row store is needed
// (measured on B300, Philox u32 2^24 x 16: 0.172 ms against 0.182).
template <int GEN, int DT, int R, bool WHOLE>
__device__ __forceinline__ void fill_run(const TileArgs &a, uint64_t lr, uint32_t a0)
{
    const uint64_t r = a.r_first + lr;
    if constexpr (WHOLE) {
        auto put = [&](int i, uint4 bits) { st_shared_v4(a0 ^ ((uint32_t)i << 4), bits); };
        if constexpr (GEN == ORAND_TYCHE) {
            orand::TycheState st = orand::tyche_init(a.seed ^ r, a.counter);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                uint4 w;
                w.x = orand::tyche_next(st);
                w.y = orand::tyche_next(st);
                w.z = orand::tyche_next(st);
                w.w = orand::tyche_next(st);
                put(i, group_bits<DT>(w));
            }
        } else if constexpr (kLockstep<GEN, DT>) {
            const StreamGen<GEN> sg(a.seed ^ r, a.counter, a.one);
            uint4 w[R];
            sg.template groups<R>(0u, w);
#pragma unroll
            for (int i = 0; i < R; ++i) put(i, group_bits<DT>(w[i]));
        } else {
            const StreamGen<GEN> sg(a.seed ^ r, a.counter, a.one);
#pragma unroll
            for (int i = 0; i < R; ++i) put(i, group_bits<DT>(sg.group((uint32_t)i)));
        }
        return;
    }
    uint64_t s, q;
    if (a.rps_shift >= 0) {
        s = r >> a.rps_shift;
        q = r & (a.rps - 1);
    } else {
        s = r / a.rps;
        q = r - s * a.rps;
    }
    const bool tail = lr * R >= a.full_chunks;
    uint4 *gout = a.out + lr * R;
    auto put = [&](int i, uint4 bits) {
        st_shared_v4(a0 ^ ((uint32_t)i << 4), bits);
        if (tail) gout[i] = bits;
    };
    if constexpr (GEN == ORAND_TYCHE) {
        // Whole stream in one run (R == G): sequential words.
        orand::TycheState st = orand::tyche_init(a.seed ^ s, a.counter);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            uint4 w;
            w.x = orand::tyche_next(st);
            w.y = orand::tyche_next(st);
            w.z = orand::tyche_next(st);
            w.w = orand::tyche_next(st);
            put(i, group_bits<DT>(w));
        }
    } else {
        const StreamGen<GEN> sg(a.seed ^ s, a.counter, a.one);
        if constexpr (kLockstep<GEN, DT>) {
            uint4 w[R];
            sg.template groups<R>(a.rps == 1 ? 0u : (uint32_t)(q * R), w);
#pragma unroll
            for (int i = 0; i < R; ++i) put(i, group_bits<DT>(w[i]));
        } else if (a.rps == 1) {
            // Every stream is one run (the same for the whole launch): the
            // group indices are the constants 0..R-1.
#pragma unroll
            for (int i = 0; i < R; ++i) put(i, group_bits<DT>(sg.group((uint32_t)i)));
        } else {
            const uint32_t b0 = (uint32_t)(q * R);
#pragma unroll
            for (int i = 0; i < R; ++i) put(i, group_bits<DT>(sg.group(b0 + (uint32_t)i)));
        }
    }
}

template <int GEN, int DT, int R, int T, int TR, bool WHOLE>
__global__ void __launch_bounds__(T) fill_tile_kernel(const __grid_constant__ CUtensorMap map, TileArgs a)
{
    constexpr uint32_t kRunsPerTile = (uint32_t)T * TR;
    constexpr uint32_t kTileBytes = kRunsPerTile * R * 16;
    constexpr uint32_t kTileRows = kTileBytes / 128;
    static_assert(kTileBytes % 1024 == 0 && kTileRows <= 256, "a tile is whole swizzle periods, at most 256 rows");
    // Two tile buffers from a 1024-byte boundary (the 128-byte swizzle's period);
    // the launch adds 1 KiB of slack for the round-up.
    extern __shared__ __align__(1024) uint8_t tile_raw[];
    const uint32_t base = ((uint32_t)__cvta_generic_to_shared(tile_raw) + 1023u) & ~1023u;
    const uint32_t x = threadIdx.x;
    int buf = 0;
    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const uint32_t sb = base + (uint32_t)buf * kTileBytes;
        // The tensor store issued two tiles ago read this buffer; wait until it has.
        if (x == 0) bulk_wait_read_1();
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TR; ++k) {
            const uint32_t slot = (uint32_t)k * T + x;
            const uint32_t row = (slot * R) >> 3;
            const uint32_t a0 = sb + row * 128u + ((((slot * R) & 7u) ^ (row & 7u)) << 4);
            const uint64_t lr = t * kRunsPerTile + slot;
            if (lr < a.n_runs) fill_run<GEN, DT, R, WHOLE>(a, lr, a0);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (x == 0) {
            tensor_store_2d(&map, sb, 0, (int)(t * kTileRows));
            bulk_commit();
        }
        buf ^= 1;
    }
    if (x == 0) bulk_wait_all();
}

// Tyche is sequential within a stream: one thread walks one whole stream.
template <int DT, bool VEC>
__global__ void __launch_bounds__(256) fill_tyche_kernel(FillArgs a)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_streams; s += stride) {
        orand::TycheState st = orand::tyche_init(a.seed ^ (a.s_first + s), a.counter);
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

// The driver's tensor-map encoder, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// Output rows per launch: tensor coordinates are signed 32-bit, so a fill
// larger than 2^30 rows (128 GiB) is split into launches of whole rows.
constexpr uint64_t kMaxRowsPerLaunch = 1ull << 30;

template <int GEN, int DT, int R, int T, int TR>
static orand_status_t launch_tile_shape(TileArgs a, const DeviceInfo &info, cudaStream_t stream)
{
    constexpr uint32_t kTileRows = (uint32_t)T * TR * R * 16 / 128;
    const size_t smem = 2u * (size_t)T * TR * R * sizeof(uint4) + 1024;
    // The shared-memory opt-in is per device: one bit per ordinal (the call is
    // idempotent, so a race only repeats it).  Ordinals past 63 set it on
    // every launch.
    // Kernel 1 serves launches where every stream is one run and the output
    // is whole rows (see fill_run); kernel 0 serves the rest.
    void (*const kernel[2])(const CUtensorMap, TileArgs) = {fill_tile_kernel<GEN, DT, R, T, TR, false>,
                                                            fill_tile_kernel<GEN, DT, R, T, TR, true>};
    static std::atomic<uint64_t> configured{0};
    const uint64_t bit = info.device < 64 ? 1ull << info.device : 0;
    if (bit == 0 || !(configured.load(std::memory_order_relaxed) & bit)) {
        for (int k = 0; k < 2; ++k) {
            cudaError_t e = cudaFuncSetAttribute(kernel[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_status(e);
        }
        configured.fetch_or(bit, std::memory_order_relaxed);
    }
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (encode == nullptr) return ORAND_ERR_CUDA;
    int per_sm[2] = {0, 0};  // resident CTAs per SM, looked up when a kernel is first used
    const uint64_t total_runs = a.n_runs;
    const uint64_t runs_per_launch = kMaxRowsPerLaunch * 8 / R;
    uint4 *const out0 = a.out;
    for (uint64_t r0 = 0; r0 < total_runs; r0 += runs_per_launch) {
        TileArgs p = a;
        p.r_first = a.r_first + r0;
        // The last launch takes a remainder of less than one row as well, so
        // every launch has at least one full row.
        const uint64_t left = total_runs - r0;
        p.n_runs = left <= runs_per_launch || left - runs_per_launch < 8 / R ? left : runs_per_launch;
        p.out = out0 + r0 * R;
        const uint64_t rows = p.n_runs * R / 8;  // >= 1: the caller sends at least 128 bytes here
        p.full_chunks = rows * 8;
        p.n_tiles = ceil_div(p.n_runs, (uint64_t)T * TR);
        // 32 words x rows, 128-byte rows, box of one tile, 128-byte swizzle.
        CUtensorMap map;
        const cuuint64_t dims[2] = {32, rows};
        const cuuint64_t strides[1] = {128};
        const cuuint32_t box[2] = {32, kTileRows};
        const cuuint32_t elem_strides[2] = {1, 1};
        if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)p.out, dims, strides, box, elem_strides,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return ORAND_ERR_CUDA;
        const int k = (a.rps == 1 && p.n_runs * R % 8 == 0) ? 1 : 0;
        if (per_sm[k] == 0) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[k], kernel[k], T, smem);
            if (e != cudaSuccess) return cuda_status(e);
            if (per_sm[k] < 1) per_sm[k] = 1;
        }
        uint64_t grid = (uint64_t)per_sm[k] * info.sm_count;
        if (grid > p.n_tiles) grid = p.n_tiles;
        kernel[k]<<<(unsigned)grid, T, smem, stream>>>(map, p);
        const orand_status_t st = launch_status();
        if (st != ORAND_OK) return st;
    }
    return ORAND_OK;
}

template <int GEN, int DT, int R>
static orand_status_t launch_tile_r(const TileArgs &a, const DeviceInfo &info, cudaStream_t stream)
{
    constexpr bool light = GEN == ORAND_PHILOX4x32_10 && (DT == ORAND_U32 || DT == ORAND_F32_UNIFORM);
    if constexpr (light) return launch_tile_shape<GEN, DT, R, 128, 8 / R>(a, info, stream);
    else return launch_tile_shape<GEN, DT, R, 256, 1>(a, info, stream);
}

template <int GEN, int DT>
static orand_status_t launch_tile_dt(int R, const TileArgs &a, const DeviceInfo &info, cudaStream_t stream)
{
    switch (R) {
    case 8: return launch_tile_r<GEN, DT, 8>(a, info, stream);
    case 4: return launch_tile_r<GEN, DT, 4>(a, info, stream);
    case 2: return launch_tile_r<GEN, DT, 2>(a, info, stream);
    default: return launch_tile_r<GEN, DT, 1>(a, info, stream);
    }
}

template <int GEN>
static orand_status_t launch_tile_gen(int dt, int R, const TileArgs &a, const DeviceInfo &info, cudaStream_t stream)
{
    switch (dt) {
    case ORAND_U32: return launch_tile_dt<GEN, ORAND_U32>(R, a, info, stream);
    case ORAND_F32_UNIFORM: return launch_tile_dt<GEN, ORAND_F32_UNIFORM>(R, a, info, stream);
    case ORAND_F64_UNIFORM: return launch_tile_dt<GEN, ORAND_F64_UNIFORM>(R, a, info, stream);
    default: return launch_tile_dt<GEN, ORAND_F32_NORMAL>(R, a, info, stream);
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

orand_status_t fill_validate(int gen, int dt, uint64_t s_first, uint64_t n_streams, uint64_t dps, const void *out,
                             uint64_t *n_values)
{
    if (gen < 0 || gen > 3 || dt < 0 || dt > 3) return ORAND_ERR_INVALID_ARG;
    uint64_t n, bytes, words, run_end;
    if (mul_overflows(n_streams, dps, &n)) return ORAND_ERR_OVERFLOW;
    const uint64_t elem = dt == ORAND_F64_UNIFORM ? 8 : 4;
    if (mul_overflows(n, elem, &bytes)) return ORAND_ERR_OVERFLOW;
    if (!stream_words(dt, dps, &words) || words > (1ull << 32)) return ORAND_ERR_OVERFLOW;
    *n_values = n;
    if (n == 0) return ORAND_OK;
    if (s_first > UINT64_MAX - n_streams) return ORAND_ERR_OVERFLOW;      // global stream ids stay below 2^64
    if (mul_overflows(s_first + n_streams, dps, &run_end)) return ORAND_ERR_OVERFLOW;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)out % elem) return ORAND_ERR_ALIGNMENT;
    return ORAND_OK;
}

// ORAND_FILL_TILE=0 selects the untiled kernels (for comparison runs).
static bool tile_path_disabled()
{
    static const bool off = [] {
        const char *v = getenv("ORAND_FILL_TILE");
        return v && v[0] == '0';
    }();
    return off;
}

orand_status_t fill_launch(int gen, int dt, uint64_t seed, uint32_t counter, uint64_t s_first, uint64_t n_streams,
                           uint64_t dps, void *out, cudaStream_t stream)
{
    uint64_t n = 0;
    orand_status_t st = fill_validate(gen, dt, s_first, n_streams, dps, out, &n);
    if (st != ORAND_OK || n == 0) return st;
    DeviceInfo info;
    if ((st = current_device(&info)) != ORAND_OK) return st;

    const uint32_t V = dt == ORAND_F64_UNIFORM ? 2u : 4u;
    const uint64_t G = ceil_div(dps, V);
    const bool vec16 = (dps % V == 0) && ((uintptr_t)out % 16 == 0);
    // Tiled path: vector-aligned output of at least one 128-byte row; Tyche
    // only when a whole stream fits a run.
    if (vec16 && n_streams * G >= 8 && !(gen == ORAND_TYCHE && G > 8) && !tile_path_disabled()) {
        int R = 1;
        if (gen == ORAND_TYCHE) R = (int)G;
        else while (R < 8 && G % (2 * R) == 0) R *= 2;
        if (gen != ORAND_TYCHE || R == 1 || R == 2 || R == 4 || R == 8) {
            TileArgs t;
            t.seed = seed;
            t.counter = counter;
            t.one = 1u;
            t.rps = G / R;
            t.n_runs = n_streams * t.rps;
            t.r_first = s_first * t.rps;   // no overflow: (s_first + n_streams) * dps was checked
            t.n_tiles = 0;      // set per launch
            t.full_chunks = 0;  // set per launch
            t.rps_shift = (t.rps & (t.rps - 1)) == 0 ? __builtin_ctzll(t.rps) : -1;
            t.out = (uint4 *)out;
            switch (gen) {
            case ORAND_PHILOX4x32_10: return launch_tile_gen<ORAND_PHILOX4x32_10>(dt, R, t, info, stream);
            case ORAND_THREEFRY4x32_20: return launch_tile_gen<ORAND_THREEFRY4x32_20>(dt, R, t, info, stream);
            case ORAND_SQUARES32: return launch_tile_gen<ORAND_SQUARES32>(dt, R, t, info, stream);
            default: return launch_tile_gen<ORAND_TYCHE>(dt, R, t, info, stream);
            }
        }
    }
    FillArgs a;
    a.seed = seed;
    a.s_first = s_first;
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

// Word -> value map over caller words: group g reads words 4g..4g+3 (the
// missing tail words of the last group read as 0; their values are not
// stored) and writes its values masked to j < n_values.
template <int DT>
__global__ void __launch_bounds__(256) map_words_kernel(const uint32_t *__restrict__ w, uint64_t n_words,
                                                        uint64_t n_values, char *__restrict__ out)
{
    constexpr uint32_t V = Vals<DT>::V;
    constexpr uint32_t E = DT == ORAND_F64_UNIFORM ? 8u : 4u;
    const uint64_t n_groups = (n_values + V - 1) / V;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = (4 * g + i < n_words) ? w[4 * g + i] : 0u;
        const uint4 bits = group_bits<DT>(make_uint4(v[0], v[1], v[2], v[3]));
        store_bits_masked<DT>(out + g * V * E, g * V, n_values, bits);
    }
}

orand_status_t map_words_launch(int dt, const uint32_t *words, uint64_t n_values, void *out, cudaStream_t stream)
{
    if (dt < 0 || dt > 3) return ORAND_ERR_INVALID_ARG;
    uint64_t n_words = 0, bytes = 0;
    if (!stream_words(dt, n_values, &n_words)) return ORAND_ERR_OVERFLOW;
    const uint64_t elem = dt == ORAND_F64_UNIFORM ? 8 : 4;
    if (mul_overflows(n_values, elem, &bytes)) return ORAND_ERR_OVERFLOW;
    if (n_values == 0) return ORAND_OK;
    if (words == nullptr || out == nullptr) return ORAND_ERR_INVALID_ARG;
    if ((uintptr_t)words % 4 || (uintptr_t)out % elem) return ORAND_ERR_ALIGNMENT;
    DeviceInfo info;
    orand_status_t st = current_device(&info);
    if (st != ORAND_OK) return st;
    const uint64_t groups = ceil_div(n_values, dt == ORAND_F64_UNIFORM ? 2 : 4);
    const unsigned grid = grid_for(groups, 256, info.sm_count, info.max_threads_per_sm / 256);
    switch (dt) {
    case ORAND_U32: map_words_kernel<ORAND_U32><<<grid, 256, 0, stream>>>(words, n_words, n_values, (char *)out); break;
    case ORAND_F32_UNIFORM:
        map_words_kernel<ORAND_F32_UNIFORM><<<grid, 256, 0, stream>>>(words, n_words, n_values, (char *)out);
        break;
    case ORAND_F64_UNIFORM:
        map_words_kernel<ORAND_F64_UNIFORM><<<grid, 256, 0, stream>>>(words, n_words, n_values, (char *)out);
        break;
    default:
        map_words_kernel<ORAND_F32_NORMAL><<<grid, 256, 0, stream>>>(words, n_words, n_values, (char *)out);
        break;
    }
    return launch_status();
}

}  // namespace orand_impl

extern "C" {

orand_status_t orand_map_words(orand_dtype_t dtype, const uint32_t *words, uint64_t n_values, void *out,
                               cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_map_words");
    return orand_impl::map_words_launch((int)dtype, words, n_values, out, stream);
}


orand_status_t orand_fill(orand_gen_t gen, orand_dtype_t dtype, uint64_t seed, uint32_t counter,
                          uint64_t n_streams, uint64_t draws_per_stream, void *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill");
    return orand_impl::fill_launch((int)gen, (int)dtype, seed, counter, 0, n_streams, draws_per_stream, out,
                                   stream);
}

orand_status_t orand_fill_streams(orand_gen_t gen, orand_dtype_t dtype, uint64_t seed, uint32_t counter,
                                  uint64_t first_stream, uint64_t n_streams, uint64_t draws_per_stream, void *out,
                                  cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_streams");
    return orand_impl::fill_launch((int)gen, (int)dtype, seed, counter, first_stream, n_streams, draws_per_stream,
                                   out, stream);
}

orand_status_t orand_fill_u32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                              uint64_t draws_per_stream, uint32_t *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_u32");
    return orand_impl::fill_launch((int)gen, ORAND_U32, seed, counter, 0, n_streams, draws_per_stream, out, stream);
}

orand_status_t orand_fill_uniform_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, float *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_uniform_f32");
    return orand_impl::fill_launch((int)gen, ORAND_F32_UNIFORM, seed, counter, 0, n_streams, draws_per_stream,
                                   out, stream);
}

orand_status_t orand_fill_uniform_f64(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                      uint64_t draws_per_stream, double *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_uniform_f64");
    return orand_impl::fill_launch((int)gen, ORAND_F64_UNIFORM, seed, counter, 0, n_streams, draws_per_stream,
                                   out, stream);
}

orand_status_t orand_fill_normal_f32(orand_gen_t gen, uint64_t seed, uint32_t counter, uint64_t n_streams,
                                     uint64_t draws_per_stream, float *out, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_normal_f32");
    return orand_impl::fill_launch((int)gen, ORAND_F32_NORMAL, seed, counter, 0, n_streams, draws_per_stream,
                                   out, stream);
}

}  // extern "C"
