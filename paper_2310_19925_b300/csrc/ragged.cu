// Ragged batched generation: many independent requests (generator, dtype,
// seed, counter, length, output offset) served by one persistent kernel
// launched from a cached CUDA graph.  A request is exactly the single-stream
// bulk fill (stream 0, key = its seed), so the two paths emit identical bits.
//
// Scheduling (host, O(n log n)):
//   * Tyche is sequential within a stream, so each Tyche request is one
//     lane's serial chain.  Requests of one dtype are sorted longest first and
//     grouped 32 to a warp item; items of all dtypes are merged longest first
//     (LPT), so the longest chains start first and a warp runs one code path.
//   * The random-access generators (Philox, Threefry, Squares) are cut into
//     chunks of `chunk_values` values.  A warp takes one chunk at a time; its
//     32 lanes write consecutive 16-byte groups, and per-stream setup (round
//     keys, Squares key hash) is paid once per chunk.
// Warps take Tyche items and chunks through two atomic cursors.  The
// latency-bound Tyche chains get SMs of their own (two chain warps each) so
// that compute-heavy chunk warps do not slow them; the other SMs
// take the chunks, then the Tyche items left.  There are no inter-block
// waits.
//
// Autotuning: block size, chunk size and store width (16/8/4-byte stores)
// are timed on the caller's batch the first time a size class is seen.  The
// output is written again each time with the same bits.  The fastest
// configuration is kept per size class in the context and, keyed by the GPU's
// name as well, in a small file that later processes read instead of tuning.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <sys/stat.h>

#include "common.cuh"
#include "ctx.cuh"
#include "values.cuh"

namespace orand_impl {

struct RaggedReq {
    uint64_t seed;
    uint64_t length;      // values
    uint64_t out_off;     // bytes from out_base
    uint64_t first_item;  // first chunk item (random-access requests)
    uint32_t counter;
    uint8_t gen, dtype, vec;
    uint8_t raw;          // Tyche lane stores raw words; the convert pass maps them in place
};
static_assert(sizeof(RaggedReq) == 40, "RaggedReq layout");

// Header at the start of the device table: everything that changes from one
// batch to the next, so the captured graph (copy + kernel) does not.
struct RaggedHeader {
    char *out;
    uint64_t n_items;
    uint64_t chunk_values;
    uint64_t off_reqs, off_items, off_tyche, off_cursors;  // bytes from the table start
    uint64_t off_conv;                                     // convert items: request index each
    uint64_t n_conv_items;
    uint64_t conv_chunk_groups;                            // groups per convert item
    uint32_t n_ty_items;                                   // Tyche warp items (32 slots each)
    uint32_t tyche_warps;                                  // warps to give the Tyche chains SMs of their own
};
static_assert(sizeof(RaggedHeader) <= 256, "header slot");
constexpr uint32_t kNoRequest = 0xFFFFFFFFu;

// 16-byte store of one group's bits as SW-byte stores (dst 16-byte aligned).
template <int SW>
__device__ __forceinline__ void store16(char *dst, uint4 v)
{
    if (SW == 16) {
        *reinterpret_cast<uint4 *>(dst) = v;
    } else if (SW == 8) {
        reinterpret_cast<uint2 *>(dst)[0] = make_uint2(v.x, v.y);
        reinterpret_cast<uint2 *>(dst)[1] = make_uint2(v.z, v.w);
    } else {
        uint32_t *o = reinterpret_cast<uint32_t *>(dst);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
}

// Store group g of a request with L values at base.
template <int DT, int SW>
__device__ __forceinline__ void store_req_group(char *base, bool vec, uint64_t g, uint64_t L, uint4 w)
{
    constexpr uint32_t V = Vals<DT>::V;
    constexpr uint32_t E = DT == ORAND_F64_UNIFORM ? 8u : 4u;
    const uint4 v = group_bits<DT>(w);
    const uint64_t j0 = g * V;
    if (vec && j0 + V <= L) store16<SW>(base + j0 * E, v);
    else store_bits_masked<DT>(base + j0 * E, j0, L, v);
}

__device__ __forceinline__ uint4 tyche_next4(orand::TycheState &st)
{
    uint4 w;
    w.x = orand::tyche_next(st);
    w.y = orand::tyche_next(st);
    w.z = orand::tyche_next(st);
    w.w = orand::tyche_next(st);
    return w;
}

// One lane serves one whole Tyche request.  The MIX chain is the critical
// path (one dependent chain of ~12 integer ops per word), so the lane is
// software-pipelined in batches of kTycheBatch groups: while the chain
// produces the words of batch k+1, the independent conversion and stores of
// batch k fill the issue slots the chain leaves idle.
constexpr int kTycheBatch = 4;

// Device table tail: the two work cursors, then the scheduler gates.
constexpr size_t kCursorBytes = 256;
constexpr unsigned kGateSlots = 1024;  // per-SM arrival counters, by SM id (folded)
// Chain warps per Tyche SM.  Measured on B300: chains alone keep full speed
// up to 8 warps per SM, but each lane's 16-byte store to its own request
// (32 distinct lines per warp store) loads the SM's store path: alone, 4
// warps per SM still ran at full speed and 8 at half; inside the
// 100,000-request batch, with the chunk warps' write traffic on the other
// SMs, 4 per SM gave 40-51 ms (run to run) and 2 per SM 31-33 ms, at the
// 29.6 ms floor of the longest chain.
constexpr unsigned kTycheWarpsPerSm = 2;
constexpr size_t kCursorAreaBytes = kCursorBytes + kGateSlots * sizeof(unsigned);

template <int DT, int SW>
__device__ __forceinline__ void tyche_request(const RaggedReq &q, char *out)
{
    constexpr uint64_t V = Vals<DT>::V;
    constexpr uint64_t E = DT == ORAND_F64_UNIFORM ? 8u : 4u;
    char *base = out + q.out_off;
    const uint64_t L = q.length, G = (L + V - 1) / V;
    orand::TycheState st = orand::tyche_init(q.seed, q.counter);
    uint64_t g = 0;
    if (q.raw) {
        // Raw words for every complete group: each value of this dtype takes
        // exactly the bytes of the words it is made from, so the convert pass
        // maps them in place.  The lane runs the bare MIX chain.
        const uint64_t full = L / V;
        for (; g < full; ++g) store16<SW>(base + g * V * E, tyche_next4(st));
    } else if (q.vec && G >= 2 * kTycheBatch) {
        // Full batches [g, g + kTycheBatch) whose groups are all complete.
        const uint64_t full = (L / V) / kTycheBatch * kTycheBatch;
        uint4 cur[kTycheBatch];
#pragma unroll
        for (int i = 0; i < kTycheBatch; ++i) cur[i] = tyche_next4(st);
        for (; g + 2 * kTycheBatch <= full; g += kTycheBatch) {
            uint4 nxt[kTycheBatch];
#pragma unroll
            for (int i = 0; i < kTycheBatch; ++i) nxt[i] = tyche_next4(st);
#pragma unroll
            for (int i = 0; i < kTycheBatch; ++i) store16<SW>(base + (g + i) * V * E, group_bits<DT, true>(cur[i]));
#pragma unroll
            for (int i = 0; i < kTycheBatch; ++i) cur[i] = nxt[i];
        }
        // The last full batch is already generated.
#pragma unroll
        for (int i = 0; i < kTycheBatch; ++i) store16<SW>(base + (g + i) * V * E, group_bits<DT, true>(cur[i]));
        g += kTycheBatch;
    }
    for (; g < G; ++g) store_bits_masked<DT>(base + g * V * E, g * V, L, group_bits<DT>(tyche_next4(st)));
}

template <int SW>
__device__ __forceinline__ void tyche_request_rt(const RaggedReq &q, char *out)
{
    switch (q.dtype) {
    case ORAND_U32: tyche_request<ORAND_U32, SW>(q, out); break;
    case ORAND_F32_UNIFORM: tyche_request<ORAND_F32_UNIFORM, SW>(q, out); break;
    case ORAND_F64_UNIFORM: tyche_request<ORAND_F64_UNIFORM, SW>(q, out); break;
    default: tyche_request<ORAND_F32_NORMAL, SW>(q, out); break;
    }
}

// A warp serves groups [g0, g1) of one random-access request.
template <int GEN, int DT, int SW>
__device__ __forceinline__ void chunk_groups(const RaggedReq &q, char *out, uint64_t g0, uint64_t g1, int lane)
{
    char *base = out + q.out_off;
    if (GEN == ORAND_PHILOX4x32_10) {
        const orand::PhiloxKeys keys(q.seed);
        for (uint64_t g = g0 + lane; g < g1; g += 32)
            store_req_group<DT, SW>(base, q.vec, g, q.length, keys.block((uint32_t)g, q.counter));
    } else if (GEN == ORAND_THREEFRY4x32_20) {
        const uint4 key = make_uint4((uint32_t)q.seed, (uint32_t)(q.seed >> 32), 0u, 0u);
        for (uint64_t g = g0 + lane; g < g1; g += 32)
            store_req_group<DT, SW>(base, q.vec, g, q.length,
                                    orand::threefry4x32_20(make_uint4((uint32_t)g, q.counter, 0u, 0u), key));
    } else {
        const uint64_t sk = orand::squares_key(q.seed);
        for (uint64_t g = g0 + lane; g < g1; g += 32)
            store_req_group<DT, SW>(base, q.vec, g, q.length, orand::squares_block(sk, q.counter, (uint32_t)g));
    }
}

template <int GEN, int SW>
__device__ __forceinline__ void chunk_dt(const RaggedReq &q, char *out, uint64_t g0, uint64_t g1, int lane)
{
    switch (q.dtype) {
    case ORAND_U32: chunk_groups<GEN, ORAND_U32, SW>(q, out, g0, g1, lane); break;
    case ORAND_F32_UNIFORM: chunk_groups<GEN, ORAND_F32_UNIFORM, SW>(q, out, g0, g1, lane); break;
    case ORAND_F64_UNIFORM: chunk_groups<GEN, ORAND_F64_UNIFORM, SW>(q, out, g0, g1, lane); break;
    default: chunk_groups<GEN, ORAND_F32_NORMAL, SW>(q, out, g0, g1, lane); break;
    }
}

// Block sizes up to 1024 threads are accepted (orand_ragged_set_config), so
// the kernels are compiled to fit 1024-thread blocks (at most 64 registers).
constexpr int kRaggedMaxBlock = 1024;

template <int SW>
__global__ void __launch_bounds__(kRaggedMaxBlock) ragged_kernel(char *table)
{
    const RaggedHeader h = *reinterpret_cast<const RaggedHeader *>(table);
    const RaggedReq *reqs = reinterpret_cast<const RaggedReq *>(table + h.off_reqs);
    const uint32_t *item_req = reinterpret_cast<const uint32_t *>(table + h.off_items);
    const uint32_t *tyche = reinterpret_cast<const uint32_t *>(table + h.off_tyche);
    unsigned long long *cursors = reinterpret_cast<unsigned long long *>(table + h.off_cursors);
    const int lane = threadIdx.x & 31;
    unsigned *sm_rank = reinterpret_cast<unsigned *>(table + h.off_cursors + kCursorBytes);
    // Tyche warp items (32 requests of one dtype, longest first) come from
    // cursor 0.  Each chain is one latency-bound dependency chain: up to
    // two per scheduler run at full speed, but compute-heavy warps on the
    // same SM (the chunks) slow it two- to four-fold, and so do more than
    // kTycheWarpsPerSm chains on one SM (their scattered stores).  So the
    // chains get SMs of their own: K SMs, spread by SM id, on which the first
    // kTycheWarpsPerSm warps to arrive take Tyche items (then chunks) and the
    // other warps leave.  On every other SM all warps take chunks first; then the first
    // two warps to have arrived take the Tyche items still left.  Each item
    // is claimed once, through the cursor, whoever takes it.
    unsigned rank = 0, tyche_sm = 0;
    if (lane == 0) {
        unsigned smid, nsmid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
        rank = atomicAdd(&sm_rank[smid & (kGateSlots - 1u)], 1u);
        const unsigned cap = nsmid / 2 > 1u ? nsmid / 2 : 1u;
        const unsigned want = (h.tyche_warps + kTycheWarpsPerSm - 1) / kTycheWarpsPerSm;
        const unsigned K = want < cap ? want : cap;
        if (K) {
            const unsigned stride = nsmid / K > 1u ? nsmid / K : 1u;
            tyche_sm = smid % stride == 0 && smid / stride < K;
        }
    }
    rank = __shfl_sync(0xFFFFFFFFu, rank, 0);
    tyche_sm = __shfl_sync(0xFFFFFFFFu, tyche_sm, 0);
    auto tyche_items = [&]() {
        for (;;) {
            unsigned long long wi = 0;
            if (lane == 0) wi = atomicAdd(&cursors[0], 1ull);
            wi = __shfl_sync(0xFFFFFFFFu, wi, 0);
            if (wi >= h.n_ty_items) break;
            const uint32_t r = tyche[wi * 32 + lane];
            if (r != kNoRequest) {
                // A register copy: the output stores could alias the table as
                // far as the compiler knows, so a reference would be re-read
                // from global memory inside the chain loop.
                const RaggedReq q = reqs[r];
                tyche_request_rt<SW>(q, h.out);
            }
        }
    };
    if (tyche_sm) {
        if (rank >= kTycheWarpsPerSm) return;
        tyche_items();
    }
    // Chunks of the random-access requests.
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&cursors[1], 1ull);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= h.n_items) break;
        const RaggedReq q = reqs[item_req[item]];
        const uint64_t V = q.dtype == ORAND_F64_UNIFORM ? 2u : 4u;
        const uint64_t v0 = (item - q.first_item) * h.chunk_values;
        const uint64_t v1 = min(q.length, v0 + h.chunk_values);
        const uint64_t g0 = v0 / V, g1 = (v1 + V - 1) / V;
        switch (q.gen) {
        case ORAND_PHILOX4x32_10: chunk_dt<ORAND_PHILOX4x32_10, SW>(q, h.out, g0, g1, lane); break;
        case ORAND_THREEFRY4x32_20: chunk_dt<ORAND_THREEFRY4x32_20, SW>(q, h.out, g0, g1, lane); break;
        default: chunk_dt<ORAND_SQUARES32, SW>(q, h.out, g0, g1, lane); break;
        }
    }
    if (!tyche_sm && rank < 2) tyche_items();
}

// In-place conversion of the raw words Tyche lanes stored: each warp takes
// one item (conv_chunk_groups complete groups of one request), loads each
// group's four words and stores its values over them.
template <int DT>
__device__ __forceinline__ void convert_groups(char *base, uint64_t g0, uint64_t g1, int lane)
{
    constexpr uint64_t V = Vals<DT>::V;
    constexpr uint64_t E = DT == ORAND_F64_UNIFORM ? 8u : 4u;
    for (uint64_t g = g0 + lane; g < g1; g += 32) {
        uint4 *p = reinterpret_cast<uint4 *>(base + g * V * E);
        *p = group_bits<DT>(*p);
    }
}

__global__ void __launch_bounds__(kRaggedMaxBlock) ragged_convert_kernel(char *table)
{
    const RaggedHeader h = *reinterpret_cast<const RaggedHeader *>(table);
    const RaggedReq *reqs = reinterpret_cast<const RaggedReq *>(table + h.off_reqs);
    const uint32_t *conv = reinterpret_cast<const uint32_t *>(table + h.off_conv);
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); it < h.n_conv_items;
         it += warps) {
        const uint32_t r = conv[it];
        const RaggedReq q = reqs[r];
        const uint64_t V = q.dtype == ORAND_F64_UNIFORM ? 2u : 4u;
        // items of one request are consecutive; its first item index is
        // first_item (set on the host for raw Tyche requests)
        const uint64_t g0 = (it - q.first_item) * h.conv_chunk_groups;
        const uint64_t g1 = min(q.length / V, g0 + h.conv_chunk_groups);
        char *base = h.out + q.out_off;
        switch (q.dtype) {
        case ORAND_F32_UNIFORM: convert_groups<ORAND_F32_UNIFORM>(base, g0, g1, lane); break;
        case ORAND_F64_UNIFORM: convert_groups<ORAND_F64_UNIFORM>(base, g0, g1, lane); break;
        default: convert_groups<ORAND_F32_NORMAL>(base, g0, g1, lane); break;
        }
    }
}

// ------------------------------------------------------------------ host

struct RaggedConfig {
    uint32_t block = 256;
    uint32_t chunk_values = 8192;
    uint32_t store_bytes = 16;
    uint32_t ctas_per_sm = 0;  // 0: as many as fit
};

struct GraphKey {
    RaggedConfig cfg;
    uint64_t copy_bytes;
    void *d_tables, *h_staging;
    bool operator==(const GraphKey &o) const
    {
        return cfg.block == o.cfg.block && cfg.chunk_values == o.cfg.chunk_values &&
               cfg.store_bytes == o.cfg.store_bytes && cfg.ctas_per_sm == o.cfg.ctas_per_sm &&
               copy_bytes == o.copy_bytes && d_tables == o.d_tables && h_staging == o.h_staging;
    }
};

struct RaggedState {
    void *d_tables = nullptr;
    size_t d_bytes = 0;
    void *h_staging = nullptr;
    size_t h_bytes = 0;
    cudaEvent_t staging_free = nullptr;  // recorded in the graph after the table copy
    cudaEvent_t batch_done = nullptr;    // recorded on the caller's stream after each batch
    bool batch_pending = false;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    GraphKey key{};
    bool have_graph = false;
    bool forced = false;
    RaggedConfig forced_cfg, last_cfg;
    std::map<std::tuple<int, int, int>, RaggedConfig> tuned;
    uint64_t graph_launches = 0, graph_builds = 0, tune_runs = 0;
};

static RaggedState *state_of(orand_ctx_t ctx)
{
    if (!ctx->ragged && !alloc_blocked()) ctx->ragged = new (std::nothrow) RaggedState();
    return (RaggedState *)ctx->ragged;
}

void ragged_state_free(orand_ctx_t ctx)
{
    RaggedState *s = (RaggedState *)ctx->ragged;
    if (!s) return;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
    if (s->staging_free) cudaEventDestroy(s->staging_free);
    if (s->batch_done) cudaEventDestroy(s->batch_done);
    if (s->d_tables) cudaFree(s->d_tables);
    if (s->h_staging) cudaFreeHost(s->h_staging);
    delete s;
    ctx->ragged = nullptr;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr uint64_t kConvChunkGroups = 2048;  // 32 KiB of output per convert item

struct Plan {
    uint64_t chunk_values = 0;
    std::vector<uint32_t> conv;   // convert items: request index each
    std::vector<RaggedReq> reqs;
    std::vector<uint32_t> tyche;  // warp items of 32 slots, kNoRequest-padded
    uint64_t n_tyche = 0;
    uint32_t tyche_warps = 0;     // warps the Tyche chains should get (0: no Tyche requests)
    uint64_t n_items = 0;
    uint64_t total_values = 0;
    size_t off_reqs = 256, off_items = 0, off_tyche = 0, off_conv = 0, off_cursors = 0, table_bytes = 0;
};

static uint64_t words_for(uint32_t dt, uint64_t len)
{
    if (dt == ORAND_F64_UNIFORM) return len > UINT64_MAX / 2 ? UINT64_MAX : 2 * len;
    if (dt == ORAND_F32_NORMAL) return len + (len & 1);
    return len;
}

// Validate every request and build the device tables' host image.
static orand_status_t plan_requests(const orand_request_t *r, size_t n, const char *out_base, uint64_t out_bytes,
                                    uint64_t chunk_values, Plan *p, bool check_overlap)
{
    p->chunk_values = chunk_values;
    p->reqs.resize(n);
    p->tyche.clear();
    p->conv.clear();
    p->n_tyche = 0;
    std::vector<uint32_t> ty[4];
    p->n_items = 0;
    p->total_values = 0;
    std::vector<std::pair<uint64_t, uint64_t>> ranges;
    if (check_overlap) ranges.reserve(n);
    for (size_t i = 0; i < n; ++i) {
        const orand_request_t &q = r[i];
        if (q.gen > 3 || q.dtype > 3 || q.reserved != 0) return ORAND_ERR_INVALID_ARG;
        if (words_for(q.dtype, q.length) > (1ull << 32)) return ORAND_ERR_OVERFLOW;
        const uint64_t elem = q.dtype == ORAND_F64_UNIFORM ? 8 : 4;
        const uint64_t bytes = q.length * elem;  // length <= 2^32, no overflow
        if (q.out_offset_bytes > out_bytes || bytes > out_bytes - q.out_offset_bytes) return ORAND_ERR_OVERFLOW;
        if (((uintptr_t)out_base + q.out_offset_bytes) % elem) return ORAND_ERR_ALIGNMENT;
        RaggedReq &d = p->reqs[i];
        d.seed = q.seed;
        d.length = q.length;
        d.out_off = q.out_offset_bytes;
        d.counter = q.counter;
        d.gen = (uint8_t)q.gen;
        d.dtype = (uint8_t)q.dtype;
        d.vec = (((uintptr_t)out_base + q.out_offset_bytes) % 16 == 0) ? 1 : 0;
        d.raw = 0;
        d.first_item = p->n_items;
        if (q.length && check_overlap) ranges.emplace_back(q.out_offset_bytes, q.out_offset_bytes + bytes);
        p->total_values += q.length;
        if (q.length == 0) continue;
        if (q.gen == ORAND_TYCHE) {
            ty[q.dtype].push_back((uint32_t)i);
            ++p->n_tyche;
            const uint64_t V = q.dtype == ORAND_F64_UNIFORM ? 2 : 4;
            const uint64_t full = q.length / V;
            if (q.dtype != ORAND_U32 && d.vec && full > 0) {
                // raw words now, converted in place by the convert pass
                d.raw = 1;
                d.first_item = p->conv.size();
                for (uint64_t c = 0; c < full; c += kConvChunkGroups) p->conv.push_back((uint32_t)i);
            }
        } else {
            p->n_items += (q.length + chunk_values - 1) / chunk_values;
        }
    }
    if (n > 0xFFFFFFFFull) return ORAND_ERR_OVERFLOW;
    if (check_overlap) {
        std::sort(ranges.begin(), ranges.end());
        for (size_t i = 1; i < ranges.size(); ++i)
            if (ranges[i].first < ranges[i - 1].second) return ORAND_ERR_INVALID_ARG;
    }
    // Tyche warp items: 32 requests of one dtype (so a warp runs one code
    // path), longest chains first within each dtype, and the items of all
    // dtypes merged longest-first (LPT).  Ties by request index keep the plan
    // deterministic.
    struct WarpItem {
        uint64_t longest;
        uint32_t dtype, first;
    };
    std::vector<WarpItem> items;
    for (uint32_t d = 0; d < 4; ++d) {
        std::sort(ty[d].begin(), ty[d].end(), [&](uint32_t a, uint32_t b) {
            if (p->reqs[a].length != p->reqs[b].length) return p->reqs[a].length > p->reqs[b].length;
            return a < b;
        });
        for (uint32_t k = 0; k < ty[d].size(); k += 32) items.push_back({p->reqs[ty[d][k]].length, d, k});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const WarpItem &a, const WarpItem &b) { return a.longest > b.longest; });
    // Warps for the chains: the longest item sets the floor of the batch's
    // time, so aim for about twice the total item cost over the longest.
    p->tyche_warps = 0;
    if (!items.empty()) {
        double total = 0.0;
        for (const WarpItem &w : items) total += (double)w.longest;
        const double want = 2.0 * total / (double)items.front().longest;
        p->tyche_warps = (uint32_t)std::min<double>((double)items.size(), std::max(8.0, std::ceil(want)));
    }
    p->tyche.assign(items.size() * 32, kNoRequest);
    for (size_t w = 0; w < items.size(); ++w)
        for (uint32_t l = 0; l < 32 && items[w].first + l < ty[items[w].dtype].size(); ++l)
            p->tyche[w * 32 + l] = ty[items[w].dtype][items[w].first + l];
    p->off_reqs = 256;
    p->off_items = align_up(p->off_reqs + n * sizeof(RaggedReq), 256);
    p->off_tyche = align_up(p->off_items + p->n_items * sizeof(uint32_t), 256);
    p->off_conv = align_up(p->off_tyche + p->tyche.size() * sizeof(uint32_t), 256);
    p->off_cursors = align_up(p->off_conv + p->conv.size() * sizeof(uint32_t), 256);
    p->table_bytes = p->off_cursors + kCursorAreaBytes;
    return ORAND_OK;
}

static void write_staging(const Plan &p, char *out, char *h)
{
    RaggedHeader hd{};
    hd.out = out;
    hd.n_items = p.n_items;
    hd.chunk_values = p.chunk_values;
    hd.off_reqs = p.off_reqs;
    hd.off_items = p.off_items;
    hd.off_tyche = p.off_tyche;
    hd.off_cursors = p.off_cursors;
    hd.n_ty_items = (uint32_t)(p.tyche.size() / 32);
    hd.tyche_warps = p.tyche_warps;
    hd.off_conv = p.off_conv;
    hd.n_conv_items = p.conv.size();
    hd.conv_chunk_groups = kConvChunkGroups;
    std::memset(h, 0, 256);
    std::memcpy(h, &hd, sizeof(hd));
    std::memcpy(h + p.off_reqs, p.reqs.data(), p.reqs.size() * sizeof(RaggedReq));
    uint32_t *items = (uint32_t *)(h + p.off_items);
    uint64_t k = 0;
    for (size_t i = 0; i < p.reqs.size(); ++i) {
        const RaggedReq &q = p.reqs[i];
        if (q.gen == ORAND_TYCHE || q.length == 0) continue;
        const uint64_t n_chunks = (q.length + p.chunk_values - 1) / p.chunk_values;
        for (uint64_t c = 0; c < n_chunks; ++c) items[k++] = (uint32_t)i;
    }
    std::memcpy(h + p.off_tyche, p.tyche.data(), p.tyche.size() * sizeof(uint32_t));
    std::memcpy(h + p.off_conv, p.conv.data(), p.conv.size() * sizeof(uint32_t));
    std::memset(h + p.off_cursors, 0, kCursorAreaBytes);
}

// Bytes the graph copies: the table rounded up to a power of two, so batches
// of similar size reuse one graph.
static size_t copy_bucket(size_t table_bytes)
{
    size_t b = 1 << 16;
    while (b < table_bytes) b <<= 1;
    return b;
}

static orand_status_t ensure_buffers(RaggedState *s, size_t bytes)
{
    if (!s->staging_free) {
        if (cudaEventCreateWithFlags(&s->staging_free, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->batch_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_status(cudaGetLastError());
    }
    if (bytes > s->d_bytes) {
        if (s->d_tables) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_status(e);
            cudaFree(s->d_tables);
            s->d_tables = nullptr;
            s->d_bytes = 0;
        }
        const size_t want = align_up(bytes + bytes / 4, (size_t)1 << 20);
        if (alloc_blocked()) return ORAND_ERR_ALLOC;
        if (cudaMalloc(&s->d_tables, want) != cudaSuccess) {
            set_last_cuda_error(cudaGetLastError());
            return ORAND_ERR_ALLOC;
        }
        s->d_bytes = want;
        s->have_graph = false;
    }
    if (bytes > s->h_bytes) {
        if (s->h_staging) {
            cudaEventSynchronize(s->staging_free);
            cudaFreeHost(s->h_staging);
            s->h_staging = nullptr;
            s->h_bytes = 0;
        }
        const size_t want = align_up(bytes + bytes / 4, (size_t)1 << 20);
        if (alloc_blocked()) return ORAND_ERR_ALLOC;
        if (cudaHostAlloc(&s->h_staging, want, cudaHostAllocDefault) != cudaSuccess) {
            set_last_cuda_error(cudaGetLastError());
            return ORAND_ERR_ALLOC;
        }
        s->h_bytes = want;
        s->have_graph = false;
    }
    return ORAND_OK;
}

// Persistent grid for a configuration: as many CTAs as fit on every SM (or
// the configured cap).  Queried outside any stream capture.
static orand_status_t ragged_grid(const RaggedConfig &c, unsigned *grid)
{
    DeviceInfo info;
    orand_status_t st = current_device(&info);
    if (st != ORAND_OK) return st;
    const void *fn = c.store_bytes == 16 ? (const void *)ragged_kernel<16>
                     : c.store_bytes == 8 ? (const void *)ragged_kernel<8> : (const void *)ragged_kernel<4>;
    int per_sm = 0;
    ORAND_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)c.block, 0));
    if (per_sm < 1) per_sm = 1;
    if (c.ctas_per_sm && (int)c.ctas_per_sm < per_sm) per_sm = (int)c.ctas_per_sm;
    *grid = (unsigned)(per_sm * info.sm_count);
    return ORAND_OK;
}

// The batch: the persistent kernel, then the in-place conversion of the raw
// Tyche words (a no-op grid when there are none).
static void launch_kernel(char *table, const RaggedConfig &c, unsigned grid, cudaStream_t stream)
{
    if (c.store_bytes == 16) ragged_kernel<16><<<grid, c.block, 0, stream>>>(table);
    else if (c.store_bytes == 8) ragged_kernel<8><<<grid, c.block, 0, stream>>>(table);
    else ragged_kernel<4><<<grid, c.block, 0, stream>>>(table);
    ragged_convert_kernel<<<grid, 256, 0, stream>>>(table);
}

static bool valid_config(const RaggedConfig &c)
{
    return (c.block == 64 || c.block == 128 || c.block == 256 || c.block == 512 || c.block == 1024) &&
           c.chunk_values >= 128 && c.chunk_values % 4 == 0 && c.chunk_values <= (1u << 24) &&
           (c.store_bytes == 4 || c.store_bytes == 8 || c.store_bytes == 16);
}

static int ilog2(uint64_t v)
{
    int r = 0;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

// Time candidate configurations on the caller's batch (tables already on the
// device) and return the fastest.  Each run rewrites the same output bits.
static orand_status_t autotune(RaggedState *s, const orand_request_t *r, size_t n, char *out, uint64_t out_bytes,
                               cudaStream_t stream, RaggedConfig *best)
{
    static const uint32_t blocks[] = {128, 256, 512};
    static const uint32_t chunks[] = {2048, 8192, 32768};
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cuda_status(cudaGetLastError());
    float best_ms = 1e30f;
    RaggedConfig cand;
    orand_status_t st = ORAND_OK;
    for (uint32_t ch : chunks) {
        Plan p;
        if ((st = plan_requests(r, n, out, out_bytes, ch, &p, false)) != ORAND_OK) break;
        if ((st = ensure_buffers(s, copy_bucket(p.table_bytes))) != ORAND_OK) break;
        cudaEventSynchronize(s->staging_free);
        write_staging(p, out, (char *)s->h_staging);
        cudaError_t e = cudaMemcpyAsync(s->d_tables, s->h_staging, p.table_bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) { st = cuda_status(e); break; }
        for (uint32_t bl : blocks) {
            for (uint32_t sw : {16u, 8u}) {
                cand.block = bl;
                cand.chunk_values = ch;
                cand.store_bytes = sw;
                cand.ctas_per_sm = 0;
                unsigned grid = 0;
                if ((st = ragged_grid(cand, &grid)) != ORAND_OK) break;
                cudaMemsetAsync((char *)s->d_tables + p.off_cursors, 0, kCursorAreaBytes, stream);
                cudaEventRecord(a, stream);
                launch_kernel((char *)s->d_tables, cand, grid, stream);
                if ((st = launch_status()) != ORAND_OK) break;
                cudaEventRecord(b, stream);
                e = cudaEventSynchronize(b);
                if (e != cudaSuccess) { st = cuda_status(e); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                ++s->tune_runs;
                if (ms < best_ms) { best_ms = ms; *best = cand; }
            }
            if (st != ORAND_OK) break;
        }
        if (st != ORAND_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    s->have_graph = false;
    return st;
}

static bool env_flag(const char *name, bool dflt)
{
    const char *v = getenv(name);
    if (!v || !*v) return dflt;
    return !(v[0] == '0' || v[0] == 'n' || v[0] == 'N' || v[0] == 'f' || v[0] == 'F');
}

// ----------------------------------------------- persistent tuning table
//
// Tuned configurations outlive the process in a small text file, one line
// per (GPU name, size class): "<gpu> <log2 values> <log2 requests> <tyche>
// <block> <chunk_values> <store_bytes> <ctas_per_sm>", GPU names with
// spaces written as '_'.  The file is ORAND_TUNE_CACHE (empty, "0" or "off":
// no file), else $XDG_CACHE_HOME/orand/ragged_tune.txt, else
// $HOME/.cache/orand/ragged_tune.txt.  It is read once per process and
// appended to after each new tuning; unreadable or malformed lines are
// skipped, so a bad file costs a re-tune, never a wrong result (every
// configuration writes the same bits).  With no file every context tunes
// its own size classes.
using TuneKey = std::tuple<std::string, int, int, int>;

struct TuneFile {
    std::mutex mu;
    bool loaded = false;
    std::string path;
    std::map<TuneKey, RaggedConfig> table;
};

static TuneFile &tune_file()
{
    static TuneFile f;
    return f;
}

static std::string tune_cache_path()
{
    const char *v = getenv("ORAND_TUNE_CACHE");
    if (v) {
        if (!*v || !strcmp(v, "0") || !strcmp(v, "off")) return std::string();
        return v;
    }
    const char *x = getenv("XDG_CACHE_HOME");
    if (x && *x) return std::string(x) + "/orand/ragged_tune.txt";
    const char *h = getenv("HOME");
    if (h && *h) return std::string(h) + "/.cache/orand/ragged_tune.txt";
    return std::string();
}

static std::string gpu_name(int device)
{
    static std::mutex mu;
    static std::map<int, std::string> names;
    std::lock_guard<std::mutex> lock(mu);
    auto it = names.find(device);
    if (it != names.end()) return it->second;
    cudaDeviceProp prop;
    std::string n = cudaGetDeviceProperties(&prop, device) == cudaSuccess ? prop.name : "unknown";
    for (char &c : n)
        if (c == ' ' || c == '\t' || c == '\n') c = '_';
    names[device] = n;
    return n;
}

// Caller holds f.mu.
static void tune_file_load(TuneFile &f)
{
    if (f.loaded) return;
    f.loaded = true;
    f.path = tune_cache_path();
    if (f.path.empty()) return;
    FILE *fp = fopen(f.path.c_str(), "r");
    if (!fp) return;
    char name[256];
    int lv, ln, ty;
    unsigned bl, ch, sw, cps;
    char line[512];
    while (fgets(line, sizeof line, fp)) {
        if (sscanf(line, "%255s %d %d %d %u %u %u %u", name, &lv, &ln, &ty, &bl, &ch, &sw, &cps) != 8) continue;
        RaggedConfig c;
        c.block = bl;
        c.chunk_values = ch;
        c.store_bytes = sw;
        c.ctas_per_sm = cps;
        if (valid_config(c)) f.table[TuneKey(name, lv, ln, ty)] = c;
    }
    fclose(fp);
}

static bool tune_file_lookup(const TuneKey &k, RaggedConfig *cfg)
{
    TuneFile &f = tune_file();
    std::lock_guard<std::mutex> lock(f.mu);
    tune_file_load(f);
    if (f.path.empty()) return false;  // no file: each context tunes for itself
    auto it = f.table.find(k);
    if (it == f.table.end()) return false;
    *cfg = it->second;
    return true;
}

static void tune_file_store(const TuneKey &k, const RaggedConfig &c)
{
    TuneFile &f = tune_file();
    std::lock_guard<std::mutex> lock(f.mu);
    tune_file_load(f);
    if (f.path.empty()) return;
    f.table[k] = c;
    // Create the parent directories if needed (best effort; existing ones stay).
    for (size_t i = f.path.find('/', 1); i != std::string::npos; i = f.path.find('/', i + 1))
        mkdir(f.path.substr(0, i).c_str(), 0755);
    FILE *fp = fopen(f.path.c_str(), "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d %d %u %u %u %u\n", std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
            c.block, c.chunk_values, c.store_bytes, c.ctas_per_sm);
    fclose(fp);
}

orand_status_t ragged_serve(orand_ctx_t ctx, const orand_request_t *reqs, size_t n, void *out_base,
                            uint64_t out_bytes, cudaStream_t stream)
{
    orand_status_t st = ctx_check(ctx);
    if (st != ORAND_OK) return st;
    if (n == 0) return ORAND_OK;
    if (reqs == nullptr) return ORAND_ERR_INVALID_ARG;
    RaggedState *s = state_of(ctx);
    if (!s) return ORAND_ERR_ALLOC;
    char *out = (char *)out_base;
    const bool check_overlap = env_flag("ORAND_CHECK_OVERLAP", false);

    // Validate and plan with the default chunk size; re-plan if the chosen
    // configuration uses another one.
    RaggedConfig cfg;
    Plan plan;
    if ((st = plan_requests(reqs, n, out, out_bytes, cfg.chunk_values, &plan, check_overlap)) != ORAND_OK)
        return st;
    if (plan.total_values == 0) return ORAND_OK;
    if (out == nullptr) return ORAND_ERR_INVALID_ARG;
    const auto klass = std::make_tuple(ilog2(plan.total_values), ilog2(n), plan.tyche.empty() ? 0 : 1);
    if (s->forced) {
        cfg = s->forced_cfg;
    } else if (s->tuned.count(klass)) {
        cfg = s->tuned[klass];
    } else if (env_flag("ORAND_AUTOTUNE", true)) {
        const TuneKey key(gpu_name(ctx->device), std::get<0>(klass), std::get<1>(klass), std::get<2>(klass));
        if (!tune_file_lookup(key, &cfg)) {
            if (s->batch_pending) cudaStreamWaitEvent(stream, s->batch_done, 0);
            if ((st = autotune(s, reqs, n, out, out_bytes, stream, &cfg)) != ORAND_OK) return st;
            tune_file_store(key, cfg);
        }
        s->tuned[klass] = cfg;
    }
    if (cfg.chunk_values != plan.chunk_values &&
        (st = plan_requests(reqs, n, out, out_bytes, cfg.chunk_values, &plan, false)) != ORAND_OK)
        return st;
    const size_t copy_bytes = copy_bucket(plan.table_bytes);
    if ((st = ensure_buffers(s, copy_bytes)) != ORAND_OK) return st;

    // The previous batch's graph must have copied the staging buffer out
    // before it is rewritten.
    cudaError_t e = cudaSuccess;
    ORAND_CUDA_TRY(cudaEventSynchronize(s->staging_free));
    write_staging(plan, out, (char *)s->h_staging);

    GraphKey key{};
    key.cfg = cfg;
    key.copy_bytes = copy_bytes;
    key.d_tables = s->d_tables;
    key.h_staging = s->h_staging;
    if (!s->have_graph || !(key == s->key)) {
        if (s->exec) {
            cudaGraphExecDestroy(s->exec);
            s->exec = nullptr;
        }
        s->have_graph = false;
        unsigned grid = 0;
        if ((st = ragged_grid(cfg, &grid)) != ORAND_OK) return st;
        cudaStream_t cs = s->capture_stream;
        ORAND_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        // Captured: table copy, an external event record (the host waits on it
        // before rewriting the staging buffer), the persistent kernel.
        cudaMemcpyAsync(s->d_tables, s->h_staging, copy_bytes, cudaMemcpyHostToDevice, cs);
        cudaEventRecordWithFlags(s->staging_free, cs, cudaEventRecordExternal);
        launch_kernel((char *)s->d_tables, cfg, grid, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) {
            log_cuda_failure("cudaStreamEndCapture", __FILE__, __LINE__, e);
            if (graph) cudaGraphDestroy(graph);
            return cuda_status(e);
        }
        e = cudaGraphInstantiate(&s->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            log_cuda_failure("cudaGraphInstantiate", __FILE__, __LINE__, e);
            return cuda_status(e);
        }
        s->key = key;
        s->have_graph = true;
        ++s->graph_builds;
    }
    if (s->batch_pending) ORAND_CUDA_TRY(cudaStreamWaitEvent(stream, s->batch_done, 0));
    ORAND_CUDA_TRY(cudaGraphLaunch(s->exec, stream));
    ORAND_CUDA_TRY(cudaEventRecord(s->batch_done, stream));
    s->batch_pending = true;
    s->last_cfg = cfg;
    ++s->graph_launches;
    return ORAND_OK;
}

orand_status_t fill_launch(int gen, int dt, uint64_t seed, uint32_t counter, uint64_t s_first, uint64_t n_streams,
                           uint64_t dps, void *out, cudaStream_t stream);

}  // namespace orand_impl

using namespace orand_impl;

extern "C" {

orand_status_t orand_fill_ragged(orand_ctx_t ctx, const orand_request_t *reqs, size_t n, void *out_base,
                                 uint64_t out_bytes, cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_ragged");
    return ragged_serve(ctx, reqs, n, out_base, out_bytes, stream);
}

orand_status_t orand_fill_ragged_serial(const orand_request_t *reqs, size_t n, void *out_base, uint64_t out_bytes,
                                        cudaStream_t stream)
{
    ORAND_NVTX_RANGE("orand_fill_ragged_serial");
    if (n == 0) return ORAND_OK;
    if (reqs == nullptr) return ORAND_ERR_INVALID_ARG;
    Plan plan;
    orand_status_t st = plan_requests(reqs, n, (const char *)out_base, out_bytes, 8192, &plan, false);
    if (st != ORAND_OK || plan.total_values == 0) return st;
    if (out_base == nullptr) return ORAND_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; ++i) {
        const orand_request_t &q = reqs[i];
        if (q.length == 0) continue;
        st = fill_launch((int)q.gen, (int)q.dtype, q.seed, q.counter, 0, 1, q.length,
                         (char *)out_base + q.out_offset_bytes, stream);
        if (st != ORAND_OK) return st;
    }
    return ORAND_OK;
}

orand_status_t orand_ragged_set_config(orand_ctx_t ctx, const orand_ragged_config_t *cfg)
{
    orand_status_t st = ctx_check(ctx);
    if (st != ORAND_OK) return st;
    RaggedState *s = state_of(ctx);
    if (!s) return ORAND_ERR_ALLOC;
    if (cfg == nullptr) {
        s->forced = false;
        return ORAND_OK;
    }
    RaggedConfig c;
    c.block = cfg->block;
    c.chunk_values = cfg->chunk_values;
    c.store_bytes = cfg->store_bytes;
    c.ctas_per_sm = cfg->ctas_per_sm;
    if (!valid_config(c)) return ORAND_ERR_INVALID_ARG;
    s->forced = true;
    s->forced_cfg = c;
    return ORAND_OK;
}

orand_status_t orand_ragged_get_config(orand_ctx_t ctx, orand_ragged_config_t *cfg)
{
    orand_status_t st = ctx_check(ctx);
    if (st != ORAND_OK) return st;
    if (cfg == nullptr) return ORAND_ERR_INVALID_ARG;
    RaggedState *s = state_of(ctx);
    if (!s) return ORAND_ERR_ALLOC;
    cfg->block = s->last_cfg.block;
    cfg->chunk_values = s->last_cfg.chunk_values;
    cfg->store_bytes = s->last_cfg.store_bytes;
    cfg->ctas_per_sm = s->last_cfg.ctas_per_sm;
    return ORAND_OK;
}

orand_status_t orand_ragged_stats(orand_ctx_t ctx, orand_ragged_stats_t *stats)
{
    orand_status_t st = ctx_check(ctx);
    if (st != ORAND_OK) return st;
    if (stats == nullptr) return ORAND_ERR_INVALID_ARG;
    RaggedState *s = state_of(ctx);
    if (!s) return ORAND_ERR_ALLOC;
    stats->graph_launches = s->graph_launches;
    stats->graph_builds = s->graph_builds;
    stats->tune_runs = s->tune_runs;
    stats->tuned_classes = s->tuned.size();
    return ORAND_OK;
}

}  // extern "C"
