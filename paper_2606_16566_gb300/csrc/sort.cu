// sort.cu -- stage 2 of the 3DGS pipeline (Local-GS Sec. II-A): a parallel
// prefix scan over tiles-touched, duplication of every visible Gaussian into
// one 64-bit key (tile_id << 32 | depth bits) per tile of its rect, a stable
// LSD radix sort of the (key, value) pairs, and per-tile ranges.
//
// The instance count K is only known on the device. Every kernel reads it from
// the caller's status words, so the whole stage is enqueued without a host
// round trip (and is capturable in a CUDA graph); grids are sized for the
// caller's capacity and blocks past K exit at once.
//
// Radix sort: 8-bit digits over the significant bits only (32 depth bits +
// ceil(log2(n_tiles)) tile bits). Each pass is reduce-then-scan: an upsweep
// builds per-block digit histograms, a scan turns each digit row into block
// offsets, and a downsweep ranks keys stably inside 4096-key blocks (warp
// __match_any_sync + per-warp counters), reorders them in shared memory and
// writes runs of equal digits contiguously.
#include "common.cuh"
#include "host.h"

#include <mutex>

namespace lgs {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 2048

constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;  // 4096

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one value per thread (blockDim.x multiple of 32).
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = THREADS / 32;
        uint32_t s = lane < NW ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) warp_sums[lane] = s;  // inclusive
    }
    __syncthreads();
    total = warp_sums[THREADS / 32 - 1];
    uint32_t excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0u);
    __syncthreads();
    return excl;
}

// ------------------------------------------------------------------ scan of tiles
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce(const uint32_t* tiles, int64_t m,
                                                            uint64_t* block_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < m) s += tiles[i];
    }
    // 64-bit reduction: warp shuffles then shared memory
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ uint64_t w64[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) w64[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += w64[w];
        block_sums[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of the block sums; K -> status. Each block sum
// is < 2^32 (at most 2048 Gaussians of at most 2^16 tiles each would exceed it
// only for absurd rects, which the capacity check then rejects).
__global__ void __launch_bounds__(1024) scan_block_sums(uint64_t* block_sums, int64_t nb,
                                                        int64_t* status, int64_t capacity) {
    __shared__ uint32_t ws[32];
    uint64_t carry = 0;
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < nb ? block_sums[i] : 0ull;
        const uint32_t v32 = v > 0xffffffffull ? 0xffffffffu : (uint32_t)v;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<1024>(v32, ws, tot);
        if (i < nb) block_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        status[LGS_ST_NUM_INSTANCES] = (int64_t)carry;
        if ((int64_t)carry > capacity) report_error(status, LGS_ERR_CAPACITY, (int64_t)carry);
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_downsweep(const uint32_t* tiles, int64_t m,
                                                               const uint64_t* block_sums,
                                                               uint32_t* offsets) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // blocked arrangement: thread t owns items [t*ITEMS, (t+1)*ITEMS) of the block
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        v[k] = i < m ? tiles[i] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<SCAN_THREADS>(s, ws, tot);
    // per block K may exceed 2^32 only if the capacity check fails; offsets wrap
    // harmlessly then because emission is skipped.
    uint32_t run = (uint32_t)block_sums[blockIdx.x] + ex;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (i < m) offsets[i] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------------ emission
// key = (global tile id << 32) | bits(depth); value = v*N + i.
__global__ void __launch_bounds__(256) emit_keys(const uint32_t* tiles, const uint32_t* offsets,
                                                 const uint64_t* rect, const float* depth,
                                                 int64_t m, int64_t n, const int64_t* status,
                                                 int64_t capacity, Views vs, uint64_t* keys,
                                                 uint32_t* vals) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m) return;
    if (status[LGS_ST_NUM_INSTANCES] > capacity) return;
    const uint32_t nt = tiles[idx];
    if (nt == 0) return;
    const int v = (int)(idx / n);
    const ViewRec& c = vs.v[v];
    const uint64_t r = rect[idx];
    const int x0 = (int)(r & 0xffff), y0 = (int)((r >> 16) & 0xffff);
    const int x1 = (int)((r >> 32) & 0xffff), y1 = (int)((r >> 48) & 0xffff);
    const uint32_t dbits = __float_as_uint(depth[idx]);
    uint32_t off = offsets[idx];
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
            const uint64_t tid = (uint64_t)(c.tile_off + (uint32_t)(ty * c.gx + tx));
            keys[off] = (tid << 32) | dbits;
            vals[off] = (uint32_t)idx;
            ++off;
        }
}

// ------------------------------------------------------------------ radix passes
__device__ __forceinline__ int64_t sort_count(const int64_t* status, int64_t capacity) {
    int64_t K = status[LGS_ST_NUM_INSTANCES];
    return K > capacity ? 0 : K;
}

__global__ void __launch_bounds__(SORT_THREADS) radix_upsweep(const uint64_t* keys,
                                                              const int64_t* status,
                                                              int64_t capacity, int shift,
                                                              uint32_t* hist, int nb) {
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t K = sort_count(status, capacity);
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const uint32_t lane = threadIdx.x & 31;
    if (base < K) {
#pragma unroll 4
        for (int k = 0; k < SORT_ITEMS; ++k) {
            const int64_t i = base + (int64_t)k * SORT_THREADS + threadIdx.x;
            const uint32_t d = i < K ? (uint32_t)((keys[i] >> shift) & 0xffu) : 0x100u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (d < 0x100u && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], __popc(peers));
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's row over blocks.
__global__ void __launch_bounds__(1024) radix_scan_rows(uint32_t* hist, int nb,
                                                        uint32_t* digit_total) {
    __shared__ uint32_t ws[32];
    uint32_t* row = hist + (int64_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? row[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<1024>(v, ws, tot);
        if (i < nb) row[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

struct DownSmem {
    uint32_t base[RADIX];            // global output base per digit for this block
    uint32_t start[RADIX];           // block-local start of each digit
    uint32_t cnt[2][SORT_THREADS / 32][RADIX];
    uint32_t ws[32];
    uint64_t keys[SORT_TILE];
    uint32_t vals[SORT_TILE];
};

__global__ void __launch_bounds__(SORT_THREADS) radix_downsweep(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const int64_t* status, int64_t capacity, int shift,
    const uint32_t* hist, int nb, const uint32_t* digit_total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem& S = *reinterpret_cast<DownSmem*>(smem_raw);
    const int64_t K = sort_count(status, capacity);
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    if (base >= K) return;
    const int n_valid = (int)min((int64_t)SORT_TILE, K - base);
    const int t = threadIdx.x, warp = t >> 5;

    // global digit bases: exclusive scan over digits of the totals + this block's row offset
    {
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<SORT_THREADS>(digit_total[t], S.ws, tot);
        S.base[t] = ex + hist[(int64_t)t * nb + blockIdx.x];
    }
#pragma unroll
    for (int w = 0; w < SORT_THREADS / 32; ++w) {
        S.cnt[0][w][t] = 0;
        S.cnt[1][w][t] = 0;
    }
    uint64_t k[SORT_ITEMS];
    uint32_t vv[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const int j = i * SORT_THREADS + t;
        if (j < n_valid) {
            k[i] = kin[base + j];
            vv[i] = vin[base + j];
        } else {
            k[i] = ~0ull;   // digit 255 and ranked after every valid key
            vv[i] = 0;
        }
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
    uint32_t run = 0;                  // thread t: running count of digit t
    uint16_t rank[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const int b = i & 1;
        const uint32_t d = (uint32_t)((k[i] >> shift) & 0xffu);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t r = __popc(peers & lt);
        if (r == 0) S.cnt[b][warp][d] = __popc(peers);
        __syncthreads();
#pragma unroll
        for (int w = 0; w < SORT_THREADS / 32; ++w) {
            const uint32_t c = S.cnt[b][w][t];
            S.cnt[b][w][t] = run;
            run += c;
            S.cnt[b ^ 1][w][t] = 0;
        }
        __syncthreads();
        rank[i] = (uint16_t)(S.cnt[b][warp][d] + r);
    }
    {
        uint32_t tot;
        S.start[t] = block_exclusive_scan<SORT_THREADS>(run, S.ws, tot);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const int j = i * SORT_THREADS + t;
        if (j < n_valid) {
            const uint32_t d = (uint32_t)((k[i] >> shift) & 0xffu);
            const uint32_t pos = S.start[d] + rank[i];
            S.keys[pos] = k[i];
            S.vals[pos] = vv[i];
        }
    }
    __syncthreads();
    for (int j = t; j < n_valid; j += SORT_THREADS) {
        const uint64_t key = S.keys[j];
        const uint32_t d = (uint32_t)((key >> shift) & 0xffu);
        const uint32_t gpos = S.base[d] + (uint32_t)j - S.start[d];
        kout[gpos] = key;
        vout[gpos] = S.vals[j];
    }
}

// ------------------------------------------------------------------ ranges
__global__ void tile_ranges(const uint64_t* keys, const int64_t* status, int64_t capacity,
                            uint32_t* ranges) {
    const int64_t K = sort_count(status, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t tile = (uint32_t)(keys[i] >> 32);
        if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[2 * (int64_t)tile] = (uint32_t)i;
        if (i == K - 1 || (uint32_t)(keys[i + 1] >> 32) != tile)
            ranges[2 * (int64_t)tile + 1] = (uint32_t)(i + 1);
    }
}

// ------------------------------------------------------------------ workspace
struct SortWs {
    uint32_t* offsets;     // [m]
    uint64_t* block_sums;  // [ceil(m/2048)]
    uint64_t* keys_alt;    // [capacity]
    uint32_t* vals_alt;    // [capacity]
    uint32_t* hist;        // [256 * nb]
    uint32_t* digit_total; // [256]
};

constexpr size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of the sort workspace for m entries and an instance capacity
// (usable in constant expressions).
constexpr size_t sort_ws_bytes(int64_t m, int64_t capacity) {
    const int64_t nscan = (m + SCAN_TILE - 1) / SCAN_TILE;
    const int64_t nb = (capacity + SORT_TILE - 1) / SORT_TILE;
    return align_up(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1)) +
           align_up(sizeof(uint64_t) * (size_t)(nscan > 0 ? nscan : 1)) +
           align_up(sizeof(uint64_t) * (size_t)(capacity > 0 ? capacity : 1)) +
           align_up(sizeof(uint32_t) * (size_t)(capacity > 0 ? capacity : 1)) +
           align_up(sizeof(uint32_t) * RADIX * (size_t)(nb > 0 ? nb : 1)) +
           align_up(sizeof(uint32_t) * RADIX);
}

inline size_t sort_ws_layout(int64_t m, int64_t capacity, char* base, SortWs* ws) {
    const int64_t nscan = (m + SCAN_TILE - 1) / SCAN_TILE;
    const int64_t nb = (capacity + SORT_TILE - 1) / SORT_TILE;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align_up(bytes); return p; };
    char* p0 = take(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    char* p1 = take(sizeof(uint64_t) * (size_t)(nscan > 0 ? nscan : 1));
    char* p2 = take(sizeof(uint64_t) * (size_t)(capacity > 0 ? capacity : 1));
    char* p3 = take(sizeof(uint32_t) * (size_t)(capacity > 0 ? capacity : 1));
    char* p4 = take(sizeof(uint32_t) * RADIX * (size_t)(nb > 0 ? nb : 1));
    char* p5 = take(sizeof(uint32_t) * RADIX);
    if (ws) {
        ws->offsets = reinterpret_cast<uint32_t*>(p0);
        ws->block_sums = reinterpret_cast<uint64_t*>(p1);
        ws->keys_alt = reinterpret_cast<uint64_t*>(p2);
        ws->vals_alt = reinterpret_cast<uint32_t*>(p3);
        ws->hist = reinterpret_cast<uint32_t*>(p4);
        ws->digit_total = reinterpret_cast<uint32_t*>(p5);
    }
    return off;
}

inline int sort_passes(uint32_t n_tiles) {
    int tile_bits = 0;
    while (tile_bits < 32 && (1ull << tile_bits) < (uint64_t)n_tiles) ++tile_bits;
    return (32 + tile_bits + 7) / 8;
}

}  // namespace lgs

using namespace lgs;

extern "C" size_t lgs_sort_workspace_size(int64_t m, int64_t capacity) {
    if (m < 0 || capacity < 0) return 0;
    return sort_ws_layout(m, capacity, nullptr, nullptr);
}

// Enqueues the full stage given a workspace layout (shared by the entry points).
static lgs_status sort_enqueue(const lgs_pre_out* pre, int64_t n, const Views* vs,
                                       int64_t capacity, uint64_t* keys, uint32_t* vals,
                                       uint32_t* ranges, const SortWs* ws, int64_t* d_status,
                                       cudaStream_t s) {
    const int64_t m = n * vs->n;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)vs->n_tiles, s);
    if (e != cudaSuccess) return LGS_ERR_CUDA;
    if (m == 0) {
        e = cudaMemsetAsync(d_status + LGS_ST_NUM_INSTANCES, 0, sizeof(int64_t), s);
        return cuda_status(e);
    }
    const int64_t nscan = (m + SCAN_TILE - 1) / SCAN_TILE;
    scan_reduce<<<(unsigned)nscan, SCAN_THREADS, 0, s>>>(pre->tiles, m, ws->block_sums);
    scan_block_sums<<<1, 1024, 0, s>>>(ws->block_sums, nscan, d_status, capacity);
    scan_downsweep<<<(unsigned)nscan, SCAN_THREADS, 0, s>>>(pre->tiles, m, ws->block_sums,
                                                            ws->offsets);
    const int passes = sort_passes(vs->n_tiles);
    // emit so that the last pass lands in the caller's buffers
    uint64_t* ka = (passes & 1) ? ws->keys_alt : keys;
    uint32_t* va = (passes & 1) ? ws->vals_alt : vals;
    uint64_t* kb = (passes & 1) ? keys : ws->keys_alt;
    uint32_t* vb = (passes & 1) ? vals : ws->vals_alt;
    emit_keys<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pre->tiles, ws->offsets, pre->rect,
                                                          pre->depth, m, n, d_status, capacity,
                                                          *vs, ka, va);
    const int nb = (int)((capacity + SORT_TILE - 1) / SORT_TILE);
    if (nb > 0) {
        static_assert(sizeof(DownSmem) < 227 * 1024, "smem");
        cudaFuncSetAttribute(radix_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(DownSmem));
        for (int p = 0; p < passes; ++p) {
            const int shift = 8 * p;
            radix_upsweep<<<nb, SORT_THREADS, 0, s>>>(ka, d_status, capacity, shift, ws->hist, nb);
            radix_scan_rows<<<RADIX, 1024, 0, s>>>(ws->hist, nb, ws->digit_total);
            radix_downsweep<<<nb, SORT_THREADS, sizeof(DownSmem), s>>>(
                ka, va, kb, vb, d_status, capacity, shift, ws->hist, nb, ws->digit_total);
            uint64_t* tk = ka; ka = kb; kb = tk;
            uint32_t* tv = va; va = vb; vb = tv;
        }
        tile_ranges<<<152 * 4, 256, 0, s>>>(keys, d_status, capacity, ranges);
    }
    return cuda_status(cudaGetLastError());
}

extern "C" lgs_status lgs_sort(const lgs_pre_out* pre, int64_t n, const lgs_camera* cams,
                               int32_t n_views, const lgs_config* cfg, int64_t capacity,
                               uint64_t* keys, uint32_t* vals, uint32_t* ranges, void* workspace,
                               size_t workspace_bytes, int64_t* d_status, void* stream) {
    if (!pre || !keys || !vals || !ranges || !d_status) return LGS_ERR_ARG;
    if (n < 0 || capacity < 0 || capacity >= (1ll << 32)) return LGS_ERR_ARG;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    if (!pre->tiles || !pre->rect || !pre->depth) return LGS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(pre->rect) & 7u) || (reinterpret_cast<uintptr_t>(keys) & 7u))
        return LGS_ERR_ALIGN;
    const int64_t m = n * (int64_t)n_views;
    if (m >= (1ll << 32)) return LGS_ERR_UNSUPPORTED;
    const size_t need = sort_ws_layout(m, capacity, nullptr, nullptr);
    if (!workspace || workspace_bytes < need) return LGS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return LGS_ERR_ALIGN;
    SortWs ws;
    sort_ws_layout(m, capacity, static_cast<char*>(workspace), &ws);
    return sort_enqueue(pre, n, &vs, capacity, keys, vals, ranges, &ws, d_status,
                            static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------ static scratch variant
// lgs_sort_static: lgs_sort for callers that cannot allocate device memory.
// Its scratch lives in a file-scope device array, so every GPU that loads the
// library holds LGS_SORT_STATIC_BYTES of it until the process exits.
namespace lgs {
constexpr size_t kSortStaticBytes =
    sort_ws_bytes(LGS_SORT_STATIC_MAX_ENTRIES, LGS_SORT_STATIC_MAX_INSTANCES);
static_assert(kSortStaticBytes <= (size_t)LGS_SORT_STATIC_BYTES,
              "LGS_SORT_STATIC_BYTES must cover the workspace at the stated maxima");
}  // namespace lgs

static __device__ __align__(256) unsigned char g_sort_static_scratch[LGS_SORT_STATIC_BYTES];

// Device address of the array on the current device. In host code the
// symbol's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
static lgs_status sort_static_scratch(void** out) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static void* ptr[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LGS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_static_scratch) != cudaSuccess || !p) return LGS_ERR_CUDA;
        ptr[dev] = p;
    }
    *out = ptr[dev];
    return LGS_OK;
}

extern "C" lgs_status lgs_sort_static(const lgs_pre_out* pre, int64_t n, const lgs_camera* cams,
                                      int32_t n_views, const lgs_config* cfg, int64_t capacity,
                                      uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                                      int64_t* d_status, void* stream) {
    if (!pre || !keys || !vals || !ranges || !d_status) return LGS_ERR_ARG;
    if (n < 0 || capacity < 0) return LGS_ERR_ARG;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    const int64_t m = n * (int64_t)n_views;
    if (m > LGS_SORT_STATIC_MAX_ENTRIES || capacity > LGS_SORT_STATIC_MAX_INSTANCES)
        return LGS_ERR_UNSUPPORTED;
    if (!pre->tiles || !pre->rect || !pre->depth) return LGS_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(pre->rect) & 7u) || (reinterpret_cast<uintptr_t>(keys) & 7u))
        return LGS_ERR_ALIGN;
    void* scratch = nullptr;
    st = sort_static_scratch(&scratch);
    if (st != LGS_OK) return st;
    SortWs ws;
    sort_ws_layout(m, capacity, static_cast<char*>(scratch), &ws);
    return sort_enqueue(pre, n, &vs, capacity, keys, vals, ranges, &ws, d_status,
                        static_cast<cudaStream_t>(stream));
}
