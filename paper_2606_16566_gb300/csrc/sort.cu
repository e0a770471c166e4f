// sort.cu -- stage 2 of the 3DGS pipeline (Local-GS Sec. II-A): duplication of
// every visible (view, Gaussian) entry into one instance per tile it touches,
// ordering of the instances by the 64-bit key (tile_id << 32 | depth bits)
// with ties kept in emission order, and per-tile ranges.
//
// The instance count K is only known on the device. Every kernel reads it from
// the caller's status words, so the whole stage is enqueued without a host
// round trip (and is capturable in a CUDA graph); grids are sized for the
// caller's capacity and blocks past K exit at once.
//
// Depth first, tiles second:
//  1. a stable LSD radix sort of the visible entries by their 32 depth bits
//     (the first pass reads tiles-touched and depth directly and drops the
//     culled entries);
//  2. an exclusive scan of tiles-touched in that order gives every entry its
//     instance offset and K (with LGS_FLAG_TIGHT the counts are those of the
//     tight box, computed here: count_tight);
//  3. emission writes (tile id, entry) pairs entry by entry in depth order;
//  4. stable LSD passes over the ceil(log2(tiles)) tile-id bits only;
//  5. per-tile ranges from the sorted tile ids.
// Inside a tile the instances keep their emission order, which is (depth,
// entry index), so the result is bit for bit the stable sort of the 64-bit
// keys -- with 4 passes over the (visible) entries instead of 4 passes over the K
// instances for the depth bits.
// Every radix pass is one "onesweep" kernel: per 6144-element block a stable
// in-shared-memory ranking and a decoupled look-back over the earlier blocks'
// digit counts (see onesweep_pass).
#include "common.cuh"
#include "host.h"

#include <mutex>

namespace lgs {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 2048

constexpr int RADIX = 256;

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

// ------------------------------------------------------------------ element counts
// Element count of a pass: the device word *cnt (0 when it exceeds the host
// bound n, e.g. K beyond the capacity) when cnt is given, else n.
__device__ __forceinline__ int64_t pass_count(const int64_t* cnt, int64_t n) {
    if (!cnt) return n;
    const int64_t k = *cnt;
    return k > n ? 0 : k;
}

__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ int64_t sort_count(const int64_t* status, int64_t capacity) {
    return pass_count(status + LGS_ST_NUM_INSTANCES, capacity);
}

// ------------------------------------------------------------------ scan of tiles
// Entries at or past the device count *mv (the visible entries) count as 0.
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce(const uint32_t* tiles, int64_t m, const int64_t* mv,
                                                            uint64_t* block_sums) {
    m = pass_count(mv, m);
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

__global__ void __launch_bounds__(SCAN_THREADS) scan_downsweep(const uint32_t* tiles, int64_t m, const int64_t* mv,
                                                               const uint64_t* block_sums,
                                                               uint32_t* offsets) {
    __shared__ uint32_t ws[32];
    m = pass_count(mv, m);
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // blocked arrangement: thread t owns items [t*ITEMS, (t+1)*ITEMS) of the
    // block, loaded 16 B at a time where they all lie below the count (the
    // block starts on a 2048-element boundary of a 256-B aligned buffer)
    static_assert(SCAN_ITEMS % 4 == 0, "whole 16-B groups per thread");
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
    const int64_t first = base + (int64_t)threadIdx.x * SCAN_ITEMS;
    if (first + SCAN_ITEMS <= m) {
        const uint4* t4 = reinterpret_cast<const uint4*>(tiles + first);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
            const uint4 w = t4[q];
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = first + k < m ? tiles[first + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) s += v[k];
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<SCAN_THREADS>(s, ws, tot);
    // per block K may exceed 2^32 only if the capacity check fails; offsets wrap
    // harmlessly then because emission is skipped.
    uint32_t run = (uint32_t)block_sums[blockIdx.x] + ex;
    uint32_t o[SCAN_ITEMS];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        o[k] = run;
        run += v[k];
    }
    if (first + SCAN_ITEMS <= m) {
        uint4* o4 = reinterpret_cast<uint4*>(offsets + first);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; ++q) o4[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k)
            if (first + k < m) offsets[first + k] = o[k];
    }
}

// ------------------------------------------------------------------ emission
// One (tile id, value) pair per tile of each visible entry's rect, entries
// taken in depth order (order[j]), tiles row-major inside the rect; value =
// entry index v*N + i. The 32 entries of a warp own one contiguous range of
// instances (their offsets come from the scan), so the warp writes that range
// cooperatively: lane l produces instances l, l+32, ... of the range, finds
// the owning entry by a binary search over the warp's inclusive prefix counts
// (shuffles), and the stores of a warp land on consecutive addresses.
template <typename KT>
__global__ void __launch_bounds__(256) emit_pairs(const uint32_t* order, const uint32_t* tiles,
                                                  const uint32_t* offsets, const uint64_t* rect,
                                                  int64_t m, int64_t n, int64_t* status,
                                                  int64_t capacity, Views vs, KT* tkey,
                                                  uint32_t* tval) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wbase = idx - (threadIdx.x & 31);
    const int lane = threadIdx.x & 31;
    const bool valid = idx < m;
    const bool fits = status[LGS_ST_NUM_INSTANCES] <= capacity;
    const uint32_t cnt = (valid && fits) ? tiles[idx] : 0u;
    const uint32_t ent = cnt ? order[idx] : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (wbase < m && total > 0) {
        const uint32_t start = __shfl_sync(0xffffffffu, valid ? offsets[idx] - (incl - cnt) : 0u, 0);
        // per-entry data the owners hand out
        uint32_t x0 = 0, y0 = 0, wd = 1, toff = 0, gx = 1;
        if (cnt) {
            const uint64_t r = rect[ent];
            x0 = (uint32_t)(r & 0xffff);
            y0 = (uint32_t)((r >> 16) & 0xffff);
            wd = (uint32_t)((r >> 32) & 0xffff) - x0;
            const ViewRec& c = vs.v[(int)(ent / (uint64_t)n)];
            toff = c.tile_off;
            gx = (uint32_t)c.gx;
        }
        const uint32_t excl = incl - cnt;
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + lane;
            // owner = first lane with incl > e
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                if (v <= e) lo += step;
            }
            const int own = lo;
            const uint32_t k = e - __shfl_sync(0xffffffffu, excl, own);
            const uint32_t ox0 = __shfl_sync(0xffffffffu, x0, own);
            const uint32_t oy0 = __shfl_sync(0xffffffffu, y0, own);
            const uint32_t ow = __shfl_sync(0xffffffffu, wd, own);
            const uint32_t otoff = __shfl_sync(0xffffffffu, toff, own);
            const uint32_t ogx = __shfl_sync(0xffffffffu, gx, own);
            const uint32_t oent = __shfl_sync(0xffffffffu, ent, own);
            if (e < total) {
                const uint32_t ry = k / ow, rx = k - ry * ow;
                const uint32_t tile = otoff + (oy0 + ry) * ogx + ox0 + rx;
                if (LGS_CHECK((int64_t)start + e < capacity, 1, status) &&
                    LGS_CHECK(tile < vs.n_tiles, 2, status) && LGS_CHECK(oent < (uint64_t)m, 3, status)) {
                    tkey[start + e] = (KT)tile;
                    tval[start + e] = oent;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ tight-box emission
// With LGS_FLAG_TIGHT an entry emits only the tiles of its rect that its tight
// box (TightBox / tight_tile_rows) reaches: column strip by column strip, tile
// rows ascending inside a column. Counting (count_tight) and emission
// (emit_pairs_tight) walk the same column items with the same function, so the
// counts the scan turns into offsets are exactly the instances emitted.
//
// Both kernels give each warp 32 consecutive entries of the depth order; each
// lane loads its entry's rect and box, the entries expand into column items
// (one per rect column), and the lanes take 32 items at a time, each finding
// its owner entry by a binary search over the warp's inclusive column counts,
// so wide and narrow Gaussians share the work evenly.
struct TightLane {
    uint32_t x0, y0, y1, wd, toff, gx, ent;
    TightBox tb;
};

// Loads a visible entry's rect, conic and mean and forms its tight box; with
// `rec`, also writes the entry's emission record at depth-order index idx.
__device__ __forceinline__ TightLane tight_lane_load(uint32_t ent, bool live, const uint64_t* rect,
                                                     const float4* xy, const float4* conic,
                                                     const Views& vs, int64_t n, uint4* rec = nullptr,
                                                     int64_t idx = 0) {
    TightLane L{};
    L.gx = 1;
    L.ent = ent;
    if (live) {
        const uint64_t r = rect[ent];
        L.x0 = (uint32_t)(r & 0xffff);
        L.y0 = (uint32_t)((r >> 16) & 0xffff);
        L.wd = (uint32_t)((r >> 32) & 0xffff) - L.x0;
        L.y1 = (uint32_t)((r >> 48) & 0xffff);
        const ViewRec& cv = vs.v[(int)(ent / (uint64_t)n)];
        L.toff = cv.tile_off;
        L.gx = (uint32_t)cv.gx;
        const float4 co = conic[ent];
        const float4 p = xy[ent];
        const float mux = __fadd_rn(p.x, p.z), muy = __fadd_rn(p.y, p.w);
        L.tb = tight_box(co.x, co.y, co.z, co.w, mux, muy);
        if (rec) {
            rec[2 * idx] = make_uint4((uint32_t)r, (uint32_t)(r >> 32), __float_as_uint(mux), __float_as_uint(muy));
            rec[2 * idx + 1] = make_uint4(__float_as_uint(co.x), __float_as_uint(co.y), __float_as_uint(co.z),
                                          __float_as_uint(co.w));
        }
    }
    return L;
}

// The same lane state from the emission record count_tight left at depth-order
// index idx ((rect, mean x, mean y), conic: two coalesced 16-B loads instead of
// a second gather of rect, conic and mean).
__device__ __forceinline__ TightLane tight_lane_from(uint32_t ent, bool live, uint4 a, uint4 c,
                                                     const Views& vs, int64_t n) {
    TightLane L{};
    L.gx = 1;
    L.ent = ent;
    if (live) {
        L.x0 = a.x & 0xffffu;
        L.y0 = a.x >> 16;
        L.wd = (a.y & 0xffffu) - L.x0;
        L.y1 = a.y >> 16;
        const ViewRec& cv = vs.v[(int)(ent / (uint64_t)n)];
        L.toff = cv.tile_off;
        L.gx = (uint32_t)cv.gx;
        L.tb = tight_box(__uint_as_float(c.x), __uint_as_float(c.y), __uint_as_float(c.z), __uint_as_float(c.w),
                         __uint_as_float(a.z), __uint_as_float(a.w));
    }
    return L;
}

__device__ __forceinline__ TightLane tight_lane_rec(uint32_t ent, bool live, const uint4* rec, int64_t idx,
                                                    const Views& vs, int64_t n) {
    uint4 a = make_uint4(0u, 0u, 0u, 0u), c = a;
    if (live) {
        a = rec[2 * idx];
        c = rec[2 * idx + 1];
    }
    return tight_lane_from(ent, live, a, c, vs, n);
}

// The tight box of lane `own`'s entry, broadcast to the calling lane.
__device__ __forceinline__ TightBox tight_box_of(const TightBox& tb, int own) {
    TightBox o;
    o.mux = __shfl_sync(0xffffffffu, tb.mux, own);
    o.muy = __shfl_sync(0xffffffffu, tb.muy, own);
    o.a = __shfl_sync(0xffffffffu, tb.a, own);
    o.b = __shfl_sync(0xffffffffu, tb.b, own);
    o.ic = __shfl_sync(0xffffffffu, tb.ic, own);
    o.det = __shfl_sync(0xffffffffu, tb.det, own);
    o.ct = __shfl_sync(0xffffffffu, tb.ct, own);
    o.xr = __shfl_sync(0xffffffffu, tb.xr, own);
    o.bdy = __shfl_sync(0xffffffffu, tb.bdy, own);
    o.dy = __shfl_sync(0xffffffffu, tb.dy, own);
    o.kind = __shfl_sync(0xffffffffu, tb.kind, own);
    return o;
}

__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// first lane whose inclusive count exceeds e
__device__ __forceinline__ int owner_lane(uint32_t incl, uint32_t e) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
        if (v <= e) lo += step;
    }
    return lo;
}

// Tight instance count of the entries the 32 lanes of a warp hold (lane
// state L; a lane without an entry has L.wd = 0), returned to each lane. The
// entries expand into column items that the lanes take 32 at a time (owner
// found by a binary search over the inclusive column counts), so wide and
// narrow Gaussians share the work evenly; cnt = the warp's 32 shared counters.
template <int TW, int TH>
__device__ __forceinline__ uint32_t warp_tight_count(const TightLane& L, uint32_t* cnt) {
    const int lane = threadIdx.x & 31;
    cnt[lane] = 0u;
    __syncwarp();
    const uint32_t iw = warp_inclusive_sum(L.wd);
    const uint32_t items = __shfl_sync(0xffffffffu, iw, 31);
    const uint32_t ew = iw - L.wd;
    for (uint32_t e0 = 0; e0 < items; e0 += 32) {
        const uint32_t e = e0 + lane;
        const int own = owner_lane(iw, e);
        const uint32_t col = e - __shfl_sync(0xffffffffu, ew, own);
        const uint32_t ox0 = __shfl_sync(0xffffffffu, L.x0, own);
        const int oy0 = (int)__shfl_sync(0xffffffffu, L.y0, own);
        const int oy1 = (int)__shfl_sync(0xffffffffu, L.y1, own);
        const TightBox ot = tight_box_of(L.tb, own);
        if (e < items) {
            int rlo, rhi;
            const int k = tight_tile_rows(ot, (int)(ox0 + col) * TW, TW, TH, oy0, oy1, &rlo, &rhi);
            if (k) atomicAdd(&cnt[own], (uint32_t)k);
        }
    }
    __syncwarp();
    const uint32_t r = cnt[lane];
    __syncwarp();
    return r;
}

// Tight instance count of every entry in depth order: tiles_sorted[j] =
// instances that emission will write for entry order[j] (0 past the visible
// entries).
template <int TW, int TH>
__global__ void __launch_bounds__(256) count_tight(const uint32_t* order,
                                                   const uint64_t* rect, const float4* xy,
                                                   const float4* conic, const uint4* emit, int64_t m,
                                                   const int64_t* mv, int64_t n, Views vs,
                                                   uint32_t* tiles_sorted, uint4* rec) {
    __shared__ uint32_t cnt[256];
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wbase = idx - (threadIdx.x & 31);
    if (wbase >= m) return;
    const bool valid = idx < m;
    const bool visible = idx < pass_count(mv, m);
    const uint32_t ent = visible ? order[idx] : 0u;
    // the first entry pass kept only visible entries, so every entry before
    // the visible count has a non-empty rect
    TightLane L;
    if (emit) {
        // one 32-B record per entry (written by the preprocess), copied to
        // the depth-ordered records of the emission
        uint4 a = make_uint4(0u, 0u, 0u, 0u), c = a;
        if (visible) {
            a = emit[2 * (int64_t)ent];
            c = emit[2 * (int64_t)ent + 1];
            rec[2 * idx] = a;
            rec[2 * idx + 1] = c;
        }
        L = tight_lane_from(ent, visible, a, c, vs, n);
    } else {
        L = tight_lane_load(ent, visible, rect, xy, conic, vs, n, rec, idx);
    }
    const uint32_t c = warp_tight_count<TW, TH>(L, cnt + (threadIdx.x & ~31));
    if (valid) tiles_sorted[idx] = c;
}

// Emission of the tight instances: entry e's instances fill exactly
// [offsets[e], offsets[e] + tiles_sorted[e]); a warp lays the runs of its column
// items out one after the other from its first offset (warp scan of the run
// lengths). Should the recount ever differ from count_tight's (it cannot: same
// function, same inputs), the warp writes only inside its own range, pads it
// with tile 0 / entry 0 and records LGS_ERR_INTERNAL.
template <int TW, int TH, typename KT>
__global__ void __launch_bounds__(256) emit_pairs_tight(const uint32_t* order, const uint32_t* tiles_sorted,
                                                        const uint32_t* offsets, const uint4* rec,
                                                        int64_t m, const int64_t* mv, int64_t n, int64_t* status,
                                                        int64_t capacity, Views vs, KT* tkey,
                                                        uint32_t* tval) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wbase = idx - (threadIdx.x & 31);
    const int lane = threadIdx.x & 31;
    const bool valid = idx < pass_count(mv, m);
    const bool fits = status[LGS_ST_NUM_INSTANCES] <= capacity;
    const uint32_t cnt = (valid && fits) ? tiles_sorted[idx] : 0u;
    const uint32_t incl = warp_inclusive_sum(cnt);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (wbase < m && total > 0) {
        const uint32_t start = __shfl_sync(0xffffffffu, valid ? offsets[idx] - (incl - cnt) : 0u, 0);
        const TightLane L = tight_lane_rec(cnt ? order[idx] : 0u, cnt != 0u, rec, idx, vs, n);
        const uint32_t iw = warp_inclusive_sum(L.wd);
        const uint32_t items = __shfl_sync(0xffffffffu, iw, 31);
        const uint32_t ew = iw - L.wd;
        uint32_t run = 0;
        for (uint32_t e0 = 0; e0 < items; e0 += 32) {
            const uint32_t e = e0 + lane;
            const int own = owner_lane(iw, e);
            const uint32_t col = e - __shfl_sync(0xffffffffu, ew, own);
            const uint32_t ox0 = __shfl_sync(0xffffffffu, L.x0, own);
            const int oy0 = (int)__shfl_sync(0xffffffffu, L.y0, own);
            const int oy1 = (int)__shfl_sync(0xffffffffu, L.y1, own);
            const uint32_t otoff = __shfl_sync(0xffffffffu, L.toff, own);
            const uint32_t ogx = __shfl_sync(0xffffffffu, L.gx, own);
            const uint32_t oent = __shfl_sync(0xffffffffu, L.ent, own);
            const TightBox ot = tight_box_of(L.tb, own);
            const uint32_t tx = ox0 + col;
            int rlo = 0, rhi = -1;
            uint32_t k = 0;
            if (e < items) k = (uint32_t)tight_tile_rows(ot, (int)tx * TW, TW, TH, oy0, oy1, &rlo, &rhi);
            const uint32_t ik = warp_inclusive_sum(k);
            const uint32_t rtot = __shfl_sync(0xffffffffu, ik, 31);
            // the round's rtot instances (column after column, rows ascending)
            // are written by consecutive lanes: output q belongs to the lane
            // whose inclusive row count first exceeds q, so the stores of a
            // warp are contiguous instead of strided by the columns' heights
            const uint32_t tfirst = otoff + (uint32_t)rlo * ogx + tx;   // tile of the column's first row
            for (uint32_t q0 = 0; q0 < rtot; q0 += 32) {
                const uint32_t q = q0 + lane;
                const int ow = owner_lane(ik, q);
                const uint32_t qb = __shfl_sync(0xffffffffu, ik - k, ow);
                const uint32_t tb = __shfl_sync(0xffffffffu, tfirst, ow);
                const uint32_t tg = __shfl_sync(0xffffffffu, ogx, ow);
                const uint32_t te = __shfl_sync(0xffffffffu, oent, ow);
                const uint32_t pos = run + q;
                const uint32_t tile = tb + (q - qb) * tg;
                if (q < rtot && pos < total && LGS_CHECK((int64_t)start + pos < capacity, 4, status) &&
                    LGS_CHECK(tile < vs.n_tiles, 5, status) && LGS_CHECK(te < (uint64_t)m, 6, status)) {
                    tkey[start + pos] = (KT)tile;
                    tval[start + pos] = te;
                }
            }
            run += rtot;
        }
        if (run != total) {
            for (uint32_t q = run + lane; q < total; q += 32) {
                tkey[start + q] = (KT)0;
                tval[start + q] = 0u;
            }
            if (lane == 0) report_error(status, LGS_ERR_INTERNAL, (int64_t)total - (int64_t)run);
        }
    }
}

// ------------------------------------------------------------------ radix passes (onesweep)
// A stable LSD pass moves (u32 key, u32 value) pairs by one 8-bit digit in a
// single kernel. Each block takes the next tile index in launch order
// (atomic counter), counts its 6144 keys' digits in shared memory and
// publishes those counts at once, obtains the count of every digit in all
// earlier tiles by looking back over their published words (decoupled
// look-back, Merrill & Garland): a word carries either the tile's own count
// (AGG) or its inclusive prefix (PRE); the walk stops at the first PRE. Only
// then does it rank its keys stably and scatter them. A block only waits on
// tiles that were handed out before its own and therefore are already
// running; every wait is bounded: after spin_limit polls (OS_SPIN_LIMIT, about
// a second of L2 round trips) the block records LGS_ERR_TIMEOUT and continues. The digit bases of all passes come from one
// histogram kernel over the input keys (digits of later passes are counted on
// the same keys, since a pass only permutes them).
//
// The first pass over the entries reads no key array: it forms each entry's
// key (the bits of its depth, which order like the positive floats they are)
// and value (the entry index) from tiles-touched and depth, and drops culled
// entries (no tile) altogether, so later passes and stages see only the
// visible entries; their number goes to a device word.
constexpr int OS_THREADS = 256;
constexpr int OS_ITEMS = 24;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;   // 6144
constexpr uint64_t OS_AGG = 1ull << 62;
constexpr uint64_t OS_PRE = 2ull << 62;
constexpr uint64_t OS_VAL = (1ull << 62) - 1;
constexpr int OS_SPIN_LIMIT = 1 << 20;
constexpr int OS_MAX_DIGITS = 4;

// Where a pass reads its pairs: key/value arrays, or (k == nullptr) the
// entries' tiles-touched and depth.
struct OsSrc {
    const uint32_t* k;
    const uint32_t* v;
    const uint32_t* tiles;
    const float* depth;
};

__device__ __forceinline__ bool os_load(const OsSrc& src, int64_t i, uint32_t& k, uint32_t& v) {
    if (src.k) {
        k = src.k[i];
        v = src.v[i];
        return true;
    }
    v = (uint32_t)i;
    const uint32_t tiles = src.tiles[i];      // both loads issued together
    const uint32_t bits = __float_as_uint(src.depth[i]);
    k = tiles ? bits : 0xffffffffu;
    return tiles != 0u;
}

// Per-digit-position histograms of the (kept) keys: ghist[p*256 + d] += count
// of kept elements whose digit p (bits 8p..8p+7) is d, for p < npass; with a
// synthesized source also the number of kept elements into *kept. One private
// histogram per warp; when all kept keys of a warp share a digit (the high
// depth bytes often do), one atomic adds them all.
__global__ void __launch_bounds__(256) onesweep_histogram(OsSrc src, const int64_t* cnt, int64_t count,
                                                          int npass, uint32_t* ghist, int64_t* kept) {
    __shared__ uint32_t h[8][OS_MAX_DIGITS][RADIX];
    __shared__ uint32_t s_kept;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * OS_MAX_DIGITS * RADIX; i += blockDim.x) (&h[0][0][0])[i] = 0;
    if (threadIdx.x == 0) s_kept = 0;
    __syncthreads();
    const int64_t K = pass_count(cnt, count);
    uint32_t my_kept = 0;
    for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 32; base < K; base += (int64_t)gridDim.x * 256) {
        const int64_t i = base + lane;
        uint32_t k = 0, v;
        const bool ok = i < K && os_load(src, i, k, v);
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (bal == 0u) continue;
        my_kept += ok;
        const int leader = __ffs(bal) - 1;
        for (int p = 0; p < npass; ++p) {
            const uint32_t d = (k >> (8 * p)) & 0xffu;
            const uint32_t first = __shfl_sync(0xffffffffu, d, leader);
            if (__all_sync(0xffffffffu, !ok || d == first)) {
                if (lane == leader) atomicAdd(&h[warp][p][first], (uint32_t)__popc(bal));
            } else if (ok) {
                atomicAdd(&h[warp][p][d], 1u);
            }
        }
    }
    if (kept && my_kept) atomicAdd(&s_kept, my_kept);
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RADIX; i += blockDim.x) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += (&h[w][0][0])[i];
        if (sum) atomicAdd(&ghist[i], sum);
    }
    if (kept && threadIdx.x == 0 && s_kept)
        atomicAdd(reinterpret_cast<unsigned long long*>(kept), (unsigned long long)s_kept);
}

// Digit histograms of a key array (the tile ids of the instances): 16-B loads,
// one private histogram per warp, and a warp-uniform fast path -- when all 128
// digits a warp loads at once are equal (instances of neighbouring Gaussians
// mostly share the high tile-id byte) one atomic adds them all.
template <typename KT>
__global__ void __launch_bounds__(256) key_histogram(const KT* keys, const int64_t* cnt,
                                                     int64_t count, int npass, uint32_t* ghist) {
    constexpr int PER = 16 / sizeof(KT);        // keys per 16-B load
    __shared__ uint32_t h[8][OS_MAX_DIGITS][RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * OS_MAX_DIGITS * RADIX; i += blockDim.x) (&h[0][0][0])[i] = 0;
    __syncthreads();
    const int64_t K = pass_count(cnt, count);
    const int64_t n4 = K / PER;
    const uint4* k4 = reinterpret_cast<const uint4*>(keys);
    for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 32; base < n4; base += (int64_t)gridDim.x * 256) {
        const int64_t q = base + lane;
        const bool ok = q < n4;
        const uint4 v4 = ok ? k4[q] : make_uint4(0u, 0u, 0u, 0u);
        uint32_t kv[PER];
        if constexpr (PER == 4) {
            kv[0] = v4.x; kv[1] = v4.y; kv[2] = v4.z; kv[3] = v4.w;
        } else {
            const uint32_t w4[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                kv[2 * r] = w4[r] & 0xffffu;
                kv[2 * r + 1] = w4[r] >> 16;
            }
        }
        const int nok = __popc(__ballot_sync(0xffffffffu, ok));
        for (int p = 0; p < npass; ++p) {
            const int sh = 8 * p;
            const uint32_t first = __shfl_sync(0xffffffffu, (kv[0] >> sh) & 0xffu, 0);
            bool uni = true;
#pragma unroll
            for (int r = 0; r < PER; ++r) uni = uni && ((kv[r] >> sh) & 0xffu) == first;
            if (__all_sync(0xffffffffu, !ok || uni)) {
                if (lane == 0) atomicAdd(&h[warp][p][first], (uint32_t)PER * (uint32_t)nok);
            } else if (ok) {
#pragma unroll
                for (int r = 0; r < PER; ++r) atomicAdd(&h[warp][p][(kv[r] >> sh) & 0xffu], 1u);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < (int)(K - PER * n4)) {       // the K mod PER tail
        const uint32_t k = keys[PER * n4 + threadIdx.x];
        for (int p = 0; p < npass; ++p) atomicAdd(&h[0][p][(k >> (8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RADIX; i += blockDim.x) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += (&h[w][0][0])[i];
        if (sum) atomicAdd(&ghist[i], sum);
    }
}

// In place: each digit position's 256 counts -> exclusive prefix (one block per position).
__global__ void __launch_bounds__(RADIX) onesweep_bases(uint32_t* ghist) {
    __shared__ uint32_t ws[32];
    uint32_t* row = ghist + blockIdx.x * RADIX;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<RADIX>(row[threadIdx.x], ws, tot);
    row[threadIdx.x] = ex;
}

struct OneSmem {
    uint32_t cnt[OS_THREADS / 32][RADIX];   // per-warp digit counters -> (digit, warp) offsets
    uint32_t ws[32];
    uint32_t start[RADIX];   // digit counts of the tile, then block-local start of each digit
    uint32_t base[RADIX];    // global output position of each digit's first element in this tile
    uint32_t tile;
    uint32_t keys[OS_TILE];
    uint32_t vals[OS_TILE];
};

// Keys are ranked warp by warp: warp w owns tile elements [w*768, (w+1)*768),
// taken 32 at a time in order; per-bit ballots group equal digits and the
// warp's private counters give each key its rank among equal digits of the
// warp's range, with no block barrier. A digit-major exclusive scan over
// (digit, warp) then gives each (digit, warp) pair its place in the tile.
__global__ void __launch_bounds__(OS_THREADS, 2) onesweep_pass(
    OsSrc src, uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const int64_t* cnt,
    int64_t count, int shift, const uint32_t* bases, unsigned long long* look, uint32_t* tile_counter,
    int64_t* err_status, int spin_limit) {
    constexpr int NW = OS_THREADS / 32;
    constexpr int PER_WARP = OS_TILE / NW;      // 768
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OneSmem& S = *reinterpret_cast<OneSmem*>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt = lanemask_lt();
    if (t == 0) S.tile = atomicAdd(tile_counter, 1u);
    for (int d = lane; d < RADIX; d += 32) S.cnt[warp][d] = 0;
    S.start[t] = 0;
    __syncthreads();
    const uint32_t tile = S.tile;
    const int64_t K = pass_count(cnt, count);
    const int64_t first = (int64_t)tile * OS_TILE;
    if (first >= K) return;
    const int n_valid = (int)min((int64_t)OS_TILE, K - first);
    uint32_t k[OS_ITEMS], v[OS_ITEMS];
    uint32_t keep = 0;      // bit i: item i is a kept element
    const int wbase = warp * PER_WARP;
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        const int j = wbase + i * 32 + lane;
        k[i] = 0xffffffffu;
        v[i] = 0u;
        if (j < n_valid && os_load(src, first + j, k[i], v[i])) keep |= 1u << i;
    }
    // early digit counts of the tile, published before ranking
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i)
        if (keep & (1u << i)) atomicAdd(&S.start[(k[i] >> shift) & 0xffu], 1u);
    __syncthreads();
    const uint32_t total = S.start[t];
    unsigned long long* my = look + (int64_t)tile * RADIX + t;
    atomicExch(my, (unsigned long long)((tile == 0 ? OS_PRE : OS_AGG) | total));
    uint64_t prefix = 0;
    if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        int spins = 0;
        while (j >= 0) {
            const uint64_t w = *reinterpret_cast<volatile unsigned long long*>(look + j * RADIX + t);
            const uint64_t f = w & ~OS_VAL;
            if (f == 0) {
                if (++spins > spin_limit) {
                    report_error(err_status, LGS_ERR_TIMEOUT, (int64_t)tile);
                    break;
                }
                continue;
            }
            prefix += w & OS_VAL;
            if (f == OS_PRE) break;
            --j;
        }
        atomicExch(my, (unsigned long long)(OS_PRE | (prefix + total)));
    }
    // stable rank of every kept key among equal digits of its warp's range; the
    // lanes holding the same digit (9 bits: 0x100 marks no key) are found with
    // one ballot per bit
    uint16_t rk[OS_ITEMS];
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        const uint32_t d = (keep & (1u << i)) ? ((k[i] >> shift) & 0xffu) : 0x100u;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        // every lane of a group reads the group's counter; the group's last
        // lane advances it
        const uint32_t b = d < 0x100u ? S.cnt[warp][d] : 0u;
        rk[i] = (uint16_t)(b + __popc(peers & lt));
        __syncwarp();
        if (d < 0x100u && (peers >> lane) == 1u) S.cnt[warp][d] = b + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t pre[NW], acc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        pre[w] = acc;
        acc += S.cnt[w][t];
    }
    uint32_t n_kept;
    const uint32_t st = block_exclusive_scan<OS_THREADS>(total, S.ws, n_kept);
    S.start[t] = st;
    S.base[t] = bases[t] + (uint32_t)prefix;
#pragma unroll
    for (int w = 0; w < NW; ++w) S.cnt[w][t] = st + pre[w];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < OS_ITEMS; ++i) {
        if (keep & (1u << i)) {
            const uint32_t pos = S.cnt[warp][(k[i] >> shift) & 0xffu] + rk[i];
            S.keys[pos] = k[i];
            S.vals[pos] = v[i];
        }
    }
    __syncthreads();
    for (int j = t; j < (int)n_kept; j += OS_THREADS) {
        const uint32_t key = S.keys[j];
        const uint32_t d = (key >> shift) & 0xffu;
        const uint32_t gpos = S.base[d] + (uint32_t)j - S.start[d];
        if (LGS_CHECK((int64_t)gpos < K, 7, err_status)) {
            kout[gpos] = key;
            vout[gpos] = S.vals[j];
        }
    }
}

// ------------------------------------------------------------------ radix passes (reduce-then-scan)
// The same stable LSD pass as onesweep_pass, split so that no block ever waits
// on another: rs_upsweep counts each 4096-element block's digits into a
// digit-major table counts[d * nb + b]; rs_scan turns every row d into an
// exclusive scan along the blocks and stores the row's total (the pass's count
// of digit d); and rs_downsweep adds each digit's base (the exclusive scan of
// the 256 totals), ranks its block's keys stably (the warp-ballot ranking of
// onesweep_pass) and scatters them to those positions, so no histogram kernel
// runs before the passes. The keys are read twice
// (4 B per element more traffic than onesweep), but every kernel runs fully
// parallel instead of along a look-back chain. Keys are u32 or, for tile ids
// of at most 2^16 tiles, u16.
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // 4096

template <typename KT>
struct RsSrc {
    const KT* k;             // keys (nullptr: synthesized from tiles and depth, u32 only)
    const uint32_t* v;
    const uint32_t* tiles;
    const float* depth;
};

template <typename KT>
__device__ __forceinline__ bool rs_load(const RsSrc<KT>& src, int64_t i, uint32_t& k, uint32_t& v) {
    if (src.k) {
        k = (uint32_t)src.k[i];
        v = src.v ? src.v[i] : 0u;
        return true;
    }
    v = (uint32_t)i;
    const uint32_t tiles = src.tiles[i];
    const uint32_t bits = __float_as_uint(src.depth[i]);
    k = tiles ? bits : 0xffffffffu;
    return tiles != 0u;
}

// Per-block digit counts. Each warp counts its 512 elements into a private
// histogram (one atomic for a whole warp when its 32 kept digits agree).
template <typename KT>
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(RsSrc<KT> src, const int64_t* cnt, int64_t count,
                                                         int shift, uint32_t* counts, int64_t nb) {
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t h[NW][RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < RADIX; d += 32) h[warp][d] = 0;
    const int64_t K = pass_count(cnt, count);
    const int64_t first = (int64_t)blockIdx.x * RS_TILE;
    if (first >= K) return;
    __syncwarp();
    const int64_t wfirst = first + warp * (RS_TILE / NW);
    // all of the thread's keys first (independent loads in flight together),
    // then the counting
    uint32_t kk[RS_ITEMS];
    uint32_t okm = 0;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t j = wfirst + i * 32 + lane;
        uint32_t v;
        kk[i] = 0;
        if (j < K && rs_load(RsSrc<KT>{src.k, nullptr, src.tiles, src.depth}, j, kk[i], v)) okm |= 1u << i;
    }
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const uint32_t k = kk[i];
        const bool ok = (okm >> i) & 1u;
        const uint32_t d = (k >> shift) & 0xffu;
        const uint32_t bal = __ballot_sync(0xffffffffu, ok);
        if (bal == 0u) continue;
        const int leader = __ffs(bal) - 1;
        const uint32_t d0 = __shfl_sync(0xffffffffu, d, leader);
        if (__all_sync(0xffffffffu, !ok || d == d0)) {
            if (lane == leader) h[warp][d0] += (uint32_t)__popc(bal);
        } else if (ok) {
            atomicAdd(&h[warp][d], 1u);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += h[w][d];
        counts[(int64_t)d * nb + blockIdx.x] = t;
    }
}

// Row d of the count table -> exclusive prefix along the live blocks, and the
// row's total (the pass's count of digit d) into totals[d] (one CTA per digit).
// rs_downsweep adds the digit's base, the exclusive prefix of the totals.
__global__ void __launch_bounds__(1024) rs_scan(uint32_t* counts, int64_t nb, const int64_t* cnt, int64_t count,
                                               uint32_t* totals) {
    __shared__ uint32_t ws[32];
    const int64_t K = pass_count(cnt, count);
    const int64_t live = ceil_div_dev(K, RS_TILE);
    uint32_t* row = counts + (int64_t)blockIdx.x * nb;
    uint32_t carry = 0u;
    for (int64_t b0 = 0; b0 < live; b0 += 1024) {
        const int64_t b = b0 + threadIdx.x;
        const uint32_t v = b < live ? row[b] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<1024>(v, ws, tot);
        if (b < live) row[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <typename KT>
struct RsSmem {
    uint32_t cnt[RS_THREADS / 32][RADIX];   // per-warp digit counters -> (digit, warp) offsets
    uint32_t ws[32];
    uint32_t start[RADIX];   // block-local start of each digit
    uint32_t base[RADIX];    // global output position of each digit's first element in this block
    uint32_t tcnt[RS_THREADS];   // per-warp tight counters of the fused count
    KT keys[RS_TILE];
    uint32_t vals[RS_TILE];
};

// What the last entry pass also does with LGS_FLAG_TIGHT (the tight count
// folded into the pass): its sorted entries are the depth order, so it writes
// their tight instance counts and depth-ordered emission records as it
// scatters them, instead of a separate kernel reading the order back.
struct RsTightCount {
    const uint64_t* rect;
    const float4* xy;
    const float4* conic;
    const uint4* emit;
    Views vs;
    int64_t n;
    uint32_t* tiles_sorted;
    uint4* rec;
};

// TW > 0: the scatter also runs the fused tight count (keys are not written).
// Stable rank of each of a warp's RS_ITEMS x 32 digits (item i of lane l is
// element i * 32 + l of the warp's range) among equal digits, with the warp's
// counters cnt advanced: one ballot per significant digit bit (NBITS: the
// digits of the pass are known to be < 2^NBITS), plus one for the kept bit
// when some element of the warp is dropped (d = 0x100).
template <int NBITS, bool WITH_DROP>
__device__ __forceinline__ void warp_rank(const uint32_t (&d)[RS_ITEMS], uint32_t* cnt, uint16_t (&rk)[RS_ITEMS]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < NBITS; ++b) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d[i] >> b) & 1u);
            peers &= ((d[i] >> b) & 1u) ? bal : ~bal;
        }
        if (WITH_DROP) {
            const uint32_t bal = __ballot_sync(0xffffffffu, d[i] >> 8);
            peers &= (d[i] >> 8) ? bal : ~bal;
        }
        const uint32_t b = d[i] < 0x100u ? cnt[d[i]] : 0u;
        rk[i] = (uint16_t)(b + __popc(peers & lt));
        __syncwarp();
        if (d[i] < 0x100u && (peers >> lane) == 1u) cnt[d[i]] = b + __popc(peers);
        __syncwarp();
    }
}

// `totals`: the pass's digit counts from rs_scan; with `kept`, block 0 also
// stores their sum, the number of elements the pass kept.
template <typename KT, int TW = 0, int TH = 0, int NBITS = 8>
__global__ void __launch_bounds__(RS_THREADS, 3) rs_downsweep(RsSrc<KT> src, KT* __restrict__ kout,
                                                              uint32_t* __restrict__ vout, const int64_t* cnt,
                                                              int64_t count, int shift, const uint32_t* offsets,
                                                              const uint32_t* totals, int64_t nb,
                                                              int64_t* err_status, int64_t* kept = nullptr,
                                                              RsTightCount tc = RsTightCount{}) {
    static_assert(RS_THREADS == RADIX, "one thread per digit");
    constexpr int NW = RS_THREADS / 32;
    constexpr int PER_WARP = RS_TILE / NW;      // 512
    __shared__ RsSmem<KT> S;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t K = pass_count(cnt, count);
    const int64_t first = (int64_t)blockIdx.x * RS_TILE;
    if (first >= K) return;
    for (int d = lane; d < RADIX; d += 32) S.cnt[warp][d] = 0;
    {
        // global position of this block's first element of digit t: the
        // digit's base (exclusive prefix of the totals) + the row prefix
        uint32_t all;
        const uint32_t dbase = block_exclusive_scan<RS_THREADS>(totals[t], S.ws, all);
        S.base[t] = dbase + offsets[(int64_t)t * nb + blockIdx.x];
        if (kept && blockIdx.x == 0 && t == 0) *kept = (int64_t)all;
    }
    const int n_valid = (int)min((int64_t)RS_TILE, K - first);
    // keys first; the values are loaded only once their slots are known, so
    // they hold no registers through the ranking
    uint32_t k[RS_ITEMS];
    uint32_t keep = 0;      // bit i: item i is a kept element
    const int wbase = warp * PER_WARP;
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int j = wbase + i * 32 + lane;
        k[i] = 0xffffffffu;
        uint32_t unused;
        if (j < n_valid && rs_load(RsSrc<KT>{src.k, nullptr, src.tiles, src.depth}, first + j, k[i], unused))
            keep |= 1u << i;
    }
    __syncwarp();
    // stable rank of every kept key among equal digits of its warp's range
    // (one ballot per digit bit; bit 8 marks a dropped element)
    uint16_t rk[RS_ITEMS];
    uint32_t dg[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) dg[i] = (keep & (1u << i)) ? ((k[i] >> shift) & 0xffu) : 0x100u;
    if (__all_sync(0xffffffffu, keep == (1u << RS_ITEMS) - 1u))
        warp_rank<NBITS, false>(dg, S.cnt[warp], rk);
    else
        warp_rank<NBITS, true>(dg, S.cnt[warp], rk);
    __syncthreads();
    uint32_t pre[NW], acc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        pre[w] = acc;
        acc += S.cnt[w][t];
    }
    uint32_t n_kept;
    const uint32_t st = block_exclusive_scan<RS_THREADS>(acc, S.ws, n_kept);
    S.start[t] = st;
#pragma unroll
    for (int w = 0; w < NW; ++w) S.cnt[w][t] = st + pre[w];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        if (keep & (1u << i)) {
            const uint32_t pos = S.cnt[warp][(k[i] >> shift) & 0xffu] + rk[i];
            const int64_t j = first + wbase + i * 32 + lane;
            S.keys[pos] = (KT)k[i];
            S.vals[pos] = src.k ? src.v[j] : (uint32_t)j;
        }
    }
    __syncthreads();
    if constexpr (TW == 0) {
#pragma unroll 4
        for (int j = t; j < (int)n_kept; j += RS_THREADS) {
            const uint32_t key = S.keys[j];
            const uint32_t d = (key >> shift) & 0xffu;
            const uint32_t gpos = S.base[d] + (uint32_t)j - S.start[d];
            if (LGS_CHECK((int64_t)gpos < K, 9, err_status)) {
                kout[gpos] = (KT)key;
                vout[gpos] = S.vals[j];
            }
        }
    } else {
        // every lane of a warp takes part in each round (the count is warp-cooperative)
        for (int j0 = 0; j0 < (int)n_kept; j0 += RS_THREADS) {
            const int j = j0 + t;
            bool live = j < (int)n_kept;
            uint32_t ent = 0u, gpos = 0u;
            if (live) {
                const uint32_t d = (S.keys[j] >> shift) & 0xffu;
                gpos = S.base[d] + (uint32_t)j - S.start[d];
                ent = S.vals[j];
                live = LGS_CHECK((int64_t)gpos < K, 9, err_status);
                if (live) vout[gpos] = ent;
            }
            TightLane L;
            if (tc.emit) {
                uint4 a = make_uint4(0u, 0u, 0u, 0u), c = a;
                if (live) {
                    a = tc.emit[2 * (int64_t)ent];
                    c = tc.emit[2 * (int64_t)ent + 1];
                    tc.rec[2 * (int64_t)gpos] = a;
                    tc.rec[2 * (int64_t)gpos + 1] = c;
                }
                L = tight_lane_from(ent, live, a, c, tc.vs, tc.n);
            } else {
                L = tight_lane_load(ent, live, tc.rect, tc.xy, tc.conic, tc.vs, tc.n, tc.rec, gpos);
            }
            const uint32_t c = warp_tight_count<TW, TH>(L, S.tcnt + (t & ~31));
            if (live) tc.tiles_sorted[gpos] = c;
        }
    }
}

// ------------------------------------------------------------------ ranges
// Per-tile [start, end) of the sorted tile ids; each thread takes 4
// consecutive instances (one 16-B load when all 4 lie below K).
template <typename KT>
__global__ void __launch_bounds__(256) tile_ranges(const KT* tkey, int64_t* status,
                                                   int64_t capacity, uint32_t n_tiles, uint2* ranges) {
    constexpr int PER = 16 / sizeof(KT);        // ids per 16-B load
    const int64_t K = sort_count(status, capacity);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; PER * q < K;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = PER * q;
        uint32_t t[PER];
        if (i0 + PER - 1 < K) {
            const uint4 v = reinterpret_cast<const uint4*>(tkey)[q];
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int r = 0; r < PER; ++r) {
                if constexpr (PER == 4) t[r] = w4[r];
                else t[r] = (w4[r / 2] >> (16 * (r & 1))) & 0xffffu;
            }
        } else {
#pragma unroll
            for (int r = 0; r < PER; ++r) t[r] = i0 + r < K ? (uint32_t)tkey[i0 + r] : 0u;
        }
        uint32_t prev = i0 > 0 ? (uint32_t)tkey[i0 - 1] : 0xffffffffu;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int64_t i = i0 + r;
            if (i >= K) break;
            if (!LGS_CHECK(t[r] < n_tiles, 8, status)) break;
            if (i == 0 || prev != t[r]) ranges[t[r]].x = (uint32_t)i;
            const uint32_t next = r < PER - 1 ? (i + 1 < K ? t[r + 1] : 0xffffffffu)
                                              : (i + 1 < K ? (uint32_t)tkey[i + 1] : 0xffffffffu);
            if (i == K - 1 || next != t[r]) ranges[t[r]].y = (uint32_t)(i + 1);
            prev = t[r];
        }
    }
}

// tiles-touched of the visible entries in depth order (0 past the mv visible ones)
__global__ void gather_tiles(const uint32_t* order, const uint32_t* tiles, int64_t m,
                             const int64_t* mv, uint32_t* tiles_sorted) {
    const int64_t nv = pass_count(mv, m);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x)
        tiles_sorted[j] = j < nv ? tiles[order[j]] : 0u;
}

// Optional 64-bit keys of the sorted instances: (tile << 32) | bits(depth).
template <typename KT>
__global__ void write_keys(const KT* tkey, const uint32_t* vals, const float* depth,
                           const int64_t* status, int64_t capacity, uint64_t* keys) {
    const int64_t K = sort_count(status, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = ((uint64_t)tkey[i] << 32) | __float_as_uint(depth[vals[i]]);
}

// ------------------------------------------------------------------ workspace
struct SortWs {
    uint32_t* ek;          // [m] entry depth keys (ping)
    uint32_t* ev;          // [m] entry indices
    uint32_t* ek2;         // [m] (pong)
    uint32_t* ev2;         // [m]
    uint32_t* tiles_s;     // [m] tiles-touched in depth order
    uint32_t* offsets;     // [m] exclusive scan of tiles_s
    uint64_t* block_sums;  // [ceil(m/2048)]
    uint32_t* ak;          // [capacity] tile ids
    uint32_t* bk;          // [capacity]
    uint32_t* bv;          // [capacity] values (the caller's vals buffer is the other one)
    unsigned long long* look;  // [256 * max tiles of a pass] look-back words
    uint32_t* counters;    // tile counter of the running pass (u32 at byte 0 of a 256-B block)
    int64_t* mvis;         // visible entries (int64 at byte 64 of the same block)
    uint32_t* bases;       // [2 * OS_MAX_DIGITS * 256]: digit bases (entry sort, tile sort)
    uint4* erec;           // [2 * m] tight-box emission records in depth order (see count_tight)
};

constexpr size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Byte offsets of the workspace buffers for m entries and an instance
// capacity. One constexpr function is the only description of the layout: the
// workspace query, the carving of a caller's buffer and the compile-time check
// of the static scratch array all read it.
struct SortWsOffsets {
    size_t ek, ev, ek2, ev2, tiles_s, offsets, erec, block_sums, ak, bk, bv, look, counters, bases;
    size_t total;
};

constexpr SortWsOffsets sort_ws_offsets(int64_t m, int64_t capacity) {
    const size_t mm = (size_t)(m > 0 ? m : 1);
    const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
    const int64_t nscan = ceil_div(m, SCAN_TILE);
    const int64_t nt = ceil_div(m > capacity ? m : capacity, OS_TILE);
    SortWsOffsets o{};
    size_t off = 0;
    o.ek = off;         off += align_up(sizeof(uint32_t) * mm);
    o.ev = off;         off += align_up(sizeof(uint32_t) * mm);
    o.ek2 = off;        off += align_up(sizeof(uint32_t) * mm);
    o.ev2 = off;        off += align_up(sizeof(uint32_t) * mm);
    o.tiles_s = off;    off += align_up(sizeof(uint32_t) * mm);
    o.offsets = off;    off += align_up(sizeof(uint32_t) * mm);
    o.erec = off;       off += align_up(2 * sizeof(uint4) * mm);
    o.block_sums = off; off += align_up(sizeof(uint64_t) * (size_t)(nscan > 0 ? nscan : 1));
    o.ak = off;         off += align_up(sizeof(uint32_t) * cap);
    o.bk = off;         off += align_up(sizeof(uint32_t) * cap);
    o.bv = off;         off += align_up(sizeof(uint32_t) * cap);
    // look-back words of a onesweep pass, or the count table of a reduce-then-scan pass
    const int64_t nr = ceil_div(m > capacity ? m : capacity, RS_TILE);
    const size_t look_b = sizeof(uint64_t) * RADIX * (size_t)(nt > 0 ? nt : 1);
    const size_t cnt_b = sizeof(uint32_t) * RADIX * (size_t)(nr > 0 ? nr : 1);
    o.look = off;       off += align_up(look_b > cnt_b ? look_b : cnt_b);
    o.counters = off;   off += align_up(8 * sizeof(uint32_t));
    o.bases = off;      off += align_up(2 * OS_MAX_DIGITS * RADIX * sizeof(uint32_t));
    o.total = off;
    return o;
}

// Carves the workspace at `base` (256-B aligned) into *ws; returns its size.
inline size_t sort_ws_layout(int64_t m, int64_t capacity, char* base, SortWs* ws) {
    const SortWsOffsets o = sort_ws_offsets(m, capacity);
    if (ws && base) {
        ws->ek = reinterpret_cast<uint32_t*>(base + o.ek);
        ws->ev = reinterpret_cast<uint32_t*>(base + o.ev);
        ws->ek2 = reinterpret_cast<uint32_t*>(base + o.ek2);
        ws->ev2 = reinterpret_cast<uint32_t*>(base + o.ev2);
        ws->tiles_s = reinterpret_cast<uint32_t*>(base + o.tiles_s);
        ws->offsets = reinterpret_cast<uint32_t*>(base + o.offsets);
        ws->erec = reinterpret_cast<uint4*>(base + o.erec);
        ws->block_sums = reinterpret_cast<uint64_t*>(base + o.block_sums);
        ws->ak = reinterpret_cast<uint32_t*>(base + o.ak);
        ws->bk = reinterpret_cast<uint32_t*>(base + o.bk);
        ws->bv = reinterpret_cast<uint32_t*>(base + o.bv);
        ws->look = reinterpret_cast<unsigned long long*>(base + o.look);
        ws->counters = reinterpret_cast<uint32_t*>(base + o.counters);
        ws->mvis = reinterpret_cast<int64_t*>(base + o.counters + 64);
        ws->bases = reinterpret_cast<uint32_t*>(base + o.bases);
    }
    return o.total;
}

inline int tile_passes(uint32_t n_tiles) {
    int bits = 0;
    while (bits < 32 && (1ull << bits) < (uint64_t)n_tiles) ++bits;
    return bits == 0 ? 0 : (bits + 7) / 8;
}

// Digit bases of `npass` LSD passes over the pairs of `src` (count from the
// device word `cnt` when given): histogram + exclusive scan into
// bases[npass * 256]; with `kept`, also the number of kept elements.
static void onesweep_prepare(const OsSrc& src, const int64_t* cnt, int64_t count, int npass,
                             uint32_t* bases, int64_t* kept, cudaStream_t s) {
    cudaMemsetAsync(bases, 0, sizeof(uint32_t) * RADIX * npass, s);
    if (kept) cudaMemsetAsync(kept, 0, sizeof(int64_t), s);
    onesweep_histogram<<<152 * 4, 256, 0, s>>>(src, cnt, count, npass, bases, kept);
    onesweep_bases<<<npass, RADIX, 0, s>>>(bases);
}

// One stable LSD pass over u32 keys carrying u32 values (element count from
// the device word `cnt` when given, else `count`; the grid covers `count`).
// With `onesweep` one look-back kernel (onesweep_pass; `bases` holds the
// pass's digit bases from onesweep_prepare), else the three reduce-then-scan
// kernels (rs_upsweep, rs_scan, rs_downsweep; `bases` is their 256-word digit
// total scratch, their count table reuses the look-back words' space, which no
// concurrent pass uses, and `kept`, when given, receives the kept count).
static void radix_pass(const OsSrc& src, uint32_t* kout, uint32_t* vout, const int64_t* cnt,
                       int64_t count, int shift, uint32_t* bases, const SortWs* ws,
                       int64_t* d_status, cudaStream_t s, bool onesweep, int nbits = 8,
                       int64_t* kept = nullptr) {
    if (onesweep) {
        const int64_t nt = ceil_div(count, OS_TILE);
        if (nt == 0) return;
        cudaMemsetAsync(ws->look, 0, sizeof(unsigned long long) * RADIX * (size_t)nt, s);
        cudaMemsetAsync(ws->counters, 0, sizeof(uint32_t), s);
        onesweep_pass<<<(unsigned)nt, OS_THREADS, sizeof(OneSmem), s>>>(
            src, kout, vout, cnt, count, shift, bases, ws->look, ws->counters, d_status, OS_SPIN_LIMIT);
        return;
    }
    const int64_t nb = ceil_div(count, RS_TILE);
    if (nb == 0) return;
    uint32_t* counts = reinterpret_cast<uint32_t*>(ws->look);
    const RsSrc<uint32_t> rs{src.k, src.v, src.tiles, src.depth};
    rs_upsweep<uint32_t><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, cnt, count, shift, counts, nb);
    rs_scan<<<RADIX, 1024, 0, s>>>(counts, nb, cnt, count, bases);
    if (nbits <= 7)
        rs_downsweep<uint32_t, 0, 0, 7><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, kout, vout, cnt, count, shift,
                                                                          counts, bases, nb, d_status, kept);
    else
        rs_downsweep<uint32_t><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, kout, vout, cnt, count, shift, counts,
                                                                   bases, nb, d_status, kept);
}

}  // namespace lgs

using namespace lgs;

extern "C" size_t lgs_sort_workspace_size(int64_t m, int64_t capacity) {
    if (m < 0 || capacity < 0) return 0;
    return sort_ws_layout(m, capacity, nullptr, nullptr);
}

struct SortTileArgs {
    const uint32_t* order;
    const lgs_pre_out* pre;
    int64_t n, m;
    const Views* vs;
    int64_t capacity;
    uint64_t* keys;
    uint32_t* vals;
    uint32_t* ranges;
    const SortWs* ws;
    int64_t* d_status;
    bool tight, onesweep;
};

// Emission of the (tile id, entry) pairs in depth order, the stable LSD
// passes over the tile-id bits, the tile ranges and (if asked for) the 64-bit
// keys, with tile ids of type KT (u16 when every id fits).
template <typename KT>
static void tile_stage(const SortTileArgs& a, cudaStream_t s) {
    const Views* vs = a.vs;
    const SortWs* ws = a.ws;
    const int64_t m = a.m, capacity = a.capacity;
    const unsigned eg = (unsigned)ceil_div(m, 256);
    // the value buffers alternate so that the last pass lands in vals
    const int passes = tile_passes(vs->n_tiles);
    KT *ka = reinterpret_cast<KT*>(ws->ak), *kb = reinterpret_cast<KT*>(ws->bk);
    uint32_t *va = (passes & 1) ? ws->bv : a.vals, *vb = (passes & 1) ? a.vals : ws->bv;
    if (a.tight) {
#define LGS_EMIT_TIGHT(TW_, TH_)                                                                          \
    emit_pairs_tight<TW_, TH_, KT><<<eg, 256, 0, s>>>(a.order, ws->tiles_s, ws->offsets, ws->erec, m, ws->mvis, \
                                                      a.n, a.d_status, capacity, *vs, ka, va)
        const int tw = vs->tile_w, th = vs->tile_h;
        if (tw == 16 && th == 16) LGS_EMIT_TIGHT(16, 16);
        else if (tw == 8 && th == 32) LGS_EMIT_TIGHT(8, 32);
        else if (tw == 32 && th == 8) LGS_EMIT_TIGHT(32, 8);
        else if (tw == 32 && th == 32) LGS_EMIT_TIGHT(32, 32);
        else if (tw == 16 && th == 32) LGS_EMIT_TIGHT(16, 32);
        else LGS_EMIT_TIGHT(32, 16);
#undef LGS_EMIT_TIGHT
    } else {
        emit_pairs<KT><<<eg, 256, 0, s>>>(a.order, ws->tiles_s, ws->offsets, a.pre->rect, m, a.n, a.d_status,
                                          capacity, *vs, ka, va);
    }
    const int64_t* kcount = a.d_status + LGS_ST_NUM_INSTANCES;
    uint32_t* tbases = ws->bases + OS_MAX_DIGITS * RADIX;
    if (passes > 0 && a.onesweep) {
        // digit bases of the look-back passes; the reduce-then-scan passes
        // take their digit totals from their own count tables
        cudaMemsetAsync(tbases, 0, sizeof(uint32_t) * RADIX * passes, s);
        key_histogram<KT><<<152 * 4, 256, 0, s>>>(ka, kcount, capacity, passes, tbases);
        onesweep_bases<<<passes, RADIX, 0, s>>>(tbases);
    }
    int tile_bits = 0;
    while ((1u << tile_bits) < vs->n_tiles) ++tile_bits;
    for (int p = 0; p < passes; ++p) {
        // significant bits of this pass's digit (tile ids are < n_tiles)
        const int nbits = tile_bits - 8 * p < 8 ? tile_bits - 8 * p : 8;
        if constexpr (sizeof(KT) == 4) {
            radix_pass(OsSrc{ka, va, nullptr, nullptr}, kb, vb, kcount, capacity, 8 * p, tbases + p * RADIX, ws,
                       a.d_status, s, a.onesweep, nbits);
        } else {
            const int64_t nb = ceil_div(capacity, RS_TILE);
            uint32_t* counts = reinterpret_cast<uint32_t*>(ws->look);
            const RsSrc<KT> rs{ka, va, nullptr, nullptr};
            rs_upsweep<KT><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, kcount, capacity, 8 * p, counts, nb);
            uint32_t* tot = tbases + p * RADIX;
            rs_scan<<<RADIX, 1024, 0, s>>>(counts, nb, kcount, capacity, tot);
            if (nbits <= 7)
                rs_downsweep<KT, 0, 0, 7><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, kb, vb, kcount, capacity, 8 * p,
                                                                              counts, tot, nb, a.d_status);
            else
                rs_downsweep<KT><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, kb, vb, kcount, capacity, 8 * p, counts,
                                                                     tot, nb, a.d_status);
        }
        KT* t = ka; ka = kb; kb = t;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    // ka holds the sorted tile ids, va == vals
    uint2* r2 = reinterpret_cast<uint2*>(a.ranges);
    tile_ranges<KT><<<152 * 4, 256, 0, s>>>(ka, a.d_status, capacity, vs->n_tiles, r2);
    if (a.keys) write_keys<KT><<<152 * 8, 256, 0, s>>>(ka, a.vals, a.pre->depth, a.d_status, capacity, a.keys);
}

// Enqueues the full stage given a workspace layout (shared by the entry points):
//  1. stable LSD sort of the visible entries by depth (the first pass drops
//     the culled ones),
//  2. scan of tiles-touched in that order -> instance offsets and K,
//  3. emission of (tile id, entry) pairs in that order,
//  4. stable LSD passes over the tile-id bits,
//  5. tile ranges (and, if asked for, the 64-bit keys).
// Inside every tile the instances are then in (depth, entry index) order,
// i.e. exactly the stable sort of the (tile << 32 | depth) keys.
static lgs_status sort_enqueue(const lgs_pre_out* pre, int64_t n, const Views* vs,
                               int64_t capacity, uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                               const SortWs* ws, int64_t* d_status, cudaStream_t s) {
    const int64_t m = n * vs->n;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)vs->n_tiles, s);
    if (e != cudaSuccess) return LGS_ERR_CUDA;
    if (m == 0) {
        e = cudaMemsetAsync(d_status + LGS_ST_NUM_INSTANCES, 0, sizeof(int64_t), s);
        return cuda_status(e);
    }
    cudaFuncSetAttribute(onesweep_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(OneSmem));
    // 1. visible entries by depth: the first pass forms (depth bits, entry)
    //    from tiles-touched and depth and drops the culled entries
    const OsSrc entries{nullptr, nullptr, pre->tiles, pre->depth};
    const bool os = (vs->flags & LGS_FLAG_ONESWEEP) != 0;
    // the look-back passes need every pass's digit bases (and the kept count)
    // up front; the reduce-then-scan passes count their own digits, and the
    // first one stores the kept count
    if (os) onesweep_prepare(entries, nullptr, m, 4, ws->bases, ws->mvis, s);
    radix_pass(entries, ws->ek2, ws->ev2, nullptr, m, 0, ws->bases, ws, d_status, s, os, 8,
               os ? nullptr : ws->mvis);
    const bool tight = (vs->flags & LGS_FLAG_TIGHT) != 0;
    const float4* pxy = reinterpret_cast<const float4*>(pre->xy);
    const float4* pco = reinterpret_cast<const float4*>(pre->conic);
    const uint4* pem = reinterpret_cast<const uint4*>(pre->emit);
    const unsigned eg = (unsigned)ceil_div(m, 256);
    // with tight emission and reduce-then-scan passes, the last entry pass
    // also computes the tight counts (fused; no count kernel afterwards)
    // Fused only for entry sets whose depth-ordered record gathers miss L2
    // (32 B per entry against the 129 MB L2): there the fused count measured
    // faster (30M-Gaussian scene: sort 28.8 -> 27.7 ms with 32x32 tiles), while
    // on the 8-view outdoor step (4M entries) the separate count kernel wins
    // (75 against 100 us for the pass and the count).
    const bool fused = tight && !os && m > (int64_t(1) << 23);
    uint32_t *k0 = ws->ek2, *v0 = ws->ev2, *k1 = ws->ek, *v1 = ws->ev;
    for (int shift = 8; shift < 32; shift += 8) {
        if (shift == 24 && fused) {
            const int64_t nb = ceil_div(m, RS_TILE);
            uint32_t* counts = reinterpret_cast<uint32_t*>(ws->look);
            const RsSrc<uint32_t> rs{k0, v0, nullptr, nullptr};
            const RsTightCount tc{pre->rect, pxy, pco, pem, *vs, n, ws->tiles_s, ws->erec};
            rs_upsweep<uint32_t><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, ws->mvis, m, shift, counts, nb);
            uint32_t* tot = ws->bases + RADIX * 3;
            rs_scan<<<RADIX, 1024, 0, s>>>(counts, nb, ws->mvis, m, tot);
#define LGS_FUSED_PASS(TW_, TH_)                                                                          \
    rs_downsweep<uint32_t, TW_, TH_, 7><<<(unsigned)nb, RS_THREADS, 0, s>>>(rs, k1, v1, ws->mvis, m, shift, counts, \
                                                                            tot, nb, d_status, nullptr, tc)
            const int tw = vs->tile_w, th = vs->tile_h;
            if (tw == 16 && th == 16) LGS_FUSED_PASS(16, 16);
            else if (tw == 8 && th == 32) LGS_FUSED_PASS(8, 32);
            else if (tw == 32 && th == 8) LGS_FUSED_PASS(32, 8);
            else if (tw == 32 && th == 32) LGS_FUSED_PASS(32, 32);
            else if (tw == 16 && th == 32) LGS_FUSED_PASS(16, 32);
            else LGS_FUSED_PASS(32, 16);
#undef LGS_FUSED_PASS
        } else {
            // the kept depths are positive floats: bit 31 of their keys is 0
            radix_pass(OsSrc{k0, v0, nullptr, nullptr}, k1, v1, ws->mvis, m, shift,
                       ws->bases + RADIX * (shift / 8), ws, d_status, s, os, shift == 24 ? 7 : 8);
        }
        uint32_t* t = k0; k0 = k1; k1 = t;
        t = v0; v0 = v1; v1 = t;
    }
    const uint32_t* order = v0;
    // 2. scan of tiles-touched (with LGS_FLAG_TIGHT: of the tight counts) in depth order
#define LGS_COUNT_TIGHT(TW_, TH_)                                                                       \
    count_tight<TW_, TH_><<<eg, 256, 0, s>>>(order, pre->rect, pxy, pco, pem, m, ws->mvis, n, *vs, ws->tiles_s, \
                                             ws->erec)
    const int tw = vs->tile_w, th = vs->tile_h;
    if (!tight) gather_tiles<<<152 * 8, 256, 0, s>>>(order, pre->tiles, m, ws->mvis, ws->tiles_s);
    else if (fused) {}
    else if (tw == 16 && th == 16) LGS_COUNT_TIGHT(16, 16);
    else if (tw == 8 && th == 32) LGS_COUNT_TIGHT(8, 32);
    else if (tw == 32 && th == 8) LGS_COUNT_TIGHT(32, 8);
    else if (tw == 32 && th == 32) LGS_COUNT_TIGHT(32, 32);
    else if (tw == 16 && th == 32) LGS_COUNT_TIGHT(16, 32);
    else LGS_COUNT_TIGHT(32, 16);
#undef LGS_COUNT_TIGHT
    const int64_t nscan = ceil_div(m, SCAN_TILE);
    scan_reduce<<<(unsigned)nscan, SCAN_THREADS, 0, s>>>(ws->tiles_s, m, ws->mvis, ws->block_sums);
    scan_block_sums<<<1, 1024, 0, s>>>(ws->block_sums, nscan, d_status, capacity);
    scan_downsweep<<<(unsigned)nscan, SCAN_THREADS, 0, s>>>(ws->tiles_s, m, ws->mvis, ws->block_sums,
                                                            ws->offsets);
    // 3-5: emission, tile-id passes and ranges, with u16 tile ids when the
    //      batch has at most 2^16 tiles (reduce-then-scan passes only)
    const SortTileArgs ta{order, pre, n, m, vs, capacity, keys, vals, ranges, ws, d_status, tight, os};
    if (!os && vs->n_tiles <= 65536u) tile_stage<uint16_t>(ta, s);
    else tile_stage<uint32_t>(ta, s);
    return cuda_status(cudaGetLastError());
}

extern "C" lgs_status lgs_sort(const lgs_pre_out* pre, int64_t n, const lgs_camera* cams,
                               int32_t n_views, const lgs_config* cfg, int64_t capacity,
                               uint64_t* keys, uint32_t* vals, uint32_t* ranges, void* workspace,
                               size_t workspace_bytes, int64_t* d_status, void* stream) {
    if (!pre || !vals || !ranges || !d_status) return LGS_ERR_ARG;
    if (n < 0 || capacity < 0 || capacity >= (1ll << 32)) return LGS_ERR_ARG;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    if (!pre->tiles || !pre->rect || !pre->depth) return LGS_ERR_ARG;
    if ((cfg->flags & LGS_FLAG_TIGHT) && (!pre->xy || !pre->conic)) return LGS_ERR_ARG;
    if ((cfg->flags & LGS_FLAG_TIGHT) && (!aligned16(pre->xy) || !aligned16(pre->conic)))
        return LGS_ERR_ALIGN;
    if (reinterpret_cast<uintptr_t>(pre->emit) & 31u) return LGS_ERR_ALIGN;
    if ((reinterpret_cast<uintptr_t>(pre->rect) & 7u) || (reinterpret_cast<uintptr_t>(keys) & 7u) ||
        (reinterpret_cast<uintptr_t>(ranges) & 7u))
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
    sort_ws_offsets(LGS_SORT_STATIC_MAX_ENTRIES, LGS_SORT_STATIC_MAX_INSTANCES).total;
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
    if (!pre || !vals || !ranges || !d_status) return LGS_ERR_ARG;
    if (n < 0 || capacity < 0) return LGS_ERR_ARG;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    const int64_t m = n * (int64_t)n_views;
    if (m > LGS_SORT_STATIC_MAX_ENTRIES || capacity > LGS_SORT_STATIC_MAX_INSTANCES)
        return LGS_ERR_UNSUPPORTED;
    if (!pre->tiles || !pre->rect || !pre->depth) return LGS_ERR_ARG;
    if ((cfg->flags & LGS_FLAG_TIGHT) && (!pre->xy || !pre->conic)) return LGS_ERR_ARG;
    if ((cfg->flags & LGS_FLAG_TIGHT) && (!aligned16(pre->xy) || !aligned16(pre->conic)))
        return LGS_ERR_ALIGN;
    if (reinterpret_cast<uintptr_t>(pre->emit) & 31u) return LGS_ERR_ALIGN;
    if ((reinterpret_cast<uintptr_t>(pre->rect) & 7u) || (reinterpret_cast<uintptr_t>(keys) & 7u) ||
        (reinterpret_cast<uintptr_t>(ranges) & 7u))
        return LGS_ERR_ALIGN;
    // the layout at these sizes must fit the array (it does whenever the
    // limits above hold; the check guards against a later layout change)
    if (sort_ws_layout(m, capacity, nullptr, nullptr) > (size_t)LGS_SORT_STATIC_BYTES)
        return LGS_ERR_INTERNAL;
    void* scratch = nullptr;
    st = sort_static_scratch(&scratch);
    if (st != LGS_OK) return st;
    SortWs ws;
    sort_ws_layout(m, capacity, static_cast<char*>(scratch), &ws);
    return sort_enqueue(pre, n, &vs, capacity, keys, vals, ranges, &ws, d_status,
                        static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------ failure-detection self-test
// Runs one onesweep block that is handed tile index 1 of a two-tile pass whose
// tile 0 never runs: its look-back waits on a word that nothing writes, gives
// up after spin_limit polls, records LGS_ERR_TIMEOUT (detail = 1) and finishes
// its pass (its output is meaningless but stays inside the scratch buffer).
extern "C" lgs_status lgs_selftest_wait_timeout(int32_t spin_limit, void* workspace,
                                               size_t workspace_bytes, int64_t* d_status,
                                               void* stream) {
    if (!workspace || !d_status || spin_limit < 0) return LGS_ERR_ARG;
    if (workspace_bytes < (size_t)LGS_SELFTEST_WORKSPACE_BYTES) return LGS_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return LGS_ERR_ALIGN;
    char* w = static_cast<char*>(workspace);
    uint32_t* kin = reinterpret_cast<uint32_t*>(w);
    uint32_t* vin = kin + 2 * OS_TILE;
    uint32_t* kout = vin + 2 * OS_TILE;
    uint32_t* vout = kout + 2 * OS_TILE;
    unsigned long long* look = reinterpret_cast<unsigned long long*>(vout + 2 * OS_TILE);
    uint32_t* bases = reinterpret_cast<uint32_t*>(look + 2 * RADIX);
    uint32_t* counter = bases + RADIX;
    static_assert(8 * 2 * OS_TILE * 4 / 2 + 2 * RADIX * 8 + RADIX * 4 + 4 <= LGS_SELFTEST_WORKSPACE_BYTES,
                  "self-test workspace");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(workspace, 0, LGS_SELFTEST_WORKSPACE_BYTES, s) != cudaSuccess) return LGS_ERR_CUDA;
    if (cudaMemsetAsync(counter, 1, 1, s) != cudaSuccess) return LGS_ERR_CUDA;   // first tile handed out: 1
    cudaFuncSetAttribute(onesweep_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(OneSmem));
    onesweep_pass<<<1, OS_THREADS, sizeof(OneSmem), s>>>(OsSrc{kin, vin, nullptr, nullptr}, kout, vout,
                                                          nullptr, 2 * OS_TILE, 0, bases, look, counter,
                                                          d_status, spin_limit);
    return cuda_status(cudaGetLastError());
}
