// render.cu -- stage 3 of the 3DGS pipeline: per-tile front-to-back alpha
// blending (Local-GS Sec. II-A render kernel).
//
// render_localgs implements the three Local-GS stages (Sec. III):
//  (1) hoisting (Sec. III-B): a batch of the tile's Gaussians is staged into
//      shared memory (their xy, conic and rgb records copied with cp.async one
//      batch ahead of the blend); each staging thread maps (a, b, c, ln o) and the
//      tile-local offset Delta to the six coefficients V = [A..F] of
//      ln(alpha) = A x'^2 + B x'y' + C y'^2 + D x' + E y' + F (Eq. hoist
//      transform), scaled by log2(e) so that alpha = 2^(V . B_local) is one
//      ex2. The pixel basis B_local = [x'^2, x'y', y'^2, x', y', 1] lives in
//      registers. The tile-local origin is the tile centre rather than its
//      corner: x' and Delta are then half as large, which divides the
//      cancellation bound of Sec. III-B4 by four at no cost.
//  (2) warp-level culling (Sec. III-C): the staging thread also evaluates the
//      tight box of the Gaussian's ellipse a x~^2 + 2b x~y~ + c y~^2 = tau,
//      tau = 2 ln(255 o), restricted to the tile column (Cases A/B/C), and turns
//      its vertical span into an 8-bit mask of warp strips. Each warp then
//      compacts the batch into its own index list (one __ballot_sync per 32
//      candidates, written to shared memory) and walks that list with a plain
//      counter (unrolled by 4), so culled Gaussians cost no issue slot in the
//      blend loop.
//  (3) warp-coherent blending (Sec. III-D): the per-pair data path is a fixed
//      branch-free sequence (5 FMA dot product, ex2, clamp, predicated
//      threshold/stop, w = alpha T, 3 FMA colour, 1 FMA transmittance); the
//      warp leaves the list when __all_sync says every lane is done.
// The alpha >= 1/255 skip and the per-pixel stop before T(1-alpha) < 1e-4 are
// kept as predicates (not branches), so results follow the per-pixel
// definition exactly; the warp-uniform exit only saves work.
//
// render_plain is the comparison baseline: the same staging and tile lists, but
// each thread evaluates every staged Gaussian in global pixel coordinates with
// per-pixel branches and per-pixel early exit (Alg. 1 left column).
#include "common.cuh"
#include "host.h"

namespace lgs {

constexpr int BATCH = 256;
constexpr float LOG2E = 1.4426950408889634f;
constexpr float LOG2_ALPHA_MIN = -7.9943534368588580f;  // log2(1/255)

struct RenderParams {
    const float4* xy;
    const float4* conic;
    const float4* rgb;
    const uint32_t* vals;
    const uint2* ranges;
    float* out_rgb;
    float* out_T;
    uint32_t* out_n;
    int64_t* status;
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct TileCtx {
    int view, X0, Y0, px, py, lx, ly;
    bool inside;
    uint32_t start, count;
};

template <int TW, int TH>
__device__ __forceinline__ TileCtx tile_ctx(const Views& vs, const RenderParams& p, uint32_t tile) {
    TileCtx t;
    t.view = view_of_tile(vs, tile);
    const ViewRec& c = vs.v[t.view];
    const uint32_t lt = tile - c.tile_off;
    const int tx = (int)(lt % (uint32_t)c.gx), ty = (int)(lt / (uint32_t)c.gx);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    t.lx = lane % TW;
    t.ly = warp * (TH / 8) + lane / TW;
    t.X0 = tx * TW;
    t.Y0 = ty * TH;
    t.px = t.X0 + t.lx;
    t.py = t.Y0 + t.ly;
    t.inside = t.px < c.W && t.py < c.H;
    const uint2 r = p.ranges[tile];
    t.start = r.x;
    t.count = r.y - r.x;
    return t;
}

__device__ __forceinline__ void write_pixel(const Views& vs, const RenderParams& p, const TileCtx& t,
                                            float C0, float C1, float C2, float T, uint32_t last) {
    if (!t.inside) return;
    const ViewRec& c = vs.v[t.view];
    const int64_t plane = (int64_t)c.W * c.H;
    const int64_t pix = (int64_t)t.py * c.W + t.px;
    float* o = p.out_rgb + 3 * (int64_t)c.pix_off;
    o[pix] = fmaf(T, c.bg[0], C0);
    o[plane + pix] = fmaf(T, c.bg[1], C1);
    o[2 * plane + pix] = fmaf(T, c.bg[2], C2);
    p.out_T[c.pix_off + pix] = T;
    p.out_n[c.pix_off + pix] = last;
}

// ------------------------------------------------------------------ Local-GS
// The three 16-B records of a staged Gaussian sit at the same byte offset in
// sV, sDE and sC, so a warp's list holds that offset and the blend loop
// addresses all three without index arithmetic.
template <int NB>
struct LocalSmem {
    float4 raw[2][3][NB];  // double-buffered cp.async landing zone: xy, conic, rgb records
    float4 sV[NB];         // (A, B, C, F), log2 domain
    float4 sDE[NB];        // (D, E, -, -)
    float4 sC[NB];         // (-r, -g, -b, list position + 1 as bits): colour negated, see the blend
    uint8_t sM[NB];        // warp-block mask
    uint16_t sL[8][NB];    // per warp: byte offsets (16 x batch index) of its set mask bits, in order
};

template <typename T>
__device__ __forceinline__ const float4& at_offset(const T* base, int off) {
    return *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(base) + off);
}

// 16-byte asynchronous global -> shared copy (cp.async, cached in L2 only:
// neighbouring tiles read the same Gaussians from L2) and its group fences.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Variants of the Local-GS tile loop:
//  VAR_CONTRACT: the per-pixel definition (1/255 skip and stop as predicates),
//                hoisted in the tile-centred frame;
//  VAR_LITERAL:  Alg. 1 right column read literally (Sec. III-D): no per-pixel
//                1/255 test (the warp mask is the only culling), w = alpha T,
//                C += f w, T -= w, and the warp leaves its list once every
//                pixel it owns has T < 1e-4 (checked before each Gaussian);
//  VAR_GLOBAL:   the contract evaluated with the hoist in global pixel
//                coordinates (origin at pixel (0, 0)): the "w/o local coord"
//                configuration of Sec. III-B4 / Table V, kept for the FP32
//                precision study.
constexpr int VAR_CONTRACT = 0, VAR_LITERAL = 1, VAR_GLOBAL = 2;
constexpr float INF_F = __builtin_huge_valf();

// One CTA region of one tile: work item w = tile * (regions per tile) + region.
// The region (CW x CH pixels at X0, Y0) walks the whole list of its tile.
template <int TW, int TH, int WX, int WY, bool COUNT, int VAR, int NB>
__device__ __forceinline__ void localgs_tile(const RenderParams& p, const Views& vs, uint32_t work,
                                             LocalSmem<NB>& S) {
    using Reg = Regions<TW, TH>;
    constexpr int CW = Reg::CW, CH = Reg::CH;
    using Lay = Layout<CW, CH, WX, WY>;
    constexpr int PPL = Lay::PPL, NT = Lay::NT;
    static_assert(NB == 64 || NB == 128 || NB == 256, "staging batch of 64, 128 or 256 Gaussians");
    static_assert(NB % NT == 0 || NT % NB == 0, "whole staging slots per thread");
    using P = Px<PPL>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const uint32_t tile = work / (uint32_t)Reg::N, reg = work % (uint32_t)Reg::N;
    const int view = view_of_tile(vs, tile);
    const ViewRec& cam = vs.v[view];
    const uint32_t lt = tile - cam.tile_off;
    const int X0 = (int)(lt % (uint32_t)cam.gx) * TW + (int)(reg % Reg::NX) * CW;
    const int Y0 = (int)(lt / (uint32_t)cam.gx) * TH + (int)(reg / Reg::NX) * CH;
    uint2 rg = p.ranges[tile];
    uint32_t start = rg.x, count = rg.y - rg.x;
    // the tile's list must lie inside the sorted instances (checked build; it
    // assumes the status words of the lgs_sort call that made the lists)
    if (!LGS_CHECK(start <= start + count &&
                   (count == 0 || (int64_t)start + count <= p.status[LGS_ST_NUM_INSTANCES]), 20, p.status))
        count = 0;

    constexpr bool global_frame = VAR == VAR_GLOBAL;
    const float Ox = global_frame ? 0.f : (float)X0 + 0.5f * (CW - 1);
    const float Oy = global_frame ? 0.f : (float)Y0 + 0.5f * (CH - 1);
    // the lane's pixels: tile-local (lx, ly[k]); basis B = [x'^2, x'y', y'^2, x', y', 1]
    const int lx = (warp % Lay::NBX) * WX + lane % WX;
    int ly[PPL];
    bool inside[PPL];
    P bx2, bxy, by2, bxl, byl, T, C0, C1, C2, thr;
    uint32_t last[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        ly[k] = (warp / Lay::NBX) * WY + lane / WX + k * (WY / 2);
        inside[k] = X0 + lx < cam.W && Y0 + ly[k] < cam.H;
        const float xl = global_frame ? (float)(X0 + lx) : (float)lx - 0.5f * (CW - 1);
        const float yl = global_frame ? (float)(Y0 + ly[k]) : (float)ly[k] - 0.5f * (CH - 1);
        bx2[k] = xl * xl;
        bxy[k] = xl * yl;
        by2[k] = yl * yl;
        bxl[k] = xl;
        byl[k] = yl;
        T[k] = 1.f;
        C0[k] = 0.f;
        C1[k] = 0.f;
        C2[k] = 0.f;
        // per-pixel 1/255 threshold in the log2 domain; +inf once the pixel
        // has stopped (or lies outside the image), so that it never blends again
        thr[k] = inside[k] ? LOG2_ALPHA_MIN : INF_F;
        last[k] = 0;
    }
    auto lane_done = [&]() {
        bool d = true;
#pragma unroll
        for (int k = 0; k < PPL; ++k) d = d && (VAR == VAR_LITERAL ? (!inside[k] || T[k] < 1e-4f) : thr[k] > 0.f);
        return d;
    };
    bool warp_done = __all_sync(0xffffffffu, lane_done());
    uint32_t pairs = 0, cands = 0;

    // Staging: thread t copies the three 16-B records of list entries b0 + t,
    // b0 + t + NT, ... with cp.async into buffer (b0 / NB) & 1, one batch ahead,
    // so the gathers of batch b+1 are in flight while batch b blends. A thread
    // reads back only the slots it copied itself, so its own group fence orders them.
    const int ti = threadIdx.x;
    auto stage = [&](uint32_t b, int buf) {
#pragma unroll
        for (int sl = ti; sl < NB; sl += NT) {
            const uint32_t jj = b + (uint32_t)sl;
            if (jj < count) {
                const uint32_t id = p.vals[start + jj];
                cp_async16(&S.raw[buf][0][sl], p.xy + id);
                cp_async16(&S.raw[buf][1][sl], p.conic + id);
                cp_async16(&S.raw[buf][2][sl], p.rgb + id);
            }
        }
        cp_async_commit();
    };
    if (count > 0 && !__syncthreads_and(warp_done)) stage(0, 0);
    int buf = 0;
    for (uint32_t b0 = 0; b0 < count; b0 += NB, buf ^= 1) {
        if (__syncthreads_and(warp_done)) break;
        if (b0 + NB < count) stage(b0 + NB, buf ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
#pragma unroll
        for (int sl = ti; sl < NB; sl += NT) {
            if (b0 + (uint32_t)sl < count) {
                const float4 xy = S.raw[buf][0][sl];
                const float4 co = S.raw[buf][1][sl];
                const float4 col = S.raw[buf][2][sl];
                const float dx = __fadd_rn(xy.x - Ox, xy.z);
                const float dy = __fadd_rn(xy.y - Oy, xy.w);
                const float Dn = fmaf(co.x, dx, co.y * dy);
                const float En = fmaf(co.y, dx, co.z * dy);
                const float Fn = -0.5f * fmaf(dx, Dn, dy * En);
                S.sV[sl] = make_float4(-0.5f * LOG2E * co.x, -LOG2E * co.y, -0.5f * LOG2E * co.z,
                                       fmaf(Fn, LOG2E, __log2f(co.w)));
                S.sDE[sl] = make_float4(Dn * LOG2E, En * LOG2E, 0.f, 0.f);
                S.sC[sl] = make_float4(-col.x, -col.y, -col.z, __uint_as_float(b0 + (uint32_t)sl + 1u));
                S.sM[sl] = (uint8_t)block_mask<CW, CH, WX, WY>(co.x, co.y, co.z, co.w, __fadd_rn(xy.x, xy.z),
                                                               __fadd_rn(xy.y, xy.w), X0, Y0);
            }
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)NB, count - b0);
        if (COUNT && !warp_done) cands += (uint32_t)nb;
        if (!warp_done) {
            // compact the warp's list: the batch indices whose mask bit for this
            // warp is set, in list order (one ballot per 32 candidates)
            uint16_t* sL = S.sL[warp];
            int nl = 0;
            for (int c0 = 0; c0 < nb; c0 += 32) {
                const int jj = c0 + lane;
                const bool hit = jj < nb && ((S.sM[jj] >> warp) & 1u);
                const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                if (hit) sL[nl + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(16 * jj);
                nl += __popc(bal);
            }
            __syncwarp();
            // walk it; the warp leaves once every lane is done (tested per 32)
            for (int i0 = 0; i0 < nl && !warp_done; i0 += 32) {
                const int iend = min(nl, i0 + 32);
#pragma unroll 8
                for (int i = i0; i < iend; ++i) {
                    const int off = sL[i];
                    if (VAR == VAR_LITERAL) {
                        if (__all_sync(0xffffffffu, lane_done())) { warp_done = true; break; }
                        if (COUNT) ++pairs;
                    } else if (COUNT) {
                        if (__all_sync(0xffffffffu, lane_done())) break;
                        ++pairs;
                    }
                    const float4 V = at_offset(S.sV, off);
                    const float4 DE = at_offset(S.sDE, off);
                    const float4 ncol = at_offset(S.sC, off);
                    const uint32_t idx = __float_as_uint(ncol.w);
                    const P pw = pfma(bcast<PPL>(V.x), bx2, pfma(bcast<PPL>(V.y), bxy, pfma(bcast<PPL>(V.z), by2,
                                 pfma(bcast<PPL>(DE.x), bxl, pfma(bcast<PPL>(DE.y), byl, bcast<PPL>(V.w))))));
                    // -alpha = -min(0.99, 2^pw), negated so that the packed
                    // updates below need no separate negation
                    P nal;
#pragma unroll
                    for (int k = 0; k < PPL; ++k) nal[k] = fmaxf(-0.99f, -ex2_approx(pw[k]));
                    if (VAR == VAR_LITERAL) {
                        const P nw = pmul(nal, T);          // -w = -alpha T
                        C0 = pfma(bcast<PPL>(ncol.x), nw, C0);
                        C1 = pfma(bcast<PPL>(ncol.y), nw, C1);
                        C2 = pfma(bcast<PPL>(ncol.z), nw, C2);
                        T = padd(T, nw);                    // T - w
#pragma unroll
                        for (int k = 0; k < PPL; ++k) last[k] = idx;
                        continue;
                    }
                    const P tT = pfma(nal, T, T);           // T (1 - alpha), one rounding
                    P nab;
#pragma unroll
                    for (int k = 0; k < PPL; ++k) {
                        const bool valid = pw[k] >= thr[k];
                        const bool blend = valid && tT[k] >= 1e-4f;
                        thr[k] = (valid && !blend) ? INF_F : thr[k];
                        // -alpha of the pixel's blend, 0 when it does not blend:
                        // the colour and T updates need no further select
                        nab[k] = blend ? nal[k] : 0.f;
                        last[k] = blend ? idx : last[k];
                    }
                    const P nw = pmul(nab, T);              // -w
                    C0 = pfma(bcast<PPL>(ncol.x), nw, C0);  // (-c)(-w) = c w exactly
                    C1 = pfma(bcast<PPL>(ncol.y), nw, C1);
                    C2 = pfma(bcast<PPL>(ncol.z), nw, C2);
                    T = pfma(nab, T, T);                    // T - alpha T, or T unchanged
                }
                if (__all_sync(0xffffffffu, lane_done())) warp_done = true;
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        if (!inside[k]) continue;
        const int64_t plane = (int64_t)cam.W * cam.H;
        const int64_t pix = (int64_t)(Y0 + ly[k]) * cam.W + (X0 + lx);
        float* o = p.out_rgb + 3 * (int64_t)cam.pix_off;
        o[pix] = fmaf(T[k], cam.bg[0], C0[k]);
        o[plane + pix] = fmaf(T[k], cam.bg[1], C1[k]);
        o[2 * plane + pix] = fmaf(T[k], cam.bg[2], C2[k]);
        p.out_T[cam.pix_off + pix] = T[k];
        p.out_n[cam.pix_off + pix] = last[k];
    }
    if (COUNT && lane == 0 && pairs)
        atomicAdd(reinterpret_cast<unsigned long long*>(p.status + LGS_ST_PAIRS),
                  (unsigned long long)pairs * 32ull * PPL);
    if (COUNT && lane == 0 && cands)
        atomicAdd(reinterpret_cast<unsigned long long*>(p.status + LGS_ST_CANDIDATES),
                  (unsigned long long)cands);
}

// One CTA per (tile, region).
template <int TW, int TH, int WX, int WY, bool COUNT, int VAR, int NB>
__global__ void __launch_bounds__(TileLayout<TW, TH, WX, WY>::NT) render_localgs(RenderParams p, Views vs) {
    __shared__ LocalSmem<NB> S;
    localgs_tile<TW, TH, WX, WY, COUNT, VAR, NB>(p, vs, blockIdx.x, S);
}

// Persistent CTAs: each pulls the next (tile, region) work item from a
// work-queue counter (status word LGS_ST_QUEUE, zeroed by the launcher) until
// all are taken, so uneven tile lists and uneven view sizes balance across
// the SMs.
template <int TW, int TH, int WX, int WY, bool COUNT, int NB>
__global__ void __launch_bounds__(TileLayout<TW, TH, WX, WY>::NT) render_localgs_persistent(RenderParams p,
                                                                                         Views vs) {
    __shared__ LocalSmem<NB> S;
    __shared__ uint32_t s_work;
    unsigned long long* q = reinterpret_cast<unsigned long long*>(p.status + LGS_ST_QUEUE);
    const uint32_t n_work = vs.n_tiles * (uint32_t)Regions<TW, TH>::N;
    for (;;) {
        if (threadIdx.x == 0) s_work = (uint32_t)atomicAdd(q, 1ull);
        __syncthreads();
        const uint32_t work = s_work;
        __syncthreads();
        if (work >= n_work) break;
        localgs_tile<TW, TH, WX, WY, COUNT, VAR_CONTRACT, NB>(p, vs, work, S);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ plain
template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(256) render_plain(RenderParams p, Views vs) {
    __shared__ float4 sXY[BATCH];
    __shared__ float4 sCO[BATCH];
    __shared__ float4 sC[BATCH];

    const TileCtx t = tile_ctx<TW, TH>(vs, p, blockIdx.x);
    const float pxf = (float)t.px, pyf = (float)t.py;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !t.inside;
    uint32_t pairs = 0;

    for (uint32_t b0 = 0; b0 < t.count; b0 += BATCH) {
        if (__syncthreads_count(done) == (int)blockDim.x) break;
        const uint32_t j = b0 + threadIdx.x;
        if (j < t.count) {
            const uint32_t id = p.vals[t.start + j];
            sXY[threadIdx.x] = p.xy[id];
            sCO[threadIdx.x] = p.conic[id];
            sC[threadIdx.x] = p.rgb[id];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)BATCH, t.count - b0);
        for (int g = 0; !done && g < nb; ++g) {
            if (COUNT && (threadIdx.x & 31) == (__ffs(__activemask()) - 1)) ++pairs;
            const float4 xy = sXY[g];
            const float dx = __fadd_rn(xy.x - pxf, xy.z);
            const float dy = __fadd_rn(xy.y - pyf, xy.w);
            const float4 co = sCO[g];
            const float power = plain_power(co, dx, dy);
            if (power > 0.f) continue;
            const float alpha = fminf(0.99f, co.w * __expf(power));
            if (alpha < 1.f / 255.f) continue;
            const float test_T = T * (1.f - alpha);
            if (test_T < 1e-4f) { done = true; continue; }
            const float4 col = sC[g];
            C0 += col.x * alpha * T;
            C1 += col.y * alpha * T;
            C2 += col.z * alpha * T;
            T = test_T;
            last = b0 + (uint32_t)g + 1u;
        }
        __syncthreads();
    }
    write_pixel(vs, p, t, C0, C1, C2, T, last);
    if (COUNT && pairs)
        atomicAdd(reinterpret_cast<unsigned long long*>(p.status + LGS_ST_PAIRS),
                  (unsigned long long)pairs * 32ull);
}

// The Local-GS contract kernel for one warp layout and staging batch size
// (one CTA per tile, or persistent CTAs pulling tiles from the work queue).
template <int TW, int TH, int WX, int WY, int NB>
lgs_status launch_contract(const RenderParams& p, const Views& vs, bool count, bool persistent,
                           cudaStream_t s) {
    constexpr int NT = TileLayout<TW, TH, WX, WY>::NT;
    const uint32_t n_work = vs.n_tiles * (uint32_t)Regions<TW, TH>::N;
    const dim3 grid(n_work), block(NT);
    if (!persistent) {
        if (count) render_localgs<TW, TH, WX, WY, true, VAR_CONTRACT, NB><<<grid, block, 0, s>>>(p, vs);
        else       render_localgs<TW, TH, WX, WY, false, VAR_CONTRACT, NB><<<grid, block, 0, s>>>(p, vs);
        return cuda_status(cudaGetLastError());
    }
    if (cudaMemsetAsync(p.status + LGS_ST_QUEUE, 0, sizeof(int64_t), s) != cudaSuccess) return LGS_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (count) {
        auto k = render_localgs_persistent<TW, TH, WX, WY, true, NB>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, 0);
        const unsigned g = (unsigned)min((int64_t)n_work, (int64_t)max(1, sms * max(per_sm, 1)));
        k<<<g, block, 0, s>>>(p, vs);
    } else {
        auto k = render_localgs_persistent<TW, TH, WX, WY, false, NB>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, 0);
        const unsigned g = (unsigned)min((int64_t)n_work, (int64_t)max(1, sms * max(per_sm, 1)));
        k<<<g, block, 0, s>>>(p, vs);
    }
    return cuda_status(cudaGetLastError());
}

template <int TW, int TH, int WX, int WY>
lgs_status launch_layout(const RenderParams& p, const Views& vs, int batch, bool count, bool persistent,
                         cudaStream_t s) {
    if (batch == 64) return launch_contract<TW, TH, WX, WY, 64>(p, vs, count, persistent, s);
    if (batch == 128) return launch_contract<TW, TH, WX, WY, 128>(p, vs, count, persistent, s);
    return launch_contract<TW, TH, WX, WY, 256>(p, vs, count, persistent, s);
}

// The study variants (literal, global frame) run in the paper's layout.
template <int TW, int TH, int VAR>
lgs_status launch_variant(const RenderParams& p, const Views& vs, bool count, cudaStream_t s) {
    constexpr int WX = TW, WY = TH / 8;
    const dim3 grid(vs.n_tiles), block(Layout<TW, TH, WX, WY>::NT);
    if (count) render_localgs<TW, TH, WX, WY, true, VAR, BATCH><<<grid, block, 0, s>>>(p, vs);
    else       render_localgs<TW, TH, WX, WY, false, VAR, BATCH><<<grid, block, 0, s>>>(p, vs);
    return cuda_status(cudaGetLastError());
}

template <int TW, int TH>
lgs_status launch_render(const RenderParams& p, const Views& vs, int mode, int batch, int wx, int wy,
                         bool count, bool persistent, cudaStream_t s) {
    if constexpr (Regions<TW, TH>::SPLIT) {
        // large tiles: Local-GS contract in 8x8 blocks only (checked on the host)
        return launch_layout<TW, TH, 8, 8>(p, vs, batch, count, persistent, s);
    } else {
    if (mode == LGS_MODE_PLAIN) {
        const dim3 grid(vs.n_tiles), block(256);
        if (count) render_plain<TW, TH, true><<<grid, block, 0, s>>>(p, vs);
        else       render_plain<TW, TH, false><<<grid, block, 0, s>>>(p, vs);
        return cuda_status(cudaGetLastError());
    }
    if (mode == LGS_MODE_LITERAL) return launch_variant<TW, TH, VAR_LITERAL>(p, vs, count, s);
    if (mode == LGS_MODE_GLOBAL) return launch_variant<TW, TH, VAR_GLOBAL>(p, vs, count, s);
    if (wx == TW && wy == TH / 8) return launch_layout<TW, TH, TW, TH / 8>(p, vs, batch, count, persistent, s);
    if constexpr (TW == 16) {
        if (wx == 8 && wy == 4) return launch_layout<16, 16, 8, 4>(p, vs, batch, count, persistent, s);
        if (wx == 16 && wy == 4) return launch_layout<16, 16, 16, 4>(p, vs, batch, count, persistent, s);
    }
    return launch_layout<TW, TH, 8, 8>(p, vs, batch, count, persistent, s);
    }
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status lgs_render_fwd(const lgs_pre_out* pre, const uint32_t* vals,
                                     const uint32_t* ranges, const lgs_camera* cams,
                                     int32_t n_views, const lgs_config* cfg, float* rgb,
                                     float* final_T, uint32_t* n_contrib, int64_t* d_status,
                                     void* stream) {
    if (!vals || !ranges || !rgb || !final_T || !n_contrib || !d_status) return LGS_ERR_ARG;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    st = check_pre(pre);
    if (st != LGS_OK) return st;
    if (cfg->mode < LGS_MODE_LOCALGS || cfg->mode > LGS_MODE_GLOBAL) return LGS_ERR_UNSUPPORTED;
    if ((cfg->flags & LGS_FLAG_PERSISTENT) && cfg->mode != LGS_MODE_LOCALGS) return LGS_ERR_UNSUPPORTED;
    if (cfg->batch != 0 && cfg->batch != 64 && cfg->batch != 128 && cfg->batch != 256) return LGS_ERR_UNSUPPORTED;
    const int batch = cfg->batch == 0 ? BATCH : cfg->batch;
    if (reinterpret_cast<uintptr_t>(ranges) & 7u) return LGS_ERR_ALIGN;
    RenderParams p;
    p.xy = reinterpret_cast<const float4*>(pre->xy);
    p.conic = reinterpret_cast<const float4*>(pre->conic);
    p.rgb = reinterpret_cast<const float4*>(pre->rgb);
    p.vals = vals;
    p.ranges = reinterpret_cast<const uint2*>(ranges);
    p.out_rgb = rgb;
    p.out_T = final_T;
    p.out_n = n_contrib;
    p.status = d_status;
    const bool count = (cfg->flags & LGS_FLAG_COUNT) != 0;
    const bool persistent = (cfg->flags & LGS_FLAG_PERSISTENT) != 0;
    int wx = 0, wy = 0;
    if (!warp_block(cfg, &wx, &wy)) return LGS_ERR_UNSUPPORTED;
    if (cfg->mode != LGS_MODE_LOCALGS &&
        (split_tile(cfg->tile_w, cfg->tile_h) || wx != cfg->tile_w || wy != cfg->tile_h / 8))
        return LGS_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tw = cfg->tile_w, th = cfg->tile_h;
    if (tw == 16 && th == 16) return launch_render<16, 16>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
    if (tw == 8 && th == 32) return launch_render<8, 32>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
    if (tw == 32 && th == 8) return launch_render<32, 8>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
    if (tw == 32 && th == 32) return launch_render<32, 32>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
    if (tw == 16 && th == 32) return launch_render<16, 32>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
    return launch_render<32, 16>(p, vs, cfg->mode, batch, wx, wy, count, persistent, s);
}
