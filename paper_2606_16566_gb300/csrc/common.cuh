// common.cuh -- device-side helpers shared by the sm_103a kernels of liblgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgs.h"

namespace lgs {

// Per-view constants, passed by value in kernel parameters (<= 64 views).
struct ViewRec {
    float R[9];          // world -> camera rotation, row-major
    float t[3];          // world -> camera translation
    float fx, fy, cx, cy;
    float campos[3];
    float bg[3];
    int32_t W, H, gx, gy;
    uint32_t tile_off;   // first global tile id of the view
    uint32_t pix_off;    // first pixel of the view in the concatenated outputs
};

struct Views {
    int32_t n;
    int32_t tile_w, tile_h;
    int32_t flags;       // lgs_config flags
    uint32_t n_tiles;    // total tiles over all views
    uint32_t n_pix;      // total pixels over all views
    ViewRec v[LGS_MAX_VIEWS];
};

// View owning a global tile id (binary search over tile offsets).
__device__ __forceinline__ int view_of_tile(const Views& vs, uint32_t tile) {
    int lo = 0, hi = vs.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vs.v[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First device-side error wins; later ones are dropped.
__device__ __forceinline__ void report_error(int64_t* st, int64_t code, int64_t detail) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(st);
    if (atomicCAS(w + LGS_ST_CODE, 0ull, (unsigned long long)code) == 0ull)
        atomicExch(w + LGS_ST_DETAIL, (unsigned long long)detail);
}

// Bounds checks of the LGS_CHECKED build (a test build; compiled out otherwise):
// a failed check records LGS_ERR_INTERNAL with detail 1000 + site in the status
// words and the caller skips the access, so an index bug shows up as a status
// code instead of a memory fault.
#ifdef LGS_CHECKED
#define LGS_CHECK(cond, site, st) \
    ((cond) ? true : (::lgs::report_error((st), LGS_ERR_INTERNAL, 1000 + (site)), false))
#else
#define LGS_CHECK(cond, site, st) true
#endif

// ---------------------------------------------------------------- float pairs
// Unevaluated sums hi + lo of two floats (Dekker / Knuth error-free
// transformations). The __f*_rn intrinsics keep the compiler from contracting
// or reassociating the compensated steps.
struct ff { float hi, lo; };

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

// a0*b0 + a1*b1 + a2*b2 + c with about twice the float precision
// (compensated dot product, Ogita-Rump-Oishi Dot2).
__device__ __forceinline__ ff dot3_plus(float a0, float b0, float a1, float b1, float a2, float b2,
                                        float c) {
    ff p0 = two_prod(a0, b0);
    ff p1 = two_prod(a1, b1);
    ff p2 = two_prod(a2, b2);
    ff s = two_sum(p0.hi, p1.hi);
    float err = __fadd_rn(__fadd_rn(p0.lo, p1.lo), s.lo);
    ff s2 = two_sum(s.hi, p2.hi);
    err = __fadd_rn(__fadd_rn(err, p2.lo), s2.lo);
    ff s3 = two_sum(s2.hi, c);
    err = __fadd_rn(err, s3.lo);
    return fast_two_sum(s3.hi, err);
}

// (a.hi + a.lo) / (b.hi + b.lo) as a float pair.
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q = __fdiv_rn(a.hi, b.hi);
    // r = a - q*b, exact leading part via fma
    float r = __fmaf_rn(-q, b.hi, a.hi);
    r = __fadd_rn(r, a.lo);
    r = __fmaf_rn(-q, b.lo, r);
    float ql = __fdiv_rn(r, b.hi);
    return fast_two_sum(q, ql);
}

// s * (a.hi + a.lo) + c for floats s, c.
__device__ __forceinline__ ff ff_mul_add(float s, ff a, float c) {
    ff p = two_prod(s, a.hi);
    float lo = __fmaf_rn(s, a.lo, p.lo);
    ff t = two_sum(p.hi, c);
    return fast_two_sum(t.hi, __fadd_rn(t.lo, lo));
}

// floor((a.hi + a.lo)) for |a| < 2^23.
__device__ __forceinline__ float ff_floor(ff a) {
    float f = floorf(a.hi);
    if (f == a.hi && a.lo < 0.f) f -= 1.f;
    return f;
}

// Gaussian exponent of the plain (global-coordinate) kernels,
// -1/2 (a dx^2 + c dy^2) - b dx dy, with explicit roundings so that the plain
// forward and backward kernels evaluate it bit for bit alike.
__device__ __forceinline__ float plain_power(float4 co, float dx, float dy) {
    const float t1 = __fmul_rn(co.x, __fmul_rn(dx, dx));
    const float t2 = __fmaf_rn(co.z, __fmul_rn(dy, dy), t1);
    const float t3 = __fmul_rn(co.y, __fmul_rn(dx, dy));
    return __fmaf_rn(-0.5f, t2, -t3);
}

// ---------------------------------------------------------------- tight box
// Integer floor division for any sign of p (q > 0).
__device__ __forceinline__ int floor_div(int p, int q) {
    return p >= 0 ? p / q : -((-p + q - 1) / q);
}

constexpr float TIGHT_LN255 = 5.5412635451584258f;  // ln 255

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-entry constants of the conservative tight box (Sec. III-C2) of a
// Gaussian's alpha >= 1/255 region: the ellipse a x~^2 + 2b x~y~ + c y~^2 = tau
// around the mean (mux, muy), tau = 2 ln(255 o), widened against FP32 rounding
// to tau' = 1.001 tau + 0.02. kind: 0 = no region (tau' <= 0), 2 = the conic is
// not positive definite (no box: every row counts), 1 = box.
struct TightBox {
    float mux, muy, a, b, ic, det, ct, xr, bdy, dy;
    int kind;
};

__device__ __forceinline__ TightBox tight_box(float a, float b, float c, float o, float mux,
                                              float muy) {
    TightBox t;
    float tau = __fmul_rn(2.f, __fadd_rn(TIGHT_LN255, __logf(o)));
    tau = __fmaf_rn(tau, 1.001f, 0.02f);
    const float det = __fmaf_rn(a, c, -__fmul_rn(b, b));
    t.kind = !(tau > 0.f) ? 0 : (!(det > 0.f) ? 2 : 1);
    const float idet = rcp_approx(det);
    t.mux = mux;
    t.muy = muy;
    t.a = a;
    t.b = b;
    t.ic = rcp_approx(c);
    t.det = det;
    t.ct = __fmul_rn(c, tau);
    t.xr = sqrt_approx(__fmul_rn(t.ct, idet));                 // half width of the ellipse
    t.dy = sqrt_approx(__fmul_rn(__fmul_rn(a, tau), idet));    // half height
    t.bdy = __fmul_rn(b, t.dy);
    return t;
}

// Rows of the tight box over one pixel column strip X0 .. X0+tw-1: the ellipse
// cut to the strip's x-range, its lowest and highest points over that range
// from Case A (the root at the strip's left edge), Case B (the right edge) or
// Case C (the ellipse's own extreme, +-d_y), widened by 1/64 px at both ends.
// Returns 0 when the strip misses the ellipse, 2 when there is no box, else 1
// with [*P, *Q] = the integer pixel rows ceil(lower), floor(upper) (clamped
// to +-2^30; empty when *P > *Q). Every step is an explicitly rounded
// intrinsic or a single approximate instruction, so every kernel that calls
// this (preprocess, emission, render, adjoint) gets bit-identical spans. The
// approximations (relative error ~1e-7) sit far inside the widening margin, so
// every pixel whose FP32 alpha clears 1/255 lies inside the box.
__device__ __forceinline__ int column_rows(const TightBox& t, int X0, int tw, int* P, int* Q) {
    if (t.kind != 1) return t.kind;
    float x0 = __fsub_rn((float)X0, t.mux), x1 = __fsub_rn((float)(X0 + tw - 1), t.mux);
    if (x1 < -t.xr || x0 > t.xr) return 0;
    x0 = fmaxf(x0, -t.xr);
    x1 = fminf(x1, t.xr);
    const float ax0 = __fmul_rn(t.a, x0), ax1 = __fmul_rn(t.a, x1);
    // roots of the ellipse at x: y = (-b x +- sqrt(c tau - det x^2)) / c
    const float r0 = sqrt_approx(fmaxf(0.f, __fmaf_rn(-t.det, __fmul_rn(x0, x0), t.ct)));
    const float r1 = sqrt_approx(fmaxf(0.f, __fmaf_rn(-t.det, __fmul_rn(x1, x1), t.ct)));
    const float bx0 = __fmul_rn(t.b, x0), bx1 = __fmul_rn(t.b, x1);
    float ymax, ymin;
    if (-t.bdy < ax0)      ymax = __fmul_rn(__fsub_rn(r0, bx0), t.ic);
    else if (-t.bdy > ax1) ymax = __fmul_rn(__fsub_rn(r1, bx1), t.ic);
    else                   ymax = t.dy;
    if (t.bdy < ax0)       ymin = __fmul_rn(__fsub_rn(-r0, bx0), t.ic);
    else if (t.bdy > ax1)  ymin = __fmul_rn(__fsub_rn(-r1, bx1), t.ic);
    else                   ymin = -t.dy;
    const float lo = __fsub_rn(__fadd_rn(t.muy, ymin), 0.015625f);
    const float hi = __fadd_rn(__fadd_rn(t.muy, ymax), 0.015625f);
    *P = (int)ceilf(fminf(fmaxf(lo, -1073741824.f), 1073741824.f));
    *Q = (int)floorf(fminf(fmaxf(hi, -1073741824.f), 1073741824.f));
    return 1;
}

// Tile rows [*lo, *hi] of the rect rows [ry0, ry1) that the tight box of
// column strip X0 .. X0+tw-1 reaches (tile height th); returns their number.
__device__ __forceinline__ int tight_tile_rows(const TightBox& t, int X0, int tw, int th, int ry0,
                                               int ry1, int* lo, int* hi) {
    int P = 0, Q = 0;
    const int r = column_rows(t, X0, tw, &P, &Q);
    int l = ry0, h = ry1 - 1;
    if (r == 0) return 0;
    if (r == 1) {
        if (P > Q) return 0;
        l = max(l, floor_div(P, th));
        h = min(h, floor_div(Q, th));
    }
    *lo = l;
    *hi = h;
    return h >= l ? h - l + 1 : 0;
}

// Warp-block mask of one Gaussian for one tile (Sec. III-C2/C3, with the
// paper's 8-bit mask of full-width row strips generalised to 2D blocks): the
// tile is cut into (TW/WX) x (TH/WY) blocks of WX x WY pixels, block
// (bx, by) owning bit by * (TW/WX) + bx. For every block column the
// conservative tight box is evaluated over that column's pixel range
// (column_rows), and the bits of the blocks whose rows it reaches are set.
// Every pixel whose FP32 alpha clears 1/255 lies in a set block. With WX = TW
// the blocks are the paper's full-width row strips.
template <int TW, int TH, int WX, int WY>
__device__ __forceinline__ uint32_t block_mask(float a, float b, float c, float o, float mux,
                                               float muy, int X0, int Y0) {
    constexpr int NBX = TW / WX, NBY = TH / WY;
    static_assert(TW % WX == 0 && TH % WY == 0 && NBX * NBY <= 8, "at most 8 blocks per tile");
    const TightBox tb = tight_box(a, b, c, o, mux, muy);
    if (tb.kind == 0) return 0u;
    if (tb.kind == 2) return (1u << (NBX * NBY)) - 1u;
    uint32_t m = 0u;
#pragma unroll
    for (int bx = 0; bx < NBX; ++bx) {
        int P = 0, Q = 0;
        if (column_rows(tb, X0 + bx * WX, WX, &P, &Q) != 1) continue;
        const int ys = max(Y0, P), ye = min(Y0 + TH - 1, Q);
        if (ys > ye) continue;
        const int bs = (ys - Y0) / WY, be = (ye - Y0) / WY;
        if (NBX == 1) {
            m |= ((1u << (be - bs + 1)) - 1u) << bs;
        } else {
#pragma unroll
            for (int by = 0; by < NBY; ++by)
                if (by >= bs && by <= be) m |= 1u << (by * NBX + bx);
        }
    }
    return m;
}

// The 8-strip mask of the paper's layout: eight full-width strips of TH/8 rows.
template <int TW, int TH>
__device__ __forceinline__ uint32_t warp_mask(float a, float b, float c, float o, float mux,
                                              float muy, int X0, int Y0) {
    return block_mask<TW, TH, TW, TH / 8>(a, b, c, o, mux, muy, X0, Y0);
}

// ---------------------------------------------------------------- warp layouts
// Warp layout of a Local-GS tile: NW = (TW/WX) * (TH/WY) warps, warp w owning
// the WX x WY pixel block (w % (TW/WX), w / (TW/WX)) and bit w of the block
// mask. Lane l evaluates pixel (l % WX, l / WX) of its block; with 64-pixel
// blocks (PPL = 2 pixels per lane) also the pixel WY/2 rows below, and the
// per-pixel FP32 arithmetic of the pair runs as packed two-wide instructions
// (fma.rn.f32x2 / mul.rn.f32x2), one issue slot for both pixels. The paper's
// layout is WX = TW, WY = TH/8 (eight full-width strips, one pixel per lane).
template <int TW, int TH, int WX, int WY>
struct Layout {
    static constexpr int NBX = TW / WX, NBY = TH / WY, NW = NBX * NBY, NT = 32 * NW;
    static constexpr int PPL = WX * WY / 32;
    static_assert(TW % WX == 0 && TH % WY == 0, "blocks tile the tile");
    static_assert(PPL == 1 || PPL == 2, "one or two pixels per lane");
    static_assert(NW == 4 || NW == 8, "4 or 8 warps per tile");
    static_assert(32 % WX == 0 || WX == 32, "a warp row is whole lanes");
};

// CTA regions of a sort tile: a tile of 256 pixels is one region; the larger
// tiles (32x32, 16x32, 32x16) are split into 16x16 regions, one CTA each, all
// walking the tile's one list. Larger tiles mean fewer (Gaussian, tile)
// instances to sort; the regions keep the warp blocks and the CTA size of the
// 256-pixel tiles.
template <int TW, int TH>
struct Regions {
    static constexpr bool SPLIT = TW * TH > 256;
    static constexpr int CW = SPLIT ? 16 : TW, CH = SPLIT ? 16 : TH;
    static constexpr int NX = TW / CW, NY = TH / CH, N = NX * NY;
};

template <int TW, int TH, int WX, int WY>
using TileLayout = Layout<Regions<TW, TH>::CW, Regions<TW, TH>::CH, WX, WY>;

// P pixels' worth of one float, with the packed FP32 operations on two.
template <int P> struct Px;
template <> struct Px<1> {
    float v;
    __device__ __forceinline__ float& operator[](int) { return v; }
    __device__ __forceinline__ float operator[](int) const { return v; }
};
template <> struct Px<2> {
    float2 v;
    __device__ __forceinline__ float& operator[](int k) { return k ? v.y : v.x; }
    __device__ __forceinline__ float operator[](int k) const { return k ? v.y : v.x; }
};
__device__ __forceinline__ Px<1> pfma(Px<1> a, Px<1> b, Px<1> c) { return {__fmaf_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ Px<2> pfma(Px<2> a, Px<2> b, Px<2> c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ Px<1> pmul(Px<1> a, Px<1> b) { return {__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ Px<2> pmul(Px<2> a, Px<2> b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ Px<1> padd(Px<1> a, Px<1> b) { return {__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ Px<2> padd(Px<2> a, Px<2> b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ Px<1> pneg(Px<1> a) { return {-a.v}; }
__device__ __forceinline__ Px<2> pneg(Px<2> a) { return {make_float2(-a.v.x, -a.v.y)}; }
template <int P> __device__ __forceinline__ Px<P> bcast(float s);
template <> __device__ __forceinline__ Px<1> bcast<1>(float s) { return {s}; }
template <> __device__ __forceinline__ Px<2> bcast<2>(float s) { return {make_float2(s, s)}; }

}  // namespace lgs
