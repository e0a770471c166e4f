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

}  // namespace lgs
