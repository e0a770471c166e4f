// preprocess.cu -- stage 1 of the 3DGS pipeline (Local-GS Sec. II-A, Fig. 2):
// per Gaussian and view, near-plane cull, EWA projection of the covariance,
// conic, radius, tile rect, SH colour and depth.
//
// One thread per Gaussian; the thread loops over the views of the batch so
// that the Gaussian's parameters (236 B at SH degree 3) are read from HBM once
// per batch instead of once per view. Outputs are view-major (v*N + i), so
// consecutive threads write consecutive entries.
//
// Precision: the camera-space position and the projected mean are computed as
// unevaluated float pairs (compensated dot product and division), so the
// depth key, the near-plane test and the tile rect take the same decisions as
// the double-precision definition except within ~1e-12 of a threshold. The 2D
// covariance is formed as M M^T + 0.3 I with M = J W R S, and its determinant
// through the Lagrange identity |m0|^2|m1|^2 - (m0.m1)^2 = |m0 x m1|^2, which
// has no cancellation.
#include "common.cuh"
#include "host.h"

#include <math.h>

namespace lgs {

struct PreParams {
    const float* means;
    const float* scales;
    const float* quats;
    const float* opac;
    const float* sh;
    int64_t n;
    float* xy;
    float* conic;
    float* rgb;
    float* depth;
    int32_t* radius;
    uint32_t* tiles;
    uint64_t* rect;
    uint8_t* flags;
    uint4* emit;      // optional emission records (2 x uint4 per entry), may be NULL
    int64_t* status;
};

// Kahan's 2x2 determinant a*d - b*c with one fma-compensated rounding.
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    float w = __fmul_rn(b, c);
    float e = __fmaf_rn(-b, c, w);
    float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

// Real SH basis times coefficients (Condon-Shortley phase; index l^2 + l + m).
template <int DEG>
__device__ __forceinline__ float3 sh_colour(const float* c, float x, float y, float z) {
    constexpr float C0 = 0.28209479177387814f;
    float3 r = make_float3(C0 * c[0], C0 * c[1], C0 * c[2]);
    if (DEG >= 1) {
        constexpr float C1 = 0.4886025119029199f;
        float b1 = -C1 * y, b2 = C1 * z, b3 = -C1 * x;
        r.x += b1 * c[3] + b2 * c[6] + b3 * c[9];
        r.y += b1 * c[4] + b2 * c[7] + b3 * c[10];
        r.z += b1 * c[5] + b2 * c[8] + b3 * c[11];
        if (DEG >= 2) {
            float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
            float b[5] = {1.0925484305920792f * xy, -1.0925484305920792f * yz,
                          0.31539156525252005f * (2.f * zz - xx - yy), -1.0925484305920792f * xz,
                          0.5462742152960396f * (xx - yy)};
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                r.x += b[k] * c[(4 + k) * 3 + 0];
                r.y += b[k] * c[(4 + k) * 3 + 1];
                r.z += b[k] * c[(4 + k) * 3 + 2];
            }
            if (DEG >= 3) {
                float e[7] = {-0.5900435899266435f * y * (3.f * xx - yy),
                              2.890611442640554f * xy * z,
                              -0.4570457994644658f * y * (4.f * zz - xx - yy),
                              0.3731763325901154f * z * (2.f * zz - 3.f * xx - 3.f * yy),
                              -0.4570457994644658f * x * (4.f * zz - xx - yy),
                              1.445305721320277f * z * (xx - yy),
                              -0.5900435899266435f * x * (xx - 3.f * yy)};
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    r.x += e[k] * c[(9 + k) * 3 + 0];
                    r.y += e[k] * c[(9 + k) * 3 + 1];
                    r.z += e[k] * c[(9 + k) * 3 + 2];
                }
            }
        }
    }
    return r;
}

template <int DEG>
__global__ void __launch_bounds__(256) preprocess_kernel(PreParams p, Views vs) {
    constexpr int NC = (DEG + 1) * (DEG + 1) * 3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t N = p.n;

    const float mx = p.means[3 * i], my = p.means[3 * i + 1], mz = p.means[3 * i + 2];
    const float sx = p.scales[3 * i], sy = p.scales[3 * i + 1], sz = p.scales[3 * i + 2];
    const float4 q4 = reinterpret_cast<const float4*>(p.quats)[i];
    const float op = p.opac[i];
    const bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(sx) &&
                        isfinite(sy) && isfinite(sz) && isfinite(q4.x) && isfinite(q4.y) &&
                        isfinite(q4.z) && isfinite(q4.w) && isfinite(op);
    if (!finite)
        atomicAdd(reinterpret_cast<unsigned long long*>(p.status + LGS_ST_NONFINITE), 1ull);

    // R(q) diag(s), view independent. q = (w, x, y, z), normalised.
    float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    float RS[9] = {(1.f - 2.f * (y * y + z * z)) * sx, 2.f * (x * y - w * z) * sy,
                   2.f * (x * z + w * y) * sz,
                   2.f * (x * y + w * z) * sx, (1.f - 2.f * (x * x + z * z)) * sy,
                   2.f * (y * z - w * x) * sz,
                   2.f * (x * z - w * y) * sx, 2.f * (y * z + w * x) * sy,
                   (1.f - 2.f * (x * x + y * y)) * sz};

    float shc[NC];
    bool sh_loaded = false, sh_ok = true;

    for (int v = 0; v < vs.n; ++v) {
        const ViewRec& c = vs.v[v];
        const int64_t m = (int64_t)v * N + i;
        ff tx = dot3_plus(c.R[0], mx, c.R[1], my, c.R[2], mz, c.t[0]);
        ff ty = dot3_plus(c.R[3], mx, c.R[4], my, c.R[5], mz, c.t[1]);
        ff tz = dot3_plus(c.R[6], mx, c.R[7], my, c.R[8], mz, c.t[2]);
        const float zf = tz.hi;
        p.depth[m] = zf;
        // near plane: cull when z <= 0.2 (the double 0.2 lies 2.98e-9 below 0.2f)
        const float dz = __fadd_rn(__fsub_rn(zf, 0.2f), tz.lo);
        uint8_t fl = 0;
        int32_t rad = 0;
        uint32_t ntiles = 0;
        uint64_t rpack = 0;
        if (finite && dz > -2.98023224e-9f) {
            // EWA Jacobian at the (clamped) direction
            const float limx = 1.3f * (0.5f * (float)c.W / c.fx);
            const float limy = 1.3f * (0.5f * (float)c.H / c.fy);
            float txz = tx.hi / zf, tyz = ty.hi / zf;
            if (txz < -limx) { txz = -limx; fl |= 8; }
            if (txz > limx) { txz = limx; fl |= 8; }
            if (tyz < -limy) { tyz = -limy; fl |= 16; }
            if (tyz > limy) { tyz = limy; fl |= 16; }
            const float iz = 1.f / zf;
            const float J00 = c.fx * iz, J02 = -c.fx * txz * iz;
            const float J11 = c.fy * iz, J12 = -c.fy * tyz * iz;
            // WRS = W * RS
            float WRS[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    WRS[r * 3 + k] = c.R[r * 3 + 0] * RS[k] + c.R[r * 3 + 1] * RS[3 + k] +
                                     c.R[r * 3 + 2] * RS[6 + k];
            float m0[3], m1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                m0[k] = J00 * WRS[k] + J02 * WRS[6 + k];
                m1[k] = J11 * WRS[3 + k] + J12 * WRS[6 + k];
            }
            const float n0 = m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2];
            const float n1 = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
            const float d01 = m0[0] * m1[0] + m0[1] * m1[1] + m0[2] * m1[2];
            const float cx0 = det2(m0[1], m0[2], m1[1], m1[2]);
            const float cx1 = det2(m0[2], m0[0], m1[2], m1[0]);
            const float cx2 = det2(m0[0], m0[1], m1[0], m1[1]);
            const float S00 = n0 + 0.3f, S11 = n1 + 0.3f;
            const float det = (cx0 * cx0 + cx1 * cx1 + cx2 * cx2) + 0.3f * (n0 + n1) + 0.09f;
            const float hd = 0.5f * (n0 - n1);
            const float disc = hd * hd + d01 * d01;
            const float lam1 = 0.5f * (S00 + S11) + sqrtf(fmaxf(0.1f, disc));
            const float rr = ceilf(3.f * sqrtf(lam1));
            // projected mean u = fx X/Z + cx as a float pair
            const ff uq = ff_div(tx, tz), vq = ff_div(ty, tz);
            const ff u = ff_mul_add(c.fx, uq, c.cx);
            const ff vv = ff_mul_add(c.fy, vq, c.cy);
            const float itw = 1.f / (float)vs.tile_w, ith = 1.f / (float)vs.tile_h;
            auto edge = [](ff a, float add, float inv) {
                ff s = two_sum(a.hi, add);
                ff t = fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
                return ff_floor(ff{t.hi * inv, t.lo * inv});
            };
            const float gxf = (float)c.gx, gyf = (float)c.gy;
            const int x0 = (int)fminf(gxf, fmaxf(0.f, edge(u, -rr, itw)));
            const int x1 = (int)fminf(gxf, fmaxf(0.f, edge(u, rr + (float)(vs.tile_w - 1), itw)));
            const int y0 = (int)fminf(gyf, fmaxf(0.f, edge(vv, -rr, ith)));
            const int y1 = (int)fminf(gyf, fmaxf(0.f, edge(vv, rr + (float)(vs.tile_h - 1), ith)));
            const uint32_t area = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
            if (area > 0) {
                if (!sh_loaded) {
                    const float* src = p.sh + i * NC;
                    if constexpr (NC % 4 == 0) {
                        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                        for (int k = 0; k < NC / 4; ++k) {
                            float4 t4 = s4[k];
                            shc[4 * k] = t4.x; shc[4 * k + 1] = t4.y;
                            shc[4 * k + 2] = t4.z; shc[4 * k + 3] = t4.w;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < NC; ++k) shc[k] = src[k];
                    }
                    sh_loaded = true;
                    // a non-finite SH coefficient culls the Gaussian in this
                    // and every later view (earlier views reached no tile, so
                    // it was culled there anyway) and is counted once; SH is
                    // read, and so checked, only for Gaussians that reach a tile
                    float probe = 0.f;
#pragma unroll
                    for (int k = 0; k < NC; ++k) probe = __fadd_rn(probe, __fmul_rn(shc[k], 0.f));
                    sh_ok = probe == 0.f;
                    if (!sh_ok)
                        atomicAdd(reinterpret_cast<unsigned long long*>(p.status + LGS_ST_NONFINITE), 1ull);
                }
            }
            if (area > 0 && sh_ok) {
                float dx = mx - c.campos[0], dy = my - c.campos[1], dzz = mz - c.campos[2];
                const float inv = 1.f / sqrtf(dx * dx + dy * dy + dzz * dzz);
                dx *= inv; dy *= inv; dzz *= inv;
                float3 col = sh_colour<DEG>(shc, dx, dy, dzz);
                col.x += 0.5f; col.y += 0.5f; col.z += 0.5f;
                if (col.x < 0.f) { col.x = 0.f; fl |= 1; }
                if (col.y < 0.f) { col.y = 0.f; fl |= 2; }
                if (col.z < 0.f) { col.z = 0.f; fl |= 4; }
                const float inv_det = 1.f / det;
                const float ca = S11 * inv_det, cb = -d01 * inv_det, cc = S00 * inv_det;
                reinterpret_cast<float4*>(p.xy)[m] = make_float4(u.hi, vv.hi, u.lo, vv.lo);
                reinterpret_cast<float4*>(p.conic)[m] = make_float4(ca, cb, cc, op);
                reinterpret_cast<float4*>(p.rgb)[m] = make_float4(col.x, col.y, col.z, zf);
                rad = (int32_t)rr;
                ntiles = area;
                rpack = (uint64_t)(uint32_t)x0 | ((uint64_t)(uint32_t)y0 << 16) |
                        ((uint64_t)(uint32_t)x1 << 32) | ((uint64_t)(uint32_t)y1 << 48);
                if (p.emit) {
                    p.emit[2 * m] = make_uint4((uint32_t)rpack, (uint32_t)(rpack >> 32),
                                               __float_as_uint(__fadd_rn(u.hi, u.lo)),
                                               __float_as_uint(__fadd_rn(vv.hi, vv.lo)));
                    p.emit[2 * m + 1] = make_uint4(__float_as_uint(ca), __float_as_uint(cb),
                                                   __float_as_uint(cc), __float_as_uint(op));
                }
            }
        }
        p.radius[m] = rad;
        p.tiles[m] = ntiles;
        p.rect[m] = rpack;
        p.flags[m] = fl;
    }
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status lgs_preprocess(const lgs_gaussians* g, const lgs_camera* cams,
                                     int32_t n_views, const lgs_config* cfg,
                                     const lgs_pre_out* out, int64_t* d_status, void* stream) {
    if (!g || !out || !d_status) return LGS_ERR_ARG;
    if (g->n < 0 || g->n >= (1ll << 31)) return LGS_ERR_ARG;
    if (g->sh_degree < 0 || g->sh_degree > LGS_MAX_SH_DEGREE) return LGS_ERR_UNSUPPORTED;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    if ((uint64_t)g->n * (uint64_t)n_views >= (1ull << 32)) return LGS_ERR_UNSUPPORTED;
    st = check_pre(out);
    if (st != LGS_OK) return st;
    if (g->n == 0) return LGS_OK;
    if (!g->means || !g->scales || !g->quats || !g->opacities || !g->sh) return LGS_ERR_ARG;
    if (!aligned16(g->quats)) return LGS_ERR_ALIGN;
    if ((g->sh_degree == 1 || g->sh_degree == 3) && !aligned16(g->sh)) return LGS_ERR_ALIGN;
    PreParams p;
    p.means = g->means; p.scales = g->scales; p.quats = g->quats; p.opac = g->opacities;
    p.sh = g->sh; p.n = g->n;
    p.xy = out->xy; p.conic = out->conic; p.rgb = out->rgb; p.depth = out->depth;
    p.radius = out->radius; p.tiles = out->tiles; p.rect = out->rect; p.flags = out->flags;
    p.emit = reinterpret_cast<uint4*>(out->emit);
    p.status = d_status;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 block(256), grid((unsigned)((p.n + 255) / 256));
    switch (g->sh_degree) {
        case 0: preprocess_kernel<0><<<grid, block, 0, s>>>(p, vs); break;
        case 1: preprocess_kernel<1><<<grid, block, 0, s>>>(p, vs); break;
        case 2: preprocess_kernel<2><<<grid, block, 0, s>>>(p, vs); break;
        default: preprocess_kernel<3><<<grid, block, 0, s>>>(p, vs); break;
    }
    return cuda_status(cudaGetLastError());
}
