// backward.cu -- adjoint of the render and preprocess stages (the paper covers
// inference only; this is the reverse-mode derivative of the same forward map,
// for L = <dL/drgb, rgb> + <dL/dT, final_T>).
//
// render_bwd_localgs: one CTA per tile, the tile list walked back to front from
// the largest contributor count in the tile. Gaussians are staged and hoisted
// exactly as in the forward kernel (same V, same warp mask, same FP32
// arithmetic), so every alpha >= 1/255 decision is reproduced bit for bit. Each
// warp compacts its list of the batch (set mask bits up to its largest
// contributor count) and walks it back to front; a lane takes part for list
// positions <= its stored n_contrib, the others get alpha 0 (branch-free), and
// a warp with no contributing lane skips the reduction after one vote. Per pixel the
// transmittance before each Gaussian is recovered as T / (1 - alpha) from the
// stored final T, and
//   dL/drgb_k  = alpha_k T_k g
//   dL/dalpha_k = T_k <rgb_k - A_k, g> - T_f (<bg, g> + gT) / (1 - alpha_k)
// with A_k the colour behind k normalised by T_{k+1} (A <- alpha rgb + (1-alpha) A).
// Since ln(alpha) = V . B_local (hoist transform), dL/dV = (dL/dalpha alpha) B_local:
// six hoisted gradients plus three colour gradients per pair. The sums over
// the warp's 32 pixels are deferred: each lane leaves dp = dL/dalpha alpha and
// w = alpha T of its pixel in a row of a per-warp buffer, and every 8 rows the
// lanes reduce the buffer with one Gaussian per lane group and one pixel row
// per lane (the monomials of B_local are constants of the lane's row), so a
// pair costs two shared stores instead of a 9-value shuffle reduction. The
// per-warp sums meet over the CTA's 8 warps in shared-memory atomics and are
// mapped once per (Gaussian, tile) through the transpose of the hoist Jacobian
// to dL/d(a, b, c, o, u, v) before one global atomic per component.
//
// preprocess_bwd: one thread per Gaussian looping over the views, chain rule
// through conic inversion (dL/dSigma' = -Q dL/dQ Q), Sigma' = M M^T + 0.3 I with
// M = J W R diag(s), the EWA Jacobian J(t) (zero slope in a clamped direction
// ratio), the projected mean, quaternion normalisation and the SH colour
// (Cartesian basis polynomials, gradient projected onto the unit sphere).
#include "common.cuh"
#include "host.h"

namespace lgs {

// Gaussians staged per round of the adjoint: 128 and 256 measured within
// 0.5 % of each other (128 ahead), 128 halves the staging arrays.
#ifndef LGS_BWD_BATCH
#define LGS_BWD_BATCH 128
#endif
constexpr int BWD_BATCH = LGS_BWD_BATCH;
constexpr float LOG2E_B = 1.4426950408889634f;
constexpr float LOG2_ALPHA_MIN_B = -7.9943534368588580f;

struct BwdParams {
    const float4* xy;
    const float4* conic;
    const float4* rgb;
    const uint32_t* vals;
    const uint2* ranges;
    const float* final_T;
    const uint32_t* n_contrib;
    const float* dL_drgb;
    const float* dL_dT;
    float* g_xy;      // [M,2]
    float* g_conic;   // [M,4]
    float* g_rgb;     // [M,4] (r, g, b, unused), 16-B rows
    int64_t* status;
};

__device__ __forceinline__ float ex2_approx_b(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sum of v[0..7] over the warp: lane L ends up holding the total of value
// ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1), i.e. lanes 4i..4i+3
// hold value i. Each halving step exchanges only the half a lane gives away.
__device__ __forceinline__ float warp_sum8_transposed(float v[8]) {
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h16 ? v[i] : v[i + 4];
        const float keep = h16 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float b2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h8 ? a[i] : a[i + 2];
        const float keep = h8 ? a[i + 2] : a[i];
        b2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const float send = h4 ? b2[0] : b2[1];
    float c1 = (h4 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    c1 += __shfl_xor_sync(0xffffffffu, c1, 2);
    c1 += __shfl_xor_sync(0xffffffffu, c1, 1);
    return c1;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Per-warp buffer of the deferred reduction: up to RED_ROWS rows, one per
// Gaussian of the warp's list. Row r holds, per lane, (-dp of its first pixel,
// -dp of its second pixel (0 with one pixel per lane), -W_r, -W_g) in R4 and
// -W_b in R1, where dp = dL/dalpha alpha of a pixel and W_c = sum over the
// lane's pixels of w g_c (w = alpha T, g = dL/drgb); the walk produces them
// negated, and the reduction negates its sums back. Lane c of row r is stored at
// column c ^ (r & 7), so that the row writes of the walk (one row, 32 lanes)
// and the reads of the reduction (8 rows, 8 lanes each) hit distinct banks.
constexpr int RED_ROWS = 8;
struct __align__(16) BwdRed {
    float4 R4[RED_ROWS][32];
    float R1[RED_ROWS][32];
    uint32_t slot[RED_ROWS];   // batch index of the row's Gaussian
};

// The three 16-B records of a staged Gaussian sit at the same byte offset in
// sV, sDE and sC; a warp's list holds that offset.
template <int NW>
struct BwdSmem {
    float4 sV[BWD_BATCH];        // (A, B, C, F), log2 domain
    float4 sDE[BWD_BATCH];       // (D, E, -, -)
    float4 sC[BWD_BATCH];        // (r, g, b, list position + 1 as bits)
    uint8_t sM[BWD_BATCH];       // warp-block mask
    uint16_t sL[NW][BWD_BATCH];  // per warp: byte offsets (16 x batch index) of its set mask bits
    uint32_t sId[BWD_BATCH];
    float sG[BWD_BATCH][9];      // per staged Gaussian: A, B, C, D, E, r, g, F, b gradients
    uint32_t sLast[NW];
    BwdRed red[NW];
};

// Reduces rows 0..ns-1 of a warp's buffer into sG. Lane (e, q) = (lane % 8,
// lane / 8) sums row e over the records of lanes 8q..8q+7, which own 8
// consecutive pixel columns of one pixel row (the block width is a multiple
// of 8): with offsets u = i - 3.5 from the group's centre column xc and the
// group's rows y_k, the sums S0 = sum dp, S1 = sum dp u, S2 = sum dp u^2 of
// each row k give the six hoisted moments (x'^2 -> xc^2 S0 + 2 xc S1 + S2,
// x'y' -> y_k (xc S0 + S1), y'^2 -> y_k^2 S0, x' -> xc S0 + S1, y' -> y_k S0,
// 1 -> S0); two shuffle levels add the four groups of a row and lanes 0..ns-1
// hold the warp's sums.
template <int TW, int TH, int WX, int WY>
__device__ __forceinline__ void reduce_rows(const BwdRed& R, int ns, float (*sG)[9], int lane, int warp) {
    using Lay = Layout<TW, TH, WX, WY>;
    constexpr int PPL = Lay::PPL;
    static_assert(WX % 8 == 0, "lane groups of 8 pixel columns");
    const int e = lane & 7, q = lane >> 3;
    const int bx = warp % Lay::NBX, by = warp / Lay::NBX;
    const float xc = (float)(bx * WX + (8 * q) % WX) + 3.5f - 0.5f * (TW - 1);
    float yk[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) yk[k] = (float)(by * WY + (8 * q) / WX + k * (WY / 2)) - 0.5f * (TH - 1);
    using P = Px<PPL>;
    float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (e < ns) {
        // per pixel row k of the lane's pixels (packed two-wide when PPL = 2)
        P S0 = bcast<PPL>(0.f), S1 = S0, S2 = S0;
        float2 W01 = make_float2(0.f, 0.f);
        float W2 = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int col = 8 * q + (i ^ e);
            const float4 r4 = R.R4[e][col];
            const float w2 = R.R1[e][col];
            const float u = (float)i - 3.5f;
            P dp;
            dp[0] = r4.x;
            if (PPL == 2) dp[PPL - 1] = r4.y;
            S0 = padd(S0, dp);
            S1 = pfma(dp, bcast<PPL>(u), S1);
            S2 = pfma(dp, bcast<PPL>(u * u), S2);
            W01 = __fadd2_rn(W01, make_float2(r4.z, r4.w));
            W2 += w2;
        }
        const float W0 = W01.x, W1 = W01.y;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const float Sx = fmaf(xc, S0[k], S1[k]);
            v[0] += fmaf(xc, fmaf(xc, S0[k], 2.f * S1[k]), S2[k]);
            v[1] = fmaf(yk[k], Sx, v[1]);
            v[2] = fmaf(yk[k] * yk[k], S0[k], v[2]);
            v[3] += Sx;
            v[4] = fmaf(yk[k], S0[k], v[4]);
            v[7] += S0[k];
        }
        v[5] = W0;
        v[6] = W1;
        v[8] = W2;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 8);
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 16);
    }
    if (q == 0 && e < ns) {
        // the buffer holds -dp and -w g: the sums are negated back here
        float* dst = sG[R.slot[e]];
#pragma unroll
        for (int k = 0; k < 9; ++k) atomicAdd(dst + k, -v[k]);
    }
}

// The adjoint of one tile in a warp-block layout (see Layout): every thread of
// the CTA calls it with the same tile. Per lane, PPL pixels; their per-pixel
// arithmetic runs packed two-wide when PPL = 2.
template <int TW, int TH, int WX, int WY>
__device__ __forceinline__ void bwd_tile(const BwdParams& p, const Views& vs, uint32_t work,
                                         BwdSmem<TileLayout<TW, TH, WX, WY>::NW>& S) {
    using Reg = Regions<TW, TH>;
    constexpr int CW = Reg::CW, CH = Reg::CH;
    using Lay = Layout<CW, CH, WX, WY>;
    constexpr int PPL = Lay::PPL, NT = Lay::NT, NW = Lay::NW;
    using P = Px<PPL>;
    // work item = tile * (regions per tile) + region; the region (CW x CH
    // pixels at X0, Y0) walks the whole list of its tile
    const uint32_t tile = work / (uint32_t)Reg::N, reg = work % (uint32_t)Reg::N;
    const int view = view_of_tile(vs, tile);
    const ViewRec& c = vs.v[view];
    const uint32_t lt = tile - c.tile_off;
    const int X0 = (int)(lt % (uint32_t)c.gx) * TW + (int)(reg % Reg::NX) * CW;
    const int Y0 = (int)(lt / (uint32_t)c.gx) * TH + (int)(reg / Reg::NX) * CH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float Ox = (float)X0 + 0.5f * (CW - 1), Oy = (float)Y0 + 0.5f * (CH - 1);
    const int lx = (warp % Lay::NBX) * WX + lane % WX;
    uint2 r = p.ranges[tile];
    if (!LGS_CHECK(r.x <= r.y && (r.y == r.x || (int64_t)r.y <= p.status[LGS_ST_NUM_INSTANCES]), 21, p.status))
        r.y = r.x;

    // carried negated (-<A, g>, -tail) so that the packed updates below need
    // no separate negations
    P bx2, bxy, by2, bxl, byl, T, g0, g1, g2, ntail, nAg;
    uint32_t last[PPL];
    uint32_t mylast = 0;
    const int64_t plane = (int64_t)c.W * c.H;
    const float* gr = p.dL_drgb + 3 * (int64_t)c.pix_off;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int ly = (warp / Lay::NBX) * WY + lane / WX + k * (WY / 2);
        const int px = X0 + lx, py = Y0 + ly;
        const float xl = (float)lx - 0.5f * (CW - 1), yl = (float)ly - 0.5f * (CH - 1);
        bx2[k] = xl * xl;
        bxy[k] = xl * yl;
        by2[k] = yl * yl;
        bxl[k] = xl;
        byl[k] = yl;
        T[k] = 1.f;
        g0[k] = g1[k] = g2[k] = ntail[k] = nAg[k] = 0.f;
        last[k] = 0;
        if (px < c.W && py < c.H) {
            const int64_t pix = (int64_t)py * c.W + px;
            g0[k] = gr[pix];
            g1[k] = gr[plane + pix];
            g2[k] = gr[2 * plane + pix];
            T[k] = p.final_T[c.pix_off + pix];
            last[k] = p.n_contrib[c.pix_off + pix];
            const float gT = p.dL_dT ? p.dL_dT[c.pix_off + pix] : 0.f;
            ntail[k] = -(T[k] * (c.bg[0] * g0[k] + c.bg[1] * g1[k] + c.bg[2] * g2[k] + gT));
        }
        mylast = max(mylast, last[k]);
    }
    BwdRed& R = S.red[warp];
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, mylast);
    if (lane == 0) S.sLast[warp] = wlast;
    __syncthreads();
    uint32_t tlast = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) tlast = max(tlast, S.sLast[w]);
    if (!LGS_CHECK(tlast <= r.y - r.x, 22, p.status)) tlast = r.y - r.x;

    for (int end = (int)tlast; end > 0; end -= BWD_BATCH) {
        const int begin = max(0, end - BWD_BATCH);
        const int nb = end - begin;
        __syncthreads();
        for (int sl = threadIdx.x; sl < nb; sl += NT) {
            const uint32_t pos = (uint32_t)(begin + sl);
            const uint32_t id = p.vals[r.x + pos];
            const float4 xy = p.xy[id];
            const float4 co = p.conic[id];
            const float4 col = p.rgb[id];
            const float dx = __fadd_rn(xy.x - Ox, xy.z);
            const float dy = __fadd_rn(xy.y - Oy, xy.w);
            const float Dn = fmaf(co.x, dx, co.y * dy);
            const float En = fmaf(co.y, dx, co.z * dy);
            const float Fn = -0.5f * fmaf(dx, Dn, dy * En);
            S.sV[sl] = make_float4(-0.5f * LOG2E_B * co.x, -LOG2E_B * co.y, -0.5f * LOG2E_B * co.z,
                                   fmaf(Fn, LOG2E_B, __log2f(co.w)));
            S.sDE[sl] = make_float4(Dn * LOG2E_B, En * LOG2E_B, 0.f, 0.f);
            S.sC[sl] = make_float4(col.x, col.y, col.z, __uint_as_float(pos + 1u));
            S.sM[sl] = (uint8_t)block_mask<CW, CH, WX, WY>(co.x, co.y, co.z, co.w, __fadd_rn(xy.x, xy.z),
                                                           __fadd_rn(xy.y, xy.w), X0, Y0);
            S.sId[sl] = id;
#pragma unroll
            for (int k = 0; k < 9; ++k) S.sG[sl][k] = 0.f;
        }
        __syncthreads();
        if (wlast > (uint32_t)begin) {
            // the warp's list of the batch (set mask bits up to its last
            // contributor), compacted in order and walked back to front
            uint16_t* sLw = S.sL[warp];
            int nl = 0;
            for (int c0 = 0; c0 < nb; c0 += 32) {
                const int jj = c0 + lane;
                const bool hit = jj < nb && ((S.sM[jj] >> warp) & 1u) && (uint32_t)(begin + jj) < wlast;
                const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                if (hit) sLw[nl + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(16 * jj);
                nl += __popc(bal);
            }
            __syncwarp();
            int ns = 0;   // rows of the warp's buffer in use
            // The T-independent front of a step (record loads, exponent,
            // alpha, 1/(1 - alpha), the contribution predicates) of list
            // entry i; the walk takes entries two at a time so that the front
            // of the second overlaps the dependent updates of the first.
            struct Front {
                float4 col;
                P nal, inv;
                bool contrib[PPL], clamp[PPL];
                int off;
                bool any;
            };
            auto front = [&](int i) {
                Front f;
                f.off = sLw[i];
                const float4 V = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(S.sV) + f.off);
                const float4 DE = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(S.sDE) + f.off);
                f.col = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(S.sC) + f.off);
                const uint32_t pos = __float_as_uint(f.col.w);
                const P pw = pfma(bcast<PPL>(V.x), bx2, pfma(bcast<PPL>(V.y), bxy, pfma(bcast<PPL>(V.z), by2,
                             pfma(bcast<PPL>(DE.x), bxl, pfma(bcast<PPL>(DE.y), byl, bcast<PPL>(V.w))))));
                f.any = false;
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    f.contrib[k] = pos <= last[k] && pw[k] >= LOG2_ALPHA_MIN_B;
                    f.any = f.any || f.contrib[k];
                    // branch-free: pixels that do not contribute get alpha 0,
                    // which leaves T and the colour behind exactly as they
                    // were. Carried negated: nal = -alpha
                    const float e2 = ex2_approx_b(pw[k]);
                    f.clamp[k] = e2 > 0.99f;
                    const float nal = fmaxf(-0.99f, -e2);
                    f.inv[k] = __fdividef(1.f, 1.f + nal);  // 1 - alpha >= 0.01
                    f.nal[k] = nal;
                }
                return f;
            };
            auto apply = [&](const Front& f) {
                P nac;
#pragma unroll
                for (int k = 0; k < PPL; ++k) nac[k] = f.contrib[k] ? f.nal[k] : 0.f;
                const P Tk = pmul(T, f.inv);
                const P nw = pmul(nac, Tk);                  // -w = -alpha T
                // <rgb_k - A_k, g>, and A <- alpha rgb + (1 - alpha) A carried as -<A, g>
                const P cg = pfma(bcast<PPL>(f.col.z), g2, pfma(bcast<PPL>(f.col.y), g1,
                                                                 pfma(bcast<PPL>(f.col.x), g0, nAg)));
                const P dal = pfma(ntail, f.inv, pmul(Tk, cg));  // dL/dalpha
                nAg = pfma(nac, cg, nAg);
                const P ndal = pmul(dal, f.nal);             // -dL/dalpha alpha
                float ndp[2] = {0.f, 0.f};
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    T[k] = f.contrib[k] ? Tk[k] : T[k];
                    ndp[k] = (f.contrib[k] && !f.clamp[k]) ? ndal[k] : 0.f;
                }
                // the lane's colour sums over its pixels (negated, like dp)
                const P wg0 = pmul(nw, g0), wg1 = pmul(nw, g1), wg2 = pmul(nw, g2);
                float W0 = wg0[0], W1 = wg1[0], W2 = wg2[0];
                if (PPL == 2) {
                    W0 += wg0[PPL - 1];
                    W1 += wg1[PPL - 1];
                    W2 += wg2[PPL - 1];
                }
                const int cc = lane ^ (ns & 7);
                R.R4[ns][cc] = make_float4(ndp[0], ndp[1], W0, W1);
                R.R1[ns][cc] = W2;
                if (lane == 0) R.slot[ns] = (uint32_t)(f.off >> 4);
                if (++ns == RED_ROWS) {
                    __syncwarp();
                    reduce_rows<CW, CH, WX, WY>(R, ns, S.sG, lane, warp);
                    __syncwarp();
                    ns = 0;
                }
            };
#pragma unroll 1
            for (int i = nl - 1; i >= 1; i -= 2) {
                const Front fa = front(i);
                const Front fb = front(i - 1);
                if (__any_sync(0xffffffffu, fa.any)) apply(fa);   // else nothing to reduce
                if (__any_sync(0xffffffffu, fb.any)) apply(fb);
            }
            if (nl & 1) {
                const Front fa = front(0);
                if (__any_sync(0xffffffffu, fa.any)) apply(fa);
            }
            if (ns > 0) {
                __syncwarp();
                reduce_rows<CW, CH, WX, WY>(R, ns, S.sG, lane, warp);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nb; t += NT) {
            // hoisted gradients (A, B, C, D, E, F in natural-log units) -> (a, b, c, ln o, Dx, Dy)
            const float gA = S.sG[t][0], gB = S.sG[t][1], gC = S.sG[t][2], gD = S.sG[t][3], gE = S.sG[t][4];
            const float gF = S.sG[t][7];
            const uint32_t id = S.sId[t];
            const float4 xy = p.xy[id];
            const float4 co = p.conic[id];
            const float dx = __fadd_rn(xy.x - Ox, xy.z);
            const float dy = __fadd_rn(xy.y - Oy, xy.w);
            const float Dn = fmaf(co.x, dx, co.y * dy);
            const float En = fmaf(co.y, dx, co.z * dy);
            const float ga = -0.5f * gA + dx * gD - 0.5f * dx * dx * gF;
            const float gbb = -gB + dy * gD + dx * gE - dx * dy * gF;
            const float gc = -0.5f * gC + dy * gE - 0.5f * dy * dy * gF;
            const float go = gF / co.w;
            const float gdx = co.x * gD + co.y * gE - Dn * gF;
            const float gdy = co.y * gD + co.z * gE - En * gF;
            if (ga != 0.f || gbb != 0.f || gc != 0.f || go != 0.f || gdx != 0.f || gdy != 0.f) {
                // one vector atomic per record (conic2d rows 16-B, xy2d rows
                // 8-B aligned, checked on the host)
                atomicAdd(reinterpret_cast<float4*>(p.g_conic) + id, make_float4(ga, gbb, gc, go));
                atomicAdd(reinterpret_cast<float2*>(p.g_xy) + id, make_float2(gdx, gdy));
            }
            const float gr0 = S.sG[t][5], gr1 = S.sG[t][6], gr2 = S.sG[t][8];
            if (gr0 != 0.f || gr1 != 0.f || gr2 != 0.f) {
                atomicAdd(reinterpret_cast<float4*>(p.g_rgb) + id, make_float4(gr0, gr1, gr2, 0.f));
            }
        }
    }
}

// One CTA per (tile, region) (shared memory: the dynamic allocation of the launch).
// Five CTAs per SM: the register bound this sets (at most 102 per thread for
// 128-thread CTAs) measured faster than the unbounded allocation (112, four
// CTAs) and than six or eight CTAs with 128-Gaussian batches.
#ifndef LGS_BWD_MIN_BLOCKS
#define LGS_BWD_MIN_BLOCKS 5
#endif
template <int TW, int TH, int WX, int WY>
__global__ void __launch_bounds__(TileLayout<TW, TH, WX, WY>::NT, LGS_BWD_MIN_BLOCKS) render_bwd_localgs(BwdParams p,
                                                                                                     Views vs) {
    extern __shared__ __align__(16) unsigned char bwd_smem[];
    auto& S = *reinterpret_cast<BwdSmem<TileLayout<TW, TH, WX, WY>::NW>*>(bwd_smem);
    bwd_tile<TW, TH, WX, WY>(p, vs, blockIdx.x, S);
}

// Persistent CTAs: each pulls the next (tile, region) work item from the
// work-queue counter LGS_ST_QUEUE_BWD (zeroed by the launcher) until all are
// taken.
template <int TW, int TH, int WX, int WY>
__global__ void __launch_bounds__(TileLayout<TW, TH, WX, WY>::NT, LGS_BWD_MIN_BLOCKS)
    render_bwd_localgs_persistent(BwdParams p, Views vs) {
    extern __shared__ __align__(16) unsigned char bwd_smem[];
    auto& S = *reinterpret_cast<BwdSmem<TileLayout<TW, TH, WX, WY>::NW>*>(bwd_smem);
    __shared__ uint32_t s_work;
    unsigned long long* q = reinterpret_cast<unsigned long long*>(p.status + LGS_ST_QUEUE_BWD);
    const uint32_t n_work = vs.n_tiles * (uint32_t)Regions<TW, TH>::N;
    for (;;) {
        if (threadIdx.x == 0) s_work = (uint32_t)atomicAdd(q, 1ull);
        __syncthreads();
        const uint32_t work = s_work;
        __syncthreads();
        if (work >= n_work) break;
        bwd_tile<TW, TH, WX, WY>(p, vs, work, S);
        __syncthreads();
    }
}

// Plain counterpart (comparison baseline): the plain forward's per-pixel
// global-coordinate arithmetic and branches (power > 0 and alpha < 1/255
// skipped, alpha = min(0.99, o exp(power))), every warp walking every Gaussian
// of the tile list up to its largest contributor count (no warp mask, no
// hoisting), gradients taken directly in (a, b, c, u, v, o, rgb) and reduced
// with the same warp/CTA machinery as the Local-GS adjoint.
template <int TW, int TH>
__global__ void __launch_bounds__(256) render_bwd_plain(BwdParams p, Views vs) {
    __shared__ float4 sXY[BWD_BATCH];
    __shared__ float4 sCO[BWD_BATCH];
    __shared__ float4 sC[BWD_BATCH];
    __shared__ uint32_t sId[BWD_BATCH];
    __shared__ float sG[BWD_BATCH][9];
    __shared__ uint32_t sLast[8];

    const uint32_t tile = blockIdx.x;
    const int view = view_of_tile(vs, tile);
    const ViewRec& c = vs.v[view];
    const uint32_t lt = tile - c.tile_off;
    const int X0 = (int)(lt % (uint32_t)c.gx) * TW, Y0 = (int)(lt / (uint32_t)c.gx) * TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = X0 + lane % TW, py = Y0 + warp * (TH / 8) + lane / TW;
    const bool inside = px < c.W && py < c.H;
    const float pxf = (float)px, pyf = (float)py;
    uint2 r = p.ranges[tile];
    if (!LGS_CHECK(r.x <= r.y && (r.y == r.x || (int64_t)r.y <= p.status[LGS_ST_NUM_INSTANCES]), 21, p.status))
        r.y = r.x;

    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, tail = 0.f;
    uint32_t last = 0;
    if (inside) {
        const int64_t plane = (int64_t)c.W * c.H;
        const int64_t pix = (int64_t)py * c.W + px;
        const float* gr = p.dL_drgb + 3 * (int64_t)c.pix_off;
        g0 = gr[pix];
        g1 = gr[plane + pix];
        g2 = gr[2 * plane + pix];
        T = p.final_T[c.pix_off + pix];
        last = p.n_contrib[c.pix_off + pix];
        const float gT = p.dL_dT ? p.dL_dT[c.pix_off + pix] : 0.f;
        tail = T * (c.bg[0] * g0 + c.bg[1] * g1 + c.bg[2] * g2 + gT);
    }
    float A0 = 0.f, A1 = 0.f, A2 = 0.f;
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0) sLast[warp] = wlast;
    __syncthreads();
    uint32_t tlast = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) tlast = max(tlast, sLast[w]);
    if (!LGS_CHECK(tlast <= r.y - r.x, 22, p.status)) tlast = r.y - r.x;

    for (int end = (int)tlast; end > 0; end -= BWD_BATCH) {
        const int begin = max(0, end - BWD_BATCH);
        const int nb = end - begin;
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const uint32_t pos = (uint32_t)(begin + threadIdx.x);
            const uint32_t id = p.vals[r.x + pos];
            sXY[threadIdx.x] = p.xy[id];
            sCO[threadIdx.x] = p.conic[id];
            const float4 col = p.rgb[id];
            sC[threadIdx.x] = make_float4(col.x, col.y, col.z, __uint_as_float(pos + 1u));
            sId[threadIdx.x] = id;
#pragma unroll
            for (int k = 0; k < 9; ++k) sG[threadIdx.x][k] = 0.f;
        }
        __syncthreads();
        for (int g = min(nb, (int)wlast - begin) - 1; g >= 0; --g) {
            const float4 col = sC[g];
            const uint32_t pos = __float_as_uint(col.w);
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.f;
            float gb = 0.f;
            const float4 xy = sXY[g];
            const float4 co = sCO[g];
            const float dx = __fadd_rn(xy.x - pxf, xy.z);
            const float dy = __fadd_rn(xy.y - pyf, xy.w);
            const float power = plain_power(co, dx, dy);
            const float G = __expf(power);
            const float alpha = fminf(0.99f, co.w * G);
            const bool contrib = pos <= last && power <= 0.f && alpha >= 1.f / 255.f;
            if (!__any_sync(0xffffffffu, contrib)) continue;           // nothing to reduce
            if (contrib) {
                {
                    {
                        const float inv = __fdividef(1.f, 1.f - alpha);
                        const float Tk = T * inv;
                        const float w = alpha * Tk;
                        v[6] = w * g0;
                        v[7] = w * g1;
                        gb = w * g2;
                        const float cg = (col.x - A0) * g0 + (col.y - A1) * g1 + (col.z - A2) * g2;
                        const float dal = Tk * cg - tail * inv;
                        A0 = fmaf(alpha, col.x - A0, A0);
                        A1 = fmaf(alpha, col.y - A1, A1);
                        A2 = fmaf(alpha, col.z - A2, A2);
                        T = Tk;
                        if (co.w * G <= 0.99f) {
                            const float dpw = dal * alpha;          // dL/dpower
                            v[0] = -0.5f * dpw * dx * dx;           // a
                            v[1] = -dpw * dx * dy;                  // b
                            v[2] = -0.5f * dpw * dy * dy;           // c
                            v[3] = -dpw * (co.x * dx + co.y * dy);  // u
                            v[4] = -dpw * (co.y * dx + co.z * dy);  // v
                            v[5] = dal * G;                         // o
                        }
                    }
                }
            }
            const float s8 = warp_sum8_transposed(v);
            const float s9 = warp_sum(gb);
            if ((lane & 3) == 0) atomicAdd(&sG[g][lane >> 2], s8);
            if (lane == 0) atomicAdd(&sG[g][8], s9);
        }
        __syncthreads();
        if ((int)threadIdx.x < nb) {
            const int t = threadIdx.x;
            const uint32_t id = sId[t];
            if (sG[t][0] != 0.f || sG[t][1] != 0.f || sG[t][2] != 0.f || sG[t][5] != 0.f) {
                atomicAdd(p.g_conic + 4 * (int64_t)id + 0, sG[t][0]);
                atomicAdd(p.g_conic + 4 * (int64_t)id + 1, sG[t][1]);
                atomicAdd(p.g_conic + 4 * (int64_t)id + 2, sG[t][2]);
                atomicAdd(p.g_conic + 4 * (int64_t)id + 3, sG[t][5]);
                atomicAdd(p.g_xy + 2 * (int64_t)id + 0, sG[t][3]);
                atomicAdd(p.g_xy + 2 * (int64_t)id + 1, sG[t][4]);
            }
            if (sG[t][6] != 0.f || sG[t][7] != 0.f || sG[t][8] != 0.f) {
                atomicAdd(p.g_rgb + 4 * (int64_t)id + 0, sG[t][6]);
                atomicAdd(p.g_rgb + 4 * (int64_t)id + 1, sG[t][7]);
                atomicAdd(p.g_rgb + 4 * (int64_t)id + 2, sG[t][8]);
            }
        }
    }
}

// ------------------------------------------------------------------ preprocess adjoint
struct PreBwdParams {
    const float* means;
    const float* scales;
    const float* quats;
    const float* sh;
    int64_t n;
    const float4* conic;   // forward conic (a, b, c, o)
    const uint32_t* tiles;
    const uint8_t* flags;
    const float* g_xy;
    const float* g_conic;
    const float* g_rgb;
    float* d_means;
    float* d_scales;
    float* d_quats;
    float* d_opac;
    float* d_sh;
};

// Basis value and Cartesian gradient of the real SH polynomials (Condon-Shortley
// phase, index l^2 + l + m) at a unit direction.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float (*dY)[3]) {
    constexpr float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    Y[0] = C0; dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (DEG >= 1) {
        Y[1] = -C1 * y; dY[1][0] = 0.f; dY[1][1] = -C1; dY[1][2] = 0.f;
        Y[2] = C1 * z;  dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = C1;
        Y[3] = -C1 * x; dY[3][0] = -C1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    }
    if (DEG >= 2) {
        constexpr float a = 1.0925484305920792f, b = 0.31539156525252005f, e = 0.5462742152960396f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = a * x * y;   dY[4][0] = a * y;  dY[4][1] = a * x;  dY[4][2] = 0.f;
        Y[5] = -a * y * z;  dY[5][0] = 0.f;    dY[5][1] = -a * z; dY[5][2] = -a * y;
        Y[6] = b * (2.f * zz - xx - yy); dY[6][0] = -2.f * b * x; dY[6][1] = -2.f * b * y; dY[6][2] = 4.f * b * z;
        Y[7] = -a * x * z;  dY[7][0] = -a * z; dY[7][1] = 0.f;    dY[7][2] = -a * x;
        Y[8] = e * (xx - yy); dY[8][0] = 2.f * e * x; dY[8][1] = -2.f * e * y; dY[8][2] = 0.f;
    }
    if (DEG >= 3) {
        constexpr float c1 = -0.5900435899266435f, c2 = 2.890611442640554f, c3 = -0.4570457994644658f,
                        c4 = 0.3731763325901154f, c6 = 1.445305721320277f;
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[9] = c1 * y * (3.f * xx - yy);
        dY[9][0] = 6.f * c1 * x * y; dY[9][1] = c1 * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
        Y[10] = c2 * x * y * z;
        dY[10][0] = c2 * y * z; dY[10][1] = c2 * x * z; dY[10][2] = c2 * x * y;
        Y[11] = c3 * y * (4.f * zz - xx - yy);
        dY[11][0] = -2.f * c3 * x * y; dY[11][1] = c3 * (4.f * zz - xx - 3.f * yy); dY[11][2] = 8.f * c3 * y * z;
        Y[12] = c4 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        dY[12][0] = -6.f * c4 * x * z; dY[12][1] = -6.f * c4 * y * z; dY[12][2] = c4 * (6.f * zz - 3.f * xx - 3.f * yy);
        Y[13] = c3 * x * (4.f * zz - xx - yy);
        dY[13][0] = c3 * (4.f * zz - 3.f * xx - yy); dY[13][1] = -2.f * c3 * x * y; dY[13][2] = 8.f * c3 * x * z;
        Y[14] = c6 * z * (xx - yy);
        dY[14][0] = 2.f * c6 * x * z; dY[14][1] = -2.f * c6 * y * z; dY[14][2] = c6 * (xx - yy);
        Y[15] = c1 * x * (xx - 3.f * yy);
        dY[15][0] = c1 * (3.f * xx - 3.f * yy); dY[15][1] = -6.f * c1 * x * y; dY[15][2] = 0.f;
    }
}

// Four CTAs per SM (at most 128 registers, no spills): 20 % faster than the
// unbounded allocation (167 registers, three CTAs); five would spill.
#ifndef LGS_PREBWD_MIN_BLOCKS
#define LGS_PREBWD_MIN_BLOCKS 4
#endif
template <int DEG>
__global__ void __launch_bounds__(128, LGS_PREBWD_MIN_BLOCKS) preprocess_bwd(PreBwdParams p, Views vs) {
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t N = p.n;
    const float mx = p.means[3 * i], my = p.means[3 * i + 1], mz = p.means[3 * i + 2];
    const float s[3] = {p.scales[3 * i], p.scales[3 * i + 1], p.scales[3 * i + 2]};
    const float4 q4 = reinterpret_cast<const float4*>(p.quats)[i];
    const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x / qn, x = q4.y / qn, y = q4.z / qn, z = q4.w / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float dmu[3] = {0.f, 0.f, 0.f}, dRS[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float dop = 0.f;
    float dsh[NK * 3];
#pragma unroll
    for (int k = 0; k < NK * 3; ++k) dsh[k] = 0.f;
    bool any = false;

    // the next view's tile count is loaded one view ahead
    uint32_t tiles_next = p.tiles[i];
    for (int v = 0; v < vs.n; ++v) {
        const int64_t m = (int64_t)v * N + i;
        const uint32_t tiles_v = tiles_next;
        if (v + 1 < vs.n) tiles_next = p.tiles[m + N];
        if (tiles_v == 0) continue;
        any = true;
        const ViewRec& c = vs.v[v];
        // the per-entry scratch gradients: xy2d rows 8-B aligned, conic2d and
        // rgb2d rows 16-B aligned (checked on the host)
        const float2 gxy = reinterpret_cast<const float2*>(p.g_xy)[m];
        const float4 gco = reinterpret_cast<const float4*>(p.g_conic)[m];
        const float4 grgb = reinterpret_cast<const float4*>(p.g_rgb)[m];
        const float gu = gxy.x, gv = gxy.y;
        const float ga = gco.x, gbq = gco.y, gc = gco.z;
        dop += gco.w;
        const uint8_t fl = p.flags[m];
        // ---- colour
        {
            // a channel clamped at 0 in the forward passes no gradient
            const float gm[3] = {(fl & 1u) ? 0.f : grgb.x, (fl & 2u) ? 0.f : grgb.y, (fl & 4u) ? 0.f : grgb.z};
            float d0 = mx - c.campos[0], d1 = my - c.campos[1], d2 = mz - c.campos[2];
            const float dn = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            const float id = 1.f / dn;
            d0 *= id; d1 *= id; d2 *= id;
            float Y[NK], dY[NK][3];
            sh_basis_grad<DEG>(d0, d1, d2, Y, dY);
            float gd[3] = {0.f, 0.f, 0.f};
            const float* shp = p.sh + i * NK * 3;
            // coefficient k: dL/dsh_k = Y_k g (masked), and its colour
            // <sh_k, g> times dY_k/d(dir) into the direction gradient
            auto coef = [&](int k, float s0, float s1, float s2) {
                dsh[k * 3 + 0] += Y[k] * gm[0];
                dsh[k * 3 + 1] += Y[k] * gm[1];
                dsh[k * 3 + 2] += Y[k] * gm[2];
                const float ck = s0 * gm[0] + s1 * gm[1] + s2 * gm[2];
                gd[0] += ck * dY[k][0];
                gd[1] += ck * dY[k][1];
                gd[2] += ck * dY[k][2];
            };
            if constexpr (NK % 4 == 0) {
                // four coefficients (12 floats) per three 16-B loads
                const float4* s4 = reinterpret_cast<const float4*>(shp);
#pragma unroll
                for (int g4 = 0; g4 < NK / 4; ++g4) {
                    const float4 u0 = s4[3 * g4], u1 = s4[3 * g4 + 1], u2 = s4[3 * g4 + 2];
                    coef(4 * g4 + 0, u0.x, u0.y, u0.z);
                    coef(4 * g4 + 1, u0.w, u1.x, u1.y);
                    coef(4 * g4 + 2, u1.z, u1.w, u2.x);
                    coef(4 * g4 + 3, u2.y, u2.z, u2.w);
                }
            } else {
#pragma unroll
                for (int k = 0; k < NK; ++k) coef(k, shp[3 * k], shp[3 * k + 1], shp[3 * k + 2]);
            }
            const float pr = gd[0] * d0 + gd[1] * d1 + gd[2] * d2;
            dmu[0] += (gd[0] - d0 * pr) * id;
            dmu[1] += (gd[1] - d1 * pr) * id;
            dmu[2] += (gd[2] - d2 * pr) * id;
        }
        // ---- camera space and Jacobian
        const float tx = c.R[0] * mx + c.R[1] * my + c.R[2] * mz + c.t[0];
        const float ty = c.R[3] * mx + c.R[4] * my + c.R[5] * mz + c.t[1];
        const float tz = c.R[6] * mx + c.R[7] * my + c.R[8] * mz + c.t[2];
        const float iz = 1.f / tz;
        const float limx = 1.3f * (0.5f * (float)c.W / c.fx), limy = 1.3f * (0.5f * (float)c.H / c.fy);
        const float rx = fminf(limx, fmaxf(-limx, tx * iz)), ry = fminf(limy, fmaxf(-limy, ty * iz));
        const bool clx = (fl & 8) != 0, cly = (fl & 16) != 0;
        const float J00 = c.fx * iz, J02 = -c.fx * rx * iz, J11 = c.fy * iz, J12 = -c.fy * ry * iz;
        float RS[9], WRS[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) RS[r * 3 + k] = R[r * 3 + k] * s[k];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                WRS[r * 3 + k] = c.R[r * 3] * RS[k] + c.R[r * 3 + 1] * RS[3 + k] + c.R[r * 3 + 2] * RS[6 + k];
        float M0[3], M1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M0[k] = J00 * WRS[k] + J02 * WRS[6 + k];
            M1[k] = J11 * WRS[3 + k] + J12 * WRS[6 + k];
        }
        // ---- conic -> Sigma': dL/dSigma' = -Q G Q, G = [[ga, gb/2], [gb/2, gc]]
        const float4 co = p.conic[m];
        const float a = co.x, b = co.y, cc = co.z;
        const float hb = 0.5f * gbq;
        const float QG00 = a * ga + b * hb, QG01 = a * hb + b * gc;
        const float QG10 = b * ga + cc * hb, QG11 = b * hb + cc * gc;
        const float S00 = -(QG00 * a + QG01 * b);
        const float S01 = -(QG00 * b + QG01 * cc);
        const float S11 = -(QG10 * b + QG11 * cc);
        // Sigma' = M M^T + 0.3 I  ->  dL/dM = 2 S M
        float dM0[3], dM1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dM0[k] = 2.f * (S00 * M0[k] + S01 * M1[k]);
            dM1[k] = 2.f * (S01 * M0[k] + S11 * M1[k]);
        }
        // M = J WRS
        const float dJ00 = dM0[0] * WRS[0] + dM0[1] * WRS[1] + dM0[2] * WRS[2];
        const float dJ02 = dM0[0] * WRS[6] + dM0[1] * WRS[7] + dM0[2] * WRS[8];
        const float dJ11 = dM1[0] * WRS[3] + dM1[1] * WRS[4] + dM1[2] * WRS[5];
        const float dJ12 = dM1[0] * WRS[6] + dM1[1] * WRS[7] + dM1[2] * WRS[8];
        float dW[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dW[k] = J00 * dM0[k];
            dW[3 + k] = J11 * dM1[k];
            dW[6 + k] = J02 * dM0[k] + J12 * dM1[k];
        }
        // RS gradient through WRS = W RS
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                dRS[r * 3 + k] += c.R[r] * dW[k] + c.R[3 + r] * dW[3 + k] + c.R[6 + r] * dW[6 + k];
        // J(t) and the projected mean
        const float iz2 = iz * iz;
        float dtx = gu * c.fx * iz, dty = gv * c.fy * iz;
        float dtz = -gu * c.fx * tx * iz2 - gv * c.fy * ty * iz2;
        dtz += -c.fx * iz2 * dJ00 - c.fy * iz2 * dJ11;
        dtz += dJ02 * (c.fx * rx * iz2 - (clx ? 0.f : c.fx * iz * (-tx * iz2)));
        dtz += dJ12 * (c.fy * ry * iz2 - (cly ? 0.f : c.fy * iz * (-ty * iz2)));
        if (!clx) dtx += dJ02 * (-c.fx * iz2);
        if (!cly) dty += dJ12 * (-c.fy * iz2);
        dmu[0] += c.R[0] * dtx + c.R[3] * dty + c.R[6] * dtz;
        dmu[1] += c.R[1] * dtx + c.R[4] * dty + c.R[7] * dtz;
        dmu[2] += c.R[2] * dtx + c.R[5] * dty + c.R[8] * dtz;
    }
    if (!any) return;
    // RS = R diag(s)
    float dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p.d_scales[3 * i + k] += dRS[k] * R[k] + dRS[3 + k] * R[3 + k] + dRS[6 + k] * R[6 + k];
        dR[k] = dRS[k] * s[k];
        dR[3 + k] = dRS[3 + k] * s[k];
        dR[6 + k] = dRS[6 + k] * s[k];
    }
    // R(q^) partials
    const float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    const float dx_ = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                             w * dR[7] - 2.f * x * dR[8]);
    const float dy_ = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                             z * dR[7] - 2.f * y * dR[8]);
    const float dz_ = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                             y * dR[5] + x * dR[6] + y * dR[7]);
    const float pr = w * dw + x * dx_ + y * dy_ + z * dz_;
    const float iq = 1.f / qn;
    // each Gaussian's gradients belong to this thread alone: plain
    // read-modify-writes, 16 B at a time where the rows are 16-B aligned
    // (quats and SH of degree 1 and 3, checked on the host)
    float4* dq = reinterpret_cast<float4*>(p.d_quats) + i;
    float4 q = *dq;
    q.x += (dw - w * pr) * iq;
    q.y += (dx_ - x * pr) * iq;
    q.z += (dy_ - y * pr) * iq;
    q.w += (dz_ - z * pr) * iq;
    *dq = q;
    p.d_means[3 * i + 0] += dmu[0];
    p.d_means[3 * i + 1] += dmu[1];
    p.d_means[3 * i + 2] += dmu[2];
    p.d_opac[i] += dop;
    float* dsp = p.d_sh + i * NK * 3;
    if constexpr (NK % 4 == 0) {
        float4* d4 = reinterpret_cast<float4*>(dsp);
#pragma unroll
        for (int k = 0; k < NK * 3 / 4; ++k) {
            float4 t = d4[k];
            t.x += dsh[4 * k];
            t.y += dsh[4 * k + 1];
            t.z += dsh[4 * k + 2];
            t.w += dsh[4 * k + 3];
            d4[k] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NK * 3; ++k) dsp[k] += dsh[k];
    }
}

template <int TW, int TH, int WX, int WY>
lgs_status launch_bwd_layout(const BwdParams& bp, const Views& vs, bool persistent, cudaStream_t s) {
    using Lay = TileLayout<TW, TH, WX, WY>;
    const int smem = (int)sizeof(BwdSmem<Lay::NW>);
    const uint32_t n_work = vs.n_tiles * (uint32_t)Regions<TW, TH>::N;
    if (!persistent) {
        auto k = render_bwd_localgs<TW, TH, WX, WY>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return LGS_ERR_CUDA;
        k<<<n_work, Lay::NT, smem, s>>>(bp, vs);
        return cuda_status(cudaGetLastError());
    }
    auto k = render_bwd_localgs_persistent<TW, TH, WX, WY>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return LGS_ERR_CUDA;
    if (cudaMemsetAsync(bp.status + LGS_ST_QUEUE_BWD, 0, sizeof(int64_t), s) != cudaSuccess)
        return LGS_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Lay::NT, smem);
    const unsigned g = (unsigned)min((int64_t)n_work, (int64_t)max(1, sms * max(per_sm, 1)));
    k<<<g, Lay::NT, smem, s>>>(bp, vs);
    return cuda_status(cudaGetLastError());
}

template <int TW, int TH>
lgs_status launch_render_bwd(const BwdParams& bp, const Views& vs, int mode, int wx, int wy, bool persistent,
                             cudaStream_t s) {
    if constexpr (Regions<TW, TH>::SPLIT) {
        // large tiles: Local-GS adjoint in 8x8 blocks only (checked on the host)
        return launch_bwd_layout<TW, TH, 8, 8>(bp, vs, persistent, s);
    } else {
    if (mode == LGS_MODE_PLAIN) {
        render_bwd_plain<TW, TH><<<vs.n_tiles, 256, 0, s>>>(bp, vs);
        return cuda_status(cudaGetLastError());
    }
    if (wx == TW && wy == TH / 8) return launch_bwd_layout<TW, TH, TW, TH / 8>(bp, vs, persistent, s);
    if constexpr (TW == 16) {
        if (wx == 8 && wy == 4) return launch_bwd_layout<16, 16, 8, 4>(bp, vs, persistent, s);
        if (wx == 16 && wy == 4) return launch_bwd_layout<16, 16, 16, 4>(bp, vs, persistent, s);
    }
    return launch_bwd_layout<TW, TH, 8, 8>(bp, vs, persistent, s);
    }
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status lgs_render_bwd(const lgs_gaussians* g, const lgs_camera* cams,
                                     int32_t n_views, const lgs_config* cfg,
                                     const lgs_pre_out* pre, const uint32_t* vals,
                                     const uint32_t* ranges, const float* final_T,
                                     const uint32_t* n_contrib, const float* dL_drgb,
                                     const float* dL_dfinal_T, const lgs_grads* grads,
                                     int64_t* d_status, void* stream) {
    if (!g || !grads || !vals || !ranges || !final_T || !n_contrib || !dL_drgb || !d_status)
        return LGS_ERR_ARG;
    if (g->n < 0 || g->sh_degree < 0 || g->sh_degree > LGS_MAX_SH_DEGREE) return LGS_ERR_UNSUPPORTED;
    Views vs;
    lgs_status st = make_views(cams, n_views, cfg, &vs);
    if (st != LGS_OK) return st;
    st = check_pre(pre);
    if (st != LGS_OK) return st;
    if (!grads->xy2d || !grads->conic2d || !grads->rgb2d) return LGS_ERR_ARG;
    if (!aligned16(grads->conic2d) || !aligned16(grads->rgb2d) || (reinterpret_cast<uintptr_t>(grads->xy2d) & 7u))
        return LGS_ERR_ALIGN;
    if (reinterpret_cast<uintptr_t>(ranges) & 7u) return LGS_ERR_ALIGN;
    if (g->n == 0) return LGS_OK;
    if (!g->means || !g->scales || !g->quats || !g->sh || !grads->means || !grads->scales ||
        !grads->quats || !grads->opacities || !grads->sh)
        return LGS_ERR_ARG;
    if (!aligned16(g->quats) || !aligned16(grads->quats)) return LGS_ERR_ALIGN;
    if ((g->sh_degree == 1 || g->sh_degree == 3) && (!aligned16(g->sh) || !aligned16(grads->sh)))
        return LGS_ERR_ALIGN;
    // every host-checkable error returns before anything is enqueued
    if (cfg->mode != LGS_MODE_LOCALGS && cfg->mode != LGS_MODE_PLAIN) return LGS_ERR_UNSUPPORTED;
    const bool persistent = (cfg->flags & LGS_FLAG_PERSISTENT) != 0;
    if (persistent && cfg->mode != LGS_MODE_LOCALGS) return LGS_ERR_UNSUPPORTED;
    int wx = 0, wy = 0;
    if (!warp_block(cfg, &wx, &wy)) return LGS_ERR_UNSUPPORTED;
    if (cfg->mode != LGS_MODE_LOCALGS &&
        (split_tile(cfg->tile_w, cfg->tile_h) || wx != cfg->tile_w || wy != cfg->tile_h / 8))
        return LGS_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t m = g->n * (int64_t)n_views;
    if (cudaMemsetAsync(grads->xy2d, 0, sizeof(float) * 2 * (size_t)m, s) != cudaSuccess ||
        cudaMemsetAsync(grads->conic2d, 0, sizeof(float) * 4 * (size_t)m, s) != cudaSuccess ||
        cudaMemsetAsync(grads->rgb2d, 0, sizeof(float) * 4 * (size_t)m, s) != cudaSuccess)
        return LGS_ERR_CUDA;
    BwdParams bp;
    bp.xy = reinterpret_cast<const float4*>(pre->xy);
    bp.conic = reinterpret_cast<const float4*>(pre->conic);
    bp.rgb = reinterpret_cast<const float4*>(pre->rgb);
    bp.vals = vals;
    bp.ranges = reinterpret_cast<const uint2*>(ranges);
    bp.final_T = final_T;
    bp.n_contrib = n_contrib;
    bp.dL_drgb = dL_drgb;
    bp.dL_dT = dL_dfinal_T;
    bp.g_xy = grads->xy2d;
    bp.g_conic = grads->conic2d;
    bp.g_rgb = grads->rgb2d;
    bp.status = d_status;
    const int tw = cfg->tile_w, th = cfg->tile_h;
    if (tw == 16 && th == 16) st = launch_render_bwd<16, 16>(bp, vs, cfg->mode, wx, wy, persistent, s);
    else if (tw == 8 && th == 32) st = launch_render_bwd<8, 32>(bp, vs, cfg->mode, wx, wy, persistent, s);
    else if (tw == 32 && th == 8) st = launch_render_bwd<32, 8>(bp, vs, cfg->mode, wx, wy, persistent, s);
    else if (tw == 32 && th == 32) st = launch_render_bwd<32, 32>(bp, vs, cfg->mode, wx, wy, persistent, s);
    else if (tw == 16 && th == 32) st = launch_render_bwd<16, 32>(bp, vs, cfg->mode, wx, wy, persistent, s);
    else st = launch_render_bwd<32, 16>(bp, vs, cfg->mode, wx, wy, persistent, s);
    if (st != LGS_OK) return st;
    PreBwdParams pp;
    pp.means = g->means; pp.scales = g->scales; pp.quats = g->quats; pp.sh = g->sh; pp.n = g->n;
    pp.conic = reinterpret_cast<const float4*>(pre->conic);
    pp.tiles = pre->tiles;
    pp.flags = pre->flags;
    pp.g_xy = grads->xy2d; pp.g_conic = grads->conic2d; pp.g_rgb = grads->rgb2d;
    pp.d_means = grads->means; pp.d_scales = grads->scales; pp.d_quats = grads->quats;
    pp.d_opac = grads->opacities; pp.d_sh = grads->sh;
    const dim3 grid((unsigned)((g->n + 127) / 128));
    switch (g->sh_degree) {
        case 0: preprocess_bwd<0><<<grid, 128, 0, s>>>(pp, vs); break;
        case 1: preprocess_bwd<1><<<grid, 128, 0, s>>>(pp, vs); break;
        case 2: preprocess_bwd<2><<<grid, 128, 0, s>>>(pp, vs); break;
        default: preprocess_bwd<3><<<grid, 128, 0, s>>>(pp, vs); break;
    }
    return cuda_status(cudaGetLastError());
}
