/*
 * lgs_oracle.c -- plain, slow FP64 CPU oracle of 3D Gaussian Splatting
 * rasterization and of the Local-GS pieces (tile-local hoisting, tight-box
 * warp masks).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. It shares no code, header, table or
 * constant with the CUDA path, and it must never be used as a fallback for it.
 *
 * Every step is written in the order and notation of the method:
 *   Sec. II-A  : the rasterization pipeline (preprocess, duplicate + sort by
 *                (tile, depth) keys, per-tile front-to-back blending).
 *   Eq. (3DGS) : alpha = o * exp(-1/2 x~^T Sigma^-1 x~), conic = [[a,b],[b,c]].
 *   Alg. 1 (baseline column): per pixel, stop when T*(1-alpha) < 1e-4,
 *                skip alpha < 1/255 (Sec. III-C2 threshold), clamp 0.99.
 *   Eq. (hoist transform), Sec. III-B2: V = M(Delta) [a b c ln o]^T.
 *   Sec. III-C2/C3: tight box Cases A/B/C and the 8-bit warp mask.
 * The paper cites standard 3DGS for projection, covariance, EWA, radius and
 * SH colour; those steps follow the standard definitions (readings listed
 * beside each function).
 *
 * Floating point: all arithmetic and all inputs in double. The Python wrapper
 * passes the float32 scene values promoted exactly to double; finite-difference
 * checks pass perturbed doubles.
 *
 * Parity status of each function is pinned by the CPU test-suite:
 *   orc_preprocess   pinned (closed form single Gaussian, EWA Jacobian by
 *                    central differences, quaternion convention, SH basis by
 *                    quadrature orthonormality)
 *   orc_sort         pinned (brute-force sort of emitted keys)
 *   orc_blend        pinned (closed form, two-Gaussian composition, alpha
 *                    stack stop rule, invariants, brute force without tiling)
 *   orc_hoist        pinned (identity with the direct quadratic form)
 *   orc_blend_literal pinned (equals orc_blend where no pixel has a sub-1/255
 *                    alpha inside its warp's box and no pixel stops; T stays
 *                    the product of (1 - alpha); brute force per strip)
 *   orc_warp_mask    pinned (brute-force sampling of the ellipse)
 *   orc_block_mask   pinned (brute-force row intersection per block column;
 *                    superset of every pixel with alpha >= 1/255)
 *   orc_localgs_pairs / orc_localgs_pairs_blocks
 *                    pinned (closed-form counts: one Gaussian without a stop,
 *                    a stack whose every pixel stops at one position)
 *   orc_tight_rows   pinned (brute-force alpha over every pixel of the rect:
 *                    no dropped tile holds a pixel with alpha >= 1/255; every
 *                    kept tile holds a pixel inside the widened ellipse)
 *   orc_backward     pinned (central finite differences of orc_* forward)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* camera layout (24 doubles): W, H, fx, fy, cx, cy, R[9] (row-major,
 * world->camera), t[3], campos[3], bg[3] */
enum { CAM_W = 0, CAM_H, CAM_FX, CAM_FY, CAM_CX, CAM_CY, CAM_R, CAM_T = 15,
       CAM_POS = 18, CAM_BG = 21, CAM_SIZE = 24 };

/* guard thresholds (see orc_preprocess / orc_blend) */
enum { G_RECT_PX = 0, G_RADIUS_REL, G_NEAR_REL, G_DEPTH_REL, G_DET_REL,
       G_ALPHA_REL, G_STOP_REL, G_TIGHT_TAU_REL, G_TIGHT_PX, G_SIZE };

/* per-Gaussian guard flag bits */
enum { GF_RECT = 1, GF_RADIUS = 2, GF_NEAR = 4, GF_DEPTH = 8, GF_DET = 16, GF_TIGHT = 32 };

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Real spherical harmonics from their definition.                     */
/* Y_lm = K_lm P_l^|m|(cos th) * {sqrt2 cos(m phi), 1, sqrt2 sin(|m| phi)}
 * with the Condon-Shortley phase inside P_l^m, ordered l^2 + l + m,
 * m = -l..l (Sloan, "Stupid Spherical Harmonics Tricks"). */
static double factorial(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

static double assoc_legendre(int l, int m, double x) {
    /* P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2}; upward recurrence in l. */
    double pmm = 1.0;
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pll;
    }
    return pll;
}

double orc_sh_basis(int l, int m, const double dir[3]) {
    int am = m < 0 ? -m : m;
    double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - am) / factorial(l + am));
    double ct = dir[2];
    double phi = atan2(dir[1], dir[0]);
    double P = assoc_legendre(l, am, ct);
    if (m > 0) return sqrt(2.0) * K * cos(m * phi) * P;
    if (m < 0) return sqrt(2.0) * K * sin(am * phi) * P;
    return K * P;
}

/* all (deg+1)^2 basis values */
void orc_sh_eval(int deg, const double* dir, double* out) {
    for (int l = 0; l <= deg; ++l)
        for (int m = -l; m <= l; ++m) out[l * l + l + m] = orc_sh_basis(l, m, dir);
}

/* ------------------------------------------------------------------ */
/* Rotation of a unit quaternion q = (w, x, y, z). Convention pinned by a
 * test: (cos 45, 0, 0, sin 45) rotates e_x onto e_y. */
void orc_quat_to_rot(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Sigma = R(q) diag(s^2) R(q)^T (row-major 3x3) */
void orc_cov3d(const double s[3], const double q[4], double S[9]) {
    double R[9];
    orc_quat_to_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];
            S[i * 3 + j] = acc;
        }
}

/* EWA: 2D covariance of the projected Gaussian before the low-pass term.
 * t = camera-space mean. J is the Jacobian of (fx x/z, fy y/z) at t with x/z
 * and y/z clamped to +-1.3 tan(fov/2) (standard 3DGS). Out: cov2d[3] =
 * (S00, S01, S11) of J W Sigma W^T J^T. */
void orc_ewa(const double* cam, const double t[3], const double Sig[9], double cov2d[3]) {
    double W = cam[CAM_W], H = cam[CAM_H], fx = cam[CAM_FX], fy = cam[CAM_FY];
    double limx = 1.3 * (W / (2.0 * fx)), limy = 1.3 * (H / (2.0 * fy));
    double tz = t[2];
    double txz = t[0] / tz, tyz = t[1] / tz;
    if (txz < -limx) txz = -limx; if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy; if (tyz > limy) tyz = limy;
    double xh = txz * tz, yh = tyz * tz;
    double J[6] = { fx / tz, 0.0, -fx * xh / (tz * tz),
                    0.0, fy / tz, -fy * yh / (tz * tz) };
    const double* Rw = cam + CAM_R;
    double T[6]; /* T = J W (2x3) */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[i * 3 + k] * Rw[k * 3 + j];
            T[i * 3 + j] = acc;
        }
    double C[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += T[i * 3 + k] * Sig[k * 3 + l] * T[j * 3 + l];
            C[i * 2 + j] = acc;
        }
    cov2d[0] = C[0];
    cov2d[1] = C[1];
    cov2d[2] = C[3];
}

static double frac_dist(double q) { double f = q - floor(q); return f < 0.5 ? f : 1.0 - f; }

/* distance (in units of q) from q to the nearest integer k with lo <= k <= hi */
static double int_dist_in(double q, int lo, int hi) {
    double k = floor(q + 0.5);
    if (k < lo) k = lo;
    if (k > hi) k = hi;
    return fabs(q - k);
}

/* ------------------------------------------------------------------ */
/* Tight-box tile rows (Sec. III-C2 tight box applied to emission; the
 * Speedy-Splat / AdR-style tightening the paper composes with, Sec. II).
 * For the column strip of pixel columns X0 .. X0 + tile_w - 1: the ellipse
 *   a x~^2 + 2 b x~ y~ + c y~^2 = tau',  tau' = 1.001 * 2 ln(255 o) + 0.02
 * (the alpha = 1/255 level set, widened by the library's stated margin) is
 * cut to the strip's x-range, its lowest and highest points over that range
 * found by Cases A/B/C (as in orc_warp_mask), and the span widened by 1/64 px
 * at both ends. The kept pixel rows are ceil(lower) .. floor(upper); the kept
 * tile rows of the rect rows [ry0, ry1) are those holding a kept pixel row.
 * Returns the number of kept tile rows, [*lo, *hi] their range.
 * `widen` moves the decision boundaries outward (> 0) or inward (< 0) by
 * |widen| * (tau' relative band) and |widen| * (pixel band), for the guard. */
static int tight_rows_at(double a, double b, double c, double o, double mux, double muy,
                         int X0, int tile_w, int tile_h, int ry0, int ry1,
                         double tau_rel, double px, int* lo, int* hi) {
    double tau = 1.001 * (2.0 * log(255.0 * o)) + 0.02;
    tau = tau * (1.0 + tau_rel) + tau_rel * 1e-3;
    if (!(tau > 0.0)) return 0;
    double det = a * c - b * b;
    double xr = sqrt(c * tau / det);
    double x0 = X0 - mux, x1 = X0 + tile_w - 1 - mux;
    if (x1 < -xr - px || x0 > xr + px) return 0;
    if (x0 < -xr) x0 = -xr;
    if (x1 > xr) x1 = xr;
    if (x0 > x1) { double m = 0.5 * (x0 + x1); x0 = x1 = m; }   /* inside the px band only */
    double dy = sqrt(a * tau / det);
    double ymax, ymin;
    if (-b * dy < a * x0)      ymax = (-b * x0 + sqrt(fmax(0.0, c * tau - det * x0 * x0))) / c;
    else if (-b * dy > a * x1) ymax = (-b * x1 + sqrt(fmax(0.0, c * tau - det * x1 * x1))) / c;
    else                       ymax = dy;
    if (b * dy < a * x0)       ymin = (-b * x0 - sqrt(fmax(0.0, c * tau - det * x0 * x0))) / c;
    else if (b * dy > a * x1)  ymin = (-b * x1 - sqrt(fmax(0.0, c * tau - det * x1 * x1))) / c;
    else                       ymin = -dy;
    double P = ceil(muy + ymin - 1.0 / 64.0 - px);
    double Q = floor(muy + ymax + 1.0 / 64.0 + px);
    if (P > Q) return 0;
    int l = ry0, h = ry1 - 1;
    double tl = floor(P / tile_h), th = floor(Q / tile_h);
    if (tl > l) l = (int)tl;
    if (th < h) h = (int)th;
    *lo = l; *hi = h;
    return h >= l ? h - l + 1 : 0;
}

/* Kept tile rows of one column strip (central decision) and, in *guard, 1 if
 * the decision changes anywhere inside the guard band (boundaries moved by
 * +-band_tau relatively on tau' and +-band_px pixels). */
int orc_tight_rows(double a, double b, double c, double o, double mux, double muy,
                   int X0, int tile_w, int tile_h, int ry0, int ry1,
                   double band_tau, double band_px, int* lo, int* hi, int* guard) {
    int l = 0, h = -1, l1 = 0, h1 = -1, l2 = 0, h2 = -1;
    int n = tight_rows_at(a, b, c, o, mux, muy, X0, tile_w, tile_h, ry0, ry1, 0.0, 0.0, &l, &h);
    int n_out = tight_rows_at(a, b, c, o, mux, muy, X0, tile_w, tile_h, ry0, ry1,
                              band_tau, band_px, &l1, &h1);
    int n_in = tight_rows_at(a, b, c, o, mux, muy, X0, tile_w, tile_h, ry0, ry1,
                             -band_tau, -band_px, &l2, &h2);
    *lo = l; *hi = h;
    if (guard) *guard = (n_out != n_in) || (n_out > 0 && (l1 != l2 || h1 != h2));
    return n;
}

/* ------------------------------------------------------------------ */
/* Preprocess: one Gaussian per iteration, standard 3DGS semantics.
 * Outputs (per Gaussian i):
 *   uv[2i..]      projected mean (pixel units, pixel (i,j) sampled at (i,j))
 *   depth[i]      camera-space z (double); depth_bits[i] = bits of (float)z
 *   conic[3i..]   (a, b, c) of Sigma'^-1
 *   radius[i]     ceil(3 sqrt(lambda_max)), 0 when culled
 *   rect[4i..]    tile rect x_lo, y_lo, x_hi, y_hi (half-open)
 *   tiles[i]      (x_hi-x_lo)*(y_hi-y_lo), 0 when culled
 *   gflags[i]     with tight != 0 also GF_TIGHT: a tight-box emission
 *                 decision of the Gaussian lies inside its guard band
 *   rgb[3i..]     max(0, SH colour + 0.5); clamped[3i..] = pre-clamp value < 0
 *   gflags[i]     guard bits (decision within its guard band)
 */
void orc_preprocess(int64_t n, int sh_degree, const double* means, const double* scales,
                    const double* quats, const double* opac, const double* sh,
                    const double* cam, int tile_w, int tile_h, int tight, const double* guard,
                    double* uv, double* depth, uint32_t* depth_bits, double* conic,
                    int32_t* radius, int32_t* rect, int64_t* tiles, double* rgb,
                    uint8_t* clamped, uint8_t* gflags) {
    int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
    int gx = (W + tile_w - 1) / tile_w, gy = (H + tile_h - 1) / tile_h;
    const double* R = cam + CAM_R;
    const double* tc = cam + CAM_T;
    int K = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint8_t gf = 0;
        double mu[3] = { means[3 * i], means[3 * i + 1], means[3 * i + 2] };
        double t[3];
        for (int r = 0; r < 3; ++r)
            t[r] = ((R[r * 3 + 0] * mu[0] + R[r * 3 + 1] * mu[1]) + R[r * 3 + 2] * mu[2]) + tc[r];
        radius[i] = 0; tiles[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        uv[2 * i] = uv[2 * i + 1] = 0.0;
        depth[i] = t[2];
        {
            float zf = (float)t[2];
            memcpy(&depth_bits[i], &zf, 4);
            /* guard: fp64 depth close to a float32 rounding midpoint */
            double lo = nextafterf(zf, -INFINITY), hi = nextafterf(zf, INFINITY);
            double mid = t[2] >= (double)zf ? 0.5 * ((double)zf + hi) : 0.5 * ((double)zf + lo);
            if (fabs(t[2] - mid) < guard[G_DEPTH_REL] * fabs(t[2])) gf |= GF_DEPTH;
        }
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0.0;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0.0;
        clamped[3 * i] = clamped[3 * i + 1] = clamped[3 * i + 2] = 0;
        if (fabs(t[2] - 0.2) < guard[G_NEAR_REL] * 0.2) gf |= GF_NEAR;
        if (t[2] <= 0.2) { gflags[i] = gf; continue; }          /* near-plane cull */
        double s[3] = { scales[3 * i], scales[3 * i + 1], scales[3 * i + 2] };
        double q[4] = { quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3] };
        double Sig[9], cv[3];
        orc_cov3d(s, q, Sig);
        orc_ewa(cam, t, Sig, cv);
        cv[0] += 0.3; cv[2] += 0.3;                              /* low-pass dilation */
        double det = cv[0] * cv[2] - cv[1] * cv[1];
        if (det < guard[G_DET_REL] * cv[0] * cv[2]) gf |= GF_DET;
        if (det <= 0.0) { gflags[i] = gf; continue; }
        double a = cv[2] / det, b = -cv[1] / det, c = cv[0] / det;
        double mid = 0.5 * (cv[0] + cv[2]);
        double lam1 = mid + sqrt(fmax(0.1, mid * mid - det));
        double r3 = 3.0 * sqrt(lam1);
        double rr = ceil(r3);
        if (frac_dist(r3) < guard[G_RADIUS_REL] * r3) gf |= GF_RADIUS;
        double u = cam[CAM_FX] * (t[0] / t[2]) + cam[CAM_CX];
        double v = cam[CAM_FY] * (t[1] / t[2]) + cam[CAM_CY];
        double qx0 = (u - rr) / tile_w, qx1 = (u + rr + tile_w - 1) / tile_w;
        double qy0 = (v - rr) / tile_h, qy1 = (v + rr + tile_h - 1) / tile_h;
        int x0 = (int)fmin(gx, fmax(0.0, floor(qx0)));
        int x1 = (int)fmin(gx, fmax(0.0, floor(qx1)));
        int y0 = (int)fmin(gy, fmax(0.0, floor(qy0)));
        int y1 = (int)fmin(gy, fmax(0.0, floor(qy1)));
        double gpx = guard[G_RECT_PX];
        if (int_dist_in(qx0, 1, gx) * tile_w < gpx || int_dist_in(qx1, 1, gx) * tile_w < gpx ||
            int_dist_in(qy0, 1, gy) * tile_h < gpx || int_dist_in(qy1, 1, gy) * tile_h < gpx)
            gf |= GF_RECT;
        gflags[i] = gf;
        int64_t area = (int64_t)(x1 - x0) * (int64_t)(y1 - y0);
        if (area == 0) continue;
        /* colour from SH in the view direction */
        double d[3] = { mu[0] - cam[CAM_POS], mu[1] - cam[CAM_POS + 1], mu[2] - cam[CAM_POS + 2] };
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dn; d[1] /= dn; d[2] /= dn;
        double Y[16];
        orc_sh_eval(sh_degree, d, Y);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += Y[k] * sh[(i * K + k) * 3 + ch];
            acc += 0.5;
            clamped[3 * i + ch] = acc < 0.0;
            rgb[3 * i + ch] = acc < 0.0 ? 0.0 : acc;
        }
        uv[2 * i] = u; uv[2 * i + 1] = v;
        conic[3 * i] = a; conic[3 * i + 1] = b; conic[3 * i + 2] = c;
        radius[i] = (int32_t)rr;
        rect[4 * i] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
        tiles[i] = area;
        if (tight) {          /* guard flag of the tight-box emission decisions */
            int any_guard = 0;
            for (int tx = x0; tx < x1; ++tx) {
                int lo, hi, gd = 0;
                orc_tight_rows(a, b, c, opac[i], u, v, tx * tile_w, tile_w, tile_h, y0, y1,
                               guard[G_TIGHT_TAU_REL], guard[G_TIGHT_PX], &lo, &hi, &gd);
                any_guard |= gd;
            }
            if (any_guard) gflags[i] |= GF_TIGHT;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Duplicate + sort (Sec. II-A): key = (tile_id << 32) | bits(float depth),
 * emitted in Gaussian order, tiles row-major inside each rect (with tight != 0
 * only the tiles orc_tight_rows keeps, from uv/conic/opac); sorted
 * ascending by key with ties kept in emission order (stable sort).
 * tile_id = tile_offset + ty*gx + tx. ranges[2t..] = [first, last+1) or (0,0). */
typedef struct { uint64_t key; int64_t pos; uint32_t val; } orc_kv;

static int kv_cmp(const void* pa, const void* pb) {
    const orc_kv* a = (const orc_kv*)pa; const orc_kv* b = (const orc_kv*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->pos < b->pos ? -1 : (a->pos > b->pos);
}

int64_t orc_sort(int64_t n, int gx, int gy, int64_t tile_offset, uint32_t val_offset,
                 const int32_t* rect, const int64_t* tiles, const uint32_t* depth_bits,
                 int64_t capacity, uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                 int tight, int tile_w, int tile_h, const double* uv, const double* conic,
                 const double* opac) {
    int64_t K = 0;
    for (int64_t i = 0; i < n; ++i) K += tiles[i];     /* upper bound with tight != 0 */
    if (K > capacity) return -K;
    orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(K > 0 ? K : 1));
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (tiles[i] == 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                if (tight) {          /* drop the tiles the tight box does not reach */
                    int lo, hi;
                    int k = orc_tight_rows(conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], opac[i],
                                           uv[2 * i], uv[2 * i + 1], tx * tile_w, tile_w, tile_h,
                                           rect[4 * i + 1], rect[4 * i + 3], 0.0, 0.0, &lo, &hi, NULL);
                    if (k == 0 || ty < lo || ty > hi) continue;
                }
                uint64_t tid = (uint64_t)(tile_offset + (int64_t)ty * gx + tx);
                kv[p].key = (tid << 32) | depth_bits[i];
                kv[p].val = (uint32_t)i + val_offset;
                kv[p].pos = p;
                ++p;
            }
    }
    K = p;                    /* instances actually emitted */
    qsort(kv, (size_t)K, sizeof(orc_kv), kv_cmp);
    int64_t nt = (int64_t)gx * gy;
    for (int64_t t = 0; t < 2 * nt; ++t) ranges[t] = 0;
    for (int64_t k = 0; k < K; ++k) {
        keys[k] = kv[k].key;
        vals[k] = kv[k].val;
        int64_t t = (int64_t)(kv[k].key >> 32) - tile_offset;
        if (k == 0 || (kv[k - 1].key >> 32) != (kv[k].key >> 32)) ranges[2 * t] = (uint32_t)k;
        ranges[2 * t + 1] = (uint32_t)(k + 1);
    }
    free(kv);
    return K;
}

/* ------------------------------------------------------------------ */
/* Front-to-back blending, Alg. 1 baseline column, one pixel at a time.
 * For each pixel (px, py) of tile t and each Gaussian k of its list in order:
 *   d = (u_k - px, v_k - py); p = -1/2 d^T Q d
 *   alpha = min(0.99, o exp(p)); skip if alpha < 1/255
 *   test_T = T (1 - alpha); stop (without blending) if test_T < 1e-4
 *   C += rgb alpha T; T = test_T; last = position of k in the list + 1
 * out: rgb [3,H,W] = C + T bg; final_T [H,W]; n_contrib [H,W] = last.
 * pguard [H,W]: 1 if an alpha or stop decision on the pixel's path lay inside
 * its relative guard band. stop_pos [H,W] (optional): list position (1-based)
 * of the Gaussian whose test_T fell below 1e-4, 0 if the pixel never stopped.
 * n_useful [H,W] (optional): blended Gaussians. vals index the per-Gaussian
 * arrays directly. tile_mask [tiles] (optional): only pixels of tiles with a
 * non-zero entry are computed (the others are left untouched). */
void orc_blend(int W, int H, int tile_w, int tile_h, const double* bg,
               const uint32_t* vals, const uint32_t* ranges, int64_t tile_offset,
               const double* uv, const double* conic, const double* opac, const double* rgb,
               const double* guard, double* out_rgb, double* final_T, uint32_t* n_contrib,
               uint8_t* pguard, uint32_t* stop_pos, uint32_t* n_useful, const uint8_t* tile_mask) {
    int gx = (W + tile_w - 1) / tile_w;
    const double a_min = 1.0 / 255.0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
        int px = (int)(pix % W), py = (int)(pix / W);
        int64_t tile = tile_offset + (int64_t)(py / tile_h) * gx + px / tile_w;
        if (tile_mask && !tile_mask[tile - tile_offset]) continue;   /* pixel not sampled */
        uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        double T = 1.0, C[3] = { 0, 0, 0 };
        uint32_t last = 0, stop = 0, useful = 0;
        uint8_t g = 0;
        for (uint32_t k = s; k < e; ++k) {
            uint32_t id = vals[k];
            double dx = uv[2 * id] - px, dy = uv[2 * id + 1] - py;
            double a = conic[3 * id], b = conic[3 * id + 1], c = conic[3 * id + 2];
            double p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
            double al = (double)opac[id] * exp(p);
            if (al > 0.99) al = 0.99;
            if (fabs(al - a_min) < guard[G_ALPHA_REL] * a_min) g = 1;
            if (al < a_min) continue;
            double test_T = T * (1.0 - al);
            if (fabs(test_T - 1e-4) < guard[G_STOP_REL] * 1e-4) g = 1;
            if (test_T < 1e-4) { stop = k - s + 1; break; }
            ++useful;
            for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * id + ch] * al * T;
            T = test_T;
            last = k - s + 1;
        }
        for (int ch = 0; ch < 3; ++ch) out_rgb[(int64_t)ch * W * H + pix] = C[ch] + T * bg[ch];
        final_T[pix] = T;
        n_contrib[pix] = last;
        pguard[pix] = g;
        if (stop_pos) stop_pos[pix] = stop;
        if (n_useful) n_useful[pix] = useful;
    }
}

/* ------------------------------------------------------------------ */
/* Paper-literal warp-coherent blending (Alg. 1 right column read literally,
 * Sec. III-D). Per tile and per warp strip (n_warps strips of tile_w x
 * tile_h/n_warps pixels), the tile list in order. A Gaussian is processed by
 * the strip iff the strip's pixel rows meet the tight box of the tile column
 * (orc_tight_rows at pixel-row granularity: the widened rule of the
 * emission). Before each processed Gaussian the strip leaves the list when
 * every pixel of it inside the image has T < 1e-4. A processed Gaussian blends
 * into every pixel of the strip, with no 1/255 test:
 *   alpha = min(0.99, o e^p), w = alpha T, C += f w, T -= w.
 * n_contrib = list position (1-based) of the last processed Gaussian.
 * pguard[pix] = 1 when a decision of the pixel's strip (a mask bit or the
 * exit test on the strip's largest T) lies inside its guard band. */
void orc_blend_literal(int W, int H, int tile_w, int tile_h, int n_warps, const double* bg,
                       const uint32_t* vals, const uint32_t* ranges, int64_t tile_offset,
                       const double* uv, const double* conic, const double* opac,
                       const double* rgb, const double* guard, double* out_rgb, double* final_T,
                       uint32_t* n_contrib, uint8_t* pguard) {
    int gx = (W + tile_w - 1) / tile_w, gy = (H + tile_h - 1) / tile_h;
    int rows = tile_h / n_warps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t ts = 0; ts < (int64_t)gx * gy * n_warps; ++ts) {
        int64_t tile = ts / n_warps;
        int w = (int)(ts % n_warps);
        int tx = (int)(tile % gx), ty = (int)(tile / gx);
        int X0 = tx * tile_w, Y0 = ty * tile_h + w * rows;
        int pxs[64], pys[64], np = 0;
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < tile_w; ++c)
                if (X0 + c < W && Y0 + r < H) { pxs[np] = X0 + c; pys[np] = Y0 + r; ++np; }
        if (np == 0) continue;
        double T[64], C[64][3];
        for (int q = 0; q < np; ++q) { T[q] = 1.0; C[q][0] = C[q][1] = C[q][2] = 0.0; }
        uint32_t s = ranges[2 * (tile_offset + tile)], e = ranges[2 * (tile_offset + tile) + 1];
        uint32_t last = 0;
        uint8_t g = 0;
        for (uint32_t k = s; k < e; ++k) {
            uint32_t id = vals[k];
            double a = conic[3 * id], b = conic[3 * id + 1], c = conic[3 * id + 2], o = opac[id];
            int lo, hi, gd = 0;
            int hit = orc_tight_rows(a, b, c, o, uv[2 * id], uv[2 * id + 1], X0, tile_w, 1, Y0, Y0 + rows,
                                     guard[G_TIGHT_TAU_REL], guard[G_TIGHT_PX], &lo, &hi, &gd);
            if (gd) g = 1;
            if (hit == 0) continue;
            double tmax = 0.0;
            for (int q = 0; q < np; ++q) if (T[q] > tmax) tmax = T[q];
            if (fabs(tmax - 1e-4) < guard[G_STOP_REL] * 1e-4) g = 1;
            if (tmax < 1e-4) break;                     /* the whole strip is done */
            for (int q = 0; q < np; ++q) {
                double dx = uv[2 * id] - pxs[q], dy = uv[2 * id + 1] - pys[q];
                double p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                double al = o * exp(p);
                if (al > 0.99) al = 0.99;
                double wgt = al * T[q];
                for (int ch = 0; ch < 3; ++ch) C[q][ch] += rgb[3 * id + ch] * wgt;
                T[q] -= wgt;
            }
            last = k - s + 1;
        }
        for (int q = 0; q < np; ++q) {
            int64_t pix = (int64_t)pys[q] * W + pxs[q];
            for (int ch = 0; ch < 3; ++ch) out_rgb[(int64_t)ch * W * H + pix] = C[q][ch] + T[q] * bg[ch];
            final_T[pix] = T[q];
            n_contrib[pix] = last;
            pguard[pix] = g;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Hoist transform (Eq. hoist transform, Sec. III-B2): with the tile-local
 * displacement Delta = mu - T_origin,
 *   [A B C D E F]^T = M(Delta) [a b c ln o]^T
 * so that ln alpha = A x'^2 + B x'y' + C y'^2 + D x' + E y' + F for a pixel at
 * tile-local x' = x - T_origin. */
void orc_hoist(double a, double b, double c, double o, double dx, double dy, double V[6]) {
    double lno = log(o);
    V[0] = -0.5 * a;
    V[1] = -1.0 * b;
    V[2] = -0.5 * c;
    V[3] = dx * a + dy * b;
    V[4] = dx * b + dy * c;
    V[5] = -0.5 * dx * dx * a - dx * dy * b - 0.5 * dy * dy * c + 1.0 * lno;
}

/* Tight box and warp mask (Sec. III-C2, III-C3) for one Gaussian and one
 * tile column of width tile_w starting at pixel column X0, rows Y0..Y0+tile_h-1
 * split into n_warps strips of tile_h/n_warps rows.
 *   tau = 2 ln(255 o); ellipse a x~^2 + 2b x~y~ + c y~^2 = tau
 *   x~ in [X0 - mu_x, X0 + tile_w - 1 - mu_x]; d_y = sqrt(a tau/(ac - b^2))
 *   upper bound: Case A (-b d_y < a x~0) -> root at x~0; Case B (-b d_y > a x~1)
 *   -> root at x~1; Case C -> d_y. Lower bound symmetric (peak at +b d_y / a).
 * Reading: the strip is first intersected with the ellipse's x-extent
 * |x~| <= sqrt(c tau/(ac - b^2)); a strip outside it gives mask 0, and the
 * clamp keeps the square roots real. Returns the warp bit mask. */
uint32_t orc_warp_mask(double a, double b, double c, double o, double mux, double muy,
                       int X0, int Y0, int tile_w, int tile_h, int n_warps) {
    double tau = 2.0 * log(255.0 * o);
    if (!(tau > 0.0)) return 0u;
    double det = a * c - b * b;
    double xr = sqrt(c * tau / det);
    double x0 = X0 - mux, x1 = X0 + tile_w - 1 - mux;
    if (x1 < -xr || x0 > xr) return 0u;
    if (x0 < -xr) x0 = -xr;
    if (x1 > xr) x1 = xr;
    double dy = sqrt(a * tau / det);
    double ymax, ymin;
    if (-b * dy < a * x0)      ymax = (-b * x0 + sqrt(fmax(0.0, c * tau - det * x0 * x0))) / c;
    else if (-b * dy > a * x1) ymax = (-b * x1 + sqrt(fmax(0.0, c * tau - det * x1 * x1))) / c;
    else                       ymax = dy;
    if (b * dy < a * x0)       ymin = (-b * x0 - sqrt(fmax(0.0, c * tau - det * x0 * x0))) / c;
    else if (b * dy > a * x1)  ymin = (-b * x1 - sqrt(fmax(0.0, c * tau - det * x1 * x1))) / c;
    else                       ymin = -dy;
    double ylo = muy + ymin, yhi = muy + ymax;
    int ys = (int)fmax((double)Y0, ceil(ylo));
    int ye = (int)fmin((double)(Y0 + tile_h - 1), floor(yhi));
    if (ys > ye) return 0u;
    int rows = tile_h / n_warps;
    int ws = (ys - Y0) / rows, we = (ye - Y0) / rows;
    return ((1u << (we - ws + 1)) - 1u) << ws;
}

/* Block mask: the tile cut into (tile_w/block_w) x (tile_h/block_h) blocks,
 * block (bx, by) owning bit by * (tile_w/block_w) + bx. Each block column is
 * the pixel-column strip of orc_warp_mask above (its own tight box over its
 * own x-range), split into strips of block_h rows; with block_w = tile_w this
 * is orc_warp_mask with tile_h/block_h strips. */
uint32_t orc_block_mask(double a, double b, double c, double o, double mux, double muy,
                        int X0, int Y0, int tile_w, int tile_h, int block_w, int block_h) {
    int nbx = tile_w / block_w, nby = tile_h / block_h;
    uint32_t m = 0u;
    for (int bx = 0; bx < nbx; ++bx) {
        uint32_t col = orc_warp_mask(a, b, c, o, mux, muy, X0 + bx * block_w, Y0, block_w, tile_h, nby);
        for (int by = 0; by < nby; ++by)
            if (col & (1u << by)) m |= 1u << (by * nbx + bx);
    }
    return m;
}

/* Work of the Local-GS schedule in pixel-Gaussian pairs, for a warp layout of
 * block_w x block_h pixel blocks (one warp each): for every tile and block,
 * the Gaussians of the tile list whose mask bit for the block is set, counted
 * up to and including the first one after which every pixel of the block has
 * stopped (or the end of the list); times the pixels of the block (the
 * evaluations its warp issues). n_contrib/stop positions come from the blend
 * above: a pixel has stopped once the list position passes its stop position.
 * stop_pos[pix] = list position (1-based) of the Gaussian that triggered the
 * stop, or 0 when the pixel never stopped; pixels outside the image count as
 * stopped. */
int64_t orc_localgs_pairs_blocks(int W, int H, int tile_w, int tile_h, int block_w, int block_h,
                                 const uint32_t* vals, const uint32_t* ranges, int64_t tile_offset,
                                 const double* uv, const double* conic, const double* opac,
                                 const uint32_t* stop_pos) {
    int gx = (W + tile_w - 1) / tile_w, gy = (H + tile_h - 1) / tile_h;
    int nbx = tile_w / block_w, nby = tile_h / block_h;
    int64_t total = 0;
    for (int ty = 0; ty < gy; ++ty)
        for (int tx = 0; tx < gx; ++tx) {
            int64_t tile = tile_offset + (int64_t)ty * gx + tx;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            int X0 = tx * tile_w, Y0 = ty * tile_h;
            for (int w = 0; w < nbx * nby; ++w) {
                int bx = w % nbx, by = w / nbx;
                /* stop position of the block = max over its pixels (0 = never) */
                uint32_t wstop = 0;
                int never = 0;
                for (int r = 0; r < block_h; ++r)
                    for (int cc = 0; cc < block_w; ++cc) {
                        int px = X0 + bx * block_w + cc, py = Y0 + by * block_h + r;
                        if (px >= W || py >= H) continue;
                        uint32_t sp = stop_pos[(int64_t)py * W + px];
                        if (sp == 0) never = 1;
                        else if (sp > wstop) wstop = sp;
                    }
                for (uint32_t k = s; k < e; ++k) {
                    uint32_t pos = k - s + 1;
                    if (!never && pos > wstop) break;
                    uint32_t id = vals[k];
                    uint32_t m = orc_block_mask(conic[3 * id], conic[3 * id + 1], conic[3 * id + 2],
                                                opac[id], uv[2 * id], uv[2 * id + 1], X0, Y0,
                                                tile_w, tile_h, block_w, block_h);
                    if (m & (1u << w)) total += (int64_t)block_w * block_h;
                }
            }
        }
    return total;
}

/* The paper's layout: n_warps full-width strips of tile_h/n_warps rows. */
int64_t orc_localgs_pairs(int W, int H, int tile_w, int tile_h, int n_warps,
                          const uint32_t* vals, const uint32_t* ranges, int64_t tile_offset,
                          const double* uv, const double* conic, const double* opac,
                          const uint32_t* stop_pos) {
    return orc_localgs_pairs_blocks(W, H, tile_w, tile_h, tile_w, tile_h / n_warps, vals, ranges,
                                    tile_offset, uv, conic, opac, stop_pos);
}

/* ------------------------------------------------------------------ */
/* Hand-derived adjoint (reverse mode) of the forward map above, for a loss
 * L = sum_pix <g_pix, rgb_pix> + sum_pix gT_pix * final_T_pix. The paper covers
 * inference only; this is the plain chain rule through each forward step, with
 * the piecewise-constant decisions (rects, 1/255 skips, stops, clamps) held
 * fixed, and the true derivative of every clamp (zero slope where clamped).
 *
 * Blend (per pixel, blended Gaussians k in order, T_k before k):
 *   dL/drgb_k = alpha_k T_k g
 *   dL/dalpha_k = T_k <rgb_k, g> - (<S_k, g> + T_f <bg, g> + T_f gT)/(1 - alpha_k),
 *                 S_k = sum_{j>k} rgb_j alpha_j T_j
 *   alpha = o e^p (unclamped): dalpha/do = e^p, dalpha/dp = alpha
 *   p = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = (u - px, v - py)
 * Conic: (a, b, c) = (S11, -S01, S00)/(S00 S11 - S01^2) differentiated in
 * (S00, S01, S11); Sigma' = T Sigma T^T + 0.3 I with T = J W:
 *   dL/dSigma = T^T G T, dL/dT = 2 G T Sigma, G = [[g00, g01/2], [g01/2, g11]].
 * J(t) with r = clamp(t_x/t_z): J00 = fx/tz, J02 = -fx r/tz (dr = 0 when
 * clamped); mean u = fx tx/tz + cx; t = W mu + t_c.
 * Sigma = M M^T, M = R(q^) diag(s): dL/dM = 2 dL/dSigma M; q^ = q/|q|.
 * SH: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5); dir = (mu - campos)/|..|;
 * the basis gradient is taken in spherical coordinates
 *   sin(th) dP_l^m/dth = l cos(th) P_l^m - (l+m) P_{l-1}^m.
 * g2d (optional, n x 9): dL/d(u, v, a, b, c, o, r, g, b). */
static void sh_grad(int deg, const double dir[3], double* Y, double (*dY)[3]) {
    double ct = dir[2], st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = atan2(dir[1], dir[0]);
    double eth[3] = { ct * cos(phi), ct * sin(phi), -st };
    double eph[3] = { -sin(phi), cos(phi), 0.0 };
    for (int l = 0; l <= deg; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int idx = l * l + l + m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, ct);
            double Pm1 = (l - 1 >= am) ? assoc_legendre(l - 1, am, ct) : 0.0;
            double dPdth = (st > 0.0) ? (l * ct * P - (l + am) * Pm1) / st : 0.0;
            double trig, dtrig;
            if (m > 0)      { trig = sqrt(2.0) * cos(m * phi); dtrig = -sqrt(2.0) * m * sin(m * phi); }
            else if (m < 0) { trig = sqrt(2.0) * sin(am * phi); dtrig = sqrt(2.0) * am * cos(am * phi); }
            else            { trig = 1.0; dtrig = 0.0; }
            Y[idx] = K * P * trig;
            double dth = K * dPdth * trig;
            double dph = (st > 0.0) ? K * P * dtrig / st : 0.0;
            for (int c = 0; c < 3; ++c) dY[idx][c] = dth * eth[c] + dph * eph[c];
        }
}

void orc_backward(int64_t n, int sh_degree, const double* means, const double* scales,
                  const double* quats, const double* opac, const double* sh, const double* cam,
                  int tile_w, int tile_h, const double* dL_drgb, const double* dL_dT,
                  double* g_means, double* g_scales, double* g_quats, double* g_opac,
                  double* g_sh, double* g2d) {
    int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
    int gx = (W + tile_w - 1) / tile_w;
    int Ksh = (sh_degree + 1) * (sh_degree + 1);
    double guard0[G_SIZE] = { 0 };
    double* uv = (double*)calloc((size_t)n * 2 + 1, sizeof(double));
    double* depth = (double*)calloc((size_t)n + 1, sizeof(double));
    uint32_t* dbits = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    double* conic = (double*)calloc((size_t)n * 3 + 1, sizeof(double));
    int32_t* radius = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t* rect = (int32_t*)calloc((size_t)n * 4 + 1, sizeof(int32_t));
    int64_t* tiles = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    double* rgb = (double*)calloc((size_t)n * 3 + 1, sizeof(double));
    uint8_t* clamped = (uint8_t*)calloc((size_t)n * 3 + 1, 1);
    uint8_t* gfl = (uint8_t*)calloc((size_t)n + 1, 1);
    orc_preprocess(n, sh_degree, means, scales, quats, opac, sh, cam, tile_w, tile_h, 0, guard0, uv,
                   depth, dbits, conic, radius, rect, tiles, rgb, clamped, gfl);
    int64_t K = 0;
    for (int64_t i = 0; i < n; ++i) K += tiles[i];
    int64_t ntile = (int64_t)gx * ((H + tile_h - 1) / tile_h);
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(K + 1));
    uint32_t* vals = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(K + 1));
    uint32_t* ranges = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * ntile + 2));
    orc_sort(n, gx, (H + tile_h - 1) / tile_h, 0, 0, rect, tiles, dbits, K, keys, vals, ranges,
             0, tile_w, tile_h, NULL, NULL, NULL);

    /* 2D gradients: du dv da db dc do dr dg db */
    double* G2 = (double*)calloc((size_t)n * 9 + 1, sizeof(double));
    const double* bg = cam + CAM_BG;
    const double a_min = 1.0 / 255.0;
    uint32_t* lid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(K + 1));
    double* lal = (double*)malloc(sizeof(double) * (size_t)(K + 1));
    double* lT = (double*)malloc(sizeof(double) * (size_t)(K + 1));
    double* lep = (double*)malloc(sizeof(double) * (size_t)(K + 1));
    uint8_t* lcl = (uint8_t*)malloc((size_t)(K + 1));
    for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
        int px = (int)(pix % W), py = (int)(pix / W);
        int64_t tile = (int64_t)(py / tile_h) * gx + px / tile_w;
        uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        double T = 1.0;
        int cnt = 0;
        for (uint32_t k = s; k < e; ++k) {
            uint32_t id = vals[k];
            double dx = uv[2 * id] - px, dy = uv[2 * id + 1] - py;
            double a = conic[3 * id], b = conic[3 * id + 1], c = conic[3 * id + 2];
            double p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
            double ep = exp(p);
            double al = (double)opac[id] * ep;
            uint8_t cl = 0;
            if (al > 0.99) { al = 0.99; cl = 1; }
            if (al < a_min) continue;
            double test_T = T * (1.0 - al);
            if (test_T < 1e-4) break;
            lid[cnt] = id; lal[cnt] = al; lT[cnt] = T; lep[cnt] = ep; lcl[cnt] = cl;
            ++cnt;
            T = test_T;
        }
        double Tf = T;
        double g[3] = { dL_drgb[pix], dL_drgb[(int64_t)W * H + pix], dL_drgb[2 * (int64_t)W * H + pix] };
        double gT = dL_dT ? dL_dT[pix] : 0.0;
        double tail = Tf * (bg[0] * g[0] + bg[1] * g[1] + bg[2] * g[2]) + Tf * gT;
        double S = 0.0; /* <S_k, g> */
        for (int j = cnt - 1; j >= 0; --j) {
            uint32_t id = lid[j];
            double al = lal[j], Tk = lT[j];
            double cg = rgb[3 * id] * g[0] + rgb[3 * id + 1] * g[1] + rgb[3 * id + 2] * g[2];
            for (int ch = 0; ch < 3; ++ch) G2[9 * id + 6 + ch] += al * Tk * g[ch];
            double dal = Tk * cg - (S + tail) / (1.0 - al);
            S += cg * al * Tk;
            if (lcl[j]) continue;
            double dx = uv[2 * id] - px, dy = uv[2 * id + 1] - py;
            double a = conic[3 * id], b = conic[3 * id + 1], c = conic[3 * id + 2];
            double dp = dal * al;
            G2[9 * id + 5] += dal * lep[j];
            G2[9 * id + 2] += dp * (-0.5 * dx * dx);
            G2[9 * id + 3] += dp * (-dx * dy);
            G2[9 * id + 4] += dp * (-0.5 * dy * dy);
            G2[9 * id + 0] += dp * (-(a * dx + b * dy));
            G2[9 * id + 1] += dp * (-(b * dx + c * dy));
        }
    }

    /* per Gaussian chain rule */
    const double* Rw = cam + CAM_R;
    double fx = cam[CAM_FX], fy = cam[CAM_FY];
    double limx = 1.3 * (W / (2.0 * fx)), limy = 1.3 * (H / (2.0 * fy));
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) { g_means[3 * i + k] = 0; g_scales[3 * i + k] = 0; }
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] = 0;
        g_opac[i] = 0;
        for (int k = 0; k < Ksh * 3; ++k) g_sh[i * Ksh * 3 + k] = 0;
        if (g2d) for (int k = 0; k < 9; ++k) g2d[9 * i + k] = G2[9 * i + k];
        if (tiles[i] == 0) continue;
        double* G = G2 + 9 * i;
        double mu[3] = { means[3 * i], means[3 * i + 1], means[3 * i + 2] };
        double t[3];
        for (int r = 0; r < 3; ++r)
            t[r] = ((Rw[r * 3 + 0] * mu[0] + Rw[r * 3 + 1] * mu[1]) + Rw[r * 3 + 2] * mu[2]) + cam[CAM_T + r];
        double s[3] = { scales[3 * i], scales[3 * i + 1], scales[3 * i + 2] };
        double q[4] = { quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3] };
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qh[4] = { q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn };
        double R[9], Sig[9];
        orc_quat_to_rot(qh, R);
        orc_cov3d(s, q, Sig);
        double tz = t[2];
        double rx = t[0] / tz, ry = t[1] / tz;
        int clx = 0, cly = 0;
        if (rx < -limx) { rx = -limx; clx = 1; } if (rx > limx) { rx = limx; clx = 1; }
        if (ry < -limy) { ry = -limy; cly = 1; } if (ry > limy) { ry = limy; cly = 1; }
        double J[6] = { fx / tz, 0.0, -fx * rx / tz, 0.0, fy / tz, -fy * ry / tz };
        double Tm[6];
        for (int r = 0; r < 2; ++r)
            for (int c2 = 0; c2 < 3; ++c2) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += J[r * 3 + k] * Rw[k * 3 + c2];
                Tm[r * 3 + c2] = acc;
            }
        double C[4];
        for (int r = 0; r < 2; ++r)
            for (int c2 = 0; c2 < 2; ++c2) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += Tm[r * 3 + k] * Sig[k * 3 + l] * Tm[c2 * 3 + l];
                C[r * 2 + c2] = acc;
            }
        double s00 = C[0] + 0.3, s01 = C[1], s11 = C[3] + 0.3;
        double D = s00 * s11 - s01 * s01, D2 = D * D;
        double ga = G[2], gb = G[3], gc = G[4];
        double g00 = ga * (-s11 * s11 / D2) + gb * (s01 * s11 / D2) + gc * (1.0 / D - s00 * s11 / D2);
        double g11 = ga * (1.0 / D - s11 * s00 / D2) + gb * (s01 * s00 / D2) + gc * (-s00 * s00 / D2);
        double g01 = ga * (2.0 * s01 * s11 / D2) + gb * (-1.0 / D - 2.0 * s01 * s01 / D2) +
                     gc * (2.0 * s01 * s00 / D2);
        double Gm[4] = { g00, 0.5 * g01, 0.5 * g01, g11 };
        /* dL/dSigma = T^T G T ; dL/dT = 2 G T Sigma */
        double dSig[9], dT[6], GT[6];
        for (int r = 0; r < 2; ++r)
            for (int c2 = 0; c2 < 3; ++c2)
                GT[r * 3 + c2] = Gm[r * 2 + 0] * Tm[c2] + Gm[r * 2 + 1] * Tm[3 + c2];
        for (int r = 0; r < 3; ++r)
            for (int c2 = 0; c2 < 3; ++c2)
                dSig[r * 3 + c2] = Tm[r] * GT[c2] + Tm[3 + r] * GT[3 + c2];
        for (int r = 0; r < 2; ++r)
            for (int c2 = 0; c2 < 3; ++c2) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += GT[r * 3 + k] * Sig[k * 3 + c2];
                dT[r * 3 + c2] = 2.0 * acc;
            }
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int c2 = 0; c2 < 3; ++c2) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += dT[r * 3 + k] * Rw[c2 * 3 + k];
                dJ[r * 3 + c2] = acc;
            }
        double dt[3] = { 0, 0, 0 };
        double drx_dtx = clx ? 0.0 : 1.0 / tz, drx_dtz = clx ? 0.0 : -t[0] / (tz * tz);
        double dry_dty = cly ? 0.0 : 1.0 / tz, dry_dtz = cly ? 0.0 : -t[1] / (tz * tz);
        dt[2] += dJ[0] * (-fx / (tz * tz)) + dJ[4] * (-fy / (tz * tz));
        dt[2] += dJ[2] * (fx * rx / (tz * tz) - fx / tz * drx_dtz);
        dt[2] += dJ[5] * (fy * ry / (tz * tz) - fy / tz * dry_dtz);
        dt[0] += dJ[2] * (-fx / tz * drx_dtx);
        dt[1] += dJ[5] * (-fy / tz * dry_dty);
        /* projected mean */
        dt[0] += G[0] * fx / tz;
        dt[1] += G[1] * fy / tz;
        dt[2] += G[0] * (-fx * t[0] / (tz * tz)) + G[1] * (-fy * t[1] / (tz * tz));
        for (int k = 0; k < 3; ++k)
            g_means[3 * i + k] += Rw[0 * 3 + k] * dt[0] + Rw[1 * 3 + k] * dt[1] + Rw[2 * 3 + k] * dt[2];
        /* Sigma = M M^T, M = R diag(s) */
        double dM[9], M[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) M[r * 3 + k] = R[r * 3 + k] * s[k];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += dSig[r * 3 + l] * M[l * 3 + k];
                dM[r * 3 + k] = 2.0 * acc;
            }
        double dR[9];
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int r = 0; r < 3; ++r) acc += dM[r * 3 + k] * R[r * 3 + k];
            g_scales[3 * i + k] = acc;
            for (int r = 0; r < 3; ++r) dR[r * 3 + k] = dM[r * 3 + k] * s[k];
        }
        double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
        double Rw_[9] = { 0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0 };
        double Rx_[9] = { 0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x };
        double Ry_[9] = { -4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y };
        double Rz_[9] = { -4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0 };
        double dqh[4] = { 0, 0, 0, 0 };
        for (int k = 0; k < 9; ++k) {
            dqh[0] += dR[k] * Rw_[k]; dqh[1] += dR[k] * Rx_[k];
            dqh[2] += dR[k] * Ry_[k]; dqh[3] += dR[k] * Rz_[k];
        }
        double proj = qh[0] * dqh[0] + qh[1] * dqh[1] + qh[2] * dqh[2] + qh[3] * dqh[3];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] = (dqh[k] - qh[k] * proj) / qn;
        g_opac[i] = G[5];
        /* SH colour */
        double d[3] = { mu[0] - cam[CAM_POS], mu[1] - cam[CAM_POS + 1], mu[2] - cam[CAM_POS + 2] };
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dir[3] = { d[0] / dn, d[1] / dn, d[2] / dn };
        double Y[16], dY[16][3];
        sh_grad(sh_degree, dir, Y, dY);
        double gdir[3] = { 0, 0, 0 };
        for (int ch = 0; ch < 3; ++ch) {
            if (clamped[3 * i + ch]) continue;
            double gr = G[6 + ch];
            for (int k = 0; k < Ksh; ++k) {
                g_sh[(i * Ksh + k) * 3 + ch] = Y[k] * gr;
                double shv = sh[(i * Ksh + k) * 3 + ch];
                for (int c2 = 0; c2 < 3; ++c2) gdir[c2] += gr * shv * dY[k][c2];
            }
        }
        double pr = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        for (int k = 0; k < 3; ++k) g_means[3 * i + k] += (gdir[k] - dir[k] * pr) / dn;
    }
    free(uv); free(depth); free(dbits); free(conic); free(radius); free(rect); free(tiles);
    free(rgb); free(clamped); free(gfl); free(keys); free(vals); free(ranges); free(G2);
    free(lid); free(lal); free(lT); free(lep); free(lcl);
}
