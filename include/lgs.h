/*
 * lgs.h -- C ABI of the GB300 (sm_103a) Local-GS 3D Gaussian Splatting
 * rasterizer.
 *
 * The library renders N anisotropic 3D Gaussians (mean, scale, rotation,
 * opacity, SH colour; Local-GS Sec. II-A) seen by one or more pinhole cameras
 * into an RGB image, its final transmittance T and the per-pixel contributor
 * count, through the three stages of the 3DGS rasterization pipeline
 * (Sec. II-A, Fig. 2): preprocess, duplicate + sort by (tile, depth) keys,
 * per-tile render. The render stage implements Local-GS (Sec. III): tile-local
 * parameter hoisting (Sec. III-B, Eq. hoist transform), warp-level culling with
 * the tight box and 8-bit warp mask (Sec. III-C), and warp-coherent blending
 * (Sec. III-D, Alg. 1 right column) -- alongside a plain per-pixel tiled
 * kernel (Alg. 1 left column) for comparison. The backward entry point is the
 * adjoint of the same forward map.
 *
 * Conventions (all entry points):
 *  - Every buffer is caller-owned. The library never allocates or frees memory;
 *    scratch comes from a caller-provided workspace whose size a *_workspace_size
 *    query returns.
 *  - Device pointers are CUDA device addresses on the current device; `stream`
 *    is a cudaStream_t (NULL = legacy default stream). All work is enqueued
 *    asynchronously on that stream; no entry point synchronises except
 *    lgs_read_status and lgs_get_device_status. Calls are therefore
 *    capturable in a CUDA graph.
 *  - Host-checkable errors (NULL pointers, bad sizes, misalignment, unsupported
 *    tile shapes or SH degrees) return a non-zero lgs_status before anything is
 *    enqueued. Errors detected on the device (instance capacity exceeded,
 *    bounded waits that gave up) are recorded in the caller's device status
 *    buffer `d_status` (LGS_STATUS_WORDS int64 words, zeroed by the caller
 *    before the first call of a frame) and read back with lgs_read_status.
 *  - Arrays loaded as float4 (marked "16-B aligned") must start on a 16-byte
 *    boundary, otherwise LGS_ERR_ALIGN.
 *  - No C++ exception crosses the ABI. The library holds no mutable global
 *    state, except the static scratch array of lgs_sort_static and its cached
 *    per-device address.
 *
 * Multi-view batches: n_views cameras (1..LGS_MAX_VIEWS) are processed in one
 * call. Per-(view, Gaussian) arrays are view-major, index v*N + i. Tile ids are
 * global across the batch: tile_id = (tiles of views 0..v-1) + ty*gx + tx.
 * Per-pixel outputs are concatenated per view: view v's image starts at pixel
 * offset P_v = sum_{u<v} W_u*H_u; rgb is channel-major within a view
 * (rgb[3*P_v + c*H_v*W_v + y*W_v + x]); final_T and n_contrib at P_v + y*W_v + x.
 */
#ifndef LGS_H
#define LGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lgs_status;
#define LGS_OK 0
#define LGS_ERR_ARG 1          /* NULL pointer, negative or inconsistent size */
#define LGS_ERR_ALIGN 2        /* a float4-loaded array is not 16-byte aligned */
#define LGS_ERR_UNSUPPORTED 3  /* tile shape, SH degree or view count not supported */
#define LGS_ERR_CAPACITY 4     /* instance capacity too small (device: needed K in detail) */
#define LGS_ERR_NONFINITE 5    /* reserved: non-finite inputs are counted, not fatal */
#define LGS_ERR_TIMEOUT 6      /* a bounded device-side wait gave up */
#define LGS_ERR_CUDA 7         /* a CUDA launch failed (detail = cudaError_t) */
#define LGS_ERR_INTERNAL 8     /* device-side consistency check failed (a library bug); outputs are invalid */

#define LGS_MAX_VIEWS 64
#define LGS_MAX_SH_DEGREE 3

/* Device status buffer: LGS_STATUS_WORDS int64 words, caller-zeroed. */
#define LGS_STATUS_WORDS 8
#define LGS_ST_CODE 0           /* first device-side error code (0 = none) */
#define LGS_ST_DETAIL 1         /* detail of that error (e.g. needed capacity) */
#define LGS_ST_NUM_INSTANCES 2  /* K, written by lgs_sort */
#define LGS_ST_NONFINITE 3      /* Gaussians with non-finite inputs (culled), accumulated */
#define LGS_ST_PAIRS 4          /* pixel-Gaussian pairs of the render schedule (LGS_FLAG_COUNT) */
#define LGS_ST_QUEUE 5          /* work-queue counter of the persistent render (library-owned) */
#define LGS_ST_QUEUE_BWD 6      /* work-queue counter of the persistent backward (library-owned) */
#define LGS_ST_CANDIDATES 7     /* (warp, Gaussian) candidates the Local-GS render's warps scanned
                                   before their exit (LGS_FLAG_COUNT); 1 - PAIRS/32/CANDIDATES is
                                   the fraction the warp mask culled */

/* Pinhole camera. Pixel (x, y) is sampled at the integer position (x, y);
 * u = fx * X/Z + cx, v = fy * Y/Z + cy for a camera-space point (X, Y, Z).
 * viewmat is the row-major 4x4 world-to-camera transform with OpenCV axes
 * (x right, y down, z forward); only its top 3x4 block is read. campos is the
 * camera centre in world space (used for the SH view direction); bg the
 * background colour composited with the final transmittance. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[16];
    float campos[3];
    float bg[3];
} lgs_camera;

/* Scene: N Gaussians, structure-of-arrays, float32, device memory.
 * means [N,3]; scales [N,3] (already exponentiated); quats [N,4] (w,x,y,z, any
 * non-zero norm); opacities [N] (already in (0,1)); sh [N,(d+1)^2,3] with
 * d = sh_degree in 0..3 (16-B aligned). */
typedef struct {
    int64_t n;
    int32_t sh_degree;
    const float* means;
    const float* scales;
    const float* quats;
    const float* opacities;
    const float* sh;
} lgs_gaussians;

#define LGS_MODE_LOCALGS 0      /* hoisting + warp culling + warp-coherent blending */
#define LGS_MODE_PLAIN 1        /* per-pixel global-coordinate loop with per-pixel branches */
/* Forward-only study variants of the Local-GS kernel (lgs_render_bwd and
 * LGS_FLAG_PERSISTENT reject them):
 * LGS_MODE_LITERAL: Alg. 1 right column read literally -- no per-pixel 1/255
 *   test (the warp mask is the only culling) and no per-pixel stop: every
 *   Gaussian whose warp bit is set blends with w = alpha T, C += f w, T -= w,
 *   until all 32 pixels of the warp have T < 1e-4 (checked before each
 *   Gaussian). n_contrib = position of the last Gaussian the warp processed.
 * LGS_MODE_GLOBAL: the contract of LGS_MODE_LOCALGS with the hoisted
 *   coefficients expressed in global pixel coordinates (origin at pixel 0,0)
 *   instead of the tile frame: the "w/o local coordinates" configuration of
 *   Sec. III-B4 / Table V, whose FP32 cancellation grows with the image size. */
#define LGS_MODE_LITERAL 2
#define LGS_MODE_GLOBAL 3

#define LGS_FLAG_COUNT 1        /* render also counts its schedule's pixel-Gaussian pairs into d_status[LGS_ST_PAIRS] */
#define LGS_FLAG_PERSISTENT 2   /* render and adjoint (LGS_MODE_LOCALGS) with persistent CTAs pulling tiles from a work queue */
/* Tight-box emission (lgs_sort): an entry is duplicated only into the tiles of
 * its rect that the conservative tight box of Sec. III-C2 reaches, evaluated
 * per tile column strip (the ellipse alpha = 1/255 widened to
 * tau' = 1.001 tau + 0.02 and by 1/64 px; the same box whose rows give the
 * render's warp mask), instead of every tile of the rect. A dropped
 * (Gaussian, tile) pair has alpha < 1/255 at every pixel of the tile, so
 * images are unchanged; K, the tile lists and the list positions in n_contrib
 * shrink. lgs_sort then also reads pre->xy and pre->conic. The other entry
 * points ignore the flag (they follow the lists they are given). */
#define LGS_FLAG_TIGHT 4
/* lgs_sort: run every radix pass as one single-kernel "onesweep" pass
 * (decoupled look-back over earlier blocks' digit counts) instead of the
 * default three fully parallel reduce-then-scan kernels. Results are
 * identical; only the speed differs. */
#define LGS_FLAG_ONESWEEP 8

/* Tile shape, render mode and flags. Tiles of 256 pixels: 16x16, 8x32, 32x8.
 * Larger tiles, 32x32, 16x32 and 32x16: sorted as one tile (fewer
 * (Gaussian, tile) instances to duplicate and sort), rendered (and
 * differentiated) by one CTA per 16x16 region, each walking the whole tile
 * list with 8x8 warp blocks; LGS_MODE_LOCALGS only (the other modes return
 * LGS_ERR_UNSUPPORTED for them).
 * batch = Gaussians the Local-GS render (LGS_MODE_LOCALGS) stages in shared
 * memory per round: 0 (= 256), 64, 128 or 256, else LGS_ERR_UNSUPPORTED; the
 * results do not depend on it. The other render modes stage 256, the adjoint 128.
 * warp_w x warp_h = the pixel block one warp of the Local-GS render owns, with
 * its own bit of the culling mask (Sec. III-C3; the paper's layout, and the
 * default 0 x 0, is eight full-width strips of tile_h/8 rows). Blocks of 32
 * pixels run one pixel per lane, blocks of 64 pixels two pixels per lane with
 * packed two-wide FP32 arithmetic (4 warps per tile). Supported: 16x16 tiles
 * with 16x2, 8x4 (2 x 4 blocks: the mask also culls by column half), 16x4 or
 * 8x8 blocks; 8x32 tiles with 8x4 or 8x8; 32x8 tiles with 32x1 or 8x8. Other
 * blocks, or a non-default block with LGS_MODE_PLAIN/LITERAL/GLOBAL, return
 * LGS_ERR_UNSUPPORTED; the larger tiles take 8x8 blocks (0 x 0 or 8 x 8).
 * Outputs do not depend on the block layout (bit for bit); only the work the
 * mask saves does. Other entry points ignore the two fields. */
typedef struct {
    int32_t tile_w, tile_h;
    int32_t mode;
    int32_t batch;
    int32_t flags;
    int32_t warp_w, warp_h;
} lgs_config;

/* Per-(view, Gaussian) preprocess outputs, M = n_views * N entries each,
 * device memory owned by the caller.
 *   xy      [M,4] f32 16-B aligned: (u_hi, v_hi, u_lo, v_lo), the projected mean
 *           as an unevaluated float pair u = u_hi + u_lo (about 48 bits)
 *   conic   [M,4] f32 16-B aligned: (a, b, c, o) with Sigma'^-1 = [[a,b],[b,c]]
 *   rgb     [M,4] f32 16-B aligned: (r, g, b, depth)
 *   depth   [M]   f32 camera-space z
 *   radius  [M]   i32 ceil(3 sqrt(lambda_max)), 0 when culled
 *   tiles   [M]   u32 number of tiles in the rect, 0 when culled
 *   rect    [M]   u64 tile rect packed as x_lo | y_lo<<16 | x_hi<<32 | y_hi<<48 (half-open)
 *   flags   [M]   u8  bit c (c<3): colour channel c was clamped at 0;
 *                     bit 3/4: x/z resp. y/z clamped to 1.3 tan(fov/2) in the EWA Jacobian
 *   emit    [M,8] u32 32-B aligned, optional (NULL = not written / not read):
 *           for visible entries the fields the tight-box emission of lgs_sort
 *           needs, in one 32-B record: (rect lo32, rect hi32, bits(u_hi + u_lo),
 *           bits(v_hi + v_lo), bits(a), bits(b), bits(c), bits(o)). lgs_sort with
 *           LGS_FLAG_TIGHT then gathers one record per entry instead of reading
 *           rect, xy and conic; results are identical either way. */
typedef struct {
    float* xy;
    float* conic;
    float* rgb;
    float* depth;
    int32_t* radius;
    uint32_t* tiles;
    uint64_t* rect;
    uint8_t* flags;
    uint32_t* emit;
} lgs_pre_out;

/* Gradients (device, caller-zeroed; the per-Gaussian ones are added to, the
 * per-entry scratch ones accumulated with atomics).
 * means [N,3], scales [N,3], quats [N,4] (16-B aligned), opacities [N],
 * sh [N,(d+1)^2,3] (16-B aligned for d = 1 and 3). The *_2d buffers are per-(view, Gaussian) scratch gradients of the render
 * stage, M = n_views*N entries: xy2d [M,2] (8-B aligned), conic2d [M,4] (a, b, c, o;
 * 16-B aligned), rgb2d [M,4] (r, g, b, unused; 16-B aligned); otherwise
 * lgs_render_bwd returns LGS_ERR_ALIGN. */
typedef struct {
    float* means;
    float* scales;
    float* quats;
    float* opacities;
    float* sh;
    float* xy2d;
    float* conic2d;
    float* rgb2d;
} lgs_grads;

/* Stage 1, preprocess (Sec. II-A; Fig. 2 "preprocessing"): per view and
 * Gaussian, near-plane cull (z <= 0.2), EWA projection of the covariance with
 * the 0.3 px low-pass term, conic, radius, tile rect, SH colour in the view
 * direction and depth. Non-finite inputs cull the Gaussian and are counted in
 * d_status[LGS_ST_NONFINITE]. Writes every field of *out for all M entries. */
lgs_status lgs_preprocess(const lgs_gaussians* g, const lgs_camera* cams, int32_t n_views,
                          const lgs_config* cfg, const lgs_pre_out* out, int64_t* d_status,
                          void* stream);

/* Workspace bytes of lgs_sort for M = n_views*N entries and an instance
 * capacity (upper bound of K = sum of tiles). */
size_t lgs_sort_workspace_size(int64_t m, int64_t capacity);

/* Stage 2, duplicate + sort (Sec. II-A: "a parallel prefix scan duplicates the
 * surviving primitives across intersecting tiles into 64-bit key-value pairs,
 * which are sorted by GPU radix sort to produce ... tile ranges"):
 * exclusive scan of tiles, emission of key = (tile_id << 32) | bits(depth) and
 * value = v*N + i in Gaussian order (tiles row-major inside the rect; with
 * LGS_FLAG_TIGHT only the tiles the tight box reaches), a stable radix sort by
 * key (ties keep emission order), and per-tile ranges [start, end) (0,0 for
 * empty tiles).
 * keys [capacity] u64 (may be NULL: the sorted keys are then not written),
 * vals [capacity] u32, ranges [n_tiles_total,2] u32 (all device, caller-owned,
 * keys and ranges 8-B aligned). K is written to d_status[LGS_ST_NUM_INSTANCES]; if
 * K > capacity nothing is sorted, d_status records LGS_ERR_CAPACITY with K as
 * detail and ranges are left empty. capacity must be < 2^32. */
lgs_status lgs_sort(const lgs_pre_out* pre, int64_t n, const lgs_camera* cams, int32_t n_views,
                    const lgs_config* cfg, int64_t capacity, uint64_t* keys, uint32_t* vals,
                    uint32_t* ranges, void* workspace, size_t workspace_bytes, int64_t* d_status,
                    void* stream);

/* lgs_sort without a workspace argument. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at all --
 * for example a plugin inside a host engine that owns every device allocation
 * and forbids third-party code from calling cudaMalloc, or a real-time render
 * loop that must never enter an allocator after start-up -- and so cannot hand
 * lgs_sort a workspace. Its scratch is a file-scope __device__ array of
 * LGS_SORT_STATIC_BYTES that every GPU loading the library holds until exit;
 * the call itself allocates nothing (no cudaMalloc, no allocating library
 * routine).
 * Limits: n * n_views <= LGS_SORT_STATIC_MAX_ENTRIES and capacity <=
 * LGS_SORT_STATIC_MAX_INSTANCES, otherwise LGS_ERR_UNSUPPORTED is returned
 * before anything is enqueued. Other arguments, outputs and errors are those of
 * lgs_sort.
 * The array belongs to the library's sort module: with CUDA's lazy module
 * loading (the default) that module, and with it the array, is loaded on a
 * device by the first call of any sort entry point there (lgs_sort,
 * lgs_sort_static or lgs_selftest_wait_timeout). The first lgs_sort_static
 * call on a device also looks up the array's device address (once per device,
 * with that device current) and caches it for the life of the process. Make a
 * first sort call on each device before any stream capture. The cached address
 * belongs to the device's primary context: resetting the device
 * (cudaDeviceReset) or making another context current on it between calls is
 * not supported. All calls share the one array, which keeps the previous call's
 * contents (nothing in it needs to start at zero: every word the sort reads is
 * written earlier in the same call), so calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller. */
#define LGS_SORT_STATIC_MAX_ENTRIES (1ll << 18)
#define LGS_SORT_STATIC_MAX_INSTANCES (1ll << 20)
#define LGS_SORT_STATIC_BYTES (28ull << 20)
lgs_status lgs_sort_static(const lgs_pre_out* pre, int64_t n, const lgs_camera* cams,
                           int32_t n_views, const lgs_config* cfg, int64_t capacity,
                           uint64_t* keys, uint32_t* vals, uint32_t* ranges, int64_t* d_status,
                           void* stream);

/* Stage 3, render (Sec. II-A render kernel; Local-GS Sec. III or the plain
 * per-pixel kernel, cfg->mode). Per pixel, front to back over its tile's list:
 * alpha = min(0.99, o exp(-1/2 d^T Sigma'^-1 d)) (Eq. 3DGS alpha); Gaussians with
 * alpha < 1/255 are skipped; the pixel stops before the first Gaussian with
 * T(1-alpha) < 1e-4; C += rgb alpha T, T *= (1-alpha).
 * Outputs (device, concatenated per view, see header comment):
 *   rgb [3*P] f32 = C + T bg; final_T [P] f32; n_contrib [P] u32 = list
 *   position (1-based) of the last blended Gaussian. */
lgs_status lgs_render_fwd(const lgs_pre_out* pre, const uint32_t* vals, const uint32_t* ranges,
                          const lgs_camera* cams, int32_t n_views, const lgs_config* cfg,
                          float* rgb, float* final_T, uint32_t* n_contrib, int64_t* d_status,
                          void* stream);

/* Adjoint of stages 1 and 3 (no counterpart in the paper, which covers
 * inference only): given dL/drgb [3*P] and optionally dL/dfinal_T [P] (NULL =
 * zero), recomputes blending back to front per tile from the stored final_T
 * and n_contrib and accumulates gradients into *grads (caller-zeroed):
 * first the per-(view, Gaussian) 2D gradients, then the chain rule through
 * conic inverse, EWA, covariance, quaternion normalisation and SH.
 * cfg->mode LGS_MODE_LOCALGS or LGS_MODE_PLAIN (else LGS_ERR_UNSUPPORTED);
 * LGS_FLAG_PERSISTENT (Local-GS only) runs the adjoint with persistent CTAs
 * pulling tiles from the work queue d_status[LGS_ST_QUEUE_BWD]; the gradients
 * then differ from the one-CTA-per-tile launch only in the order of float
 * atomics. */
lgs_status lgs_render_bwd(const lgs_gaussians* g, const lgs_camera* cams, int32_t n_views,
                          const lgs_config* cfg, const lgs_pre_out* pre, const uint32_t* vals,
                          const uint32_t* ranges, const float* final_T, const uint32_t* n_contrib,
                          const float* dL_drgb, const float* dL_dfinal_T, const lgs_grads* grads,
                          int64_t* d_status, void* stream);

/* Failure-detection self-test (no counterpart in the paper). Every device-side
 * wait of the library (the look-back of the sort's radix passes) is bounded:
 * after a spin limit it records LGS_ERR_TIMEOUT in d_status and returns
 * instead of hanging. This entry point makes one such wait run out on purpose:
 * it launches a single radix-pass block that waits on a predecessor that never
 * runs, with the given spin limit (polls of an L2 word, ~0.5 us each), inside
 * the caller's workspace of LGS_SELFTEST_WORKSPACE_BYTES (device, 256-B
 * aligned). Afterwards d_status holds LGS_ERR_TIMEOUT with detail 1. Nothing
 * faults or traps; the context stays usable. */
#define LGS_SELFTEST_WORKSPACE_BYTES (256ull << 10)
lgs_status lgs_selftest_wait_timeout(int32_t spin_limit, void* workspace, size_t workspace_bytes,
                                     int64_t* d_status, void* stream);

/* Throughput probe of one SM pipe (a measurement utility; no counterpart in
 * the paper): enqueues `blocks` CTAs of 256 threads, each thread running 8
 * independent chains of 16 * iters dependent operations of the chosen kind,
 * and writes the operation count of the launch to *ops (host): FP32 flops for
 * LGS_PROBE_FFMA (scalar fused multiply-add, 2 flops each) and LGS_PROBE_FFMA2
 * (packed fma.rn.f32x2, 4 flops each), ex2.approx results for LGS_PROBE_EX2.
 * Dividing *ops by the launch's duration (caller-timed, e.g. CUDA events on
 * `stream`) gives the pipe's throughput at the clock the GPU ran at. d_sink
 * (device, >= blocks floats) only keeps the chains live; it is practically
 * never written. */
#define LGS_PROBE_FFMA 0
#define LGS_PROBE_FFMA2 1
#define LGS_PROBE_EX2 2
lgs_status lgs_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float* d_sink, double* ops,
                          void* stream);

/* Copies the LGS_STATUS_WORDS device status words into h_status after
 * synchronising `stream`. Returns LGS_ERR_CUDA if the copy fails. */
lgs_status lgs_read_status(const int64_t* d_status, int64_t* h_status, void* stream);

/* The first device-side error of d_status: synchronises `stream` and writes
 * the code word (LGS_ST_CODE, 0 = none) to *code and its detail word
 * (LGS_ST_DETAIL, e.g. the capacity the sort needed) to *detail. Either output
 * pointer may be NULL. Returns LGS_ERR_ARG for a NULL d_status, LGS_ERR_CUDA
 * if the copy fails. */
lgs_status lgs_get_device_status(const int64_t* d_status, void* stream, int32_t* code, int64_t* detail);

/* Static description of a status code. */
const char* lgs_status_string(lgs_status s);

/* Library version, (major << 16) | minor. */
int32_t lgs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LGS_H */
