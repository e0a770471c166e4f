// host.h -- host-side helpers of the liblgs entry points: view-table
// construction and argument validation. No allocation, no synchronisation.
#pragma once

#include <stdint.h>
#include <string.h>

#include "common.cuh"

namespace lgs {

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline bool tile_shape_ok(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 8 && th == 32) || (tw == 32 && th == 8) ||
           (tw == 32 && th == 32) || (tw == 16 && th == 32) || (tw == 32 && th == 16);
}

// Tiles of more than 256 pixels: sorted as one tile, rendered as 16x16 regions.
inline bool split_tile(int tw, int th) { return tw * th > 256; }

// The Local-GS render's warp block (see lgs_config): 0 x 0 selects the
// paper's full-width strips; returns false for an unsupported block.
inline bool warp_block(const lgs_config* cfg, int* wx, int* wy) {
    const int tw = cfg->tile_w, th = cfg->tile_h;
    int x = cfg->warp_w, y = cfg->warp_h;
    if (split_tile(tw, th)) {
        // the 16x16 regions of a large tile run in 8x8 blocks
        if (!((x == 0 && y == 0) || (x == 8 && y == 8))) return false;
        *wx = 8;
        *wy = 8;
        return true;
    }
    if (x == 0 && y == 0) { x = tw; y = th / 8; }
    const bool ok = (x == tw && y == th / 8) || (x == 8 && y == 8) ||
                    (tw == 16 && th == 16 && ((x == 8 && y == 4) || (x == 16 && y == 4)));
    if (!ok) return false;
    *wx = x;
    *wy = y;
    return true;
}

// Builds the per-view constant table. Tile ids and pixel offsets are global
// across the batch (views concatenated in order).
inline lgs_status make_views(const lgs_camera* cams, int32_t n_views, const lgs_config* cfg,
                             Views* vs) {
    if (!cams || !cfg || !vs) return LGS_ERR_ARG;
    if (n_views < 1 || n_views > LGS_MAX_VIEWS) return LGS_ERR_UNSUPPORTED;
    if (!tile_shape_ok(cfg->tile_w, cfg->tile_h)) return LGS_ERR_UNSUPPORTED;
    memset(vs, 0, sizeof(Views));
    vs->n = n_views;
    vs->tile_w = cfg->tile_w;
    vs->tile_h = cfg->tile_h;
    vs->flags = cfg->flags;
    uint64_t toff = 0, poff = 0;
    for (int v = 0; v < n_views; ++v) {
        const lgs_camera& c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 32768 || c.height > 32768) return LGS_ERR_ARG;
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return LGS_ERR_ARG;
        ViewRec& r = vs->v[v];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) r.R[i * 3 + j] = c.viewmat[i * 4 + j];
            r.t[i] = c.viewmat[i * 4 + 3];
            r.campos[i] = c.campos[i];
            r.bg[i] = c.bg[i];
        }
        r.fx = c.fx; r.fy = c.fy; r.cx = c.cx; r.cy = c.cy;
        r.W = c.width; r.H = c.height;
        r.gx = (c.width + cfg->tile_w - 1) / cfg->tile_w;
        r.gy = (c.height + cfg->tile_h - 1) / cfg->tile_h;
        r.tile_off = (uint32_t)toff;
        r.pix_off = (uint32_t)poff;
        toff += (uint64_t)r.gx * r.gy;
        poff += (uint64_t)c.width * c.height;
    }
    if (toff >= (1ull << 31) || poff >= (1ull << 31)) return LGS_ERR_UNSUPPORTED;
    vs->n_tiles = (uint32_t)toff;
    vs->n_pix = (uint32_t)poff;
    return LGS_OK;
}

inline lgs_status check_pre(const lgs_pre_out* pre) {
    if (!pre || !pre->xy || !pre->conic || !pre->rgb || !pre->depth || !pre->radius ||
        !pre->tiles || !pre->rect || !pre->flags)
        return LGS_ERR_ARG;
    if (!aligned16(pre->xy) || !aligned16(pre->conic) || !aligned16(pre->rgb))
        return LGS_ERR_ALIGN;
    if ((reinterpret_cast<uintptr_t>(pre->rect) & 7u) != 0) return LGS_ERR_ALIGN;
    if ((reinterpret_cast<uintptr_t>(pre->emit) & 31u) != 0) return LGS_ERR_ALIGN;
    return LGS_OK;
}

inline lgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LGS_OK : LGS_ERR_CUDA; }

}  // namespace lgs
