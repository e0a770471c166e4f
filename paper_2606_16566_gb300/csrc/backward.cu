// backward.cu -- adjoint of the render and preprocess stages.
#include "common.cuh"
#include "host.h"

extern "C" lgs_status lgs_render_bwd(const lgs_gaussians* g, const lgs_camera* cams,
                                     int32_t n_views, const lgs_config* cfg,
                                     const lgs_pre_out* pre, const uint32_t* vals,
                                     const uint32_t* ranges, const float* final_T,
                                     const uint32_t* n_contrib, const float* dL_drgb,
                                     const float* dL_dfinal_T, const lgs_grads* grads,
                                     int64_t* d_status, void* stream) {
    (void)g; (void)cams; (void)n_views; (void)cfg; (void)pre; (void)vals; (void)ranges;
    (void)final_T; (void)n_contrib; (void)dL_drgb; (void)dL_dfinal_T; (void)grads;
    (void)d_status; (void)stream;
    return LGS_ERR_UNSUPPORTED;
}
