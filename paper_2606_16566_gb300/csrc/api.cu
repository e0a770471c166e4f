// api.cu -- status and version entry points of liblgs.
#include "common.cuh"
#include "host.h"

extern "C" lgs_status lgs_read_status(const int64_t* d_status, int64_t* h_status, void* stream) {
    if (!d_status || !h_status) return LGS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return LGS_ERR_CUDA;
    if (cudaMemcpy(h_status, d_status, sizeof(int64_t) * LGS_STATUS_WORDS, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return LGS_ERR_CUDA;
    return LGS_OK;
}

extern "C" lgs_status lgs_get_device_status(const int64_t* d_status, void* stream, int32_t* code,
                                            int64_t* detail) {
    if (!d_status) return LGS_ERR_ARG;
    int64_t h[2];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return LGS_ERR_CUDA;
    if (cudaMemcpy(h, d_status + LGS_ST_CODE, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LGS_ERR_CUDA;
    if (code) *code = (int32_t)h[0];
    if (detail) *detail = h[1];
    return LGS_OK;
}

extern "C" const char* lgs_status_string(lgs_status s) {
    switch (s) {
        case LGS_OK: return "ok";
        case LGS_ERR_ARG: return "invalid argument (null pointer or bad size)";
        case LGS_ERR_ALIGN: return "misaligned buffer (float4 arrays need 16-byte alignment)";
        case LGS_ERR_UNSUPPORTED: return "unsupported tile shape, SH degree or view count";
        case LGS_ERR_CAPACITY: return "instance capacity too small";
        case LGS_ERR_NONFINITE: return "non-finite input";
        case LGS_ERR_TIMEOUT: return "bounded device wait gave up";
        case LGS_ERR_CUDA: return "CUDA launch or copy failed";
        case LGS_ERR_INTERNAL: return "device-side consistency check failed";
        default: return "unknown status";
    }
}

extern "C" int32_t lgs_version(void) { return (0 << 16) | 1; }
