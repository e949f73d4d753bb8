// device.cu -- host-side helpers of the library: the per-device SM count cache,
// error strings and the version query.
#include "nacc_internal.cuh"

namespace nacc {

DeviceInfo current_device() {
    static int sm_cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    DeviceInfo info{dev, 0};
    if (dev >= 0 && dev < 64) {
        if (sm_cache[dev] == 0) {
            int n = 0;
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            sm_cache[dev] = n > 0 ? n : 1;
        }
        info.sm_count = sm_cache[dev];
    } else {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        info.sm_count = n > 0 ? n : 1;
    }
    return info;
}

}  // namespace nacc

extern "C" const char* nacc_error_string(int code) {
    switch (code) {
        case NACC_OK: return "ok";
        case NACC_ERR_INVALID_ARG: return "invalid argument";
        case NACC_ERR_CAPACITY: return "output capacity exceeded";
        case NACC_ERR_CUDA: return "CUDA launch or runtime error";
        case NACC_ERR_TIMEOUT: return "bounded device wait timed out";
        case NACC_ERR_INTERNAL: return "internal error";
        default: return "unknown error code";
    }
}

extern "C" int nacc_version(void) { return NACC_VERSION; }
