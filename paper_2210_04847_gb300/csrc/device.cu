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

namespace {
// Tuned launch-shape table: one int per knob, read at every launch.
int g_tune[NACC_TUNE_COUNT] = {
    0,  // NACC_TUNE_RENDER_FWD_PREFETCH
    4,  // NACC_TUNE_MARCH_TILE_RAYS (upper bound; long lattices use fewer)
    8,  // NACC_TUNE_PRUNE_TILE_RAYS
    0,  // NACC_TUNE_MARCH_OCCUPANCY
    2,  // NACC_TUNE_PRUNE_OCCUPANCY
    2,  // NACC_TUNE_RENDER_OCCUPANCY
    2,  // NACC_TUNE_RENDER_BWD_OCCUPANCY
    0,  // NACC_TUNE_MARCH_UNROLL
    2,  // NACC_TUNE_PRUNE_INTERLEAVE
    0,  // NACC_TUNE_RENDER_BWD_PREFETCH
    0,  // NACC_TUNE_MARCH_COARSE
    1,  // NACC_TUNE_FUSED_OCCUPANCY
    0,  // NACC_TUNE_MARCH_BOX_TILE
    0,  // NACC_TUNE_RENDER_FWD_STAGES
    2,  // NACC_TUNE_RENDER_BWD_STAGES
    2,  // NACC_TUNE_RENDER_MSE_OCCUPANCY
};
const int g_tune_lo[NACC_TUNE_COUNT] = {0, 1, 2, 0, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0};
const int g_tune_hi[NACC_TUNE_COUNT] = {1, 32, 32, 1, 2, 2, 2, 1, 4, 1, 1, 1, 3, 4, 4, 2};
}  // namespace

int tune_get(int knob) { return (knob >= 0 && knob < NACC_TUNE_COUNT) ? g_tune[knob] : 0; }

namespace {
// Test hooks of the look-back waits, read at every launch (defaults: the full
// poll budget, every tile publishes).
int g_hook[NACC_TEST_HOOK_COUNT] = {kSpinLimit, 0, 0};
const int g_hook_lo[NACC_TEST_HOOK_COUNT] = {0, 0, 0};
const int g_hook_hi[NACC_TEST_HOOK_COUNT] = {kSpinLimit, 1, 1};
}  // namespace

LookbackHooks lookback_hooks() {
    return LookbackHooks{g_hook[NACC_TEST_HOOK_WITHHOLD_FIRST_TILE] ? 0ull : kFlagInc, g_hook[NACC_TEST_HOOK_SPIN_LIMIT],
                         g_hook[NACC_TEST_HOOK_OVERSTATE_STAGE_BYTES]};
}

}  // namespace nacc

extern "C" int nacc_tune_set(int knob, int value) {
    if (knob < 0 || knob >= NACC_TUNE_COUNT) return NACC_ERR_INVALID_ARG;
    if (value < nacc::g_tune_lo[knob] || value > nacc::g_tune_hi[knob]) return NACC_ERR_INVALID_ARG;
    if (knob == NACC_TUNE_PRUNE_TILE_RAYS && (value & 1)) return NACC_ERR_INVALID_ARG;
    if (knob == NACC_TUNE_PRUNE_INTERLEAVE && value != 2 && value != 4) return NACC_ERR_INVALID_ARG;
    if ((knob == NACC_TUNE_RENDER_FWD_STAGES || knob == NACC_TUNE_RENDER_BWD_STAGES) && value == 1)
        return NACC_ERR_INVALID_ARG;
    nacc::g_tune[knob] = value;
    return NACC_OK;
}

extern "C" int nacc_tune_get(int knob) {
    if (knob < 0 || knob >= NACC_TUNE_COUNT) return NACC_ERR_INVALID_ARG;
    return nacc::g_tune[knob];
}

extern "C" int nacc_test_hook_set(int hook, int value) {
    if (hook < 0 || hook >= NACC_TEST_HOOK_COUNT) return NACC_ERR_INVALID_ARG;
    if (value < nacc::g_hook_lo[hook] || value > nacc::g_hook_hi[hook]) return NACC_ERR_INVALID_ARG;
    nacc::g_hook[hook] = value;
    return NACC_OK;
}

extern "C" int nacc_test_hook_get(int hook) {
    if (hook < 0 || hook >= NACC_TEST_HOOK_COUNT) return NACC_ERR_INVALID_ARG;
    return nacc::g_hook[hook];
}

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
