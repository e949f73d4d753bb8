// march_static.cu -- ray marching for callers that cannot allocate device memory.
//
// nacc_march_rays takes its scratch (the tile ticket and the per-tile look-back
// words) from a workspace the caller allocates. Some callers cannot do that: code
// running where every allocation must be planned up front (a real-time renderer
// with a fixed memory budget, a plugin inside a host application that owns the
// CUDA allocator, a process whose allocator is locked after start-up).
// nacc_march_rays_static gives them the same marching with the scratch held in a
// fixed array in this library's own device memory, so a call allocates nothing.
// The caller still provides the inputs and outputs.
#include <mutex>

#include "nacc_internal.cuh"

namespace {

// Ticket (256 bytes) + one look-back word per ray, for up to NACC_STATIC_MAX_RAYS
// rays, then the cone-step lattice table (t_0 .. t_max_steps, float32) for the
// largest max_steps any marching call accepts (32768), each part rounded up to
// 256 bytes as nacc_march_workspace_size lays them out. Every valid call fits.
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticStatusBytes =
    (256 + (size_t)NACC_STATIC_MAX_RAYS * sizeof(unsigned long long) + 255) / 256 * 256;
constexpr size_t kStaticTableBytes = ((size_t)(NACC_STATIC_MAX_STEPS + 1) * sizeof(float) + 255) / 256 * 256;
constexpr size_t kStaticScratchBytes = kStaticStatusBytes + kStaticTableBytes;
static __device__ __align__(256) unsigned char g_march_scratch[kStaticScratchBytes];

// Device address of g_march_scratch per device. In host code the array's name is
// only a host-side stand-in, never a device address: the address is looked up
// with cudaGetSymbolAddress once per device, with that device current.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NACC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_march_scratch) != cudaSuccess || !p) return NACC_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NACC_OK;
}

}  // namespace

extern "C" int nacc_march_rays_static(const float* rays_o, const float* rays_d, const float* ray_time,
                                      const int32_t* ray_slot, int32_t n_rays, const nacc_grid* grid,
                                      const nacc_march_params* params, int32_t* packed_info, float* t_starts,
                                      float* t_ends, int32_t* ray_indices, int64_t capacity, int64_t* n_samples,
                                      int32_t* d_status, void* stream) {
    if (n_rays < 0 || n_rays > NACC_STATIC_MAX_RAYS) return NACC_ERR_INVALID_ARG;
    void* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != NACC_OK) return rc;
    if (nacc_march_workspace_size(n_rays, params) > kStaticScratchBytes) return NACC_ERR_INVALID_ARG;
    // nacc_march_rays clears the ticket and look-back words it uses on `stream`
    // before its kernel runs, so the previous call's contents do not matter.
    return nacc_march_rays(rays_o, rays_d, ray_time, ray_slot, n_rays, grid, params, packed_info, t_starts, t_ends,
                           ray_indices, capacity, n_samples, d_status, scratch, kStaticScratchBytes, stream);
}
