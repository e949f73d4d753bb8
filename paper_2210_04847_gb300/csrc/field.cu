// field.cu -- procedural radiance field standing in for the user's network in
// benchmarks (sum of Gaussian density blobs, sigmoid-linear colour). Not part
// of the marching/rendering method; built as its own library.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nacc_field.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlobs = 1024;

__device__ __forceinline__ float blob_density(const float* tab, int n_blobs, float x, float y, float z, float t) {
    float s = 0.0f;
    for (int b = 0; b < n_blobs; ++b) {
        const float* q = tab + 8 * b;
        const float dx = x - (q[0] + q[5] * t);
        const float dy = y - (q[1] + q[6] * t);
        const float dz = z - (q[2] + q[7] * t);
        s += q[4] * __expf(-(dx * dx + dy * dy + dz * dz) * q[3]);
    }
    return s;
}

__global__ void __launch_bounds__(kThreads) samples_kernel(const float* rays_o, const float* rays_d,
                                                          const float* ray_time, const int32_t* ri,
                                                          const float* ts, const float* te, int64_t n,
                                                          const float* blobs, int n_blobs, const float* wb,
                                                          float* sigmas, float* rgbs) {
    extern __shared__ float tab[];
    for (int k = threadIdx.x; k < 8 * n_blobs; k += blockDim.x) tab[k] = blobs[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int r = ri[i];
        const float mid = (ts[i] + te[i]) * 0.5f;
        const float x = rays_o[3 * (size_t)r] + rays_d[3 * (size_t)r] * mid;
        const float y = rays_o[3 * (size_t)r + 1] + rays_d[3 * (size_t)r + 1] * mid;
        const float z = rays_o[3 * (size_t)r + 2] + rays_d[3 * (size_t)r + 2] * mid;
        const float t = ray_time ? ray_time[r] : 0.0f;
        sigmas[i] = blob_density(tab, n_blobs, x, y, z, t);
        if (rgbs) {
            for (int c = 0; c < 3; ++c) {
                const float v = wb[3 * c] * x + wb[3 * c + 1] * y + wb[3 * c + 2] * z + wb[9 + c];
                rgbs[3 * i + c] = 1.0f / (1.0f + __expf(-v));
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) points_kernel(const float* xyz, const float* times, int64_t n,
                                                         const float* blobs, int n_blobs, float* sigmas) {
    extern __shared__ float tab[];
    for (int k = threadIdx.x; k < 8 * n_blobs; k += blockDim.x) tab[k] = blobs[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        sigmas[i] = blob_density(tab, n_blobs, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], times ? times[i] : 0.0f);
}

// Field at sample midpoints for a batch of scenes: the scene of sample i is the
// slot of its ray; scene s uses blob rows [blob_off[s], blob_off[s+1]) and colour
// weights rgb_wb[12 s .. 12 s + 11]. The sample count is read on the device
// (*n_dev, at most n_max), so the call can be captured in a CUDA graph.
__global__ void __launch_bounds__(kThreads) samples_multi_kernel(const float* rays_o, const float* rays_d,
                                                                const float* ray_time, const int32_t* ray_slot,
                                                                const int32_t* ri, const float* ts, const float* te,
                                                                const int64_t* n_dev, int64_t n_max,
                                                                const float* blobs, const int32_t* blob_off,
                                                                const float* wb_all, float* sigmas, float* rgbs) {
    int64_t n = *n_dev;
    if (n > n_max) n = n_max;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int r = ri[i];
        const int s = ray_slot ? ray_slot[r] : 0;
        const float mid = (ts[i] + te[i]) * 0.5f;
        const float x = rays_o[3 * (size_t)r] + rays_d[3 * (size_t)r] * mid;
        const float y = rays_o[3 * (size_t)r + 1] + rays_d[3 * (size_t)r + 1] * mid;
        const float z = rays_o[3 * (size_t)r + 2] + rays_d[3 * (size_t)r + 2] * mid;
        const float t = ray_time ? ray_time[r] : 0.0f;
        const int b0 = blob_off[s], b1 = blob_off[s + 1];
        sigmas[i] = blob_density(blobs + 8 * (size_t)b0, b1 - b0, x, y, z, t);
        if (rgbs) {
            const float* wb = wb_all + 12 * (size_t)s;
            for (int c = 0; c < 3; ++c) {
                const float v = wb[3 * c] * x + wb[3 * c + 1] * y + wb[3 * c + 2] * z + wb[9 + c];
                rgbs[3 * i + c] = 1.0f / (1.0f + __expf(-v));
            }
        }
    }
}

int grid_size(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

extern "C" int nacc_field_samples(const float* rays_o, const float* rays_d, const float* ray_time,
                                  const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                                  int64_t n, const float* blobs, int32_t n_blobs, const float* rgb_wb,
                                  float* sigmas, float* rgbs, void* stream) {
    if (n < 0 || n_blobs < 0 || n_blobs > kMaxBlobs) return -1;
    if (n == 0) return 0;
    const size_t smem = sizeof(float) * 8 * (size_t)n_blobs;
    if (smem > 48 * 1024) cudaFuncSetAttribute(samples_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    samples_kernel<<<grid_size(n), kThreads, smem, (cudaStream_t)stream>>>(
        rays_o, rays_d, ray_time, ray_indices, t_starts, t_ends, n, blobs, n_blobs, rgb_wb, sigmas, rgbs);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int nacc_field_samples_multi(const float* rays_o, const float* rays_d, const float* ray_time,
                                        const int32_t* ray_slot, const int32_t* ray_indices, const float* t_starts,
                                        const float* t_ends, const int64_t* n_dev, int64_t n_max, const float* blobs,
                                        const int32_t* blob_off, const float* rgb_wb, float* sigmas, float* rgbs,
                                        void* stream) {
    if (n_max < 0 || !n_dev) return -1;
    if (n_max == 0) return 0;
    samples_multi_kernel<<<grid_size(n_max), kThreads, 0, (cudaStream_t)stream>>>(
        rays_o, rays_d, ray_time, ray_slot, ray_indices, t_starts, t_ends, n_dev, n_max, blobs, blob_off, rgb_wb,
        sigmas, rgbs);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

extern "C" int nacc_field_points(const float* xyz, const float* times, int64_t n, const float* blobs,
                                 int32_t n_blobs, float* sigmas, void* stream) {
    if (n < 0 || n_blobs < 0 || n_blobs > kMaxBlobs) return -1;
    if (n == 0) return 0;
    const size_t smem = sizeof(float) * 8 * (size_t)n_blobs;
    if (smem > 48 * 1024) cudaFuncSetAttribute(points_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    points_kernel<<<grid_size(n), kThreads, smem, (cudaStream_t)stream>>>(xyz, times, n, blobs, n_blobs, sigmas);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
