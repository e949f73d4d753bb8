/*
 * nacc_field.h -- procedural stand-in for the user's radiance field (the
 * paper's sigma_fn / rgb_sigma_fn callbacks, Sec. 3 listing), used only to
 * drive benchmarks and examples on the GPU. It is NOT part of the method: the
 * marching/rendering library never calls it.
 *
 * Field: sigma(x, t) = sum_b p_b exp(-|x - (c_b + v_b t)|^2 k_b) with
 * k_b = 1/(2 s_b^2); rgb(x) = sigmoid(W x + b). Blob table rows are
 * (cx, cy, cz, k, p, vx, vy, vz) float32; rgb_wb is W (3x3, row-major) then b.
 * Pointers are device pointers; `stream` is a cudaStream_t as void*.
 */
#ifndef NACC_FIELD_H
#define NACC_FIELD_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Field at sample midpoints x = o_r + d_r (t_s + t_e)/2, r = ray_indices[i]
 * (the point the paper's callbacks query). ray_time nullable (t = 0).
 * sigmas (n,) out; rgbs (n,3) out or NULL. Returns 0 or a negative error. */
int nacc_field_samples(const float* rays_o, const float* rays_d, const float* ray_time,
                       const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                       int64_t n, const float* blobs, int32_t n_blobs, const float* rgb_wb,
                       float* sigmas, float* rgbs, void* stream);

/* Batch of scenes: the scene of a sample is the slot of its ray (ray_slot nullable =
 * scene 0); scene s owns blob rows [blob_off[s], blob_off[s+1]) and colour weights
 * rgb_wb[12 s ...]. The sample count is read from the device (*n_dev, at most
 * n_max), so the call can be captured in a CUDA graph. */
int nacc_field_samples_multi(const float* rays_o, const float* rays_d, const float* ray_time,
                             const int32_t* ray_slot, const int32_t* ray_indices, const float* t_starts,
                             const float* t_ends, const int64_t* n_dev, int64_t n_max, const float* blobs,
                             const int32_t* blob_off, const float* rgb_wb, float* sigmas, float* rgbs,
                             void* stream);

/* Density at points xyz (n,3); times (n,) nullable (t = 0). */
int nacc_field_points(const float* xyz, const float* times, int64_t n, const float* blobs,
                      int32_t n_blobs, float* sigmas, void* stream);

#ifdef __cplusplus
}
#endif
#endif
