/*
 * nacc.h -- C ABI of the GB300 (sm_103a) occupancy-grid ray marcher and packed
 * differentiable volume renderer (the method of NerfAcc, arXiv 2210.04847).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every pointer named in a signature is a DEVICE pointer into memory the
 *   caller owns (cudaMalloc / torch), unless the comment says "host". The
 *   library never allocates device memory; scratch comes from a caller
 *   workspace whose size is returned by the matching *_workspace_size() call.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call only enqueues work on that stream and returns; nothing
 *   synchronises the host. Results are valid once the stream reaches them.
 * - Return value (host): NACC_OK, or a negative NACC_ERR_* for arguments the
 *   host can reject (null pointer where one is required, negative size,
 *   unsupported parameter) and for launch failures (NACC_ERR_CUDA). Nothing is
 *   enqueued when the call fails.
 * - Device-side conditions (capacity exceeded, a bounded wait that gave up,
 *   inconsistent packed_info) are OR-ed into `*d_status` (a device int32 the
 *   caller zeroes; nullable = not reported) as NACC_STATUS_* bits. Kernels
 *   never trap; on such a condition they skip the offending access and finish.
 * - Arrays are contiguous, C order. Reals are float32, indices int32.
 *   "Samples" are packed ray-major: packed_info (n_rays, 2) int32 holds
 *   (offset, count) of each ray's run in the per-sample arrays
 *   t_starts (n,), t_ends (n,), ray_indices (n,) -- the layout of the paper's
 *   API listing (Sec. 3): packed_info, t_starts, t_ends, ray_indices.
 *   Sample totals must stay below 2^31 (offsets are int32).
 * - The sample interval of a ray r is [t_start, t_end] along o_r + t d_r;
 *   rays_d are expected to be unit length (Sec. 3 listing: "normalized
 *   directions"), but nothing depends on it.
 */
#ifndef NACC_H
#define NACC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NACC_VERSION 300

/* host return codes */
#define NACC_OK 0
#define NACC_ERR_INVALID_ARG (-1)
#define NACC_ERR_CAPACITY (-2)
#define NACC_ERR_CUDA (-3)
#define NACC_ERR_TIMEOUT (-4)
#define NACC_ERR_INTERNAL (-5)

/* device status bits, OR-ed into *d_status */
#define NACC_STATUS_CAPACITY 0x1    /* more samples than `capacity`; total still reported */
#define NACC_STATUS_TIMEOUT 0x2     /* a bounded inter-block wait gave up; outputs invalid */
#define NACC_STATUS_BAD_PACKED 0x4  /* a packed_info run lies outside [0, n_samples) */
#define NACC_STATUS_BAD_INDEX 0x8   /* a grid slot or cell index out of range (skipped) */
#define NACC_STATUS_OVERFLOW 0x10   /* a sample total reached 2^31 (int32 offsets) */

#define NACC_MAX_LEVELS 16

/*
 * Binary occupancy grid (Sec. 2.1, "Pruning Empty and Occluded Regions"; the
 * multi-level form follows the cascaded grids the paper's footnote cites for
 * large scenes). One bit per cell, packed into uint32 words over the flat cell
 * index
 *     cell = ((slot * n_levels + level) * res[0] + ix) * res[1] + iy) * res[2] + iz
 * (bit cell & 31 of word cell >> 5). Level 0 covers aabb = (lo xyz, hi xyz);
 * level l >= 1 covers the level-0 box scaled by 2^l about its centre. A slot is
 * an independent grid: a time bin of a dynamic scene, or a scene of a batch.
 *
 * contraction = 1 (unbounded scenes, Sec. 2.1 "Scene Contraction", with the
 * contraction of Mip-NeRF 360, its Eq. 10): one level; a point x is normalised
 * by the box, x_n = (x - c) * (1 / h) (c = (lo + hi) / 2, h = (hi - lo) / 2),
 * contracted, x_c = x_n if |x_n|^2 <= 1 else x_n * (2 - 1/|x_n|) / |x_n|, and
 * looked up in a grid spanning [-2, 2]^3: cell i = floor((x_c + 2) * res / 4).
 * All in float32, every operation rounded ((x0^2 + x1^2) + x2^2, IEEE sqrt and
 * division). Rays are not clipped by the box: they march [near_plane, far_plane].
 */
typedef struct nacc_grid {
    const uint32_t* bits; /* device, ceil(n_slots*n_levels*res0*res1*res2 / 32) words */
    int32_t res[3];       /* 1 .. 2^22 cells per axis; total cells over all slots and levels < 2^31 */
    int32_t n_levels; /* 1 .. NACC_MAX_LEVELS (1 with contraction) */
    int32_t n_slots;  /* >= 1 */
    float aabb[6];
    int32_t contraction; /* 0: boxes (cascade); 1: contracted unbounded space */
    const uint16_t* sat; /* device or NULL: the summed-area table of `bits`, see nacc_build_grid_sat */
} nacc_grid;

/*
 * Summed-area table of a grid (an acceleration structure of this library, not
 * part of the paper's method): for each slot and level g, one uint16 entry per
 * cell corner (x, y, z) in [0, res0] x [0, res1] x [0, res2],
 *     S_g[x][y][z] = number of occupied cells (i, j, k) of g with i < x, j < y, k < z
 * modulo 2^16, corners x-major and z fastest, grids in slot-major, level order.
 * Built from grid->bits on `stream`; rebuild it whenever the bits change.
 * Marching an uncontracted grid of up to four levels that carries its table
 * (nacc_grid.sat) decides every 32-point lattice chunk whose box of cells (from
 * the chunk's first point to the point after the chunk: every cell index of
 * every level is monotone along the ray) is all occupied or all empty from one
 * box count (exact for boxes of fewer than 2^16 cells). In a cascade the box is
 * taken at the first level the chunk can reach; it decides when every point
 * lies in that level (its box inside the level) or outside all levels (the
 * outermost). The other chunks are tested point by point. Results are identical
 * with and without the table (shared lattices; rays with their own cone
 * recurrence are always tested point by point). After the corners, from the
 * first 16-byte boundary of the buffer, the build also writes a brick summary:
 * 2 bits per block of 8^3 cells (clipped at the grid's faces; bit 0: no cell
 * occupied, bit 1: every cell occupied), 8 bricks per uint16 entry, bricks
 * x-major and z fastest, ceil(nb0 nb1 nb2 / 8) entries per grid with
 * nb_k = ceil(res_k / 8), grids in the table's order. When the summary of all
 * grids fits 16 KiB, marching keeps it in shared memory and decides a box that
 * lies within 2 x 2 x 2 bricks from it, without reading the table (same
 * decisions). sat: nacc_grid_sat_bytes() bytes (corners, then the summary),
 * 2-byte aligned; the corners over all slots and levels must number below 2^31.
 */
size_t nacc_grid_sat_bytes(const nacc_grid* grid);
int nacc_build_grid_sat(const nacc_grid* grid, uint16_t* sat, void* stream);

/*
 * Marching parameters (Sec. 3 listing: near_plane, far_plane; the step rule is
 * the paper's dense 1024-sample lattice of Sec. 4.1 generalised to
 * cone-growing steps). cone == 0: uniform steps t_k = near + k * dt_min.
 * cone > 0: t_{k+1} = t_k + clamp(t_k * cone, dt_min, dt_max).
 */
typedef struct nacc_march_params {
    float near_plane;
    float far_plane;
    float dt_min;
    float dt_max;
    float cone;
    int32_t max_steps; /* 1 .. 32768 lattice intervals per ray */
} nacc_march_params;

/* ------------------------------------------------------------------------- */
/* Ray marching (Sec. 2.1 "Ray Marching", "GPU Memory Efficiency")           */
/* ------------------------------------------------------------------------- */

/* Bytes of device workspace nacc_march_rays needs for n_rays rays. */
size_t nacc_march_workspace_size(int32_t n_rays, const nacc_march_params* params);

/*
 * Occupancy-grid ray marching with empty-space skipping, pruned while
 * marching (Sec. 2.1: samples are produced only in non-empty space, so memory
 * is never over-allocated). For every ray r (input order):
 *   1. clip o_r + t d_r against the outermost level box (slab test, float32),
 *      near = max(t_in, near_plane), far = min(t_out, far_plane); a ray that
 *      misses, has near >= far, or holds a non-finite component gets none;
 *   2. walk the lattice intervals [t_k, min(t_{k+1}, far)], t_k < far,
 *      k < max_steps;
 *   3. emit interval k iff the grid bit of the cell holding its midpoint
 *      o + d (t_s + t_e)/2 is set, looking up the finest level whose box holds
 *      the midpoint, in the grid slot of the ray.
 * Every floating-point step is a separately rounded IEEE float32 operation
 * (no contraction), so results are bit-reproducible.
 *
 * rays_o, rays_d   (n_rays, 3) float32.
 * ray_time         (n_rays,) float32 or NULL: slot = clamp(floor(time*n_slots), 0, n_slots-1).
 * ray_slot         (n_rays,) int32 or NULL: explicit slot (wins over ray_time);
 *                  with both NULL every ray uses slot 0. Out-of-range slots emit
 *                  nothing and raise NACC_STATUS_BAD_INDEX.
 * grid, params     host structs (read during the call only).
 * packed_info      (n_rays, 2) int32 out: (offset, count), offsets ray-major.
 * t_starts, t_ends (capacity,) float32 out; ray_indices (capacity,) int32 out.
 *                  Samples beyond `capacity` are not written.
 * n_samples        device int64 out: the total number of samples (also when it
 *                  exceeds capacity; then NACC_STATUS_CAPACITY is raised).
 * workspace        nacc_march_workspace_size() bytes, 256-byte aligned; the
 *                  call clears what it needs on `stream`. After the call, the
 *                  uint64 at byte offset 8 holds the number of lattice points
 *                  the call examined (summed over rays; a diagnostic).
 * Errors: NACC_ERR_INVALID_ARG for null required pointers, n_rays < 0,
 * capacity < 0, n_levels or max_steps out of range, res <= 0, a workspace too
 * small; NACC_ERR_CUDA if a launch fails.
 */
int nacc_march_rays(const float* rays_o, const float* rays_d, const float* ray_time,
                    const int32_t* ray_slot, int32_t n_rays, const nacc_grid* grid,
                    const nacc_march_params* params, int32_t* packed_info, float* t_starts,
                    float* t_ends, int32_t* ray_indices, int64_t capacity, int64_t* n_samples,
                    int32_t* d_status, void* workspace, size_t workspace_bytes, void* stream);

/*
 * One scene of a batch whose scenes each have their own occupancy grid
 * (Sec. 2.1: the grid is kept per scene). Same meaning as nacc_grid with one
 * slot: bits (device) holds the scene's levels from word 0, res, n_levels, aabb
 * and contraction as there. n_rays: the scene's rays, which are consecutive in
 * the batch, scenes in array order.
 */
typedef struct nacc_scene_desc {
    const uint32_t* bits;
    int32_t res[3];
    int32_t n_levels;
    float aabb[6];
    int32_t contraction; /* the same for every scene of a call */
    int32_t n_rays;
    const uint16_t* sat; /* NULL or the scene's summed-area table (nacc_build_grid_sat, one slot) */
} nacc_scene_desc;

/* Bytes of device workspace nacc_march_rays_batched needs. */
size_t nacc_march_batched_workspace_size(int32_t n_scenes, int32_t n_rays, const nacc_march_params* params);

/*
 * nacc_march_rays over a batch of scenes with per-scene grids, in one
 * persistent launch: ray r of scene s (rays of scene s are the n_rays of
 * scenes[s] that follow those of scenes 0..s-1) is clipped against scene s's
 * outermost box and looked up in scene s's grid; everything else (step rule,
 * outputs, capacity, status, bit-exact float32 arithmetic) is as in
 * nacc_march_rays. The output is packed ray-major over the whole batch, so it is
 * also scene-major; ray_indices are indices into the batch.
 * scenes           host array of n_scenes >= 1 descriptors (read during the
 *                  call only; the library copies their geometry into the
 *                  workspace with a kernel launch on `stream`, so the call can be
 *                  captured in a CUDA graph).
 * workspace        nacc_march_batched_workspace_size() bytes, 256-byte aligned.
 * Errors: those of nacc_march_rays; NACC_ERR_INVALID_ARG for an invalid scene
 * grid, negative or inconsistent ray counts (their sum must be n_rays), or
 * scenes that differ in contraction.
 */
int nacc_march_rays_batched(const nacc_scene_desc* scenes, int32_t n_scenes, const float* rays_o,
                            const float* rays_d, int32_t n_rays, const nacc_march_params* params,
                            int32_t* packed_info, float* t_starts, float* t_ends, int32_t* ray_indices,
                            int64_t capacity, int64_t* n_samples, int32_t* d_status, void* workspace,
                            size_t workspace_bytes, void* stream);

/*
 * Ray marching without any device allocation by the caller. The paper has no
 * counterpart: this is an integration aid for callers that cannot allocate
 * device memory at call time (a renderer with a fixed, pre-planned memory
 * budget, a plugin inside a host application that owns the CUDA allocator).
 * Same arguments, results and errors as nacc_march_rays, minus the workspace:
 * the scratch lives in a fixed array of this library's device memory, held by
 * every GPU that loads the library until the process exits: the look-back words
 * of up to NACC_STATIC_MAX_RAYS rays (256 + 8 * NACC_STATIC_MAX_RAYS bytes) and
 * the cone-step lattice table of up to NACC_STATIC_MAX_STEPS steps
 * (4 * (NACC_STATIC_MAX_STEPS + 1) bytes, rounded up to 256), about 8.1 MiB in
 * all. Every call nacc_march_rays accepts fits, uniform or cone steps, for any
 * n_rays up to the limit; n_rays above NACC_STATIC_MAX_RAYS is rejected with
 * NACC_ERR_INVALID_ARG before anything is enqueued.
 * - The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture on the device.
 * - Every call on a device shares the one array. Each call clears the part it
 *   uses on `stream` before use, but calls that overlap on the GPU (concurrent
 *   streams, or host threads racing) corrupt each other's scratch: serialise
 *   them, e.g. on one stream.
 * - Nothing is allocated: no cudaMalloc, no cudaFree, no allocating library call.
 */
#define NACC_STATIC_MAX_RAYS (1 << 20)
#define NACC_STATIC_MAX_STEPS 32768 /* = the largest max_steps of nacc_march_params */
int nacc_march_rays_static(const float* rays_o, const float* rays_d, const float* ray_time,
                           const int32_t* ray_slot, int32_t n_rays, const nacc_grid* grid,
                           const nacc_march_params* params, int32_t* packed_info, float* t_starts,
                           float* t_ends, int32_t* ray_indices, int64_t capacity, int64_t* n_samples,
                           int32_t* d_status, void* stream);

/* ------------------------------------------------------------------------- */
/* Pruning by transmittance and opacity (Sec. 2.1 "Pruning Empty and         */
/* Occluded Regions"; arguments early_stop_eps, alpha_thre of Sec. 3)        */
/* ------------------------------------------------------------------------- */

size_t nacc_prune_workspace_size(int32_t n_rays, int64_t n_samples);

/*
 * Keeps sample i of a ray iff T_i >= early_stop_eps and alpha_i >= alpha_thre,
 * with tau_i = sigma_i (t_end,i - t_start,i), T_i = exp(-sum_{j<i} tau_j) over
 * ALL input samples of the ray, alpha_i = 1 - exp(-tau_i) (Eq. 1), and writes
 * the kept samples re-packed (ray-major, order preserved). The decision is
 * taken in float32 as O_i <= -ln(eps) and tau_i >= -ln(1 - thre), both
 * thresholds rounded once to float32; eps <= 0 (thre <= 0) switches that test
 * off. sigmas must be >= 0 (the density of the user's field, queried without
 * gradient per Sec. 2.1); once a ray's optical depth passes -ln(eps) the rest
 * of the ray is not read.
 *
 * packed_info (n_rays,2), t_starts, t_ends, sigmas (n_samples,): input samples,
 *   each 8-byte aligned; runs ascending and disjoint in ray order (as produced
 *   by nacc_march_rays), else the ray is skipped and NACC_STATUS_BAD_PACKED set.
 * packed_info_out (n_rays, 2); t_starts_out, t_ends_out, ray_indices_out
 *   (capacity,): output; n_kept: device int64 out (total, also past capacity).
 * keep_mask (n_samples,) uint8 or NULL: 1 where kept.
 * workspace        nacc_prune_workspace_size() bytes, 256-byte aligned. After
 *                  the call, the uint64 at byte offset 8 of the workspace holds
 *                  the number of input samples the pass read (samples past a
 *                  ray's termination point are not read).
 */
int nacc_prune_samples(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                       const float* t_ends, const float* sigmas, int64_t n_samples,
                       float early_stop_eps, float alpha_thre, int32_t* packed_info_out,
                       float* t_starts_out, float* t_ends_out, int32_t* ray_indices_out,
                       int64_t capacity, int64_t* n_kept, uint8_t* keep_mask, int32_t* d_status,
                       void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Inference: marching that stops on the field's transmittance (Sec. 2.1     */
/* "Pruning Empty and Occluded Regions", "GPU Memory Efficiency")            */
/* ------------------------------------------------------------------------- */

/*
 * A density field the library evaluates itself (for instance a trained
 * radiance field's density baked onto a grid): float32 sigma at the vertices
 * of a res[0] x res[1] x res[2] lattice over the box aabb = (lo xyz, hi xyz),
 * vertex (i, j, k) at lo + (hi - lo) * (i, j, k) / (res - 1), stored x-major,
 * z fastest. Between vertices sigma is trilinear; outside the box it is 0.
 * Float32, in this order per axis a: s_a = (res_a - 1) / (hi_a - lo_a),
 * u_a = (x_a - lo_a) * s_a (outside unless 0 <= u_a <= res_a - 1),
 * i_a = min(floor(u_a), res_a - 2), f_a = u_a - i_a; then
 * lerp(p, q, f) = p + f (q - p) along z, then y, then x (no contraction).
 * Values must be finite and >= 0 (a density).
 */
typedef struct nacc_density_field {
    const float* sigma; /* device, res[0]*res[1]*res[2] float32 (caller-owned) */
    int32_t res[3];     /* vertices per axis, each >= 2, product < 2^31 */
    float aabb[6];      /* lo x, y, z, hi x, y, z; lo < hi, finite */
} nacc_density_field;

/*
 * Marching with the field's transmittance for inference: the samples kept are
 * exactly those nacc_prune_samples(early_stop_eps, alpha_thre) keeps of the
 * samples nacc_march_rays emits, with sigma_i = the field at each sample's
 * midpoint x = o + d (t_s + t_e)/2 (the point the occupancy lookup uses). The
 * march of a ray ends where its optical depth passes -ln(eps) (Sec. 2.1: the
 * transmittance needs the density, queried without gradient), and samples that
 * are dropped are never written, so memory holds only the kept set.
 * Differences to the two-call path: the keep decisions are taken on the same
 * float32 tau_i; the optical depth O_i is summed in another order (32 lattice
 * points per warp-wide shuffle scan), so a decision can differ only where O_i
 * lies within float32 summation error of -ln(eps).
 *
 * Arguments as nacc_march_rays (rays use grid slot 0; no time or slot input),
 * plus:
 * field            host struct (read during the call only), see above.
 * early_stop_eps, alpha_thre  as nacc_prune_samples (<= 0 switches a test off).
 * sigmas           (capacity,) float32 out or NULL: sigma of each kept sample.
 * n_samples        device int64 out: the number of KEPT samples.
 * workspace        nacc_march_workspace_size(n_rays, params) bytes, 256-byte
 *                  aligned. After the call the uint64 at byte offset 8 holds
 *                  the number of lattice points examined (up to each ray's end).
 * Errors: those of nacc_march_rays; NACC_ERR_INVALID_ARG for a missing or
 * malformed field or NaN thresholds.
 */
int nacc_march_fused(const float* rays_o, const float* rays_d, int32_t n_rays, const nacc_grid* grid,
                     const nacc_march_params* params, const nacc_density_field* field, float early_stop_eps,
                     float alpha_thre, int32_t* packed_info, float* t_starts, float* t_ends,
                     int32_t* ray_indices, float* sigmas, int64_t capacity, int64_t* n_samples,
                     int32_t* d_status, void* workspace, size_t workspace_bytes, void* stream);

/*
 * sigma of the field at each sample's midpoint: sigmas[s] = field at
 * o_r + d_r (t_starts[s] + t_ends[s]) / 2 with r = ray_indices[s] (the same
 * float32 operations as nacc_march_fused). rays_o, rays_d (n_rays, 3);
 * ray_indices, t_starts, t_ends, sigmas (n_samples,). A ray index outside
 * [0, n_rays) gives sigma 0 and raises NACC_STATUS_BAD_INDEX in d_status.
 */
int nacc_density_field_at_samples(const nacc_density_field* field, const float* rays_o, const float* rays_d,
                                  int32_t n_rays, const int32_t* ray_indices, const float* t_starts,
                                  const float* t_ends, int64_t n_samples, float* sigmas, int32_t* d_status,
                                  void* stream);

/* sigma of the field at points xyz (n, 3) float32 into sigmas (n,). */
int nacc_density_field_query(const nacc_density_field* field, const float* xyz, int64_t n, float* sigmas,
                             void* stream);

/* ------------------------------------------------------------------------- */
/* Differentiable rendering (Sec. 2.2, Eq. 1)                                */
/* ------------------------------------------------------------------------- */

/*
 * Per-sample weights of Eq. 1: w_i = T_i alpha_i with T_i = exp(-sum_{j<i}
 * sigma_j delta_j), alpha_i = 1 - exp(-sigma_i delta_i), delta_i = t_end -
 * t_start (the printed formula drops the minus sign inside alpha; only this
 * reading lies in [0, 1)). Parallel over samples within each ray (Sec. 2.2).
 * weights, trans: (n_samples,) float32 out, each nullable.
 */
int nacc_render_weights(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                        const float* t_ends, const float* sigmas, int64_t n_samples,
                        float* weights, float* trans, int32_t* d_status, void* stream);

/*
 * Accumulates any per-sample attribute along rays (Sec. 2.2: "Any sample
 * attributes ... can be rendered"): out[r, c] = sum_{i in ray r} w_i v_i[c].
 * values (n_samples, n_channels) float32, or NULL for v = 1 (opacity).
 * out (n_rays, n_channels) float32.
 */
int nacc_accumulate_along_rays(const int32_t* packed_info, int32_t n_rays, const float* weights,
                               const float* values, int32_t n_channels, int64_t n_samples,
                               float* out, int32_t* d_status, void* stream);

/*
 * Gradient of nacc_render_weights for any upstream gradient g_i = dL/dw_i
 * (Sec. 2.2: gradients reach the field through the weights of any attribute):
 *   dL/dsigma_k = delta_k (g_k T_{k+1} - sum_{i>k} g_i w_i),
 * by the same reverse segmented scan and centred form as nacc_render_bwd
 * (with a_i = g_i); T recomputed from sigmas.
 * g_weights (n_samples,) float32 in; d_sigmas (n_samples,) float32 out; the
 * float arrays and packed_info 8-byte aligned.
 * g_ref (n_rays,) float32 in, or NULL. When given, the upstream gradient is
 * split in two parts, g_i = g_ref[r] + g_weights[i] (sample i in ray r), the
 * form nacc_accumulate_along_rays_bwd writes in its centred mode: the scan takes
 * g_ref[r] as its reference and g_weights[i] as the centred term, so the float32
 * error of the result scales with the variation of g along the ray.
 */
int nacc_render_weights_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                            const float* t_ends, const float* sigmas, int64_t n_samples,
                            const float* g_weights, const float* g_ref, float* d_sigmas,
                            int32_t* d_status, void* stream);

/*
 * Gradient of nacc_accumulate_along_rays for g = dL/dout (n_rays, n_channels):
 *   dL/dw_i = sum_c g[r, c] v_i[c] (v = 1 when values is NULL),
 *   dL/dv_i[c] = w_i g[r, c]   (sample i in ray r).
 * d_weights (n_samples,) and d_values (n_samples, n_channels) float32 out,
 * each nullable (d_values needs values).
 * g_ref (n_rays,) float32 in/out, or NULL (needs d_weights). Centred mode: the
 * gradient of each ray's weights is written in two parts, d_weights[i] =
 * sum_c g[r, c] (v_i[c] - v_1[c]) with v_1 the values of the ray's first sample,
 * and sum_c g[r, c] v_1[c] ADDED to g_ref[r] (rays without samples leave it
 * unchanged); the parts sum to dL/dw_i. The per-sample part is formed from value
 * differences before any rounding, so nacc_render_weights_bwd given both parts
 * keeps the precision of the fused nacc_render_bwd. Adding lets several
 * accumulations of the same weights share one g_ref (the caller zeroes it once).
 */
int nacc_accumulate_along_rays_bwd(const int32_t* packed_info, int32_t n_rays, const float* weights,
                                   const float* values, int32_t n_channels, int64_t n_samples,
                                   const float* g_out, float* d_weights, float* d_values, float* g_ref,
                                   int32_t* d_status, void* stream);

/*
 * Fused forward rendering, Eq. 1 (render_weights + accumulate_along_rays):
 *   color[r] = sum w_i rgb_i (n_rays,3); opacity[r] = sum w_i (n_rays,);
 *   depth[r] = sum w_i (t_s + t_e)/2 (n_rays,), unnormalised, black background.
 * optical_depth (n_samples,) float32 out or NULL: O_i = sum_{j<i} tau_j, the
 * state nacc_render_bwd can reuse instead of recomputing it.
 */
int nacc_render_fwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                    const float* t_ends, const float* sigmas, const float* rgbs,
                    int64_t n_samples, float* color, float* opacity, float* depth,
                    float* optical_depth, int32_t* d_status, void* stream);

/*
 * Gradient of nacc_render_fwd (Sec. 2.2: every output of the radiance field
 * receives gradients). With a_i = <g_color, rgb_i> + g_opacity + g_depth tmid_i:
 *   dL/dsigma_k = delta_k (a_k T_{k+1} - sum_{i>k} a_i w_i),  dL/drgb_k = w_k g_color,
 * the suffix sum taken as a true reverse segmented scan (no total-minus-prefix
 * cancellation) and evaluated in the centred form a_ref T_end + b_k T_{k+1} -
 * sum_{i>k} b_i w_i, b_i = a_i - a_ref (a_ref: the ray's first sample), which
 * equals the expression above exactly but keeps float32 error proportional to
 * the variation of a along the ray. T is recomputed from sigmas, or read from
 * optical_depth when the forward pass saved it (bit-identical results either
 * way).
 * g_color (n_rays,3), g_opacity (n_rays,), g_depth (n_rays,): nullable (zero).
 * d_sigmas (n_samples,), d_rgbs (n_samples,3): float32 out.
 */
int nacc_render_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                    const float* t_ends, const float* sigmas, const float* rgbs,
                    const float* optical_depth, int64_t n_samples, const float* g_color,
                    const float* g_opacity, const float* g_depth, float* d_sigmas,
                    float* d_rgbs, int32_t* d_status, void* stream);

/*
 * Forward rendering, the gradient of a squared-error loss on the colours and the
 * backward, in one pass (Eq. 1 and Sec. 2.2, for the photometric loss of the
 * Sec. 3 listing). With L = (grad_scale / 2) * sum_r |C_r - C*_r|^2 (grad_scale =
 * 2 / (3 n_rays): the mean squared error over rays and channels), dL/dC_r =
 * grad_scale * (C_r - C*_r) is known once ray r is rendered, so each ray is
 * rendered forward and then differentiated while its samples are still cached:
 * the samples are read from memory once and no optical depth is stored.
 * Outputs equal nacc_render_fwd's (color, opacity, depth; each nullable) and
 * nacc_render_bwd's for g_color = (C - C*) * grad_scale formed in float32 (two
 * roundings), g_opacity = g_depth = 0 (d_sigmas (n_samples,), d_rgbs
 * (n_samples,3)). target (n_rays,3) float32; sq_err (n_rays,) or NULL: sum over
 * channels of (C - C*)^2 per ray (the loss is grad_scale / 2 times its sum).
 * Float arrays and packed_info 8-byte aligned; grad_scale finite.
 */
int nacc_render_mse_fused(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                          const float* t_ends, const float* sigmas, const float* rgbs, int64_t n_samples,
                          const float* target, float grad_scale, float* color, float* opacity, float* depth,
                          float* sq_err, float* d_sigmas, float* d_rgbs, int32_t* d_status, void* stream);

/*
 * Capacity-sized sample arrays whose count stays on the device (a training step
 * without host reads): value into arr[i * width + c] for every i in
 * [*n_dev, capacity) and c < width, *n_dev read on the device (clamped to
 * [0, capacity]). For example the gradients of samples past the kept count,
 * which no packed run covers. arr (capacity, width) float32; n_dev device int64.
 */
int nacc_fill_tail_f32(float* arr, int64_t width, int64_t capacity, const int64_t* n_dev, float value,
                       void* stream);

/* ray_indices[i] = r for every sample i of ray r (the inverse of packed_info). */
int nacc_unpack_info(const int32_t* packed_info, int32_t n_rays, int64_t n_samples,
                     int32_t* ray_indices, int32_t* d_status, void* stream);

/* ------------------------------------------------------------------------- */
/* Occupancy-grid update (Sec. 2.1: the binary grid is "cached and updated   */
/* during training", following Instant-NGP's Appendix E.2)                   */
/* ------------------------------------------------------------------------- */

/*
 * ema[c] <- decay * ema[c] for every cell c in [0, n_cells), then
 * ema[cell_s] <- max(ema[cell_s], sigma_s) for every sample s (NaN sigmas are
 * ignored), then bits = (ema > thre) packed as in nacc_grid. The caller draws
 * the cells (uniform random cells in Instant-NGP's scheme) and evaluates its
 * field at points inside them. Float32 state, one rounding per product:
 * bit-exact and independent of sample order.
 * alpha_step = 0: thre is a density threshold (bits = ema > thre).
 * alpha_step > 0: the paper's criterion (Sec. 2.1), a cell is empty where the
 * opacity of a step of length alpha_step is below thre (0 <= thre < 1): bit =
 * 1 - exp(-ema alpha_step) > thre, applied as its equivalent density threshold
 * nacc_density_threshold(thre, alpha_step). Negative or NaN alpha_step, or thre
 * outside [0, 1) with alpha_step > 0: NACC_ERR_INVALID_ARG.
 * ema (n_cells,) float32 in/out, values >= 0; bits ceil(n_cells/32) uint32 out;
 * cells (n_samples,) int32 in [0, n_cells) (others raise NACC_STATUS_BAD_INDEX
 * and are skipped); sigmas (n_samples,) float32.
 */
int nacc_update_occupancy_grid(float* ema, uint32_t* bits, int64_t n_cells, const int32_t* cells,
                               const float* sigmas, int64_t n_samples, float decay, float thre,
                               float alpha_step, int32_t* d_status, void* stream);

/*
 * Density threshold of the opacity criterion (host only, no device work): for
 * steps of length dt > 0, 1 - exp(-sigma dt) > alpha_thre exactly when
 * sigma > -ln(1 - alpha_thre) / dt; returned computed in double and rounded once
 * to float32 (the precision of the grid's comparison). NaN unless
 * 0 <= alpha_thre < 1 and 0 < dt < inf.
 */
float nacc_density_threshold(float alpha_thre, float dt);

/*
 * The update's random inputs (Instant-NGP's scheme that Sec. 2.1 follows):
 * n uniform random cells of the whole grid (with replacement) and a uniform
 * point inside each, at which the caller evaluates its field. Counter-based
 * SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): draw i of stream k of seed s
 * is mix(mix(s) + k * 0xD1B54A32D192ED03 + (i + 1) * 0x9E3779B97F4A7C15), mix
 * the splitmix64 output function. Sample i: draws 2i, 2i+1 of stream `stream`
 * give its cell coordinates by multiply-shift range reduction of their 32-bit
 * halves, (h * extent) >> 32 (x, y: high, low half of the first draw; z and
 * sl = slot * n_levels + level: high, low half of the second), cell =
 * ((sl * res_x + x) * res_y + y) * res_z + z; draws 2i, 2i+1 of stream
 * `stream` + 1 give its jitter (24-bit fields at bits 40 and 16 of the first
 * and 40 of the second, times 2^-24); xyz_a = lo_a + (i_a + jitter_a) * cs_a in
 * float32 (each operation rounded), with the level box formed as for marching
 * (c = (lo + hi) / 2, h = (hi - lo) / 2, level l >= 1: c -+ h 2^l) and
 * cs = (hi - lo) / res. With contraction the cell and point are drawn in
 * contracted space (box [-2, 2]^3) and the point is mapped back to the world:
 * r^2 = (p0^2 + p1^2) + p2^2; r^2 <= 1: x_n = p; else x_n = p / ((2 - r) r)
 * (NaN for r >= 2, cells the contraction never reaches); xyz = c + h x_n with
 * the box's c, h. Deterministic: the same arguments give the same bits.
 * grid: the bits pointer is not read; cells (n,) int32 out; xyz (n,3) float32 out.
 */
int nacc_sample_grid_cells(uint64_t seed, uint64_t stream, int64_t n, const nacc_grid* grid,
                           int32_t* cells, float* xyz, void* cuda_stream);

/* ------------------------------------------------------------------------- */
/* Launch-shape tuning (process-wide table, read at each launch)             */
/* ------------------------------------------------------------------------- */

/*
 * Knobs select among launch shapes that compute identical results; they only
 * change speed. Defaults are valid for any input; an autotuner measures the
 * variants on the caller's workload and sets the fastest. Not synchronised:
 * change knobs only while no other host thread launches library work.
 */
#define NACC_TUNE_RENDER_FWD_PREFETCH 0 /* 0/1: issue the next chunk's loads early */
#define NACC_TUNE_MARCH_TILE_RAYS 1     /* 1..32: rays per warp tile (upper bound) */
#define NACC_TUNE_PRUNE_TILE_RAYS 2     /* 2..32, even: rays per warp tile */
#define NACC_TUNE_MARCH_OCCUPANCY 3     /* 0: compiler's register use; 1: registers capped at 64 (4 blocks/SM);
                                          the one-level uniform-step walk is always capped */
#define NACC_TUNE_PRUNE_OCCUPANCY 4     /* 0: compiler's; 1: capped for 8 blocks/SM; 2: for 6 */
#define NACC_TUNE_RENDER_OCCUPANCY 5    /* forward: 0: compiler's; 1: capped for 16 blocks/SM; 2: for 12 */
#define NACC_TUNE_RENDER_BWD_OCCUPANCY 6 /* backward: 0: compiler's; 1: capped for 16 blocks/SM; 2: for 12 */
#define NACC_TUNE_MARCH_UNROLL 7        /* 0/1: uniform steps, two lattice chunks per loop iteration */
#define NACC_TUNE_PRUNE_INTERLEAVE 8    /* 2 or 4: rays a pruning warp walks at once */
#define NACC_TUNE_RENDER_BWD_PREFETCH 9 /* 0/1: backward issues the next chunk's loads early */
#define NACC_TUNE_MARCH_COARSE 10       /* 0/1: first test one lattice point in 32, fill chunks that lie in one cell */
#define NACC_TUNE_FUSED_OCCUPANCY 11    /* 0: compiler's register use; 1: nacc_march_fused capped at 64 registers */
#define NACC_TUNE_MARCH_BOX_TILE 12     /* box walk (grid with its summed-area table, uniform steps): 0 ray by ray;
                                          1, 2, 3 over all chunks of a tile at once, for 4, 5, 6 blocks per SM */
#define NACC_TUNE_RENDER_FWD_STAGES 13  /* forward: 0 loads into registers; 2, 3, 4: chunks staged in shared
                                          memory by bulk copies, that many stages per warp (16-byte aligned
                                          arrays; others take the register path) */
#define NACC_TUNE_RENDER_BWD_STAGES 14  /* backward with the saved optical depth: as NACC_TUNE_RENDER_FWD_STAGES */
#define NACC_TUNE_RENDER_MSE_OCCUPANCY 15 /* nacc_render_mse_fused: 0 compiler's register use; capped for 1: 8,
                                            2: 12 blocks/SM */
#define NACC_TUNE_COUNT 16

/* Set a knob; NACC_ERR_INVALID_ARG for an unknown knob or out-of-range value. */
int nacc_tune_set(int knob, int value);
/* Current value of a knob (NACC_ERR_INVALID_ARG for an unknown knob). */
int nacc_tune_get(int knob);

/* ------------------------------------------------------------------------- */
/* Test hooks of the bounded inter-warp waits (process-wide, read at launch)  */
/* ------------------------------------------------------------------------- */

/*
 * Marching, pruning and the fused inference march find each tile's output
 * offset by a decoupled look-back: a warp waits for the tiles before it to
 * publish their totals. Every wait is bounded: after a poll budget it gives up,
 * raises NACC_STATUS_TIMEOUT, and publishes a prefix no larger than the true one,
 * so the call still returns and every store stays below the true total (and
 * below capacity). These hooks exist so a test can make the waits run out on
 * purpose and check that path; they are not for production use and compute
 * invalid results while set to anything but their defaults.
 * NACC_TEST_HOOK_SPIN_LIMIT: polls before a wait gives up, 0 .. 2^22
 *   (default 2^22: about a second with the back-off between polls).
 * NACC_TEST_HOOK_WITHHOLD_FIRST_TILE: 0 (default) or 1. With 1 the first tile
 *   never publishes its total, so every wait that reaches it runs out.
 * The render passes with staged chunks (NACC_TUNE_RENDER_*_STAGES) wait, a
 * bounded number of polls, for each chunk's bulk copies to land; a wait that
 * gives up raises NACC_STATUS_TIMEOUT, waits (bounded) for the warp's copies in
 * flight and ends the warp's walk, leaving its rays' outputs unwritten.
 * NACC_TEST_HOOK_SPIN_LIMIT also sets that poll budget when below its default.
 * NACC_TEST_HOOK_OVERSTATE_STAGE_BYTES: 0 (default) or 1. With 1 each warp's
 *   first chunk announces 16 bytes more than it copies, so its wait runs out.
 * Not synchronised: change hooks only while no other host thread launches
 * library work. NACC_ERR_INVALID_ARG for an unknown hook or a value out of range.
 */
#define NACC_TEST_HOOK_SPIN_LIMIT 0
#define NACC_TEST_HOOK_WITHHOLD_FIRST_TILE 1
#define NACC_TEST_HOOK_OVERSTATE_STAGE_BYTES 2
#define NACC_TEST_HOOK_COUNT 3
int nacc_test_hook_set(int hook, int value);
int nacc_test_hook_get(int hook);

/* ------------------------------------------------------------------------- */
/* Utilities                                                                 */
/* ------------------------------------------------------------------------- */

/* Static, human-readable text of a host return code. */
const char* nacc_error_string(int code);
/* NACC_VERSION of the built library. */
int nacc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NACC_H */
