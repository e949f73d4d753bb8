// march.cu -- occupancy-grid ray marching with empty-space skipping (NerfAcc,
// arXiv 2210.04847, Sec. 2.1 "Ray Marching" and "GPU Memory Efficiency":
// samples are emitted only in occupied cells, pruned while marching).
//
// Compiled with -fmad=false; every float operation on the sample path is an
// explicitly rounded __f*_rn intrinsic so that the emitted set is
// bit-reproducible (it is an integer result decided by float arithmetic).
//
// Design (single pass, no count/fill split):
//   * A persistent grid of blocks takes tiles of rays in ticket order.
//   * Uniform steps: one warp per ray, lane j evaluates lattice point 32c + j
//     (the lattice is closed-form, t_k = near + k*dt), the occupancy test of
//     the 32 midpoints is turned into one __ballot_sync word kept in shared
//     memory, and __popc gives the ray's count.
//   * Cone steps (t_{k+1} = t_k + clamp(t_k*cone, dt_min, dt_max)): the
//     lattice is a sequential float32 recurrence, so one thread walks one ray;
//     it counts first and walks again to write.
//   * The tile's sample total is turned into a global offset by a bounded
//     decoupled look-back over earlier tiles; the warp then re-expands the
//     ballot words into compacted, coalesced stores of (t_start, t_end, ray).
#include <math.h>
#include <string.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTileUniform = 32;   // rays per tile, warp-per-ray walk
constexpr int kTileCone = kThreads;  // rays per tile, thread-per-ray walk

struct Levels {
    float lo[NACC_MAX_LEVELS][3];
    float scale[NACC_MAX_LEVELS][3];
    float box_lo[3];  // clipping box = outermost level
    float box_hi[3];
};

struct MarchArgs {
    const float* rays_o;
    const float* rays_d;
    const float* ray_time;
    const int32_t* ray_slot;
    int32_t n_rays;
    const uint32_t* bits;
    int32_t res0, res1, res2;
    float fres0, fres1, fres2;
    int32_t n_levels;
    int32_t n_slots;
    float near_plane, far_plane, dt_min, dt_max, cone;
    int32_t max_steps;
    int32_t* packed_info;
    float* t_starts;
    float* t_ends;
    int32_t* ray_indices;
    int64_t capacity;
    int64_t* n_samples;
    int32_t* d_status;
    unsigned long long* tile_status;
    unsigned int* ticket;
    int32_t n_tiles;
    int32_t mask_words;
    Levels L;
};

__device__ __forceinline__ bool finite32(float v) { return fabsf(v) <= 3.402823466e+38f; }

// Slab clip against the outermost level box, float32 (ties and zero
// directions as the oracle defines them).
__device__ __forceinline__ bool clip_ray(const MarchArgs& a, const float o[3], const float d[3],
                                         float& near, float& far) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!finite32(o[k]) || !finite32(d[k])) return false;
    float t_in = -INFINITY, t_out = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) {
            if (o[k] < a.L.box_lo[k] || o[k] > a.L.box_hi[k]) return false;
            continue;
        }
        float inv = __fdiv_rn(1.0f, d[k]);
        float t0 = __fmul_rn(__fsub_rn(a.L.box_lo[k], o[k]), inv);
        float t1 = __fmul_rn(__fsub_rn(a.L.box_hi[k], o[k]), inv);
        float tmin = t0 < t1 ? t0 : t1;
        float tmax = t0 < t1 ? t1 : t0;
        if (tmin > t_in) t_in = tmin;
        if (tmax < t_out) t_out = tmax;
    }
    near = t_in > a.near_plane ? t_in : a.near_plane;
    far = t_out < a.far_plane ? t_out : a.far_plane;
    return near < far;
}

__device__ __forceinline__ int slot_of(const MarchArgs& a, int r) {
    if (a.ray_slot) return a.ray_slot[r];
    if (a.ray_time) {
        float fn = __int2float_rn(a.n_slots);
        float v = __fmul_rn(a.ray_time[r], fn);
        if (v >= 0.0f && v < fn) return (int)v;
        if (v >= fn) return a.n_slots - 1;
        return 0;
    }
    return 0;
}

// Occupancy bit of point x: finest level whose box holds x, floor cell index.
template <int MAXL>
__device__ __forceinline__ bool occupied(const MarchArgs& a, float x0, float x1, float x2,
                                         unsigned slot_level0) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) {
        if (l >= a.n_levels) break;
        float u0 = __fmul_rn(__fsub_rn(x0, a.L.lo[l][0]), a.L.scale[l][0]);
        float u1 = __fmul_rn(__fsub_rn(x1, a.L.lo[l][1]), a.L.scale[l][1]);
        float u2 = __fmul_rn(__fsub_rn(x2, a.L.lo[l][2]), a.L.scale[l][2]);
        if (u0 >= 0.0f && u0 < a.fres0 && u1 >= 0.0f && u1 < a.fres1 && u2 >= 0.0f && u2 < a.fres2) {
            unsigned ix = (unsigned)u0, iy = (unsigned)u1, iz = (unsigned)u2;
            unsigned cell = (((slot_level0 + l) * a.res0 + ix) * a.res1 + iy) * a.res2 + iz;
            unsigned w = __ldg(a.bits + (cell >> 5));
            return (w >> (cell & 31u)) & 1u;
        }
    }
    return false;
}

__device__ __forceinline__ float lattice_t(float near, int k, float dt) {
    return __fadd_rn(near, __fmul_rn(__int2float_rn(k), dt));
}

// ---------------------------------------------------------------------------
// uniform steps: warp per ray
// ---------------------------------------------------------------------------

template <int MAXL>
__global__ void __launch_bounds__(kThreads) march_uniform_kernel(const MarchArgs a) {
    extern __shared__ uint32_t s_masks[];  // [kTileUniform][mask_words]
    __shared__ int s_count[kTileUniform];
    __shared__ int s_nchunks[kTileUniform];
    __shared__ float s_near[kTileUniform];
    __shared__ float s_far[kTileUniform];
    __shared__ int s_excl[kTileUniform];
    __shared__ int s_tile;
    __shared__ int s_next;
    __shared__ long long s_tile_excl;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const float dt = a.dt_min;

    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(a.ticket, 1u);
            s_next = 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= a.n_tiles) break;
        const int ray0 = tile * kTileUniform;
        const int nr = min(kTileUniform, a.n_rays - ray0);

        // phase 1: walk the lattice of every ray of the tile, ballot words -> smem
        for (;;) {
            int i = 0;
            if (lane == 0) i = atomicAdd(&s_next, 1);
            i = __shfl_sync(FULL, i, 0);
            if (i >= nr) break;
            const int r = ray0 + i;
            float o[3], d[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
                d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
            }
            float near = 0.0f, far = 0.0f;
            int count = 0, c = 0;
            const int slot = slot_of(a, r);
            const bool slot_ok = slot >= 0 && slot < a.n_slots;
            if (!slot_ok && lane == 0) raise_status(a.d_status, NACC_STATUS_BAD_INDEX);
            if (slot_ok && clip_ray(a, o, d, near, far)) {
                const unsigned sl0 = (unsigned)slot * (unsigned)a.n_levels;
                uint32_t* row = s_masks + (size_t)i * a.mask_words;
                for (; c < a.mask_words; ++c) {
                    const int k = (c << 5) + lane;
                    const float ts = lattice_t(near, k, dt);
                    const bool valid = (k < a.max_steps) && (ts < far);
                    if (__ballot_sync(FULL, valid) == 0u) break;
                    bool occ = false;
                    if (valid) {
                        const float tn = lattice_t(near, k + 1, dt);
                        const float te = tn < far ? tn : far;
                        const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                        const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
                        const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
                        const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
                        occ = occupied<MAXL>(a, x0, x1, x2, sl0);
                    }
                    const unsigned m = __ballot_sync(FULL, occ);
                    if (lane == 0) row[c] = m;
                    count += __popc(m);
                }
            }
            if (lane == 0) {
                s_count[i] = count;
                s_nchunks[i] = c;
                s_near[i] = near;
                s_far[i] = far;
            }
        }
        __syncthreads();

        // phase 2: tile prefix, then the tile's global offset by look-back
        if (warp == 0) {
            const int cnt = lane < nr ? s_count[lane] : 0;
            const int incl = warp_incl_scan_int(cnt, lane);
            s_excl[lane] = incl - cnt;
            const int agg = __shfl_sync(FULL, incl, 31);
            const unsigned long long excl =
                lookback(a.tile_status, tile, (unsigned long long)agg, lane, a.d_status);
            if (lane == 0) {
                s_tile_excl = (long long)excl;
                if (tile == a.n_tiles - 1) {
                    const long long total = (long long)excl + agg;
                    *a.n_samples = total;
                    if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
                    if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
                }
            }
        }
        __syncthreads();

        // phase 3: expand the ballot words into compacted, coalesced stores
        const long long tile_excl = s_tile_excl;
        for (int i = warp; i < nr; i += kWarps) {
            const int r = ray0 + i;
            const int cnt = s_count[i];
            const long long off = tile_excl + s_excl[i];
            if (lane == 0) {
                a.packed_info[2 * (size_t)r] = (int32_t)off;
                a.packed_info[2 * (size_t)r + 1] = cnt;
            }
            if (cnt == 0) continue;
            const float near = s_near[i], far = s_far[i];
            const uint32_t* row = s_masks + (size_t)i * a.mask_words;
            const int nch = s_nchunks[i];
            long long base = off;
            for (int c = 0; c < nch; ++c) {
                const unsigned m = row[c];
                if (m == 0u) continue;
                if ((m >> lane) & 1u) {
                    const int k = (c << 5) + lane;
                    const long long pos = base + __popc(m & lanemask_lt());
                    if (pos < a.capacity) {
                        const float ts = lattice_t(near, k, dt);
                        const float tn = lattice_t(near, k + 1, dt);
                        a.t_starts[pos] = ts;
                        a.t_ends[pos] = tn < far ? tn : far;
                        a.ray_indices[pos] = r;
                    }
                }
                base += __popc(m);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// cone steps: thread per ray (sequential float32 recurrence)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float cone_step(const MarchArgs& a, float t) {
    float dt = __fmul_rn(t, a.cone);
    if (dt < a.dt_min) dt = a.dt_min;
    if (dt > a.dt_max) dt = a.dt_max;
    return __fadd_rn(t, dt);
}

template <int MAXL>
__device__ int walk_cone(const MarchArgs& a, const float o[3], const float d[3], float near, float far,
                         unsigned sl0, int r, long long out, bool write) {
    int count = 0;
    float t = near;
    for (int k = 0; k < a.max_steps; ++k) {
        const float ts = t;
        const float tn = cone_step(a, t);
        t = tn;
        if (!(ts < far)) break;
        const float te = tn < far ? tn : far;
        const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
        const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
        const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
        const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
        if (occupied<MAXL>(a, x0, x1, x2, sl0)) {
            if (write) {
                const long long pos = out + count;
                if (pos < a.capacity) {
                    a.t_starts[pos] = ts;
                    a.t_ends[pos] = te;
                    a.ray_indices[pos] = r;
                }
            }
            ++count;
        }
    }
    return count;
}

template <int MAXL>
__global__ void __launch_bounds__(kThreads) march_cone_kernel(const MarchArgs a) {
    __shared__ int s_warp_tot[kWarps];
    __shared__ int s_tile;
    __shared__ long long s_tile_excl;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= a.n_tiles) break;
        const int r = tile * kTileCone + threadIdx.x;
        const bool have = r < a.n_rays;
        float o[3] = {0, 0, 0}, d[3] = {0, 0, 0};
        float near = 0.0f, far = 0.0f;
        bool live = false;
        unsigned sl0 = 0;
        if (have) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
                d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
            }
            const int slot = slot_of(a, r);
            if (slot >= 0 && slot < a.n_slots) {
                sl0 = (unsigned)slot * (unsigned)a.n_levels;
                live = clip_ray(a, o, d, near, far);
            } else {
                raise_status(a.d_status, NACC_STATUS_BAD_INDEX);
            }
        }
        const int cnt = live ? walk_cone<MAXL>(a, o, d, near, far, sl0, r, 0, false) : 0;

        // block-wide exclusive scan of the 256 counts
        const int incl = warp_incl_scan_int(cnt, lane);
        if (lane == 31) s_warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int wt = lane < kWarps ? s_warp_tot[lane] : 0;
            const int wincl = warp_incl_scan_int(wt, lane);
            if (lane < kWarps) s_warp_tot[lane] = wincl - wt;
            const int agg = __shfl_sync(FULL, wincl, kWarps - 1);
            const unsigned long long excl =
                lookback(a.tile_status, tile, (unsigned long long)agg, lane, a.d_status);
            if (lane == 0) {
                s_tile_excl = (long long)excl;
                if (tile == a.n_tiles - 1) {
                    const long long total = (long long)excl + agg;
                    *a.n_samples = total;
                    if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
                    if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
                }
            }
        }
        __syncthreads();
        const long long off = s_tile_excl + s_warp_tot[warp] + (incl - cnt);
        if (have) {
            a.packed_info[2 * (size_t)r] = (int32_t)off;
            a.packed_info[2 * (size_t)r + 1] = cnt;
        }
        if (cnt > 0) walk_cone<MAXL>(a, o, d, near, far, sl0, r, off, true);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

constexpr size_t kTicketBytes = 256;

int mask_words_for(int32_t max_steps) { return (max_steps + 31) / 32; }

size_t workspace_bytes_for(int32_t n_rays) {
    const size_t tiles = (size_t)(n_rays + kTileUniform - 1) / kTileUniform;
    return align_up(kTicketBytes + tiles * sizeof(unsigned long long), 256);
}

// Level boxes and cell scales, float32, in the order the method defines them.
void make_levels(const nacc_grid& g, Levels& L) {
    for (int k = 0; k < 3; ++k) {
        const float lo = g.aabb[k], hi = g.aabb[3 + k];
        const float c = (lo + hi) * 0.5f;
        const float h = (hi - lo) * 0.5f;
        for (int l = 0; l < g.n_levels; ++l) {
            float llo, lhi;
            if (l == 0) {
                llo = lo;
                lhi = hi;
            } else {
                const float hl = h * ldexpf(1.0f, l);
                llo = c - hl;
                lhi = c + hl;
            }
            L.lo[l][k] = llo;
            L.scale[l][k] = (float)g.res[k] / (lhi - llo);
            if (l == g.n_levels - 1) {
                L.box_lo[k] = llo;
                L.box_hi[k] = lhi;
            }
        }
    }
}

template <typename K>
int blocks_for(K kernel, size_t smem, int n_tiles) {
    const DeviceInfo dev = current_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int want = dev.sm_count * per_sm;
    return n_tiles < want ? n_tiles : want;
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_march_workspace_size(int32_t n_rays, const nacc_march_params* params) {
    (void)params;
    if (n_rays < 0) return 0;
    return workspace_bytes_for(n_rays);
}

extern "C" int nacc_march_rays(const float* rays_o, const float* rays_d, const float* ray_time,
                               const int32_t* ray_slot, int32_t n_rays, const nacc_grid* grid,
                               const nacc_march_params* p, int32_t* packed_info, float* t_starts,
                               float* t_ends, int32_t* ray_indices, int64_t capacity,
                               int64_t* n_samples, int32_t* d_status, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (n_rays < 0 || capacity < 0 || !grid || !p || !n_samples) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d || !packed_info || !grid->bits)) return NACC_ERR_INVALID_ARG;
    if (capacity > 0 && (!t_starts || !t_ends || !ray_indices)) return NACC_ERR_INVALID_ARG;
    if (grid->n_levels < 1 || grid->n_levels > NACC_MAX_LEVELS || grid->n_slots < 1) return NACC_ERR_INVALID_ARG;
    if (grid->res[0] < 1 || grid->res[1] < 1 || grid->res[2] < 1) return NACC_ERR_INVALID_ARG;
    const long long cells = (long long)grid->res[0] * grid->res[1] * grid->res[2] * grid->n_levels * grid->n_slots;
    if (cells >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    if (p->max_steps < 1 || p->max_steps > 32768) return NACC_ERR_INVALID_ARG;
    if (!(p->dt_min > 0.0f) || !(p->dt_min < INFINITY) || p->cone < 0.0f || !(p->cone < INFINITY))
        return NACC_ERR_INVALID_ARG;
    if (p->cone > 0.0f && !(p->dt_max >= p->dt_min)) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 6; ++k)
        if (!(fabsf(grid->aabb[k]) < INFINITY)) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(grid->aabb[k] < grid->aabb[3 + k])) return NACC_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < workspace_bytes_for(n_rays)) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return NACC_ERR_INVALID_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays == 0) return launch_status(cudaMemsetAsync(n_samples, 0, sizeof(int64_t), st));

    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.rays_o = rays_o;
    a.rays_d = rays_d;
    a.ray_time = ray_time;
    a.ray_slot = ray_slot;
    a.n_rays = n_rays;
    a.bits = grid->bits;
    a.res0 = grid->res[0];
    a.res1 = grid->res[1];
    a.res2 = grid->res[2];
    a.fres0 = (float)grid->res[0];
    a.fres1 = (float)grid->res[1];
    a.fres2 = (float)grid->res[2];
    a.n_levels = grid->n_levels;
    a.n_slots = grid->n_slots;
    a.near_plane = p->near_plane;
    a.far_plane = p->far_plane;
    a.dt_min = p->dt_min;
    a.dt_max = p->dt_max;
    a.cone = p->cone;
    a.max_steps = p->max_steps;
    a.packed_info = packed_info;
    a.t_starts = t_starts;
    a.t_ends = t_ends;
    a.ray_indices = ray_indices;
    a.capacity = capacity;
    a.n_samples = n_samples;
    a.d_status = d_status;
    a.ticket = (unsigned int*)workspace;
    a.tile_status = (unsigned long long*)((char*)workspace + kTicketBytes);
    a.mask_words = mask_words_for(p->max_steps);
    make_levels(*grid, a.L);

    const bool cone = p->cone > 0.0f;
    a.n_tiles = cone ? (n_rays + kTileCone - 1) / kTileCone : (n_rays + kTileUniform - 1) / kTileUniform;
    const size_t clear = kTicketBytes + (size_t)a.n_tiles * sizeof(unsigned long long);
    cudaError_t e = cudaMemsetAsync(workspace, 0, clear, st);
    if (e != cudaSuccess) return NACC_ERR_CUDA;

    if (cone) {
        if (a.n_levels == 1) {
            const int blocks = blocks_for(march_cone_kernel<1>, 0, a.n_tiles);
            march_cone_kernel<1><<<blocks, kThreads, 0, st>>>(a);
        } else {
            const int blocks = blocks_for(march_cone_kernel<NACC_MAX_LEVELS>, 0, a.n_tiles);
            march_cone_kernel<NACC_MAX_LEVELS><<<blocks, kThreads, 0, st>>>(a);
        }
    } else {
        const size_t smem = (size_t)kTileUniform * a.mask_words * sizeof(uint32_t);
        if (a.n_levels == 1) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(march_uniform_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            const int blocks = blocks_for(march_uniform_kernel<1>, smem, a.n_tiles);
            march_uniform_kernel<1><<<blocks, kThreads, smem, st>>>(a);
        } else {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(march_uniform_kernel<NACC_MAX_LEVELS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            const int blocks = blocks_for(march_uniform_kernel<NACC_MAX_LEVELS>, smem, a.n_tiles);
            march_uniform_kernel<NACC_MAX_LEVELS><<<blocks, kThreads, smem, st>>>(a);
        }
    }
    return launch_status(cudaGetLastError());
}
