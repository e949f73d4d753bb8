// march_common.cuh -- what the marching kernels share: the argument block, the
// float32 ray-box clip, the occupancy lookup, the step lattices (uniform and
// cone), and the host-side sizing, level boxes and argument checks (NerfAcc,
// arXiv 2210.04847, Sec. 2.1 "Ray Marching"). Included by march.cu (marching)
// and fused.cu (marching with the density field's transmittance, for inference).
// Every float operation here is an explicitly rounded __f*_rn intrinsic: the
// emitted set is an integer result decided by float arithmetic.
#pragma once

#include <math.h>
#include <string.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct Levels {
    float lo[NACC_MAX_LEVELS][3];
    float scale[NACC_MAX_LEVELS][3];
    float box_lo[3];  // clipping box = outermost level
    float box_hi[3];
};

// One scene of a batch with per-scene grids (nacc_march_rays_batched), as the
// kernels read it from the workspace: the scene's bitfield (its level 0 at word
// 0), resolution, level boxes and contraction constants, formed on the host by
// the same float32 operations as a single grid's.
struct SceneGeom {
    const uint32_t* bits;
    const uint16_t* sat;  // summed-area table of bits, or null
    int32_t res[3];
    int32_t n_levels;
    Levels L;
    float cc[3], inv_h[3], qres[3];
    int32_t pad;
};
static_assert(sizeof(SceneGeom) % 16 == 0, "scene table entries stay 16-byte aligned");

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
    int32_t vec_out;          // the three outputs are 16-byte aligned (16-byte stores for runs of full words)
    int64_t capacity;
    int64_t* n_samples;
    int32_t* d_status;
    unsigned long long* tile_status;
    unsigned int* ticket;
    unsigned long long* lattice_points;  // diagnostic: lattice points examined, summed over rays
    int32_t n_tiles;
    int32_t mask_words;       // ballot words a ray's row can hold
    int32_t row_stride;       // words between consecutive rows in shared memory (= mask_words)
    int32_t tile_rays;
    const float* cone_table;  // t_0 = near_plane, t_1, ..., t_max_steps (cone steps only)
    int32_t cone_smem_at;     // float offset of the table's copy in dynamic shared memory, or -1
    int32_t contract;         // contracted unbounded space (one level, no box clip)
    float cc[3], inv_h[3];    // contraction: box centre and 1 / half size
    float qres[3];            // contraction: res / 4 (the grid spans [-2, 2])
    float inv_dt;             // 1 / dt_min, for the first guess of a uniform lattice's length
    LookbackHooks hooks;      // look-back poll budget (test hooks)
    const uint16_t* sat;      // summed-area table of the grid's bits, or null
    const uint16_t* bricks;   // the table's brick summary (global), when the walk keeps it in shared memory
    int32_t brick_entries;    // uint16 entries of the summary over all grids
    int32_t brick_nb1, brick_nb2, brick_per_grid;  // bricks along y and z; summary entries per grid
    const SceneGeom* scenes;  // batch of scenes with their own grids (else null)
    const int32_t* scene_end; // exclusive end of each scene's consecutive rays
    int32_t n_scenes;
    Levels L;
};

// ---------------------------------------------------------------------------
// grid geometry as the lookup reads it
// ---------------------------------------------------------------------------
// The call's grid lives in the kernel parameters (ArgGeom). For a batch of
// scenes with their own grids the walk reads the current ray's scene from
// registers (RegGeom: one level or contracted space) or from the warp's copy of
// the scene in shared memory (SmemGeom: cascades). The lookup arithmetic is the
// same for all three.

struct ArgGeom {
    const MarchArgs& a;
    const uint16_t* s_bricks = nullptr;  // the brick summary in shared memory, or null
    __device__ __forceinline__ float lo(int l, int k) const { return a.L.lo[l][k]; }
    __device__ __forceinline__ float scale(int l, int k) const { return a.L.scale[l][k]; }
    __device__ __forceinline__ float box_lo(int k) const { return a.L.box_lo[k]; }
    __device__ __forceinline__ float box_hi(int k) const { return a.L.box_hi[k]; }
    __device__ __forceinline__ float cc(int k) const { return a.cc[k]; }
    __device__ __forceinline__ float inv_h(int k) const { return a.inv_h[k]; }
    __device__ __forceinline__ float qres(int k) const { return a.qres[k]; }
    __device__ __forceinline__ int res0() const { return a.res0; }
    __device__ __forceinline__ int res1() const { return a.res1; }
    __device__ __forceinline__ int res2() const { return a.res2; }
    __device__ __forceinline__ int n_levels() const { return a.n_levels; }
    __device__ __forceinline__ const uint32_t* bits() const { return a.bits; }
    __device__ __forceinline__ const uint16_t* sat() const { return a.sat; }
    __device__ __forceinline__ const uint16_t* bricks() const { return s_bricks; }
    __device__ __forceinline__ int brick_nb1() const { return a.brick_nb1; }
    __device__ __forceinline__ int brick_nb2() const { return a.brick_nb2; }
    __device__ __forceinline__ int brick_per_grid() const { return a.brick_per_grid; }
};

struct SmemGeom {
    const SceneGeom* g;
    __device__ __forceinline__ float lo(int l, int k) const { return g->L.lo[l][k]; }
    __device__ __forceinline__ float scale(int l, int k) const { return g->L.scale[l][k]; }
    __device__ __forceinline__ float box_lo(int k) const { return g->L.box_lo[k]; }
    __device__ __forceinline__ float box_hi(int k) const { return g->L.box_hi[k]; }
    __device__ __forceinline__ float cc(int k) const { return g->cc[k]; }
    __device__ __forceinline__ float inv_h(int k) const { return g->inv_h[k]; }
    __device__ __forceinline__ float qres(int k) const { return g->qres[k]; }
    __device__ __forceinline__ int res0() const { return g->res[0]; }
    __device__ __forceinline__ int res1() const { return g->res[1]; }
    __device__ __forceinline__ int res2() const { return g->res[2]; }
    __device__ __forceinline__ int n_levels() const { return g->n_levels; }
    __device__ __forceinline__ const uint32_t* bits() const { return g->bits; }
    __device__ __forceinline__ const uint16_t* sat() const { return g->sat; }
    __device__ __forceinline__ const uint16_t* bricks() const { return nullptr; }
    __device__ __forceinline__ int brick_nb1() const { return 0; }
    __device__ __forceinline__ int brick_nb2() const { return 0; }
    __device__ __forceinline__ int brick_per_grid() const { return 0; }
};

// One level (or contracted space) in registers, loaded once per ray.
struct RegGeom {
    float lo_[3], scale_[3], blo_[3], bhi_[3], cc_[3], ih_[3], q_[3];
    int r_[3];
    const uint32_t* b_;
    const uint16_t* sat_;
    __device__ __forceinline__ explicit RegGeom(const SceneGeom& s) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo_[k] = s.L.lo[0][k];
            scale_[k] = s.L.scale[0][k];
            blo_[k] = s.L.box_lo[k];
            bhi_[k] = s.L.box_hi[k];
            cc_[k] = s.cc[k];
            ih_[k] = s.inv_h[k];
            q_[k] = s.qres[k];
            r_[k] = s.res[k];
        }
        b_ = s.bits;
        sat_ = s.sat;
    }
    __device__ __forceinline__ float lo(int, int k) const { return lo_[k]; }
    __device__ __forceinline__ float scale(int, int k) const { return scale_[k]; }
    __device__ __forceinline__ float box_lo(int k) const { return blo_[k]; }
    __device__ __forceinline__ float box_hi(int k) const { return bhi_[k]; }
    __device__ __forceinline__ float cc(int k) const { return cc_[k]; }
    __device__ __forceinline__ float inv_h(int k) const { return ih_[k]; }
    __device__ __forceinline__ float qres(int k) const { return q_[k]; }
    __device__ __forceinline__ int res0() const { return r_[0]; }
    __device__ __forceinline__ int res1() const { return r_[1]; }
    __device__ __forceinline__ int res2() const { return r_[2]; }
    __device__ __forceinline__ int n_levels() const { return 1; }
    __device__ __forceinline__ const uint32_t* bits() const { return b_; }
    __device__ __forceinline__ const uint16_t* sat() const { return sat_; }
    __device__ __forceinline__ const uint16_t* bricks() const { return nullptr; }
    __device__ __forceinline__ int brick_nb1() const { return 0; }
    __device__ __forceinline__ int brick_nb2() const { return 0; }
    __device__ __forceinline__ int brick_per_grid() const { return 0; }
};

__device__ __forceinline__ bool finite32(float v) { return fabsf(v) <= 3.402823466e+38f; }

// Slab clip against the outermost level box, float32 (ties and zero
// directions as the oracle defines them). CONTRACT: contracted space has no box.
template <bool CONTRACT, typename G>
__device__ __forceinline__ bool clip_ray_in(const MarchArgs& a, const G& g, const float o[3], const float d[3],
                                            float& near, float& far) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!finite32(o[k]) || !finite32(d[k])) return false;
    if (CONTRACT) {  // unbounded: the whole [near_plane, far_plane]
        near = a.near_plane;
        far = a.far_plane;
        return near < far;
    }
    float t_in = -INFINITY, t_out = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0f) {
            if (o[k] < g.box_lo(k) || o[k] > g.box_hi(k)) return false;
            continue;
        }
        float inv = __frcp_rn(d[k]);  // the correctly rounded 1/d, as the IEEE division gives
        float t0 = __fmul_rn(__fsub_rn(g.box_lo(k), o[k]), inv);
        float t1 = __fmul_rn(__fsub_rn(g.box_hi(k), o[k]), inv);
        float tmin = t0 < t1 ? t0 : t1;
        float tmax = t0 < t1 ? t1 : t0;
        if (tmin > t_in) t_in = tmin;
        if (tmax < t_out) t_out = tmax;
    }
    near = t_in > a.near_plane ? t_in : a.near_plane;
    far = t_out < a.far_plane ? t_out : a.far_plane;
    return near < far;
}

template <bool CONTRACT>
__device__ __forceinline__ bool clip_ray(const MarchArgs& a, const float o[3], const float d[3], float& near,
                                         float& far) {
    return clip_ray_in<CONTRACT>(a, ArgGeom{a}, o, d, near, far);
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
// i = floor(u) with 0 <= i < res is the same test as 0 <= u < res followed by
// truncation (u is finite here: o, d and the lattice are finite).
// MAXL == 0: contracted unbounded space (one level, see nacc_grid).
template <int MAXL, typename G>
__device__ __forceinline__ bool occupied_in(const G& g, float x0, float x1, float x2, unsigned slot_level0) {
    if constexpr (MAXL == 0) {
        float x[3] = {__fmul_rn(__fsub_rn(x0, g.cc(0)), g.inv_h(0)), __fmul_rn(__fsub_rn(x1, g.cc(1)), g.inv_h(1)),
                      __fmul_rn(__fsub_rn(x2, g.cc(2)), g.inv_h(2))};
        const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(x[0], x[0]), __fmul_rn(x[1], x[1])), __fmul_rn(x[2], x[2]));
        if (!(n2 <= 1.0f)) {
            const float n = __fsqrt_rn(n2);
            const float s = __fdiv_rn(__fsub_rn(2.0f, __frcp_rn(n)), n);  // __frcp_rn(n) is the correctly rounded 1/n
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = __fmul_rn(x[k], s);
        }
        const int i0 = __float2int_rd(__fmul_rn(__fadd_rn(x[0], 2.0f), g.qres(0)));
        const int i1 = __float2int_rd(__fmul_rn(__fadd_rn(x[1], 2.0f), g.qres(1)));
        const int i2 = __float2int_rd(__fmul_rn(__fadd_rn(x[2], 2.0f), g.qres(2)));
        if ((unsigned)i0 < (unsigned)g.res0() && (unsigned)i1 < (unsigned)g.res1() && (unsigned)i2 < (unsigned)g.res2()) {
            const unsigned cell = ((slot_level0 * g.res0() + i0) * g.res1() + i1) * g.res2() + i2;
            const unsigned w = __ldg(g.bits() + (cell >> 5));
            return (w >> (cell & 31u)) & 1u;
        }
        return false;
    } else {
#pragma unroll
        for (int l = 0; l < MAXL; ++l) {
            if (MAXL > 1 && l >= g.n_levels()) break;  // single-level kernels run only for n_levels == 1
            const int i0 = __float2int_rd(__fmul_rn(__fsub_rn(x0, g.lo(l, 0)), g.scale(l, 0)));
            const int i1 = __float2int_rd(__fmul_rn(__fsub_rn(x1, g.lo(l, 1)), g.scale(l, 1)));
            const int i2 = __float2int_rd(__fmul_rn(__fsub_rn(x2, g.lo(l, 2)), g.scale(l, 2)));
            if ((unsigned)i0 < (unsigned)g.res0() && (unsigned)i1 < (unsigned)g.res1() &&
                (unsigned)i2 < (unsigned)g.res2()) {
                const unsigned cell = (((slot_level0 + l) * g.res0() + i0) * g.res1() + i1) * g.res2() + i2;
                const unsigned w = __ldg(g.bits() + (cell >> 5));
                return (w >> (cell & 31u)) & 1u;
            }
        }
        return false;
    }
}

template <int MAXL>
__device__ __forceinline__ bool occupied(const MarchArgs& a, float x0, float x1, float x2, unsigned slot_level0) {
    return occupied_in<MAXL>(ArgGeom{a}, x0, x1, x2, slot_level0);
}

__device__ __forceinline__ float lattice_t(float near, int k, float dt) {
    return __fadd_rn(near, __fmul_rn(__int2float_rn(k), dt));
}

// Number of lattice intervals of a ray: the k < max_steps with t_k < far. t_k is
// non-decreasing in k, so it is the first k with t_k >= far (capped): a guess from
// real arithmetic (the span times 1/dt), then the exact float32 test moves it to
// the boundary (the guess is off by at most a few steps).
__device__ __forceinline__ int lattice_count(const MarchArgs& a, float near, float far, float dt) {
    float g = (far - near) * a.inv_dt;
    int e = g < (float)a.max_steps ? (int)g : a.max_steps;
    if (e < 0) e = 0;
    while (e > 0 && !(lattice_t(near, e - 1, dt) < far)) --e;
    while (e < a.max_steps && lattice_t(near, e, dt) < far) ++e;
    return e;
}

// ---------------------------------------------------------------------------
// cone lattice
// ---------------------------------------------------------------------------

__device__ __forceinline__ float cone_step(const MarchArgs& a, float t) {
    float dt = __fmul_rn(t, a.cone);
    if (dt < a.dt_min) dt = a.dt_min;
    if (dt > a.dt_max) dt = a.dt_max;
    return __fadd_rn(t, dt);
}

// The lattice of rays starting at near_plane: table[k] = t_k, k = 0..max_steps.
__global__ void cone_table_kernel(const MarchArgs a, float* table) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    float t = a.near_plane;
    for (int k = 0; k <= a.max_steps; ++k) {
        table[k] = t;
        t = cone_step(a, t);
    }
}

// First k in [0, max_steps] with table[k] >= far (max_steps if none below it; the
// table is non-decreasing), found by the whole warp: each round probes 32 evenly
// spaced candidates, and the probes below far form a prefix of the lanes, which
// narrows the range by a factor of 32 (three rounds for 4096 steps).
__device__ __forceinline__ int table_count(const float* table, int max_steps, float far, int lane) {
    int lo = 0, hi = max_steps;  // table[k] < far for every k < lo; the answer is in [lo, hi]
    while (lo < hi) {
        const int step = (hi - lo + 31) >> 5;
        const int k = lo + lane * step;
        const unsigned below = __ballot_sync(FULL, k < hi && __ldg(table + k) < far);
        const int nb = __popc(below);
        if (nb == 0) break;  // table[lo] >= far
        hi = min(lo + nb * step, hi);
        lo = lo + (nb - 1) * step + 1;
    }
    return lo;
}

// Lane 0 extends a ray's own cone recurrence by 32 steps: buf[j] = t_{32c + j},
// j = 0..32, starting from *t (t_{32c}); *t becomes t_{32c + 32}.
__device__ __forceinline__ void cone_extend(const MarchArgs& a, float* buf, float& t, int lane) {
    if (lane == 0) {
        float v = t;
#pragma unroll 1
        for (int j = 0; j <= 32; ++j) {
            buf[j] = v;
            if (j < 32) v = cone_step(a, v);
        }
        t = v;
    }
    t = __shfl_sync(FULL, t, 0);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

constexpr size_t kTicketBytes = 256;

// Ballot words of the longest lattice. With cone steps the lattice from
// near_plane is the densest (a later start only lengthens every step: the step
// is non-decreasing in t) and no ray's far exceeds far_plane, so its length up
// to far_plane bounds every ray's; 32 points of margin, and kernels check it.
int mask_words_for(const nacc_march_params* p) {
    const int full = (p->max_steps + 31) / 32;
    if (!(p->cone > 0.0f)) return full;
    float t = p->near_plane;
    int k = 0;
    while (k < p->max_steps && t < p->far_plane) {
        float dt = t * p->cone;
        if (dt < p->dt_min) dt = p->dt_min;
        if (dt > p->dt_max) dt = p->dt_max;
        t = t + dt;
        ++k;
    }
    const int words = (k + 32 + 31) / 32;
    return words < full ? words : full;
}

// Rays per warp tile: at most the knob, fewer when long lattices make the ballot
// rows big (each of the warp's two tile buffers stays within kWarpSmemBudget bytes).
constexpr size_t kWarpSmemBudget = 2048;
int tile_rays_for(int mask_words) {
    int t = (int)(kWarpSmemBudget / ((size_t)mask_words * sizeof(uint32_t)));
    const int cap = tune_get(NACC_TUNE_MARCH_TILE_RAYS);
    if (t > cap) t = cap;
    if (t < 1) t = 1;
    return t;
}

size_t status_bytes_for(int32_t n_rays) {
    // the smallest warp tile is one ray: size for one status word per ray
    return align_up(kTicketBytes + (size_t)n_rays * sizeof(unsigned long long), 256);
}

size_t workspace_bytes_for(int32_t n_rays, const nacc_march_params* p) {
    size_t b = status_bytes_for(n_rays);
    if (p && p->cone > 0.0f && p->max_steps >= 1)
        b += align_up(((size_t)p->max_steps + 1) * sizeof(float), 256);
    return b;
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
int blocks_for(K kernel, size_t smem, int n_work_blocks) {
    const DeviceInfo dev = current_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int want = dev.sm_count * per_sm;
    return n_work_blocks < want ? n_work_blocks : want;
}

// The shape of a grid (levels, slots, resolution, box, contraction); bits are
// checked by the caller.
int check_grid(const nacc_grid* grid) {
    if (!grid) return NACC_ERR_INVALID_ARG;
    if (grid->n_levels < 1 || grid->n_levels > NACC_MAX_LEVELS || grid->n_slots < 1) return NACC_ERR_INVALID_ARG;
    if (grid->contraction != 0 && (grid->contraction != 1 || grid->n_levels != 1)) return NACC_ERR_INVALID_ARG;
    if (grid->res[0] < 1 || grid->res[1] < 1 || grid->res[2] < 1) return NACC_ERR_INVALID_ARG;
    if (grid->res[0] > (1 << 22) || grid->res[1] > (1 << 22) || grid->res[2] > (1 << 22)) return NACC_ERR_INVALID_ARG;
    const long long cells = (long long)grid->res[0] * grid->res[1] * grid->res[2] * grid->n_levels * grid->n_slots;
    if (cells >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    const long long corners = (grid->res[0] + 1LL) * (grid->res[1] + 1LL) * (grid->res[2] + 1LL) * grid->n_levels *
                              grid->n_slots;  // entries of the summed-area table
    if (grid->sat && (corners >= (1LL << 31) || ((uintptr_t)grid->sat & 1u))) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 6; ++k)
        if (!(fabsf(grid->aabb[k]) < INFINITY)) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(grid->aabb[k] < grid->aabb[3 + k])) return NACC_ERR_INVALID_ARG;
    return NACC_OK;
}

// Contraction constants of a grid's box: centre, 1 / half size, res / 4.
void contraction_consts(const nacc_grid& grid, float cc[3], float inv_h[3], float qres[3]) {
    for (int k = 0; k < 3; ++k) {
        const float lo = grid.aabb[k], hi = grid.aabb[3 + k];
        cc[k] = (lo + hi) * 0.5f;
        inv_h[k] = 1.0f / ((hi - lo) * 0.5f);
        qres[k] = (float)grid.res[k] * 0.25f;
    }
}

// A scene's geometry as the batched kernels read it (the grid checked already).
void scene_geom_for(const nacc_grid& grid, SceneGeom& g) {
    memset(&g, 0, sizeof(g));
    g.bits = grid.bits;
    g.sat = grid.sat;
    for (int k = 0; k < 3; ++k) g.res[k] = grid.res[k];
    g.n_levels = grid.n_levels;
    make_levels(grid, g.L);
    contraction_consts(grid, g.cc, g.inv_h, g.qres);
}

// Checks the arguments every marching entry point shares (rays, grid, step
// parameters) and fills the corresponding fields of `a` (zeroing the rest).
int march_setup(const float* rays_o, const float* rays_d, const float* ray_time, const int32_t* ray_slot,
                int32_t n_rays, const nacc_grid* grid, const nacc_march_params* p, MarchArgs& a) {
    if (n_rays < 0 || !grid || !p) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!rays_o || !rays_d || !grid->bits)) return NACC_ERR_INVALID_ARG;
    if (check_grid(grid) != NACC_OK) return NACC_ERR_INVALID_ARG;
    if (p->max_steps < 1 || p->max_steps > 32768) return NACC_ERR_INVALID_ARG;
    if (!(p->dt_min > 0.0f) || !(p->dt_min < INFINITY) || p->cone < 0.0f || !(p->cone < INFINITY))
        return NACC_ERR_INVALID_ARG;
    if (p->cone > 0.0f && !(p->dt_max >= p->dt_min)) return NACC_ERR_INVALID_ARG;

    memset(&a, 0, sizeof(a));
    a.rays_o = rays_o;
    a.rays_d = rays_d;
    a.ray_time = ray_time;
    a.ray_slot = ray_slot;
    a.n_rays = n_rays;
    a.bits = grid->bits;
    a.sat = grid->sat;
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
    a.inv_dt = 1.0f / p->dt_min;
    a.dt_max = p->dt_max;
    a.cone = p->cone;
    a.max_steps = p->max_steps;
    a.mask_words = mask_words_for(p);
    a.row_stride = a.mask_words;
    make_levels(*grid, a.L);
    a.contract = grid->contraction;
    contraction_consts(*grid, a.cc, a.inv_h, a.qres);
    return NACC_OK;
}

}  // namespace
}  // namespace nacc
