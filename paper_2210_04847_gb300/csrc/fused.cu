// fused.cu -- marching with the density field's transmittance, for inference
// (NerfAcc, arXiv 2210.04847, Sec. 2.1 "Pruning Empty and Occluded Regions":
// empty space is skipped with the occupancy grid and marching stops where the
// transmittance from the field's density falls below eps; "GPU Memory
// Efficiency": only the samples that matter are ever written).
//
// The field is a density grid the kernel can evaluate itself: float32 sigma at
// the vertices of a lattice over a box, trilinear in between, zero outside
// (nacc_density_field). Result: exactly what nacc_march_rays followed by
// nacc_prune_samples keeps with sigma_i = the field at each sample's midpoint;
// the work stops at each ray's termination point instead of the far plane, and
// the marched-but-dropped samples are never stored.
//
// Layout of the work is the marcher's (march.cu): a warp takes tiles of
// consecutive rays from an atomic ticket, walks each ray 32 lattice points at
// a time (lane j: point 32c + j), and turns the decisions into one ballot word
// per chunk in its private shared memory; tiles go two deep through a bounded
// decoupled look-back; the words are then expanded into compacted stores. Per
// chunk the lanes whose midpoint is occupied also evaluate the field, form
// tau = sigma * delta, and the warp scans tau (float32 shuffle scan plus the
// ray's running optical depth) to decide T_i >= eps and alpha_i >= thre. The
// walk of a ray ends once its optical depth passes -ln(eps). Compiled with
// -fmad=false; every float operation on the decision path is explicitly rounded.
#include "march_common.cuh"

namespace nacc {
namespace {

struct FieldArgs {
    const float* sigma;
    int32_t g1, g2;         // vertices along y and z (x-major, z fastest)
    int32_t im0, im1, im2;  // largest lower vertex index per axis: res - 2
    float lo[3];            // box corner
    float s[3];             // (res - 1) / (hi - lo), float32
    float umax[3];          // res - 1
};

struct FusedArgs {
    MarchArgs m;
    FieldArgs f;
    float* sigmas_out;
    int32_t use_t, use_a;
    float thr_o, thr_tau;
};

__device__ __forceinline__ float lerp_rn(float p, float q, float t) {
    return __fadd_rn(p, __fmul_rn(t, __fsub_rn(q, p)));
}

// sigma at x: trilinear between the eight vertices around x (z, then y, then x),
// zero outside the box (and for NaN coordinates).
__device__ __forceinline__ float field_sigma(const FieldArgs& f, float x0, float x1, float x2) {
    const float u0 = __fmul_rn(__fsub_rn(x0, f.lo[0]), f.s[0]);
    const float u1 = __fmul_rn(__fsub_rn(x1, f.lo[1]), f.s[1]);
    const float u2 = __fmul_rn(__fsub_rn(x2, f.lo[2]), f.s[2]);
    if (!(u0 >= 0.0f && u0 <= f.umax[0] && u1 >= 0.0f && u1 <= f.umax[1] && u2 >= 0.0f && u2 <= f.umax[2]))
        return 0.0f;
    const int i0 = min(__float2int_rd(u0), f.im0);
    const int i1 = min(__float2int_rd(u1), f.im1);
    const int i2 = min(__float2int_rd(u2), f.im2);
    const float f0 = __fsub_rn(u0, __int2float_rn(i0));
    const float f1 = __fsub_rn(u1, __int2float_rn(i1));
    const float f2 = __fsub_rn(u2, __int2float_rn(i2));
    const size_t sy = (size_t)f.g2, sx = (size_t)f.g1 * f.g2;
    const float* p = f.sigma + (size_t)i0 * sx + (size_t)i1 * sy + i2;
    const float c00 = lerp_rn(__ldg(p), __ldg(p + 1), f2);
    const float c01 = lerp_rn(__ldg(p + sy), __ldg(p + sy + 1), f2);
    const float c10 = lerp_rn(__ldg(p + sx), __ldg(p + sx + 1), f2);
    const float c11 = lerp_rn(__ldg(p + sx + sy), __ldg(p + sx + sy + 1), f2);
    return lerp_rn(lerp_rn(c00, c01, f1), lerp_rn(c10, c11, f1), f0);
}

// Lattice interval k of a ray: [ts, tn) before the clip at far. Own cone
// lattices come from the warp's shared buffer (extended by the caller).
template <bool CONE>
__device__ __forceinline__ void interval(const MarchArgs& a, bool shared, float near, int k, const float* lat, int lane,
                                         float& ts, float& tn) {
    if (!CONE) {
        const float kf = __int2float_rn(k);
        ts = __fadd_rn(near, __fmul_rn(kf, a.dt_min));
        tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), a.dt_min));
    } else if (shared) {
        ts = __ldg(a.cone_table + min(k, a.max_steps));
        tn = __ldg(a.cone_table + min(k + 1, a.max_steps));
    } else {
        ts = lat[lane];
        tn = lat[lane + 1];
    }
}

// Phase 1 of one ray, all 32 lanes: one word of keep decisions per 32 lattice
// points into row[c]. count = kept samples, nch = words written, pts = lattice
// points examined (up to the termination point).
template <int MAXL, bool CONE>
__device__ __forceinline__ void fused_walk(const FusedArgs& A, const float o[3], const float d[3], float near,
                                           float far, uint32_t* row, float* lat, int lane, int& count_out,
                                           int& nch_out, int& pts_out) {
    const MarchArgs& a = A.m;
    const bool shared = !CONE || near == a.near_plane;
    int nk = !CONE ? lattice_count(a, near, far, a.dt_min)
                   : (shared ? table_count(a.cone_table, a.max_steps, far, lane) : a.max_steps);
    if (CONE && shared && nk > 32 * a.mask_words) {
        if (lane == 0) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
        nk = 32 * a.mask_words;
    }
    const int max_ch = min((nk + 31) >> 5, a.mask_words);
    float carry = 0.0f;  // optical depth of the ray's samples before this chunk
    float tcur = near;
    int count = 0, nch = 0, pts = 0, c = 0;
    bool ended = false;
    for (; c < max_ch; ++c) {
        const int k = (c << 5) + lane;
        if (CONE && !shared) cone_extend(a, lat, tcur, lane);
        float ts, tn;
        interval<CONE>(a, shared, near, k, lat, lane, ts, tn);
        const bool valid = k < nk && ts < far;
        const unsigned vmask = __ballot_sync(FULL, valid);
        if (CONE && !shared && vmask == 0u) {
            ended = true;
            break;
        }
        pts += __popc(vmask);
        bool occ = false;
        float tau = 0.0f;
        if (valid) {
            const float te = tn < far ? tn : far;
            const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
            const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
            const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
            const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
            occ = occupied<MAXL>(a, x0, x1, x2, 0u);
            if (occ) tau = __fmul_rn(field_sigma(A.f, x0, x1, x2), __fsub_rn(te, ts));
        }
        nch = c + 1;
        if (__ballot_sync(FULL, occ) == 0u) {  // an empty chunk: no sample, the optical depth is unchanged
            if (lane == 0) row[c] = 0u;
            continue;
        }
        const float incl = warp_incl_scan(tau, lane);
        float excl = __shfl_up_sync(FULL, incl, 1);
        if (lane == 0) excl = 0.0f;
        bool keep = occ;
        if (A.use_t) keep = keep && __fadd_rn(carry, excl) <= A.thr_o;
        if (A.use_a) keep = keep && tau >= A.thr_tau;
        const unsigned m = __ballot_sync(FULL, keep);
        if (lane == 0) row[c] = m;
        count += __popc(m);
        carry = __fadd_rn(carry, __shfl_sync(FULL, incl, 31));
        // every later sample has O_i >= carry (tau >= 0): the rest of the ray is not marched
        if (A.use_t && !(carry <= A.thr_o)) {
            ended = true;
            break;
        }
    }
    // an own cone lattice that still had points beyond the rows' capacity
    if (CONE && !shared && !ended && c == a.mask_words && (c << 5) < a.max_steps && tcur < far && lane == 0)
        raise_status(a.d_status, NACC_STATUS_OVERFLOW);
    count_out = count;
    nch_out = nch;
    pts_out = pts;
}

struct FusedTile {
    int tile, ray0, nr, agg;
    int my_count, my_nch, incl;
    float my_near, my_far;
};

// The tile's offset by look-back, then the decision words expanded into
// compacted, coalesced stores of (t_start, t_end, ray[, sigma]).
template <bool CONE>
__device__ __forceinline__ void fused_finish(const FusedArgs& A, const uint32_t* wmask, const FusedTile& t, float* lat,
                                             int lane) {
    const MarchArgs& a = A.m;
    const unsigned lt = lanemask_lt();
    const long long excl =
        (long long)resolve_prefix(a.tile_status, t.tile, (unsigned long long)t.agg, lane, a.d_status, a.hooks);
    const int my_excl = t.incl - t.my_count;
    if (lane < t.nr) {
        const int2 pi = make_int2((int)(excl + my_excl), t.my_count);
        reinterpret_cast<int2*>(a.packed_info)[t.ray0 + lane] = pi;
    }
    if (lane == 0 && t.tile == a.n_tiles - 1) {
        const long long total = excl + t.agg;
        *a.n_samples = total;
        if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
        if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
    }
    if (excl >= a.capacity) return;
    const unsigned cap = (unsigned)(a.capacity < 0x7fffffffLL ? a.capacity : 0x7fffffffLL);
    for (int i = 0; i < t.nr; ++i) {
        const int cnt = __shfl_sync(FULL, t.my_count, i);
        if (cnt == 0) continue;
        const int nch = __shfl_sync(FULL, t.my_nch, i);
        const float near = __shfl_sync(FULL, t.my_near, i);
        const float far = __shfl_sync(FULL, t.my_far, i);
        const bool shared = !CONE || near == a.near_plane;
        const int r = t.ray0 + i;
        float o[3], d[3];
        if (A.sigmas_out) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
                d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
            }
        }
        const uint32_t* row = wmask + i * a.row_stride;
        unsigned base = (unsigned)excl + (unsigned)__shfl_sync(FULL, my_excl, i);
        float tcur = near;
        for (int c = 0; c < nch; ++c) {
            const unsigned m = row[c];
            if (shared && m == 0u) continue;  // an own cone lattice is extended chunk by chunk
            if (CONE && !shared) cone_extend(a, lat, tcur, lane);
            if (m == 0u) continue;
            const int k = (c << 5) + lane;
            float ts, tn;
            interval<CONE>(a, shared, near, k, lat, lane, ts, tn);
            const unsigned pos = base + __popc(m & lt);
            if (((m >> lane) & 1u) && pos < cap) {
                const float te = tn < far ? tn : far;
                a.t_starts[pos] = ts;
                a.t_ends[pos] = te;
                a.ray_indices[pos] = r;
                if (A.sigmas_out) {
                    const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                    A.sigmas_out[pos] = field_sigma(A.f, __fadd_rn(o[0], __fmul_rn(d[0], mid)),
                                                    __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                                    __fadd_rn(o[2], __fmul_rn(d[2], mid)));
                }
            }
            base += __popc(m);
        }
    }
}

template <int MAXL, int MINB, bool CONE>
__global__ void __launch_bounds__(kThreads, MINB) march_fused_kernel(const FusedArgs A) {
    extern __shared__ uint32_t s_masks[];  // per warp: 2 x [tile_rays][row_stride]
    __shared__ float s_lat[kWarps][36];
    const MarchArgs& a = A.m;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t tile_words = (size_t)a.tile_rays * a.row_stride;
    uint32_t* wbase = s_masks + (size_t)warp * 2 * tile_words;
    float* lat = s_lat[warp];

    FusedTile prev;
    bool have_prev = false;
    int buf = 0;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = (int)atomicAdd(a.ticket, 1u);
        tile = __shfl_sync(FULL, tile, 0);
        const bool have = tile < a.n_tiles;
        FusedTile cur;
        if (have) {
            uint32_t* wmask = wbase + buf * tile_words;
            cur.tile = tile;
            cur.ray0 = tile * a.tile_rays;
            cur.nr = min(a.tile_rays, a.n_rays - cur.ray0);
            int my_count = 0, my_nch = 0;
            float my_near = 0.0f, my_far = 0.0f;
            int tile_pts = 0;  // at most tile_rays * max_steps
            for (int i = 0; i < cur.nr; ++i) {
                const int r = cur.ray0 + i;
                float o[3], d[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
                    d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
                }
                float near = 0.0f, far = 0.0f;
                int count = 0, nch = 0, pts = 0;
                if (clip_ray<MAXL == 0>(a, o, d, near, far))
                    fused_walk<MAXL, CONE>(A, o, d, near, far, wmask + i * a.row_stride, lat, lane, count, nch, pts);
                tile_pts += pts;
                if (lane == i) {
                    my_count = count;
                    my_nch = nch;
                    my_near = near;
                    my_far = far;
                }
            }
            __syncwarp();
            if (lane == 0 && tile_pts > 0) atomicAdd(a.lattice_points, (unsigned long long)tile_pts);
            cur.my_count = my_count;
            cur.my_nch = my_nch;
            cur.my_near = my_near;
            cur.my_far = my_far;
            cur.incl = warp_incl_scan_int(cur.my_count, lane);
            cur.agg = __shfl_sync(FULL, cur.incl, 31);
            publish_aggregate(a.tile_status, cur.tile, (unsigned long long)cur.agg, lane, a.hooks);
        }
        if (have_prev) {
            fused_finish<CONE>(A, wbase + (buf ^ 1) * tile_words, prev, lat, lane);
            __syncwarp();
        }
        if (!have) break;
        prev = cur;
        have_prev = true;
        buf ^= 1;
    }
}

// sigma of the field at each sample's midpoint x = o + d * (t_start + t_end) / 2
// (the point the marcher looks up), one thread per sample.
__global__ void field_at_samples_kernel(const FieldArgs f, const float* __restrict__ rays_o,
                                        const float* __restrict__ rays_d, const int32_t* __restrict__ ray_indices,
                                        const float* __restrict__ t_starts, const float* __restrict__ t_ends,
                                        int64_t n, int32_t n_rays, float* __restrict__ sigmas,
                                        int32_t* d_status) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int r = __ldg(ray_indices + s);
        if ((unsigned)r >= (unsigned)n_rays) {
            raise_status(d_status, NACC_STATUS_BAD_INDEX);
            sigmas[s] = 0.0f;
            continue;
        }
        const float mid = __fmul_rn(__fadd_rn(__ldg(t_starts + s), __ldg(t_ends + s)), 0.5f);
        float x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            x[k] = __fadd_rn(__ldg(rays_o + 3 * (size_t)r + k), __fmul_rn(__ldg(rays_d + 3 * (size_t)r + k), mid));
        sigmas[s] = field_sigma(f, x[0], x[1], x[2]);
    }
}

// sigma of the field at points xyz (n, 3).
__global__ void field_at_points_kernel(const FieldArgs f, const float* __restrict__ xyz, int64_t n,
                                       float* __restrict__ sigmas) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        sigmas[s] = field_sigma(f, __ldg(xyz + 3 * s), __ldg(xyz + 3 * s + 1), __ldg(xyz + 3 * s + 2));
}

int field_setup(const nacc_density_field* field, FieldArgs& f) {
    if (!field || !field->sigma) return NACC_ERR_INVALID_ARG;
    long long n = 1;
    for (int k = 0; k < 3; ++k) {
        if (field->res[k] < 2) return NACC_ERR_INVALID_ARG;
        if (!(fabsf(field->aabb[k]) < INFINITY) || !(fabsf(field->aabb[3 + k]) < INFINITY)) return NACC_ERR_INVALID_ARG;
        if (!(field->aabb[k] < field->aabb[3 + k])) return NACC_ERR_INVALID_ARG;
        n *= field->res[k];
        if (n >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    }
    f.sigma = field->sigma;
    f.g1 = field->res[1];
    f.g2 = field->res[2];
    f.im0 = field->res[0] - 2;
    f.im1 = field->res[1] - 2;
    f.im2 = field->res[2] - 2;
    for (int k = 0; k < 3; ++k) {
        const float lo = field->aabb[k], hi = field->aabb[3 + k];
        f.lo[k] = lo;
        f.s[k] = (float)(field->res[k] - 1) / (hi - lo);
        f.umax[k] = (float)(field->res[k] - 1);
    }
    return NACC_OK;
}

template <int MAXL>
void launch_fused(bool cone, size_t smem, int need, cudaStream_t st, const FusedArgs& A) {
    const bool cap = tune_get(NACC_TUNE_FUSED_OCCUPANCY) != 0;  // 4 blocks of 256 threads: <= 64 registers
    auto kernel = cone ? (cap ? march_fused_kernel<MAXL, 4, true> : march_fused_kernel<MAXL, 1, true>)
                       : (cap ? march_fused_kernel<MAXL, 4, false> : march_fused_kernel<MAXL, 1, false>);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = blocks_for(kernel, smem, need);
    kernel<<<blocks, kThreads, smem, st>>>(A);
}

int grid_blocks(int64_t n) {
    const DeviceInfo dev = current_device();
    const int64_t want = (n + 255) / 256;
    const int64_t cap = (int64_t)dev.sm_count * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_march_fused(const float* rays_o, const float* rays_d, int32_t n_rays, const nacc_grid* grid,
                                const nacc_march_params* p, const nacc_density_field* field, float early_stop_eps,
                                float alpha_thre, int32_t* packed_info, float* t_starts, float* t_ends,
                                int32_t* ray_indices, float* sigmas, int64_t capacity, int64_t* n_samples,
                                int32_t* d_status, void* workspace, size_t workspace_bytes, void* stream) {
    if (capacity < 0 || !n_samples) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (capacity > 0 && (!t_starts || !t_ends || !ray_indices)) return NACC_ERR_INVALID_ARG;
    if (early_stop_eps != early_stop_eps || alpha_thre != alpha_thre) return NACC_ERR_INVALID_ARG;
    FusedArgs A;
    const int setup = march_setup(rays_o, rays_d, nullptr, nullptr, n_rays, grid, p, A.m);
    if (setup != NACC_OK) return setup;
    const int fs = field_setup(field, A.f);
    if (fs != NACC_OK) return fs;
    if (!workspace || workspace_bytes < workspace_bytes_for(n_rays, p)) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)packed_info & 7u) != 0) return NACC_ERR_INVALID_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays == 0) return launch_status(cudaMemsetAsync(n_samples, 0, sizeof(int64_t), st));

    MarchArgs& a = A.m;
    a.packed_info = packed_info;
    a.t_starts = t_starts;
    a.t_ends = t_ends;
    a.ray_indices = ray_indices;
    a.capacity = capacity;
    a.n_samples = n_samples;
    a.d_status = d_status;
    a.ticket = (unsigned int*)workspace;
    a.lattice_points = (unsigned long long*)((char*)workspace + 8);
    a.tile_status = (unsigned long long*)((char*)workspace + kTicketBytes);
    a.hooks = lookback_hooks();
    a.tile_rays = tile_rays_for(a.mask_words);
    A.sigmas_out = capacity > 0 ? sigmas : nullptr;
    A.use_t = early_stop_eps > 0.0f;
    A.use_a = alpha_thre > 0.0f;
    A.thr_o = A.use_t ? (float)(-log((double)early_stop_eps)) : INFINITY;
    A.thr_tau = A.use_a ? (float)(-log1p(-(double)alpha_thre)) : 0.0f;

    a.n_tiles = (n_rays + a.tile_rays - 1) / a.tile_rays;
    const size_t clear = kTicketBytes + (size_t)a.n_tiles * sizeof(unsigned long long);
    if (cudaMemsetAsync(workspace, 0, clear, st) != cudaSuccess) return NACC_ERR_CUDA;
    const bool cone = p->cone > 0.0f;
    if (cone) {
        float* table = (float*)((char*)workspace + status_bytes_for(n_rays));
        a.cone_table = table;
        cone_table_kernel<<<1, 32, 0, st>>>(a, table);
    }
    const size_t smem = (size_t)kWarps * 2 * a.tile_rays * a.row_stride * sizeof(uint32_t);
    const int need = (a.n_tiles + kWarps - 1) / kWarps;
    if (a.contract) launch_fused<0>(cone, smem, need, st, A);
    else if (a.n_levels == 1) launch_fused<1>(cone, smem, need, st, A);
    else if (a.n_levels <= 4) launch_fused<4>(cone, smem, need, st, A);
    else launch_fused<NACC_MAX_LEVELS>(cone, smem, need, st, A);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_density_field_at_samples(const nacc_density_field* field, const float* rays_o,
                                             const float* rays_d, int32_t n_rays, const int32_t* ray_indices,
                                             const float* t_starts, const float* t_ends, int64_t n_samples,
                                             float* sigmas, int32_t* d_status, void* stream) {
    FieldArgs f;
    const int fs = field_setup(field, f);
    if (fs != NACC_OK) return fs;
    if (n_samples < 0 || n_rays < 0) return NACC_ERR_INVALID_ARG;
    if (n_samples == 0) return NACC_OK;
    if (!rays_o || !rays_d || !ray_indices || !t_starts || !t_ends || !sigmas) return NACC_ERR_INVALID_ARG;
    field_at_samples_kernel<<<grid_blocks(n_samples), 256, 0, (cudaStream_t)stream>>>(
        f, rays_o, rays_d, ray_indices, t_starts, t_ends, n_samples, n_rays, sigmas, d_status);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_density_field_query(const nacc_density_field* field, const float* xyz, int64_t n, float* sigmas,
                                        void* stream) {
    FieldArgs f;
    const int fs = field_setup(field, f);
    if (fs != NACC_OK) return fs;
    if (n < 0) return NACC_ERR_INVALID_ARG;
    if (n == 0) return NACC_OK;
    if (!xyz || !sigmas) return NACC_ERR_INVALID_ARG;
    field_at_points_kernel<<<grid_blocks(n), 256, 0, (cudaStream_t)stream>>>(f, xyz, n, sigmas);
    return launch_status(cudaGetLastError());
}
