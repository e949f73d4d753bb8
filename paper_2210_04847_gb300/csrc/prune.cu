// prune.cu -- pruning of marched samples by transmittance (early stop) and
// opacity (alpha threshold), then re-packing (NerfAcc, arXiv 2210.04847,
// Sec. 2.1 "Pruning Empty and Occluded Regions"; early_stop_eps and
// alpha_thre of the Sec. 3 listing).
//
// Single pass over the input samples. Each warp takes tiles of consecutive rays
// from an atomic ticket and keeps two (or four) rays in flight (independent
// load streams; a slot whose ray has ended takes the tile's next ray), in
// chunks of 64 samples: lane j loads samples 2j and 2j+1 of
// the chunk as one 8-byte vector per array (chunks start at an even index).
// It forms tau = sigma*delta, the exclusive optical depth by a warp shuffle
// scan of the lane pairs plus a running carry, and the keep decisions; two
// __ballot_sync words per chunk (even and odd samples) go to a workspace row of
// the ray. Once the optical depth passes -ln(eps) the rest of the ray is
// dropped without being read. A bounded decoupled look-back run by the warp
// turns the tile's kept count into its output offset, and the warp re-expands
// the ballot words into compacted stores. Compiled with -fmad=false (tau and the
// scan are explicitly rounded float32 operations).
#include <math.h>
#include <string.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr size_t kTicketBytes = 256;

struct PruneArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* t_starts;
    const float* t_ends;
    const float* sigmas;
    int64_t n_samples;
    int use_t, use_a;
    float thr_o, thr_tau;
    int32_t* packed_info_out;
    float* t_starts_out;
    float* t_ends_out;
    int32_t* ray_indices_out;
    int64_t capacity;
    int64_t* n_kept;
    uint8_t* keep_mask;
    int32_t* d_status;
    unsigned long long* tile_status;
    unsigned int* ticket;
    unsigned long long* examined;  // input samples read, summed over rays (diagnostic)
    uint32_t* masks;
    int32_t n_tiles;
    int32_t tile_rays;
    LookbackHooks hooks;  // look-back poll budget (test hooks)
};

// Row of ballot words of ray r whose run starts at `off`: two words per 64-sample
// chunk. Rows of rays with ascending, disjoint runs never overlap: ray r needs at
// most floor(cnt/32) + 2 words and the next row starts at least that far on.
__device__ __forceinline__ uint32_t* mask_row(const PruneArgs& a, int off, int r) {
    return a.masks + (off >> 5) + 2 * (size_t)r;
}

// One ray's walk state inside phase 1 (32-bit indices: n_samples < 2^31).
struct RayWalk {
    int j;        // this lane's first sample of the current chunk: (off & ~1) + 64 c + 2 lane
    int off, cnt; // the ray's run [off, off + cnt)
    int nch, c, count;
    float carry;
    uint32_t* row;
    bool live;
};

__device__ __forceinline__ void walk_init(RayWalk& w, const PruneArgs& a, int off, int cnt, int r, int lane) {
    w.off = off;
    w.cnt = cnt;
    w.j = (off & ~1) + 2 * lane;
    w.nch = cnt > 0 ? (cnt + (off & 1) + 63) >> 6 : 0;
    w.c = 0;
    w.count = 0;
    w.carry = 0.0f;
    w.row = mask_row(a, off, r);
    w.live = w.nch > 0;
}

struct Pair {
    float s0[2], s1[2], sg[2];
    bool v0, v1;  // samples j and j + 1 belong to the ray
};

// Samples j and j + 1 of the lane in the current chunk (only those inside the ray
// are read; a pair whose second sample is inside is read as one 8-byte vector).
__device__ __forceinline__ void walk_load(const RayWalk& w, const PruneArgs& a, Pair& p) {
    p.s0[0] = p.s0[1] = p.s1[0] = p.s1[1] = p.sg[0] = p.sg[1] = 0.0f;
    p.v0 = w.live && (unsigned)(w.j - w.off) < (unsigned)w.cnt;
    p.v1 = w.live && (unsigned)(w.j + 1 - w.off) < (unsigned)w.cnt;
    if (p.v1) {
        const float2 u = __ldg(reinterpret_cast<const float2*>(a.t_starts + w.j));
        const float2 v = __ldg(reinterpret_cast<const float2*>(a.t_ends + w.j));
        const float2 g = __ldg(reinterpret_cast<const float2*>(a.sigmas + w.j));
        p.s0[0] = u.x; p.s0[1] = u.y;
        p.s1[0] = v.x; p.s1[1] = v.y;
        p.sg[0] = g.x; p.sg[1] = g.y;
    } else if (p.v0) {
        p.s0[0] = __ldg(a.t_starts + w.j);
        p.s1[0] = __ldg(a.t_ends + w.j);
        p.sg[0] = __ldg(a.sigmas + w.j);
    }
}

// Decide one chunk of 64 samples of the ray (call with w.live, warp-uniform).
__device__ __forceinline__ void walk_step(RayWalk& w, const PruneArgs& a, int lane, const Pair& p) {
    const float tau0 = p.v0 ? __fmul_rn(p.sg[0], __fsub_rn(p.s1[0], p.s0[0])) : 0.0f;
    const float tau1 = p.v1 ? __fmul_rn(p.sg[1], __fsub_rn(p.s1[1], p.s0[1])) : 0.0f;
    const float incl = warp_incl_scan(__fadd_rn(tau0, tau1), lane);
    float excl = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) excl = 0.0f;
    const float O0 = __fadd_rn(w.carry, excl);
    const float O1 = __fadd_rn(O0, tau0);
    bool k0 = p.v0, k1 = p.v1;
    if (a.use_t) {
        k0 = k0 && (O0 <= a.thr_o);
        k1 = k1 && (O1 <= a.thr_o);
    }
    if (a.use_a) {
        k0 = k0 && (tau0 >= a.thr_tau);
        k1 = k1 && (tau1 >= a.thr_tau);
    }
    const unsigned m0 = __ballot_sync(FULL, k0);
    const unsigned m1 = __ballot_sync(FULL, k1);
    if (lane == 0) {
        w.row[2 * w.c] = m0;
        w.row[2 * w.c + 1] = m1;
    }
    w.count += __popc(m0) + __popc(m1);
    w.carry = __fadd_rn(w.carry, __shfl_sync(FULL, incl, 31));
    ++w.c;
    w.j += 64;
    // every later O_i >= carry once tau >= 0: the rest of the ray is dropped unread
    if (w.c >= w.nch || (a.use_t && !(w.carry <= a.thr_o))) w.live = false;
}

// ---------------------------------------------------------------------------
// phase 1, register walk: IL rays at a time, their chunks loaded into registers
// ---------------------------------------------------------------------------

template <int IL>
__device__ __forceinline__ void phase1_walk(const PruneArgs& a, int ray0, int nr, int my_off, int my_cnt, int lane,
                                            int& my_count, int& my_nch) {
    // IL rays in flight; a slot whose ray has ended takes the tile's next ray, so
    // the warp keeps IL load streams going while the tile has rays left
    RayWalk W[IL];
    int held[IL];  // tile-local index of the ray in each slot, -1 when empty
    int next = 0;
    auto start = [&](int j) {
        held[j] = -1;
        W[j].live = false;
        while (next < nr) {
            const int r = next++;
            const int off = __shfl_sync(FULL, my_off, r & 31);
            const int cnt = __shfl_sync(FULL, my_cnt, r & 31);
            walk_init(W[j], a, off, cnt, ray0 + r, lane);
            if (W[j].live) {
                held[j] = r;
                return;
            }
            if (lane == r) {  // a ray without samples
                my_count = 0;
                my_nch = 0;
            }
        }
    };
#pragma unroll
    for (int j = 0; j < IL; ++j) start(j);
    for (;;) {
        bool any = false;
#pragma unroll
        for (int j = 0; j < IL; ++j) any |= W[j].live;
        if (!any) break;
        Pair P[IL];
#pragma unroll
        for (int j = 0; j < IL; ++j) walk_load(W[j], a, P[j]);
#pragma unroll
        for (int j = 0; j < IL; ++j)
            if (W[j].live) walk_step(W[j], a, lane, P[j]);
#pragma unroll
        for (int j = 0; j < IL; ++j) {
            if (!W[j].live && held[j] >= 0) {
                if (lane == held[j]) {
                    my_count = W[j].count;
                    my_nch = W[j].c;
                }
                start(j);
            }
        }
    }
}

// One tile between its decisions and its stores. Lane i holds ray i's run,
// kept count, chunks read and inclusive kept prefix within the tile.
struct TileState {
    int tile, ray0, nr, agg;
    int my_off, my_cnt, my_count, my_nch, incl;
};

// Phases 0 and 1 of a tile: validate the runs, decide every chunk (ballot rows
// in the workspace), then publish the tile's kept total for the look-back.
template <int IL>
__device__ __forceinline__ void decide_tile(const PruneArgs& a, int tile, int lane, TileState& t) {
    t.tile = tile;
    t.ray0 = tile * a.tile_rays;
    t.nr = min(a.tile_rays, a.n_rays - t.ray0);
    const int ray0 = t.ray0, nr = t.nr;

    // runs of the tile's rays: must be in bounds, ascending and disjoint in ray
    // order (the layout marching and pruning produce), so that the ballot rows
    // of different rays never overlap
    int my_off = 0, my_cnt = 0;
    if (lane < nr) {
        const int2 v = reinterpret_cast<const int2*>(a.packed_info)[ray0 + lane];
        my_off = v.x;
        my_cnt = v.y;
    }
    long long prev_end = __shfl_up_sync(FULL, (long long)my_off + my_cnt, 1);
    if (lane == 0) {
        prev_end = 0;
        if (ray0 > 0) {
            const int2 v = reinterpret_cast<const int2*>(a.packed_info)[ray0 - 1];
            prev_end = (long long)v.x + v.y;
        }
    }
    if (lane < nr) {
        bool bad = my_off < 0 || my_cnt < 0 || (long long)my_off + my_cnt > a.n_samples;
        if (my_cnt > 0 && (long long)my_off < prev_end && (ray0 + lane) > 0) bad = true;
        if (bad) {
            raise_status(a.d_status, NACC_STATUS_BAD_PACKED);
            my_off = 0;
            my_cnt = 0;
        }
    }

    // phase 1: keep decisions into the ballot rows, kept counts per ray
    int my_count = 0, my_nch = 0;
    phase1_walk<IL>(a, ray0, nr, my_off, my_cnt, lane, my_count, my_nch);
    __syncwarp();
    t.my_off = my_off;
    t.my_cnt = my_cnt;
    t.my_count = my_count;
    t.my_nch = my_nch;
    t.incl = warp_incl_scan_int(my_count, lane);
    t.agg = __shfl_sync(FULL, t.incl, 31);
    publish_aggregate(a.tile_status, tile, (unsigned long long)t.agg, lane, a.hooks);
}

// Phases 2 and 3 of a tile: its offset from the look-back, then the compacted
// stores of the kept samples (and the optional mask).
__device__ __forceinline__ void finish_tile(const PruneArgs& a, const TileState& t, int lane, unsigned lt) {
    const int ray0 = t.ray0, nr = t.nr;
    int seen = lane < nr ? min(t.my_cnt, (t.my_nch << 6) - (t.my_off & 1)) : 0;
    if (seen < 0) seen = 0;
    for (int o = 16; o > 0; o >>= 1) seen += __shfl_xor_sync(FULL, seen, o);
    const long long excl =
        (long long)resolve_prefix(a.tile_status, t.tile, (unsigned long long)t.agg, lane, a.d_status, a.hooks);
    const int my_excl = t.incl - t.my_count;
    if (lane < nr) {
        const int2 pi = make_int2((int)(excl + my_excl), t.my_count);
        reinterpret_cast<int2*>(a.packed_info_out)[ray0 + lane] = pi;
    }
    if (lane == 0) {
        atomicAdd(a.examined, (unsigned long long)seen);
        if (t.tile == a.n_tiles - 1) {
            const long long total = excl + t.agg;
            *a.n_kept = total;
            if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
            if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
        }
    }

    for (int i = 0; i < nr; ++i) {
        const int off = __shfl_sync(FULL, t.my_off, i);
        const int cnt = __shfl_sync(FULL, t.my_cnt, i);
        const int nch = __shfl_sync(FULL, t.my_nch, i);
        const int r = ray0 + i;
        const long long end = (long long)off + cnt;
        const long long abase = off & ~1;
        const uint32_t* row = mask_row(a, off, r);
        long long base = excl + __shfl_sync(FULL, my_excl, i);
        for (int c0 = 0; c0 < nch; c0 += 16) {
            // 16 chunks' ballot word pairs at once; two chunks per step, both
            // chunks' kept samples loaded (one 8-byte load per array per sample
            // pair) before either is stored
            const unsigned mw = (c0 + (lane >> 1) < nch) ? row[2 * c0 + lane] : 0u;
            const int n = min(16, nch - c0);
            for (int q = 0; q < n; q += 2) {
                unsigned m[2][2];
                long long j[2];
                float2 ts[2], te[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool ex = q + h < n;
                    m[h][0] = __shfl_sync(FULL, mw, (2 * (q + h)) & 31);
                    m[h][1] = __shfl_sync(FULL, mw, (2 * (q + h) + 1) & 31);
                    if (!ex) m[h][0] = m[h][1] = 0u;
                    j[h] = abase + ((long long)(c0 + q + h) << 6) + 2 * lane;
                    const bool k0 = (m[h][0] >> lane) & 1u, k1 = (m[h][1] >> lane) & 1u;
                    ts[h] = te[h] = make_float2(0.0f, 0.0f);
                    if (k0 || k1) {
                        if (j[h] + 1 < a.n_samples) {
                            ts[h] = __ldg(reinterpret_cast<const float2*>(a.t_starts + j[h]));
                            te[h] = __ldg(reinterpret_cast<const float2*>(a.t_ends + j[h]));
                        } else {  // the array's last sample, alone in its pair
                            ts[h].x = __ldg(a.t_starts + j[h]);
                            te[h].x = __ldg(a.t_ends + j[h]);
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const unsigned m0 = m[h][0], m1 = m[h][1];
                    const long long j0 = j[h];
                    const bool b0 = (m0 >> lane) & 1u, b1 = (m1 >> lane) & 1u;
                    if (a.keep_mask && q + h < n) {
                        if (j0 >= off && j0 < end) a.keep_mask[j0] = (uint8_t)b0;
                        if (j0 + 1 >= off && j0 + 1 < end) a.keep_mask[j0 + 1] = (uint8_t)b1;
                    }
                    const long long pos0 = base + __popc(m0 & lt) + __popc(m1 & lt);
                    if (b0 && pos0 < a.capacity) {
                        a.t_starts_out[pos0] = ts[h].x;
                        a.t_ends_out[pos0] = te[h].x;
                        a.ray_indices_out[pos0] = r;
                    }
                    const long long pos1 = pos0 + (b0 ? 1 : 0);
                    if (b1 && pos1 < a.capacity) {
                        a.t_starts_out[pos1] = ts[h].y;
                        a.t_ends_out[pos1] = te[h].y;
                        a.ray_indices_out[pos1] = r;
                    }
                    base += __popc(m0) + __popc(m1);
                }
            }
        }
        if (a.keep_mask) {
            const long long from = abase + ((long long)nch << 6);
            for (long long j = (from > off ? from : off) + lane; j < end; j += 32) a.keep_mask[j] = 0;
        }
    }
    __syncwarp();
}

// Tiles of consecutive rays taken from an atomic ticket, two deep: the warp
// decides a new tile and publishes its total before it waits for the offset of
// the tile it decided before (by then its predecessors have almost always
// published), so the look-back rarely stalls.
template <int IL>
__device__ __forceinline__ void prune_body(const PruneArgs& a) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    TileState prev;
    bool have_prev = false;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = (int)atomicAdd(a.ticket, 1u);
        tile = __shfl_sync(FULL, tile, 0);
        const bool have = tile < a.n_tiles;
        TileState cur;
        if (have) decide_tile<IL>(a, tile, lane, cur);
        if (have_prev) finish_tile(a, prev, lane, lt);
        if (!have) break;
        prev = cur;
        have_prev = true;
    }
}

// Register-budget variants (minimum resident blocks per SM), chosen by a tuning knob.
template <int MINB, int IL>
__global__ void __launch_bounds__(kThreads, MINB) prune_kernel(const PruneArgs a) {
    prune_body<IL>(a);
}

template <typename K>
void launch_persistent(K kernel, int need, cudaStream_t st, const PruneArgs& a) {
    const DeviceInfo dev = current_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int blocks = dev.sm_count * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kernel<<<blocks, kThreads, 0, st>>>(a);
}

template <int MINB>
void launch_variant(bool il4, int need, cudaStream_t st, const PruneArgs& a) {
    if (il4) launch_persistent(prune_kernel<MINB, 4>, need, st, a);
    else launch_persistent(prune_kernel<MINB, 2>, need, st, a);
}


// Persistent launch: as many blocks as fit on the GPU, at most `need`.

size_t workspace_bytes_for(int32_t n_rays, int64_t n_samples) {
    const size_t tiles = (size_t)(n_rays + 1) / 2;  // smallest tile: 2 rays
    const size_t head = align_up(kTicketBytes + tiles * sizeof(unsigned long long), 256);
    const size_t words = (size_t)(n_samples >> 5) + 2 * (size_t)n_rays + 4;
    return align_up(head + words * sizeof(uint32_t), 256);
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_prune_workspace_size(int32_t n_rays, int64_t n_samples) {
    if (n_rays < 0 || n_samples < 0) return 0;
    return workspace_bytes_for(n_rays, n_samples);
}

extern "C" int nacc_prune_samples(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                                  const float* t_ends, const float* sigmas, int64_t n_samples,
                                  float early_stop_eps, float alpha_thre, int32_t* packed_info_out,
                                  float* t_starts_out, float* t_ends_out, int32_t* ray_indices_out,
                                  int64_t capacity, int64_t* n_kept, uint8_t* keep_mask,
                                  int32_t* d_status, void* workspace, size_t workspace_bytes,
                                  void* stream) {
    if (n_rays < 0 || n_samples < 0 || capacity < 0 || !n_kept) return NACC_ERR_INVALID_ARG;
    if (n_samples >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!packed_info || !packed_info_out)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas)) return NACC_ERR_INVALID_ARG;
    if (capacity > 0 && (!t_starts_out || !t_ends_out || !ray_indices_out)) return NACC_ERR_INVALID_ARG;
    if (early_stop_eps != early_stop_eps || alpha_thre != alpha_thre) return NACC_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < workspace_bytes_for(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return NACC_ERR_INVALID_ARG;
    if ((((uintptr_t)packed_info | (uintptr_t)packed_info_out | (uintptr_t)t_starts | (uintptr_t)t_ends |
          (uintptr_t)sigmas) & 7u) != 0)
        return NACC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays == 0) return launch_status(cudaMemsetAsync(n_kept, 0, sizeof(int64_t), st));

    PruneArgs a;
    memset(&a, 0, sizeof(a));
    a.packed_info = packed_info;
    a.n_rays = n_rays;
    a.t_starts = t_starts;
    a.t_ends = t_ends;
    a.sigmas = sigmas;
    a.n_samples = n_samples;
    // thresholds of the decision, each rounded once to float32:
    // T_i >= eps  <=>  O_i <= -ln(eps);  alpha_i >= thre  <=>  tau_i >= -ln(1 - thre)
    a.use_t = early_stop_eps > 0.0f;
    a.use_a = alpha_thre > 0.0f;
    a.thr_o = a.use_t ? (float)(-log((double)early_stop_eps)) : INFINITY;
    a.thr_tau = a.use_a ? (float)(-log1p(-(double)alpha_thre)) : 0.0f;
    a.packed_info_out = packed_info_out;
    a.t_starts_out = t_starts_out;
    a.t_ends_out = t_ends_out;
    a.ray_indices_out = ray_indices_out;
    a.capacity = capacity;
    a.n_kept = n_kept;
    a.keep_mask = keep_mask;
    a.d_status = d_status;
    a.tile_rays = tune_get(NACC_TUNE_PRUNE_TILE_RAYS);
    a.n_tiles = (n_rays + a.tile_rays - 1) / a.tile_rays;
    a.ticket = (unsigned int*)workspace;
    a.examined = (unsigned long long*)((char*)workspace + 8);
    a.tile_status = (unsigned long long*)((char*)workspace + kTicketBytes);
    a.hooks = lookback_hooks();
    const size_t head = align_up(kTicketBytes + (size_t)a.n_tiles * sizeof(unsigned long long), 256);
    a.masks = (uint32_t*)((char*)workspace + head);

    cudaError_t e = cudaMemsetAsync(workspace, 0, kTicketBytes + (size_t)a.n_tiles * 8, st);
    if (e != cudaSuccess) return NACC_ERR_CUDA;
    const int need = (a.n_tiles + kThreads / 32 - 1) / (kThreads / 32);
    const bool il4 = tune_get(NACC_TUNE_PRUNE_INTERLEAVE) == 4;
    switch (tune_get(NACC_TUNE_PRUNE_OCCUPANCY)) {
        case 1: launch_variant<8>(il4, need, st, a); break;
        case 2: launch_variant<6>(il4, need, st, a); break;
        default: launch_variant<1>(il4, need, st, a); break;
    }
    return launch_status(cudaGetLastError());
}
