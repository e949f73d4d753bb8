// prune.cu -- pruning of marched samples by transmittance (early stop) and
// opacity (alpha threshold), then re-packing (NerfAcc, arXiv 2210.04847,
// Sec. 2.1 "Pruning Empty and Occluded Regions"; early_stop_eps and
// alpha_thre of the Sec. 3 listing).
//
// Single pass over the input samples: per ray, a warp walks its samples in
// chunks of 32 with coalesced loads, forms tau = sigma*delta, the exclusive
// optical depth by a warp shuffle scan plus a running carry, and the keep
// decision; one __ballot_sync word per chunk goes to a workspace row of the
// ray. Once the optical depth passes -ln(eps) the rest of the ray is dropped
// without being read. A bounded decoupled look-back turns the tile's kept
// count into its output offset, and the warps re-expand the ballot words into
// compacted stores. Compiled with -fmad=false (tau and the scan are explicitly
// rounded float32 operations).
#include <math.h>
#include <string.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 32;
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
};

__global__ void __launch_bounds__(kThreads) prune_kernel(const PruneArgs a) {
    __shared__ int s_count[kTile];
    __shared__ int s_nch[kTile];
    __shared__ int s_off[kTile];
    __shared__ int s_cnt[kTile];
    __shared__ int s_excl[kTile];
    __shared__ int s_tile;
    __shared__ int s_next;
    __shared__ int s_examined;
    __shared__ long long s_tile_excl;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = (int)atomicAdd(a.ticket, 1u);
            s_next = 0;
            s_examined = 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= a.n_tiles) break;
        const int ray0 = tile * kTile;
        const int nr = min(kTile, a.n_rays - ray0);

        // phase 1: decisions, one ballot word per 32 samples
        for (;;) {
            int i = 0;
            if (lane == 0) i = atomicAdd(&s_next, 1);
            i = __shfl_sync(FULL, i, 0);
            if (i >= nr) break;
            const int r = ray0 + i;
            int off = a.packed_info[2 * (size_t)r];
            int cnt = a.packed_info[2 * (size_t)r + 1];
            // runs must be in bounds, ascending and disjoint in ray order (the
            // layout marching and pruning produce): the ballot rows of the rays
            // then never overlap
            bool bad = off < 0 || cnt < 0 || (long long)off + cnt > a.n_samples;
            if (r > 0) {
                const long long prev_end = (long long)a.packed_info[2 * (size_t)r - 2] + a.packed_info[2 * (size_t)r - 1];
                if ((long long)off < prev_end && cnt > 0) bad = true;
            }
            if (bad) {
                if (lane == 0) raise_status(a.d_status, NACC_STATUS_BAD_PACKED);
                off = 0;
                cnt = 0;
            }
            uint32_t* row = a.masks + (off >> 5) + r;
            const int nch = (cnt + 31) >> 5;
            float carry = 0.0f;
            int count = 0, c = 0;
            for (; c < nch; ++c) {
                const int j = (c << 5) + lane;
                const bool valid = j < cnt;
                float tau = 0.0f;
                if (valid) {
                    const size_t idx = (size_t)off + j;
                    const float s0 = __ldg(a.t_starts + idx);
                    const float s1 = __ldg(a.t_ends + idx);
                    const float sg = __ldg(a.sigmas + idx);
                    tau = __fmul_rn(sg, __fsub_rn(s1, s0));
                }
                const float incl = warp_incl_scan(tau, lane);
                float excl = __shfl_up_sync(FULL, incl, 1);
                if (lane == 0) excl = 0.0f;
                const float O = __fadd_rn(carry, excl);
                bool keep = valid;
                if (a.use_t && !(O <= a.thr_o)) keep = false;
                if (a.use_a && !(tau >= a.thr_tau)) keep = false;
                const unsigned m = __ballot_sync(FULL, keep);
                if (lane == 0) row[c] = m;
                count += __popc(m);
                carry = __fadd_rn(carry, __shfl_sync(FULL, incl, 31));
                if (a.use_t && !(carry <= a.thr_o)) {  // every later O_i >= carry: all dropped
                    ++c;
                    break;
                }
            }
            if (lane == 0) {
                s_count[i] = count;
                s_nch[i] = c;
                s_off[i] = off;
                s_cnt[i] = cnt;
                atomicAdd(&s_examined, min(cnt, c << 5));
            }
        }
        __syncthreads();

        if (warp == 0) {
            const int cnt = lane < nr ? s_count[lane] : 0;
            const int incl = warp_incl_scan_int(cnt, lane);
            s_excl[lane] = incl - cnt;
            const int agg = __shfl_sync(FULL, incl, 31);
            const unsigned long long excl =
                lookback(a.tile_status, tile, (unsigned long long)agg, lane, a.d_status);
            if (lane == 0) {
                s_tile_excl = (long long)excl;
                atomicAdd(a.examined, (unsigned long long)s_examined);
                if (tile == a.n_tiles - 1) {
                    const long long total = (long long)excl + agg;
                    *a.n_kept = total;
                    if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
                    if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
                }
            }
        }
        __syncthreads();

        // phase 3: compacted stores of the kept samples
        const long long tile_excl = s_tile_excl;
        for (int i = warp; i < nr; i += kWarps) {
            const int r = ray0 + i;
            const int count = s_count[i];
            const long long out = tile_excl + s_excl[i];
            if (lane == 0) {
                a.packed_info_out[2 * (size_t)r] = (int32_t)out;
                a.packed_info_out[2 * (size_t)r + 1] = count;
            }
            const int off = s_off[i];
            const int cnt = s_cnt[i];
            const int nch = s_nch[i];
            const uint32_t* row = a.masks + (off >> 5) + r;
            long long base = out;
            for (int c = 0; c < nch; ++c) {
                const unsigned m = row[c];
                const int j = (c << 5) + lane;
                if (a.keep_mask && j < cnt) a.keep_mask[(size_t)off + j] = (uint8_t)((m >> lane) & 1u);
                if (m == 0u) continue;
                if ((m >> lane) & 1u) {
                    const long long pos = base + __popc(m & lanemask_lt());
                    if (pos < a.capacity) {
                        const size_t idx = (size_t)off + j;
                        a.t_starts_out[pos] = a.t_starts[idx];
                        a.t_ends_out[pos] = a.t_ends[idx];
                        a.ray_indices_out[pos] = r;
                    }
                }
                base += __popc(m);
            }
            if (a.keep_mask)
                for (int j = (nch << 5) + lane; j < cnt; j += 32) a.keep_mask[(size_t)off + j] = 0;
        }
        __syncthreads();
    }
}

size_t workspace_bytes_for(int32_t n_rays, int64_t n_samples) {
    const size_t tiles = (size_t)(n_rays + kTile - 1) / kTile;
    const size_t head = align_up(kTicketBytes + tiles * sizeof(unsigned long long), 256);
    const size_t words = (size_t)(n_samples >> 5) + (size_t)n_rays + 2;
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
    a.n_tiles = (n_rays + kTile - 1) / kTile;
    a.ticket = (unsigned int*)workspace;
    a.examined = (unsigned long long*)((char*)workspace + 8);
    a.tile_status = (unsigned long long*)((char*)workspace + kTicketBytes);
    const size_t head = align_up(kTicketBytes + (size_t)a.n_tiles * sizeof(unsigned long long), 256);
    a.masks = (uint32_t*)((char*)workspace + head);

    cudaError_t e = cudaMemsetAsync(workspace, 0, kTicketBytes + (size_t)a.n_tiles * 8, st);
    if (e != cudaSuccess) return NACC_ERR_CUDA;
    const DeviceInfo dev = current_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prune_kernel, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int blocks = dev.sm_count * per_sm;
    if (blocks > a.n_tiles) blocks = a.n_tiles;
    prune_kernel<<<blocks, kThreads, 0, st>>>(a);
    return launch_status(cudaGetLastError());
}
