// render.cu -- differentiable volume rendering of packed samples (NerfAcc,
// arXiv 2210.04847, Sec. 2.2 and Eq. 1): per-sample weights, accumulation of
// sample attributes along rays, the fused forward pass and its hand-written
// backward pass.
//
// Every kernel gives one warp to one ray at a time and walks the ray's run of
// samples in chunks of 32 (parallel over samples inside the ray, Sec. 2.2),
// with coalesced loads. The exclusive optical depth O_i = sum_{j<i} tau_j is a
// warp shuffle scan plus a carry between chunks; the operations that form it
// are explicitly rounded, so the forward and backward kernels (and the saved
// optical-depth path) produce the same O_i bit for bit.
#include <math.h>
#include <string.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCarryCap = 128;  // chunk carries kept in shared memory per warp (4096 samples)

__device__ __forceinline__ bool load_run(const int32_t* packed_info, int r, int64_t n_samples,
                                         int32_t* d_status, int lane, int& off, int& cnt) {
    off = packed_info[2 * (size_t)r];
    cnt = packed_info[2 * (size_t)r + 1];
    if (off < 0 || cnt < 0 || (long long)off + cnt > n_samples) {
        if (lane == 0) raise_status(d_status, NACC_STATUS_BAD_PACKED);
        off = 0;
        cnt = 0;
        return false;
    }
    return true;
}

// tau = sigma * (t_end - t_start), one rounding each.
__device__ __forceinline__ float tau_of(float s0, float s1, float sg) {
    return __fmul_rn(sg, __fsub_rn(s1, s0));
}

// Exclusive optical depth of each lane's sample within the chunk, given the
// carry of earlier chunks; also returns the chunk total.
__device__ __forceinline__ float chunk_optical_depth(float tau, float carry, int lane, float& total,
                                                     float& incl_out) {
    const float incl = warp_incl_scan(tau, lane);
    float excl = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) excl = 0.0f;
    total = __shfl_sync(FULL, incl, 31);
    incl_out = incl;
    return __fadd_rn(carry, excl);
}

__device__ __forceinline__ int global_warp() { return (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int n_global_warps() { return (int)((gridDim.x * (size_t)blockDim.x) >> 5); }

// ---------------------------------------------------------------------------
// forward (fused weights + accumulation)
// ---------------------------------------------------------------------------

struct FwdArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* t_starts;
    const float* t_ends;
    const float* sigmas;
    const float* rgbs;
    int64_t n_samples;
    float* color;
    float* opacity;
    float* depth;
    float* optical_depth;
    int32_t* d_status;
};

__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const FwdArgs a) {
    const int lane = threadIdx.x & 31;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        float carry = 0.0f;
        float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, op = 0.0f, dp = 0.0f;
        for (int base = 0; base < cnt; base += 32) {
            const int j = base + lane;
            const bool valid = j < cnt;
            const size_t i = (size_t)off + j;
            float s0 = 0.0f, s1 = 0.0f, sg = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
            if (valid) {
                s0 = __ldg(a.t_starts + i);
                s1 = __ldg(a.t_ends + i);
                sg = __ldg(a.sigmas + i);
                cr = __ldg(a.rgbs + 3 * i);
                cg = __ldg(a.rgbs + 3 * i + 1);
                cb = __ldg(a.rgbs + 3 * i + 2);
            }
            const float tau = valid ? tau_of(s0, s1, sg) : 0.0f;
            float total, incl;
            const float O = chunk_optical_depth(tau, carry, lane, total, incl);
            carry = __fadd_rn(carry, total);
            if (valid) {
                const float T = expf(-O);
                const float alpha = -expm1f(-tau);
                const float w = T * alpha;
                const float tmid = (s0 + s1) * 0.5f;
                c0 += w * cr;
                c1 += w * cg;
                c2 += w * cb;
                op += w;
                dp += w * tmid;
                if (a.optical_depth) a.optical_depth[i] = O;
            }
        }
        c0 = warp_sum(c0);
        c1 = warp_sum(c1);
        c2 = warp_sum(c2);
        op = warp_sum(op);
        dp = warp_sum(dp);
        if (lane == 0) {
            if (a.color) {
                a.color[3 * (size_t)r] = c0;
                a.color[3 * (size_t)r + 1] = c1;
                a.color[3 * (size_t)r + 2] = c2;
            }
            if (a.opacity) a.opacity[r] = op;
            if (a.depth) a.depth[r] = dp;
        }
    }
}

// ---------------------------------------------------------------------------
// weights only (Eq. 1)
// ---------------------------------------------------------------------------

struct WeightsArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* t_starts;
    const float* t_ends;
    const float* sigmas;
    int64_t n_samples;
    float* weights;
    float* trans;
    int32_t* d_status;
};

__global__ void __launch_bounds__(kThreads) render_weights_kernel(const WeightsArgs a) {
    const int lane = threadIdx.x & 31;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        float carry = 0.0f;
        for (int base = 0; base < cnt; base += 32) {
            const int j = base + lane;
            const bool valid = j < cnt;
            const size_t i = (size_t)off + j;
            float tau = 0.0f;
            if (valid) tau = tau_of(__ldg(a.t_starts + i), __ldg(a.t_ends + i), __ldg(a.sigmas + i));
            float total, incl;
            const float O = chunk_optical_depth(tau, carry, lane, total, incl);
            carry = __fadd_rn(carry, total);
            if (valid) {
                const float T = expf(-O);
                if (a.weights) a.weights[i] = T * -expm1f(-tau);
                if (a.trans) a.trans[i] = T;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// accumulate any attribute: out[r, c] = sum_i w_i v_i[c]
// ---------------------------------------------------------------------------

struct AccArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* weights;
    const float* values;
    int32_t n_channels;
    int64_t n_samples;
    float* out;
    int32_t* d_status;
};

__global__ void __launch_bounds__(kThreads) accumulate_kernel(const AccArgs a) {
    const int lane = threadIdx.x & 31;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        for (int c = 0; c < a.n_channels; ++c) {
            float acc = 0.0f;
            for (int j = lane; j < cnt; j += 32) {
                const size_t i = (size_t)off + j;
                const float w = __ldg(a.weights + i);
                acc += a.values ? w * __ldg(a.values + i * a.n_channels + c) : w;
            }
            acc = warp_sum(acc);
            if (lane == 0) a.out[(size_t)r * a.n_channels + c] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// backward: reverse segmented scan
// ---------------------------------------------------------------------------

struct BwdArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* t_starts;
    const float* t_ends;
    const float* sigmas;
    const float* rgbs;
    const float* optical_depth;
    int64_t n_samples;
    const float* g_color;
    const float* g_opacity;
    const float* g_depth;
    float* d_sigmas;
    float* d_rgbs;
    int32_t* d_status;
};

__device__ __forceinline__ float chunk_tau(const BwdArgs& a, int off, int cnt, int c, int lane) {
    const int j = (c << 5) + lane;
    if (j >= cnt) return 0.0f;
    const size_t i = (size_t)off + j;
    return tau_of(__ldg(a.t_starts + i), __ldg(a.t_ends + i), __ldg(a.sigmas + i));
}

__global__ void __launch_bounds__(kThreads) render_bwd_kernel(const BwdArgs a) {
    __shared__ float s_carry[kWarps][kCarryCap];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* carries = s_carry[wib];
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        if (cnt == 0) continue;
        const int nch = (cnt + 31) >> 5;
        const float gc0 = a.g_color ? a.g_color[3 * (size_t)r] : 0.0f;
        const float gc1 = a.g_color ? a.g_color[3 * (size_t)r + 1] : 0.0f;
        const float gc2 = a.g_color ? a.g_color[3 * (size_t)r + 2] : 0.0f;
        const float ga = a.g_opacity ? a.g_opacity[r] : 0.0f;
        const float gd = a.g_depth ? a.g_depth[r] : 0.0f;
        const bool saved = a.optical_depth != nullptr;

        // pass A (recompute mode): carry of optical depth at the start of each chunk
        if (!saved) {
            float carry = 0.0f;
            const int keep = nch < kCarryCap ? nch : kCarryCap;
            for (int c = 0; c < keep; ++c) {
                if (lane == 0) carries[c] = carry;
                const float tau = chunk_tau(a, off, cnt, c, lane);
                float total, incl;
                chunk_optical_depth(tau, carry, lane, total, incl);
                carry = __fadd_rn(carry, total);
            }
            __syncwarp();
        }

        // Reference sample of the ray (its first): with b_i = a_i - a_ref and the
        // telescoping sum_{i>k} w_i = T_{k+1} - T_end, the gradient
        //   a_k T_{k+1} - sum_{i>k} a_i w_i = a_ref T_end + b_k T_{k+1} - sum_{i>k} b_i w_i
        // is the same quantity, but the large near-cancelling terms a_ref T_{k+1}
        // and a_ref sum w_i never appear: the float32 error scales with |b| (the
        // variation of a along the ray), not with |a|.
        const float r_ref = __ldg(a.rgbs + 3 * (size_t)off);
        const float g_ref = __ldg(a.rgbs + 3 * (size_t)off + 1);
        const float b_ref = __ldg(a.rgbs + 3 * (size_t)off + 2);
        const float tm_ref = (__ldg(a.t_starts + off) + __ldg(a.t_ends + off)) * 0.5f;
        const float a_ref = gc0 * r_ref + gc1 * g_ref + gc2 * b_ref + ga + gd * tm_ref;
        float t_end = 0.0f;

        // pass B: chunks in reverse order, suffix sums of b_i w_i carried backwards
        float carry_s = 0.0f;
        for (int c = nch - 1; c >= 0; --c) {
            float carry_o = 0.0f;
            if (!saved) {
                if (c < kCarryCap) {
                    carry_o = carries[c];
                } else {  // rays longer than the shared-memory record: rescan from the last record
                    carry_o = carries[kCarryCap - 1];
                    for (int q = kCarryCap - 1; q < c; ++q) {
                        float total, incl;
                        chunk_optical_depth(chunk_tau(a, off, cnt, q, lane), carry_o, lane, total, incl);
                        carry_o = __fadd_rn(carry_o, total);
                    }
                }
            }
            const int j = (c << 5) + lane;
            const bool valid = j < cnt;
            const size_t i = (size_t)off + j;
            float s0 = 0.0f, s1 = 0.0f, sg = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f, Os = 0.0f;
            if (valid) {
                s0 = __ldg(a.t_starts + i);
                s1 = __ldg(a.t_ends + i);
                sg = __ldg(a.sigmas + i);
                cr = __ldg(a.rgbs + 3 * i);
                cg = __ldg(a.rgbs + 3 * i + 1);
                cb = __ldg(a.rgbs + 3 * i + 2);
                if (saved) Os = __ldg(a.optical_depth + i);
            }
            const float tau = valid ? tau_of(s0, s1, sg) : 0.0f;
            float O;
            if (saved) {
                O = Os;
            } else {
                float total, incl;
                O = chunk_optical_depth(tau, carry_o, lane, total, incl);
            }
            const float T = expf(-O);
            const float T_next = expf(-__fadd_rn(O, tau));
            if (c == nch - 1) t_end = __shfl_sync(FULL, T_next, (cnt - 1) & 31);
            const float w = T * -expm1f(-tau);
            const float tmid = (s0 + s1) * 0.5f;
            const float bv = gc0 * (cr - r_ref) + gc1 * (cg - g_ref) + gc2 * (cb - b_ref) + gd * (tmid - tm_ref);
            const float bw = valid ? bv * w : 0.0f;
            const float suf = warp_incl_suffix(bw, lane);
            float suf_excl = __shfl_down_sync(FULL, suf, 1);
            if (lane == 31) suf_excl = 0.0f;
            const float S = carry_s + suf_excl;
            carry_s = carry_s + __shfl_sync(FULL, suf, 0);
            if (valid) {
                const float dtau = a_ref * t_end + (bv * T_next - S);
                a.d_sigmas[i] = (s1 - s0) * dtau;
                a.d_rgbs[3 * i] = w * gc0;
                a.d_rgbs[3 * i + 1] = w * gc1;
                a.d_rgbs[3 * i + 2] = w * gc2;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// ray index of every sample
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) unpack_kernel(const int32_t* packed_info, int32_t n_rays,
                                                         int64_t n_samples, int32_t* ray_indices,
                                                         int32_t* d_status) {
    const int lane = threadIdx.x & 31;
    for (int r = global_warp(); r < n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(packed_info, r, n_samples, d_status, lane, off, cnt);
        for (int j = lane; j < cnt; j += 32) ray_indices[(size_t)off + j] = r;
    }
}

template <typename K>
int grid_for(K kernel, int n_rays) {
    const DeviceInfo dev = current_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long need = ((long long)n_rays + kWarps - 1) / kWarps;
    const long long cap = (long long)dev.sm_count * per_sm;
    return (int)(need < cap ? need : cap);
}

bool sizes_ok(int32_t n_rays, int64_t n_samples) {
    return n_rays >= 0 && n_samples >= 0 && n_samples < (1LL << 31);
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_render_fwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                               const float* t_ends, const float* sigmas, const float* rgbs,
                               int64_t n_samples, float* color, float* opacity, float* depth,
                               float* optical_depth, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas || !rgbs)) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    FwdArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, rgbs, n_samples, color, opacity, depth, optical_depth, d_status};
    render_fwd_kernel<<<grid_for(render_fwd_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_render_weights(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                                   const float* t_ends, const float* sigmas, int64_t n_samples,
                                   float* weights, float* trans, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas)) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    WeightsArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, n_samples, weights, trans, d_status};
    render_weights_kernel<<<grid_for(render_weights_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_accumulate_along_rays(const int32_t* packed_info, int32_t n_rays, const float* weights,
                                          const float* values, int32_t n_channels, int64_t n_samples,
                                          float* out, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples) || n_channels < 1) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!packed_info || !out)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && !weights) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    AccArgs a{packed_info, n_rays, weights, values, n_channels, n_samples, out, d_status};
    accumulate_kernel<<<grid_for(accumulate_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_render_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                               const float* t_ends, const float* sigmas, const float* rgbs,
                               const float* optical_depth, int64_t n_samples, const float* g_color,
                               const float* g_opacity, const float* g_depth, float* d_sigmas,
                               float* d_rgbs, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas || !rgbs || !d_sigmas || !d_rgbs))
        return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    BwdArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, rgbs, optical_depth, n_samples,
              g_color, g_opacity, g_depth, d_sigmas, d_rgbs, d_status};
    render_bwd_kernel<<<grid_for(render_bwd_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_unpack_info(const int32_t* packed_info, int32_t n_rays, int64_t n_samples,
                                int32_t* ray_indices, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!packed_info || (n_samples > 0 && !ray_indices))) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    unpack_kernel<<<grid_for(unpack_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(
        packed_info, n_rays, n_samples, ray_indices, d_status);
    return launch_status(cudaGetLastError());
}
