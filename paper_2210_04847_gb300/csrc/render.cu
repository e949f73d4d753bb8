// render.cu -- differentiable volume rendering of packed samples (NerfAcc,
// arXiv 2210.04847, Sec. 2.2 and Eq. 1): per-sample weights, accumulation of
// sample attributes along rays, the fused forward pass and its hand-written
// backward pass.
//
// Every kernel gives one warp to one ray at a time and walks the ray's run of
// samples in chunks (parallel over samples inside the ray, Sec. 2.2), with
// coalesced loads: the fused forward and backward take 64 samples per chunk, two
// consecutive samples per lane as 8-byte loads; the weights and accumulation
// kernels take 32. The exclusive optical depth O_i = sum_{j<i} tau_j is a
// warp shuffle scan plus a carry between chunks; the operations that form it
// are explicitly rounded, so the forward and backward kernels (and the saved
// optical-depth path) produce the same O_i bit for bit.
#include <math.h>
#include <string.h>

#include "bulk_copy.cuh"
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCarryCap = 128;  // chunk carries kept in shared memory per warp (8192 samples)

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
    int stage_polls;       // staged kernel: polls of a stage's barrier before the walk gives up
    unsigned stage_extra;  // staged kernel, test hook: bytes announced beyond the first chunk's copies
};

constexpr int kRenderThreads = 128;
constexpr int kRayVals = 9;  // backward: per-ray values staged in shared memory
constexpr int kGroup = 4;  // consecutive rays per warp (lane i holds ray i's run)

// Runs of the warp's group of rays; lanes >= nr and invalid runs hold (0, 0).
__device__ __forceinline__ void load_group(const int32_t* packed_info, int ray0, int nr, int64_t n_samples,
                                           int32_t* d_status, int lane, int& off, int& cnt) {
    off = 0;
    cnt = 0;
    if (lane < nr) {
        const int2 v = reinterpret_cast<const int2*>(packed_info)[ray0 + lane];
        off = v.x;
        cnt = v.y;
        if (off < 0 || cnt < 0 || (long long)off + cnt > n_samples) {
            raise_status(d_status, NACC_STATUS_BAD_PACKED);
            off = 0;
            cnt = 0;
        }
    }
}

// alpha = 1 - exp(-tau) for tau >= 0. Below 1/16 the Taylor series
// t (1 - t/2 (1 - t/3 (1 - t/4 (1 - t/5)))) (truncation below t^5/6! < 2e-8
// relative); from 1/16 on 1 - exp(-tau) with the fast exponential (absolute
// error below 2.5e-7, relative below 4e-6 since alpha > 0.06 there).
__device__ __forceinline__ float alpha_of(float t) {
    float p = 1.0f - t * (1.0f / 5.0f);
    p = 1.0f - t * (1.0f / 4.0f) * p;
    p = 1.0f - t * (1.0f / 3.0f) * p;
    p = 1.0f - t * 0.5f * p;
    p = t * p;
    const float q = 1.0f - __expf(-t);
    return t < 0.0625f ? p : q;
}

// Sum of 5 values over the warp with a butterfly that halves the number of
// values a lane carries at each of the first steps (9 shuffles instead of 25).
// Returns in lane 0 the total of v[0] and in lanes 4, 8, 12, 16 those of v[1..4].
__device__ __forceinline__ float warp_sum5(float v0, float v1, float v2, float v3, float v4, int lane) {
    float v[8] = {v0, v1, v2, v3, v4, 0.0f, 0.0f, 0.0f};
    // step 16: keep half k in {4b..4b+3}, b = bit 4 of lane
    const bool h16 = (lane & 16) != 0;
    float u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = h16 ? v[k] : v[4 + k];
        const float keep = h16 ? v[4 + k] : v[k];
        u[k] = keep + __shfl_xor_sync(FULL, send, 16);
    }
    const bool h8 = (lane & 8) != 0;
    float w2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = h8 ? u[k] : u[2 + k];
        const float keep = h8 ? u[2 + k] : u[k];
        w2[k] = keep + __shfl_xor_sync(FULL, send, 8);
    }
    const bool h4 = (lane & 4) != 0;
    float x = (h4 ? w2[1] : w2[0]) + __shfl_xor_sync(FULL, h4 ? w2[0] : w2[1], 4);
    x += __shfl_xor_sync(FULL, x, 2);
    x += __shfl_xor_sync(FULL, x, 1);
    // lane bits (4,3,2) select the value index 4*b4 + 2*b3 + b2
    return x;
}

// Two consecutive samples j0, j0 + 1 (j0 even) of a ray with run [lo, hi).
// Sample indices are below 2^31 (checked on the host), so 32-bit unsigned
// arithmetic cannot wrap even 64 samples past the end.
struct Pair {
    float s0[2], s1[2], sg[2], rgb[6];
    bool v0, v1;
};

__device__ __forceinline__ void load_pair(const float* __restrict__ ts, const float* __restrict__ te,
                                          const float* __restrict__ sig, const float* __restrict__ rgbs,
                                          unsigned j0, unsigned lo, unsigned hi, Pair& q) {
    q.v0 = j0 >= lo && j0 < hi;
    q.v1 = j0 + 1 >= lo && j0 + 1 < hi;
#pragma unroll
    for (int k = 0; k < 2; ++k) q.s0[k] = q.s1[k] = q.sg[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) q.rgb[k] = 0.0f;
    if (q.v0 && q.v1) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(ts + j0));
        const float2 b = __ldg(reinterpret_cast<const float2*>(te + j0));
        const float2 g = __ldg(reinterpret_cast<const float2*>(sig + j0));
        const float2 c0 = __ldg(reinterpret_cast<const float2*>(rgbs + 3 * j0));
        const float2 c1 = __ldg(reinterpret_cast<const float2*>(rgbs + 3 * j0 + 2));
        const float2 c2 = __ldg(reinterpret_cast<const float2*>(rgbs + 3 * j0 + 4));
        q.s0[0] = a.x; q.s0[1] = a.y;
        q.s1[0] = b.x; q.s1[1] = b.y;
        q.sg[0] = g.x; q.sg[1] = g.y;
        q.rgb[0] = c0.x; q.rgb[1] = c0.y; q.rgb[2] = c1.x;
        q.rgb[3] = c1.y; q.rgb[4] = c2.x; q.rgb[5] = c2.y;
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 0 ? q.v0 : q.v1) {
                const unsigned j = j0 + k;
                q.s0[k] = __ldg(ts + j);
                q.s1[k] = __ldg(te + j);
                q.sg[k] = __ldg(sig + j);
                q.rgb[3 * k] = __ldg(rgbs + 3 * j);
                q.rgb[3 * k + 1] = __ldg(rgbs + 3 * j + 1);
                q.rgb[3 * k + 2] = __ldg(rgbs + 3 * j + 2);
            }
        }
    }
}

// As load_pair, with the upstream weight gradients of the two samples in
// rgb[0] and rgb[3] (weights mode of the backward).
__device__ __forceinline__ void load_pair_w(const float* __restrict__ ts, const float* __restrict__ te,
                                            const float* __restrict__ sig, const float* __restrict__ gw,
                                            unsigned j0, unsigned lo, unsigned hi, Pair& q) {
    q.v0 = j0 >= lo && j0 < hi;
    q.v1 = j0 + 1 >= lo && j0 + 1 < hi;
#pragma unroll
    for (int k = 0; k < 2; ++k) q.s0[k] = q.s1[k] = q.sg[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) q.rgb[k] = 0.0f;
    if (q.v0 && q.v1) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(ts + j0));
        const float2 b = __ldg(reinterpret_cast<const float2*>(te + j0));
        const float2 g = __ldg(reinterpret_cast<const float2*>(sig + j0));
        const float2 w = __ldg(reinterpret_cast<const float2*>(gw + j0));
        q.s0[0] = a.x; q.s0[1] = a.y;
        q.s1[0] = b.x; q.s1[1] = b.y;
        q.sg[0] = g.x; q.sg[1] = g.y;
        q.rgb[0] = w.x; q.rgb[3] = w.y;
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 0 ? q.v0 : q.v1) {
                const unsigned j = j0 + k;
                q.s0[k] = __ldg(ts + j);
                q.s1[k] = __ldg(te + j);
                q.sg[k] = __ldg(sig + j);
                q.rgb[3 * k] = __ldg(gw + j);
            }
        }
    }
}

// Exclusive optical depth of both samples of each lane's pair, given the carry of
// earlier chunks; updates the carry. The same explicitly rounded operations in
// every kernel, so forward, backward and saved values agree bit for bit.
__device__ __forceinline__ void pair_optical_depth(float tau0, float tau1, float& carry, int lane, float& O0,
                                                   float& O1) {
    const float incl = warp_incl_scan(__fadd_rn(tau0, tau1), lane);
    float excl = __shfl_up_sync(FULL, incl, 1);
    if (lane == 0) excl = 0.0f;
    O0 = __fadd_rn(carry, excl);
    O1 = __fadd_rn(O0, tau0);
    carry = __fadd_rn(carry, __shfl_sync(FULL, incl, 31));
}

// The warp walks the 64-sample chunks of its rays as one stream (lane j holds
// samples 2j, 2j + 1 of a chunk, chunks start at an even index); the loads of
// the next chunk (of the same ray or of the next one) are issued before the
// current chunk is computed.
template <bool PREFETCH, int MINB>
__global__ void __launch_bounds__(kRenderThreads, MINB) render_fwd_kernel(const FwdArgs a) {
    const int lane = threadIdx.x & 31;
    const int ray0 = global_warp() * kGroup;
    if (ray0 >= a.n_rays) return;
    const int nr = min(kGroup, a.n_rays - ray0);
    int my_off, my_cnt;
    load_group(a.packed_info, ray0, nr, a.n_samples, a.d_status, lane, my_off, my_cnt);
    if (lane < nr && my_cnt == 0) {
        const int r = ray0 + lane;
        if (a.color) {
            a.color[3 * (size_t)r] = 0.0f;
            a.color[3 * (size_t)r + 1] = 0.0f;
            a.color[3 * (size_t)r + 2] = 0.0f;
        }
        if (a.opacity) a.opacity[r] = 0.0f;
        if (a.depth) a.depth[r] = 0.0f;
    }
    unsigned todo = __ballot_sync(FULL, my_cnt > 0);
    if (todo == 0u) return;
    int i = __ffs(todo) - 1;
    todo &= todo - 1;
    unsigned lo = __shfl_sync(FULL, my_off, i);
    unsigned hi = lo + __shfl_sync(FULL, my_cnt, i);
    unsigned j0 = (lo & ~1u) + 2 * lane;
    Pair nx;
    if (PREFETCH) load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, lo, hi, nx);
    float carry = 0.0f;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, op = 0.0f, dp = 0.0f;
    for (;;) {
        Pair q;
        if (PREFETCH) {
            q = nx;
        } else {
            load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, lo, hi, q);
        }
        const int qi = i;
        const unsigned qj0 = j0;
        j0 += 64;
        const bool ray_done = (j0 - 2 * lane) >= hi;
        bool more = true;
        if (ray_done) {
            if (todo) {
                i = __ffs(todo) - 1;
                todo &= todo - 1;
                lo = __shfl_sync(FULL, my_off, i);
                hi = lo + __shfl_sync(FULL, my_cnt, i);
                j0 = (lo & ~1u) + 2 * lane;
            } else {
                more = false;
            }
        }
        if (PREFETCH && more) load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, lo, hi, nx);

        const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
        const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
        float O0, O1;
        pair_optical_depth(tau0, tau1, carry, lane, O0, O1);
        const float w0 = q.v0 ? __expf(-O0) * alpha_of(tau0) : 0.0f;
        const float w1 = q.v1 ? __expf(-O1) * alpha_of(tau1) : 0.0f;
        c0 += w0 * q.rgb[0] + w1 * q.rgb[3];
        c1 += w0 * q.rgb[1] + w1 * q.rgb[4];
        c2 += w0 * q.rgb[2] + w1 * q.rgb[5];
        op += w0 + w1;
        dp += w0 * ((q.s0[0] + q.s1[0]) * 0.5f) + w1 * ((q.s0[1] + q.s1[1]) * 0.5f);
        if (a.optical_depth) {
            if (q.v0) a.optical_depth[qj0] = O0;
            if (q.v1) a.optical_depth[qj0 + 1] = O1;
        }
        if (ray_done) {
            const float sum = warp_sum5(c0, c1, c2, op, dp, lane);
            const size_t r = (size_t)ray0 + qi;
            if (lane == 0 && a.color) a.color[3 * r] = sum;
            if (lane == 4 && a.color) a.color[3 * r + 1] = sum;
            if (lane == 8 && a.color) a.color[3 * r + 2] = sum;
            if (lane == 12 && a.opacity) a.opacity[r] = sum;
            if (lane == 16 && a.depth) a.depth[r] = sum;
            carry = 0.0f;
            c0 = c1 = c2 = op = dp = 0.0f;
        }
        if (!more) break;
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
                const float T = __expf(-O);
                if (a.weights) a.weights[i] = T * alpha_of(tau);
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

// Warp per ray; each lane keeps one channel. For C <= 32 a step covers P = 32 / C
// consecutive samples (lane l: channel l % C of sample l / C), so the warp reads one
// contiguous run of P*C values; the P partial sums of a channel are then added
// over lanes C apart. For C > 32 a step is one sample, 32 channels at a time.
__global__ void __launch_bounds__(kThreads) accumulate_kernel(const AccArgs a) {
    const int lane = threadIdx.x & 31;
    const int C = a.n_channels;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        if (C <= 32) {
            const int P = 32 / C, L = P * C;
            const int ch = lane % C;
            float acc = 0.0f;
            if (lane < L) {
#pragma unroll 4
                for (int s = lane / C; s < cnt; s += P) {
                    const size_t i = (size_t)off + s;
                    const float w = __ldg(a.weights + i);
                    acc += a.values ? w * __ldg(a.values + i * C + ch) : w;
                }
            }
            for (int o = C; o < L; o <<= 1) {
                const float y = __shfl_down_sync(FULL, acc, o);
                if (lane + o < L) acc += y;
            }
            if (lane < C) a.out[(size_t)r * C + lane] = acc;
        } else {
            for (int cg = 0; cg < C; cg += 32) {
                const int c = cg + lane;
                if (c >= C) continue;
                float acc = 0.0f;
#pragma unroll 4
                for (int s = 0; s < cnt; ++s) {
                    const size_t i = (size_t)off + s;
                    const float w = __ldg(a.weights + i);
                    acc += a.values ? w * __ldg(a.values + i * C + c) : w;
                }
                a.out[(size_t)r * C + c] = acc;
            }
        }
    }
}

struct AccBwdArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* weights;
    const float* values;
    int32_t n_channels;
    int64_t n_samples;
    const float* g_out;
    float* d_weights;
    float* d_values;
    float* g_ref;  // centred mode: per-ray dL/dw of the first sample, added in
    int32_t* d_status;
};

// Centred mode (g_ref given): dL/dw_i is written as sum_c g[r,c] (v_i[c] - v_1[c]),
// v_1 the values of the ray's first sample, and sum_c g[r,c] v_1[c] is added to
// g_ref[r]. The two parts add up to dL/dw_i, but the per-sample part is formed
// from value differences before any rounding, so its float32 error scales with
// how much the values vary along the ray rather than with their size. The
// weights backward takes g_ref as the reference of its centred scan.
__device__ __forceinline__ void add_g_ref(const AccBwdArgs& a, int r, int off, int cnt, int lane) {
    if (!a.g_ref || cnt == 0) return;
    const int C = a.n_channels;
    const float* g = a.g_out + (size_t)r * C;
    float ref = 0.0f;
    for (int c = lane; c < C; c += 32) ref += __ldg(g + c) * (a.values ? __ldg(a.values + (size_t)off * C + c) : 1.0f);
    ref = warp_sum(ref);
    if (lane == 0) a.g_ref[r] += ref;
}

// The same gradient for C <= 4 channels: a lane per sample, its values one short
// run (no shared memory, so more warps per SM than the tiled kernel).
__global__ void __launch_bounds__(kThreads) accumulate_bwd_narrow_kernel(const AccBwdArgs a) {
    const int lane = threadIdx.x & 31;
    const int C = a.n_channels;
    const bool centre = a.g_ref != nullptr;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        add_g_ref(a, r, off, cnt, lane);
        const float* g = a.g_out + (size_t)r * C;
        const float* v1 = a.values ? a.values + (size_t)off * C : nullptr;  // the ray's first sample
        for (int j = lane; j < cnt; j += 32) {
            const size_t i = (size_t)off + j;
            const float w = __ldg(a.weights + i);
            float dw = 0.0f;
            for (int c = 0; c < C; ++c) {
                const float gc = __ldg(g + c);
                if (centre) {
                    if (a.values) dw += gc * (__ldg(a.values + i * C + c) - __ldg(v1 + c));
                } else {
                    dw += a.values ? gc * __ldg(a.values + i * C + c) : gc;
                }
                if (a.d_values) a.d_values[i * C + c] = w * gc;
            }
            if (a.d_weights) a.d_weights[i] = dw;
        }
    }
}

// Gradient of accumulate_along_rays, warp per ray: dL/dw_i = sum_c g[r,c] v_i[c]
// and dL/dv_i[c] = w_i g[r,c]. For 4 < C <= 32 the ray goes in tiles of 32 samples:
// the warp reads the tile's values as one contiguous run (four loads in flight
// per lane), writes dL/dv in the same order, and stages the values in shared
// memory with an odd row stride. Lane j then sums sample j's C products from
// there, with no bank conflicts. For C > 32 a step is one sample, 32 channels at
// a time.
__global__ void __launch_bounds__(kThreads) accumulate_bwd_kernel(const AccBwdArgs a) {
    __shared__ float s_v[kWarps][32 * 33];
    __shared__ float s_g[kWarps][32];
    __shared__ float s_w[kWarps][32];
    __shared__ float s_v1[kWarps][32];  // centred mode: the ray's first sample's values
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int C = a.n_channels;
    const bool centre = a.g_ref != nullptr;
    float* sv = s_v[warp];
    float* sg = s_g[warp];
    float* sw = s_w[warp];
    float* sv1 = s_v1[warp];
    const int stride = C | 1;
    const int q = C <= 32 ? 32 / C : 0, rem = C <= 32 ? 32 - q * C : 0;  // +32 elements: +q samples, +rem channels
    const int s_first = C <= 32 ? lane / C : 0, c_first = C <= 32 ? lane - s_first * C : 0;
    for (int r = global_warp(); r < a.n_rays; r += n_global_warps()) {
        int off, cnt;
        load_run(a.packed_info, r, a.n_samples, a.d_status, lane, off, cnt);
        const float* g = a.g_out + (size_t)r * C;
        add_g_ref(a, r, off, cnt, lane);
        if (C <= 32) {
            if (lane < C) sg[lane] = __ldg(g + lane);
            if (centre && lane < C) sv1[lane] = cnt > 0 && a.values ? __ldg(a.values + (size_t)off * C + lane) : 1.0f;
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const int n = min(32, cnt - j0);
                const size_t sbase = (size_t)off + j0;
                const size_t ebase = sbase * C;
                const int E = n * C;
                if (lane < n) sw[lane] = __ldg(a.weights + sbase + lane);
                __syncwarp();
                int s = s_first, c = c_first;
                for (int e0 = 0; e0 < E; e0 += 128) {
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + 32 * u + lane;
                        v[u] = e < E ? (a.values ? __ldg(a.values + ebase + e) : 1.0f) : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + 32 * u + lane;
                        if (e < E) {
                            sv[s * stride + c] = v[u];
                            if (a.d_values) a.d_values[ebase + e] = sw[s] * sg[c];
                        }
                        s += q;
                        c += rem;
                        if (c >= C) {
                            c -= C;
                            ++s;
                        }
                    }
                }
                __syncwarp();
                if (a.d_weights && lane < n) {
                    float dw = 0.0f;
                    if (centre) {
                        for (int k = 0; k < C; ++k) dw += sg[k] * (sv[lane * stride + k] - sv1[k]);
                    } else {
                        for (int k = 0; k < C; ++k) dw += sg[k] * sv[lane * stride + k];
                    }
                    a.d_weights[sbase + lane] = dw;
                }
                __syncwarp();
            }
        } else {
            for (int s = 0; s < cnt; ++s) {
                const size_t i = (size_t)off + s;
                const float w = __ldg(a.weights + i);
                float dw = 0.0f;
                for (int cg = 0; cg < C; cg += 32) {
                    const int c = cg + lane;
                    if (c < C) {
                        const float gc = __ldg(g + c);
                        if (centre) {
                            if (a.values) dw += gc * (__ldg(a.values + i * C + c) - __ldg(a.values + (size_t)off * C + c));
                        } else {
                            dw += a.values ? gc * __ldg(a.values + i * C + c) : gc;
                        }
                        if (a.d_values) a.d_values[i * C + c] = w * gc;
                    }
                }
                if (a.d_weights) {
                    dw = warp_sum(dw);
                    if (lane == 0) a.d_weights[i] = dw;
                }
            }
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
    const float* g_weights;  // weights mode: dL/dw_i (no rgb, g_color, d_rgbs)
    const float* g_ref;      // weights mode, centred input: dL/dw_i = g_ref[r] + g_weights[i]
    int stage_polls;         // as FwdArgs
    unsigned stage_extra;
};

// tau of both samples of the lane's pair in chunk c of a ray (pass A of the backward).
__device__ __forceinline__ void pair_tau(const BwdArgs& a, unsigned abase, unsigned lo, unsigned hi, int c, int lane,
                                         float& tau0, float& tau1) {
    const unsigned j0 = abase + ((unsigned)c << 6) + 2 * lane;
    const bool v0 = j0 >= lo && j0 < hi, v1 = j0 + 1 >= lo && j0 + 1 < hi;
    tau0 = tau1 = 0.0f;
    if (v0 && v1) {
        const float2 u = __ldg(reinterpret_cast<const float2*>(a.t_starts + j0));
        const float2 v = __ldg(reinterpret_cast<const float2*>(a.t_ends + j0));
        const float2 g = __ldg(reinterpret_cast<const float2*>(a.sigmas + j0));
        tau0 = tau_of(u.x, v.x, g.x);
        tau1 = tau_of(u.y, v.y, g.y);
    } else if (v0) {
        tau0 = tau_of(__ldg(a.t_starts + j0), __ldg(a.t_ends + j0), __ldg(a.sigmas + j0));
    } else if (v1) {
        tau1 = tau_of(__ldg(a.t_starts + j0 + 1), __ldg(a.t_ends + j0 + 1), __ldg(a.sigmas + j0 + 1));
    }
}

// WEIGHTS: the gradient of nacc_render_weights (a_i = dL/dw_i read from
// g_weights; only d_sigmas is written).
template <int MINB, bool PREFETCH, bool WEIGHTS = false>
__global__ void __launch_bounds__(kRenderThreads, MINB) render_bwd_kernel(const BwdArgs a) {
    __shared__ float s_carry[kRenderThreads / 32][kCarryCap];
    // per ray of the group: its upstream gradients and first sample, loaded by
    // lane i for ray i before any ray is processed (one round trip for the group)
    __shared__ float s_ray[kRenderThreads / 32][kGroup][kRayVals];
    const int lane = threadIdx.x & 31;
    float* carries = s_carry[threadIdx.x >> 5];
    float(*ray_vals)[kRayVals] = s_ray[threadIdx.x >> 5];
    const int ray0 = global_warp() * kGroup;
    if (ray0 >= a.n_rays) return;
    const int nr = min(kGroup, a.n_rays - ray0);
    int my_off, my_cnt;
    load_group(a.packed_info, ray0, nr, a.n_samples, a.d_status, lane, my_off, my_cnt);
    const bool saved = a.optical_depth != nullptr;
    if (lane < nr && my_cnt > 0) {
        const size_t r = (size_t)ray0 + lane;
        float* v = ray_vals[lane];
        if constexpr (WEIGHTS) {
            v[0] = a.g_ref ? __ldg(a.g_ref + r) : __ldg(a.g_weights + my_off);
        } else {
            v[0] = a.g_color ? a.g_color[3 * r] : 0.0f;
            v[1] = a.g_color ? a.g_color[3 * r + 1] : 0.0f;
            v[2] = a.g_color ? a.g_color[3 * r + 2] : 0.0f;
            v[3] = a.g_opacity ? a.g_opacity[r] : 0.0f;
            v[4] = a.g_depth ? a.g_depth[r] : 0.0f;
            v[5] = __ldg(a.rgbs + 3 * (size_t)my_off);
            v[6] = __ldg(a.rgbs + 3 * (size_t)my_off + 1);
            v[7] = __ldg(a.rgbs + 3 * (size_t)my_off + 2);
            v[8] = (__ldg(a.t_starts + my_off) + __ldg(a.t_ends + my_off)) * 0.5f;
        }
    }
    __syncwarp();
    for (int ri = 0; ri < nr; ++ri) {
        const unsigned lo = __shfl_sync(FULL, my_off, ri);
        const int cnt = __shfl_sync(FULL, my_cnt, ri);
        if (cnt == 0) continue;
        const unsigned hi = lo + cnt;
        const unsigned abase = lo & ~1u;
        const int nch = (int)((hi - abase + 63) >> 6);
        const float* rv = ray_vals[ri];
        const float gc0 = WEIGHTS ? 0.0f : rv[0];
        const float gc1 = WEIGHTS ? 0.0f : rv[1];
        const float gc2 = WEIGHTS ? 0.0f : rv[2];
        const float ga = WEIGHTS ? 0.0f : rv[3];
        const float gd = WEIGHTS ? 0.0f : rv[4];

        // pass A (recompute mode): optical-depth carry at the start of each chunk,
        // the next chunk's loads in flight while the current one is scanned
        if (!saved) {
            float carry = 0.0f;
            const int keep = nch < kCarryCap ? nch : kCarryCap;
            float n0, n1;
            pair_tau(a, abase, lo, hi, 0, lane, n0, n1);
            for (int c = 0; c < keep; ++c) {
                const float t0 = n0, t1 = n1;
                if (c + 1 < keep) pair_tau(a, abase, lo, hi, c + 1, lane, n0, n1);
                if (lane == 0) carries[c] = carry;
                float O0, O1;
                pair_optical_depth(t0, t1, carry, lane, O0, O1);
            }
            __syncwarp();
        }

        // Reference sample of the ray (its first): with b_i = a_i - a_ref and the
        // telescoping sum_{i>k} w_i = T_{k+1} - T_end, the gradient
        //   a_k T_{k+1} - sum_{i>k} a_i w_i = a_ref T_end + b_k T_{k+1} - sum_{i>k} b_i w_i
        // is the same quantity, but the large near-cancelling terms a_ref T_{k+1}
        // and a_ref sum w_i never appear: the float32 error scales with |b| (the
        // variation of a along the ray), not with |a|.
        // with PREFETCH the last chunk's loads (pass B starts there) go out
        // together with the reference sample's, so their latencies overlap
        Pair nx;
        if (PREFETCH && !WEIGHTS)
            load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, abase + ((unsigned)(nch - 1) << 6) + 2 * lane, lo, hi,
                      nx);
        // weights mode: a_i = g_weights[i] with a_ref = a_1 (b_i = a_i - a_1), or,
        // with g_ref, a_i = g_ref[r] + g_weights[i], the reference given and b_i the
        // centred input itself
        float r_ref = 0.0f, g_ref = 0.0f, b_ref = 0.0f, tm_ref = 0.0f, a_ref, a_sub = 0.0f;
        if constexpr (WEIGHTS) {
            a_ref = rv[0];
            if (!a.g_ref) a_sub = a_ref;
        } else {
            r_ref = rv[5];
            g_ref = rv[6];
            b_ref = rv[7];
            tm_ref = rv[8];
            a_ref = gc0 * r_ref + gc1 * g_ref + gc2 * b_ref + ga + gd * tm_ref;
        }
        const unsigned last = hi - 1 - abase;  // position of the ray's last sample in its chunks
        const int last_lane = (int)((last >> 1) & 31);
        const bool last_odd = (last & 1) != 0;
        float t_end = 0.0f;

        // pass B: chunks in reverse order, suffix sums of b_i w_i carried backwards;
        // with PREFETCH the next (earlier) chunk's loads are issued before this one
        // is computed
        float carry_s = 0.0f;
        for (int c = nch - 1; c >= 0; --c) {
            float carry_o = 0.0f;
            if (!saved) {
                if (c < kCarryCap) {
                    carry_o = carries[c];
                } else {  // rays longer than the shared-memory record: rescan from the last record
                    carry_o = carries[kCarryCap - 1];
                    for (int p = kCarryCap - 1; p < c; ++p) {
                        float t0, t1, O0, O1;
                        pair_tau(a, abase, lo, hi, p, lane, t0, t1);
                        pair_optical_depth(t0, t1, carry_o, lane, O0, O1);
                    }
                }
            }
            const unsigned j0 = abase + ((unsigned)c << 6) + 2 * lane;
            Pair q;
            if constexpr (WEIGHTS) {
                load_pair_w(a.t_starts, a.t_ends, a.sigmas, a.g_weights, j0, lo, hi, q);
            } else if (PREFETCH) {
                q = nx;
                if (c > 0) load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0 - 64, lo, hi, nx);
            } else {
                load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, lo, hi, q);
            }
            const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
            const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
            float O0, O1;
            if (saved) {
                O0 = q.v0 ? __ldg(a.optical_depth + j0) : 0.0f;
                O1 = q.v1 ? __ldg(a.optical_depth + j0 + 1) : 0.0f;
                if (!q.v0) O1 = q.v1 ? O1 : 0.0f;
            } else {
                pair_optical_depth(tau0, tau1, carry_o, lane, O0, O1);
            }
            // T of each sample and of the sample after it: T_{k+1} of the even
            // sample is T of the odd one (O1 = O0 + tau0 by construction)
            const float T0 = __expf(-O0);
            const float T1 = __expf(-O1);
            const float T2 = __expf(-__fadd_rn(O1, tau1));
            const float Tn0 = q.v1 ? T1 : __expf(-__fadd_rn(O0, tau0));
            if (c == nch - 1) t_end = __shfl_sync(FULL, last_odd ? T2 : Tn0, last_lane);
            const float w0 = q.v0 ? T0 * alpha_of(tau0) : 0.0f;
            const float w1 = q.v1 ? T1 * alpha_of(tau1) : 0.0f;
            const float tm0 = (q.s0[0] + q.s1[0]) * 0.5f, tm1 = (q.s0[1] + q.s1[1]) * 0.5f;
            float b0, b1;
            if constexpr (WEIGHTS) {
                b0 = q.rgb[0] - a_sub;
                b1 = q.rgb[3] - a_sub;
            } else {
                b0 = gc0 * (q.rgb[0] - r_ref) + gc1 * (q.rgb[1] - g_ref) + gc2 * (q.rgb[2] - b_ref) +
                     gd * (tm0 - tm_ref);
                b1 = gc0 * (q.rgb[3] - r_ref) + gc1 * (q.rgb[4] - g_ref) + gc2 * (q.rgb[5] - b_ref) +
                     gd * (tm1 - tm_ref);
            }
            const float bw0 = q.v0 ? b0 * w0 : 0.0f;
            const float bw1 = q.v1 ? b1 * w1 : 0.0f;
            const float suf = warp_incl_suffix(bw0 + bw1, lane);
            float later = __shfl_down_sync(FULL, suf, 1);  // pairs of lanes > this one
            if (lane == 31) later = 0.0f;
            const float S1 = carry_s + later;
            const float S0 = S1 + bw1;
            carry_s = carry_s + __shfl_sync(FULL, suf, 0);
            const float base_g = a_ref * t_end;
            const float ds0 = (q.s1[0] - q.s0[0]) * (base_g + (b0 * Tn0 - S0));
            const float ds1 = (q.s1[1] - q.s0[1]) * (base_g + (b1 * T2 - S1));
            if constexpr (WEIGHTS) {
                if (q.v0 && q.v1) {
                    *reinterpret_cast<float2*>(a.d_sigmas + j0) = make_float2(ds0, ds1);
                } else if (q.v0) {
                    a.d_sigmas[j0] = ds0;
                } else if (q.v1) {
                    a.d_sigmas[j0 + 1] = ds1;
                }
            } else if (q.v0 && q.v1) {
                *reinterpret_cast<float2*>(a.d_sigmas + j0) = make_float2(ds0, ds1);
                float2* dr = reinterpret_cast<float2*>(a.d_rgbs + 3 * j0);
                dr[0] = make_float2(w0 * gc0, w0 * gc1);
                dr[1] = make_float2(w0 * gc2, w1 * gc0);
                dr[2] = make_float2(w1 * gc1, w1 * gc2);
            } else if (q.v0) {
                a.d_sigmas[j0] = ds0;
                a.d_rgbs[3 * j0] = w0 * gc0;
                a.d_rgbs[3 * j0 + 1] = w0 * gc1;
                a.d_rgbs[3 * j0 + 2] = w0 * gc2;
            } else if (q.v1) {
                a.d_sigmas[j0 + 1] = ds1;
                a.d_rgbs[3 * j0 + 3] = w1 * gc0;
                a.d_rgbs[3 * j0 + 4] = w1 * gc1;
                a.d_rgbs[3 * j0 + 5] = w1 * gc2;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// forward and backward with the chunks staged in shared memory by bulk copies
// ---------------------------------------------------------------------------
//
// The same walk, lane mapping and arithmetic as the register kernels above (so
// the results are bit-identical), but a chunk's arrays reach the warp through
// a ring of NST shared-memory stages: lane 0 issues one bulk copy per array and
// chunk, up to NST - 1 chunks ahead of the chunk being computed, across the
// rays of the warp's group (the backward walks each ray's chunks last to
// first). Several chunks' loads are then in flight per warp without holding
// registers. A forward stage holds a 68-sample window: the chunk's 64 samples
// from the 16-byte boundary at or below its first pair; a backward stage holds
// two consecutive chunks of a ray (132 samples), halving the per-chunk cost of
// the waits, copies and cursors. Samples from n4 =
// n_samples & ~3 on (the arrays' last partial 16 bytes) are read from global
// memory directly. Needs t_starts, t_ends, sigmas, rgbs (and the optical
// depth in the backward) 16-byte aligned; the entry points use the register
// kernels otherwise.

constexpr int kSpan = 68;                        // forward: samples per stage window (one chunk)
constexpr int kBwdSpan = 132;                    // backward: two consecutive chunks per stage
constexpr int kFwdStage = 3 * kSpan + 3 * kSpan;  // t_s, t_e, sigma, rgb (floats)
constexpr int kBwdStage = 4 * kBwdSpan + 3 * kBwdSpan;  // t_s, t_e, sigma, O, rgb
constexpr int kBarBytes = 256;                   // mbarriers of the block (up to 8 stages x 4 warps)
constexpr int kStageWaitPolls = 1 << 20;         // polls of a stage's barrier before the walk gives up
constexpr int kBulkMinBlocks = 8;                // register cap of the staged kernels (64 per thread)

static_assert((kRenderThreads / 32) * 8 * 8 <= kBarBytes, "barrier area");
static_assert(kSpan % 4 == 0 && kBwdSpan % 4 == 0 && kFwdStage % 4 == 0 && kBwdStage % 4 == 0,
              "16-byte stage layout");

size_t bulk_smem_bytes(int nst, bool bwd) {
    return kBarBytes + (size_t)(kRenderThreads / 32) * nst * (bwd ? kBwdStage : kFwdStage) * sizeof(float);
}

// Copied window [lo, hi) of chunk c of the run [rlo, rhi): from the 16-byte
// boundary at or below the chunk's first pair to the one at or above its last
// sample, clipped to n4.
struct Win {
    unsigned lo, hi;
};

__device__ __forceinline__ Win chunk_window(unsigned rlo, unsigned rhi, int c, unsigned n4) {
    const unsigned c0 = (rlo & ~1u) + ((unsigned)c << 6);
    const unsigned end = min(c0 + 64u, rhi);
    Win w;
    w.lo = c0 & ~3u;
    w.hi = min((end + 3u) & ~3u, n4);
    if (w.hi < w.lo) w.hi = w.lo;
    return w;
}

// The window of chunks c - 1 and c (c alone when c = 0): from the 16-byte boundary
// at or below chunk c - 1's first pair to the one at or above chunk c's last
// sample, clipped to n4 (at most 132 samples).
__device__ __forceinline__ Win pair_window(unsigned rlo, unsigned rhi, int c, unsigned n4) {
    const unsigned c1 = (rlo & ~1u) + ((unsigned)c << 6);
    const unsigned c0 = c > 0 ? c1 - 64u : c1;
    const unsigned end = min(c1 + 64u, rhi);
    Win w;
    w.lo = c0 & ~3u;
    w.hi = min((end + 3u) & ~3u, n4);
    if (w.hi < w.lo) w.hi = w.lo;
    return w;
}

// Lane 0: announce the window's bytes on the stage's barrier and copy the arrays
// (od may be null: forward layout). (Copies issued by lanes 0 .. 4 at once, one
// array each, measured slower.)
template <int SPAN>
__device__ __forceinline__ void issue_window(float* st, uint64_t* bar, Win w, const float* ts, const float* te,
                                             const float* sg, const float* od, const float* rgb, unsigned extra = 0) {
    const unsigned n = w.hi - w.lo, b = 4u * n;
    mbar_arrive_expect_tx(bar, (od ? 7u * b : 6u * b) + extra);
    if (n) {
        bulk_copy_g2s(st, ts + w.lo, b, bar);
        bulk_copy_g2s(st + SPAN, te + w.lo, b, bar);
        bulk_copy_g2s(st + 2 * SPAN, sg + w.lo, b, bar);
        if (od) {
            bulk_copy_g2s(st + 3 * SPAN, od + w.lo, b, bar);
            bulk_copy_g2s(st + 4 * SPAN, rgb + 3 * (size_t)w.lo, 3u * b, bar);
        } else {
            bulk_copy_g2s(st + 3 * SPAN, rgb + 3 * (size_t)w.lo, 3u * b, bar);
        }
    }
}

// The lane's pair j0, j0 + 1 of a run [lo, hi) from a stage whose window starts
// at wlo (rgb at st + rgb_at), as load_pair gives it. Every sample of the
// chunk below n4 is in the window; those at or beyond n4 come from global memory.
template <int SPAN>
__device__ __forceinline__ void stage_pair(const float* st, int rgb_at, unsigned wlo, unsigned n4,
                                           const float* __restrict__ ts, const float* __restrict__ te,
                                           const float* __restrict__ sig, const float* __restrict__ rgbs,
                                           unsigned j0, unsigned lo, unsigned hi, Pair& q) {
    q.v0 = j0 >= lo && j0 < hi;
    q.v1 = j0 + 1 >= lo && j0 + 1 < hi;
#pragma unroll
    for (int k = 0; k < 2; ++k) q.s0[k] = q.s1[k] = q.sg[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) q.rgb[k] = 0.0f;
    const unsigned p = j0 - wlo;  // even: j0 and wlo are
    if (q.v0 && q.v1 && j0 + 1 < n4) {
        const float2 u = *reinterpret_cast<const float2*>(st + p);
        const float2 v = *reinterpret_cast<const float2*>(st + SPAN + p);
        const float2 g = *reinterpret_cast<const float2*>(st + 2 * SPAN + p);
        const float2* c = reinterpret_cast<const float2*>(st + rgb_at + 3 * p);
        const float2 c0 = c[0], c1 = c[1], c2 = c[2];
        q.s0[0] = u.x; q.s0[1] = u.y;
        q.s1[0] = v.x; q.s1[1] = v.y;
        q.sg[0] = g.x; q.sg[1] = g.y;
        q.rgb[0] = c0.x; q.rgb[1] = c0.y; q.rgb[2] = c1.x;
        q.rgb[3] = c1.y; q.rgb[4] = c2.x; q.rgb[5] = c2.y;
    } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 0 ? q.v0 : q.v1) {
                const unsigned j = j0 + k;
                if (j < n4) {
                    const unsigned l = p + k;
                    q.s0[k] = st[l];
                    q.s1[k] = st[SPAN + l];
                    q.sg[k] = st[2 * SPAN + l];
                    q.rgb[3 * k] = st[rgb_at + 3 * l];
                    q.rgb[3 * k + 1] = st[rgb_at + 3 * l + 1];
                    q.rgb[3 * k + 2] = st[rgb_at + 3 * l + 2];
                } else {
                    q.s0[k] = __ldg(ts + j);
                    q.s1[k] = __ldg(te + j);
                    q.sg[k] = __ldg(sig + j);
                    q.rgb[3 * k] = __ldg(rgbs + 3 * (size_t)j);
                    q.rgb[3 * k + 1] = __ldg(rgbs + 3 * (size_t)j + 1);
                    q.rgb[3 * k + 2] = __ldg(rgbs + 3 * (size_t)j + 2);
                }
            }
        }
    }
}

// Cursor over the chunks of the rays of a warp's group: rays in order (set bits
// of `todo`, lane i = ray i), chunks first to last, or last to first (REV).
template <bool REV, int STEP = 1>
struct ChunkCursor {
    unsigned todo, lo, hi;
    int i, c, nch;
    __device__ __forceinline__ void ray(int my_off, int my_cnt, int my_nch) {
        i = __ffs(todo) - 1;
        todo &= todo - 1;
        lo = (unsigned)__shfl_sync(FULL, my_off, i);
        hi = lo + (unsigned)__shfl_sync(FULL, my_cnt, i);
        nch = __shfl_sync(FULL, my_nch, i);
        c = REV ? nch - 1 : 0;
    }
    // next chunk (STEP chunks on); returns true when it starts a new ray
    __device__ __forceinline__ bool next(int my_off, int my_cnt, int my_nch) {
        c += REV ? -STEP : STEP;
        if (REV ? c < 0 : c >= nch) {
            if (todo) ray(my_off, my_cnt, my_nch);
            return true;
        }
        return false;
    }
};

// After a stage wait gave up: report it, then wait (bounded) for the copies the
// warp has in flight, so that none lands after the block has exited. A first
// chunk whose announced bytes were overstated by the test hook never completes
// and has no copy outstanding: it is not waited for.
template <int NST>
__device__ __forceinline__ void drain_stages(uint64_t* bars, int k, int total, bool poisoned, int32_t* d_status,
                                             int lane) {
    if (lane == 0) raise_status(d_status, NACC_STATUS_TIMEOUT);
    const int end = min(k + NST, total);
    for (int d = k; d < end; ++d)
        if (!(d == 0 && poisoned)) mbar_wait_bounded(&bars[d % NST], (unsigned)(d / NST) & 1u, kSpinLimit);
    __syncwarp();
}

template <int NST>
__global__ void __launch_bounds__(kRenderThreads, kBulkMinBlocks) render_fwd_bulk_kernel(const FwdArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(dyn_smem) + wib * NST;
    float* stages = reinterpret_cast<float*>(dyn_smem + kBarBytes) + (size_t)wib * NST * kFwdStage;
    const int ray0 = global_warp() * kGroup;
    if (ray0 >= a.n_rays) return;
    const int nr = min(kGroup, a.n_rays - ray0);
    int my_off, my_cnt;
    load_group(a.packed_info, ray0, nr, a.n_samples, a.d_status, lane, my_off, my_cnt);
    if (lane < nr && my_cnt == 0) {
        const int r = ray0 + lane;
        if (a.color) {
            a.color[3 * (size_t)r] = 0.0f;
            a.color[3 * (size_t)r + 1] = 0.0f;
            a.color[3 * (size_t)r + 2] = 0.0f;
        }
        if (a.opacity) a.opacity[r] = 0.0f;
        if (a.depth) a.depth[r] = 0.0f;
    }
    const unsigned todo = __ballot_sync(FULL, my_cnt > 0);
    if (todo == 0u) return;
    const int my_nch = my_cnt > 0 ? (int)(((unsigned)my_off + my_cnt - ((unsigned)my_off & ~1u) + 63u) >> 6) : 0;
    int total = my_nch;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULL, total, o);
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncwarp();
    const unsigned n4 = (unsigned)a.n_samples & ~3u;

    ChunkCursor<false> P;  // producer: the next chunk to copy
    P.todo = todo;
    P.ray(my_off, my_cnt, my_nch);
    const int pre = min(NST, total);
    for (int k = 0; k < pre; ++k) {
        if (lane == 0)
            issue_window<kSpan>(stages + k * kFwdStage, &bars[k], chunk_window(P.lo, P.hi, P.c, n4), a.t_starts,
                                a.t_ends,
                         a.sigmas, nullptr, a.rgbs, k == 0 ? a.stage_extra : 0u);
        P.next(my_off, my_cnt, my_nch);
    }

    ChunkCursor<false> C;  // consumer: the chunk being computed
    C.todo = todo;
    C.ray(my_off, my_cnt, my_nch);
    float carry = 0.0f;
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, op = 0.0f, dp = 0.0f;
    for (int k = 0; k < total; ++k) {
        const int s = k % NST;
        float* st = stages + s * kFwdStage;
        const bool ok = mbar_wait_bounded(&bars[s], (unsigned)(k / NST) & 1u, a.stage_polls);
        if (!__all_sync(FULL, ok)) {
            drain_stages<NST>(bars, k, total, a.stage_extra != 0u, a.d_status, lane);
            return;
        }
        const unsigned qj0 = (C.lo & ~1u) + ((unsigned)C.c << 6) + 2 * lane;
        Pair q;
        stage_pair<kSpan>(st, 3 * kSpan, ((C.lo & ~1u) + ((unsigned)C.c << 6)) & ~3u, n4, a.t_starts, a.t_ends, a.sigmas,
                   a.rgbs, qj0, C.lo, C.hi, q);
        const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
        const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
        float O0, O1;
        pair_optical_depth(tau0, tau1, carry, lane, O0, O1);
        const float w0 = q.v0 ? __expf(-O0) * alpha_of(tau0) : 0.0f;
        const float w1 = q.v1 ? __expf(-O1) * alpha_of(tau1) : 0.0f;
        c0 += w0 * q.rgb[0] + w1 * q.rgb[3];
        c1 += w0 * q.rgb[1] + w1 * q.rgb[4];
        c2 += w0 * q.rgb[2] + w1 * q.rgb[5];
        op += w0 + w1;
        dp += w0 * ((q.s0[0] + q.s1[0]) * 0.5f) + w1 * ((q.s0[1] + q.s1[1]) * 0.5f);
        if (a.optical_depth) {
            if (q.v0) a.optical_depth[qj0] = O0;
            if (q.v1) a.optical_depth[qj0 + 1] = O1;
        }
        // the stage is read: refill it with the chunk NST ahead
        __syncwarp();
        if (k + NST < total) {
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_window<kSpan>(st, &bars[s], chunk_window(P.lo, P.hi, P.c, n4), a.t_starts, a.t_ends, a.sigmas, nullptr,
                             a.rgbs);
            }
            P.next(my_off, my_cnt, my_nch);
        }
        if (C.c + 1 == C.nch) {
            const float sum = warp_sum5(c0, c1, c2, op, dp, lane);
            const size_t r = (size_t)ray0 + C.i;
            if (lane == 0 && a.color) a.color[3 * r] = sum;
            if (lane == 4 && a.color) a.color[3 * r + 1] = sum;
            if (lane == 8 && a.color) a.color[3 * r + 2] = sum;
            if (lane == 12 && a.opacity) a.opacity[r] = sum;
            if (lane == 16 && a.depth) a.depth[r] = sum;
            carry = 0.0f;
            c0 = c1 = c2 = op = dp = 0.0f;
        }
        C.next(my_off, my_cnt, my_nch);
    }
}

// Backward with the optical depth saved by the forward (colour mode).
template <int NST>
__global__ void __launch_bounds__(kRenderThreads, kBulkMinBlocks) render_bwd_bulk_kernel(const BwdArgs a) {
    __shared__ float s_ray[kRenderThreads / 32][kGroup][kRayVals];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float(*ray_vals)[kRayVals] = s_ray[wib];
    uint64_t* bars = reinterpret_cast<uint64_t*>(dyn_smem) + wib * NST;
    float* stages = reinterpret_cast<float*>(dyn_smem + kBarBytes) + (size_t)wib * NST * kBwdStage;
    const int ray0 = global_warp() * kGroup;
    if (ray0 >= a.n_rays) return;
    const int nr = min(kGroup, a.n_rays - ray0);
    int my_off, my_cnt;
    load_group(a.packed_info, ray0, nr, a.n_samples, a.d_status, lane, my_off, my_cnt);
    if (lane < nr && my_cnt > 0) {
        const size_t r = (size_t)ray0 + lane;
        float* v = ray_vals[lane];
        v[0] = a.g_color ? a.g_color[3 * r] : 0.0f;
        v[1] = a.g_color ? a.g_color[3 * r + 1] : 0.0f;
        v[2] = a.g_color ? a.g_color[3 * r + 2] : 0.0f;
        v[3] = a.g_opacity ? a.g_opacity[r] : 0.0f;
        v[4] = a.g_depth ? a.g_depth[r] : 0.0f;
        v[5] = __ldg(a.rgbs + 3 * (size_t)my_off);
        v[6] = __ldg(a.rgbs + 3 * (size_t)my_off + 1);
        v[7] = __ldg(a.rgbs + 3 * (size_t)my_off + 2);
        v[8] = (__ldg(a.t_starts + my_off) + __ldg(a.t_ends + my_off)) * 0.5f;
    }
    const unsigned todo = __ballot_sync(FULL, my_cnt > 0);
    if (todo == 0u) return;
    const int my_nch = my_cnt > 0 ? (int)(((unsigned)my_off + my_cnt - ((unsigned)my_off & ~1u) + 63u) >> 6) : 0;
    // a stage holds chunks c and c - 1 of a ray (c alone when c = 0), walked c first
    int total = (my_nch + 1) >> 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(FULL, total, o);
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncwarp();
    const unsigned n4 = (unsigned)a.n_samples & ~3u;

    ChunkCursor<true, 2> P;
    P.todo = todo;
    P.ray(my_off, my_cnt, my_nch);
    const int pre = min(NST, total);
    for (int k = 0; k < pre; ++k) {
        if (lane == 0)
            issue_window<kBwdSpan>(stages + k * kBwdStage, &bars[k], pair_window(P.lo, P.hi, P.c, n4), a.t_starts,
                                   a.t_ends, a.sigmas, a.optical_depth, a.rgbs, k == 0 ? a.stage_extra : 0u);
        P.next(my_off, my_cnt, my_nch);
    }

    ChunkCursor<true, 2> C;
    C.todo = todo;
    C.ray(my_off, my_cnt, my_nch);
    // per-ray values (see render_bwd_kernel for the centred form)
    float gc0 = 0.0f, gc1 = 0.0f, gc2 = 0.0f, gd = 0.0f;
    float r_ref = 0.0f, g_ref = 0.0f, b_ref = 0.0f, tm_ref = 0.0f, a_ref = 0.0f;
    int last_lane = 0;
    bool last_odd = false;
    float t_end = 0.0f, carry_s = 0.0f;
    auto begin_ray = [&]() {
        const float* rv = ray_vals[C.i];
        gc0 = rv[0];
        gc1 = rv[1];
        gc2 = rv[2];
        const float ga = rv[3];
        gd = rv[4];
        r_ref = rv[5];
        g_ref = rv[6];
        b_ref = rv[7];
        tm_ref = rv[8];
        a_ref = gc0 * r_ref + gc1 * g_ref + gc2 * b_ref + ga + gd * tm_ref;
        const unsigned last = C.hi - 1 - (C.lo & ~1u);
        last_lane = (int)((last >> 1) & 31);
        last_odd = (last & 1) != 0;
        t_end = 0.0f;
        carry_s = 0.0f;
    };
    __syncwarp();  // ray_vals written by their lanes
    begin_ray();
    for (int k = 0; k < total; ++k) {
        const int s = k % NST;
        float* st = stages + s * kBwdStage;
        const bool ok = mbar_wait_bounded(&bars[s], (unsigned)(k / NST) & 1u, a.stage_polls);
        if (!__all_sync(FULL, ok)) {
            drain_stages<NST>(bars, k, total, a.stage_extra != 0u, a.d_status, lane);
            return;
        }
        const unsigned abase = C.lo & ~1u;
        const unsigned wlo = (abase + ((unsigned)(C.c > 0 ? C.c - 1 : 0) << 6)) & ~3u;
        const int n_in = C.c > 0 ? 2 : 1;
        for (int u = 0; u < n_in; ++u) {
            const int c = C.c - u;
            const unsigned j0 = abase + ((unsigned)c << 6) + 2 * lane;
            Pair q;
            stage_pair<kBwdSpan>(st, 4 * kBwdSpan, wlo, n4, a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, C.lo, C.hi,
                                 q);
            float O0 = 0.0f, O1 = 0.0f;
            {
                const unsigned p = j0 - wlo;
                if (q.v0) O0 = j0 < n4 ? st[3 * kBwdSpan + p] : __ldg(a.optical_depth + j0);
                if (q.v1) O1 = j0 + 1 < n4 ? st[3 * kBwdSpan + p + 1] : __ldg(a.optical_depth + j0 + 1);
            }
            const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
            const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
            if (u == n_in - 1) {  // the stage is read: refill it with the stage NST ahead
                __syncwarp();
                if (k + NST < total) {
                    if (lane == 0) {
                        fence_proxy_async_smem();
                        issue_window<kBwdSpan>(st, &bars[s], pair_window(P.lo, P.hi, P.c, n4), a.t_starts, a.t_ends,
                                               a.sigmas, a.optical_depth, a.rgbs);
                    }
                    P.next(my_off, my_cnt, my_nch);
                }
            }
            const float T0 = __expf(-O0);
            const float T1 = __expf(-O1);
            const float T2 = __expf(-__fadd_rn(O1, tau1));
            const float Tn0 = q.v1 ? T1 : __expf(-__fadd_rn(O0, tau0));
            if (c == C.nch - 1) t_end = __shfl_sync(FULL, last_odd ? T2 : Tn0, last_lane);
            const float w0 = q.v0 ? T0 * alpha_of(tau0) : 0.0f;
            const float w1 = q.v1 ? T1 * alpha_of(tau1) : 0.0f;
            const float tm0 = (q.s0[0] + q.s1[0]) * 0.5f, tm1 = (q.s0[1] + q.s1[1]) * 0.5f;
            const float b0 = gc0 * (q.rgb[0] - r_ref) + gc1 * (q.rgb[1] - g_ref) + gc2 * (q.rgb[2] - b_ref) +
                             gd * (tm0 - tm_ref);
            const float b1 = gc0 * (q.rgb[3] - r_ref) + gc1 * (q.rgb[4] - g_ref) + gc2 * (q.rgb[5] - b_ref) +
                             gd * (tm1 - tm_ref);
            const float bw0 = q.v0 ? b0 * w0 : 0.0f;
            const float bw1 = q.v1 ? b1 * w1 : 0.0f;
            const float suf = warp_incl_suffix(bw0 + bw1, lane);
            float later = __shfl_down_sync(FULL, suf, 1);
            if (lane == 31) later = 0.0f;
            const float S1 = carry_s + later;
            const float S0 = S1 + bw1;
            carry_s = carry_s + __shfl_sync(FULL, suf, 0);
            const float base_g = a_ref * t_end;
            const float ds0 = (q.s1[0] - q.s0[0]) * (base_g + (b0 * Tn0 - S0));
            const float ds1 = (q.s1[1] - q.s0[1]) * (base_g + (b1 * T2 - S1));
            if (q.v0 && q.v1) {
                *reinterpret_cast<float2*>(a.d_sigmas + j0) = make_float2(ds0, ds1);
                float2* dr = reinterpret_cast<float2*>(a.d_rgbs + 3 * (size_t)j0);
                dr[0] = make_float2(w0 * gc0, w0 * gc1);
                dr[1] = make_float2(w0 * gc2, w1 * gc0);
                dr[2] = make_float2(w1 * gc1, w1 * gc2);
            } else if (q.v0) {
                a.d_sigmas[j0] = ds0;
                a.d_rgbs[3 * (size_t)j0] = w0 * gc0;
                a.d_rgbs[3 * (size_t)j0 + 1] = w0 * gc1;
                a.d_rgbs[3 * (size_t)j0 + 2] = w0 * gc2;
            } else if (q.v1) {
                a.d_sigmas[j0 + 1] = ds1;
                a.d_rgbs[3 * (size_t)j0 + 3] = w1 * gc0;
                a.d_rgbs[3 * (size_t)j0 + 4] = w1 * gc1;
                a.d_rgbs[3 * (size_t)j0 + 5] = w1 * gc2;
            }
        }
        if (C.next(my_off, my_cnt, my_nch) && k + 1 < total) begin_ray();
    }
}

// ---------------------------------------------------------------------------
// forward, squared-error loss gradient and backward in one pass
// ---------------------------------------------------------------------------
//
// For a loss L = (s / 2) sum_r |C_r - C*_r|^2 (s = 2 / (3 R): the mean squared
// error of the colours) dL/dC_r = s (C_r - C*_r) is known as soon as ray r's
// colour is: the warp renders the ray forward (render_fwd_kernel's arithmetic,
// keeping each chunk's optical-depth carry in shared memory), forms the
// gradient, and runs the reverse scan (render_bwd_kernel's recompute path) over
// the same samples while they are still in L2. The samples are read from DRAM
// once instead of twice and no optical depth is stored; the results equal those
// of nacc_render_fwd, the gradient formed as (C - C*) * s in float32, and
// nacc_render_bwd.

struct MseArgs {
    const int32_t* packed_info;
    int32_t n_rays;
    const float* t_starts;
    const float* t_ends;
    const float* sigmas;
    const float* rgbs;
    int64_t n_samples;
    const float* target;  // (n_rays, 3)
    float grad_scale;     // s
    float* color;
    float* opacity;
    float* depth;
    float* sq_err;  // per ray sum_c (C - C*)^2, or null
    float* d_sigmas;
    float* d_rgbs;
    int32_t* d_status;
};

template <int MINB>
__global__ void __launch_bounds__(kRenderThreads, MINB) render_mse_kernel(const MseArgs a) {
    __shared__ float s_carry[kRenderThreads / 32][kCarryCap];
    const int lane = threadIdx.x & 31;
    float* carries = s_carry[threadIdx.x >> 5];
    const int ray0 = global_warp() * kGroup;
    if (ray0 >= a.n_rays) return;
    const int nr = min(kGroup, a.n_rays - ray0);
    int my_off, my_cnt;
    load_group(a.packed_info, ray0, nr, a.n_samples, a.d_status, lane, my_off, my_cnt);
    for (int ri = 0; ri < nr; ++ri) {
        const unsigned lo = __shfl_sync(FULL, my_off, ri);
        const int cnt = __shfl_sync(FULL, my_cnt, ri);
        const size_t r = (size_t)ray0 + ri;
        const unsigned hi = lo + cnt;
        const unsigned abase = lo & ~1u;
        const int nch = cnt > 0 ? (int)((hi - abase + 63) >> 6) : 0;

        // forward: chunks in order, the carry at the start of each chunk kept
        float carry = 0.0f;
        float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, op = 0.0f, dp = 0.0f;
        for (int c = 0; c < nch; ++c) {
            if (lane == 0 && c < kCarryCap) carries[c] = carry;
            Pair q;
            load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, abase + ((unsigned)c << 6) + 2 * lane, lo, hi, q);
            const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
            const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
            float O0, O1;
            pair_optical_depth(tau0, tau1, carry, lane, O0, O1);
            const float w0 = q.v0 ? __expf(-O0) * alpha_of(tau0) : 0.0f;
            const float w1 = q.v1 ? __expf(-O1) * alpha_of(tau1) : 0.0f;
            c0 += w0 * q.rgb[0] + w1 * q.rgb[3];
            c1 += w0 * q.rgb[1] + w1 * q.rgb[4];
            c2 += w0 * q.rgb[2] + w1 * q.rgb[5];
            op += w0 + w1;
            dp += w0 * ((q.s0[0] + q.s1[0]) * 0.5f) + w1 * ((q.s0[1] + q.s1[1]) * 0.5f);
        }
        const float sum = warp_sum5(c0, c1, c2, op, dp, lane);
        if (lane == 0 && a.color) a.color[3 * r] = sum;
        if (lane == 4 && a.color) a.color[3 * r + 1] = sum;
        if (lane == 8 && a.color) a.color[3 * r + 2] = sum;
        if (lane == 12 && a.opacity) a.opacity[r] = sum;
        if (lane == 16 && a.depth) a.depth[r] = sum;
        const float e0 = __fsub_rn(__shfl_sync(FULL, sum, 0), __ldg(a.target + 3 * r));
        const float e1 = __fsub_rn(__shfl_sync(FULL, sum, 4), __ldg(a.target + 3 * r + 1));
        const float e2 = __fsub_rn(__shfl_sync(FULL, sum, 8), __ldg(a.target + 3 * r + 2));
        if (lane == 0 && a.sq_err) a.sq_err[r] = e0 * e0 + e1 * e1 + e2 * e2;
        if (nch == 0) continue;
        const float gc0 = __fmul_rn(e0, a.grad_scale);
        const float gc1 = __fmul_rn(e1, a.grad_scale);
        const float gc2 = __fmul_rn(e2, a.grad_scale);
        const float ga = 0.0f, gd = 0.0f;
        __syncwarp();  // the carries

        // backward (render_bwd_kernel, recompute path): chunks in reverse order
        const float r_ref = __ldg(a.rgbs + 3 * (size_t)lo);
        const float g_ref = __ldg(a.rgbs + 3 * (size_t)lo + 1);
        const float b_ref = __ldg(a.rgbs + 3 * (size_t)lo + 2);
        const float tm_ref = (__ldg(a.t_starts + lo) + __ldg(a.t_ends + lo)) * 0.5f;
        const float a_ref = gc0 * r_ref + gc1 * g_ref + gc2 * b_ref + ga + gd * tm_ref;
        const unsigned last = hi - 1 - abase;
        const int last_lane = (int)((last >> 1) & 31);
        const bool last_odd = (last & 1) != 0;
        float t_end = 0.0f;
        float carry_s = 0.0f;
        for (int c = nch - 1; c >= 0; --c) {
            float carry_o;
            if (c < kCarryCap) {
                carry_o = carries[c];
            } else {  // rays longer than the shared-memory record: rescan from the last record
                carry_o = carries[kCarryCap - 1];
                for (int p = kCarryCap - 1; p < c; ++p) {
                    const unsigned pj = abase + ((unsigned)p << 6) + 2 * lane;
                    const bool pv0 = pj >= lo && pj < hi, pv1 = pj + 1 >= lo && pj + 1 < hi;
                    const float t0 = pv0 ? tau_of(__ldg(a.t_starts + pj), __ldg(a.t_ends + pj), __ldg(a.sigmas + pj))
                                         : 0.0f;
                    const float t1 = pv1 ? tau_of(__ldg(a.t_starts + pj + 1), __ldg(a.t_ends + pj + 1),
                                                  __ldg(a.sigmas + pj + 1))
                                         : 0.0f;
                    float O0, O1;
                    pair_optical_depth(t0, t1, carry_o, lane, O0, O1);
                }
            }
            const unsigned j0 = abase + ((unsigned)c << 6) + 2 * lane;
            Pair q;
            load_pair(a.t_starts, a.t_ends, a.sigmas, a.rgbs, j0, lo, hi, q);
            const float tau0 = q.v0 ? tau_of(q.s0[0], q.s1[0], q.sg[0]) : 0.0f;
            const float tau1 = q.v1 ? tau_of(q.s0[1], q.s1[1], q.sg[1]) : 0.0f;
            float O0, O1;
            pair_optical_depth(tau0, tau1, carry_o, lane, O0, O1);
            const float T0 = __expf(-O0);
            const float T1 = __expf(-O1);
            const float T2 = __expf(-__fadd_rn(O1, tau1));
            const float Tn0 = q.v1 ? T1 : __expf(-__fadd_rn(O0, tau0));
            if (c == nch - 1) t_end = __shfl_sync(FULL, last_odd ? T2 : Tn0, last_lane);
            const float w0 = q.v0 ? T0 * alpha_of(tau0) : 0.0f;
            const float w1 = q.v1 ? T1 * alpha_of(tau1) : 0.0f;
            const float tm0 = (q.s0[0] + q.s1[0]) * 0.5f, tm1 = (q.s0[1] + q.s1[1]) * 0.5f;
            const float b0 = gc0 * (q.rgb[0] - r_ref) + gc1 * (q.rgb[1] - g_ref) + gc2 * (q.rgb[2] - b_ref) +
                             gd * (tm0 - tm_ref);
            const float b1 = gc0 * (q.rgb[3] - r_ref) + gc1 * (q.rgb[4] - g_ref) + gc2 * (q.rgb[5] - b_ref) +
                             gd * (tm1 - tm_ref);
            const float bw0 = q.v0 ? b0 * w0 : 0.0f;
            const float bw1 = q.v1 ? b1 * w1 : 0.0f;
            const float suf = warp_incl_suffix(bw0 + bw1, lane);
            float later = __shfl_down_sync(FULL, suf, 1);
            if (lane == 31) later = 0.0f;
            const float S1 = carry_s + later;
            const float S0 = S1 + bw1;
            carry_s = carry_s + __shfl_sync(FULL, suf, 0);
            const float base_g = a_ref * t_end;
            const float ds0 = (q.s1[0] - q.s0[0]) * (base_g + (b0 * Tn0 - S0));
            const float ds1 = (q.s1[1] - q.s0[1]) * (base_g + (b1 * T2 - S1));
            if (q.v0 && q.v1) {
                *reinterpret_cast<float2*>(a.d_sigmas + j0) = make_float2(ds0, ds1);
                float2* dr = reinterpret_cast<float2*>(a.d_rgbs + 3 * (size_t)j0);
                dr[0] = make_float2(w0 * gc0, w0 * gc1);
                dr[1] = make_float2(w0 * gc2, w1 * gc0);
                dr[2] = make_float2(w1 * gc1, w1 * gc2);
            } else if (q.v0) {
                a.d_sigmas[j0] = ds0;
                a.d_rgbs[3 * (size_t)j0] = w0 * gc0;
                a.d_rgbs[3 * (size_t)j0 + 1] = w0 * gc1;
                a.d_rgbs[3 * (size_t)j0 + 2] = w0 * gc2;
            } else if (q.v1) {
                a.d_sigmas[j0 + 1] = ds1;
                a.d_rgbs[3 * (size_t)j0 + 3] = w1 * gc0;
                a.d_rgbs[3 * (size_t)j0 + 4] = w1 * gc1;
                a.d_rgbs[3 * (size_t)j0 + 5] = w1 * gc2;
            }
        }
        __syncwarp();  // the carries are read before the next ray writes them
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

// value into arr[i * width + c] for n <= i < capacity (n read on the device,
// clamped to [0, capacity]).
__global__ void __launch_bounds__(kThreads) fill_tail_kernel(float* arr, int64_t width, int64_t capacity,
                                                             const int64_t* n_dev, float value) {
    int64_t n = *n_dev;
    n = n < 0 ? 0 : (n > capacity ? capacity : n);
    const int64_t begin = n * width, end = capacity * width;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) arr[i] = value;
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

// one warp per group of kGroup consecutive rays
int group_blocks(int n_rays) {
    const long long groups = ((long long)n_rays + kGroup - 1) / kGroup;
    return (int)((groups + kRenderThreads / 32 - 1) / (kRenderThreads / 32));
}

// Launch of a bulk-staged render kernel (the shared-memory carveout raised once
// per kernel, so that the stages of several blocks fit on an SM).
template <typename K, typename A>
int launch_bulk(K kernel, bool& carveout_set, int nst, bool bwd, int n_rays, cudaStream_t st, const A& a) {
    const size_t smem = bulk_smem_bytes(nst, bwd);
    if (!carveout_set) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        // static and dynamic shared memory together are limited to 48 KB without the opt-in
        if (smem > 40 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        carveout_set = true;
    }
    kernel<<<group_blocks(n_rays), kRenderThreads, smem, st>>>(a);
    return launch_status(cudaGetLastError());
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Stages 2, 3 or 4 per warp. (Registers capped for 12 blocks per SM instead of 8
// spill and measured slower in both passes.)
// Poll budget of the stage waits and the test hook's overstated bytes.
template <typename A>
void set_stage_hooks(A& a) {
    const LookbackHooks h = lookback_hooks();
    a.stage_polls = h.spin_limit < kSpinLimit ? h.spin_limit : kStageWaitPolls;
    a.stage_extra = h.overstate_stage ? 16u : 0u;
}

int launch_fwd_bulk(int nst, int n_rays, cudaStream_t st, FwdArgs a) {
    set_stage_hooks(a);
    static bool set2, set3, set4;
    switch (nst) {
        case 2: return launch_bulk(render_fwd_bulk_kernel<2>, set2, 2, false, n_rays, st, a);
        case 3: return launch_bulk(render_fwd_bulk_kernel<3>, set3, 3, false, n_rays, st, a);
        default: return launch_bulk(render_fwd_bulk_kernel<4>, set4, 4, false, n_rays, st, a);
    }
}

int launch_bwd_bulk(int nst, int n_rays, cudaStream_t st, BwdArgs a) {
    set_stage_hooks(a);
    static bool set2, set3, set4;
    switch (nst) {
        case 2: return launch_bulk(render_bwd_bulk_kernel<2>, set2, 2, true, n_rays, st, a);
        case 3: return launch_bulk(render_bwd_bulk_kernel<3>, set3, 3, true, n_rays, st, a);
        default: return launch_bulk(render_bwd_bulk_kernel<4>, set4, 4, true, n_rays, st, a);
    }
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
    if ((((uintptr_t)packed_info | (uintptr_t)t_starts | (uintptr_t)t_ends | (uintptr_t)sigmas | (uintptr_t)rgbs |
          (uintptr_t)optical_depth) & 7u) != 0)
        return NACC_ERR_INVALID_ARG;
    FwdArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, rgbs, n_samples, color, opacity, depth, optical_depth, d_status};
    const int nb = group_blocks(n_rays);
    cudaStream_t st = (cudaStream_t)stream;
    const int nst = tune_get(NACC_TUNE_RENDER_FWD_STAGES);
    if (nst >= 2 && n_samples > 0 && aligned16(t_starts) && aligned16(t_ends) && aligned16(sigmas) && aligned16(rgbs))
        return launch_fwd_bulk(nst, n_rays, st, a);
    const bool pf = tune_get(NACC_TUNE_RENDER_FWD_PREFETCH) != 0;
    switch (tune_get(NACC_TUNE_RENDER_OCCUPANCY)) {
        case 1:
            if (pf) render_fwd_kernel<true, 16><<<nb, kRenderThreads, 0, st>>>(a);
            else render_fwd_kernel<false, 16><<<nb, kRenderThreads, 0, st>>>(a);
            break;
        case 2:
            if (pf) render_fwd_kernel<true, 12><<<nb, kRenderThreads, 0, st>>>(a);
            else render_fwd_kernel<false, 12><<<nb, kRenderThreads, 0, st>>>(a);
            break;
        default:
            if (pf) render_fwd_kernel<true, 1><<<nb, kRenderThreads, 0, st>>>(a);
            else render_fwd_kernel<false, 1><<<nb, kRenderThreads, 0, st>>>(a);
            break;
    }
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

extern "C" int nacc_accumulate_along_rays_bwd(const int32_t* packed_info, int32_t n_rays, const float* weights,
                                              const float* values, int32_t n_channels, int64_t n_samples,
                                              const float* g_out, float* d_weights, float* d_values,
                                              float* g_ref, int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples) || n_channels < 1) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!packed_info || !g_out)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && !weights) return NACC_ERR_INVALID_ARG;
    if (d_values && !values) return NACC_ERR_INVALID_ARG;
    if (g_ref && !d_weights) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0 || (!d_weights && !d_values)) return NACC_OK;
    AccBwdArgs a{packed_info, n_rays, weights, values, n_channels, n_samples, g_out, d_weights, d_values, g_ref,
                 d_status};
    if (n_channels <= 4)
        accumulate_bwd_narrow_kernel<<<grid_for(accumulate_bwd_narrow_kernel, n_rays), kThreads, 0,
                                       (cudaStream_t)stream>>>(a);
    else
        accumulate_bwd_kernel<<<grid_for(accumulate_bwd_kernel, n_rays), kThreads, 0, (cudaStream_t)stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_render_weights_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                                       const float* t_ends, const float* sigmas, int64_t n_samples,
                                       const float* g_weights, const float* g_ref, float* d_sigmas,
                                       int32_t* d_status, void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas || !g_weights || !d_sigmas)) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    if ((((uintptr_t)packed_info | (uintptr_t)t_starts | (uintptr_t)t_ends | (uintptr_t)sigmas |
          (uintptr_t)g_weights | (uintptr_t)d_sigmas) & 7u) != 0)
        return NACC_ERR_INVALID_ARG;
    BwdArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, nullptr, nullptr, n_samples,
              nullptr, nullptr, nullptr, d_sigmas, nullptr, d_status, g_weights, g_ref};
    const int nb = group_blocks(n_rays);
    cudaStream_t st = (cudaStream_t)stream;
    switch (tune_get(NACC_TUNE_RENDER_BWD_OCCUPANCY)) {
        case 1: render_bwd_kernel<16, false, true><<<nb, kRenderThreads, 0, st>>>(a); break;
        case 2: render_bwd_kernel<12, false, true><<<nb, kRenderThreads, 0, st>>>(a); break;
        default: render_bwd_kernel<1, false, true><<<nb, kRenderThreads, 0, st>>>(a); break;
    }
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
    if ((((uintptr_t)packed_info | (uintptr_t)t_starts | (uintptr_t)t_ends | (uintptr_t)sigmas | (uintptr_t)rgbs |
          (uintptr_t)optical_depth | (uintptr_t)d_sigmas | (uintptr_t)d_rgbs) & 7u) != 0)
        return NACC_ERR_INVALID_ARG;
    BwdArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, rgbs, optical_depth, n_samples,
              g_color, g_opacity, g_depth, d_sigmas, d_rgbs, d_status, nullptr, nullptr};
    const int nb = group_blocks(n_rays);
    cudaStream_t st = (cudaStream_t)stream;
    const int nst = tune_get(NACC_TUNE_RENDER_BWD_STAGES);
    if (nst >= 2 && n_samples > 0 && optical_depth && aligned16(t_starts) && aligned16(t_ends) && aligned16(sigmas) &&
        aligned16(rgbs) && aligned16(optical_depth))
        return launch_bwd_bulk(nst, n_rays, st, a);
    const bool pf = tune_get(NACC_TUNE_RENDER_BWD_PREFETCH) != 0;
    switch (tune_get(NACC_TUNE_RENDER_BWD_OCCUPANCY)) {
        case 1:
            if (pf) render_bwd_kernel<16, true><<<nb, kRenderThreads, 0, st>>>(a);
            else render_bwd_kernel<16, false><<<nb, kRenderThreads, 0, st>>>(a);
            break;
        case 2:
            if (pf) render_bwd_kernel<12, true><<<nb, kRenderThreads, 0, st>>>(a);
            else render_bwd_kernel<12, false><<<nb, kRenderThreads, 0, st>>>(a);
            break;
        default:
            if (pf) render_bwd_kernel<1, true><<<nb, kRenderThreads, 0, st>>>(a);
            else render_bwd_kernel<1, false><<<nb, kRenderThreads, 0, st>>>(a);
            break;
    }
    return launch_status(cudaGetLastError());
}

extern "C" int nacc_render_mse_fused(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                                     const float* t_ends, const float* sigmas, const float* rgbs, int64_t n_samples,
                                     const float* target, float grad_scale, float* color, float* opacity,
                                     float* depth, float* sq_err, float* d_sigmas, float* d_rgbs, int32_t* d_status,
                                     void* stream) {
    if (!sizes_ok(n_rays, n_samples)) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && (!packed_info || !target)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!t_starts || !t_ends || !sigmas || !rgbs || !d_sigmas || !d_rgbs))
        return NACC_ERR_INVALID_ARG;
    if (!(fabsf(grad_scale) <= 3.402823466e+38f)) return NACC_ERR_INVALID_ARG;
    if (n_rays == 0) return NACC_OK;
    if ((((uintptr_t)packed_info | (uintptr_t)t_starts | (uintptr_t)t_ends | (uintptr_t)sigmas | (uintptr_t)rgbs |
          (uintptr_t)d_sigmas | (uintptr_t)d_rgbs) & 7u) != 0)
        return NACC_ERR_INVALID_ARG;
    MseArgs a{packed_info, n_rays, t_starts, t_ends, sigmas, rgbs, n_samples, target, grad_scale,
              color, opacity, depth, sq_err, d_sigmas, d_rgbs, d_status};
    const int nb = group_blocks(n_rays);
    cudaStream_t st = (cudaStream_t)stream;
    switch (tune_get(NACC_TUNE_RENDER_MSE_OCCUPANCY)) {
        case 1: render_mse_kernel<8><<<nb, kRenderThreads, 0, st>>>(a); break;
        case 2: render_mse_kernel<12><<<nb, kRenderThreads, 0, st>>>(a); break;
        default: render_mse_kernel<1><<<nb, kRenderThreads, 0, st>>>(a); break;
    }
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

extern "C" int nacc_fill_tail_f32(float* arr, int64_t width, int64_t capacity, const int64_t* n_dev, float value,
                                  void* stream) {
    if (width < 1 || capacity < 0 || !n_dev || (capacity > 0 && !arr)) return NACC_ERR_INVALID_ARG;
    if (capacity == 0) return NACC_OK;
    const DeviceInfo dev = current_device();
    const long long blocks = (long long)dev.sm_count * 4;
    fill_tail_kernel<<<(int)blocks, kThreads, 0, (cudaStream_t)stream>>>(arr, width, capacity, n_dev, value);
    return launch_status(cudaGetLastError());
}
