// grid.cu -- occupancy-grid update (NerfAcc, arXiv 2210.04847, Sec. 2.1: the
// binary grid is cached and updated during training, following Instant-NGP's
// Appendix E.2).
//
//   ema <- decay * ema                 (every cell)
//   ema[c] <- max(ema[c], sigma_s)     (every sample s in cell c)
//   bits  = ema > thre
//
// The update's inputs come from nacc_sample_grid_cells (uniform random cells, a
// uniform point in each, from a counter-based generator) and the caller's field.
//
// Two launches, 8.125 bytes of HBM traffic per cell plus the samples:
//   1. decay_pack: one pass over the float32 grid, decays in place and writes
//      the bit words of the decayed values (four cells per thread with 16-byte
//      accesses over whole 128-cell steps of an aligned grid; elsewhere one cell
//      per thread, __ballot_sync giving a word per 32 cells);
//   2. scatter: per sample, atomicMax on the float bits (valid because every
//      value is >= 0, so the int order is the float order) and, when the sample
//      alone passes the threshold, atomicOr of its bit. Since max only grows,
//      bit(max(decay*e, s)) = bit(decay*e) OR bit(s): the words equal the
//      threshold of the final grid, independent of sample order.
#include <math.h>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) decay_pack_kernel(float* ema, uint32_t* bits, int64_t n_cells,
                                                              float decay, float thre) {
    const int lane = threadIdx.x & 31;
    const int64_t n_words = (n_cells + 31) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_words; w += warps) {
        const int64_t c = (w << 5) + lane;
        bool on = false;
        if (c < n_cells) {
            const float e = __fmul_rn(decay, ema[c]);
            ema[c] = e;
            on = e > thre;
        }
        const unsigned m = __ballot_sync(FULL, on);
        if (lane == 0) bits[w] = m;
    }
}

// The same pass, four cells per thread (one 16-byte load and store) over whole
// warp steps of 128 cells, two steps in flight per thread: cell 4 lane + j of a
// step is bit 4 (lane % 8) + j of the step's word lane / 8, so each word gathers
// the four-bit groups of eight lanes by three shuffles.
__global__ void __launch_bounds__(kThreads) decay_pack4_kernel(float4* __restrict__ ema4,
                                                               uint32_t* __restrict__ bits, int64_t n_steps,
                                                               float decay, float thre) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_steps; w += 2 * warps) {
        const int64_t w2 = w + warps;
        const bool two = w2 < n_steps;
        float4 v = ema4[(w << 5) + lane];
        float4 u = two ? ema4[(w2 << 5) + lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4& q = h ? u : v;
            if (h && !two) break;
            q.x = __fmul_rn(decay, q.x);
            q.y = __fmul_rn(decay, q.y);
            q.z = __fmul_rn(decay, q.z);
            q.w = __fmul_rn(decay, q.w);
            const int64_t step = h ? w2 : w;
            ema4[(step << 5) + lane] = q;
            unsigned word = ((unsigned)(q.x > thre) | ((unsigned)(q.y > thre) << 1) | ((unsigned)(q.z > thre) << 2) |
                             ((unsigned)(q.w > thre) << 3))
                            << (4 * (lane & 7));
            word |= __shfl_xor_sync(FULL, word, 1);
            word |= __shfl_xor_sync(FULL, word, 2);
            word |= __shfl_xor_sync(FULL, word, 4);
            if ((lane & 7) == 0) bits[(step << 2) + (lane >> 3)] = word;
        }
    }
}

__global__ void __launch_bounds__(kThreads) scatter_max_kernel(float* ema, uint32_t* bits, int64_t n_cells,
                                                               const int32_t* __restrict__ cells,
                                                               const float* __restrict__ sigmas, int64_t n, float thre,
                                                               int32_t* d_status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const int c = __ldg(cells + s);
        const float v = __ldg(sigmas + s);
        if (c < 0 || (int64_t)c >= n_cells) {
            raise_status(d_status, NACC_STATUS_BAD_INDEX);
            continue;
        }
        if (!(v > 0.0f)) continue;  // NaN, zero and negative values never raise a cell (ema >= 0)
        atomicMax(reinterpret_cast<int*>(ema) + c, __float_as_int(v));
        if (v > thre) atomicOr(bits + (c >> 5), 1u << (c & 31));
    }
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014; the 64-bit output mix of Vigna's splitmix64):
// draw i (from 0) of stream k of seed s is mix(key + (i + 1) * gamma) with
// key = mix(s) + k * kStreamMul. Counter-based: any draw is computed directly.
constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kStreamMul = 0xD1B54A32D192ED03ull;

__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

struct SampleArgs {
    unsigned long long key_cells, key_jitter;
    long long n;
    int res[3];
    int n_levels, n_sl;             // levels, levels * slots
    int contraction;                // points drawn in contracted space, mapped back to the world
    float cc[3], hh[3];             // contraction: box centre and half size
    float lo[NACC_MAX_LEVELS][3];   // level boxes in float32, formed as the marcher forms them
    float cs[NACC_MAX_LEVELS][3];   // cell size (hi - lo) / res of each level
    int32_t* cells;
    float* xyz;
};

// Sample i: draws 2i, 2i+1 of the cell stream give the cell's coordinates by
// multiply-shift range reduction of their 32-bit halves, (h * extent) >> 32:
// x, y from the first draw's high and low halves, z and the (slot, level)
// index sl from the second's; draws 2i, 2i+1 of the jitter stream give three
// 24-bit fields (bits 40.., 16.. of the first, 40.. of the second) times 2^-24.
// point_a = lo_a + (i_a + jitter_a) * cs_a in float32, each operation rounded.
__global__ void __launch_bounds__(kThreads) sample_cells_kernel(const SampleArgs a) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += stride) {
        const unsigned long long c0 = mix64(a.key_cells + (unsigned long long)(2 * s + 1) * kGamma);
        const unsigned long long c1 = mix64(a.key_cells + (unsigned long long)(2 * s + 2) * kGamma);
        // (h * extent) >> 32 of a 32-bit half h: the high word of the 32 x 32-bit product
        const unsigned ix = __umulhi((unsigned)(c0 >> 32), (unsigned)a.res[0]);
        const unsigned iy = __umulhi((unsigned)c0, (unsigned)a.res[1]);
        const unsigned iz = __umulhi((unsigned)(c1 >> 32), (unsigned)a.res[2]);
        const unsigned sl = __umulhi((unsigned)c1, (unsigned)a.n_sl);
        a.cells[s] = (int32_t)(((sl * (unsigned)a.res[0] + ix) * (unsigned)a.res[1] + iy) * (unsigned)a.res[2] + iz);
        const int lvl = (int)(sl % (unsigned)a.n_levels);
        const unsigned long long q0 = mix64(a.key_jitter + (unsigned long long)(2 * s + 1) * kGamma);
        const unsigned long long q1 = mix64(a.key_jitter + (unsigned long long)(2 * s + 2) * kGamma);
        const float j[3] = {__uint2float_rn((unsigned)(q0 >> 40)) * (1.0f / 16777216.0f),
                            __uint2float_rn((unsigned)((q0 >> 16) & 0xFFFFFFull)) * (1.0f / 16777216.0f),
                            __uint2float_rn((unsigned)(q1 >> 40)) * (1.0f / 16777216.0f)};
        const unsigned idx[3] = {ix, iy, iz};
        float p[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float lo = a.lo[0][k], cs = a.cs[0][k];
            for (int l = 1; l < a.n_levels; ++l)
                if (l == lvl) {
                    lo = a.lo[l][k];
                    cs = a.cs[l][k];
                }
            p[k] = __fadd_rn(lo, __fmul_rn(__fadd_rn(__uint2float_rn(idx[k]), j[k]), cs));
        }
        if (a.contraction) {
            // p is in contracted space [-2, 2]^3: back to the world, x_c / ((2 - r) r)
            // outside the unit ball, then c + h x_n; unreachable points (r >= 2) are NaN
            const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(p[0], p[0]), __fmul_rn(p[1], p[1])), __fmul_rn(p[2], p[2]));
            float sc = 1.0f;
            if (!(r2 <= 1.0f)) {
                const float r = __fsqrt_rn(r2);
                sc = r < 2.0f ? __frcp_rn(__fmul_rn(__fsub_rn(2.0f, r), r)) : __int_as_float(0x7fc00000);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] = __fadd_rn(a.cc[k], __fmul_rn(a.hh[k], __fmul_rn(p[k], sc)));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) a.xyz[3 * s + k] = p[k];
    }
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_sample_grid_cells(uint64_t seed, uint64_t stream, int64_t n, const nacc_grid* grid,
                                      int32_t* cells, float* xyz, void* cuda_stream) {
    if (n < 0 || !grid) return NACC_ERR_INVALID_ARG;
    if (grid->n_levels < 1 || grid->n_levels > NACC_MAX_LEVELS || grid->n_slots < 1) return NACC_ERR_INVALID_ARG;
    if (grid->contraction != 0 && (grid->contraction != 1 || grid->n_levels != 1)) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (grid->res[k] < 1 || !(grid->aabb[k] < grid->aabb[3 + k])) return NACC_ERR_INVALID_ARG;
    const long long n_cells =
        (long long)grid->res[0] * grid->res[1] * grid->res[2] * grid->n_levels * grid->n_slots;
    if (n_cells >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    if (n == 0) return NACC_OK;
    if (!cells || !xyz) return NACC_ERR_INVALID_ARG;
    SampleArgs a;
    a.key_cells = mix64(seed) + stream * kStreamMul;
    a.key_jitter = mix64(seed) + (stream + 1) * kStreamMul;
    a.n = n;
    a.n_levels = grid->n_levels;
    a.n_sl = grid->n_levels * grid->n_slots;
    a.contraction = grid->contraction;
    for (int k = 0; k < 3; ++k) {
        a.res[k] = grid->res[k];
        // level l: the level-0 box scaled by 2^l about its centre, in float32
        // (contraction: one level spanning [-2, 2] in contracted space)
        const float lo = grid->contraction ? -2.0f : grid->aabb[k];
        const float hi = grid->contraction ? 2.0f : grid->aabb[3 + k];
        const float c = (lo + hi) * 0.5f, h = (hi - lo) * 0.5f;
        a.cc[k] = (grid->aabb[k] + grid->aabb[3 + k]) * 0.5f;
        a.hh[k] = (grid->aabb[3 + k] - grid->aabb[k]) * 0.5f;
        for (int l = 0; l < NACC_MAX_LEVELS; ++l) {
            float llo = lo, lhi = hi;
            if (l > 0) {
                const float hl = h * ldexpf(1.0f, l);
                llo = c - hl;
                lhi = c + hl;
            }
            a.lo[l][k] = llo;
            a.cs[l][k] = (lhi - llo) / (float)grid->res[k];
        }
    }
    a.cells = cells;
    a.xyz = xyz;
    const DeviceInfo dev = current_device();
    long long blocks = (n + kThreads - 1) / kThreads;
    const long long cap = (long long)dev.sm_count * 8;
    if (blocks > cap) blocks = cap;
    sample_cells_kernel<<<(int)blocks, kThreads, 0, (cudaStream_t)cuda_stream>>>(a);
    return launch_status(cudaGetLastError());
}

extern "C" float nacc_density_threshold(float alpha_thre, float dt) {
    // 1 - exp(-sigma dt) > alpha  <=>  sigma > -ln(1 - alpha) / dt  (dt > 0), in
    // double, rounded once to the float32 of the grid's comparison
    if (!(alpha_thre >= 0.0f && alpha_thre < 1.0f) || !(dt > 0.0f) || !(dt < INFINITY)) return NAN;
    return (float)(-log1p(-(double)alpha_thre) / (double)dt);
}

extern "C" int nacc_update_occupancy_grid(float* ema, uint32_t* bits, int64_t n_cells, const int32_t* cells,
                                          const float* sigmas, int64_t n_samples, float decay, float thre,
                                          float alpha_step, int32_t* d_status, void* stream) {
    if (n_cells < 0 || n_samples < 0 || n_cells >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    if (n_cells > 0 && (!ema || !bits)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!cells || !sigmas)) return NACC_ERR_INVALID_ARG;
    if (decay != decay || thre != thre || alpha_step != alpha_step || alpha_step < 0.0f) return NACC_ERR_INVALID_ARG;
    if (alpha_step > 0.0f) {  // thre is the opacity threshold of a step of length alpha_step
        thre = nacc_density_threshold(thre, alpha_step);
        if (thre != thre) return NACC_ERR_INVALID_ARG;
    }
    if (n_cells == 0 && n_samples == 0) return NACC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const DeviceInfo dev = current_device();
    if (n_cells > 0) {
        const int64_t cap = (int64_t)dev.sm_count * 8;
        // whole 128-cell steps four cells per thread when the state is 16-byte aligned,
        // the rest (and unaligned states) one cell per thread
        const int64_t steps = (((uintptr_t)ema & 15u) == 0) ? n_cells >> 7 : 0;
        if (steps > 0) {
            int64_t blocks = (steps * 32 + kThreads - 1) / kThreads;
            if (blocks > cap) blocks = cap;
            decay_pack4_kernel<<<(int)blocks, kThreads, 0, st>>>(reinterpret_cast<float4*>(ema), bits, steps, decay,
                                                                  thre);
        }
        const int64_t done = steps << 7;
        if (done < n_cells) {
            const int64_t words = ((n_cells - done) + 31) >> 5;
            int64_t blocks = (words * 32 + kThreads - 1) / kThreads;
            if (blocks > cap) blocks = cap;
            decay_pack_kernel<<<(int)blocks, kThreads, 0, st>>>(ema + done, bits + (done >> 5), n_cells - done,
                                                                 decay, thre);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return NACC_ERR_CUDA;
    }
    if (n_samples > 0) {
        // one sample per thread (up to 2^31 - 1 blocks): every thread's loads and
        // fire-and-forget atomics are in flight at once; the latency of the random
        // updates, not the issue rate, bounds this pass
        int64_t blocks = (n_samples + kThreads - 1) / kThreads;
        if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
        scatter_max_kernel<<<(int)blocks, kThreads, 0, st>>>(ema, bits, n_cells, cells, sigmas, n_samples, thre,
                                                             d_status);
    }
    return launch_status(cudaGetLastError());
}
