// grid.cu -- occupancy-grid update (NerfAcc, arXiv 2210.04847, Sec. 2.1: the
// binary grid is cached and updated during training, following Instant-NGP's
// Appendix E.2).
//
//   ema <- decay * ema                 (every cell)
//   ema[c] <- max(ema[c], sigma_s)     (every sample s in cell c)
//   bits  = ema > thre
//
// Two launches, 8.125 bytes of HBM traffic per cell plus the samples:
//   1. decay_pack: one pass over the float32 grid, decays in place and writes
//      the bit words of the decayed values (__ballot_sync gives a word per 32
//      cells);
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

__global__ void __launch_bounds__(kThreads) scatter_max_kernel(float* ema, uint32_t* bits, int64_t n_cells,
                                                               const int32_t* cells, const float* sigmas,
                                                               int64_t n, float thre, int32_t* d_status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const int c = cells[s];
        const float v = sigmas[s];
        if (c < 0 || (int64_t)c >= n_cells) {
            raise_status(d_status, NACC_STATUS_BAD_INDEX);
            continue;
        }
        if (!(v > 0.0f)) continue;  // NaN, zero and negative values never raise a cell (ema >= 0)
        atomicMax(reinterpret_cast<int*>(ema) + c, __float_as_int(v));
        if (v > thre) atomicOr(bits + (c >> 5), 1u << (c & 31));
    }
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_update_occupancy_grid(float* ema, uint32_t* bits, int64_t n_cells, const int32_t* cells,
                                          const float* sigmas, int64_t n_samples, float decay, float thre,
                                          int32_t* d_status, void* stream) {
    if (n_cells < 0 || n_samples < 0 || n_cells >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    if (n_cells > 0 && (!ema || !bits)) return NACC_ERR_INVALID_ARG;
    if (n_samples > 0 && (!cells || !sigmas)) return NACC_ERR_INVALID_ARG;
    if (decay != decay || thre != thre) return NACC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const DeviceInfo dev = current_device();
    if (n_cells > 0) {
        const int64_t words = (n_cells + 31) >> 5;
        int64_t blocks = (words * 32 + kThreads - 1) / kThreads;
        const int64_t cap = (int64_t)dev.sm_count * 8;
        if (blocks > cap) blocks = cap;
        decay_pack_kernel<<<(int)blocks, kThreads, 0, st>>>(ema, bits, n_cells, decay, thre);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return NACC_ERR_CUDA;
    }
    if (n_samples > 0) {
        int64_t blocks = (n_samples + kThreads - 1) / kThreads;
        const int64_t cap = (int64_t)dev.sm_count * 8;
        if (blocks > cap) blocks = cap;
        scatter_max_kernel<<<(int)blocks, kThreads, 0, st>>>(ema, bits, n_cells, cells, sigmas, n_samples, thre,
                                                             d_status);
    }
    return launch_status(cudaGetLastError());
}
