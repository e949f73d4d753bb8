// sat.cu -- summed-area table of an occupancy grid, the acceleration structure
// of the marcher's box test (an addition of this library; the paper's method
// (Sec. 2.1) only needs the bitfield itself).
//
// For every grid g (slot x level) of res0 x res1 x res2 cells, the table holds
// one entry per cell corner (x, y, z) in [0, res0] x [0, res1] x [0, res2]:
//     S_g[x][y][z] = #{ occupied cells (i, j, k) of g : i < x, j < y, k < z }
// stored as uint16 modulo 2^16, corners x-major, z fastest, grids one after the
// other. Any box of fewer than 2^16 cells then has its exact count from eight
// entries by inclusion-exclusion in modular arithmetic (the true count is below
// 2^16, so it equals its residue).
//
// Two passes, each staging a slice of the table in shared memory so that every
// global access is a coalesced sweep and every scan runs on chip:
//   1. planes: a block per corner plane x forms the plane's own 2D table
//      P[y][z] = occupied cells (x - 1, j, k) with j < y, k < z: the plane's bits
//      are copied to shared memory in one sweep, each warp takes whole rows
//      (lane l counts four consecutive cells, a warp scan gives the row's
//      prefix), then a running sum along y; plane 0 is zero;
//   2. slabs: a block per (g, y) loads the (x, z) slab of those plane tables and
//      runs the sum along x.
// The running sums are warp scans over columns (a warp per column).
// Four or more grids have enough planes to fill the GPU with a warp per plane
// instead: a lane keeps four running sums along y in registers, then a warp per
// (g, y, z block) runs the sums along x. Planes or slabs too large for shared
// memory take slower global-memory passes.
// A last pass writes the brick summary after the table (see sat_layout): for
// every block of 8^3 cells, whether none or all of its cells are occupied. It is
// small enough for the marcher to keep in shared memory and decide most boxes
// without reading the table.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kSliceThreads = 1024;  // a plane or slab per block: one block per SM for a single grid, so many warps
constexpr int kSliceMax = 20 * 1024;  // uint16 entries of a plane or slab held in shared memory
constexpr int kPlaneWordsMax = 2048;  // bit words of a cell plane held in shared memory

struct SatArgs {
    const uint32_t* bits;
    uint16_t* sat;
    int32_t r0, r1, r2;
    int32_t n_grids;
};

// Bits [b, b + n) (n <= 25) of a word array as the low bits of a word.
__device__ __forceinline__ uint32_t bit_run(const uint32_t* words, int64_t b, int n) {
    const int off = (int)(b & 31);
    const uint64_t w0 = words[b >> 5];
    const uint64_t w1 = off + n > 32 ? (uint64_t)words[(b >> 5) + 1] : 0ull;
    return (uint32_t)((w0 | (w1 << 32)) >> off) & ((1u << n) - 1u);
}

// out[z] = occupied cells among the first z cells of the row starting at bit
// `base` of `words`, z = 0 .. r2. Whole warp.
__device__ __forceinline__ void row_prefix(const uint32_t* words, int64_t base, int r2, uint16_t* out, int lane) {
    if (lane == 0) out[0] = 0;
    uint32_t carry = 0;
    for (int s = 0; s < r2; s += 128) {
        const int z0 = s + 4 * lane;  // this lane's four cells z0 .. z0 + 3
        const int n = z0 < r2 ? min(4, r2 - z0) : 0;
        const uint32_t run = n > 0 ? bit_run(words, base + z0, n) : 0u;
        const uint32_t incl = (uint32_t)warp_incl_scan_int(__popc(run), lane);
        uint32_t c = carry + incl - __popc(run);  // cells before z0
        for (int j = 0; j < n; ++j) {
            c += (run >> j) & 1u;
            out[z0 + j + 1] = (uint16_t)c;
        }
        carry += __shfl_sync(FULL, incl, 31);
    }
}

// In-place running sum (modulo 2^16) along the first axis of an n x m array of
// uint16 in shared memory (row stride m), for every column: a warp per column,
// lane l summing a stretch of ceil(n / 32) consecutive entries, then a warp scan
// of the stretch totals.
__device__ __forceinline__ void column_scan(uint16_t* p, int n, int m, int lane, int warp, int warps) {
    const int per = (n + 31) / 32;
    for (int col = warp; col < m; col += warps) {
        const int y0 = lane * per;
        int s = 0;
        for (int j = 0; j < per; ++j)
            if (y0 + j < n) s += p[(y0 + j) * m + col];
        int run = warp_incl_scan_int(s, lane) - s;
        for (int j = 0; j < per; ++j) {
            if (y0 + j < n) {
                run += p[(y0 + j) * m + col];
                p[(y0 + j) * m + col] = (uint16_t)run;
            }
        }
    }
}

// Pass 1: corner plane x of grid g (block g * (r0 + 1) + x).
__global__ void __launch_bounds__(kSliceThreads) sat_plane_kernel(const SatArgs a) {
    __shared__ uint16_t p[kSliceMax];
    __shared__ uint32_t wbits[kPlaneWordsMax];
    const int64_t plane = blockIdx.x;
    const int x = (int)(plane % (a.r0 + 1));
    const int64_t g = plane / (a.r0 + 1);
    const int ny = a.r1 + 1, nz = a.r2 + 1, n = ny * nz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    uint16_t* out = a.sat + plane * (int64_t)n;
    if (x == 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = 0;
        return;
    }
    // the bits of cell plane x - 1, from the word holding its first bit
    const int64_t first = (g * a.r0 + (x - 1)) * (int64_t)a.r1 * a.r2;
    const int64_t w0 = first >> 5;
    const int nw = (int)(((first + (int64_t)a.r1 * a.r2 + 31) >> 5) - w0);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) wbits[i] = __ldg(a.bits + w0 + i);
    for (int z = threadIdx.x; z < nz; z += blockDim.x) p[z] = 0;  // y = 0
    __syncthreads();
    for (int y = 1 + warp; y < ny; y += warps)
        row_prefix(wbits, (first & 31) + (int64_t)(y - 1) * a.r2, a.r2, p + y * nz, lane);
    __syncthreads();
    column_scan(p, ny, nz, lane, warp, warps);  // running sum along y
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = p[i];
}

// Pass 2: the (x, z) slab of row y of grid g (block g * (r1 + 1) + y).
__global__ void __launch_bounds__(kSliceThreads) sat_slab_kernel(const SatArgs a) {
    __shared__ uint16_t p[kSliceMax];
    const int64_t slab = blockIdx.x;
    const int y = (int)(slab % (a.r1 + 1));
    const int64_t g = slab / (a.r1 + 1);
    const int nx = a.r0 + 1, nz = a.r2 + 1;
    const int64_t plane = (int64_t)(a.r1 + 1) * nz;
    uint16_t* base = a.sat + g * nx * plane + (int64_t)y * nz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const int total = nx * nz;
    for (int i0 = threadIdx.x; i0 < total; i0 += 8 * blockDim.x) {  // eight loads in flight per thread
        uint16_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * blockDim.x;
            const int xx = i / nz;
            v[u] = i < total ? base[xx * plane + (i - xx * nz)] : (uint16_t)0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u * blockDim.x < total) p[i0 + u * blockDim.x] = v[u];
    }
    __syncthreads();
    column_scan(p, nx, nz, lane, warp, warps);  // running sum along x
    __syncthreads();
    for (int xx = warp; xx < nx; xx += warps)
        for (int z = lane; z < nz; z += 32) base[xx * plane + z] = p[xx * nz + z];
}

// Many grids, pass 1: a warp per corner plane (g, x). For each block of 128
// cells along z, lane l takes corners z = zb + 4l + 1 .. zb + 4l + 4: every row's
// 128 bits of the block are read by all lanes (broadcast), realigned to the
// block's first cell by funnel shifts, and a lane's counts are the popcounts of
// the words below its own plus the masked part of its word; running sums along y
// are kept in the lane's registers. Bits before the block (zb > 0) are counted by
// the warp, one word per lane.
__global__ void __launch_bounds__(kThreads) sat_plane_warp_kernel(const SatArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // g (r0 + 1) + x
    if (p >= (int64_t)a.n_grids * (a.r0 + 1)) return;                         // whole warps
    const int x = (int)(p % (a.r0 + 1));
    const int64_t g = p / (a.r0 + 1);
    const int ny = a.r1 + 1, nz = a.r2 + 1;
    uint16_t* out = a.sat + p * (int64_t)ny * nz;
    const int64_t n_words = ((int64_t)a.n_grids * a.r0 * a.r1 * a.r2 + 31) >> 5;
    for (int y = lane; y < ny; y += 32) out[(int64_t)y * nz] = 0;  // z = 0
    const int64_t first = (g * a.r0 + (x - 1)) * (int64_t)a.r1 * a.r2;  // bit of cell (x - 1, 0, 0)
    const int q = lane >> 3, j0 = 4 * (lane & 7);  // the lane's word of the block and first bit in it
    constexpr int kRows = 4;  // rows whose words are loaded together
    for (int zb = 0; zb < a.r2; zb += 128) {
        uint32_t run[4] = {0u, 0u, 0u, 0u};
        for (int y0 = 0; y0 < ny; y0 += kRows) {
            uint32_t w[kRows][5];
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const int y = y0 + u;
                const int64_t k = (first + (int64_t)(y - 1) * a.r2 + zb) >> 5;
                const bool live = y > 0 && y < ny && x > 0;
#pragma unroll
                for (int i = 0; i < 5; ++i) w[u][i] = live && k + i < n_words ? __ldg(a.bits + k + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const int y = y0 + u;
                if (y >= ny) break;  // uniform
                if (y > 0 && x > 0) {
                    const int64_t row = first + (int64_t)(y - 1) * a.r2;
                    uint32_t before = 0;  // bits [row, row + zb)
                    if (zb > 0) {
                        for (int64_t w0 = row >> 5; (w0 << 5) < row + zb; w0 += 32) {
                            const int64_t k = w0 + lane, lo = k << 5;
                            if (lo < row + zb) {
                                uint32_t m = k < n_words ? __ldg(a.bits + k) : 0u;
                                if (lo < row) m &= ~0u << (int)(row - lo);
                                if (lo + 32 > row + zb) m &= (1u << (int)(row + zb - lo)) - 1u;
                                before += __popc(m);
                            }
                        }
                        for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(FULL, before, o);
                    }
                    const unsigned off = (unsigned)((row + zb) & 31);
                    uint32_t v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = __funnelshift_r(w[u][i], w[u][i + 1], off);
                    const uint32_t c1 = __popc(v[0]), c2 = c1 + __popc(v[1]), c3 = c2 + __popc(v[2]);
                    const uint32_t mine = q == 0 ? v[0] : q == 1 ? v[1] : q == 2 ? v[2] : v[3];
                    const uint32_t below = before + (q == 0 ? 0u : q == 1 ? c1 : q == 2 ? c2 : c3);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int nb = j0 + i + 1;  // bits of the lane's word below its corner
                        run[i] += below + __popc(mine & (nb >= 32 ? ~0u : (1u << nb) - 1u));
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int z = zb + 4 * lane + i + 1;
                    if (z <= a.r2) out[(int64_t)y * nz + z] = (uint16_t)run[i];
                }
            }
        }
    }
}

// Many grids, pass 2: a warp per (g, y, block of 128 z); lane l runs the sums
// along x of corners z = zb + 4l + 1 .. zb + 4l + 4, eight planes loaded ahead.
__global__ void __launch_bounds__(kThreads) sat_xsum_warp_kernel(const SatArgs a) {
    const int lane = threadIdx.x & 31;
    const int zblocks = (a.r2 + 127) / 128;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)a.n_grids * (a.r1 + 1) * zblocks) return;  // whole warps
    const int zb = 128 * (int)(w % zblocks);
    const int64_t gy = w / zblocks;  // g (r1 + 1) + y
    const int y = (int)(gy % (a.r1 + 1));
    const int64_t g = gy / (a.r1 + 1);
    const int nx = a.r0 + 1, nz = a.r2 + 1;
    const int64_t plane = (int64_t)(a.r1 + 1) * nz;
    const int nv = min(4, a.r2 - (zb + 4 * lane));  // the lane's corners inside the grid (may be <= 0)
    uint16_t* col = a.sat + g * nx * plane + (int64_t)y * nz + (nv > 0 ? zb + 4 * lane + 1 : 0);
    uint32_t run[4] = {0u, 0u, 0u, 0u};
    constexpr int kPlanes = 8;  // planes loaded ahead
    int x = 0;
    for (; x + kPlanes <= nx; x += kPlanes) {
        uint32_t v[kPlanes][4];
#pragma unroll
        for (int u = 0; u < kPlanes; ++u)
#pragma unroll
            for (int i = 0; i < 4; ++i) v[u][i] = i < nv ? col[(int64_t)(x + u) * plane + i] : 0u;
#pragma unroll
        for (int u = 0; u < kPlanes; ++u)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                run[i] += v[u][i];
                if (i < nv) col[(int64_t)(x + u) * plane + i] = (uint16_t)run[i];
            }
    }
    for (; x < nx; ++x) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < nv) {
                run[i] += col[(int64_t)x * plane + i];
                col[(int64_t)x * plane + i] = (uint16_t)run[i];
            }
        }
    }
}

// Fallback pass 1: rows straight from global memory (one warp per corner row).
__global__ void __launch_bounds__(32) sat_rows_kernel(const SatArgs a) {
    const int64_t row = blockIdx.x;  // (g * (r0 + 1) + x) * (r1 + 1) + y
    const int y = (int)(row % (a.r1 + 1));
    const int64_t gx = row / (a.r1 + 1);
    const int x = (int)(gx % (a.r0 + 1));
    const int64_t g = gx / (a.r0 + 1);
    uint16_t* out = a.sat + row * (a.r2 + 1);
    if (x == 0 || y == 0) {
        for (int z = threadIdx.x; z <= a.r2; z += 32) out[z] = 0;
        return;
    }
    row_prefix(a.bits, ((g * a.r0 + (x - 1)) * (int64_t)a.r1 + (y - 1)) * a.r2, a.r2, out, threadIdx.x);
}

// Fallback running sums along y (AXIS 1) or x (AXIS 0), one thread per line,
// consecutive threads on consecutive z, eight entries loaded ahead.
template <int AXIS>
__global__ void __launch_bounds__(kThreads) sat_sum_kernel(const SatArgs a) {
    const int64_t lines = (int64_t)a.n_grids * (AXIS == 1 ? (a.r0 + 1) : (a.r1 + 1)) * (a.r2 + 1);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= lines) return;
    const int z = (int)(t % (a.r2 + 1));
    const int64_t rest = t / (a.r2 + 1);
    const int64_t plane = (int64_t)(a.r1 + 1) * (a.r2 + 1);
    int64_t start, step;
    int n;
    if (AXIS == 1) {  // rest = g * (r0 + 1) + x
        start = rest * plane + z;
        step = a.r2 + 1;
        n = a.r1 + 1;
    } else {  // rest = g * (r1 + 1) + y
        start = rest / (a.r1 + 1) * (a.r0 + 1) * plane + (rest % (a.r1 + 1)) * (a.r2 + 1) + z;
        step = plane;
        n = a.r0 + 1;
    }
    uint16_t* q = a.sat + start;
    uint32_t s = 0;
    int i = 0;
    for (; i + 8 <= n; i += 8) {
        uint16_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = q[(i + u) * step];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            s += v[u];
            q[(i + u) * step] = (uint16_t)s;
        }
    }
    for (; i < n; ++i) {
        s += q[i * step];
        q[i * step] = (uint16_t)s;
    }
}


// Brick summary (layout: sat_layout): a thread per brick forms its 2-bit state
// from its box count in the finished table (a brick holds at most 512 cells, so
// the modular count is exact); groups of 8 lanes pack their states into one entry.
__global__ void __launch_bounds__(kThreads) brick_summary_kernel(const SatArgs a, uint16_t* out, int nb0, int nb1,
                                                                int nb2, int per_grid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (grid, brick slot)
    const long long slots = (long long)a.n_grids * per_grid * 8;
    const int g = (int)(i / ((long long)per_grid * 8)), b = (int)(i % ((long long)per_grid * 8));
    unsigned v = 0u;
    if (i < slots && b < nb0 * nb1 * nb2) {
        const unsigned sy = (unsigned)(a.r2 + 1), sx = (unsigned)(a.r1 + 1) * sy;
        const uint16_t* t = a.sat + (size_t)g * sx * (unsigned)(a.r0 + 1);
        const int bz = b % nb2, by = (b / nb2) % nb1, bx = b / (nb1 * nb2);
        const int x0 = 8 * bx, y0 = 8 * by, z0 = 8 * bz;
        const int x1 = min(x0 + 8, a.r0), y1 = min(y0 + 8, a.r1), z1 = min(z0 + 8, a.r2);
        const unsigned xa = x0 * sx, xb = x1 * sx, ya = y0 * sy, yb = y1 * sy;
        const unsigned cnt = ((unsigned)t[xb + yb + z1] - (unsigned)t[xa + yb + z1] - (unsigned)t[xb + ya + z1] -
                              (unsigned)t[xb + yb + z0] + (unsigned)t[xa + ya + z1] + (unsigned)t[xa + yb + z0] +
                              (unsigned)t[xb + ya + z0] - (unsigned)t[xa + ya + z0]) &
                             0xffffu;
        const unsigned vol = (unsigned)((x1 - x0) * (y1 - y0) * (z1 - z0));
        v = (cnt == 0u ? 1u : 0u) | (cnt == vol ? 2u : 0u);
    }
    // slots are whole warps' worth of entries (8 per entry, entries never straddle warps)
    v <<= 2 * (threadIdx.x & 7);
    v |= __shfl_xor_sync(FULL, v, 1);
    v |= __shfl_xor_sync(FULL, v, 2);
    v |= __shfl_xor_sync(FULL, v, 4);
    if ((threadIdx.x & 7) == 0 && i < slots) out[i >> 3] = (uint16_t)v;
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_grid_sat_bytes(const nacc_grid* grid) {
    if (!grid || grid->n_levels < 1 || grid->n_slots < 1) return 0;
    for (int k = 0; k < 3; ++k)
        if (grid->res[k] < 1) return 0;
    return sat_layout((long long)grid->n_slots * grid->n_levels, grid->res[0], grid->res[1], grid->res[2])
               .total_entries * sizeof(uint16_t);
}

extern "C" int nacc_build_grid_sat(const nacc_grid* grid, uint16_t* sat, void* stream) {
    if (!grid || !sat || !grid->bits) return NACC_ERR_INVALID_ARG;
    if (grid->n_levels < 1 || grid->n_levels > NACC_MAX_LEVELS || grid->n_slots < 1) return NACC_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (grid->res[k] < 1 || grid->res[k] > (1 << 22)) return NACC_ERR_INVALID_ARG;
    const long long grids = (long long)grid->n_slots * grid->n_levels;
    const long long r0 = grid->res[0], r1 = grid->res[1], r2 = grid->res[2];
    const long long corners = grids * (r0 + 1) * (r1 + 1) * (r2 + 1);
    if (corners >= (1LL << 31) || grids * r0 * r1 * r2 >= (1LL << 31)) return NACC_ERR_INVALID_ARG;
    SatArgs a{grid->bits, sat, grid->res[0], grid->res[1], grid->res[2], (int32_t)grids};
    cudaStream_t st = (cudaStream_t)stream;
    const long long planes = grids * (r0 + 1);
    // up to three grids: a block per plane and slab (few blocks, so each short);
    // more grids: a warp per plane, then a warp per row of z blocks
    const bool many = grids >= 4;
    if (many) {
        const long long zblocks = (r2 + 127) / 128, w1 = planes, w2 = grids * (r1 + 1) * zblocks;
        sat_plane_warp_kernel<<<(unsigned)((w1 * 32 + kThreads - 1) / kThreads), kThreads, 0, st>>>(a);
        sat_xsum_warp_kernel<<<(unsigned)((w2 * 32 + kThreads - 1) / kThreads), kThreads, 0, st>>>(a);
    } else if ((r1 + 1) * (r2 + 1) <= kSliceMax && r1 * r2 / 32 + 2 <= kPlaneWordsMax) {
        // a plane's bits span at most r1 r2 / 32 + 2 words
        sat_plane_kernel<<<(unsigned)planes, kSliceThreads, 0, st>>>(a);
    } else {
        sat_rows_kernel<<<(unsigned)(planes * (r1 + 1)), 32, 0, st>>>(a);
        const long long ly = planes * (r2 + 1);
        sat_sum_kernel<1><<<(unsigned)((ly + kThreads - 1) / kThreads), kThreads, 0, st>>>(a);
    }
    if (!many) {
        if ((r0 + 1) * (r2 + 1) <= kSliceMax) {
            sat_slab_kernel<<<(unsigned)(grids * (r1 + 1)), kSliceThreads, 0, st>>>(a);
        } else {
            const long long lx = grids * (r1 + 1) * (r2 + 1);
            sat_sum_kernel<0><<<(unsigned)((lx + kThreads - 1) / kThreads), kThreads, 0, st>>>(a);
        }
    }
    // the brick summary, from the finished table
    const SatLayout L = sat_layout(grids, grid->res[0], grid->res[1], grid->res[2]);
    const long long slots = grids * (long long)L.per_grid * 8;
    brick_summary_kernel<<<(unsigned)((slots + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        a, sat + L.summary_offset, L.nb0, L.nb1, L.nb2, (int)L.per_grid);
    return launch_status(cudaGetLastError());
}
