// nacc_internal.cuh -- device helpers shared by the CUDA kernels of the library:
// warp scans, status reporting, the bounded decoupled look-back used by the
// single-pass compaction kernels, and host-side launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nacc.h"

namespace nacc {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// status
// ---------------------------------------------------------------------------

__device__ __forceinline__ void raise_status(int32_t* d_status, int bits) {
    if (d_status) atomicOr(d_status, bits);
}

// ---------------------------------------------------------------------------
// warp scans (float32 and int)
// ---------------------------------------------------------------------------

// Inclusive prefix sum over the 32 lanes (Hillis-Steele, 5 shuffle steps).
__device__ __forceinline__ float warp_incl_scan(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v = v + n;
    }
    return v;
}

// Inclusive suffix sum (lane i gets sum over lanes i..31).
__device__ __forceinline__ float warp_incl_suffix(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float n = __shfl_down_sync(FULL, v, o);
        if (lane + o < 32) v = v + n;
    }
    return v;
}

__device__ __forceinline__ int warp_incl_scan_int(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// decoupled look-back (single-pass scan over tiles taken in ticket order)
// ---------------------------------------------------------------------------
//
// Tile j publishes one 64-bit word: flag in bits 62..63 (1 = aggregate of the
// tile alone, 2 = inclusive prefix through the tile), value in bits 0..61.
// Tiles are numbered by an atomic ticket taken when a warp starts work on
// them, so every tile a warp waits for is held by a warp that is already
// running and publishes its aggregate without waiting: the wait always ends.
// It is still bounded: after spin_limit polls (2^22 by default, about a second
// with the back-off below) the warp reports NACC_STATUS_TIMEOUT, stops waiting,
// and publishes a (too small) prefix so that no other warp waits on it either.
// Every prefix is then at most the true one, so every store stays below the
// true total.
//
// Two test hooks (nacc_test_hook_set) reach these waits: the poll budget, and a
// switch under which tile 0 never publishes its prefix, so that every wait that
// reaches it runs out. A test uses them to check the timeout path on the GPU
// without any fault, trap or unbounded loop.

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

struct LookbackHooks {
    unsigned long long first_flag;  // flag tile 0 publishes: kFlagInc, or 0 ("pending") to withhold it (test only)
    int spin_limit;                 // polls before a wait gives up (default kSpinLimit)
    int overstate_stage;            // staged render kernels: first chunk announces 16 bytes too many (test only)
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Publishes a tile's aggregate (tile 0: its inclusive prefix). Never waits.
__device__ __forceinline__ void publish_aggregate(unsigned long long* status, int tile,
                                                  unsigned long long aggregate, int lane,
                                                  const LookbackHooks& hooks) {
    // (a branch around the store instead of the flag value costs the pruning
    // kernel hundreds of bytes of register spills under its 6-blocks cap)
    if (lane == 0) st_relaxed_u64(&status[tile], (tile == 0 ? hooks.first_flag : kFlagAgg) | (aggregate & kValMask));
}

// Called by one full warp after publish_aggregate(tile). Returns the exclusive
// prefix of the tile (sum of the aggregates of tiles 0..tile-1) and publishes
// its inclusive prefix. A warp may publish further tiles' aggregates before
// resolving an earlier one: every tile it waits for has a lower ticket, and
// the warp holding that ticket publishes its aggregate before it waits.
__device__ __forceinline__ unsigned long long resolve_prefix(unsigned long long* status, int tile,
                                                             unsigned long long aggregate, int lane,
                                                             int32_t* d_status, const LookbackHooks& hooks) {
    const int spin_limit = hooks.spin_limit;
    if (tile == 0) return 0ull;
    unsigned long long excl = 0;
    int base = tile - 1;
    int spins = 0;
    bool timed_out = false;
    while (true) {
        int j = base - lane;
        unsigned long long s = j >= 0 ? ld_relaxed_u64(&status[j]) : (kFlagInc | 0ull);
        unsigned pending = __ballot_sync(FULL, (s >> 62) == 0ull);
        while (pending) {
            if (++spins > spin_limit) {
                timed_out = true;
                break;
            }
            __nanosleep(spins < 64 ? 32 : 256);
            if ((pending >> lane) & 1u) s = ld_relaxed_u64(&status[j]);
            pending = __ballot_sync(FULL, (s >> 62) == 0ull);
        }
        if (timed_out) break;
        unsigned inc = __ballot_sync(FULL, (s >> 62) == 2ull);
        unsigned long long v = s & kValMask;
        if (inc) {
            int first = __ffs(inc) - 1;  // nearest predecessor holding an inclusive prefix
            if (lane > first) v = 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            excl += v;
            break;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        excl += v;
        base -= 32;
    }
    if (timed_out && lane == 0) raise_status(d_status, NACC_STATUS_TIMEOUT);
    if (lane == 0) st_relaxed_u64(&status[tile], kFlagInc | ((excl + aggregate) & kValMask));
    return excl;
}


// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

struct DeviceInfo {
    int device;
    int sm_count;
};

DeviceInfo current_device();

// Current value of a tuning knob (NACC_TUNE_*), the library default unless set.
int tune_get(int knob);

// The look-back settings in force (test hooks; defaults unless a test set them).
LookbackHooks lookback_hooks();

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Layout of a grid's summed-area table buffer (nacc_build_grid_sat): the table's
// uint16 corner entries for every grid, then, from the first 16-byte boundary,
// the brick summary: 2 bits per brick of 8^3 cells (bit 0: no cell occupied,
// bit 1: every in-grid cell occupied), 8 bricks per uint16 entry, bricks
// x-major and z fastest, ceil(nb0 nb1 nb2 / 8) entries per grid, nb_k = ceil(res_k / 8).
struct SatLayout {
    size_t table_entries;   // uint16 corner entries over all grids
    size_t summary_offset;  // uint16 entries before the brick summary
    int nb0, nb1, nb2;      // bricks per axis
    size_t per_grid;        // summary entries per grid
    size_t total_entries;   // uint16 entries of the whole buffer
};

inline SatLayout sat_layout(long long grids, int r0, int r1, int r2) {
    SatLayout L;
    L.table_entries = (size_t)grids * (size_t)(r0 + 1) * (size_t)(r1 + 1) * (size_t)(r2 + 1);
    L.summary_offset = align_up(L.table_entries, 8);
    L.nb0 = (r0 + 7) >> 3;
    L.nb1 = (r1 + 7) >> 3;
    L.nb2 = (r2 + 7) >> 3;
    L.per_grid = ((size_t)L.nb0 * L.nb1 * L.nb2 + 7) >> 3;
    L.total_entries = L.summary_offset + (size_t)grids * L.per_grid;
    return L;
}

inline int launch_status(cudaError_t e) { return e == cudaSuccess ? NACC_OK : NACC_ERR_CUDA; }

}  // namespace nacc
