// march.cu -- occupancy-grid ray marching with empty-space skipping (NerfAcc,
// arXiv 2210.04847, Sec. 2.1 "Ray Marching" and "GPU Memory Efficiency":
// samples are emitted only in occupied cells, pruned while marching).
//
// Compiled with -fmad=false; every float operation on the sample path is an
// explicitly rounded __f*_rn intrinsic so that the emitted set is
// bit-reproducible (it is an integer result decided by float arithmetic).
//
// Design (single pass, no count/fill split):
//   * Every warp works on its own tiles of consecutive rays, taken from a
//     global atomic ticket (tile order = ticket order). No block-wide barrier
//     is ever taken: each warp keeps its tile's ballot words in a private
//     slice of shared memory.
//   * Uniform steps: the warp walks one ray at a time, lane j evaluating
//     lattice point 32c + j (the lattice is closed-form, t_k = near + k*dt);
//     the occupancy test of the 32 midpoints becomes one __ballot_sync word and
//     __popc gives the count. Lane i of the warp keeps ray i's count, chunk
//     count and [near, far]. On a one-level grid each chunk's bitfield word is
//     loaded one chunk ahead, so that load overlaps the ballot of the chunk
//     before it.
//   * Cone steps (t_{k+1} = t_k + clamp(t_k*cone, dt_min, dt_max)): the
//     lattice is a sequential float32 recurrence that depends only on its start.
//     Every ray that starts inside the outermost box starts at near_plane, so a
//     one-thread prologue writes that shared lattice once per call into the
//     workspace and the warps read t_k from it, lane-parallel, exactly as for
//     uniform steps (each block first copies it into shared memory when it
//     fits). A ray with another start has lane 0 extend its own recurrence 32
//     steps at a time into the warp's shared memory.
//   * The tile's total becomes its global offset through a bounded decoupled
//     look-back run by the warp itself; the warp then re-expands the ballot
//     words into compacted, coalesced stores of (t_start, t_end, ray).
#include "march_common.cuh"

namespace nacc {
namespace {

// The shared cone lattice t_0 .. t_max_steps as the block reads it: its copy in
// the block's shared memory when it fits (kConeSmemMax entries), else the table in
// global memory. Set by the kernel before any walk (cone steps only).
constexpr int kConeSmemMax = 8193;
__shared__ const float* s_cone;

__device__ __forceinline__ float cone_t(const MarchArgs& a, int k) { return s_cone[min(k, a.max_steps)]; }

// The contracted walk reads the global table through the read-only path (its
// blocks keep no copy: that measured slower there).
template <bool GLOBAL>
__device__ __forceinline__ float lattice_t(const MarchArgs& a, int k) {
    if constexpr (GLOBAL) return __ldg(a.cone_table + min(k, a.max_steps));
    else return cone_t(a, k);
}

// table_count (march_common.cuh) on the block's copy (plain loads: it may be
// shared memory).
__device__ __forceinline__ int cone_count(float far, int max_steps, int lane) {
    int lo = 0, hi = max_steps;
    while (lo < hi) {
        const int step = (hi - lo + 31) >> 5;
        const int k = lo + lane * step;
        const unsigned below = __ballot_sync(FULL, k < hi && s_cone[k] < far);
        const int nb = __popc(below);
        if (nb == 0) break;
        hi = min(lo + nb * step, hi);
        lo = lo + (nb - 1) * step + 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// lattice walk: the warp evaluates 32 lattice points of one ray at a time
// ---------------------------------------------------------------------------

// occupied<1> in two halves, so that a caller can have the load in flight while it
// works on another point: the bitfield word that holds x's cell (0 when x is
// outside the grid) and the cell's index. Bit (cell & 31) of the word is the
// occupancy bit of x.
template <typename G>
__device__ __forceinline__ unsigned level0_word(const G& g, float x0, float x1, float x2, unsigned slot_level0,
                                                unsigned& cell) {
    const int i0 = __float2int_rd(__fmul_rn(__fsub_rn(x0, g.lo(0, 0)), g.scale(0, 0)));
    const int i1 = __float2int_rd(__fmul_rn(__fsub_rn(x1, g.lo(0, 1)), g.scale(0, 1)));
    const int i2 = __float2int_rd(__fmul_rn(__fsub_rn(x2, g.lo(0, 2)), g.scale(0, 2)));
    cell = ((slot_level0 * g.res0() + i0) * g.res1() + i1) * g.res2() + i2;
    const bool in =
        (unsigned)i0 < (unsigned)g.res0() && (unsigned)i1 < (unsigned)g.res1() && (unsigned)i2 < (unsigned)g.res2();
    return in ? __ldg(g.bits() + (cell >> 5)) : 0u;
}

// Box test of the walks that use a grid's summed-area table. Every cell index
// along each axis is a monotone function of the lattice index k (t_k, the
// midpoints and the rounded index arithmetic all are), so the cells of the points
// between two points lie in the box their cells span (indices clamped to
// [-1, res]). If every cell of that box is inside the grid and occupied, every
// point between is occupied; if no in-grid cell of the box is occupied, none is
// (points outside the grid are empty). The table gives the box's count from eight
// entries, exactly when the box has fewer than 2^16 cells.

// Clamped cell indices of point x of the level-0 grid.
template <typename G>
__device__ __forceinline__ void clamped_cell(const G& g, float x0, float x1, float x2, int& i0, int& i1, int& i2) {
    i0 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x0, g.lo(0, 0)), g.scale(0, 0))), -1), g.res0());
    i1 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x1, g.lo(0, 1)), g.scale(0, 1))), -1), g.res1());
    i2 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x2, g.lo(0, 2)), g.scale(0, 2))), -1), g.res2());
}

// Decides the box spanned by cells (i0, i1, i2) and (n0, n1, n2) of grid slot
// sl0: full (all inside and occupied), empty (no in-grid cell occupied), or
// neither (undecided: test the points).
template <typename G>
__device__ __forceinline__ void box_decide(const G& g, unsigned sl0, int i0, int i1, int i2, int n0, int n1, int n2,
                                           bool& full, bool& empty) {
    const int r0 = g.res0(), r1 = g.res1(), r2 = g.res2();
    const int lo0 = min(i0, n0), hi0 = max(i0, n0);
    const int lo1 = min(i1, n1), hi1 = max(i1, n1);
    const int lo2 = min(i2, n2), hi2 = max(i2, n2);
    const bool inside = lo0 >= 0 && lo1 >= 0 && lo2 >= 0 && hi0 < r0 && hi1 < r1 && hi2 < r2;
    // in-grid part of the box: corners [a, b) per axis
    const int a0 = max(lo0, 0), a1 = max(lo1, 0), a2 = max(lo2, 0);
    const int b0 = min(hi0, r0 - 1) + 1, b1 = min(hi1, r1 - 1) + 1, b2 = min(hi2, r2 - 1) + 1;
    full = empty = false;
    if (b0 <= a0 || b1 <= a1 || b2 <= a2) {
        empty = true;  // no point lies inside the grid
        return;
    }
    // the brick summary first (shared memory, no table reads): a box within
    // 2 x 2 x 2 bricks of 8^3 cells is empty when they all are, and, inside the
    // grid, full when they all are
    if (const uint16_t* bm = g.bricks()) {
        const int x0 = a0 >> 3, x1 = (b0 - 1) >> 3, y0 = a1 >> 3, y1 = (b1 - 1) >> 3, z0 = a2 >> 3, z1 = (b2 - 1) >> 3;
        if (x1 - x0 <= 1 && y1 - y0 <= 1 && z1 - z0 <= 1) {
            const int nb1 = g.brick_nb1(), nb2 = g.brick_nb2();
            const uint16_t* gm = bm + sl0 * (unsigned)g.brick_per_grid();
            unsigned acc = 3u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int bx = (q & 4) ? x1 : x0, by = (q & 2) ? y1 : y0, bz = (q & 1) ? z1 : z0;
                const unsigned b = (unsigned)((bx * nb1 + by) * nb2 + bz);
                acc &= (unsigned)gm[b >> 3] >> ((b & 7u) * 2u);
            }
            if (acc & 1u) {
                empty = true;
                return;
            }
            if ((acc & 2u) && inside) {
                full = true;
                return;
            }
        }
    }
    const unsigned long long vol =
        (unsigned long long)(b0 - a0) * (unsigned long long)(b1 - a1) * (unsigned long long)(b2 - a2);
    if (vol >= 65536ull) return;
    const unsigned sy = (unsigned)(r2 + 1), sx = (unsigned)(r1 + 1) * sy;  // corner strides
    const uint16_t* t = g.sat() + sl0 * sx * (unsigned)(r0 + 1);
    const unsigned xa = (unsigned)a0 * sx, xb = (unsigned)b0 * sx, ya = (unsigned)a1 * sy, yb = (unsigned)b1 * sy;
    const unsigned za = (unsigned)a2, zb = (unsigned)b2;
    const unsigned cnt = ((unsigned)__ldg(t + xb + yb + zb) - (unsigned)__ldg(t + xa + yb + zb) -
                          (unsigned)__ldg(t + xb + ya + zb) - (unsigned)__ldg(t + xb + yb + za) +
                          (unsigned)__ldg(t + xa + ya + zb) + (unsigned)__ldg(t + xa + yb + za) +
                          (unsigned)__ldg(t + xb + ya + za) - (unsigned)__ldg(t + xa + ya + za)) &
                         0xffffu;
    empty = cnt == 0u;
    full = inside && cnt == (unsigned)vol;
}

// Box walk of one ray (a one-level grid with its table; shared lattices): lane j
// takes the first point of chunk grp + j (31 chunks per group) and the box up to
// the next chunk's first point (the lattice's last point for the last chunk);
// chunks whose box is full or empty take their ballot word from it, the others
// are tested point by point. Writes row[0 .. max_ch) and returns the sample
// count (summed over the warp).
template <bool CONE, typename G>
__device__ __forceinline__ int walk_box(const MarchArgs& a, const G& g, const float o[3], const float d[3],
                                        float near, float far, int nk, int max_ch, unsigned sl0, uint32_t* row,
                                        int lane) {
    const float dt = a.dt_min;
    int part = 0, count = 0;
    for (int grp = 0; grp < max_ch; grp += 31) {
        const int kp = min((grp + lane) << 5, nk - 1);
        float ts, tn;
        if (!CONE) {
            const float kf = __int2float_rn(kp);
            ts = __fadd_rn(near, __fmul_rn(kf, dt));
            tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
        } else {
            ts = cone_t(a, kp);
            tn = cone_t(a, kp + 1);
        }
        const float te = tn < far ? tn : far;
        const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
        int i0, i1, i2;
        clamped_cell(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)), __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                     __fadd_rn(o[2], __fmul_rn(d[2], mid)), i0, i1, i2);
        const int n0 = __shfl_down_sync(FULL, i0, 1);
        const int n1 = __shfl_down_sync(FULL, i1, 1);
        const int n2 = __shfl_down_sync(FULL, i2, 1);
        const int c = grp + lane;
        const bool exists = lane < 31 && c < max_ch;
        bool full = false, empty = false;
        if (exists) box_decide(g, sl0, i0, i1, i2, n0, n1, n2, full, empty);
        if (full || empty) {
            const int n = min(32, nk - (c << 5));
            const uint32_t m = full ? (n >= 32 ? ~0u : (1u << n) - 1u) : 0u;
            row[c] = m;
            part += __popc(m);
        }
        unsigned pend = __ballot_sync(FULL, exists && !full && !empty);
        while (pend) {
            const int cc = grp + __ffs(pend) - 1;
            pend &= pend - 1;
            const int k = (cc << 5) + lane;
            float ks, kn;
            if (!CONE) {
                const float kf = __int2float_rn(k);
                ks = __fadd_rn(near, __fmul_rn(kf, dt));
                kn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else {
                ks = cone_t(a, k);
                kn = cone_t(a, k + 1);
            }
            bool occ = false;
            if (k < nk) {
                const float ke = kn < far ? kn : far;
                const float km = __fmul_rn(__fadd_rn(ks, ke), 0.5f);
                occ = occupied_in<1>(g, __fadd_rn(o[0], __fmul_rn(d[0], km)), __fadd_rn(o[1], __fmul_rn(d[1], km)),
                                     __fadd_rn(o[2], __fmul_rn(d[2], km)), sl0);
            }
            const unsigned m = __ballot_sync(FULL, occ);
            if (lane == 0) row[cc] = m;
            count += __popc(m);
        }
    }
    return count + __reduce_add_sync(FULL, part);
}

// Box walk of one ray over a cascade (2..MAXL levels, each with its table;
// shared lattices). A point's level is the first whose cell indices are all in
// range, and every level's clamped index along each axis is monotone along the
// ray, so for the box of a chunk (lane j: chunk grp + j, from its first point to
// the next chunk's first point) at level l:
//   - an axis on which both ends are below 0 (or both at res) puts no point of
//     the chunk inside level l (the level is excluded);
//   - with L the first level not excluded, no point lies in a finer level; if
//     L's box is inside the grid, every point lies in L and its cells are in the
//     box, which the table of L decides as full or empty; if L is the outermost
//     level, points outside it lie outside every level (empty), so the in-grid
//     part's count decides empty;
//   - every level excluded: the chunk is empty.
// Other chunks are tested point by point.
template <int MAXL, bool CONE, typename G>
__device__ __forceinline__ int walk_box_levels(const MarchArgs& a, const G& g, const float o[3], const float d[3],
                                               float near, float far, int nk, int max_ch, unsigned sl0,
                                               uint32_t* row, int lane) {
    const float dt = a.dt_min;
    const int nl = g.n_levels();
    const int r0 = g.res0(), r1 = g.res1(), r2 = g.res2();
    int part = 0, count = 0;
    for (int grp = 0; grp < max_ch; grp += 31) {
        const int kp = min((grp + lane) << 5, nk - 1);
        float ts, tn;
        if (!CONE) {
            const float kf = __int2float_rn(kp);
            ts = __fadd_rn(near, __fmul_rn(kf, dt));
            tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
        } else {
            ts = cone_t(a, kp);
            tn = cone_t(a, kp + 1);
        }
        const float te = tn < far ? tn : far;
        const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
        const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
        const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
        const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
        // the first level not excluded, with both ends' clamped cells there
        int L = -1, i0 = 0, i1 = 0, i2 = 0, n0 = 0, n1 = 0, n2 = 0;
#pragma unroll
        for (int l = 0; l < MAXL; ++l) {
            if (l >= nl) break;  // uniform
            const int c0 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x0, g.lo(l, 0)), g.scale(l, 0))), -1), r0);
            const int c1 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x1, g.lo(l, 1)), g.scale(l, 1))), -1), r1);
            const int c2 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x2, g.lo(l, 2)), g.scale(l, 2))), -1), r2);
            const int e0 = __shfl_down_sync(FULL, c0, 1);
            const int e1 = __shfl_down_sync(FULL, c1, 1);
            const int e2 = __shfl_down_sync(FULL, c2, 1);
            const bool excluded = (c0 < 0 && e0 < 0) || (c0 >= r0 && e0 >= r0) || (c1 < 0 && e1 < 0) ||
                                  (c1 >= r1 && e1 >= r1) || (c2 < 0 && e2 < 0) || (c2 >= r2 && e2 >= r2);
            if (L < 0 && !excluded) {
                L = l;
                i0 = c0;
                i1 = c1;
                i2 = c2;
                n0 = e0;
                n1 = e1;
                n2 = e2;
            }
        }
        const int c = grp + lane;
        const bool exists = lane < 31 && c < max_ch;
        bool full = false, empty = false;
        if (exists) {
            if (L < 0) {
                empty = true;
            } else {
                const bool inside = min(i0, n0) >= 0 && min(i1, n1) >= 0 && min(i2, n2) >= 0 && max(i0, n0) < r0 &&
                                    max(i1, n1) < r1 && max(i2, n2) < r2;
                if (inside || L == nl - 1) box_decide(g, sl0 + (unsigned)L, i0, i1, i2, n0, n1, n2, full, empty);
            }
        }
        if (full || empty) {
            const int n = min(32, nk - (c << 5));
            const uint32_t m = full ? (n >= 32 ? ~0u : (1u << n) - 1u) : 0u;
            row[c] = m;
            part += __popc(m);
        }
        unsigned pend = __ballot_sync(FULL, exists && !full && !empty);
        while (pend) {
            const int cc = grp + __ffs(pend) - 1;
            pend &= pend - 1;
            const int k = (cc << 5) + lane;
            float ks, kn;
            if (!CONE) {
                const float kf = __int2float_rn(k);
                ks = __fadd_rn(near, __fmul_rn(kf, dt));
                kn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else {
                ks = cone_t(a, k);
                kn = cone_t(a, k + 1);
            }
            bool occ = false;
            if (k < nk) {
                const float ke = kn < far ? kn : far;
                const float km = __fmul_rn(__fadd_rn(ks, ke), 0.5f);
                occ = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], km)),
                                        __fadd_rn(o[1], __fmul_rn(d[1], km)), __fadd_rn(o[2], __fmul_rn(d[2], km)),
                                        sl0);
            }
            const unsigned m = __ballot_sync(FULL, occ);
            if (lane == 0) row[cc] = m;
            count += __popc(m);
        }
    }
    return count + __reduce_add_sync(FULL, part);
}

// One ray, all 32 lanes: one ballot word per 32 lattice points into row[c].
// count = samples, nch = ballot words written (row[0..nch)).
// COARSE (shared lattices): first one point every 32 per lane, and chunks that
// lie in a single cell take their word from one occupancy test (see below).
template <int MAXL, bool CONE, bool UNROLL2, bool COARSE, int BOX, typename G>
__device__ __forceinline__ void walk_lattice(const MarchArgs& a, const G& g, const float o[3], const float d[3],
                                             float near, float far, unsigned sl0, uint32_t* row, float* lat, int lane,
                                             int& count_out, int& nch_out, int& pts_out) {
    const float dt = a.dt_min;
    const bool shared = !CONE || near == a.near_plane;
    // shared lattices know their length; an own cone lattice ends when t_k >= far
    int nk = !CONE ? lattice_count(a, near, far, dt)
                   : (shared ? (MAXL == 0 ? table_count(a.cone_table, a.max_steps, far, lane) : cone_count(far, a.max_steps, lane)) : a.max_steps);
    if (CONE && shared && nk > 32 * a.mask_words) {  // the host's bound on cone lattices was passed
        if (lane == 0) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
        nk = 32 * a.mask_words;
    }
    const int max_ch = min((nk + 31) >> 5, a.mask_words);
    int count = 0, nch = 0;
    pts_out = shared ? nk : 0;  // own cone lattices are counted as they are walked
    if constexpr (BOX != 0 && MAXL == 1) {
        if (shared && g.sat()) {
            count_out = max_ch > 0 ? walk_box<CONE>(a, g, o, d, near, far, nk, max_ch, sl0, row, lane) : 0;
            nch_out = max_ch;
            return;
        }
    }
    if constexpr (BOX != 0 && MAXL > 1) {
        if (shared && g.sat()) {
            count_out = max_ch > 0 ? walk_box_levels<MAXL, CONE>(a, g, o, d, near, far, nk, max_ch, sl0, row, lane)
                                   : 0;
            nch_out = max_ch;
            return;
        }
    }
    if (COARSE && MAXL > 0 && shared) {  // contracted indices are not monotone along a ray
        // Every cell index along each axis, at each level, is a monotone function
        // of k (t_k, the midpoints and the rounded index arithmetic all are), and so
        // is the index clamped to [-1, res]. If two points have the same clamped
        // indices at every level, so does every point between them: they share the
        // level that holds them and its cell. Lane j takes point 32(g + j) (the last
        // point where that is past the lattice); chunk g + j (j < 31) whose first
        // point and the next chunk's first point agree lies in one cell, and its
        // ballot word follows from one occupancy test. The other chunks are tested
        // point by point. Groups of 31 chunks.
        int part = 0;  // samples of this lane's single-cell chunks
        for (int grp = 0; grp < max_ch; grp += 31) {
            const int kp = min((grp + lane) << 5, nk - 1);
            float ts, tn;
            if (!CONE) {
                const float kf = __int2float_rn(kp);
                ts = __fadd_rn(near, __fmul_rn(kf, dt));
                tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else {
                ts = lattice_t<MAXL == 0>(a, kp);
                tn = lattice_t<MAXL == 0>(a, kp + 1);
            }
            const float te = tn < far ? tn : far;
            const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
            const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
            const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
            const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
            bool same = true;
#pragma unroll
            for (int l = 0; l < MAXL; ++l) {
                if (l >= g.n_levels()) break;
                const int i0 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x0, g.lo(l, 0)), g.scale(l, 0))), -1),
                                   g.res0());
                const int i1 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x1, g.lo(l, 1)), g.scale(l, 1))), -1),
                                   g.res1());
                const int i2 = min(max(__float2int_rd(__fmul_rn(__fsub_rn(x2, g.lo(l, 2)), g.scale(l, 2))), -1),
                                   g.res2());
                const int n0 = __shfl_down_sync(FULL, i0, 1);
                const int n1 = __shfl_down_sync(FULL, i1, 1);
                const int n2 = __shfl_down_sync(FULL, i2, 1);
                same = same && i0 == n0 && i1 == n1 && i2 == n2;
            }
            const bool occ_p = occupied_in<MAXL>(g, x0, x1, x2, sl0);
            const int c = grp + lane;
            const bool exists = lane < 31 && c < max_ch;
            const bool uni = exists && same;
            if (uni) {
                const int n = min(32, nk - (c << 5));
                const uint32_t m = occ_p ? (n >= 32 ? ~0u : (1u << n) - 1u) : 0u;
                row[c] = m;
                part += __popc(m);
            }
            unsigned pend = __ballot_sync(FULL, exists && !uni);
            while (pend) {
                const int cc = grp + __ffs(pend) - 1;
                pend &= pend - 1;
                const int k = (cc << 5) + lane;
                float ks, kn;
                if (!CONE) {
                    const float kf = __int2float_rn(k);
                    ks = __fadd_rn(near, __fmul_rn(kf, dt));
                    kn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                } else {
                    ks = lattice_t<MAXL == 0>(a, k);
                    kn = lattice_t<MAXL == 0>(a, k + 1);
                }
                bool occ = false;
                if (k < nk && ks < far) {
                    const float ke = kn < far ? kn : far;
                    const float km = __fmul_rn(__fadd_rn(ks, ke), 0.5f);
                    occ = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], km)), __fadd_rn(o[1], __fmul_rn(d[1], km)),
                                         __fadd_rn(o[2], __fmul_rn(d[2], km)), sl0);
                }
                const unsigned m = __ballot_sync(FULL, occ);
                if (lane == 0) row[cc] = m;
                count += __popc(m);
            }
        }
        count += __reduce_add_sync(FULL, part);
        nch = max_ch;
    } else if (!CONE && UNROLL2) {
        // two chunks per iteration: two independent chains and two grid loads in flight per lane
        for (int c = 0; c < max_ch; c += 2) {
            const int k0 = (c << 5) + lane, k1 = k0 + 32;
            const float kf0 = __int2float_rn(k0), kf1 = __int2float_rn(k1);
            bool occ0 = false, occ1 = false;
            if (k0 < nk) {
                const float ts = __fadd_rn(near, __fmul_rn(kf0, dt));
                const float tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf0, 1.0f), dt));
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                occ0 = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)), __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                      __fadd_rn(o[2], __fmul_rn(d[2], mid)), sl0);
            }
            if (k1 < nk) {
                const float ts = __fadd_rn(near, __fmul_rn(kf1, dt));
                const float tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf1, 1.0f), dt));
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                occ1 = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)), __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                      __fadd_rn(o[2], __fmul_rn(d[2], mid)), sl0);
            }
            const unsigned m0 = __ballot_sync(FULL, occ0);
            const unsigned m1 = __ballot_sync(FULL, occ1);
            if (lane == 0) {
                row[c] = m0;
                if (c + 1 < max_ch) row[c + 1] = m1;
            }
            count += __popc(m0) + __popc(m1);
        }
        nch = max_ch;
    } else if (shared) {
        // closed-form or tabulated lattice: t_k < far for every k < nk, so every
        // chunk below nk/32 is full and only the last one needs the bound test; the
        // count is summed from the finished row
        const int nfull = nk >> 5;
        if constexpr (!CONE && MAXL == 1) {
            // Uniform steps on one level: each chunk's bitfield word is loaded one
            // chunk ahead, so that load's latency overlaps the ballot and row store
            // of the chunk before it. The last look-ahead is the partial chunk's (or
            // one past the lattice): its load stays inside the grid and its result
            // is not used.
            auto probe = [&](int k, unsigned& cell) -> unsigned {
                const float kf = __int2float_rn(k);
                const float ts = __fadd_rn(near, __fmul_rn(kf, dt));
                const float tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                return level0_word(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)), __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                   __fadd_rn(o[2], __fmul_rn(d[2], mid)), sl0, cell);
            };
            if (nfull > 0) {
                unsigned cell;
                unsigned w = probe(lane, cell);
                for (int c = 0; c < nfull; ++c) {
                    unsigned cell_n;
                    const unsigned w_n = probe(((c + 1) << 5) + lane, cell_n);
                    const unsigned m = __ballot_sync(FULL, (w >> (cell & 31u)) & 1u);
                    if (lane == 0) row[c] = m;
                    cell = cell_n;
                    w = w_n;
                }
            }
        } else {
            for (int c = 0; c < nfull; ++c) {
                const int k = (c << 5) + lane;
                float ts, tn;
                if (!CONE) {
                    const float kf = __int2float_rn(k);
                    ts = __fadd_rn(near, __fmul_rn(kf, dt));
                    tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                } else {
                    ts = lattice_t<MAXL == 0>(a, k);
                    tn = lattice_t<MAXL == 0>(a, k + 1);
                }
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                const bool occ = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)),
                                                __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                                __fadd_rn(o[2], __fmul_rn(d[2], mid)), sl0);
                const unsigned m = __ballot_sync(FULL, occ);
                if (lane == 0) row[c] = m;
            }
        }
        if (nfull < max_ch) {
            const int k = (nfull << 5) + lane;
            float ts, tn;
            if (!CONE) {
                const float kf = __int2float_rn(k);
                ts = __fadd_rn(near, __fmul_rn(kf, dt));
                tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else {
                ts = lattice_t<MAXL == 0>(a, k);
                tn = lattice_t<MAXL == 0>(a, k + 1);
            }
            bool occ = false;
            if (k < nk && ts < far) {
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                occ = occupied_in<MAXL>(g, __fadd_rn(o[0], __fmul_rn(d[0], mid)), __fadd_rn(o[1], __fmul_rn(d[1], mid)),
                                     __fadd_rn(o[2], __fmul_rn(d[2], mid)), sl0);
            }
            const unsigned m = __ballot_sync(FULL, occ);
            if (lane == 0) row[nfull] = m;
        }
        nch = max_ch;
        __syncwarp();
        int part = 0;
        for (int w = lane; w < nch; w += 32) part += __popc(row[w]);
        count = __reduce_add_sync(FULL, part);
    } else {
        float tcur = near;
        int c = 0;
        for (; c < max_ch; ++c) {
            const int k = (c << 5) + lane;
            float ts, tn;
            if (!CONE) {
                const float kf = __int2float_rn(k);
                ts = __fadd_rn(near, __fmul_rn(kf, dt));
                tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else if (shared) {
                ts = lattice_t<MAXL == 0>(a, k);
                tn = lattice_t<MAXL == 0>(a, k + 1);
            } else {
                cone_extend(a, lat, tcur, lane);
                ts = lat[lane];
                tn = lat[lane + 1];
            }
            const bool valid = k < nk && ts < far;
            const unsigned vmask = __ballot_sync(FULL, valid);
            if (CONE && !shared && vmask == 0u) break;
            if (!shared) pts_out += __popc(vmask);
            bool occ = false;
            if (valid) {
                const float te = tn < far ? tn : far;
                const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
                const float x0 = __fadd_rn(o[0], __fmul_rn(d[0], mid));
                const float x1 = __fadd_rn(o[1], __fmul_rn(d[1], mid));
                const float x2 = __fadd_rn(o[2], __fmul_rn(d[2], mid));
                occ = occupied_in<MAXL>(g, x0, x1, x2, sl0);
            }
            const unsigned m = __ballot_sync(FULL, occ);
            if (lane == 0) row[c] = m;
            count += __popc(m);
            nch = c + 1;
        }
        // an own cone lattice that still had points beyond the rows' capacity
        if (CONE && !shared && c == a.mask_words && (c << 5) < a.max_steps && tcur < far && lane == 0)
            raise_status(a.d_status, NACC_STATUS_OVERFLOW);
    }
    count_out = count;
    nch_out = nch;
}

// Point k of a uniform lattice: its midpoint's position.
__device__ __forceinline__ void uniform_midpoint(float near, float far, float dt, int k, float o0, float o1,
                                                 float o2, float d0, float d1, float d2, float& x0, float& x1,
                                                 float& x2) {
    const float kf = __int2float_rn(k);
    const float ts = __fadd_rn(near, __fmul_rn(kf, dt));
    const float tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
    const float te = tn < far ? tn : far;
    const float mid = __fmul_rn(__fadd_rn(ts, te), 0.5f);
    x0 = __fadd_rn(o0, __fmul_rn(d0, mid));
    x1 = __fadd_rn(o1, __fmul_rn(d1, mid));
    x2 = __fadd_rn(o2, __fmul_rn(d2, mid));
}

// Phase 1 of a tile for the box walk with uniform steps on one grid: the whole
// tile at once. Lane i clips ray i and sizes its lattice; the tile's chunks then
// form one list, ray after ray, taken 32 at a time: lane j evaluates the first
// point of its chunk and the point after the chunk (the next chunk's first, or
// the lattice's last) and decides the chunk from the box of the two cells. The
// chunks left undecided are tested point by point by the whole warp. The ray
// loads and the table loads of 32 chunks are in flight together, instead of a
// few dependent round trips per ray.
__device__ __forceinline__ void box_tile_uniform(const MarchArgs& a, const uint16_t* s_bricks, int ray0, int nr,
                                                 uint32_t* wmask, int lane, int& my_count, int& my_nch,
                                                 float& my_near, float& my_far, int& tile_pts) {
    const ArgGeom g{a, s_bricks};
    const float dt = a.dt_min;
    float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f, d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, near = 0.0f, far = 0.0f;
    int nk = 0;
    unsigned sl0 = 0;
    if (lane < nr) {
        const int r = ray0 + lane;
        float o[3], d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
            d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
        }
        const int slot = slot_of(a, r);
        if (slot >= 0 && slot < a.n_slots) {
            sl0 = (unsigned)slot * (unsigned)a.n_levels;
            if (clip_ray_in<false>(a, g, o, d, near, far)) nk = lattice_count(a, near, far, dt);
        } else {
            raise_status(a.d_status, NACC_STATUS_BAD_INDEX);
        }
        o0 = o[0], o1 = o[1], o2 = o[2], d0 = d[0], d1 = d[1], d2 = d[2];
    }
    const int nch = min((nk + 31) >> 5, a.mask_words);
    const int incl = warp_incl_scan_int(nch, lane);  // lanes past the tile's rays add 0
    const int start = incl - nch;
    const int total = __shfl_sync(FULL, incl, 31);
    for (int f0 = 0; f0 < total; f0 += 32) {
        const int f = f0 + lane;
        const bool valid = f < total;
        int ri = 0;  // the ray of chunk f: the last ray whose chunks start at or before f
        for (int q = 1; q < nr; ++q)
            if (__shfl_sync(FULL, start, q) <= f) ri = q;
        const float r_o0 = __shfl_sync(FULL, o0, ri), r_o1 = __shfl_sync(FULL, o1, ri);
        const float r_o2 = __shfl_sync(FULL, o2, ri), r_d0 = __shfl_sync(FULL, d0, ri);
        const float r_d1 = __shfl_sync(FULL, d1, ri), r_d2 = __shfl_sync(FULL, d2, ri);
        const float r_near = __shfl_sync(FULL, near, ri), r_far = __shfl_sync(FULL, far, ri);
        const int r_nk = __shfl_sync(FULL, nk, ri), r_start = __shfl_sync(FULL, start, ri);
        const unsigned r_sl0 = __shfl_sync(FULL, sl0, ri);
        const int c = f - r_start;
        const int ka = c << 5, kb = min(ka + 32, r_nk - 1);
        bool full = false, empty = false;
        if (valid) {
            float x0, x1, x2;
            int i0, i1, i2, n0, n1, n2;
            uniform_midpoint(r_near, r_far, dt, ka, r_o0, r_o1, r_o2, r_d0, r_d1, r_d2, x0, x1, x2);
            clamped_cell(g, x0, x1, x2, i0, i1, i2);
            uniform_midpoint(r_near, r_far, dt, kb, r_o0, r_o1, r_o2, r_d0, r_d1, r_d2, x0, x1, x2);
            clamped_cell(g, x0, x1, x2, n0, n1, n2);
            box_decide(g, r_sl0, i0, i1, i2, n0, n1, n2, full, empty);
            if (full || empty) {
                const int n = min(32, r_nk - ka);
                wmask[ri * a.row_stride + c] = full ? (n >= 32 ? ~0u : (1u << n) - 1u) : 0u;
            }
        }
        unsigned pend = __ballot_sync(FULL, valid && !full && !empty);
        while (pend) {
            const int p = __ffs(pend) - 1;
            pend &= pend - 1;
            const int pri = __shfl_sync(FULL, ri, p), pc = __shfl_sync(FULL, c, p);
            const float p_o0 = __shfl_sync(FULL, o0, pri), p_o1 = __shfl_sync(FULL, o1, pri);
            const float p_o2 = __shfl_sync(FULL, o2, pri), p_d0 = __shfl_sync(FULL, d0, pri);
            const float p_d1 = __shfl_sync(FULL, d1, pri), p_d2 = __shfl_sync(FULL, d2, pri);
            const float p_near = __shfl_sync(FULL, near, pri), p_far = __shfl_sync(FULL, far, pri);
            const int p_nk = __shfl_sync(FULL, nk, pri);
            const unsigned p_sl0 = __shfl_sync(FULL, sl0, pri);
            const int k = (pc << 5) + lane;
            bool occ = false;
            if (k < p_nk) {
                float x0, x1, x2;
                uniform_midpoint(p_near, p_far, dt, k, p_o0, p_o1, p_o2, p_d0, p_d1, p_d2, x0, x1, x2);
                occ = occupied_in<1>(g, x0, x1, x2, p_sl0);
            }
            const unsigned m = __ballot_sync(FULL, occ);
            if (lane == 0) wmask[pri * a.row_stride + pc] = m;
        }
    }
    __syncwarp();
    for (int i = 0; i < nr; ++i) {  // samples per ray from its finished row
        const int n_i = __shfl_sync(FULL, nch, i);
        const uint32_t* row = wmask + i * a.row_stride;
        int part = 0;
        for (int w = lane; w < n_i; w += 32) part += __popc(row[w]);
        const int cnt = __reduce_add_sync(FULL, part);
        if (lane == i) my_count = cnt;
    }
    my_nch = nch;
    my_near = near;
    my_far = far;
    tile_pts = __reduce_add_sync(FULL, nk);
}

// ---------------------------------------------------------------------------
// phases 2 and 3 of a tile (shared by both phase-1 strategies)
// ---------------------------------------------------------------------------

// One tile between its ballot pass and its stores. Lane i holds ray i's sample
// count, ballot words written, [near, far] and inclusive count within the tile.
struct TileState {
    int tile, ray0, nr, agg;
    int my_count, my_nch, incl;
    float my_near, my_far;
};

// After phase 1: counts within the tile, and the tile's total published for the
// look-back (never waits).
__device__ __forceinline__ void publish_tile(const MarchArgs& a, TileState& t, int lane) {
    t.incl = warp_incl_scan_int(t.my_count, lane);
    t.agg = __shfl_sync(FULL, t.incl, 31);
    publish_aggregate(a.tile_status, t.tile, (unsigned long long)t.agg, lane, a.hooks);
}

// The tile's offset by look-back, then the ballot words expanded into
// compacted, coalesced stores of (t_start, t_end, ray).
template <bool CONE>
__device__ __forceinline__ void finish_tile(const MarchArgs& a, const uint32_t* wmask, const TileState& t,
                                            float* lat, int lane) {
    const float dt = a.dt_min;
    const unsigned lt = lanemask_lt();
    const int tile = t.tile, ray0 = t.ray0, nr = t.nr, agg = t.agg;
    const int my_count = t.my_count, my_nch = t.my_nch;
    const float my_near = t.my_near, my_far = t.my_far;
    const long long excl =
        (long long)resolve_prefix(a.tile_status, tile, (unsigned long long)agg, lane, a.d_status, a.hooks);
    const int my_excl = t.incl - my_count;
    if (lane < nr) {
        const int2 pi = make_int2((int)(excl + my_excl), my_count);
        reinterpret_cast<int2*>(a.packed_info)[ray0 + lane] = pi;
    }
    if (lane == 0 && tile == a.n_tiles - 1) {
        const long long total = excl + agg;
        *a.n_samples = total;
        if (total > a.capacity) raise_status(a.d_status, NACC_STATUS_CAPACITY);
        if (total > 0x7fffffffLL) raise_status(a.d_status, NACC_STATUS_OVERFLOW);
    }
    // Output positions fit 32 bits: the tile starts below capacity <= 2^31 - 1
    // and adds at most tile_rays * max_steps <= 2^20 samples.
    if (excl >= a.capacity) return;
    const unsigned cap = (unsigned)(a.capacity < 0x7fffffffLL ? a.capacity : 0x7fffffffLL);
    for (int i = 0; i < nr; ++i) {
        const int cnt = __shfl_sync(FULL, my_count, i);
        if (cnt == 0) continue;
        const int nch = __shfl_sync(FULL, my_nch, i);
        const float near = __shfl_sync(FULL, my_near, i);
        const float far = __shfl_sync(FULL, my_far, i);
        const bool shared = !CONE || near == a.near_plane;
        const int r = ray0 + i;
        const uint32_t* row = wmask + i * a.row_stride;
        unsigned base = (unsigned)excl + (unsigned)__shfl_sync(FULL, my_excl, i);
        if (shared && a.vec_out) {
            // a shared lattice with 16-byte aligned outputs: the words are taken 32 at a
            // time; in a run of full words output p holds lattice point
            // k = k_run + (p - p_run), so lane l writes four consecutive samples with one
            // 16-byte store per array (t_k .. t_{k+4} give their four intervals), after
            // a scalar head up to the 16-byte boundary; other words as below
            const bool fits = (unsigned long long)base + (unsigned)cnt <= (unsigned long long)cap;
            for (int c0 = 0; c0 < nch; c0 += 32) {
                const uint32_t mw = c0 + lane < nch ? row[c0 + lane] : 0u;
                const unsigned fullb = __ballot_sync(FULL, mw == ~0u);
                const unsigned nonz = __ballot_sync(FULL, mw != 0u);
                int w = 0;
                const int nw = min(32, nch - c0);
                while (w < nw) {
                    const unsigned rest = nonz >> w;
                    if (rest == 0u) break;
                    w += __ffs(rest) - 1;  // the next non-empty word
                    if ((fullb >> w) & 1u) {
                        const unsigned fr = ~(fullb >> w);
                        const int run = fr ? __ffs(fr) - 1 : 32 - w;  // consecutive full words from w
                        const unsigned n = 32u * (unsigned)run;
                        const int k0 = (c0 + w) << 5;
                        const unsigned head = min((4u - (base & 3u)) & 3u, n);
                        const unsigned groups = (n - head) >> 2;
                        for (unsigned q = (unsigned)lane; q < groups; q += 32u) {
                            const unsigned p = base + head + 4u * q;
                            const int k = k0 + (int)(head + 4u * q);
                            float t[5];
#pragma unroll
                            for (int j = 0; j < 5; ++j) {
                                if (!CONE) {
                                    t[j] = __fadd_rn(near, __fmul_rn(__int2float_rn(k + j), dt));
                                } else {
                                    t[j] = cone_t(a, k + j);
                                }
                            }
                            const float4 ts4 = make_float4(t[0], t[1], t[2], t[3]);
                            const float4 te4 = make_float4(t[1] < far ? t[1] : far, t[2] < far ? t[2] : far,
                                                           t[3] < far ? t[3] : far, t[4] < far ? t[4] : far);
                            if (fits || p + 3u < cap) {
                                *reinterpret_cast<float4*>(a.t_starts + p) = ts4;
                                *reinterpret_cast<float4*>(a.t_ends + p) = te4;
                                *reinterpret_cast<int4*>(a.ray_indices + p) = make_int4(r, r, r, r);
                            } else {
                                const float sv[4] = {ts4.x, ts4.y, ts4.z, ts4.w};
                                const float ev[4] = {te4.x, te4.y, te4.z, te4.w};
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    if (p + j < cap) {
                                        a.t_starts[p + j] = sv[j];
                                        a.t_ends[p + j] = ev[j];
                                        a.ray_indices[p + j] = r;
                                    }
                                }
                            }
                        }
                        // head (lanes 0 .. head - 1) and tail (the last (n - head) & 3 samples)
                        const unsigned tail = (n - head) & 3u;
                        const int sl = lane < (int)head ? lane : lane - (int)head;
                        const bool is_head = lane < (int)head;
                        const bool is_tail = !is_head && sl < (int)tail;
                        if (is_head || is_tail) {
                            const unsigned off = is_head ? (unsigned)lane : head + 4u * groups + (unsigned)sl;
                            const unsigned pos = base + off;
                            const int k = k0 + (int)off;
                            float ts, tn;
                            if (!CONE) {
                                const float kf = __int2float_rn(k);
                                ts = __fadd_rn(near, __fmul_rn(kf, dt));
                                tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                            } else {
                                ts = cone_t(a, k);
                                tn = cone_t(a, k + 1);
                            }
                            if (fits || pos < cap) {
                                a.t_starts[pos] = ts;
                                a.t_ends[pos] = tn < far ? tn : far;
                                a.ray_indices[pos] = r;
                            }
                        }
                        base += n;
                        w += run;
                    } else {
                        const unsigned m = __shfl_sync(FULL, mw, w);
                        const int k = ((c0 + w) << 5) + lane;
                        float ts, tn;
                        if (!CONE) {
                            const float kf = __int2float_rn(k);
                            ts = __fadd_rn(near, __fmul_rn(kf, dt));
                            tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                        } else {
                            ts = cone_t(a, k);
                            tn = cone_t(a, k + 1);
                        }
                        const unsigned pos = base + __popc(m & lt);
                        if (((m >> lane) & 1u) && (fits || pos < cap)) {
                            a.t_starts[pos] = ts;
                            a.t_ends[pos] = tn < far ? tn : far;
                            a.ray_indices[pos] = r;
                        }
                        base += __popc(m);
                        ++w;
                    }
                }
            }
            continue;
        }
        if (shared) {
            // a shared lattice: four chunks' words read before any is used, so the
            // shared-memory reads overlap the stores of the chunks before; a full
            // word (most chunks) stores lane l at base + l; when the whole ray lands
            // below capacity no store checks it
            const bool fits = (unsigned long long)base + (unsigned)cnt <= (unsigned long long)cap;
            for (int c0 = 0; c0 < nch; c0 += 4) {
                uint32_t m4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) m4[u] = c0 + u < nch ? row[c0 + u] : 0u;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned m = m4[u];
                    if (m == 0u) continue;
                    const int k = ((c0 + u) << 5) + lane;
                    float ts, tn;
                    if (!CONE) {
                        const float kf = __int2float_rn(k);
                        ts = __fadd_rn(near, __fmul_rn(kf, dt));
                        tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
                    } else {
                        ts = cone_t(a, k);
                        tn = cone_t(a, k + 1);
                    }
                    const float te = tn < far ? tn : far;
                    if (m == ~0u) {
                        const unsigned pos = base + (unsigned)lane;
                        if (fits || pos < cap) {
                            a.t_starts[pos] = ts;
                            a.t_ends[pos] = te;
                            a.ray_indices[pos] = r;
                        }
                        base += 32u;
                    } else {
                        const unsigned pos = base + __popc(m & lt);
                        if (((m >> lane) & 1u) && (fits || pos < cap)) {
                            a.t_starts[pos] = ts;
                            a.t_ends[pos] = te;
                            a.ray_indices[pos] = r;
                        }
                        base += __popc(m);
                    }
                }
            }
            continue;
        }
        float tcur = near;
        for (int c = 0; c < nch; ++c) {
            const unsigned m = row[c];
            if (shared && m == 0u) continue;  // an own cone lattice is extended chunk by chunk
            const int k = (c << 5) + lane;
            float ts, tn;
            if (!CONE) {
                const float kf = __int2float_rn(k);
                ts = __fadd_rn(near, __fmul_rn(kf, dt));
                tn = __fadd_rn(near, __fmul_rn(__fadd_rn(kf, 1.0f), dt));
            } else if (shared) {
                ts = cone_t(a, k);
                tn = cone_t(a, k + 1);
            } else {
                cone_extend(a, lat, tcur, lane);
                ts = lat[lane];
                tn = lat[lane + 1];
            }
            const unsigned pos = base + __popc(m & lt);
            if (((m >> lane) & 1u) && pos < cap) {
                a.t_starts[pos] = ts;
                a.t_ends[pos] = tn < far ? tn : far;
                a.ray_indices[pos] = r;
            }
            base += __popc(m);
        }
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Batch of scenes with their own grids: the scene of ray r, the first whose
// consecutive rays end after r, found by the whole warp 32 scenes at a time
// starting from `from` (a scene that starts at or before r: the warp's rays only
// grow).
__device__ __forceinline__ int scene_of(const MarchArgs& a, int r, int from, int lane) {
    for (int base = from; base < a.n_scenes; base += 32) {
        const int s = base + lane;
        const unsigned past = __ballot_sync(FULL, s < a.n_scenes && __ldg(a.scene_end + s) > r);
        if (past) return base + __ffs(past) - 1;
    }
    return a.n_scenes - 1;  // not reached: the last scene's rays end at n_rays
}

// The warp's copy of a scene's geometry in shared memory.
__device__ __forceinline__ void load_scene(const MarchArgs& a, int scene, SceneGeom* dst, int lane) {
    constexpr int kWords = (int)(sizeof(SceneGeom) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.scenes + scene);
    uint32_t* out = reinterpret_cast<uint32_t*>(dst);
    __syncwarp();
    for (int k = lane; k < kWords; k += 32) out[k] = __ldg(src + k);
    __syncwarp();
}

// Lattice walk: the warp takes the tile's rays one at a time. Tiles go two deep:
// the warp runs the ballot pass of a new tile and publishes its total before it
// waits for the offset of the tile it did before (whose rows sit in the other
// half of the warp's shared memory), so the look-back rarely stalls.
// BATCHED: every ray looks up its scene's own grid (nacc_march_rays_batched).
// BOX: 0 no table; 1 the box walk ray by ray; 2 the whole tile's chunks at once
// (uniform steps, one grid; otherwise as 1).
template <int MAXL, int MINB, bool CONE, bool UNROLL2 = false, bool COARSE = false, bool BATCHED = false,
          int BOX = 0>
__global__ void __launch_bounds__(kThreads, MINB) march_uniform_kernel(const MarchArgs a) {
    extern __shared__ uint32_t s_masks[];  // per warp: 2 x [tile_rays][row_stride]; then the brick summary
    __shared__ float s_lat[kWarps][36];    // cone steps with a ray-specific start
    __shared__ SceneGeom s_scene[BATCHED ? kWarps : 1];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t tile_words = (size_t)a.tile_rays * a.row_stride;
    uint16_t* s_bricks = nullptr;
    if (!BATCHED && a.bricks) {
        s_bricks = reinterpret_cast<uint16_t*>(s_masks + (size_t)kWarps * 2 * tile_words);
        for (int k = threadIdx.x; k < a.brick_entries; k += kThreads) s_bricks[k] = __ldg(a.bricks + k);
        __syncthreads();
    }
    if constexpr (CONE) {
        if (a.cone_smem_at >= 0) {
            float* tab = reinterpret_cast<float*>(s_masks) + a.cone_smem_at;
            for (int k = threadIdx.x; k <= a.max_steps; k += kThreads) tab[k] = __ldg(a.cone_table + k);
            if (threadIdx.x == 0) s_cone = tab;
        } else if (threadIdx.x == 0) {
            s_cone = a.cone_table;
        }
        __syncthreads();
    }
    uint32_t* wbase = s_masks + (size_t)warp * 2 * tile_words;
    float* lat = s_lat[warp];
    int scene = 0, held = -1;  // BATCHED: scene of the current ray; scene held in s_scene[warp]

    TileState prev;
    bool have_prev = false;
    int buf = 0;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = (int)atomicAdd(a.ticket, 1u);
        tile = __shfl_sync(FULL, tile, 0);
        const bool have = tile < a.n_tiles;
        TileState cur;
        if (have) {
            uint32_t* wmask = wbase + buf * tile_words;
            cur.tile = tile;
            cur.ray0 = tile * a.tile_rays;
            cur.nr = min(a.tile_rays, a.n_rays - cur.ray0);
            int my_count = 0, my_nch = 0;
            float my_near = 0.0f, my_far = 0.0f;
            int tile_pts = 0;  // at most tile_rays * max_steps
            constexpr bool kTileBox = BOX == 2 && !CONE && !BATCHED && MAXL == 1;
            if constexpr (kTileBox)
                box_tile_uniform(a, s_bricks, cur.ray0, cur.nr, wmask, lane, my_count, my_nch, my_near, my_far,
                                 tile_pts);
            for (int i = 0; i < (kTileBox ? 0 : cur.nr); ++i) {
                const int r = cur.ray0 + i;
                float o[3], d[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    o[k] = __ldg(a.rays_o + 3 * (size_t)r + k);
                    d[k] = __ldg(a.rays_d + 3 * (size_t)r + k);
                }
                float near = 0.0f, far = 0.0f;
                int count = 0, nch = 0, pts = 0;
                uint32_t* row = wmask + i * a.row_stride;
                if constexpr (BATCHED) {
                    scene = scene_of(a, r, scene, lane);
                    if (scene != held) {
                        load_scene(a, scene, &s_scene[warp], lane);
                        held = scene;
                    }
                    if constexpr (MAXL <= 1) {
                        const RegGeom g(s_scene[warp]);
                        if (clip_ray_in<MAXL == 0>(a, g, o, d, near, far))
                            walk_lattice<MAXL, CONE, UNROLL2, COARSE, BOX>(a, g, o, d, near, far, 0u, row, lat, lane,
                                                                      count, nch, pts);
                    } else {
                        const SmemGeom g{&s_scene[warp]};
                        if (clip_ray_in<false>(a, g, o, d, near, far))
                            walk_lattice<MAXL, CONE, UNROLL2, COARSE, BOX>(a, g, o, d, near, far, 0u, row, lat, lane,
                                                                      count, nch, pts);
                    }
                } else {
                    const int slot = slot_of(a, r);
                    const bool slot_ok = slot >= 0 && slot < a.n_slots;
                    if (!slot_ok && lane == 0) raise_status(a.d_status, NACC_STATUS_BAD_INDEX);
                    const ArgGeom g{a, s_bricks};
                    if (slot_ok && clip_ray_in<MAXL == 0>(a, g, o, d, near, far))
                        walk_lattice<MAXL, CONE, UNROLL2, COARSE, BOX>(a, g, o, d, near, far,
                                                                  (unsigned)slot * (unsigned)a.n_levels, row, lat,
                                                                  lane, count, nch, pts);
                }
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
            publish_tile(a, cur, lane);
        }
        if (have_prev) {
            finish_tile<CONE>(a, wbase + (buf ^ 1) * tile_words, prev, lat, lane);
            __syncwarp();
        }
        if (!have) break;
        prev = cur;
        have_prev = true;
        buf ^= 1;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename K>
void launch_uniform(K kernel, size_t smem, int need, cudaStream_t st, const MarchArgs& a) {
    // without the opt-in, static and dynamic shared memory together are limited to
    // 48 KB; the kernels' static part is below 8 KB
    if (smem > 40 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = blocks_for(kernel, smem, need);
    kernel<<<blocks, kThreads, smem, st>>>(a);
}

// Kernel variant for a level count, step rule and the tuning knobs.
template <int MAXL, int MINB>
void launch_variant(bool cone, bool unroll, bool coarse, size_t smem, int need, cudaStream_t st,
                    const MarchArgs& a) {
    if constexpr (MAXL == 0) coarse = false;  // contracted space: no coarse pass
    if (cone) {
        if constexpr (MAXL > 0)
            if (coarse) {
                launch_uniform(march_uniform_kernel<MAXL, MINB, true, false, true>, smem, need, st, a);
                return;
            }
        launch_uniform(march_uniform_kernel<MAXL, MINB, true>, smem, need, st, a);
    } else if (coarse) {
        if constexpr (MAXL > 0) launch_uniform(march_uniform_kernel<MAXL, MINB, false, false, true>, smem, need, st, a);
    } else {
        if constexpr (MAXL == 1) {  // two-chunk unrolling exists for the single-level uniform walk
            if (unroll) {
                launch_uniform(march_uniform_kernel<MAXL, MINB, false, true>, smem, need, st, a);
                return;
            }
        }
        launch_uniform(march_uniform_kernel<MAXL, MINB, false>, smem, need, st, a);
    }
}

template <int MAXL>
void launch_walk(bool cone, bool occ, bool unroll, bool coarse, size_t smem, int need, cudaStream_t st,
                 const MarchArgs& a) {
    // The single-level uniform walk keeps one bitfield load in flight; it is built
    // for 64 registers (4 blocks of 256 threads per SM) and always launched so.
    if (MAXL == 1 && !cone && !unroll && !coarse) occ = true;
    if (occ) launch_variant<MAXL, 4>(cone, unroll, coarse, smem, need, st, a);
    else launch_variant<MAXL, 1>(cone, unroll, coarse, smem, need, st, a);
}


// Scene table upload for a batch of scenes: the host-formed SceneGeom entries
// reach the workspace as kernel parameters (no host buffer has to outlive the
// call, and the upload can be captured in a CUDA graph).
constexpr int kSceneChunk = 16;
struct SceneUpload {
    SceneGeom g[kSceneChunk];
    int32_t end[kSceneChunk];
    int32_t first, count;
    SceneGeom* dst;
    int32_t* dst_end;
};

__global__ void scene_upload_kernel(const __grid_constant__ SceneUpload u) {
    constexpr int kWords = (int)(sizeof(SceneGeom) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(u.g);
    uint32_t* dst = reinterpret_cast<uint32_t*>(u.dst + u.first);
    for (int i = threadIdx.x; i < u.count * kWords; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x < u.count) u.dst_end[u.first + threadIdx.x] = u.end[threadIdx.x];
}

// Batched variants: the uniform or cone walk, no two-chunk unrolling or coarse
// pass; one-level scenes with summed-area tables take the box walk.
template <int MAXL, int MINB, int BOX = 0>
void launch_batched(bool cone, size_t smem, int need, cudaStream_t st, const MarchArgs& a) {
    if (cone) launch_uniform(march_uniform_kernel<MAXL, MINB, true, false, false, true, BOX>, smem, need, st, a);
    else launch_uniform(march_uniform_kernel<MAXL, MINB, false, false, false, true, BOX>, smem, need, st, a);
}

// Resident blocks per SM the box walks are compiled for (their registers fit
// without spills).
constexpr int kBoxMinBlocks = 4;
constexpr size_t kBrickSmemMax = 16 * 1024;  // largest brick summary the walk keeps in shared memory
constexpr int kBoxBatchedMinBlocks = 3;

// One-level grid with its summed-area table: the box walk, ray by ray or (uniform
// steps, tuning knob: 1, 2, 3) the whole tile's chunks at once, compiled for 4, 5
// or 6 resident blocks per SM (55 registers; 48 and 40 with a few spills).
void launch_box(bool cone, int tile, size_t smem, int need, cudaStream_t st, const MarchArgs& a) {
    if (cone)
        launch_uniform(march_uniform_kernel<1, kBoxMinBlocks, true, false, false, false, 1>, smem, need, st, a);
    else if (tile == 1)
        launch_uniform(march_uniform_kernel<1, 4, false, false, false, false, 2>, smem, need, st, a);
    else if (tile == 2)
        launch_uniform(march_uniform_kernel<1, 5, false, false, false, false, 2>, smem, need, st, a);
    else if (tile == 3)
        launch_uniform(march_uniform_kernel<1, 6, false, false, false, false, 2>, smem, need, st, a);
    else
        launch_uniform(march_uniform_kernel<1, kBoxMinBlocks, false, false, false, false, 1>, smem, need, st, a);
}

// A scene's grid as a one-slot nacc_grid.
nacc_grid grid_of(const nacc_scene_desc& d) {
    nacc_grid g;
    g.bits = d.bits;
    for (int k = 0; k < 3; ++k) g.res[k] = d.res[k];
    g.n_levels = d.n_levels;
    g.n_slots = 1;
    for (int k = 0; k < 6; ++k) g.aabb[k] = d.aabb[k];
    g.contraction = d.contraction;
    g.sat = d.sat;
    return g;
}

size_t batched_table_bytes(int32_t n_scenes) {
    return align_up((size_t)n_scenes * sizeof(SceneGeom), 256) + align_up((size_t)n_scenes * sizeof(int32_t), 256);
}

// What nacc_march_rays and nacc_march_rays_batched share once the arguments are
// checked and `a` holds rays, step rule and geometry: outputs, workspace
// pointers, the cone table prologue, and the walk's launch.
int march_launch(MarchArgs& a, const nacc_march_params* p, int32_t* packed_info, float* t_starts, float* t_ends,
                 int32_t* ray_indices, int64_t capacity, int64_t* n_samples, int32_t* d_status, void* workspace,
                 cudaStream_t st, bool batched, bool box) {
    a.packed_info = packed_info;
    a.t_starts = t_starts;
    a.t_ends = t_ends;
    a.ray_indices = ray_indices;
    a.vec_out = ((((uintptr_t)t_starts | (uintptr_t)t_ends | (uintptr_t)ray_indices) & 15u) == 0) ? 1 : 0;
    a.capacity = capacity;
    a.n_samples = n_samples;
    a.d_status = d_status;
    a.ticket = (unsigned int*)workspace;
    a.lattice_points = (unsigned long long*)((char*)workspace + 8);
    a.tile_status = (unsigned long long*)((char*)workspace + kTicketBytes);
    a.hooks = lookback_hooks();
    const bool cone = p->cone > 0.0f;
    const bool occ = tune_get(NACC_TUNE_MARCH_OCCUPANCY) != 0;
    a.tile_rays = tile_rays_for(a.mask_words);

    a.n_tiles = (a.n_rays + a.tile_rays - 1) / a.tile_rays;
    const size_t clear = kTicketBytes + (size_t)a.n_tiles * sizeof(unsigned long long);
    cudaError_t e = cudaMemsetAsync(workspace, 0, clear, st);
    if (e != cudaSuccess) return NACC_ERR_CUDA;
    if (cone) {
        float* table = (float*)((char*)workspace + status_bytes_for(a.n_rays));
        a.cone_table = table;
        cone_table_kernel<<<1, 32, 0, st>>>(a, table);
    }
    size_t smem = (size_t)kWarps * 2 * a.tile_rays * a.row_stride * sizeof(uint32_t);
    // the box walk keeps the table's brick summary in shared memory when it is small
    a.bricks = nullptr;
    a.brick_entries = 0;
    if (!batched && box && a.sat && !a.contract) {
        const SatLayout L = sat_layout((long long)a.n_slots * a.n_levels, a.res0, a.res1, a.res2);
        const size_t entries = (size_t)a.n_slots * a.n_levels * L.per_grid;
        if (entries * sizeof(uint16_t) <= kBrickSmemMax) {
            a.bricks = a.sat + L.summary_offset;
            a.brick_entries = (int32_t)entries;
            a.brick_nb1 = L.nb1;
            a.brick_nb2 = L.nb2;
            a.brick_per_grid = (int32_t)L.per_grid;
            smem += align_up(entries * sizeof(uint16_t), 16);
        }
    }
    // cone steps over uncontracted grids: each block keeps the shared lattice in
    // shared memory when it fits
    a.cone_smem_at = -1;
    if (cone && !a.contract && a.max_steps + 1 <= kConeSmemMax) {
        smem = align_up(smem, 16);
        a.cone_smem_at = (int32_t)(smem / sizeof(float));
        smem += align_up((size_t)(a.max_steps + 1) * sizeof(float), 16);
    }
    const int need = (a.n_tiles + kWarps - 1) / kWarps;
    if (batched) {
        // one level in registers fits 4 blocks of 256 threads per SM like the
        // single-grid walk; cascades and contracted space run uncapped
        if (a.contract) launch_batched<0, 1>(cone, smem, need, st, a);
        else if (a.n_levels == 1 && box) launch_batched<1, kBoxBatchedMinBlocks, 1>(cone, smem, need, st, a);
        else if (a.n_levels == 1) launch_batched<1, 4>(cone, smem, need, st, a);
        else if (a.n_levels <= 4) launch_batched<4, 1>(cone, smem, need, st, a);
        else launch_batched<NACC_MAX_LEVELS, 1>(cone, smem, need, st, a);
        return launch_status(cudaGetLastError());
    }
    if (box && !a.contract && a.n_levels == 1) {
        launch_box(cone, tune_get(NACC_TUNE_MARCH_BOX_TILE), smem, need, st, a);
        return launch_status(cudaGetLastError());
    }
    if (box && !a.contract && a.n_levels <= 4) {  // cascades: the box walk over levels, 64 registers
        if (cone) launch_uniform(march_uniform_kernel<4, 4, true, false, false, false, 1>, smem, need, st, a);
        else launch_uniform(march_uniform_kernel<4, 4, false, false, false, false, 1>, smem, need, st, a);
        return launch_status(cudaGetLastError());
    }
    const bool unroll = tune_get(NACC_TUNE_MARCH_UNROLL) != 0;
    const bool coarse = tune_get(NACC_TUNE_MARCH_COARSE) != 0;
    if (a.contract) launch_walk<0>(cone, occ, false, false, smem, need, st, a);
    else if (a.n_levels == 1) launch_walk<1>(cone, occ, unroll, coarse, smem, need, st, a);
    else if (a.n_levels <= 4) launch_walk<4>(cone, occ, unroll, coarse, smem, need, st, a);
    else launch_walk<NACC_MAX_LEVELS>(cone, occ, unroll, coarse, smem, need, st, a);
    return launch_status(cudaGetLastError());
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_march_workspace_size(int32_t n_rays, const nacc_march_params* params) {
    if (n_rays < 0) return 0;
    return workspace_bytes_for(n_rays, params);
}

extern "C" int nacc_march_rays(const float* rays_o, const float* rays_d, const float* ray_time,
                               const int32_t* ray_slot, int32_t n_rays, const nacc_grid* grid,
                               const nacc_march_params* p, int32_t* packed_info, float* t_starts,
                               float* t_ends, int32_t* ray_indices, int64_t capacity,
                               int64_t* n_samples, int32_t* d_status, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (capacity < 0 || !n_samples) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (capacity > 0 && (!t_starts || !t_ends || !ray_indices)) return NACC_ERR_INVALID_ARG;
    MarchArgs a;
    const int setup = march_setup(rays_o, rays_d, ray_time, ray_slot, n_rays, grid, p, a);
    if (setup != NACC_OK) return setup;
    if (!workspace || workspace_bytes < workspace_bytes_for(n_rays, p)) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)packed_info & 7u) != 0) return NACC_ERR_INVALID_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays == 0) return launch_status(cudaMemsetAsync(n_samples, 0, sizeof(int64_t), st));
    return march_launch(a, p, packed_info, t_starts, t_ends, ray_indices, capacity, n_samples, d_status, workspace,
                        st, false, grid->sat != nullptr);
}

extern "C" size_t nacc_march_batched_workspace_size(int32_t n_scenes, int32_t n_rays,
                                                    const nacc_march_params* params) {
    if (n_rays < 0 || n_scenes < 0) return 0;
    return workspace_bytes_for(n_rays, params) + batched_table_bytes(n_scenes);
}

extern "C" int nacc_march_rays_batched(const nacc_scene_desc* scenes, int32_t n_scenes, const float* rays_o,
                                       const float* rays_d, int32_t n_rays, const nacc_march_params* p,
                                       int32_t* packed_info, float* t_starts, float* t_ends, int32_t* ray_indices,
                                       int64_t capacity, int64_t* n_samples, int32_t* d_status, void* workspace,
                                       size_t workspace_bytes, void* stream) {
    if (capacity < 0 || !n_samples || n_scenes < 1 || !scenes || !p || n_rays < 0) return NACC_ERR_INVALID_ARG;
    if (n_rays > 0 && !packed_info) return NACC_ERR_INVALID_ARG;
    if (capacity > 0 && (!t_starts || !t_ends || !ray_indices)) return NACC_ERR_INVALID_ARG;
    // every scene: a valid grid of its own, its consecutive rays; one contraction mode
    long long total = 0;
    int max_levels = 1, first_with_rays = -1;
    bool any_sat = false;
    for (int s = 0; s < n_scenes; ++s) {
        const nacc_scene_desc& d = scenes[s];
        const nacc_grid g = grid_of(d);
        if (check_grid(&g) != NACC_OK || d.n_rays < 0) return NACC_ERR_INVALID_ARG;
        if (d.contraction != scenes[0].contraction) return NACC_ERR_INVALID_ARG;
        if (d.n_rays > 0 && !d.bits) return NACC_ERR_INVALID_ARG;
        if (d.n_rays > 0 && first_with_rays < 0) first_with_rays = s;
        any_sat = any_sat || d.sat != nullptr;
        max_levels = d.n_levels > max_levels ? d.n_levels : max_levels;
        total += d.n_rays;
    }
    if (total != n_rays) return NACC_ERR_INVALID_ARG;
    const nacc_scene_desc& d0 = scenes[first_with_rays < 0 ? 0 : first_with_rays];
    const nacc_grid g0 = grid_of(d0);
    MarchArgs a;
    const int setup = march_setup(rays_o, rays_d, nullptr, nullptr, n_rays, &g0, p, a);
    if (setup != NACC_OK) return setup;
    const size_t base = workspace_bytes_for(n_rays, p);
    if (!workspace || workspace_bytes < base + batched_table_bytes(n_scenes)) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return NACC_ERR_INVALID_ARG;
    if (((uintptr_t)packed_info & 7u) != 0) return NACC_ERR_INVALID_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    if (n_rays == 0) return launch_status(cudaMemsetAsync(n_samples, 0, sizeof(int64_t), st));

    SceneGeom* table = (SceneGeom*)((char*)workspace + base);
    int32_t* ends = (int32_t*)((char*)table + align_up((size_t)n_scenes * sizeof(SceneGeom), 256));
    SceneUpload u;
    memset(&u, 0, sizeof(u));
    u.dst = table;
    u.dst_end = ends;
    int32_t end = 0;
    for (int s0 = 0; s0 < n_scenes; s0 += kSceneChunk) {
        u.first = s0;
        u.count = n_scenes - s0 < kSceneChunk ? n_scenes - s0 : kSceneChunk;
        for (int j = 0; j < u.count; ++j) {
            const nacc_scene_desc& d = scenes[s0 + j];
            scene_geom_for(grid_of(d), u.g[j]);
            end += d.n_rays;
            u.end[j] = end;
        }
        scene_upload_kernel<<<1, 256, 0, st>>>(u);
    }
    a.scenes = table;
    a.scene_end = ends;
    a.n_scenes = n_scenes;
    a.n_levels = max_levels;
    a.contract = scenes[0].contraction;
    return march_launch(a, p, packed_info, t_starts, t_ends, ray_indices, capacity, n_samples, d_status, workspace,
                        st, true, any_sat);
}
