/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for occupancy-grid ray
 * marching and packed differentiable volume rendering (NerfAcc, arXiv
 * 2210.04847, Sec. 2 "Design": 2.1 Ray Marching, 2.2 Differentiable Rendering,
 * Eq. 1).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference arm may load this file's library. It shares no code,
 * header, table or constant generator with the CUDA library; the two agree
 * only because both follow the paper and the readings listed below.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -lm
 * (-ffp-contract=off keeps every float product and sum separately rounded;
 * GCC contracts a*b+c into an FMA by default on aarch64.)
 *
 * Precision, per step:
 *   marching         IEEE float32 replica (its output is integer: which lattice
 *                    intervals are emitted); no skipping, every lattice point
 *                    of every ray is visited.
 *   prune decision   float32 (the decision T_i >= eps, alpha_i >= thre decides
 *                    an integer mask, so it is taken in the kernel's precision).
 *   rendering, its gradient, accumulation: float64.
 *   grid update      float64 product of two float32 numbers (exact), stored to
 *                    the float32 state grid (so it equals a correctly rounded
 *                    float32 product); bits thresholded on the stored value.
 *   density field    float32 replica of a fixed operation order (its values
 *                    feed the fused path's keep decision, an integer result).
 *
 * Readings of the paper (it is silent on all of these):
 *   M1 ray-box clip: slab test per axis in float32; an axis with d == 0 keeps
 *      the ray iff lo <= o <= hi; t_in = max of per-axis entries, t_out = min
 *      of exits; near = max(t_in, near_plane), far = min(t_out, far_plane);
 *      no samples unless near < far; a ray with a non-finite component emits
 *      nothing. The clipping box is the outermost cascade level.
 *   M2 lattice: uniform t_k = near + k*dt (product then sum); cone
 *      t_{k+1} = t_k + clamp(t_k*cone, dt_min, dt_max). Interval k is
 *      [t_k, min(t_{k+1}, far)], a candidate iff t_k < far and k < max_steps.
 *   M3 lookup at the interval midpoint (the point the paper's callbacks query):
 *      mid = (t_s + t_e)*0.5, x = o + d*mid; the level is the finest level
 *      whose box holds x; cell i_a = floor((x_a - lo_a) * scale_a) with
 *      scale_a = res_a / (hi_a - lo_a); out of every box = empty.
 *   M4 output ray-major, ascending k; packed_info[r] = (offset, count).
 *   M5 grid slot of a ray: ray_slot[r] if given, else the time bin
 *      clamp(floor(time * n_slots), 0, n_slots-1) if ray_time is given, else 0.
 *   V1 prune (Sec. 2.1 "Pruning Empty and Occluded Regions"): with
 *      tau_i = sigma_i*(t_e - t_s) and O_i = sum_{j<i} tau_j over all marched
 *      samples of the ray, keep iff T_i = exp(-O_i) >= eps and
 *      alpha_i = 1 - exp(-tau_i) >= thre, taken as O_i <= -ln(eps) and
 *      tau_i >= -ln(1 - thre) (thresholds rounded once to float32);
 *      eps <= 0 or thre <= 0 switches that test off.
 *   R1 Eq. 1 with alpha_i = 1 - exp(-sigma_i delta_i) (the printed formula
 *      drops the minus sign), delta_i = t_e - t_s.
 *   R2 w_i = T_i alpha_i; color = sum w rgb; opacity = sum w;
 *      depth = sum w (t_s + t_e)/2 (unnormalised, black background).
 *   R5 gradient (ours, calculus on Eq. 1): with a_i = <g_C, rgb_i> + g_A +
 *      g_D tmid_i, dL/dtau_k = a_k T_{k+1} - sum_{i>k} a_i w_i,
 *      dL/dsigma_k = delta_k dL/dtau_k, dL/drgb_k = w_k g_C.
 *   F1 density field of the fused inference path: trilinear between the
 *      vertex values of a lattice over a box, zero outside (see F1 below).
 *   F2 fused march + prune: V1 applied to the M1-M4 samples with F1's sigma
 *      at each sample's midpoint (see F2 below).
 *   G2 grid update: ema <- decay*ema for every cell, then
 *      ema[c] <- max(ema[c], sigma_s) for each sample s in cell c (NaN sigma
 *      ignored); bits = ema > thre.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_LEVELS 16

/* ----- marching: float32 replica ----------------------------------------- */

typedef struct {
    float lo[OR_MAX_LEVELS][3];
    float hi[OR_MAX_LEVELS][3];
    float scale[OR_MAX_LEVELS][3];
} or_levels;

/* Level boxes (M3): level 0 is the given box; level l >= 1 is the level-0 box
 * scaled by 2^l about its centre, c +- h*2^l with c = (lo+hi)/2, h = (hi-lo)/2. */
static void or_make_levels(const float aabb[6], int n_levels, const int32_t res[3], or_levels* L) {
    for (int a = 0; a < 3; ++a) {
        float lo = aabb[a], hi = aabb[3 + a];
        float c = (lo + hi) * 0.5f;
        float h = (hi - lo) * 0.5f;
        for (int l = 0; l < n_levels; ++l) {
            float llo, lhi;
            if (l == 0) {
                llo = lo;
                lhi = hi;
            } else {
                float hl = h * ldexpf(1.0f, l);
                llo = c - hl;
                lhi = c + hl;
            }
            L->lo[l][a] = llo;
            L->hi[l][a] = lhi;
            L->scale[l][a] = (float)res[a] / (lhi - llo);
        }
    }
}

static int or_finite(float v) { return fabsf(v) <= 3.402823466e+38f; }

/* M1: returns 1 and sets near/far when the ray has samples to march. */
static int or_clip(const float o[3], const float d[3], const float lo[3], const float hi[3],
                   float near_plane, float far_plane, float* near_out, float* far_out) {
    for (int a = 0; a < 3; ++a)
        if (!or_finite(o[a]) || !or_finite(d[a])) return 0;
    float t_in = -INFINITY, t_out = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
            continue;
        }
        float inv = 1.0f / d[a];
        float t0 = (lo[a] - o[a]) * inv;
        float t1 = (hi[a] - o[a]) * inv;
        float tmin = t0 < t1 ? t0 : t1;
        float tmax = t0 < t1 ? t1 : t0;
        if (tmin > t_in) t_in = tmin;
        if (tmax < t_out) t_out = tmax;
    }
    float near = t_in > near_plane ? t_in : near_plane;
    float far = t_out < far_plane ? t_out : far_plane;
    if (!(near < far)) return 0;
    *near_out = near;
    *far_out = far;
    return 1;
}

static int or_slot(const float* ray_time, const int32_t* ray_slot, int32_t r, int32_t n_slots) {
    if (ray_slot) return ray_slot[r];
    if (ray_time) {
        float v = ray_time[r] * (float)n_slots;
        if (v >= 0.0f && v < (float)n_slots) return (int)v;
        if (v >= (float)n_slots) return n_slots - 1;
        return 0;
    }
    return 0;
}

/* M3: occupancy bit of point x for grid slot `slot`. */
static int or_occupied(const float x[3], int slot, const uint32_t* bits, const int32_t res[3],
                       int n_levels, const or_levels* L) {
    for (int l = 0; l < n_levels; ++l) {
        float u[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            u[a] = (x[a] - L->lo[l][a]) * L->scale[l][a];
            if (!(u[a] >= 0.0f && u[a] < (float)res[a])) inside = 0;
        }
        if (!inside) continue;
        int64_t ix = (int64_t)u[0], iy = (int64_t)u[1], iz = (int64_t)u[2];
        int64_t cell = (((int64_t)slot * n_levels + l) * res[0] + ix) * res[1];
        cell = (cell + iy) * res[2] + iz;
        return (int)((bits[cell >> 5] >> (cell & 31)) & 1u);
    }
    return 0;
}

/* M3 for unbounded scenes (Sec. 2.1 "Scene Contraction", the contraction of
 * Mip-NeRF 360's Eq. 10): x normalised by the box, x_n = (x - c) * (1/h); inside
 * the unit ball (|x_n|^2 <= 1) unchanged, outside scaled by (2 - 1/|x_n|)/|x_n|;
 * the grid spans [-2, 2]^3: u = (x_c + 2) * (res/4), empty outside [0, res). */
static int or_occupied_contracted(const float x[3], int slot, const uint32_t* bits, const int32_t res[3],
                                  const float c[3], const float inv_h[3]) {
    float xn[3], u[3];
    for (int a = 0; a < 3; ++a) xn[a] = (x[a] - c[a]) * inv_h[a];
    float n2 = (xn[0] * xn[0] + xn[1] * xn[1]) + xn[2] * xn[2];
    if (!(n2 <= 1.0f)) {
        float n = sqrtf(n2);
        float sc = (2.0f - 1.0f / n) / n;
        for (int a = 0; a < 3; ++a) xn[a] = xn[a] * sc;
    }
    for (int a = 0; a < 3; ++a) {
        u[a] = (xn[a] + 2.0f) * ((float)res[a] * 0.25f);
        if (!(u[a] >= 0.0f && u[a] < (float)res[a])) return 0;
    }
    int64_t ix = (int64_t)u[0], iy = (int64_t)u[1], iz = (int64_t)u[2];
    int64_t cell = (((int64_t)slot * res[0] + ix) * res[1] + iy) * res[2] + iz;
    return (int)((bits[cell >> 5] >> (cell & 31)) & 1u);
}

/* Ray marching (Sec. 2.1): returns the total number of emitted samples;
 * writes packed_info for every ray and samples up to `capacity`. With
 * contraction (one level) rays are not clipped: they march [near_plane, far_plane]. */
int64_t oracle_march(const float* rays_o, const float* rays_d, const float* ray_time,
                     const int32_t* ray_slot, int32_t n_rays, const uint32_t* bits,
                     const int32_t res[3], int32_t n_levels, int32_t n_slots, const float aabb[6],
                     float near_plane, float far_plane, float dt_min, float dt_max, float cone,
                     int32_t max_steps, int32_t contraction, int32_t* packed_info, float* t_starts,
                     float* t_ends, int32_t* ray_indices, int64_t capacity) {
    or_levels L;
    if (n_levels < 1 || n_levels > OR_MAX_LEVELS) return -1;
    if (contraction && n_levels != 1) return -1;
    or_make_levels(aabb, n_levels, res, &L);
    float cc[3], inv_h[3];
    for (int a = 0; a < 3; ++a) {
        cc[a] = (aabb[a] + aabb[3 + a]) * 0.5f;
        inv_h[a] = 1.0f / ((aabb[3 + a] - aabb[a]) * 0.5f);
    }
    const float* blo = L.lo[n_levels - 1];
    const float* bhi = L.hi[n_levels - 1];
    int64_t total = 0;
    for (int32_t r = 0; r < n_rays; ++r) {
        const float* o = rays_o + 3 * (int64_t)r;
        const float* d = rays_d + 3 * (int64_t)r;
        int64_t start = total;
        float near, far;
        int slot = or_slot(ray_time, ray_slot, r, n_slots);
        int marching;
        if (contraction) {
            marching = or_finite(o[0]) && or_finite(o[1]) && or_finite(o[2]) && or_finite(d[0]) &&
                       or_finite(d[1]) && or_finite(d[2]) && near_plane < far_plane;
            near = near_plane;
            far = far_plane;
        } else {
            marching = or_clip(o, d, blo, bhi, near_plane, far_plane, &near, &far);
        }
        if (slot >= 0 && slot < n_slots && marching) {
            float t = near;
            for (int32_t k = 0; k < max_steps; ++k) {
                float ts, tn;
                if (cone == 0.0f) {
                    ts = near + (float)k * dt_min;
                    tn = near + (float)(k + 1) * dt_min;
                } else {
                    float dt = t * cone;
                    if (dt < dt_min) dt = dt_min;
                    if (dt > dt_max) dt = dt_max;
                    ts = t;
                    tn = t + dt;
                    t = tn;
                }
                if (!(ts < far)) break;
                float te = tn < far ? tn : far;
                float mid = (ts + te) * 0.5f;
                float x[3];
                for (int a = 0; a < 3; ++a) x[a] = o[a] + d[a] * mid;
                if (contraction ? or_occupied_contracted(x, slot, bits, res, cc, inv_h)
                                : or_occupied(x, slot, bits, res, n_levels, &L)) {
                    if (total < capacity) {
                        t_starts[total] = ts;
                        t_ends[total] = te;
                        ray_indices[total] = r;
                    }
                    ++total;
                }
            }
        }
        packed_info[2 * (int64_t)r] = (int32_t)start;
        packed_info[2 * (int64_t)r + 1] = (int32_t)(total - start);
    }
    return total;
}

/* ----- prune (early stop + alpha threshold), float32 decision ------------- */

int64_t oracle_prune(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                     const float* t_ends, const float* sigmas, float early_stop_eps, float alpha_thre,
                     uint8_t* keep /* nullable, per input sample */,
                     float* optical_depth /* nullable, per input sample: O_i */,
                     int32_t* packed_info_out, float* t_starts_out, float* t_ends_out,
                     int32_t* ray_indices_out, int64_t capacity) {
    int use_t = early_stop_eps > 0.0f;
    int use_a = alpha_thre > 0.0f;
    float thr_o = use_t ? (float)(-log((double)early_stop_eps)) : INFINITY;
    float thr_tau = use_a ? (float)(-log1p(-(double)alpha_thre)) : 0.0f;
    int64_t total = 0;
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        int64_t start = total;
        float o_acc = 0.0f;
        for (int64_t i = off; i < off + cnt; ++i) {
            float delta = t_ends[i] - t_starts[i];
            float tau = sigmas[i] * delta;
            int k = 1;
            if (use_t && !(o_acc <= thr_o)) k = 0;
            if (use_a && !(tau >= thr_tau)) k = 0;
            if (keep) keep[i] = (uint8_t)k;
            if (optical_depth) optical_depth[i] = o_acc;
            if (k) {
                if (total < capacity) {
                    t_starts_out[total] = t_starts[i];
                    t_ends_out[total] = t_ends[i];
                    ray_indices_out[total] = r;
                }
                ++total;
            }
            o_acc = o_acc + tau;
        }
        packed_info_out[2 * (int64_t)r] = (int32_t)start;
        packed_info_out[2 * (int64_t)r + 1] = (int32_t)(total - start);
    }
    return total;
}

/* ----- rendering: float64 -------------------------------------------------- */

/* Eq. 1 weights of one ray (R1, R2): T_i = exp(-sum_{j<i} tau_j),
 * alpha_i = 1 - exp(-tau_i), w_i = T_i alpha_i. */
static void or_ray_weights(int64_t off, int64_t cnt, const float* ts, const float* te, const float* sg,
                           double* w, double* T, double* T_next) {
    double o_acc = 0.0;
    for (int64_t i = 0; i < cnt; ++i) {
        double delta = (double)te[off + i] - (double)ts[off + i];
        double tau = (double)sg[off + i] * delta;
        double Ti = exp(-o_acc);
        double ai = 1.0 - exp(-tau);
        T[i] = Ti;
        w[i] = Ti * ai;
        o_acc += tau;
        if (T_next) T_next[i] = exp(-o_acc);
    }
}

static int64_t or_max_count(const int32_t* packed_info, int32_t n_rays) {
    int64_t m = 1;
    for (int32_t r = 0; r < n_rays; ++r)
        if (packed_info[2 * (int64_t)r + 1] > m) m = packed_info[2 * (int64_t)r + 1];
    return m;
}

/* render_weights: per-sample weights and transmittance (nullable outputs). */
int oracle_render_weights(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                          const float* t_ends, const float* sigmas, double* weights, double* trans) {
    int64_t m = or_max_count(packed_info, n_rays);
    double* w = (double*)malloc(sizeof(double) * m);
    double* T = (double*)malloc(sizeof(double) * m);
    if (!w || !T) { free(w); free(T); return -1; }
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        or_ray_weights(off, cnt, t_starts, t_ends, sigmas, w, T, NULL);
        for (int64_t i = 0; i < cnt; ++i) {
            if (weights) weights[off + i] = w[i];
            if (trans) trans[off + i] = T[i];
        }
    }
    free(w);
    free(T);
    return 0;
}

/* accumulate_along_rays: out[r, c] = sum_i w_i v_i[c]; v == NULL means v = 1. */
int oracle_accumulate(const int32_t* packed_info, int32_t n_rays, const double* weights,
                      const float* values, int32_t n_channels, double* out) {
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        for (int32_t c = 0; c < n_channels; ++c) {
            double acc = 0.0;
            for (int64_t i = off; i < off + cnt; ++i)
                acc += weights[i] * (values ? (double)values[i * n_channels + c] : 1.0);
            out[(int64_t)r * n_channels + c] = acc;
        }
    }
    return 0;
}

/* Forward rendering (Eq. 1, R2): color (R,3), opacity (R,), depth (R,). */
int oracle_render_fwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                      const float* t_ends, const float* sigmas, const float* rgbs, double* color,
                      double* opacity, double* depth) {
    int64_t m = or_max_count(packed_info, n_rays);
    double* w = (double*)malloc(sizeof(double) * m);
    double* T = (double*)malloc(sizeof(double) * m);
    if (!w || !T) { free(w); free(T); return -1; }
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        or_ray_weights(off, cnt, t_starts, t_ends, sigmas, w, T, NULL);
        double c0 = 0, c1 = 0, c2 = 0, a = 0, dd = 0;
        for (int64_t i = 0; i < cnt; ++i) {
            const float* rgb = rgbs + 3 * (off + i);
            double tmid = ((double)t_starts[off + i] + (double)t_ends[off + i]) * 0.5;
            c0 += w[i] * rgb[0];
            c1 += w[i] * rgb[1];
            c2 += w[i] * rgb[2];
            a += w[i];
            dd += w[i] * tmid;
        }
        color[3 * (int64_t)r] = c0;
        color[3 * (int64_t)r + 1] = c1;
        color[3 * (int64_t)r + 2] = c2;
        opacity[r] = a;
        depth[r] = dd;
    }
    free(w);
    free(T);
    return 0;
}

/* Gradient of the forward rendering (R5). g_* nullable (zero). */
int oracle_render_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                      const float* t_ends, const float* sigmas, const float* rgbs,
                      const double* g_color, const double* g_opacity, const double* g_depth,
                      double* d_sigmas, double* d_rgbs) {
    int64_t m = or_max_count(packed_info, n_rays);
    double* w = (double*)malloc(sizeof(double) * m);
    double* T = (double*)malloc(sizeof(double) * m);
    double* Tn = (double*)malloc(sizeof(double) * m);
    if (!w || !T || !Tn) { free(w); free(T); free(Tn); return -1; }
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        or_ray_weights(off, cnt, t_starts, t_ends, sigmas, w, T, Tn);
        double gc0 = g_color ? g_color[3 * (int64_t)r] : 0.0;
        double gc1 = g_color ? g_color[3 * (int64_t)r + 1] : 0.0;
        double gc2 = g_color ? g_color[3 * (int64_t)r + 2] : 0.0;
        double ga = g_opacity ? g_opacity[r] : 0.0;
        double gd = g_depth ? g_depth[r] : 0.0;
        /* sum_{i>k} a_i w_i, accumulated from the end of the ray */
        double suffix = 0.0;
        for (int64_t k = cnt - 1; k >= 0; --k) {
            const float* rgb = rgbs + 3 * (off + k);
            double tmid = ((double)t_starts[off + k] + (double)t_ends[off + k]) * 0.5;
            double ak = gc0 * rgb[0] + gc1 * rgb[1] + gc2 * rgb[2] + ga + gd * tmid;
            double delta = (double)t_ends[off + k] - (double)t_starts[off + k];
            double dtau = ak * Tn[k] - suffix;
            d_sigmas[off + k] = delta * dtau;
            d_rgbs[3 * (off + k)] = w[k] * gc0;
            d_rgbs[3 * (off + k) + 1] = w[k] * gc1;
            d_rgbs[3 * (off + k) + 2] = w[k] * gc2;
            suffix += ak * w[k];
        }
    }
    free(w);
    free(T);
    free(Tn);
    return 0;
}

/* Gradient of the weights alone for an upstream g_i = dL/dw_i: with
 * w_i = T_i alpha_i, dw_i/dtau_k = -w_i (k < i), T_{i+1} (k = i), 0 (k > i), so
 * dL/dtau_k = g_k T_{k+1} - sum_{i>k} g_i w_i and dL/dsigma_k = delta_k dL/dtau_k
 * (the R5 derivation with a_i = g_i). */
int oracle_render_weights_bwd(const int32_t* packed_info, int32_t n_rays, const float* t_starts,
                              const float* t_ends, const float* sigmas, const double* g_weights,
                              double* d_sigmas) {
    int64_t m = or_max_count(packed_info, n_rays);
    double* w = (double*)malloc(sizeof(double) * m);
    double* T = (double*)malloc(sizeof(double) * m);
    double* Tn = (double*)malloc(sizeof(double) * m);
    if (!w || !T || !Tn) { free(w); free(T); free(Tn); return -1; }
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        or_ray_weights(off, cnt, t_starts, t_ends, sigmas, w, T, Tn);
        double suffix = 0.0;
        for (int64_t k = cnt - 1; k >= 0; --k) {
            double gk = g_weights[off + k];
            double delta = (double)t_ends[off + k] - (double)t_starts[off + k];
            d_sigmas[off + k] = delta * (gk * Tn[k] - suffix);
            suffix += gk * w[k];
        }
    }
    free(w);
    free(T);
    free(Tn);
    return 0;
}

/* Gradient of the accumulation out[r, c] = sum_i w_i v_i[c]:
 * dL/dw_i = sum_c g[r, c] v_i[c] (v = 1 without values), dL/dv_i[c] = w_i g[r, c]. */
int oracle_accumulate_bwd(const int32_t* packed_info, int32_t n_rays, const double* weights,
                          const float* values, int32_t n_channels, const double* g_out, double* d_weights,
                          double* d_values) {
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        for (int64_t i = off; i < off + cnt; ++i) {
            double dw = 0.0;
            for (int32_t c = 0; c < n_channels; ++c) {
                double g = g_out[(int64_t)r * n_channels + c];
                dw += values ? g * (double)values[i * n_channels + c] : g;
                if (d_values) d_values[i * n_channels + c] = weights[i] * g;
            }
            d_weights[i] = dw;
        }
    }
    return 0;
}

/* Ray index of every packed sample (the inverse of packed_info). */
int oracle_unpack_info(const int32_t* packed_info, int32_t n_rays, int32_t* ray_indices) {
    for (int32_t r = 0; r < n_rays; ++r) {
        int64_t off = packed_info[2 * (int64_t)r], cnt = packed_info[2 * (int64_t)r + 1];
        for (int64_t i = off; i < off + cnt; ++i) ray_indices[i] = r;
    }
    return 0;
}

/* ----- occupancy-grid update (G2) ----------------------------------------- */

int oracle_update_grid(float* ema, uint32_t* bits, int64_t n_cells, const int32_t* cells,
                       const float* sigmas, int64_t n_samples, float decay, float thre) {
    for (int64_t c = 0; c < n_cells; ++c) ema[c] = (float)((double)decay * (double)ema[c]);
    for (int64_t s = 0; s < n_samples; ++s) {
        int64_t c = cells[s];
        if (c < 0 || c >= n_cells) return -1;
        float v = sigmas[s];
        if (v == v && v > ema[c]) ema[c] = v;
    }
    int64_t n_words = (n_cells + 31) / 32;
    memset(bits, 0, sizeof(uint32_t) * (size_t)n_words);
    for (int64_t c = 0; c < n_cells; ++c)
        if (ema[c] > thre) bits[c >> 5] |= 1u << (c & 31);
    return 0;
}

/* ----- density field and the fused march + prune (inference) ------------- */

/* F1: the density field of the fused path is a grid of sigma values at the
 * vertices of a G0 x G1 x G2 lattice over the box [lo, hi] (vertex (i, j, k) at
 * lo + (hi - lo) * (i, j, k) / (G - 1), z fastest in memory), interpolated
 * trilinearly between vertices, and zero outside the box. Float32 in this order:
 * s_a = (G_a - 1) / (hi_a - lo_a); u_a = (x_a - lo_a) * s_a; outside unless
 * 0 <= u_a <= G_a - 1; i_a = min(floor(u_a), G_a - 2); f_a = u_a - i_a;
 * lerp(p, q, f) = p + f * (q - p) along z, then y, then x. */
static float or_lerp(float p, float q, float f) { return p + f * (q - p); }

float oracle_field_sigma(const float* grid, const int32_t G[3], const float box[6], const float x[3]) {
    int i[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
        float s = (float)(G[a] - 1) / (box[3 + a] - box[a]);
        float u = (x[a] - box[a]) * s;
        if (!(u >= 0.0f && u <= (float)(G[a] - 1))) return 0.0f;
        i[a] = (int)floorf(u);
        if (i[a] > G[a] - 2) i[a] = G[a] - 2;
        f[a] = u - (float)i[a];
    }
    float v[2][2][2];
    for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
            for (int dz = 0; dz < 2; ++dz)
                v[dx][dy][dz] = grid[((int64_t)(i[0] + dx) * G[1] + (i[1] + dy)) * G[2] + (i[2] + dz)];
    float c00 = or_lerp(v[0][0][0], v[0][0][1], f[2]);
    float c01 = or_lerp(v[0][1][0], v[0][1][1], f[2]);
    float c10 = or_lerp(v[1][0][0], v[1][0][1], f[2]);
    float c11 = or_lerp(v[1][1][0], v[1][1][1], f[2]);
    float c0 = or_lerp(c00, c01, f[1]);
    float c1 = or_lerp(c10, c11, f[1]);
    return or_lerp(c0, c1, f[0]);
}

static int or_field_ok(const int32_t G[3], const float box[6]) {
    for (int a = 0; a < 3; ++a)
        if (G[a] < 2 || !(box[a] < box[3 + a])) return 0;
    return 1;
}

int oracle_field_query(const float* grid, const int32_t G[3], const float box[6], const float* xyz, int64_t n,
                       float* sigmas) {
    if (!or_field_ok(G, box)) return -1;
    for (int64_t s = 0; s < n; ++s) sigmas[s] = oracle_field_sigma(grid, G, box, xyz + 3 * s);
    return 0;
}

/* F2, the fused path (Sec. 2.1 "Pruning Empty and Occluded Regions": the
 * transmittance is taken from the field's density while marching, and marching
 * ends where it falls below eps). Its result is, by definition, what V1 keeps of
 * the samples M1-M4 emit, with sigma_i = F1 at the midpoint x = o + d*mid that
 * M3 looks up: the march stops where the optical depth passes -ln(eps), which
 * changes the work done but not the samples kept. Written here as exactly that
 * composition. sigmas_out (nullable) receives sigma of each kept sample. */
int64_t oracle_march_fused(const float* rays_o, const float* rays_d, int32_t n_rays, const uint32_t* bits,
                           const int32_t res[3], int32_t n_levels, const float aabb[6], float near_plane,
                           float far_plane, float dt_min, float dt_max, float cone, int32_t max_steps,
                           int32_t contraction, const float* field, const int32_t G[3], const float fbox[6],
                           float early_stop_eps, float alpha_thre, int32_t* packed_info_out, float* t_starts_out,
                           float* t_ends_out, int32_t* ray_indices_out, float* sigmas_out, int64_t capacity) {
    if (!or_field_ok(G, fbox)) return -1;
    int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(n_rays > 0 ? n_rays : 1));
    if (!pi) return -1;
    int64_t m = oracle_march(rays_o, rays_d, NULL, NULL, n_rays, bits, res, n_levels, 1, aabb, near_plane, far_plane,
                             dt_min, dt_max, cone, max_steps, contraction, pi, NULL, NULL, NULL, 0);
    if (m < 0) {
        free(pi);
        return -1;
    }
    size_t mm = (size_t)(m > 0 ? m : 1);
    float* ts = (float*)malloc(sizeof(float) * mm);
    float* te = (float*)malloc(sizeof(float) * mm);
    int32_t* ri = (int32_t*)malloc(sizeof(int32_t) * mm);
    float* sg = (float*)malloc(sizeof(float) * mm);
    uint8_t* keep = (uint8_t*)malloc(mm);
    int64_t total = -1;
    if (ts && te && ri && sg && keep) {
        oracle_march(rays_o, rays_d, NULL, NULL, n_rays, bits, res, n_levels, 1, aabb, near_plane, far_plane, dt_min,
                     dt_max, cone, max_steps, contraction, pi, ts, te, ri, m);
        for (int64_t i = 0; i < m; ++i) {
            const float* o = rays_o + 3 * (int64_t)ri[i];
            const float* d = rays_d + 3 * (int64_t)ri[i];
            float mid = (ts[i] + te[i]) * 0.5f;
            float x[3];
            for (int a = 0; a < 3; ++a) x[a] = o[a] + d[a] * mid;
            sg[i] = oracle_field_sigma(field, G, fbox, x);
        }
        total = oracle_prune(pi, n_rays, ts, te, sg, early_stop_eps, alpha_thre, keep, NULL, packed_info_out,
                             t_starts_out, t_ends_out, ray_indices_out, capacity);
        if (sigmas_out) {
            int64_t j = 0;
            for (int64_t i = 0; i < m; ++i)
                if (keep[i]) {
                    if (j < capacity) sigmas_out[j] = sg[i];
                    ++j;
                }
        }
    }
    free(pi);
    free(ts);
    free(te);
    free(ri);
    free(sg);
    free(keep);
    return total;
}
