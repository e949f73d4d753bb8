"""Pins of the oracle's rendering (Eq. 1, Sec. 2.2), its gradient, pruning (Sec. 2.1
"Pruning Empty and Occluded Regions") and grid update against closed forms,
hand-derived values, central finite differences and exact float64 decisions.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _packed(counts):
    counts = np.asarray(counts, np.int64)
    off = np.concatenate([[0], np.cumsum(counts)[:-1]])
    return np.stack([off, counts], 1).astype(np.int32)


# ---------------------------------------------------------------------------
# forward quadrature
# ---------------------------------------------------------------------------


def test_worked_example(orc):
    g = json.load(open(os.path.join(GOLDEN, "render_worked_example.json")))
    sig = np.array([2 * math.log(2), 0.0, 2 * math.log(4)], np.float32)
    col, op, dp = orc.render_fwd(g["packed_info"], g["t_starts"], g["t_ends"], sig, g["rgbs"])
    assert np.allclose(col, g["color"], atol=1e-6)
    assert np.allclose(op, g["opacity"], atol=1e-6)
    assert np.allclose(dp, g["depth"], atol=1e-6)
    w, T = orc.render_weights(g["packed_info"], g["t_starts"], g["t_ends"], sig)
    assert np.allclose(w, g["weights"], atol=1e-6) and np.allclose(T, g["transmittance"], atol=1e-6)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 1000])
def test_constant_density_slab(orc, n):
    """Constant sigma on [near, far]: opacity = 1 - exp(-sigma L) for ANY split of L."""
    sigma, near, L = 1.75, 0.5, 2.0
    cuts = np.sort(synth.rand_uniform(n, 1, n - 1, near, near + L)) if n > 1 else np.array([])
    edges = np.concatenate([[near], cuts, [near + L]]).astype(np.float32)
    ts, te = edges[:-1], edges[1:]
    Lf = float(np.float64(te[-1]) - np.float64(ts[0]))
    col, op, dp = orc.render_fwd(_packed([n]), ts, te, np.full(n, sigma, np.float32), np.full((n, 3), 0.3, np.float32))
    assert abs(op[0] - (1 - math.exp(-np.float32(sigma) * Lf))) < 1e-12
    assert np.allclose(col[0], 0.3 * op[0], atol=1e-6)  # constant colour: color = c * opacity
    w, T = orc.render_weights(_packed([n]), ts, te, np.full(n, sigma, np.float32))
    assert np.all(w >= 0) and abs(w.sum() - op[0]) < 1e-12
    # telescoping: sum w = 1 - T_{N+1}
    assert abs(w.sum() - (1 - T[-1] * math.exp(-np.float32(sigma) * (np.float64(te[-1]) - ts[-1])))) < 1e-12


def test_constant_density_depth_geometric_series(orc):
    """Uniform delta, constant sigma: D = sum_i q^i (1-q) tmid_i, q = exp(-sigma delta), in closed form."""
    n, near, delta, sigma = 50, 1.0, 0.0625, 3.0
    ts = (near + delta * np.arange(n)).astype(np.float32)
    te = (near + delta * np.arange(1, n + 1)).astype(np.float32)
    _, op, dp = orc.render_fwd(_packed([n]), ts, te, np.full(n, sigma, np.float32), np.zeros((n, 3), np.float32))
    q = math.exp(-sigma * delta)
    geo = (1 - q**n) / (1 - q)
    ar = q * (1 - n * q ** (n - 1) + (n - 1) * q**n) / (1 - q) ** 2  # sum_{i<n} i q^i
    D = (1 - q) * ((near + 0.5 * delta) * geo + delta * ar)
    assert abs(dp[0] - D) < 1e-12
    assert abs(op[0] - (1 - q**n)) < 1e-12


def test_special_cases(orc):
    # zero density: nothing; one sample: w = alpha; huge density on sample 1: w_1 = 1
    pi = _packed([3, 1, 4, 0])
    ts = np.array([0, 1, 2, 5, 0, 0.5, 1.0, 1.5], np.float32)
    te = ts + np.float32(0.5)
    sg = np.array([0, 0, 0, 2.0, 1e30, 1, 1, 1], np.float32)
    rgb = synth.rand_uniform(1, 1, 24).reshape(8, 3).astype(np.float32)
    col, op, dp = orc.render_fwd(pi, ts, te, sg, rgb)
    assert op[0] == 0 and np.all(col[0] == 0) and dp[0] == 0
    assert abs(op[1] - (1 - math.exp(-1.0))) < 1e-15
    assert op[2] == 1.0 and np.allclose(col[2], rgb[4]) and dp[2] == 0.25
    assert op[3] == 0 and dp[3] == 0
    w, T = orc.render_weights(pi, ts, te, sg)
    assert np.all((w >= 0) & (w <= 1)) and np.all(T[5:8] == 0)


def test_accumulate_is_linear_and_matches_render(orc):
    rng = synth.rand_uniform(3, 1, 200)
    counts = [5, 0, 17, 1, 9]
    M = sum(counts)
    pi = _packed(counts)
    ts = np.sort(rng[:M]).astype(np.float32)
    te = ts + np.float32(0.05)
    sg = (rng[M : 2 * M] * 20).astype(np.float32)
    rgb = rng[2 * M : 5 * M].reshape(M, 3).astype(np.float32)
    w, _ = orc.render_weights(pi, ts, te, sg)
    col, op, dp = orc.render_fwd(pi, ts, te, sg, rgb)
    assert np.allclose(orc.accumulate(pi, w)[:, 0], op, atol=1e-15)
    assert np.allclose(orc.accumulate(pi, w, rgb), col, atol=1e-15)
    mid = ((ts.astype(np.float64) + te) * 0.5).astype(np.float32)
    assert np.allclose(orc.accumulate(pi, w, mid)[:, 0], dp, atol=1e-6)
    v2 = np.concatenate([rgb, 2 * rgb], 1)
    acc2 = orc.accumulate(pi, w, v2)
    assert np.allclose(acc2[:, 3:], 2 * acc2[:, :3], atol=1e-15)


# ---------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------


def _loss(orc, pi, ts, te, sg, rgb, gc, ga, gd):
    col, op, dp = orc.render_fwd(pi, ts, te, sg, rgb)
    return float((col * gc).sum() + (op * ga).sum() + (dp * gd).sum())


@pytest.mark.parametrize("seed", range(4))
def test_gradient_central_differences(orc, seed):
    """Analytic gradient vs central differences of the float64 forward. Inputs are dyadic
    (multiples of 2^-10) and the step is 2^-12, so sigma +- h and rgb +- h are exact in float32."""
    counts = [1 + int(v) for v in synth.rand_int(seed, 1, 6, 16)]
    counts[0] = 16
    M = sum(counts)
    pi = _packed(counts)
    q = 2.0**-10
    ts = np.zeros(M, np.float32)
    te = np.zeros(M, np.float32)
    for r, (off, cnt) in enumerate(pi):
        d = (1 + synth.rand_int(seed, 10 + r, cnt, 64)) * q * 4
        e = 1.0 + np.concatenate([[0], np.cumsum(d)])
        ts[off : off + cnt], te[off : off + cnt] = e[:-1], e[1:]
    sg = (synth.rand_int(seed, 2, M, 4096) * q).astype(np.float32)
    rgb = (synth.rand_int(seed, 3, 3 * M, 1024) * q).reshape(M, 3).astype(np.float32)
    R = len(counts)
    gc = synth.rand_uniform(seed, 4, 3 * R, -1, 1).reshape(R, 3)
    ga = synth.rand_uniform(seed, 5, R, -1, 1)
    gd = synth.rand_uniform(seed, 6, R, -1, 1)
    ds, dr = orc.render_bwd(pi, ts, te, sg, rgb, gc, ga, gd)
    h = 2.0**-12
    fd_s = np.zeros(M)
    for i in range(M):
        sp, sm = sg.copy(), sg.copy()
        sp[i] += np.float32(h)
        sm[i] -= np.float32(h)
        assert sp[i] - sg[i] == np.float32(h)
        fd_s[i] = (_loss(orc, pi, ts, te, sp, rgb, gc, ga, gd) - _loss(orc, pi, ts, te, sm, rgb, gc, ga, gd)) / (2 * h)
    scale = max(np.abs(fd_s).max(), 1e-12)
    assert np.max(np.abs(ds - fd_s)) / scale < 1e-6
    for i in range(0, M, 3):
        for c in range(3):
            rp, rm = rgb.copy(), rgb.copy()
            rp[i, c] += np.float32(h)
            rm[i, c] -= np.float32(h)
            fd = (_loss(orc, pi, ts, te, sg, rp, gc, ga, gd) - _loss(orc, pi, ts, te, sg, rm, gc, ga, gd)) / (2 * h)
            assert abs(dr[i, c] - fd) < 1e-9


def test_gradient_slab_closed_form(orc):
    """Constant sigma on L: d opacity / d sigma (all samples together) = L exp(-sigma L)."""
    n, sigma = 40, 0.75
    edges = (0.25 + np.linspace(0, 3.0, n + 1)).astype(np.float32)
    ts, te = edges[:-1], edges[1:]
    L = float(np.float64(te[-1]) - np.float64(ts[0]))
    ds, dr = orc.render_bwd(_packed([n]), ts, te, np.full(n, sigma, np.float32), np.ones((n, 3), np.float32),
                            None, np.ones(1), None)
    assert abs(ds.sum() - L * math.exp(-np.float32(sigma) * L)) < 1e-12
    assert np.all(dr == 0)


def _ragged_dyadic(seed, n_rays=6):
    """Rays of 1..16 samples (the first 16) with dyadic edges and densities, as above."""
    counts = [1 + int(v) for v in synth.rand_int(seed, 1, n_rays, 16)]
    counts[0] = 16
    M = sum(counts)
    pi = _packed(counts)
    q = 2.0**-10
    ts = np.zeros(M, np.float32)
    te = np.zeros(M, np.float32)
    for r, (off, cnt) in enumerate(pi):
        d = (1 + synth.rand_int(seed, 10 + r, cnt, 64)) * q * 4
        e = 1.0 + np.concatenate([[0], np.cumsum(d)])
        ts[off : off + cnt], te[off : off + cnt] = e[:-1], e[1:]
    sg = (synth.rand_int(seed, 2, M, 4096) * q).astype(np.float32)
    return pi, ts, te, sg


@pytest.mark.parametrize("seed", range(3))
def test_weights_gradient_central_differences(orc, seed):
    """dL/dsigma of L = sum_i g_i w_i against central differences of the float64 weights."""
    pi, ts, te, sg = _ragged_dyadic(seed)
    M = sg.shape[0]
    g = synth.rand_uniform(seed, 7, M, -1, 1)
    ds = orc.render_weights_bwd(pi, ts, te, sg, g)
    h = 2.0**-12
    fd = np.zeros(M)
    for i in range(M):
        sp, sm = sg.copy(), sg.copy()
        sp[i] += np.float32(h)
        sm[i] -= np.float32(h)
        fd[i] = (float((orc.render_weights(pi, ts, te, sp)[0] * g).sum())
                 - float((orc.render_weights(pi, ts, te, sm)[0] * g).sum())) / (2 * h)
    assert np.max(np.abs(ds - fd)) / max(np.abs(fd).max(), 1e-12) < 1e-6


def test_weights_gradient_single_sample_closed_form(orc):
    """One sample: w = 1 - exp(-sigma delta), so dL/dsigma = g delta exp(-sigma delta)."""
    ts = np.array([0.5, 1.0, 2.0], np.float32)
    te = np.array([0.75, 1.5, 2.125], np.float32)
    sg = np.array([0.0, 2.0, 40.0], np.float32)
    g = np.array([1.5, -0.25, 3.0])
    ds = orc.render_weights_bwd(_packed([1, 1, 1]), ts, te, sg, g)
    delta = te.astype(np.float64) - ts
    np.testing.assert_allclose(ds, g * delta * np.exp(-sg.astype(np.float64) * delta), rtol=1e-14, atol=0)


@pytest.mark.parametrize("C", [1, 3, 7])
def test_accumulate_gradient_central_differences(orc, C):
    """dL/dw and dL/dv of L = sum g * accumulate(w, v): central differences of the forward (linear)."""
    pi, ts, te, sg = _ragged_dyadic(11 + C)
    M = sg.shape[0]
    w = synth.rand_uniform(C, 1, M, 0, 1)
    v = (synth.rand_int(C, 2, M * C, 1024) * 2.0**-10).astype(np.float32).reshape(M, C)
    g = synth.rand_uniform(C, 3, pi.shape[0] * C, -1, 1).reshape(-1, C)
    dw, dv = orc.accumulate_bwd(pi, w, v, g)
    h = 2.0**-10  # L is linear in w: a large step has no truncation error and little rounding
    for i in range(0, M, 2):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (float((orc.accumulate(pi, wp, v) * g).sum()) - float((orc.accumulate(pi, wm, v) * g).sum())) / (2 * h)
        assert abs(dw[i] - fd) < 1e-9
        for c in range(C):
            vp, vm = v.copy(), v.copy()
            vp[i, c] += np.float32(2.0**-12)
            vm[i, c] -= np.float32(2.0**-12)
            fd = (float((orc.accumulate(pi, w, vp) * g).sum())
                  - float((orc.accumulate(pi, w, vm) * g).sum())) / (2 * 2.0**-12)
            assert abs(dv[i, c] - fd) < 1e-9
    dw1, dv1 = orc.accumulate_bwd(pi, w, None, g[:, :1])
    assert dv1 is None
    np.testing.assert_allclose(dw1, np.repeat(g[:, 0], pi[:, 1]), rtol=0, atol=0)


def test_render_gradient_is_the_composition(orc):
    """render = accumulate(render_weights): the fused gradient equals weights_bwd of
    accumulate_bwd's dL/dw, and its d rgb equals accumulate_bwd's d values."""
    pi, ts, te, sg = _ragged_dyadic(21)
    M, R = sg.shape[0], pi.shape[0]
    rgb = (synth.rand_int(21, 3, 3 * M, 1024) * 2.0**-10).reshape(M, 3).astype(np.float32)
    gc = synth.rand_uniform(21, 4, 3 * R, -1, 1).reshape(R, 3)
    ga = synth.rand_uniform(21, 5, R, -1, 1)
    gd = synth.rand_uniform(21, 6, R, -1, 1)
    ds, dr = orc.render_bwd(pi, ts, te, sg, rgb, gc, ga, gd)
    w, _ = orc.render_weights(pi, ts, te, sg)
    tm = ((ts.astype(np.float64) + te) * 0.5).astype(np.float32)
    vals = np.concatenate([rgb, np.ones((M, 1), np.float32), tm[:, None]], axis=1)
    g = np.concatenate([gc, ga[:, None], gd[:, None]], axis=1)
    dw, dv = orc.accumulate_bwd(pi, w, vals, g)
    ds2 = orc.render_weights_bwd(pi, ts, te, sg, dw)
    np.testing.assert_allclose(ds2, ds, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dv[:, :3], dr, rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# pruning
# ---------------------------------------------------------------------------


def test_prune_hand_built_sequence(orc):
    """tau_i = 3 per sample: O_i = 3i <= -ln(1e-4) = 9.21 for i <= 3 -> keep samples 0..3;
    alpha threshold 1e-2 <=> tau >= 0.01005: tau = 0.02 kept, tau = 0.005 dropped."""
    ts = np.arange(8, dtype=np.float32)
    te = ts + 1
    p, keep, od = orc.prune(_packed([8]), ts, te, np.full(8, 3.0, np.float32), 1e-4, 1e-2)
    assert keep.tolist() == [True] * 4 + [False] * 4 and p.packed_info.tolist() == [[0, 4]]
    assert p.t_starts.tolist() == [0, 1, 2, 3] and od.tolist() == [0, 3, 6, 9, 12, 15, 18, 21]
    sg = np.array([0.02, 0.005, 0.02, 0.0100503, 0.0100504, 0.0, 1.0, 0.02], np.float32)
    p, keep, _ = orc.prune(_packed([3, 5]), ts, te, sg, 1e-4, 1e-2)
    # -ln(0.99) = 0.01005034; the 4th value rounds below it, the 5th above
    assert keep.tolist() == [True, False, True, False, True, False, True, True]
    assert p.packed_info.tolist() == [[0, 2], [2, 3]] and p.ray_indices.tolist() == [0, 0, 1, 1, 1]


def test_prune_off_keeps_everything(orc):
    counts = [3, 0, 5]
    ts = np.arange(8, dtype=np.float32)
    sg = np.array([0, 100, 0, 5, 5, 0, 1, 2], np.float32)
    p, keep, _ = orc.prune(_packed(counts), ts, ts + 1, sg, 0.0, 0.0)
    assert keep.all() and p.packed_info.tolist() == _packed(counts).tolist()


def test_prune_matches_exact_decisions(orc):
    """Float32 decisions equal the exact (float64) ones except within the float32
    summation error bound of the threshold (Higham: |error| <= n u sum|tau|)."""
    counts = synth.rand_int(9, 1, 300, 200)
    pi = _packed(counts)
    M = int(counts.sum())
    ts = synth.rand_uniform(9, 2, M, 0, 5).astype(np.float32)
    te = ts + synth.rand_uniform(9, 3, M, 0.001, 0.02).astype(np.float32)
    sg = (synth.rand_uniform(9, 4, M) ** 4 * 60).astype(np.float32)
    eps, thre = 1e-4, 1e-2
    p, keep, od = orc.prune(pi, ts, te, sg, eps, thre)
    tau = sg.astype(np.float64) * (te.astype(np.float64) - ts.astype(np.float64))
    flips = 0
    for r, (off, cnt) in enumerate(pi):
        t = tau[off : off + cnt]
        O = np.concatenate([[0.0], np.cumsum(t)[:-1]])
        exact = (np.exp(-O) >= eps) & (1 - np.exp(-t) >= thre)
        bound = (np.arange(cnt) + 2) * 2.0**-23 * np.concatenate([[0.0], np.cumsum(np.abs(t))[:-1]]) + 1e-6
        near = (np.abs(O + math.log(eps)) <= bound) | (np.abs(t + math.log1p(-thre)) <= 1e-6 * np.maximum(1, t))
        bad = (keep[off : off + cnt] != exact) & ~near
        assert not bad.any(), (r, np.nonzero(bad))
        flips += int(((keep[off : off + cnt] != exact) & near).sum())
    assert flips <= 2
    assert p.n_samples == int(keep.sum())


# ---------------------------------------------------------------------------
# grid update
# ---------------------------------------------------------------------------


def test_grid_decay_only(orc):
    ema = synth.rand_uniform(4, 1, 1000, 0, 0.05).astype(np.float32)
    e2, bits = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 0.95, 0.01)
    assert np.array_equal(e2, ema * np.float32(0.95))
    assert np.array_equal(synth.unpack_bits(bits, 1000), e2 > np.float32(0.01))


def test_grid_scatter_max_and_threshold(orc):
    ema = np.zeros(64, np.float32)
    ema[5] = 1.0
    cells = np.array([3, 3, 3, 5, 7, 7, 9, 9], np.int32)
    sig = np.array([0.5, 2.0, 1.0, 0.1, 0.005, np.nan, -1.0, 0.0105], np.float32)
    e2, bits = orc.update_grid(ema, cells, sig, 0.5, 0.01)
    want = np.zeros(64, np.float32)
    want[3], want[5], want[7], want[9] = 2.0, 0.5, 0.005, np.float32(0.0105)
    assert np.array_equal(e2, want)
    assert np.nonzero(synth.unpack_bits(bits, 64))[0].tolist() == [3, 5, 9]
    # a hand-made grid of 70 cells (ragged last word): bits = ema > thre
    ema = np.zeros(70, np.float32)
    ema[[0, 31, 32, 63, 64, 69]] = [1, 0.02, 0.01, 0.011, 5, 0.0099]
    _, bits = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 1.0, 0.01)
    assert bits.tolist() == [(1 << 0) | (1 << 31), 1 << 31, 1 << 0]


def test_grid_opacity_criterion(orc):
    """alpha mode: occupied where a step of length dt would be at least that opaque.
    Dyadic densities on either side of -ln(1 - 0.5)/dt = ln 2/dt (dt = 1/4: 2.7726),
    including 0 (never occupied with alpha >= 0) and a decay that moves one across."""
    ema = np.array([0.0, 2.5, 2.75, 2.78125, 3.0, 100.0, 5.5, 5.5625], np.float32)
    _, bits = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 1.0, 0.5, alpha_step=0.25)
    assert np.nonzero(synth.unpack_bits(bits, 8))[0].tolist() == [3, 4, 5, 6, 7]
    e2, bits = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 0.5, 0.5, alpha_step=0.25)
    assert np.nonzero(synth.unpack_bits(bits, 8))[0].tolist() == [5, 7]  # 5.5625 -> 2.78125 stays, 5.5 -> 2.75 not
    # away from the threshold the criterion and its density form agree
    ema = synth.rand_uniform(4, 9, 5000, 0, 0.05).astype(np.float32)
    _, b_alpha = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 1.0, 0.01, alpha_step=0.5)
    _, b_dens = orc.update_grid(ema, np.zeros(0, np.int32), np.zeros(0, np.float32), 1.0,
                                float(np.float32(-np.log1p(-0.01) / 0.5)))
    assert np.array_equal(b_alpha, b_dens)
