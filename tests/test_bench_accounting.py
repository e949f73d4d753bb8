"""The benchmark's byte and launch accounting, on CPU: each stage's algorithmic
bytes (the roofline's numerator) computed by hand for one set of sizes, the
per-stage sum against the per-step formula 104R + 24M + 76S, and the library
launches one bounded training step makes."""
from types import SimpleNamespace

import bench

R, M, M_READ, S = 1000, 50000, 30000, 12000
CELLS = 128 ** 3
GRID_SAMPLES = 1 << 21
BITS = CELLS // 8


def test_stage_bytes_by_hand():
    sb = bench.stage_bytes(R, M, M_READ, S, BITS, CELLS, GRID_SAMPLES)
    # rays in (24R), packed_info out (8R), three 4-byte arrays per marched sample, the bitfield once
    assert sb["march"] == 32_000 + 600_000 + 262_144
    # packed_info in and out (16R), three arrays per sample read up to termination, three per kept sample
    assert sb["prune"] == 16_000 + 360_000 + 144_000
    # packed_info (8R) and colour, opacity, depth (20R); sigma, rgb, t_start, t_end per kept sample
    assert sb["render_fwd"] == 28_000 + 288_000
    # dL/dcolour (12R) and packed_info (8R); the kept samples in (24S) and dsigma, drgb out (16S)
    assert sb["render_bwd"] == 20_000 + 480_000
    # cells + points out and cells + sigmas in per update sample, the float grid in and out, the bits
    assert sb["grid_update"] == 24 * GRID_SAMPLES + 8 * CELLS + CELLS // 8
    saved = bench.stage_bytes(R, M, M_READ, S, BITS, CELLS, GRID_SAMPLES, saved_od=True)
    assert saved["render_fwd"] - sb["render_fwd"] == 4 * S
    assert saved["render_bwd"] - sb["render_bwd"] == 4 * S
    # forward, loss gradient and backward in one pass: the kept samples read once
    assert sb["render_fused"] == 40 * R + 40 * S


def test_stage_sum_matches_the_step_formula():
    """With every marched sample read by pruning, the four path stages add up to
    104R + 24M + 76S plus the bitfield, less the 8R of opacity and depth gradients
    that the benchmark's backward does not take (its loss is on the colour only)."""
    sb = bench.stage_bytes(R, M, M, S, BITS, CELLS, GRID_SAMPLES)
    path = sum(sb[s] for s in ("march", "prune", "render_fwd", "render_bwd"))
    assert path + 8 * R == 104 * R + 24 * M + 76 * S + BITS


def test_launches_of_a_bounded_step():
    w = SimpleNamespace(cone=0.0, res=(128, 128, 128), n_levels=1, n_slots=1)
    # the table's build: one pass over planes, the sum along x, the brick summary
    assert bench.sat_launches(w.res, 1) == 3
    # march, prune, forward, backward, sampler, scatter, the decay over whole 128-cell
    # steps of an aligned grid, and the table's three launches
    assert bench.launches_per_step(w, CELLS, GRID_SAMPLES, 256, sat=True) == 10
    assert bench.launches_per_step(w, CELLS, GRID_SAMPLES, 256, sat=True, fused=True) == 9
    # a grid not 16-byte aligned is decayed one cell per thread: still one decay launch
    assert bench.launches_per_step(w, CELLS, GRID_SAMPLES, 260, sat=False) == 7
    # cone steps add the lattice table's prologue
    cone = SimpleNamespace(cone=1.0 / 256, res=(128, 128, 128), n_levels=4, n_slots=1)
    assert bench.launches_per_step(cone, 4 * CELLS, GRID_SAMPLES, 256, sat=False) == 8
