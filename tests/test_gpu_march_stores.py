"""The marcher's store phase: runs of full ballot words are written as 16-byte
vectors when the three outputs are 16-byte aligned, lane by lane otherwise.
Both must give the oracle's samples bit for bit, at every alignment of the output
arrays, with and without the grid's summed-area table, and a capacity that cuts
a run anywhere (at every residue modulo 4) must store exactly the prefix below it
and nothing past it."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import dev, oracle_march  # noqa: E402

GUARD = 64


def _march(w, capacity, shift, use_sat):
    """March into output views that start `shift` elements past a 256-byte boundary;
    returns numpy (packed_info, t_starts, t_ends, ray_indices incl. a guard region, total, status)."""
    R = w.n_rays
    o, d = dev(w.rays_o), dev(w.rays_d)
    bits = dev(w.bits)
    grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)
    if use_sat:
        grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction,
                              sat=_lib.build_grid_sat(grid))
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    ws = torch.zeros(max(_lib.march_workspace_size(R, params), 256), dtype=torch.uint8, device="cuda")
    n = capacity + GUARD
    bts = torch.full((n + shift,), np.nan, device="cuda")
    bte = torch.full((n + shift,), np.nan, device="cuda")
    bri = torch.full((n + shift,), -1, dtype=torch.int32, device="cuda")
    ts, te, ri = bts[shift:shift + n], bte[shift:shift + n], bri[shift:shift + n]
    pi = torch.full((R, 2), -7, dtype=torch.int32, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.march_rays(o, d, grid, params, pi, ts[:capacity], te[:capacity], ri[:capacity], total, st, ws)
    torch.cuda.synchronize()
    return (pi.cpu().numpy(), ts.cpu().numpy(), te.cpu().numpy(), ri.cpu().numpy(), int(total.item()),
            int(st.item()))


def _workloads():
    bounded = synth.bounded_config(4, n_rays=1500)
    cone = synth.unbounded_config(2, n_rays=700)
    return {"bounded": bounded, "cascade_cone": cone}


@pytest.fixture(scope="module")
def cases(orc):
    out = {}
    for name, w in _workloads().items():
        out[name] = (w, oracle_march(orc, w))
    return out


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("name", ["bounded", "cascade_cone"])
@pytest.mark.parametrize("use_sat", [False, True])
@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_every_output_alignment_is_bit_exact(cases, name, use_sat, shift):
    """shift 0: 16-byte aligned outputs (vector stores of full runs); 1..3: lane by lane."""
    w, ora = cases[name]
    old = _lib.tune_get("march_box_tile")
    try:
        for box_tile in (0, 1):
            _lib.tune_set("march_box_tile", box_tile)
            pi, ts, te, ri, n, st = _march(w, ora.n_samples, shift, use_sat)
            assert st == 0 and n == ora.n_samples
            assert np.array_equal(pi, ora.packed_info)
            assert np.array_equal(_bits(ts[:n]), _bits(ora.t_starts))
            assert np.array_equal(_bits(te[:n]), _bits(ora.t_ends))
            assert np.array_equal(ri[:n], ora.ray_indices)
            assert np.all(np.isnan(ts[n:])) and np.all(np.isnan(te[n:])) and np.all(ri[n:] == -1)
    finally:
        _lib.tune_set("march_box_tile", old)


@pytest.mark.parametrize("shift", [0, 3])
def test_capacity_cuts_a_run_at_every_residue(cases, shift):
    """Capacities inside the output (every residue modulo 4, near the start, the
    middle and the end): the prefix below the capacity is the oracle's, nothing
    at or past it is written, and the total and the capacity flag are reported."""
    w, ora = cases["bounded"]
    N = ora.n_samples
    caps = sorted({c for base in (5, N // 2, N - 9) for c in range(base, base + 4) if 0 < c < N})
    for cap in caps:
        pi, ts, te, ri, n, st = _march(w, cap, shift, True)
        assert st & _lib.STATUS_CAPACITY and n == N
        assert np.array_equal(pi, ora.packed_info)
        assert np.array_equal(_bits(ts[:cap]), _bits(ora.t_starts[:cap]))
        assert np.array_equal(_bits(te[:cap]), _bits(ora.t_ends[:cap]))
        assert np.array_equal(ri[:cap], ora.ray_indices[:cap])
        assert np.all(np.isnan(ts[cap:])) and np.all(np.isnan(te[cap:])) and np.all(ri[cap:] == -1)


@pytest.mark.parametrize("tile_rays", [1, 2, 4, 8, 16, 32])
def test_cone_cascade_every_tile_size(cases, tile_rays):
    """Cone steps keep the shared lattice in each block's shared memory next to the
    tile rows and the brick summary: every tile size (the largest need more than
    the default 48 KB of shared memory per block) marches bit-exactly."""
    w, ora = cases["cascade_cone"]
    old = _lib.tune_get("march_tile_rays")
    try:
        _lib.tune_set("march_tile_rays", tile_rays)
        for use_sat in (False, True):
            pi, ts, te, ri, n, st = _march(w, ora.n_samples, 0, use_sat)
            assert st == 0 and n == ora.n_samples
            assert np.array_equal(pi, ora.packed_info)
            assert np.array_equal(_bits(ts[:n]), _bits(ora.t_starts)) and np.array_equal(ri[:n], ora.ray_indices)
    finally:
        _lib.tune_set("march_tile_rays", old)
