"""GPU marching vs the oracle, bit-exact (Sec. 2.1 "Ray Marching"): sample counts,
packed offsets, ray indices and the float32 interval bounds all identical."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import assert_march_equal, gpu_march, oracle_march  # noqa: E402


@pytest.fixture(autouse=True, params=[0, 1, 2, 4], ids=["plain", "box", "box_tile", "box_tile6"])
def box_walk(request):
    """Every case without and with the grid's summed-area table (the box walk on
    one-level grids, ray by ray or over a whole tile; other grids ignore it)."""
    import gpu_util

    old = _lib.tune_get("march_box_tile")
    _lib.tune_set("march_box_tile", {0: 0, 1: 0, 2: 1, 4: 3}[request.param])
    gpu_util.USE_SAT = request.param > 0
    yield request.param
    gpu_util.USE_SAT = False
    _lib.tune_set("march_box_tile", old)


def test_tiny_config_bitexact(orc):
    w = synth.tiny_config(0, device="cuda")
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


@pytest.mark.parametrize("seed", range(4))
def test_random_tiny_grids(orc, seed):
    """Grids 2^3..8^3 with random bits; 1000 rays (32 tiles, ragged last tile) incl.
    axis-parallel, inside-the-box, grazing and non-finite rays."""
    res = [(2, 2, 2), (3, 5, 4), (8, 8, 8), (7, 3, 6)][seed]
    n_cells = res[0] * res[1] * res[2]
    occ = synth.rand_uniform(seed, 1, n_cells) < 0.4
    n = 1000
    o = synth.random_unit_vectors(seed, 2, n) * 3.0
    tgt = synth.rand_uniform(seed, 3, 3 * n, -1.2, 1.2).reshape(n, 3)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:6] = np.eye(3)[[0, 1, 2, 0, 1, 2]] * np.array([1, 1, 1, -1, -1, -1])[:, None]
    o[:6] = [[-2, 0.1, -0.3], [0.3, -2, -0.4], [0.2, 0.3, -2], [2, -0.2, 0.1], [-0.1, 2, 0.2], [0.1, 0.2, 2]]
    o[6:40] = synth.rand_uniform(seed, 4, 102, -0.9, 0.9).reshape(34, 3)
    o[40] = [np.nan, 0, 0]
    d[41] = [np.inf, 0, 0]
    o[42], d[42] = [-2, 1.0, 0.0], [1, 0, 0]  # grazing the y = 1 face
    w = synth.Workload("tiny-random", o.astype(np.float32), d.astype(np.float32), synth.pack_bits(occ), res, 1, 1,
                       (-1.0, -0.75, -1.25, 1.0, 1.25, 0.5), 0.0, 1e10, 0.05, 0.05, 0.0, 1024, 0.0, 0.0)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_bounded_subset_bitexact(orc):
    w = synth.bounded_config(0, n_rays=1 << 12, device="cuda")
    g = gpu_march(w)
    assert g[4] > 1000 * 100
    assert_march_equal(g, oracle_march(orc, w))


def test_near_far_planes_and_max_steps(orc):
    w = synth.bounded_config(1, n_rays=2000, device="cuda")
    w.near_plane, w.far_plane, w.max_steps = 3.1, 4.6, 200
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_cone_cascade_bitexact(orc):
    """Unbounded scene: 4-level cascade of 128^3, cone steps clamp(t/256, 1e-3, 10)."""
    w = synth.unbounded_config(0, n_rays=1 << 11, device="cuda")
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


def test_time_bins_bitexact(orc):
    w = synth.dynamic_config(0, n_rays=1 << 11, n_bins=16, device="cuda")
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_scene_slots_bitexact(orc):
    w = synth.batched_config(0, n_scenes=6, device="cuda", ray_scale=1.0 / 32)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_capacity_overflow_reports_total(orc):
    w = synth.tiny_config(0, device="cuda")
    ora = oracle_march(orc, w)
    cap = ora.n_samples // 3
    pi, ts, te, ri, n, status = gpu_march(w, capacity=cap)
    assert status & _lib.STATUS_CAPACITY
    assert n == ora.n_samples
    assert np.array_equal(pi, ora.packed_info)
    assert np.array_equal(ts, ora.t_starts[:cap]) and np.array_equal(ri, ora.ray_indices[:cap])


def test_empty_and_all_missing(orc):
    w = synth.tiny_config(0, device="cuda")
    w.rays_o = np.zeros((0, 3), np.float32)
    w.rays_d = np.zeros((0, 3), np.float32)
    pi, ts, te, ri, n, status = gpu_march(w, capacity=16)
    assert n == 0 and status == 0
    w = synth.tiny_config(0, device="cuda")
    w.rays_o = np.tile(np.array([[5, 5, 5]], np.float32), (77, 1))
    w.rays_d = np.tile(np.array([[1, 0, 0]], np.float32), (77, 1))
    pi, ts, te, ri, n, status = gpu_march(w, capacity=16)
    assert n == 0 and status == 0 and np.all(pi == 0)


def test_max_steps_many_chunks(orc):
    """max_steps = 32768 with a tiny step: long rays span 1024 ballot words."""
    w = synth.tiny_config(0, device="cuda")
    w.rays_o, w.rays_d = w.rays_o[:300], w.rays_d[:300]
    w.dt_min = w.dt_max = 2e-4
    w.max_steps = 32768
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_cone_mixed_starts_bitexact(orc):
    """Cone steps with rays starting outside the box (each ray its own recurrence from
    t_in) and inside it (the lattice shared from near_plane), in one launch."""
    w = synth.bounded_config(2, n_rays=3000, device="cuda")
    inside = synth.rand_uniform(2, 7, 3 * 1000, -1.2, 1.2).reshape(1000, 3).astype(np.float32)
    w.rays_o = np.ascontiguousarray(np.concatenate([w.rays_o[:2000], inside]))
    w.cone, w.dt_min, w.dt_max, w.near_plane, w.max_steps = 1.0 / 64, 1e-3, 0.05, 0.05, 2048
    g = gpu_march(w)
    assert g[4] > 100000
    assert_march_equal(g, oracle_march(orc, w))


@pytest.mark.parametrize("cfg", ["bounded", "cone"])
def test_lattice_point_counter(orc, cfg, box_walk):
    """The workspace's lattice-point counter equals the samples the oracle emits on
    the same rays over an all-ones grid (where every lattice point is a sample)."""
    if cfg == "bounded":
        w = synth.bounded_config(3, n_rays=3000, device="cuda")
    else:
        w = synth.unbounded_config(3, n_rays=1500, device="cuda")
        inside = w.rays_o.copy()
        inside[:500] = inside[:500] * 20.0  # some rays start outside the outermost box (own lattices)
        w.rays_o = np.ascontiguousarray(inside)
    o, d = torch.from_numpy(w.rays_o).cuda(), torch.from_numpy(w.rays_d).cuda()
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    R = w.n_rays
    ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
    cap = 8_000_000
    pi = torch.zeros((R, 2), dtype=torch.int32, device="cuda")
    ts, te = torch.zeros(cap, device="cuda"), torch.zeros(cap, device="cuda")
    ri = torch.zeros(cap, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    bits = torch.from_numpy(w.bits.view(np.int32)).cuda()
    grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots)
    if box_walk:
        grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, sat=_lib.build_grid_sat(grid))
    _lib.march_rays(o, d, grid, params, pi, ts, te, ri, n, st, ws)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    counted = int(ws[8:16].cpu().numpy().view(np.uint64)[0])
    ones = np.full_like(w.bits, 0xFFFFFFFF)
    full = orc.march(w.rays_o, w.rays_d, ones, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone,
                     w.max_steps, n_levels=w.n_levels, n_slots=w.n_slots)
    assert counted == full.n_samples > 0


def test_shared_time_grid_bitexact(orc):
    """One grid for all times (the maximum over time) with per-ray times: every ray reads slot 0."""
    w = synth.dynamic_shared_config(0, n_rays=1 << 11, device="cuda")
    assert w.n_slots == 1 and w.ray_time is not None
    assert_march_equal(gpu_march(w), oracle_march(orc, w))
