"""The fused inference path (nacc_march_fused: marching that stops on the density
field's transmittance, Sec. 2.1) and the density field it evaluates, against the
oracle through the C ABI.

Bars: the field's sigma is bit-exact (a float32 replica of one operation order);
every kept sample (t_start, t_end, ray, sigma) is bit-exact, except on rays where
a keep decision flips between the two float32 summation orders of the optical
depth, which may happen only for samples within the float32 summation error of
-ln(eps) (the same rule as pruning); such rays are few.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, dev, gpu_march, near_threshold, oracle_march  # noqa: E402


def _subset(w, step, offset=0):
    w.rays_o = np.ascontiguousarray(w.rays_o[offset::step])
    w.rays_d = np.ascontiguousarray(w.rays_d[offset::step])
    return w


@pytest.fixture(scope="module")
def inf():
    """Every 97th pixel of a whole 800x800 image of the bounded scene (6598 rays),
    the scene's density baked at 65^3 vertices."""
    return _subset(synth.inference_config(0, field_res=65), 97)


def _field(w):
    return dev(w.field), w.field_box


def gpu_fused(w, eps=None, thre=None, capacity=None, field=None, rays=None):
    o = dev(w.rays_o if rays is None else rays[0])
    d = dev(w.rays_d if rays is None else rays[1])
    R = o.shape[0]
    eps = w.early_stop_eps if eps is None else eps
    thre = w.alpha_thre if thre is None else thre
    ft, fbox = _field(w) if field is None else field
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    ws = torch.zeros(max(_lib.march_workspace_size(R, params), 256), dtype=torch.uint8, device="cuda")
    bits = dev(w.bits)
    grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)
    cap = max(R * w.max_steps, 1) if capacity is None else capacity
    packed = torch.full((R, 2), -7, dtype=torch.int32, device="cuda")
    ts = torch.full((cap,), np.nan, device="cuda")
    te = torch.full((cap,), np.nan, device="cuda")
    ri = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    sg = torch.full((cap,), np.nan, device="cuda")
    n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.march_fused(o, d, grid, params, _lib.make_density_field(ft, fbox), eps, thre, packed, ts, te, ri, sg, n, st,
                     ws)
    torch.cuda.synchronize()
    k = min(int(n.item()), cap)
    lattice = int(ws[8:16].view(torch.int64).item())
    return dict(pi=packed.cpu().numpy(), ts=ts[:k].cpu().numpy(), te=te[:k].cpu().numpy(), ri=ri[:k].cpu().numpy(),
                sg=sg[:k].cpu().numpy(), n=int(n.item()), status=int(st.item()), lattice=lattice)


def _midpoints(o, d, ts, te, ri):
    mid = ((ts + te) * np.float32(0.5)).astype(np.float32)
    return (o[ri] + d[ri] * mid[:, None]).astype(np.float32)


def oracle_reference(orc, w, eps=None, thre=None, field=None):
    """march -> field at midpoints -> prune, all by the oracle; returns the marched
    set, its sigma and optical depth, and the kept set with its sigma."""
    eps = w.early_stop_eps if eps is None else eps
    thre = w.alpha_thre if thre is None else thre
    fld, fbox = (w.field, w.field_box) if field is None else field
    m = oracle_march(orc, w)
    sig = orc.field_query(fld, fbox, _midpoints(w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices))
    p, keep, od = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, eps, thre)
    return m, sig, od, p, sig[keep]


def assert_fused_matches(g, m, sig, od, p, p_sig, eps, max_flipped=2):
    assert g["status"] == 0, "device status 0x%x" % g["status"]
    near = near_threshold(m.packed_info, m.t_starts, m.t_ends, sig, eps, od) if eps > 0 else np.zeros(0, bool)
    flipped = 0
    for r in range(m.packed_info.shape[0]):
        (og, cg), (oo, co) = g["pi"][r], p.packed_info[r]
        same = (cg == co and bits_equal(g["ts"][og : og + cg], p.t_starts[oo : oo + co])
                and bits_equal(g["te"][og : og + cg], p.t_ends[oo : oo + co]))
        if same:
            assert np.all(g["ri"][og : og + cg] == r)
            assert bits_equal(g["sg"][og : og + cg], p_sig[oo : oo + co]), "sigma differs on ray %d" % r
            continue
        mo, mc = m.packed_info[r]
        assert eps > 0 and near[mo : mo + mc].any(), "ray %d differs away from the early-stop threshold" % r
        flipped += 1
    assert flipped <= max_flipped, flipped
    assert g["n"] == int(g["pi"][:, 1].sum())


def test_field_query_bit_exact(orc, inf):
    rng = np.random.default_rng(5)
    lo, hi = np.array(inf.field_box[:3]), np.array(inf.field_box[3:])
    x = lo + (hi - lo) * rng.uniform(-0.05, 1.05, (50000, 3))
    faces = np.array([[lo[0], 0, 0], [hi[0], 0, 0], [0, hi[1], 0], [0, 0, lo[2]], [hi[0], hi[1], hi[2]],
                      [np.nan, 0, 0], [0, np.inf, 0]])
    x = np.concatenate([x, faces]).astype(np.float32)
    ft, fbox = _field(inf)
    out = torch.full((x.shape[0],), np.nan, device="cuda")
    _lib.density_field_query(_lib.make_density_field(ft, fbox), dev(x), x.shape[0], out)
    torch.cuda.synchronize()
    ref = orc.field_query(inf.field, fbox, x)
    assert bits_equal(out.cpu().numpy(), ref)
    assert (ref > 0).mean() > 0.5


def test_field_at_samples_bit_exact(orc, inf):
    m = oracle_march(orc, inf)
    ft, fbox = _field(inf)
    out = torch.full((m.n_samples,), np.nan, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.density_field_at_samples(_lib.make_density_field(ft, fbox), dev(inf.rays_o), dev(inf.rays_d),
                                  dev(m.ray_indices), dev(m.t_starts), dev(m.t_ends), m.n_samples, out, st)
    torch.cuda.synchronize()
    ref = orc.field_query(inf.field, fbox, _midpoints(inf.rays_o, inf.rays_d, m.t_starts, m.t_ends, m.ray_indices))
    assert int(st.item()) == 0
    assert bits_equal(out.cpu().numpy(), ref)
    # a ray index out of range gives sigma 0 and a status bit, nothing else
    bad = m.ray_indices[:4].copy()
    bad[1] = inf.n_rays
    out2 = torch.full((4,), np.nan, device="cuda")
    _lib.density_field_at_samples(_lib.make_density_field(ft, fbox), dev(inf.rays_o), dev(inf.rays_d), dev(bad),
                                  dev(m.t_starts[:4]), dev(m.t_ends[:4]), 4, out2, st)
    torch.cuda.synchronize()
    assert int(st.item()) & _lib.STATUS_BAD_INDEX
    o2 = out2.cpu().numpy()
    assert o2[1] == 0.0 and bits_equal(o2[[0, 2, 3]], ref[[0, 2, 3]])


def test_fused_parity_bounded_image(orc, inf):
    m, sig, od, p, p_sig = oracle_reference(orc, inf)
    g = gpu_fused(inf)
    assert_fused_matches(g, m, sig, od, p, p_sig, inf.early_stop_eps)
    assert p.n_samples < 0.5 * m.n_samples  # the field really terminates rays and drops samples
    assert g["lattice"] > 0


@pytest.mark.parametrize("tile_rays", [1, 4, 32])
def test_fused_tile_shapes_agree(inf, tile_rays):
    old = _lib.tune_get("march_tile_rays")
    try:
        _lib.tune_set("march_tile_rays", 4)
        a = gpu_fused(inf)
        _lib.tune_set("march_tile_rays", tile_rays)
        b = gpu_fused(inf)
    finally:
        _lib.tune_set("march_tile_rays", old)
    for k in ("pi", "ri"):
        assert np.array_equal(a[k], b[k])
    for k in ("ts", "te", "sg"):
        assert bits_equal(a[k], b[k])


def test_fused_register_cap_agrees(inf):
    old = _lib.tune_get("fused_occupancy")
    try:
        _lib.tune_set("fused_occupancy", 0)
        a = gpu_fused(inf)
        _lib.tune_set("fused_occupancy", 1)
        b = gpu_fused(inf)
    finally:
        _lib.tune_set("fused_occupancy", old)
    for k in ("pi", "ri"):
        assert np.array_equal(a[k], b[k])
    for k in ("ts", "te", "sg"):
        assert bits_equal(a[k], b[k])


def test_fused_without_thresholds_is_the_march(orc, inf):
    g = gpu_fused(inf, eps=0.0, thre=0.0)
    mg = gpu_march(inf)
    assert g["status"] == 0 and g["n"] == mg[4]
    assert np.array_equal(g["pi"], mg[0]) and np.array_equal(g["ri"], mg[3])
    assert bits_equal(g["ts"], mg[1]) and bits_equal(g["te"], mg[2])
    ref = orc.field_query(inf.field, inf.field_box, _midpoints(inf.rays_o, inf.rays_d, mg[1], mg[2], mg[3]))
    assert bits_equal(g["sg"], ref)


def test_fused_alpha_only_and_early_stop_only(orc, inf):
    for eps, thre in ((0.0, inf.alpha_thre), (inf.early_stop_eps, 0.0)):
        m, sig, od, p, p_sig = oracle_reference(orc, inf, eps, thre)
        g = gpu_fused(inf, eps, thre)
        assert_fused_matches(g, m, sig, od, p, p_sig, eps)


def test_fused_matches_two_call_gpu_path(inf):
    """march -> field at samples -> prune on the GPU keeps the same samples."""
    w = inf
    mg = gpu_march(w)
    pi, ts, te, ri, M = mg[0], mg[1], mg[2], mg[3], mg[4]
    ft, fbox = _field(w)
    sig = torch.empty(M, device="cuda")
    _lib.density_field_at_samples(_lib.make_density_field(ft, fbox), dev(w.rays_o), dev(w.rays_d), dev(ri), dev(ts),
                                  dev(te), M, sig)
    R = pi.shape[0]
    ws = torch.zeros(_lib.prune_workspace_size(R, M), dtype=torch.uint8, device="cuda")
    out = dict(pi=torch.zeros((R, 2), dtype=torch.int32, device="cuda"), ts=torch.zeros(M, device="cuda"),
               te=torch.zeros(M, device="cuda"), ri=torch.zeros(M, dtype=torch.int32, device="cuda"),
               n=torch.zeros(1, dtype=torch.int64, device="cuda"))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.prune_samples(dev(pi), dev(ts), dev(te), sig, M, w.early_stop_eps, w.alpha_thre, out["pi"], out["ts"],
                       out["te"], out["ri"], out["n"], st, ws)
    torch.cuda.synchronize()
    two = {k: v.cpu().numpy() for k, v in out.items()}
    g = gpu_fused(w)
    sg = sig.cpu().numpy()
    tau = sg.astype(np.float64) * (te.astype(np.float64) - ts.astype(np.float64))
    od = np.zeros(M)
    for off, cnt in pi:
        if cnt:
            od[off : off + cnt] = np.concatenate([[0.0], np.cumsum(tau[off : off + cnt])[:-1]])
    near = near_threshold(pi, ts, te, sg, w.early_stop_eps, od)
    flipped = 0
    for r in range(R):
        (a, ca), (b, cb) = g["pi"][r], two["pi"][r]
        if ca == cb and bits_equal(g["ts"][a : a + ca], two["ts"][b : b + cb]):
            continue
        o, c = pi[r]
        assert near[o : o + c].any(), "ray %d differs away from the threshold" % r
        flipped += 1
    assert flipped <= 2


def test_fused_cone_cascade(orc):
    w = synth.unbounded_config(0, n_rays=1024)
    box = w.aabb  # level-0 box of the cascade; sigma is 0 outside it
    w.field = synth.density_at_vertices(w.scenes[0], box, (33, 33, 33))
    w.field_box = tuple(box)
    m, sig, od, p, p_sig = oracle_reference(orc, w)
    g = gpu_fused(w)
    assert_fused_matches(g, m, sig, od, p, p_sig, w.early_stop_eps)
    assert p.n_samples > 0


def test_fused_contracted(orc):
    w = synth.contracted_config(0, n_rays=1024)
    w.field = synth.density_at_vertices(w.scenes[0], w.aabb, (33, 33, 33))
    w.field_box = tuple(w.aabb)
    m, sig, od, p, p_sig = oracle_reference(orc, w)
    g = gpu_fused(w)
    assert_fused_matches(g, m, sig, od, p, p_sig, w.early_stop_eps)
    assert p.n_samples > 0


def test_fused_capacity_overflow_and_empty(orc, inf):
    full = gpu_fused(inf)
    cap = full["n"] // 3
    g = gpu_fused(inf, capacity=cap)
    assert g["status"] & _lib.STATUS_CAPACITY and g["n"] == full["n"]
    assert np.array_equal(g["pi"], full["pi"])
    assert bits_equal(g["ts"], full["ts"][:cap]) and bits_equal(g["sg"], full["sg"][:cap])
    # no rays
    z = np.zeros((0, 3), np.float32)
    e = gpu_fused(inf, rays=(z, z))
    assert e["n"] == 0 and e["status"] == 0
    # a transparent field keeps nothing under the opacity threshold ...
    zero = (dev(np.zeros((3, 3, 3), np.float32)), inf.field_box)
    t = gpu_fused(inf, field=zero)
    assert t["n"] == 0 and not t["pi"][:, 1].any()
    # ... and every marched sample without it (T stays 1)
    t2 = gpu_fused(inf, thre=0.0, field=zero)
    mg = gpu_march(inf)
    assert t2["n"] == mg[4] and np.array_equal(t2["pi"], mg[0]) and not t2["sg"].any()


def test_fused_rejects_bad_fields(inf):
    ft, fbox = _field(inf)
    ok = _lib.make_density_field(ft, fbox)
    bad_res = _lib.make_density_field(ft, fbox)
    bad_res.res[1] = 1
    bad_box = _lib.make_density_field(ft, fbox)
    bad_box.aabb[0], bad_box.aabb[3] = 1.0, -1.0
    out = torch.zeros(4, device="cuda")
    x = torch.zeros((4, 3), device="cuda")
    _lib.density_field_query(ok, x, 4, out)
    for f in (bad_res, bad_box):
        with pytest.raises(_lib.NaccError):
            _lib.density_field_query(f, x, 4, out)


def test_api_march_with_density_then_render(inf):
    from paper_2210_04847_gb300 import api

    grid = api.OccupancyGrid.from_bits(inf.bits, inf.res, inf.aabb, device="cuda")
    dens = api.DensityGrid(dev(inf.field), inf.field_box)
    o, d = dev(inf.rays_o), dev(inf.rays_d)
    packed, ts, te, sg, ri = api.march_with_density(o, d, grid, dens, render_step_size=inf.dt_min, max_steps=1024,
                                                    early_stop_eps=inf.early_stop_eps, alpha_thre=inf.alpha_thre,
                                                    return_ray_indices=True)
    g = gpu_fused(inf)
    assert np.array_equal(packed.cpu().numpy(), g["pi"]) and bits_equal(sg.view(-1).cpu().numpy(), g["sg"])
    # the two-call API path with the same field as sigma_fn keeps the same samples (up to threshold flips)
    p2, ts2, te2, ri2 = api.ray_marching(o, d, grid, sigma_fn=lambda a, b, r: dens.at_samples(o, d, a, b, r),
                                         render_step_size=inf.dt_min, max_steps=1024,
                                         early_stop_eps=inf.early_stop_eps, alpha_thre=inf.alpha_thre,
                                         return_ray_indices=True)
    differ = (packed[:, 1].cpu().numpy() != p2[:, 1].cpu().numpy()).sum()  # per-ray kept counts
    assert differ <= 2
    # rendering the kept samples: colour from the field's rgb stand-in, sigma from the fused output
    rgb = torch.sigmoid(torch.randn(ts.shape[0], 3, device="cuda"))
    color, opacity, depth = api.render_packed(sg.view(-1), rgb, packed, ts.view(-1), te.view(-1))
    assert torch.isfinite(color).all() and float(opacity.max()) <= 1.0 + 1e-6
    assert float(opacity.mean()) > 0.05


@pytest.mark.parametrize("eps,thre", [(1.0, 0.0), (0.5, 0.5), (1e-8, 0.999), (0.9999, 1e-6)])
def test_fused_extreme_thresholds(orc, eps, thre):
    w = _subset(synth.inference_config(0, field_res=33), 401)
    m, sig, od, p, p_sig = oracle_reference(orc, w, eps, thre)
    g = gpu_fused(w, eps, thre)
    assert_fused_matches(g, m, sig, od, p, p_sig, eps)


def test_fused_multislot_grid_uses_slot_zero(inf):
    """A grid with several slots: the fused path (no time or slot input) uses slot 0."""
    w = inf
    other = np.zeros_like(w.bits)  # slot 1: empty
    two = np.concatenate([w.bits, other])
    o, d = dev(w.rays_o), dev(w.rays_d)
    ft = dev(w.field)
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    R = o.shape[0]
    out = []
    for bits_np, slots in ((w.bits, 1), (two, 2)):
        bits = dev(bits_np)
        grid = _lib.make_grid(bits, w.res, w.aabb, 1, slots, 0)
        ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
        pi = torch.zeros((R, 2), dtype=torch.int32, device="cuda")
        cap = R * 1024
        ts, te, sg = (torch.zeros(cap, device="cuda") for _ in range(3))
        ri = torch.zeros(cap, dtype=torch.int32, device="cuda")
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        _lib.march_fused(o, d, grid, params, _lib.make_density_field(ft, w.field_box), w.early_stop_eps,
                         w.alpha_thre, pi, ts, te, ri, sg, n, st, ws)
        torch.cuda.synchronize()
        k = int(n.item())
        out.append((pi.cpu().numpy(), ts[:k].cpu().numpy(), sg[:k].cpu().numpy(), int(st.item())))
    assert out[0][3] == 0 and out[1][3] == 0
    assert np.array_equal(out[0][0], out[1][0]) and bits_equal(out[0][1], out[1][1]) and bits_equal(out[0][2], out[1][2])


def test_fused_nonfinite_rays_emit_nothing(inf):
    o = inf.rays_o[:64].copy()
    d = inf.rays_d[:64].copy()
    o[3, 0] = np.nan
    d[7, 1] = np.inf
    o[11, 2] = -np.inf
    g = gpu_fused(inf, rays=(o, d))
    ref = gpu_fused(inf, rays=(inf.rays_o[:64], inf.rays_d[:64]))
    assert g["status"] == 0
    for r in (3, 7, 11):
        assert g["pi"][r, 1] == 0
    keep = [r for r in range(64) if r not in (3, 7, 11)]
    assert np.array_equal(g["pi"][keep, 1], ref["pi"][keep, 1])


def test_api_march_with_density_empty_batch(inf):
    from paper_2210_04847_gb300 import api

    grid = api.OccupancyGrid.from_bits(inf.bits, inf.res, inf.aabb, device="cuda")
    dens = api.DensityGrid(dev(inf.field), inf.field_box)
    z = torch.zeros((0, 3), device="cuda")
    packed, ts, te, sg = api.march_with_density(z, z, grid, dens, render_step_size=inf.dt_min)
    assert packed.shape == (0, 2) and ts.shape == (0, 1) and sg.shape == (0, 1)
    # rays that miss the box: packed counts zero, no samples
    o = torch.tensor([[5.0, 5.0, 5.0], [0.0, 9.0, 0.0]], device="cuda")
    d = torch.tensor([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], device="cuda")
    packed, ts, te, sg = api.march_with_density(o, d, grid, dens, render_step_size=inf.dt_min)
    assert packed[:, 1].sum().item() == 0 and ts.numel() == 0
