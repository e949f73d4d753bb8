"""The paper-shaped Python API (Sec. 3 listing) on the GPU: ray_marching with a
density callback and pruning, rendering with autograd, the occupancy grid's
update; compared with the oracle on seeded inputs."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, dev, grad_rel_err, oracle_march, render_tol_ok  # noqa: E402
from paper_2210_04847_gb300 import api  # noqa: E402


def _host_field(scene, rays_o, rays_d):
    """Callbacks backed by the host generator (values identical for both sides)."""

    def sigma_fn(ts, te, ri):
        s, _ = synth.sample_field(scene, rays_o, rays_d, ts.view(-1).cpu().numpy(), te.view(-1).cpu().numpy(),
                                  ri.cpu().numpy())
        return torch.from_numpy(s).cuda().view(-1, 1)

    def rgb_sigma_fn(ts, te, ri):
        s, c = synth.sample_field(scene, rays_o, rays_d, ts.view(-1).cpu().numpy(), te.view(-1).cpu().numpy(),
                                  ri.cpu().numpy())
        return torch.from_numpy(c).cuda().requires_grad_(True), torch.from_numpy(s).cuda().view(-1, 1).requires_grad_(True)

    return sigma_fn, rgb_sigma_fn


def test_api_train_step_matches_oracle(orc):
    w = synth.bounded_config(4, n_rays=1500, device="cuda")
    scene = w.scenes[0]
    grid = api.OccupancyGrid.from_bits(w.bits, w.res, w.aabb)
    o, d = torch.from_numpy(w.rays_o).cuda(), torch.from_numpy(w.rays_d).cuda()
    sigma_fn, rgb_sigma_fn = _host_field(scene, w.rays_o, w.rays_d)
    packed, ts, te = api.ray_marching(o, d, grid, sigma_fn=sigma_fn, near_plane=w.near_plane,
                                      far_plane=w.far_plane, render_step_size=w.dt_min, max_steps=w.max_steps,
                                      early_stop_eps=w.early_stop_eps, alpha_thre=w.alpha_thre)
    assert ts.shape[1] == 1 and packed.shape == (1500, 2)
    # oracle: march, field, prune
    m = orc.march(w.rays_o, w.rays_d, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, 0.0,
                  w.max_steps)
    sg, _ = synth.sample_field(scene, w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    p, keep, _ = orc.prune(m.packed_info, m.t_starts, m.t_ends, sg, w.early_stop_eps, w.alpha_thre)
    if not np.array_equal(packed.cpu().numpy(), p.packed_info):
        pytest.skip("a prune decision fell within rounding of the threshold on this seed")
    assert bits_equal(ts.view(-1).cpu().numpy(), p.t_starts) and bits_equal(te.view(-1).cpu().numpy(), p.t_ends)
    rgbs, sigmas = rgb_sigma_fn(ts, te, api.unpack_info(packed, ts.shape[0]))
    color, opacity, depth = api.render_packed(sigmas, rgbs, packed, ts, te)
    target = torch.from_numpy(w.target_rgb).cuda()
    loss = torch.nn.functional.mse_loss(color, target)
    loss.backward()
    sg2, rgb2 = synth.sample_field(scene, w.rays_o, w.rays_d, p.t_starts, p.t_ends, p.ray_indices)
    c_o, a_o, d_o = orc.render_fwd(p.packed_info, p.t_starts, p.t_ends, sg2, rgb2)
    assert render_tol_ok(color.detach().cpu().numpy(), c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(opacity.detach().cpu().numpy()[:, 0], a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(depth.detach().cpu().numpy()[:, 0], d_o) <= 1.0
    gc = 2.0 * (color.detach().cpu().numpy().astype(np.float64) - w.target_rgb) / color.numel()
    ds_o, dr_o = orc.render_bwd(p.packed_info, p.t_starts, p.t_ends, sg2, rgb2, gc)
    assert grad_rel_err(sigmas.grad.view(-1).cpu().numpy(), ds_o) <= 1e-4
    assert grad_rel_err(rgbs.grad.cpu().numpy(), dr_o) <= 1e-4
    # saved optical depth path gives identical gradients
    sig_b = sigmas.detach().clone().requires_grad_(True)
    rgb_b = rgbs.detach().clone().requires_grad_(True)
    c2, _, _ = api.render_packed(sig_b, rgb_b, packed, ts, te, save_optical_depth=True)
    torch.nn.functional.mse_loss(c2, target).backward()
    assert torch.equal(sig_b.grad, sigmas.grad) and torch.equal(rgb_b.grad, rgbs.grad)


def test_api_grid_update_and_weights(orc):
    g = api.OccupancyGrid((-1, -1, -1, 1, 1, 1), 32)
    g.ema.copy_(torch.from_numpy(synth.rand_uniform(3, 1, 32 ** 3, 0, 0.02).astype(np.float32)))
    ema0 = g.ema.cpu().numpy()
    cells = synth.rand_int(3, 2, 5000, 32 ** 3).astype(np.int32)
    sig = synth.rand_uniform(3, 3, 5000, 0, 0.05).astype(np.float32)
    g.update(torch.from_numpy(cells).cuda(), torch.from_numpy(sig).cuda(), 0.9, 0.01)
    e_o, b_o = orc.update_grid(ema0, cells, sig, 0.9, 0.01)
    assert bits_equal(g.ema.cpu().numpy(), e_o) and np.array_equal(g.bits.cpu().numpy().view(np.uint32), b_o)
    # the opacity criterion (alpha of a step dt above 0.01) is the converted density threshold
    ga = api.OccupancyGrid((-1, -1, -1, 1, 1, 1), 32)
    ga.ema.copy_(torch.from_numpy(ema0))
    ga.update(torch.from_numpy(cells).cuda(), torch.from_numpy(sig).cuda(), 0.9, 0.01, alpha_step=0.5)
    e_a, b_a = orc.update_grid(ema0, cells, sig, 0.9, 0.01, alpha_step=0.5)
    assert bits_equal(ga.ema.cpu().numpy(), e_a)
    # the oracle decides with the opacity criterion in float64; the library with its
    # float32 density threshold: they may differ only within rounding of the threshold
    got = np.unpackbits(ga.bits.cpu().numpy().view(np.uint32).view(np.uint8), bitorder="little")[:32 ** 3]
    ref = np.unpackbits(b_a.view(np.uint8), bitorder="little")[:32 ** 3]
    near = np.abs(e_a.astype(np.float64) - (-np.log1p(-0.01) / 0.5)) <= 1e-6 * 0.0201
    assert np.array_equal(got[~near], ref[~near]) and near.sum() <= 2
    assert not np.array_equal(b_a, b_o)  # a different threshold (0.0201 against 0.01)
    sd = g.state_dict()
    g2 = api.OccupancyGrid((-1, -1, -1, 1, 1, 1), 32)
    g2.load_state_dict(sd)
    assert torch.equal(g2.ema, g.ema) and torch.equal(g2.bits, g.bits)
    pi = torch.tensor([[0, 3], [3, 2]], dtype=torch.int32, device="cuda")
    ts = torch.tensor([0.0, 0.5, 1.0, 2.0, 2.5], device="cuda")
    sgm = torch.tensor([1.0, 2.0, 0.5, 4.0, 0.0], device="cuda")
    wts, T = api.render_weights(pi, ts, ts + 0.5, sgm)
    w_o, T_o = orc.render_weights(pi.cpu().numpy(), ts.cpu().numpy(), (ts + 0.5).cpu().numpy(), sgm.cpu().numpy())
    assert np.max(np.abs(wts.cpu().numpy() - w_o)) < 1e-6 and np.max(np.abs(T.cpu().numpy() - T_o)) < 1e-6
    acc = api.accumulate_along_rays(wts, pi, torch.ones(5, 2, device="cuda"))
    assert np.allclose(acc.cpu().numpy(), np.stack([orc.accumulate(pi.cpu().numpy(), w_o)[:, 0]] * 2, 1), atol=1e-6)


def test_weights_and_accumulate_compose_to_render(orc):
    """Autograd through render_weights + accumulate_along_rays (any attributes) gives the
    fused render's outputs and gradients: colour, opacity and depth as three accumulations."""
    w = synth.bounded_config(4, n_rays=600, device="cuda")
    m = oracle_march(orc, w)
    sig, rgb = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    pi, ts, te = dev(m.packed_info), dev(m.t_starts), dev(m.t_ends)
    tgt = torch.rand((w.n_rays, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(3))

    def loss_of(col, op, dp):
        return ((col - tgt) ** 2).mean() + 0.1 * op.sum() / w.n_rays + 0.01 * dp.sum() / w.n_rays

    s1 = dev(sig).requires_grad_(True)
    r1 = dev(rgb).requires_grad_(True)
    col, op, dp = api.render_packed(s1, r1, pi, ts, te)
    loss_of(col, op.view(-1), dp.view(-1)).backward()
    s2 = dev(sig).requires_grad_(True)
    r2 = dev(rgb).requires_grad_(True)
    wts, _ = api.render_weights(pi, ts, te, s2)
    tm = ((ts + te) * 0.5).view(-1, 1)
    col2 = api.accumulate_along_rays(wts, pi, r2)
    op2 = api.accumulate_along_rays(wts, pi)
    dp2 = api.accumulate_along_rays(wts, pi, tm)
    loss_of(col2, op2.view(-1), dp2.view(-1)).backward()
    assert torch.allclose(col, col2, atol=1e-5) and torch.allclose(op.view(-1), op2.view(-1), atol=1e-5)
    # both paths against the oracle's gradient for the same upstream gradients (the
    # loss's, from the fused colours), both at the 1e-4 bar: the three accumulations
    # hand render_weights dL/dw centred on each ray's first sample (their per-ray
    # parts summed on the side), so the scan never subtracts nearly equal float32
    # values.
    R = w.n_rays
    gc = 2.0 * (col.detach().double() - tgt.double()).cpu().numpy() / (3 * R)
    ds_o, dr_o = orc.render_bwd(m.packed_info, m.t_starts, m.t_ends, sig, rgb, gc, np.full(R, 0.1 / R),
                                np.full(R, 0.01 / R))
    assert grad_rel_err(s1.grad.cpu().numpy(), ds_o) <= 1e-4
    assert grad_rel_err(s2.grad.cpu().numpy(), ds_o) <= 1e-4
    for r_ in (r1, r2):
        assert grad_rel_err(r_.grad.cpu().numpy(), dr_o) <= 1e-4
    # a second backward through the same graph gives the same gradient (the side
    # buffer is handed over and cleared by each backward)
    s3 = dev(sig).requires_grad_(True)
    wts3, _ = api.render_weights(pi, ts, te, s3)
    lo3 = ((api.accumulate_along_rays(wts3, pi, r2.detach()) - tgt) ** 2).mean()
    lo3.backward(retain_graph=True)
    g_first = s3.grad.clone()
    s3.grad = None
    lo3.backward()
    assert torch.equal(s3.grad, g_first)
    # weights that are not render_weights' own tensor (here scaled) take the
    # uncentred path, still exact up to float32 rounding
    s4 = dev(sig).requires_grad_(True)
    wts4, _ = api.render_weights(pi, ts, te, s4)
    ((api.accumulate_along_rays(wts4 * 1.0, pi, r2.detach()) - tgt) ** 2).mean().backward()
    assert grad_rel_err(s4.grad.cpu().numpy(), g_first.cpu().numpy()) <= 1e-3


def test_march_without_a_grid_then_render_with_gradients(orc):
    """ray_marching accepts no occupancy grid (Sec. 3): every lattice step between
    near_plane and far_plane is marched, pruned with the field's density queried
    without gradients, and rendered with gradients reaching the field's weights."""
    from paper_2210_04847_gb300 import api as nacc

    rng = np.random.default_rng(8)
    n = 300
    rays_o = torch.from_numpy(rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32)).cuda()
    d = rng.normal(size=(n, 3))
    rays_d = torch.from_numpy((d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)).cuda()
    w_field = torch.tensor([[2.0, -1.0, 0.5], [0.3, 0.2, -0.4], [-0.6, 0.9, 0.1]], device="cuda", requires_grad=True)

    def field(ts, te, ri):
        pos = rays_o[ri] + rays_d[ri] * (ts + te) / 2.0
        density = 30.0 * torch.exp(-4.0 * (pos * pos).sum(-1, keepdim=True))
        return torch.sigmoid(pos @ w_field), density

    # planes 0.2 .. 1.0 with the default 1e-2 step: 81 lattice steps per ray
    # before pruning; eps and the opacity threshold at values that prune some
    packed_info, t_starts, t_ends = nacc.ray_marching(rays_o, rays_d, sigma_fn=lambda *a: field(*a)[1],
                                                      near_plane=0.2, far_plane=1.0, early_stop_eps=1e-3,
                                                      alpha_thre=5e-3)
    assert int(packed_info[:, 1].max()) <= 81
    color, opacity, depth = nacc.rendering(field, packed_info, t_starts, t_ends)
    loss = torch.nn.functional.mse_loss(color, torch.full_like(color, 0.5))
    loss.backward()
    assert torch.isfinite(w_field.grad).all() and float(w_field.grad.abs().sum()) > 0
    # marching without a grid: every step of the lattice between the planes
    m = orc.march(rays_o.cpu().numpy(), rays_d.cpu().numpy(), np.array([1], np.uint32), (1, 1, 1),
                  (-1e6, -1e6, -1e6, 1e6, 1e6, 1e6), 0.2, 1.0, 1e-2, 1e-2, 0.0, 1024, contraction=1)
    near, dt = np.float32(0.2), np.float32(0.01)
    k_max = sum(1 for k in range(200) if near + np.float32(k) * dt < np.float32(1.0))  # float32 lattice: 81
    assert np.all(m.packed_info[:, 1] == k_max)
    packed, ts, te, ri = nacc.march_rays(rays_o, rays_d, near_plane=0.2, far_plane=1.0)
    assert np.array_equal(packed.cpu().numpy(), m.packed_info) and bits_equal(ts.cpu().numpy(), m.t_starts)
    assert float(opacity.detach().max()) > 0.5 and float(opacity.detach().min()) >= 0.0


def test_capacity_mode_step_matches_exact_mode():
    """ray_marching(capacity=...) + rendering(n_samples=...): no host read during the
    step; the same packed samples, colours and gradients as the exact mode, zero
    gradients on the padding past the device count, and a capacity too small
    reported in the step's status word."""
    w = synth.bounded_config(4, n_rays=2000, device="cuda")
    scene = w.scenes[0]
    grid = api.OccupancyGrid.from_bits(w.bits, w.res, w.aabb)
    o, d = torch.from_numpy(w.rays_o).cuda(), torch.from_numpy(w.rays_d).cuda()
    from paper_2210_04847_gb300.pipeline import StandInField

    field = StandInField(scene, "cuda")

    def sigma_fn(ts, te, ri):
        sig = torch.empty(ts.shape[0], device="cuda")
        field.samples(o, d, ri, ts.view(-1), te.view(-1), ts.shape[0], sig)
        return sig.view(-1, 1)

    def rgb_sigma_fn(ts, te, ri):
        sig = torch.empty(ts.shape[0], device="cuda")
        rgb = torch.empty((ts.shape[0], 3), device="cuda")
        field.samples(o, d, ri, ts.view(-1), te.view(-1), ts.shape[0], sig, rgb)
        return rgb.requires_grad_(True), sig.view(-1, 1).requires_grad_(True)

    kw = dict(near_plane=w.near_plane, far_plane=w.far_plane, render_step_size=w.dt_min, max_steps=w.max_steps,
              early_stop_eps=w.early_stop_eps, alpha_thre=w.alpha_thre)
    tgt = torch.from_numpy(w.target_rgb).cuda()
    grads = {}

    def grab(name):
        def fn(ts, te, ri):
            rgb, sig = rgb_sigma_fn(ts, te, ri)
            grads[name] = (rgb, sig)
            return rgb, sig
        return fn

    packed, ts, te, ri = api.ray_marching(o, d, grid, sigma_fn=sigma_fn, return_ray_indices=True, **kw)
    col, _, _ = api.rendering(grab("exact"), packed, ts, te, ray_indices=ri)
    torch.nn.functional.mse_loss(col, tgt).backward()
    S = ts.shape[0]
    cap = S + 5000  # room for the marched samples too (pruning keeps fewer)
    cap = max(cap, int(1.3 * 2000 * 500))
    api.check_status("cuda")
    packed_c, ts_c, te_c, ri_c, n_c = api.ray_marching(o, d, grid, sigma_fn=sigma_fn, capacity=cap,
                                                       kept_capacity=S + 777, **kw)
    col_c, _, _ = api.rendering(grab("cap"), packed_c, ts_c, te_c, ray_indices=ri_c, n_samples=n_c)
    torch.nn.functional.mse_loss(col_c, tgt).backward()
    api.check_status("cuda")
    assert int(n_c.item()) == S and torch.equal(packed_c, packed)
    assert torch.equal(ts_c[:S].view(-1), ts.view(-1)) and torch.equal(ri_c[:S], ri)
    assert torch.equal(col_c, col)
    (r_e, s_e), (r_c, s_c) = grads["exact"], grads["cap"]
    assert torch.equal(s_c.grad[:S], s_e.grad) and torch.equal(r_c.grad[:S], r_e.grad)
    assert (s_c.grad[S:] == 0).all() and (r_c.grad[S:] == 0).all()
    # a capacity below the marched count: reported, nothing written past it
    api.ray_marching(o, d, grid, sigma_fn=sigma_fn, capacity=1000, **kw)
    with pytest.raises(_lib_error()):
        api.check_status("cuda")


def _lib_error():
    from paper_2210_04847_gb300 import _lib

    return _lib.NaccError
