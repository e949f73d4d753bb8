"""The batched training step captured in one CUDA graph, against the eager calls
and the oracle.

64 scenes, each with its own 128^3 grid (slots of one grid), lognormal ray counts
at 1/8 of the benchmark's scale. The graph holds march -> field -> prune -> field
-> render forward -> loss gradient -> render backward with the buffer capacities
as sample bounds and the counts on the device, so no host read happens inside
it. Two replays must give exactly what the eager sequence (exact counts, host
reads between stages) gives, and sampled rays of every scene must match the
oracle: marching and pruning bit for bit, colours within 1e-5, gradients within
1e-4.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, grad_rel_err, near_threshold, render_tol_ok  # noqa: E402
from paper_2210_04847_gb300.pipeline import HotPath  # noqa: E402
from paper_2210_04847_gb300.scenarios import Scenario  # noqa: E402

RAYS_PER_SCENE_SAMPLED = 4


@pytest.fixture(scope="module")
def batched():
    w = synth.batched_config(0, device="cuda", ray_scale=0.125)
    sc = Scenario("batched", [w], w.scenes, "cuda", n_grid_samples=0)
    return w, sc


def _eager(sc, hp):
    """The step as plain calls with exact sample counts (host reads between stages)."""
    bt = sc.batches[0]
    hp.march(bt["o"], bt["d"], bt["time"], bt["slot"])
    M = int(hp.n_m.item())
    sc.field_marched_dev(hp, 0)
    hp.prune(M)
    S = int(hp.n_k.item())
    sc.field_kept_dev(hp, 0)
    hp.render_fwd(S)
    hp.loss_grad(bt["tgt"])
    hp.render_bwd(S)
    torch.cuda.synchronize()
    hp.check_status("eager")
    return M, S


def _snapshot(hp, M, S):
    c = lambda t: t.detach().clone()
    return dict(pi_m=c(hp.pi_m), ts_m=c(hp.ts_m[:M]), te_m=c(hp.te_m[:M]), ri_m=c(hp.ri_m[:M]), sig_m=c(hp.sig_m[:M]),
                pi_k=c(hp.pi_k), ts_k=c(hp.ts_k[:S]), te_k=c(hp.te_k[:S]), ri_k=c(hp.ri_k[:S]), sig_k=c(hp.sig_k[:S]),
                rgb_k=c(hp.rgb_k[:S]), color=c(hp.color), opacity=c(hp.opacity), depth=c(hp.depth),
                g_color=c(hp.g_color), d_sig=c(hp.d_sig[:S]), d_rgb=c(hp.d_rgb[:S]), M=M, S=S)


def test_graph_replay_matches_eager_and_oracle(batched, orc):
    w, sc = batched
    R = w.n_rays
    bt = sc.batches[0]
    probe = HotPath(w, cap_marched=R * 700, cap_kept=R * 700, device="cuda")
    M0, S0 = _eager(sc, probe)
    eager = _snapshot(probe, M0, S0)
    del probe
    torch.cuda.empty_cache()

    hp = HotPath(w, cap_marched=int(M0 * 1.3) + 4096, cap_kept=int(S0 * 1.3) + 4096, device="cuda")

    def body():
        hp.march(bt["o"], bt["d"], bt["time"], bt["slot"])
        sc.field_marched_dev(hp, 0)
        hp.prune(hp.cap_m)
        sc.field_kept_dev(hp, 0)
        hp.render_fwd(hp.cap_k)
        hp.loss_grad(bt["tgt"])
        hp.render_bwd(hp.cap_k)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        body()  # warm-up outside the capture (library attributes, torch kernels)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()
    for replay in range(2):
        for t in (hp.ts_m, hp.te_m, hp.sig_k, hp.color, hp.d_sig, hp.d_rgb):
            t.fill_(float("nan"))  # a replay must write everything that is compared
        hp.pi_m.fill_(-1)
        hp.pi_k.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        hp.check_status("graph replay %d" % replay)
        M, S = int(hp.n_m.item()), int(hp.n_k.item())
        assert M == eager["M"] and S == eager["S"], (replay, M, S)
        got = _snapshot(hp, M, S)
        for k in ("pi_m", "ri_m", "pi_k", "ri_k"):
            assert torch.equal(got[k], eager[k]), (replay, k)
        for k in ("ts_m", "te_m", "sig_m", "ts_k", "te_k", "sig_k", "rgb_k"):
            assert torch.equal(got[k].view(torch.int32), eager[k].view(torch.int32)), (replay, k)
        for k in ("color", "opacity", "depth"):
            assert render_tol_ok(got[k].cpu().numpy(), eager[k].cpu().numpy()) <= 1.0, (replay, k)
        for k in ("d_sig", "d_rgb"):
            assert grad_rel_err(got[k].cpu().numpy(), eager[k].cpu().numpy()) <= 1e-4, (replay, k)

    # every scene against the oracle on sampled rays
    counts = np.asarray(w.meta["rays_per_scene"])
    first = np.concatenate([[0], np.cumsum(counts)[:-1]])
    pick = np.concatenate([f + synth.rand_int(17, s, RAYS_PER_SCENE_SAMPLED, int(n))
                           for s, (f, n) in enumerate(zip(first, counts))]).astype(np.int64)
    pick = np.unique(pick)
    o, d, slot = w.rays_o[pick], w.rays_d[pick], w.ray_slot[pick]
    m = orc.march(o, d, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps,
                  n_levels=1, n_slots=w.n_slots, ray_slot=slot)
    pi_m = got["pi_m"].cpu().numpy()
    ts_m, te_m, sig_m = (got[k].cpu().numpy() for k in ("ts_m", "te_m", "sig_m"))
    assert np.array_equal(pi_m[pick, 1], m.packed_info[:, 1])
    sub = np.concatenate([np.arange(a, a + n) for a, n in pi_m[pick]]).astype(np.int64)
    assert bits_equal(ts_m[sub], m.t_starts) and bits_equal(te_m[sub], m.t_ends)
    # pruning: the oracle's decision on the GPU's marched samples and field values
    sg = sig_m[sub]
    pr, _, _ = orc.prune(m.packed_info, m.t_starts, m.t_ends, sg, w.early_stop_eps, w.alpha_thre)
    tau = sg.astype(np.float64) * (m.t_ends.astype(np.float64) - m.t_starts.astype(np.float64))
    od = np.zeros_like(tau)
    for a, n in m.packed_info:
        if n:
            od[a:a + n] = np.concatenate([[0.0], np.cumsum(tau[a:a + n])[:-1]])
    flip = near_threshold(m.packed_info, m.t_starts, m.t_ends, sg, w.early_stop_eps, od)
    pi_k = got["pi_k"].cpu().numpy()
    ts_k, te_k = got["ts_k"].cpu().numpy(), got["te_k"].cpu().numpy()
    clean = np.array([not flip[a:a + n].any() for a, n in m.packed_info])
    assert clean.mean() > 0.9
    for j in np.nonzero(clean)[0]:
        a, n = pi_k[pick[j]]
        b, nn = pr.packed_info[j]
        assert n == nn
        assert bits_equal(ts_k[a:a + n], pr.t_starts[b:b + nn]) and bits_equal(te_k[a:a + n], pr.t_ends[b:b + nn])
    # rendering and its gradient: the oracle on the GPU's kept samples of the sampled rays
    keep = np.concatenate([np.arange(a, a + n) for a, n in pi_k[pick]]).astype(np.int64)
    cnt = pi_k[pick, 1]
    pk = np.stack([np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt], 1).astype(np.int32)
    sgk, rgbk = got["sig_k"].cpu().numpy()[keep], got["rgb_k"].cpu().numpy()[keep]
    c_o, a_o, d_o = orc.render_fwd(pk, ts_k[keep], te_k[keep], sgk, rgbk)
    assert render_tol_ok(got["color"].cpu().numpy()[pick], c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["opacity"].cpu().numpy()[pick], a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["depth"].cpu().numpy()[pick], d_o) <= 1.0
    gc = got["g_color"].cpu().numpy()[pick].astype(np.float64)
    ds_o, dr_o = orc.render_bwd(pk, ts_k[keep], te_k[keep], sgk, rgbk, gc)
    assert grad_rel_err(got["d_sig"].cpu().numpy()[keep], ds_o) <= 1e-4
    assert grad_rel_err(got["d_rgb"].cpu().numpy()[keep], dr_o) <= 1e-4
