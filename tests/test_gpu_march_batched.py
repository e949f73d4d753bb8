"""nacc_march_rays_batched: scenes with their own grids (resolution, box, level
count, contraction) marched in one persistent launch, bit-exact against the
oracle run scene by scene (Sec. 2.1: each scene keeps its own occupancy grid)."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import assert_march_equal, dev  # noqa: E402


def _scene(seed, res, aabb, n_levels, n_rays, contraction=0):
    """A blob scene in the box, its grid, and rays from outside the outermost box
    aimed at random points inside the level-0 box (a few aimed past it)."""
    lo, hi = np.array(aabb[:3]), np.array(aabb[3:])
    c, h = (lo + hi) / 2, (hi - lo) / 2
    sc = synth.make_blob_scene(seed, 24)
    sc.centers = c + sc.centers * h  # move the unit-cube blobs into this box
    sc.scales = sc.scales * float(np.mean(h))
    if contraction:
        bits = synth.occupancy_bits_contracted(sc, aabb, res, 0.01)
    else:
        bits = synth.occupancy_bits(sc, aabb, res, n_levels, 0.01)
    u = synth.random_unit_vectors(seed, 50, n_rays)
    o = c + u * (np.linalg.norm(h) * 2.0 ** n_levels * 1.1)
    tgt = c + (synth.rand_uniform(seed, 51, 3 * n_rays, -1.2, 1.2).reshape(n_rays, 3)) * h
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return dict(bits=bits, res=res, aabb=aabb, n_levels=n_levels, contraction=contraction,
                o=o.astype(np.float32), d=d.astype(np.float32))


def _run(orc, scenes, near, far, dt_min, dt_max, cone, max_steps):
    o = np.concatenate([s["o"] for s in scenes])
    d = np.concatenate([s["d"] for s in scenes])
    R = o.shape[0]
    params = _lib.make_params(near, far, dt_min, dt_max, cone, max_steps)
    bits_t = [dev(s["bits"]) for s in scenes]
    descs = _lib.make_scenes([(b, s["res"], s["aabb"], s["n_levels"], s["contraction"], s["o"].shape[0],
                               s.get("sat")) for b, s in zip(bits_t, scenes)])
    # the oracle, scene by scene, stitched into one packed batch
    pis, ts, te, ri = [], [], [], []
    off, base = 0, 0
    for s in scenes:
        n = s["o"].shape[0]
        if n == 0:
            continue
        m = orc.march(s["o"], s["d"], s["bits"], s["res"], s["aabb"], near, far, dt_min, dt_max, cone, max_steps,
                      n_levels=s["n_levels"], contraction=s["contraction"])
        pi = m.packed_info.copy()
        pi[:, 0] += off
        pis.append(pi)
        ts.append(m.t_starts)
        te.append(m.t_ends)
        ri.append(m.ray_indices + base)
        off += m.n_samples
        base += n

    class Ref:
        packed_info = np.concatenate(pis)
        t_starts, t_ends, ray_indices = np.concatenate(ts), np.concatenate(te), np.concatenate(ri)
        n_samples = off

    cap = max(off, 1)
    ws = torch.zeros(_lib.march_batched_workspace_size(len(scenes), R, params), dtype=torch.uint8, device="cuda")
    out = (torch.full((R, 2), -1, dtype=torch.int32, device="cuda"), torch.full((cap,), np.nan, device="cuda"),
           torch.full((cap,), np.nan, device="cuda"), torch.full((cap,), -1, dtype=torch.int32, device="cuda"))
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.march_rays_batched(descs, dev(o), dev(d), params, *out, n, st, ws)
    torch.cuda.synchronize()
    k = int(n.item())
    got = (out[0].cpu().numpy(), out[1][:k].cpu().numpy(), out[2][:k].cpu().numpy(), out[3][:k].cpu().numpy(), k,
           int(st.item()))
    assert_march_equal(got, Ref)
    assert off > 1000
    return descs, dev(o), dev(d), params, ws, got


def test_one_level_scenes_of_different_resolution_and_box(orc):
    scenes = [_scene(1, (64, 64, 64), (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5), 1, 700),
              _scene(2, (96, 80, 128), (-2.0, -1.0, -1.5, 2.0, 1.0, 1.5), 1, 900),
              _scene(3, (16, 16, 16), (0.0, 0.0, 0.0, 1.0, 1.0, 1.0), 1, 0),  # a scene without rays
              _scene(4, (33, 47, 29), (-0.5, -3.0, 2.0, 0.5, -1.0, 2.5), 1, 400)]
    _run(orc, scenes, 0.0, 1e10, 0.0051, 0.0051, 0.0, 1024)


def test_cascades_and_cone_steps(orc):
    scenes = [_scene(5, (32, 32, 32), (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0), 3, 500),
              _scene(6, (48, 40, 56), (-2.0, -2.0, -1.0, 2.0, 2.0, 1.0), 1, 600),
              _scene(7, (24, 24, 24), (-0.5, -0.5, -0.5, 0.5, 0.5, 0.5), 5, 400)]
    _run(orc, scenes, 0.02, 50.0, 1e-3, 0.5, 1.0 / 128.0, 4096)
    _run(orc, scenes, 0.0, 1e10, 0.004, 0.004, 0.0, 2048)


def test_contracted_scenes(orc):
    scenes = [_scene(8, (64, 64, 64), (-10.0, -10.0, -10.0, 10.0, 10.0, 10.0), 1, 500, contraction=1),
              _scene(9, (32, 48, 40), (-4.0, -2.0, -3.0, 4.0, 2.0, 3.0), 1, 500, contraction=1)]
    _run(orc, scenes, 0.05, 200.0, 1e-3, 1.0, 1.0 / 256.0, 4096)


def test_batched_march_replays_in_a_cuda_graph(orc):
    scenes = [_scene(1, (64, 64, 64), (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5), 1, 700),
              _scene(2, (96, 80, 128), (-2.0, -1.0, -1.5, 2.0, 1.0, 1.5), 1, 900)]
    descs, o, d, params, ws, ref = _run(orc, scenes, 0.0, 1e10, 0.0051, 0.0051, 0.0, 1024)
    R, k = o.shape[0], ref[4]
    out = (torch.zeros((R, 2), dtype=torch.int32, device="cuda"), torch.zeros(k, device="cuda"),
           torch.zeros(k, device="cuda"), torch.zeros(k, dtype=torch.int32, device="cuda"))
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _lib.march_rays_batched(descs, o, d, params, *out, n, st, ws)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        _lib.march_rays_batched(descs, o, d, params, *out, n, st, ws)
    for _ in range(2):
        out[1].fill_(np.nan)
        out[0].fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert int(n.item()) == k and int(st.item()) == 0
        assert np.array_equal(out[0].cpu().numpy(), ref[0])
        assert np.array_equal(out[1].cpu().numpy().view(np.uint32), ref[1].view(np.uint32))
