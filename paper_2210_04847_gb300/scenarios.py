"""Benchmark scenarios: seeded inputs of each workload, ready on the device.

A scenario bundles what a training step needs besides the library: ray batches
(origins, directions, targets, per-ray time or scene slot), the stand-in field of
the user's network (one blob scene, a batch of scenes, or moving blobs), and the
inputs of the occupancy-grid update (random cells, a point inside each, the
time of the point). Workloads:

* ``bounded``   2^18 rays, 100 cameras at 800x800, 64 blobs, one 128^3 grid
* ``tiny``      one 64x64 camera, 8 blobs, 64^3 grid, no pruning
* ``unbounded`` 2^20 rays from inside a radius-1000 scene, 4-level cascade, cone steps
* ``contracted`` the unbounded scene and rays, one 128^3 grid over contracted space
* ``batched``   64 scenes (8-256 blobs, own 128^3 grid each), lognormal rays per scene
* ``dynamic``   2^19 rays over 16 time bins of 128 moving blobs, one grid per bin
* ``dynamic_shared`` the same with one grid for all times (maximum over time)
"""
from __future__ import annotations

import numpy as np
import torch

from . import synth
from .pipeline import StandInField, to_device

N_GRID_SAMPLES = 1 << 21


class Scenario:
    def __init__(self, name, workloads, scenes, device, n_grid_samples=N_GRID_SAMPLES, rank=0):
        self.name = name
        self.device = device
        self.w = workloads[0]
        self.batches = []
        for w in workloads:
            self.batches.append(dict(
                o=to_device(w.rays_o, device), d=to_device(w.rays_d, device), tgt=to_device(w.target_rgb, device)
                if w.target_rgb is not None else None, time=to_device(w.ray_time, device),
                slot=to_device(w.ray_slot, device), host=w))
        self.scenes = scenes
        self.fields = [StandInField(s, device) for s in scenes]
        w = self.w
        self.n_cells = int(np.prod(w.res)) * w.n_levels * w.n_slots
        self.n_grid = n_grid_samples
        self.rank = rank
        # scene of each slot (batched) or one scene for every slot (time bins)
        self.slot_scene = list(range(len(scenes))) if len(scenes) == w.n_slots and len(scenes) > 1 else [0] * w.n_slots
        self.rays_per_scene = w.meta.get("rays_per_scene")

    @property
    def n_rays(self):
        return self.w.n_rays

    # -- the user's network -----------------------------------------------
    def _scene_ranges(self, packed_info, total):
        """Sample ranges of each scene (rays are scene-major) -> [(scene, start, end)]."""
        if len(self.fields) == 1:
            return [(0, 0, total)]
        counts = np.asarray(self.rays_per_scene)
        first = np.concatenate([[0], np.cumsum(counts)[:-1]])
        starts = packed_info[torch.from_numpy(first).to(packed_info.device).long(), 0].cpu().numpy()
        ends = list(starts[1:]) + [total]
        return [(s, int(a), int(b)) for s, (a, b) in enumerate(zip(starts, ends))]

    def field_marched(self, hp, b, M):
        bt = self.batches[b]
        for s, a, e in self._scene_ranges(hp.pi_m, M):
            if e > a:
                self.fields[s].samples(bt["o"], bt["d"], hp.ri_m[a:e], hp.ts_m[a:e], hp.te_m[a:e], e - a,
                                       hp.sig_m[a:e], None, ray_time=bt["time"])

    def field_kept(self, hp, b, S):
        bt = self.batches[b]
        for s, a, e in self._scene_ranges(hp.pi_k, S):
            if e > a:
                self.fields[s].samples(bt["o"], bt["d"], hp.ri_k[a:e], hp.ts_k[a:e], hp.te_k[a:e], e - a,
                                       hp.sig_k[a:e], hp.rgb_k[a:e], ray_time=bt["time"])

    # -- occupancy-grid update inputs ---------------------------------------
    def grid_inputs(self, step):
        """Uniform random cells over every slot and level, a jittered point in each, its time."""
        w = self.w
        cells, jit = synth.grid_update_samples(self.rank, step, self.n_grid, w.res, w.n_levels, w.n_slots)
        xyz = synth.cell_positions(cells, jit, w.aabb, w.res, w.n_levels, contraction=w.contraction)
        per_slot = int(np.prod(w.res)) * w.n_levels
        slot = cells.astype(np.int64) // per_slot
        times = None
        if w.ray_time is not None:  # time bins: the point's time is the bin centre
            times = to_device(((slot + 0.5) / w.n_slots).astype(np.float32), self.device)
        return dict(cells=to_device(cells, self.device), xyz=to_device(xyz.astype(np.float32), self.device),
                    times=times, slot=slot)

    def grid_field(self, gi, out, xyz=None, cells=None):
        """Density of each grid-update point under its slot's scene. ``xyz`` /
        ``cells``: the device sampler's output for the same step (equal to
        gi's); with one scene the field reads those directly."""
        if len(self.fields) == 1:
            times = gi["times"]
            if times is not None and cells is not None:  # the point's time is its bin centre
                per_slot = int(np.prod(self.w.res)) * self.w.n_levels
                times = (((cells.long() // per_slot).double() + 0.5) / self.w.n_slots).float()
            self.fields[0].points(gi["xyz"] if xyz is None else xyz, self.n_grid, out, times=times)
            return
        order = np.argsort(gi["slot"], kind="stable")
        # evaluate scene by scene on gathered points, then scatter back
        for s in range(len(self.fields)):
            idx = order[np.searchsorted(gi["slot"][order], s, "left"):np.searchsorted(gi["slot"][order], s, "right")]
            if idx.size == 0:
                continue
            it = torch.from_numpy(idx).to(self.device)
            xyz = gi["xyz"][it].contiguous()
            tmp = torch.empty(idx.size, dtype=torch.float32, device=self.device)
            self.fields[s].points(xyz, idx.size, tmp)
            out[it] = tmp

    # -- graph-capturable field (device-side counts, scene chosen per ray) ----
    def _multi_tables(self):
        if not hasattr(self, "_mt"):
            tabs = [sc.device_params() for sc in self.scenes]
            off = np.concatenate([[0], np.cumsum([t.shape[0] for t in tabs])]).astype(np.int32)
            wb = np.stack([np.concatenate([sc.rgb_w.reshape(-1), sc.rgb_b]) for sc in self.scenes]).astype(np.float32)
            self._mt = (to_device(np.concatenate(tabs), self.device), to_device(off, self.device),
                        to_device(wb, self.device))
        return self._mt

    def field_marched_dev(self, hp, b):
        from . import _lib

        bt = self.batches[b]
        blobs, off, wb = self._multi_tables()
        _lib.field_samples_multi(bt["o"], bt["d"], bt["slot"], hp.ri_m, hp.ts_m, hp.te_m, hp.n_m, hp.cap_m, blobs,
                                 off, wb, hp.sig_m, None, ray_time=bt["time"])

    def field_kept_dev(self, hp, b):
        from . import _lib

        bt = self.batches[b]
        blobs, off, wb = self._multi_tables()
        _lib.field_samples_multi(bt["o"], bt["d"], bt["slot"], hp.ri_k, hp.ts_k, hp.te_k, hp.n_k, hp.cap_k, blobs,
                                 off, wb, hp.sig_k, hp.rgb_k, ray_time=bt["time"])

    def ema_init(self):
        """float32 EMA grid initialised from the densities at the cell centres (the rule that built the bits)."""
        w = self.w
        if w.contraction:
            return synth.density_at_contracted_centres(self.scenes[0], w.aabb, w.res, self.device).float()
        if w.n_slots == 1:
            return synth.density_at_cell_centres(self.scenes[0], w.aabb, w.res, w.n_levels, None,
                                                 self.device).float()
        parts = []
        for k in range(w.n_slots):
            scene = self.scenes[self.slot_scene[k]]
            t = (k + 0.5) / w.n_slots if w.ray_time is not None else None
            parts.append(synth.density_at_cell_centres(scene, w.aabb, w.res, w.n_levels, t, self.device).float())
        return torch.cat(parts)


def make_scenario(name: str, rank: int = 0, device="cuda", n_rays=None, pool: int = 4, ray_scale: float = 1.0) -> Scenario:
    """Seeded scenario; each rank draws its own ray batches (ranks share no work).
    ray_scale: the batched workload's rays per scene scaled (a smaller case)."""
    batches = [rank * 1000 + b for b in range(pool)]
    if name == "bounded":
        sg = synth.bounded_scene(0, device=device)
        ws = [synth.bounded_config(0, n_rays=n_rays or (1 << 18), scene_grid=sg, batch=b) for b in batches]
        return Scenario(name, ws, [sg[0]], device, rank=rank)
    if name == "tiny":
        w = synth.tiny_config(0, device=device)
        w.target_rgb = synth.rand_uniform(0, 77, 3 * w.n_rays).reshape(-1, 3).astype(np.float32)
        return Scenario(name, [w], w.scenes, device, n_grid_samples=1 << 16, rank=rank)
    if name == "contracted":
        ws = [synth.contracted_config(0, n_rays=n_rays or (1 << 20), device=device, batch=b) for b in batches[:1]]
        return Scenario(name, ws, ws[0].scenes, device, rank=rank)
    if name == "unbounded":
        ws = [synth.unbounded_config(0, n_rays=n_rays or (1 << 20), device=device, batch=b) for b in batches[:1]]
        return Scenario(name, ws, ws[0].scenes, device, rank=rank)
    if name == "batched":
        w = synth.batched_config(0, device=device, ray_scale=ray_scale)
        return Scenario(name, [w], w.scenes, device, rank=rank)
    if name == "dynamic_shared":
        ws = [synth.dynamic_shared_config(0, n_rays=n_rays or (1 << 19), device=device, batch=b) for b in batches[:2]]
        return Scenario(name, ws, ws[0].scenes, device, rank=rank)
    if name == "dynamic":
        ws = [synth.dynamic_config(0, n_rays=n_rays or (1 << 19), device=device, batch=b) for b in batches[:2]]
        return Scenario(name, ws, ws[0].scenes, device, rank=rank)
    raise ValueError("unknown workload " + name)
