"""One training step of the marching + rendering path on preallocated buffers.

``HotPath`` holds capacity-sized device buffers for a workload and runs the
paper's pipeline (Sec. 2 and the Sec. 3 listing) as separate stages through the
C ABI:

    march  -> [field: density, no gradient] -> prune -> [field: rgb + density]
           -> render_fwd -> [loss gradient] -> render_bwd -> update_occupancy_grid

The bracketed steps belong to the user (the radiance field and the loss); here
the procedural stand-in field of ``libnacc_field.so`` plays that part. Each
stage can be bracketed by CUDA events on the launching stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _lib, synth


def to_device(a, device="cuda"):
    if a is None:
        return None
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(device)


@dataclass
class StepCounts:
    n_marched: int
    n_kept: int


class StandInField:
    """Procedural radiance field of a blob scene on the device (user side of the API)."""

    def __init__(self, scene: synth.BlobScene, device="cuda"):
        self.blobs = to_device(scene.device_params(), device)
        self.wb = to_device(np.concatenate([scene.rgb_w.reshape(-1), scene.rgb_b]).astype(np.float32), device)

    def samples(self, rays_o, rays_d, ray_indices, t_starts, t_ends, n, sigmas, rgbs=None, ray_time=None):
        _lib.field_samples(rays_o, rays_d, ray_indices, t_starts, t_ends, n, self.blobs, self.wb, sigmas, rgbs,
                           ray_time=ray_time)

    def points(self, xyz, n, sigmas, times=None):
        _lib.field_points(xyz, n, self.blobs, sigmas, times=times)


class HotPath:
    """Capacity-sized buffers and stage launchers for one workload."""

    def __init__(self, w: synth.Workload, cap_marched: int, cap_kept: int, n_grid_samples: int = 0,
                 device="cuda"):
        R = w.n_rays
        self.w = w
        self.R = R
        self.device = device
        self.bits = to_device(w.bits, device)
        self.n_cells = int(np.prod(w.res)) * w.n_levels * w.n_slots
        self.ema = torch.zeros(self.n_cells, dtype=torch.float32, device=device)
        self.params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
        self.grid = _lib.make_grid(self.bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)
        # uncontracted grids of up to four levels can march with their summed-area
        # table (the box walk); every grid update rebuilds the table of the bits it writes
        self.sat_ok = w.n_levels <= 4 and not w.contraction
        self.use_sat = self.sat_ok
        self.sat = _lib.build_grid_sat(self.grid) if self.sat_ok else None
        self.grid_sat = (_lib.make_grid(self.bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction, sat=self.sat)
                         if self.sat_ok else self.grid)
        self.upd_sat = None
        f32, i32 = torch.float32, torch.int32
        z = lambda n, dt=f32: torch.zeros(max(int(n), 1), dtype=dt, device=device)
        self.cap_m, self.cap_k = int(cap_marched), int(cap_kept)
        self.ws_march = z(_lib.march_workspace_size(R, self.params), torch.uint8)
        self.pi_m = torch.zeros((R, 2), dtype=i32, device=device)
        self.ts_m, self.te_m, self.ri_m, self.sig_m = z(self.cap_m), z(self.cap_m), z(self.cap_m, i32), z(self.cap_m)
        self.ws_prune = z(_lib.prune_workspace_size(R, self.cap_m), torch.uint8)
        self.pi_k = torch.zeros((R, 2), dtype=i32, device=device)
        self.ts_k, self.te_k, self.ri_k = z(self.cap_k), z(self.cap_k), z(self.cap_k, i32)
        self.sig_k, self.rgb_k = z(self.cap_k), torch.zeros((max(self.cap_k, 1), 3), dtype=f32, device=device)
        self.color = torch.zeros((R, 3), dtype=f32, device=device)
        self.opacity = torch.zeros(R, dtype=f32, device=device)
        self.depth = torch.zeros(R, dtype=f32, device=device)
        self.g_color = torch.zeros((R, 3), dtype=f32, device=device)
        self.d_sig, self.d_rgb = z(self.cap_k), torch.zeros((max(self.cap_k, 1), 3), dtype=f32, device=device)
        self.n_m = torch.zeros(1, dtype=torch.int64, device=device)
        self.n_k = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=i32, device=device)
        self.save_optical_depth = False  # forward stores O_i for the backward (instead of a recompute pass)
        self.od = None
        self.n_grid = int(n_grid_samples)
        self.cells = z(self.n_grid, i32)
        self.cell_xyz = torch.zeros((max(self.n_grid, 1), 3), dtype=f32, device=device)
        self.cell_sig = z(self.n_grid)

    # -- stages ------------------------------------------------------------
    # Each stage runs now, or with defer=True returns the marshalled call to run
    # later (so a timed region can start right before the C call).
    def march(self, rays_o, rays_d, ray_time=None, ray_slot=None, defer=False):
        grid = self.grid_sat if self.use_sat else self.grid
        return _lib.march_rays(rays_o, rays_d, grid, self.params, self.pi_m, self.ts_m[: self.cap_m],
                               self.te_m[: self.cap_m], self.ri_m[: self.cap_m], self.n_m, self.status, self.ws_march,
                               ray_time=ray_time, ray_slot=ray_slot, defer=defer)

    def prune(self, n_marched: int, defer=False):
        M = min(int(n_marched), self.cap_m)
        return _lib.prune_samples(self.pi_m, self.ts_m[:M], self.te_m[:M], self.sig_m[:M], M, self.w.early_stop_eps,
                                  self.w.alpha_thre, self.pi_k, self.ts_k[: self.cap_k], self.te_k[: self.cap_k],
                                  self.ri_k[: self.cap_k], self.n_k, self.status, self.ws_prune, defer=defer)

    def _od(self):
        if self.od is None:
            self.od = torch.zeros(max(self.cap_k, 1), dtype=torch.float32, device=self.device)
        return self.od

    def render_fwd(self, n_kept: int, defer=False):
        S = min(int(n_kept), self.cap_k)
        od = self._od()[:S] if self.save_optical_depth else None
        return _lib.render_fwd(self.pi_k, self.ts_k[:S], self.te_k[:S], self.sig_k[:S], self.rgb_k[:S], S, self.color,
                               self.opacity, self.depth, optical_depth=od, d_status=self.status, defer=defer)

    def render_bwd(self, n_kept: int, defer=False):
        S = min(int(n_kept), self.cap_k)
        od = self._od()[:S] if self.save_optical_depth else None
        return _lib.render_bwd(self.pi_k, self.ts_k[:S], self.te_k[:S], self.sig_k[:S], self.rgb_k[:S], S, self.g_color,
                               None, None, self.d_sig[:S], self.d_rgb[:S], optical_depth=od, d_status=self.status,
                               defer=defer)

    def render_mse(self, n_kept: int, target, defer=False):
        """Forward, the mean-squared-error gradient against ``target`` and the backward in one call."""
        S = min(int(n_kept), self.cap_k)
        return _lib.render_mse_fused(self.pi_k, self.ts_k[:S], self.te_k[:S], self.sig_k[:S], self.rgb_k[:S], S,
                                     target, 2.0 / (3.0 * self.R), self.color, self.d_sig[:S], self.d_rgb[:S],
                                     opacity=self.opacity, depth=self.depth, d_status=self.status, defer=defer)

    def sample_cells(self, seed: int, step: int, defer=False):
        """Random cells of the grid and a point in each for the update (``cells``, ``cell_xyz``)."""
        if self.n_grid:
            return _lib.sample_grid_cells(seed, 50000 + 4 * step, self.n_grid, self.grid, self.cells, self.cell_xyz,
                                          defer=defer)
        return (lambda: None) if defer else None

    def sat_rebuild_call(self):
        """The marshalled rebuild of the marched grid's summed-area table (what every
        grid update adds when the path marches with the table)."""
        return _lib.build_grid_sat(self.grid, self.sat, defer=True)

    def grid_update(self, decay=0.95, thre=0.01, bits=None, defer=False):
        """EMA update of ``self.ema``; writes ``bits`` (default: the bitfield marched by this
        path) and, when the path marches with a summed-area table, rebuilds the table of
        the bits written (into the marched table when ``bits`` is the marched bitfield)."""
        out = self.bits if bits is None else bits
        upd = _lib.update_occupancy_grid(self.ema, out, self.cells[: self.n_grid], self.cell_sig[: self.n_grid], decay,
                                         thre, self.status, defer=True)
        sat_call = lambda: None
        if self.use_sat:
            w = self.w
            g = _lib.make_grid(out, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)
            if out is self.bits:
                target = self.sat
            else:
                if self.upd_sat is None:
                    self.upd_sat = torch.empty_like(self.sat)
                target = self.upd_sat
            sat_call = _lib.build_grid_sat(g, target, defer=True)
            sat_call._grid = g  # the call holds a pointer into g

        def run():
            upd()
            sat_call()
        if defer:
            return run
        run()
        return None

    # -- user side (stand-in field, loss) ----------------------------------
    def field_marched(self, field: StandInField, rays_o, rays_d, n_marched, ray_time=None):
        M = min(int(n_marched), self.cap_m)
        field.samples(rays_o, rays_d, self.ri_m, self.ts_m, self.te_m, M, self.sig_m, None, ray_time=ray_time)

    def field_kept(self, field: StandInField, rays_o, rays_d, n_kept, ray_time=None):
        S = min(int(n_kept), self.cap_k)
        field.samples(rays_o, rays_d, self.ri_k, self.ts_k, self.te_k, S, self.sig_k, self.rgb_k, ray_time=ray_time)

    def loss_grad(self, target):
        # L = mean over rays and channels of (C - C*)^2  ->  dL/dC = 2 (C - C*) / (3R)
        torch.sub(self.color, target, out=self.g_color)
        self.g_color.mul_(2.0 / (3.0 * self.R))

    def check_status(self, what=""):
        s = int(self.status.item())
        if s:
            raise _lib.NaccError("%s: device status 0x%x" % (what, s))
