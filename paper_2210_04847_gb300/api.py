"""User-facing API in the shape of the paper's listing (Sec. 3):

    packed_info, t_starts, t_ends = ray_marching(rays_o, rays_d, grid=grid, sigma_fn=sigma_fn,
                                                 near_plane=0.2, far_plane=1.0,
                                                 early_stop_eps=1e-4, alpha_thre=1e-2)
    color, opacity, depth = rendering(rgb_sigma_fn, packed_info, t_starts, t_ends)

``sigma_fn(t_starts, t_ends, ray_indices) -> sigmas`` and
``rgb_sigma_fn(t_starts, t_ends, ray_indices) -> (rgbs, sigmas)`` are the
user's radiance field, queried at packed samples ((n, 1) interval tensors).
Marching, pruning and rendering (forward and backward) run in the CUDA
library; PyTorch only supplies device memory, streams and autograd plumbing.

The plain (eager) path has one host synchronisation per stage that produces a
data-dependent number of samples: reading the sample count to size the
outputs. Capacity-based calls without that synchronisation are available in
``paper_2210_04847_gb300._lib`` (and used by ``Pipeline``).
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import numpy as np
import torch

from . import _lib


class OccupancyGrid:
    """Binary occupancy grid with its float32 EMA density (Sec. 2.1).

    ``bits`` is an int32 tensor holding the uint32 words of the bitfield
    (layout of ``nacc_grid``); ``ema`` the per-cell float32 state the update
    maintains.
    """

    def __init__(self, aabb: Sequence[float], res=128, n_levels: int = 1, n_slots: int = 1, device="cuda",
                 contraction: int = 0):
        self.aabb = tuple(float(v) for v in aabb)
        self.res = (int(res),) * 3 if np.isscalar(res) else tuple(int(v) for v in res)
        self.n_levels = int(n_levels)
        self.n_slots = int(n_slots)
        self.contraction = int(contraction)  # 1: unbounded scene, contracted space (Sec. 2.1)
        self.n_cells = self.res[0] * self.res[1] * self.res[2] * self.n_levels * self.n_slots
        self.ema = torch.zeros(self.n_cells, dtype=torch.float32, device=device)
        self.bits = torch.zeros((self.n_cells + 31) // 32, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        # uncontracted grids of up to four levels keep the summed-area table of their
        # bits, so marching takes the box walk; rebuilt after every update and
        # whenever the bits tensor is modified by torch (its version counter moves)
        self.use_sat = self.n_levels <= 4 and not self.contraction
        self.sat = None
        self._sat_version = None

    @classmethod
    def from_bits(cls, bits: np.ndarray, res, aabb, n_levels=1, n_slots=1, device="cuda", contraction=0):
        g = cls(aabb, res, n_levels, n_slots, device, contraction)
        w = np.ascontiguousarray(bits, dtype=np.uint32).view(np.int32)
        assert w.size == g.bits.numel(), "bit words do not match the grid size"
        g.bits.copy_(torch.from_numpy(w))
        return g

    def _plain(self) -> _lib.Grid:
        s = getattr(self, "_struct", None)
        if s is None or s._keepalive is not self.bits:  # built once per bits tensor
            s = _lib.make_grid(self.bits, self.res, self.aabb, self.n_levels, self.n_slots, self.contraction)
            self._struct = s
        return s

    def _rebuild_sat(self):
        g = self._plain()
        if self.sat is None or self.sat.numel() * 2 != _lib.grid_sat_bytes(g):
            self.sat = torch.empty(_lib.grid_sat_bytes(g) // 2, dtype=torch.int16, device=self.bits.device)
            self._sat_struct = None
        _lib.build_grid_sat(g, self.sat)
        self._sat_version = (id(self.bits), self.bits._version)

    def struct(self) -> _lib.Grid:
        """The nacc_grid of this grid (with its summed-area table when it keeps one)."""
        if not self.use_sat:
            return self._plain()
        if self._sat_version != (id(self.bits), self.bits._version):
            self._rebuild_sat()
        s = getattr(self, "_sat_struct", None)
        if s is None or s._keepalive is not self.bits or s._keepalive_sat is not self.sat:
            s = _lib.make_grid(self.bits, self.res, self.aabb, self.n_levels, self.n_slots, self.contraction,
                               sat=self.sat)
            self._sat_struct = s
        return s

    def sample_cells(self, n: int, seed: int = 0, step: int = 0):
        """n uniform random cells of the grid (all levels and slots) and a uniform
        point inside each, for the update: returns (cells (n,) int32, xyz (n,3)
        float32). Deterministic in (seed, step): streams 50000 + 4*step (cells)
        and 50001 + 4*step (points) of the counter-based generator."""
        dev = self.bits.device
        cells = torch.empty(n, dtype=torch.int32, device=dev)
        xyz = torch.empty((n, 3), dtype=torch.float32, device=dev)
        _lib.sample_grid_cells(seed, 50000 + 4 * step, n, self.struct(), cells, xyz)
        return cells, xyz

    def update(self, cells: torch.Tensor, sigmas: torch.Tensor, decay: float = 0.95, thre: float = 0.01,
               alpha_step: Optional[float] = None):
        """EMA update: ema = max(decay * ema, sigma at sampled cells); bits = ema > thre.
        With ``alpha_step`` = dt the criterion is the opacity of a step of that
        length, 1 - exp(-ema dt) > thre (the paper's "empty where alpha < 1e-2",
        Sec. 2.1), applied by the library as the equivalent density threshold."""
        _lib.update_occupancy_grid(self.ema, self.bits, cells, sigmas, decay, thre, self.status,
                                   alpha_step=0.0 if alpha_step is None else float(alpha_step))
        if self.use_sat:
            self._rebuild_sat()

    def state_dict(self):
        return {"ema": self.ema.clone(), "bits": self.bits.clone(), "res": self.res, "aabb": self.aabb,
                "n_levels": self.n_levels, "n_slots": self.n_slots, "contraction": self.contraction}

    def load_state_dict(self, sd):
        self.ema.copy_(sd["ema"])
        self.bits.copy_(sd["bits"])


class _Scratch:
    """Per-device cache of workspaces and counters, grown on demand."""

    def __init__(self):
        self.bufs = {}

    def get(self, name, nbytes, device):
        key = (name, str(device))
        b = self.bufs.get(key)
        if b is None or b.numel() < nbytes:
            b = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
            self.bufs[key] = b
        return b


_SCRATCH = _Scratch()
_CAP_HINT = {}
_PARAMS = {}


def _params(near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps) -> _lib.MarchParams:
    key = (near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps)
    p = _PARAMS.get(key)
    if p is None:
        p = _PARAMS[key] = _lib.make_params(near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps)
    return p


def _count_and_status(dev):
    """One int64 pair on the device: [count, status]; the status word is the low
    half of the second element (read back together, one synchronisation). One
    buffer per device, zeroed on the stream before each use (every caller reads it
    back before returning)."""
    cs = _SCRATCH.bufs.get(("count_status", str(dev)))
    if cs is None:
        cs = _SCRATCH.bufs[("count_status", str(dev))] = torch.zeros(2, dtype=torch.int64, device=dev)
    else:
        cs.zero_()
    return cs, cs[0:1], cs[1:2].view(torch.int32)[:1]


def _read_count(cs: torch.Tensor, what: str) -> int:
    n, s = cs.tolist()
    if s & (_lib.STATUS_TIMEOUT | _lib.STATUS_BAD_PACKED | _lib.STATUS_OVERFLOW | _lib.STATUS_BAD_INDEX):
        raise _lib.NaccError("%s: device status 0x%x" % (what, s))
    return int(n)


_NO_GRID = {}


def _no_grid(device) -> OccupancyGrid:
    """Marching without an occupancy grid (the paper's listing calls ray_marching
    without one): every lattice step between near_plane and far_plane is a sample.
    Realised as a one-cell grid over contracted space with its bit set: contracted
    rays are not clipped to a box, and every contracted point (|x_c| < 2) falls in
    the one cell of [-2, 2]^3. The box is +-1e6, so points within that radius are
    not contracted at all and points far beyond it stay below |x_c| = 2 in float32."""
    key = str(device)
    g = _NO_GRID.get(key)
    if g is None:
        g = OccupancyGrid((-1e6, -1e6, -1e6, 1e6, 1e6, 1e6), 1, device=device, contraction=1)
        g.bits.fill_(1)
        _NO_GRID[key] = g
    return g


def march_rays(rays_o, rays_d, grid: Optional[OccupancyGrid] = None, near_plane=0.0, far_plane=1e10,
               render_step_size=1e-2, cone_angle=0.0, dt_max=None, max_steps=1024, ray_time=None, ray_slot=None):
    """Occupancy-grid marching only (grid None: every step between the planes).
    Returns (packed_info (R,2), t_starts (M,), t_ends (M,), ray_indices (M,))."""
    dev = rays_o.device
    if grid is None:
        grid = _no_grid(dev)
    rays_o = rays_o.contiguous().float()
    rays_d = rays_d.contiguous().float()
    R = rays_o.shape[0]
    params = _params(near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps)
    ws = _SCRATCH.get("march_ws", _lib.march_workspace_size(R, params), dev)
    packed = torch.empty((R, 2), dtype=torch.int32, device=dev)
    cs, counter, status = _count_and_status(dev)
    # output capacity: the last call's count on this batch size plus headroom, so
    # batches of similar size march once (a larger one marches again, exactly sized)
    cap = max(_CAP_HINT.get(("march", R), 64 * R), 1)
    for attempt in range(2):
        ts = torch.empty(cap, dtype=torch.float32, device=dev)
        te = torch.empty(cap, dtype=torch.float32, device=dev)
        ri = torch.empty(cap, dtype=torch.int32, device=dev)
        if attempt:
            cs.zero_()
        _lib.march_rays(rays_o, rays_d, grid.struct(), params, packed, ts, te, ri, counter, status, ws,
                        ray_time=ray_time, ray_slot=ray_slot)
        n = _read_count(cs, "march_rays")  # the one host synchronisation of the eager path
        if n <= cap:
            break
        cap = n
    _CAP_HINT[("march", R)] = max(int(n * 1.08) + 1024, 1)
    return packed, ts[:n], te[:n], ri[:n]


class DensityGrid:
    """A density field the library evaluates inside its kernels (the fused
    inference path): float32 sigma at the vertices of a lattice over ``aabb``
    (``sigma[i, j, k]`` at lo + (hi - lo) (i, j, k) / (res - 1)), trilinear in
    between, zero outside (``nacc_density_field``)."""

    def __init__(self, sigma: torch.Tensor, aabb: Sequence[float]):
        if sigma.dim() != 3 or min(sigma.shape) < 2:
            raise ValueError("sigma must be (G0, G1, G2) vertex values with every G >= 2")
        self.sigma = sigma.contiguous().float()
        self.aabb = tuple(float(v) for v in aabb)

    def struct(self) -> _lib.DensityField:
        s = getattr(self, "_struct", None)
        if s is None or s._keepalive is not self.sigma:
            s = self._struct = _lib.make_density_field(self.sigma, self.aabb)
        return s

    def __call__(self, xyz: torch.Tensor) -> torch.Tensor:
        """sigma at points xyz (n, 3)."""
        x = xyz.contiguous().float().view(-1, 3)
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _lib.density_field_query(self.struct(), x, x.shape[0], out)
        return out

    def at_samples(self, rays_o, rays_d, t_starts, t_ends, ray_indices) -> torch.Tensor:
        """sigma at each sample's midpoint (the point the marcher looks up)."""
        n = t_starts.numel()
        out = torch.empty(n, dtype=torch.float32, device=t_starts.device)
        _lib.density_field_at_samples(self.struct(), rays_o.contiguous().float(), rays_d.contiguous().float(),
                                      ray_indices.contiguous(), t_starts.contiguous().view(-1),
                                      t_ends.contiguous().view(-1), n, out)
        return out


def march_with_density(rays_o, rays_d, grid: OccupancyGrid, density: DensityGrid, near_plane=0.0, far_plane=1e10,
                       render_step_size=1e-2, cone_angle=0.0, dt_max=None, max_steps=1024, early_stop_eps=1e-4,
                       alpha_thre=0.0, return_ray_indices=False):
    """Inference: march the occupancy grid with the density field's transmittance
    evaluated in the same kernel, so each ray stops where T < early_stop_eps and
    only the kept samples are written (Sec. 2.1). Same samples as ``ray_marching``
    with ``sigma_fn = density.at_samples``. Returns (packed_info, t_starts (n,1),
    t_ends (n,1), sigmas (n,1)[, ray_indices])."""
    dev = rays_o.device
    rays_o = rays_o.contiguous().float()
    rays_d = rays_d.contiguous().float()
    R = rays_o.shape[0]
    params = _params(near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps)
    ws = _SCRATCH.get("march_ws", _lib.march_workspace_size(R, params), dev)
    packed = torch.empty((R, 2), dtype=torch.int32, device=dev)
    cs, counter, status = _count_and_status(dev)
    cap = max(_CAP_HINT.get(("fused", R), 16 * R), 1)
    for attempt in range(2):
        ts = torch.empty(cap, dtype=torch.float32, device=dev)
        te = torch.empty(cap, dtype=torch.float32, device=dev)
        ri = torch.empty(cap, dtype=torch.int32, device=dev)
        sg = torch.empty(cap, dtype=torch.float32, device=dev)
        if attempt:
            cs.zero_()
        _lib.march_fused(rays_o, rays_d, grid.struct(), params, density.struct(), early_stop_eps, alpha_thre,
                         packed, ts, te, ri, sg, counter, status, ws)
        n = _read_count(cs, "march_with_density")
        if n <= cap:
            break
        cap = n
    _CAP_HINT[("fused", R)] = max(int(n * 1.08) + 1024, 1)
    out = (packed, ts[:n].view(-1, 1), te[:n].view(-1, 1), sg[:n].view(-1, 1))
    return out + (ri[:n],) if return_ray_indices else out


def prune_samples(packed_info, t_starts, t_ends, sigmas, early_stop_eps=1e-4, alpha_thre=0.0):
    """Early-stop / alpha pruning and re-packing. Returns (packed_info, t_starts, t_ends, ray_indices)."""
    dev = packed_info.device
    R = packed_info.shape[0]
    M = t_starts.numel()
    ws = _SCRATCH.get("prune_ws", _lib.prune_workspace_size(R, M), dev)
    packed = torch.empty((R, 2), dtype=torch.int32, device=dev)
    cs, counter, status = _count_and_status(dev)
    ts = torch.empty(M, dtype=torch.float32, device=dev)
    te = torch.empty(M, dtype=torch.float32, device=dev)
    ri = torch.empty(M, dtype=torch.int32, device=dev)
    _lib.prune_samples(packed_info.contiguous(), t_starts.contiguous().view(-1), t_ends.contiguous().view(-1),
                       sigmas.contiguous().view(-1).float(), M, early_stop_eps, alpha_thre, packed, ts, te, ri,
                       counter, status, ws)
    n = _read_count(cs, "prune_samples")
    return packed, ts[:n], te[:n], ri[:n]


def _dev_key(device) -> str:
    d = torch.device(device)
    if d.type == "cuda" and d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return str(d)


def step_status(device) -> torch.Tensor:
    """The device status word (int32, NACC_STATUS_* bits) that calls in capacity mode
    accumulate on ``device``; read it with the step's results and pass it to
    ``check_status``, or call ``check_status(device)`` (one host read)."""
    key = ("step_status", _dev_key(device))
    st = _SCRATCH.bufs.get(key)
    if st is None:
        st = _SCRATCH.bufs[key] = torch.zeros(1, dtype=torch.int32, device=device)
    return st


def check_status(device, value: Optional[int] = None):
    """Raise if the capacity-mode calls on ``device`` reported a problem (a capacity
    too small for the samples, a timed-out wait, bad indices); then clear the word.
    ``value``: the word already read back (no further host read)."""
    st = step_status(device)
    v = int(st.item()) if value is None else int(value)
    st.zero_()
    if v:
        raise _lib.NaccError("device status 0x%x%s" % (v, " (capacity too small)" if v & _lib.STATUS_CAPACITY else ""))


def _capacity_buffers(tag, device, R: int, capacity: int):
    """Sample buffers reused by every capacity-mode call of the same shape. The
    sample arrays start zeroed, so entries past a call's count always hold valid
    ray indices and finite intervals (a previous call's samples or zeros)."""
    key = ("cap", tag, _dev_key(device), R, capacity)
    b = _SCRATCH.bufs.get(key)
    if b is None:
        z = lambda dt: torch.zeros(max(capacity, 1), dtype=dt, device=device)
        b = _SCRATCH.bufs[key] = dict(packed=torch.zeros((R, 2), dtype=torch.int32, device=device),
                                      ts=z(torch.float32), te=z(torch.float32), ri=z(torch.int32),
                                      n=torch.zeros(1, dtype=torch.int64, device=device))
    return b


def _ray_marching_capacity(rays_o, rays_d, grid, sigma_fn, params, early_stop_eps, alpha_thre, ray_time, ray_slot,
                           capacity: int, kept_capacity: int):
    dev = rays_o.device
    R = rays_o.shape[0]
    st = step_status(dev)
    m = _capacity_buffers("march", dev, R, capacity)
    ws = _SCRATCH.get("march_ws", _lib.march_workspace_size(R, params), dev)
    _lib.march_rays(rays_o, rays_d, grid.struct(), params, m["packed"], m["ts"][:capacity], m["te"][:capacity],
                    m["ri"][:capacity], m["n"], st, ws, ray_time=ray_time, ray_slot=ray_slot)
    if sigma_fn is None or not (early_stop_eps > 0 or alpha_thre > 0):
        return m["packed"], m["ts"][:capacity].view(-1, 1), m["te"][:capacity].view(-1, 1), m["ri"][:capacity], m["n"]
    with torch.no_grad():
        sig = sigma_fn(m["ts"][:capacity].view(-1, 1), m["te"][:capacity].view(-1, 1), m["ri"][:capacity])
    kc = kept_capacity
    k = _capacity_buffers("prune", dev, R, kc)
    wsp = _SCRATCH.get("prune_ws", _lib.prune_workspace_size(R, capacity), dev)
    _lib.prune_samples(m["packed"], m["ts"][:capacity], m["te"][:capacity], sig.contiguous().view(-1).float(),
                       capacity, early_stop_eps, alpha_thre, k["packed"], k["ts"][:kc], k["te"][:kc], k["ri"][:kc],
                       k["n"], st, wsp)
    return k["packed"], k["ts"][:kc].view(-1, 1), k["te"][:kc].view(-1, 1), k["ri"][:kc], k["n"]


def ray_marching(rays_o, rays_d, grid: Optional[OccupancyGrid] = None, sigma_fn: Optional[Callable] = None,
                 near_plane=0.0, far_plane=1e10, render_step_size=1e-2, cone_angle=0.0, dt_max=None, max_steps=1024,
                 early_stop_eps=1e-4, alpha_thre=0.0, ray_time=None, ray_slot=None, return_ray_indices=False,
                 capacity: Optional[int] = None, kept_capacity: Optional[int] = None):
    """March rays through the occupancy grid (or, with grid None, every step between
    the planes), then (if sigma_fn is given) prune by transmittance < early_stop_eps
    and opacity < alpha_thre, with the density queried without gradients (Sec. 2.1).
    Returns (packed_info, t_starts (n,1), t_ends (n,1)).

    capacity: a step with no host read. The outputs are then capacity-sized views
    of buffers the next call with the same ray count and capacity reuses, and the
    call returns (packed_info, t_starts, t_ends, ray_indices, n_samples) with
    n_samples a device int64 tensor: samples past it are padding that no packed
    run covers (valid ray indices, finite intervals). sigma_fn is called on the
    capacity-sized marched samples; kept_capacity (default: capacity) sizes the
    samples pruning keeps, which is what rendering and its gradient then run
    over. A capacity that is too small is reported in ``step_status`` (check it
    with the step's results)."""
    if capacity is not None:
        dev = rays_o.device
        return _ray_marching_capacity(rays_o.contiguous().float(), rays_d.contiguous().float(),
                                      _no_grid(dev) if grid is None else grid, sigma_fn,
                                      _params(near_plane, far_plane, render_step_size, dt_max, cone_angle, max_steps),
                                      early_stop_eps, alpha_thre, ray_time, ray_slot, int(capacity),
                                      int(capacity if kept_capacity is None else kept_capacity))
    packed, ts, te, ri = march_rays(rays_o, rays_d, grid, near_plane, far_plane, render_step_size, cone_angle,
                                    dt_max, max_steps, ray_time, ray_slot)
    if sigma_fn is not None and (early_stop_eps > 0 or alpha_thre > 0) and ts.numel() > 0:
        with torch.no_grad():
            sig = sigma_fn(ts.view(-1, 1), te.view(-1, 1), ri)
        packed, ts, te, ri = prune_samples(packed, ts, te, sig, early_stop_eps, alpha_thre)
    out = (packed, ts.view(-1, 1), te.view(-1, 1))
    return out + (ri,) if return_ray_indices else out


def unpack_info(packed_info: torch.Tensor, n_samples: int) -> torch.Tensor:
    ri = torch.empty(n_samples, dtype=torch.int32, device=packed_info.device)
    _lib.unpack_info(packed_info.contiguous(), n_samples, ri)
    return ri


class _RenderFn(torch.autograd.Function):
    """Eq. 1 forward and its hand-written backward (reverse segmented scan).
    ``n_dev`` (capacity mode): the device count of valid samples; the gradients of
    the padding past it are set to zero."""

    @staticmethod
    def forward(ctx, sigmas, rgbs, packed_info, t_starts, t_ends, save_optical_depth: bool, n_dev=None):
        R = packed_info.shape[0]
        M = t_starts.numel()
        dev = packed_info.device
        sg = sigmas.detach().contiguous().view(-1).float()
        rgb = rgbs.detach().contiguous().view(-1, 3).float()
        color = torch.empty((R, 3), dtype=torch.float32, device=dev)
        opacity = torch.empty((R, 1), dtype=torch.float32, device=dev)
        depth = torch.empty((R, 1), dtype=torch.float32, device=dev)
        od = torch.empty(M, dtype=torch.float32, device=dev) if save_optical_depth else None
        _lib.render_fwd(packed_info, t_starts, t_ends, sg, rgb, M, color, opacity, depth, optical_depth=od)
        ctx.save_for_backward(sg, rgb, packed_info, t_starts, t_ends, *( [od] if od is not None else [] ))
        ctx.sig_shape = sigmas.shape
        ctx.rgb_shape = rgbs.shape
        ctx.n_dev = n_dev
        return color, opacity, depth

    @staticmethod
    def backward(ctx, g_color, g_opacity, g_depth):
        saved = ctx.saved_tensors
        sg, rgb, packed_info, t_starts, t_ends = saved[:5]
        od = saved[5] if len(saved) > 5 else None
        M = t_starts.numel()
        d_sig = torch.empty(M, dtype=torch.float32, device=sg.device)
        d_rgb = torch.empty((M, 3), dtype=torch.float32, device=sg.device)
        f = lambda g: None if g is None else g.contiguous().float()
        _lib.render_bwd(packed_info, t_starts, t_ends, sg, rgb, M, f(g_color), f(g_opacity), f(g_depth), d_sig, d_rgb,
                        optical_depth=od)
        if ctx.n_dev is not None:  # padding past the device count: no run covers it
            _lib.fill_tail(d_sig, ctx.n_dev)
            _lib.fill_tail(d_rgb, ctx.n_dev)
        return d_sig.view(ctx.sig_shape), d_rgb.view(ctx.rgb_shape), None, None, None, None, None


def render_packed(sigmas, rgbs, packed_info, t_starts, t_ends, save_optical_depth=False, n_samples=None):
    """Differentiable Eq. 1 over packed samples: (color (R,3), opacity (R,1), depth (R,1)).
    n_samples: the device count of capacity-sized inputs (their padding gets zero gradients)."""
    return _RenderFn.apply(sigmas, rgbs, packed_info.contiguous(), t_starts.contiguous().view(-1),
                           t_ends.contiguous().view(-1), save_optical_depth, n_samples)


class _RenderMseFn(torch.autograd.Function):
    """Eq. 1 forward, the mean squared error of the colours against a target and
    its gradient in one call (nacc_render_mse_fused); the backward scales the
    gradients the call formed by the loss's incoming gradient."""

    @staticmethod
    def forward(ctx, sigmas, rgbs, packed_info, t_starts, t_ends, target, n_dev=None):
        R = packed_info.shape[0]
        M = t_starts.numel()
        dev = packed_info.device
        sg = sigmas.detach().contiguous().view(-1).float()
        rgb = rgbs.detach().contiguous().view(-1, 3).float()
        tgt = target.detach().contiguous().view(-1, 3).float()
        color = torch.empty((R, 3), dtype=torch.float32, device=dev)
        opacity = torch.empty((R, 1), dtype=torch.float32, device=dev)
        depth = torch.empty((R, 1), dtype=torch.float32, device=dev)
        sq_err = torch.empty(R, dtype=torch.float32, device=dev)
        d_sig = torch.empty(M, dtype=torch.float32, device=dev)
        d_rgb = torch.empty((M, 3), dtype=torch.float32, device=dev)
        # L = mean over rays and channels of (C - C*)^2: dL/dC = 2 (C - C*) / (3 R)
        _lib.render_mse_fused(packed_info, t_starts, t_ends, sg, rgb, M, tgt, 2.0 / (3.0 * max(R, 1)), color, d_sig,
                              d_rgb, opacity=opacity, depth=depth, sq_err=sq_err)
        if n_dev is not None:  # padding past the device count: no run covers it
            _lib.fill_tail(d_sig, n_dev)
            _lib.fill_tail(d_rgb, n_dev)
        ctx.save_for_backward(d_sig, d_rgb)
        ctx.sig_shape = sigmas.shape
        ctx.rgb_shape = rgbs.shape
        loss = sq_err.sum() / (3.0 * max(R, 1))
        ctx.mark_non_differentiable(color, opacity, depth)
        return loss, color, opacity, depth

    @staticmethod
    def backward(ctx, g_loss, g_color, g_opacity, g_depth):
        d_sig, d_rgb = ctx.saved_tensors
        g = g_loss.float()
        return (d_sig * g).view(ctx.sig_shape), (d_rgb * g).view(ctx.rgb_shape), None, None, None, None, None


def render_packed_mse(sigmas, rgbs, packed_info, t_starts, t_ends, target, n_samples=None):
    """Eq. 1 over packed samples with the mean-squared-error loss against ``target``
    (R,3) in one call: (loss, color (R,3), opacity (R,1), depth (R,1)). Only the loss
    is differentiable; its gradient w.r.t. sigmas and rgbs is formed in the same
    pass as the colours, reading the samples once (the loss of the Sec. 3 listing,
    fused with rendering). n_samples: as in ``render_packed``."""
    return _RenderMseFn.apply(sigmas, rgbs, packed_info.contiguous(), t_starts.contiguous().view(-1),
                              t_ends.contiguous().view(-1), target, n_samples)


def rendering_mse(rgb_sigma_fn: Callable, packed_info, t_starts, t_ends, target, ray_indices=None, n_samples=None):
    """``rendering`` with the mean-squared-error loss against ``target`` fused in:
    (loss, color, opacity, depth), the loss differentiable w.r.t. the field."""
    if ray_indices is None:
        if n_samples is not None:
            raise ValueError("capacity mode: pass the ray_indices ray_marching returned (padding needs valid indices)")
        ray_indices = unpack_info(packed_info, t_starts.numel())
    rgbs, sigmas = rgb_sigma_fn(t_starts.view(-1, 1), t_ends.view(-1, 1), ray_indices)
    return render_packed_mse(sigmas, rgbs, packed_info, t_starts, t_ends, target, n_samples)


def rendering(rgb_sigma_fn: Callable, packed_info, t_starts, t_ends, ray_indices=None, save_optical_depth=False,
              n_samples=None):
    """Query the user's field with gradients and render (Sec. 2.2). Returns (color, opacity, depth).
    n_samples: the device count that ``ray_marching(capacity=...)`` returned."""
    if ray_indices is None:
        if n_samples is not None:
            raise ValueError("capacity mode: pass the ray_indices ray_marching returned (padding needs valid indices)")
        ray_indices = unpack_info(packed_info, t_starts.numel())
    rgbs, sigmas = rgb_sigma_fn(t_starts.view(-1, 1), t_ends.view(-1, 1), ray_indices)
    return render_packed(sigmas, rgbs, packed_info, t_starts, t_ends, save_optical_depth, n_samples)


class _WeightsFn(torch.autograd.Function):
    """Eq. 1 weights; backward: any dL/dw to dL/dsigma (reverse segmented scan).

    ``g_ref`` (n_rays,) collects the per-ray part of dL/dw that centred
    accumulations of these weights hand over (see ``accumulate_along_rays``); the
    backward adds it back: dL/dw_i = g_ref[ray of i] + (incoming gradient)_i."""

    @staticmethod
    def forward(ctx, sigmas, packed_info, t_starts, t_ends, g_ref):
        M = t_starts.numel()
        dev = packed_info.device
        sg = sigmas.detach().contiguous().view(-1).float()
        w = torch.empty(M, dtype=torch.float32, device=dev)
        T = torch.empty(M, dtype=torch.float32, device=dev)
        _lib.render_weights(packed_info, t_starts, t_ends, sg, M, w, T)
        ctx.save_for_backward(sg, packed_info, t_starts, t_ends)
        ctx.g_ref = g_ref
        ctx.sig_shape = sigmas.shape
        ctx.mark_non_differentiable(T)
        return w, T

    @staticmethod
    def backward(ctx, g_w, g_T):
        sg, packed_info, t_starts, t_ends = ctx.saved_tensors
        M = t_starts.numel()
        d_sig = torch.empty(M, dtype=torch.float32, device=sg.device)
        g = torch.zeros(M, dtype=torch.float32, device=sg.device) if g_w is None else g_w.contiguous().float()
        g_ref = ctx.g_ref
        _lib.render_weights_bwd(packed_info, t_starts, t_ends, sg, M, g, d_sig, g_ref=g_ref)
        g_ref.zero_()  # handed over: a second backward through the graph starts from zero again
        return d_sig.view(ctx.sig_shape), None, None, None, None


def render_weights(packed_info, t_starts, t_ends, sigmas):
    """Per-sample Eq. 1 weights and transmittance, differentiable w.r.t. sigmas
    through the weights (Sec. 2.2). Returns (weights (M,), trans (M,)).

    When the returned ``weights`` tensor itself is passed to
    ``accumulate_along_rays`` (with the same ``packed_info``), the gradient
    between the two is carried in centred form: the accumulation's backward hands
    autograd dL/dw_i minus the value at the ray's first sample and keeps that
    per-ray value on the side, and this function's backward adds it back. Errors
    then scale with how much dL/dw varies along a ray, as in the fused
    ``render_packed``. The gradient is exact either way; only a hook or
    ``retain_grad`` on ``weights`` sees the centred values."""
    pi = packed_info.contiguous()
    g_ref = torch.zeros(pi.shape[0], dtype=torch.float32, device=pi.device)
    w, T = _WeightsFn.apply(sigmas, pi, t_starts.contiguous().view(-1), t_ends.contiguous().view(-1), g_ref)
    w._nacc_centre = (g_ref, pi, w._version)
    return w, T


class _AccumulateFn(torch.autograd.Function):
    """sum_i w_i v_i per ray; backward: dL/dw_i = <g_r, v_i>, dL/dv_i = w_i g_r.
    With ``g_ref`` (weights straight from ``render_weights``) dL/dw is handed back
    centred: <g_r, v_i - v_first>, and <g_r, v_first> is added to g_ref[r]."""

    @staticmethod
    def forward(ctx, weights, values, packed_info, g_ref):
        M = weights.numel()
        w = weights.detach().contiguous().view(-1).float()
        v = None if values is None else values.detach().contiguous().view(M, -1).float()
        C = 1 if v is None else v.shape[1]
        out = torch.empty((packed_info.shape[0], C), dtype=torch.float32, device=w.device)
        _lib.accumulate_along_rays(packed_info, w, v, C, M, out)
        ctx.save_for_backward(w, *([] if v is None else [v]), packed_info)
        ctx.g_ref = g_ref
        ctx.has_values = v is not None
        ctx.shapes = (weights.shape, None if values is None else values.shape)
        return out

    @staticmethod
    def backward(ctx, g_out):
        saved = ctx.saved_tensors
        w, packed_info = saved[0], saved[-1]
        v = saved[1] if ctx.has_values else None
        M = w.numel()
        C = 1 if v is None else v.shape[1]
        dw = torch.empty(M, dtype=torch.float32, device=w.device) if ctx.needs_input_grad[0] else None
        dv = (torch.empty((M, C), dtype=torch.float32, device=w.device)
              if v is not None and ctx.needs_input_grad[1] else None)
        g_ref = ctx.g_ref if dw is not None else None
        if dw is not None or dv is not None:
            _lib.accumulate_along_rays_bwd(packed_info, w, v, C, M, g_out.contiguous().float(), dw, dv, g_ref=g_ref)
        return (None if dw is None else dw.view(ctx.shapes[0]),
                None if dv is None else dv.view(ctx.shapes[1]), None, None)


def accumulate_along_rays(weights, packed_info, values=None):
    """sum_i w_i v_i per ray for any attribute (Sec. 2.2), differentiable w.r.t.
    weights and values. values (M, C) or None (opacity). Returns (R, C)."""
    pi = packed_info.contiguous()
    g_ref = None
    centre = getattr(weights, "_nacc_centre", None)
    if centre is not None:
        ref, ref_pi, version = centre
        # the centred hand-over only for the weights tensor render_weights returned,
        # unmodified, over the same rays
        if version == weights._version and (ref_pi is pi or (ref_pi.data_ptr() == pi.data_ptr()
                                                             and ref_pi.shape == pi.shape)):
            g_ref = ref
    return _AccumulateFn.apply(weights, values, pi, g_ref)
