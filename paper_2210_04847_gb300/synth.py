"""Seeded synthetic workloads: procedural scenes, cameras, rays, occupancy bits.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle's tests. It holds none of the method's arithmetic (no marching, no
quadrature, no grid update): it only *draws inputs*.

* Randomness: a counter-based generator, SplitMix64 (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014), applied to
  ``key(seed, stream) + counter * golden_gamma``. Every array is a pure
  function of ``(seed, stream, index)``.
* Scenes: sums of isotropic Gaussian density blobs, ``sigma(x) = sum_b p_b
  exp(-|x - c_b|^2 / (2 s_b^2))``, with ``rgb(x) = sigmoid(W x + b)``; the
  stand-in for the user's radiance field (the paper's ``sigma_fn`` /
  ``rgb_sigma_fn``, Sec. 3). All of it in float64.
* Cameras: pinhole cameras on a sphere looking at the origin (bounded
  scenes) or inside a large ball (unbounded scenes), unit ray directions
  (the paper's listing, Sec. 3, passes normalised directions).
* Occupancy bits: the density at each cell centre thresholded, packed into
  uint32 words over the flat cell index
  ``((slot * n_levels + level) * rx + ix) * ry + iy) * rz + iz`` (bit
  ``i & 31`` of word ``i >> 5``).

Functions accept ``device=`` where a large array is built with torch; the
default builds on the CPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_KEY_STREAM = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (vectorised, wrapping uint64 arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def rand_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uint64 draws of stream ``stream`` of seed ``seed`` (counter-based)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        key = key + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _KEY_STREAM
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GAMMA)


def rand_uniform(seed: int, stream: int, n: int, lo=0.0, hi=1.0) -> np.ndarray:
    """float64 uniform draws in [lo, hi) from the top 53 bits."""
    u = (rand_u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def rand_normal(seed: int, stream: int, n: int) -> np.ndarray:
    """float64 standard normals (Box-Muller on two uniform streams)."""
    u1 = rand_uniform(seed, stream, n)
    u2 = rand_uniform(seed, stream + 0x5151, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def rand_int(seed: int, stream: int, n: int, hi: int) -> np.ndarray:
    """int64 draws uniform in [0, hi) (modulo reduction of 64-bit draws)."""
    return (rand_u64(seed, stream, n) % np.uint64(hi)).astype(np.int64)


# ----------------------------------------------------------------------------
# Procedural scenes
# ----------------------------------------------------------------------------


@dataclass
class BlobScene:
    """Sum of isotropic Gaussian density blobs with a sigmoid-linear colour.

    ``velocities`` (optional) moves each centre linearly in time:
    ``c_b(t) = c_b + v_b t``.
    """

    centers: np.ndarray  # (B, 3)
    scales: np.ndarray  # (B,)
    peaks: np.ndarray  # (B,)
    rgb_w: np.ndarray  # (3, 3)
    rgb_b: np.ndarray  # (3,)
    velocities: Optional[np.ndarray] = None  # (B, 3)

    @property
    def n_blobs(self) -> int:
        return int(self.centers.shape[0])

    def _centers_at(self, t):
        if self.velocities is None or t is None:
            return self.centers
        return self.centers + self.velocities * float(t)

    def density(self, x: np.ndarray, t: Optional[float] = None, chunk: int = 1 << 16) -> np.ndarray:
        """sigma(x) for points x (N, 3), float64."""
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        c = self._centers_at(t)
        inv2s2 = 1.0 / (2.0 * self.scales * self.scales)
        c2 = (c * c).sum(1)
        out = np.empty(x.shape[0], dtype=np.float64)
        for s in range(0, x.shape[0], chunk):
            xs = x[s : s + chunk]
            # |x - c|^2 = |x|^2 - 2 x.c + |c|^2 (one matrix product per chunk)
            d2 = np.maximum((xs * xs).sum(1)[:, None] - 2.0 * (xs @ c.T) + c2[None, :], 0.0)
            out[s : s + chunk] = np.exp(-d2 * inv2s2[None, :]) @ self.peaks
        return out

    def rgb(self, x: np.ndarray) -> np.ndarray:
        """rgb(x) = sigmoid(W x + b) for points x (N, 3), float64."""
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        with np.errstate(over="ignore"):  # far points saturate the sigmoid to 0 or 1
            return 1.0 / (1.0 + np.exp(-(x @ self.rgb_w.T + self.rgb_b[None, :])))

    def device_params(self) -> np.ndarray:
        """Blob table as float32 rows (cx, cy, cz, 1/(2 s^2), peak, vx, vy, vz)."""
        v = self.velocities if self.velocities is not None else np.zeros_like(self.centers)
        tab = np.concatenate(
            [self.centers, (1.0 / (2.0 * self.scales**2))[:, None], self.peaks[:, None], v], axis=1
        )
        return np.ascontiguousarray(tab, dtype=np.float32)


def make_blob_scene(
    seed: int,
    n_blobs: int,
    center_radius: float = 1.0,
    scale_range=(0.1, 0.3),
    peak_range=(10.0, 50.0),
    log_scale: bool = False,
    ball: bool = False,
    speed: float = 0.0,
    stream_base: int = 0,
    peak_scale_ref: Optional[float] = None,
) -> BlobScene:
    """Draw a blob scene.

    Centres uniform in the cube [-r, r]^3 (or the ball of radius r when
    ``ball``); scales uniform (or log-uniform) in ``scale_range``; peaks
    uniform in ``peak_range``; colour weights W ~ U[-2, 2]^{3x3},
    b ~ U[-1, 1]^3; velocities U[-speed, speed]^3 when ``speed > 0``. With
    ``peak_scale_ref`` the peak is multiplied by ref / s, so every blob has the same
    order of optical depth through its centre whatever its size.
    """
    s0 = stream_base
    if ball:
        g = rand_normal(seed, s0 + 1, 3 * n_blobs).reshape(n_blobs, 3)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        rad = center_radius * rand_uniform(seed, s0 + 2, n_blobs) ** (1.0 / 3.0)
        centers = g * rad[:, None]
    else:
        centers = rand_uniform(seed, s0 + 1, 3 * n_blobs, -center_radius, center_radius).reshape(n_blobs, 3)
    if log_scale:
        lo, hi = math.log(scale_range[0]), math.log(scale_range[1])
        scales = np.exp(rand_uniform(seed, s0 + 3, n_blobs, lo, hi))
    else:
        scales = rand_uniform(seed, s0 + 3, n_blobs, *scale_range)
    peaks = rand_uniform(seed, s0 + 4, n_blobs, *peak_range)
    if peak_scale_ref is not None:
        peaks = peaks * (peak_scale_ref / scales)
    w = rand_uniform(seed, s0 + 5, 9, -2.0, 2.0).reshape(3, 3)
    b = rand_uniform(seed, s0 + 6, 3, -1.0, 1.0)
    vel = None
    if speed > 0.0:
        vel = rand_uniform(seed, s0 + 7, 3 * n_blobs, -speed, speed).reshape(n_blobs, 3)
    return BlobScene(centers, scales, peaks, w, b, vel)


# ----------------------------------------------------------------------------
# Cameras and rays
# ----------------------------------------------------------------------------


def _look_at_frames(positions: np.ndarray, targets: np.ndarray):
    """Right/up/forward unit frames (world z up, fallback y) for each camera."""
    f = targets - positions
    f /= np.linalg.norm(f, axis=-1, keepdims=True)
    up = np.broadcast_to(np.array([0.0, 0.0, 1.0]), f.shape).copy()
    bad = np.abs((f * up).sum(-1)) > 0.999
    up[bad] = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r, axis=-1, keepdims=True)
    u = np.cross(r, f)
    return r, u, f


def sphere_cameras(seed: int, n_cams: int, radius: float, stream: int = 100) -> np.ndarray:
    """Camera centres uniform on the sphere of radius ``radius``."""
    g = rand_normal(seed, stream, 3 * n_cams).reshape(n_cams, 3)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g * radius


def pinhole_rays(
    cam_pos: np.ndarray,
    cam_target: np.ndarray,
    px: np.ndarray,
    py: np.ndarray,
    fx: float,
    fy: float,
    cx: float,
    cy: float,
):
    """Rays through pixel centres (px + 0.5, py + 0.5) of pinhole cameras.

    ``cam_pos``/``cam_target`` are (N, 3) per ray. Returns float64 origins
    and unit directions, (N, 3) each.
    """
    r, u, f = _look_at_frames(cam_pos, cam_target)
    xc = (px + 0.5 - cx) / fx
    yc = -(py + 0.5 - cy) / fy
    d = r * xc[:, None] + u * yc[:, None] + f
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return cam_pos.copy(), d


def random_unit_vectors(seed: int, stream: int, n: int) -> np.ndarray:
    g = rand_normal(seed, stream, 3 * n).reshape(n, 3)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


# ----------------------------------------------------------------------------
# Occupancy bits from a density field
# ----------------------------------------------------------------------------


def level_boxes(aabb: Sequence[float], n_levels: int):
    """float64 boxes of a cascade: level l is the level-0 box scaled 2^l about its centre."""
    lo = np.asarray(aabb[:3], dtype=np.float64)
    hi = np.asarray(aabb[3:], dtype=np.float64)
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    out = []
    for lvl in range(n_levels):
        if lvl == 0:
            out.append((lo.copy(), hi.copy()))
        else:
            out.append((c - h * 2.0**lvl, c + h * 2.0**lvl))
    return out


def pack_bits(occ: np.ndarray) -> np.ndarray:
    """Pack a flat boolean array into uint32 words (bit i & 31 of word i >> 5)."""
    occ = np.asarray(occ, dtype=bool).reshape(-1)
    n = occ.size
    n_words = (n + 31) // 32
    padded = np.zeros(n_words * 32, dtype=np.uint64)
    padded[:n] = occ
    w = padded.reshape(n_words, 32) << np.arange(32, dtype=np.uint64)[None, :]
    return w.sum(axis=1).astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32).astype(np.uint64)
    bits = (words[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)
    return bits.reshape(-1)[:n].astype(bool)


def density_at_cell_centres(scene: BlobScene, aabb, res, n_levels=1, t=None, device="cpu"):
    """float64 density at every cell centre of every level, flat cell order.

    Uses the separability of the isotropic Gaussian: per blob, the product
    of three 1-D factors, contracted over blobs with one matrix product.
    """
    import torch

    rx, ry, rz = (int(v) for v in res)
    c = scene._centers_at(t)
    inv2s2 = 1.0 / (2.0 * scene.scales**2)
    out = []
    for lo, hi in level_boxes(aabb, n_levels):
        axes = []
        for a, r in enumerate((rx, ry, rz)):
            xs = lo[a] + (np.arange(r, dtype=np.float64) + 0.5) * ((hi[a] - lo[a]) / r)
            axes.append(np.exp(-((xs[None, :] - c[:, a : a + 1]) ** 2) * inv2s2[:, None]))  # (B, r)
        gx = torch.as_tensor(axes[0] * scene.peaks[:, None], device=device)
        gy = torch.as_tensor(axes[1], device=device)
        gz = torch.as_tensor(axes[2], device=device)
        yz = (gy[:, :, None] * gz[:, None, :]).reshape(gy.shape[0], -1)  # (B, ry*rz)
        dens = gx.T @ yz  # (rx, ry*rz)
        out.append(dens.reshape(-1))
    return torch.cat(out)


def occupancy_bits(scene: BlobScene, aabb, res, n_levels=1, thre=0.01, t=None, device="cpu") -> np.ndarray:
    """uint32 words: bit = density(cell centre) > thre, flat cell order."""
    dens = density_at_cell_centres(scene, aabb, res, n_levels, t, device)
    return pack_bits((dens > thre).cpu().numpy())


def density_at_vertices(scene: BlobScene, aabb, res, device="cpu") -> np.ndarray:
    """The stand-in field's density at the vertices of a res[0] x res[1] x res[2]
    lattice over ``aabb`` (vertex (i, j, k) at lo + (hi - lo) (i, j, k) / (res - 1)),
    float64 evaluation stored as float32 (G0, G1, G2): a density grid of the kind
    a trained field is baked into for inference. Separable per blob, as above."""
    import torch

    c = scene.centers
    inv2s2 = 1.0 / (2.0 * scene.scales**2)
    axes = []
    for a in range(3):
        lo, hi, g = float(aabb[a]), float(aabb[3 + a]), int(res[a])
        xs = lo + np.arange(g, dtype=np.float64) * ((hi - lo) / (g - 1))
        axes.append(np.exp(-((xs[None, :] - c[:, a : a + 1]) ** 2) * inv2s2[:, None]))
    gx = torch.as_tensor(axes[0] * scene.peaks[:, None], device=device)
    gy = torch.as_tensor(axes[1], device=device)
    gz = torch.as_tensor(axes[2], device=device)
    yz = (gy[:, :, None] * gz[:, None, :]).reshape(gy.shape[0], -1)
    dens = (gx.T @ yz).reshape(int(res[0]), int(res[1]), int(res[2]))
    return np.ascontiguousarray(dens.cpu().numpy(), dtype=np.float32)


def uncontract(xc: np.ndarray) -> np.ndarray:
    """Inverse of the Mip-NeRF 360 contraction (Eq. 10 there) for points of the
    open radius-2 ball, float64: |x_c| <= 1 unchanged, else x_c / ((2 - |x_c|) |x_c|)."""
    xc = np.asarray(xc, dtype=np.float64)
    r = np.linalg.norm(xc, axis=-1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(r <= 1.0, 1.0, 1.0 / ((2.0 - r) * r))
    return xc * s


def contracted_cell_centres(aabb, res) -> tuple:
    """World points of the cell centres of a contracted grid over [-2, 2]^3 (the box
    normalises the unit ball: world = c + h * uncontract(x_c)) and the mask of
    cells whose centre lies inside the radius-2 ball (the others are unreachable)."""
    rx, ry, rz = (int(v) for v in res)
    axes = [-2.0 + (np.arange(r, dtype=np.float64) + 0.5) * (4.0 / r) for r in (rx, ry, rz)]
    xc = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    inside = np.linalg.norm(xc, axis=1) < 2.0
    lo = np.asarray(aabb[:3], np.float64)
    hi = np.asarray(aabb[3:], np.float64)
    world = 0.5 * (lo + hi) + 0.5 * (hi - lo) * uncontract(np.where(inside[:, None], xc, 0.0))
    return world, inside


def density_at_contracted_centres(scene: BlobScene, aabb, res, device="cpu"):
    """float64 density at the world point of every cell centre of a contracted grid
    (flat cell order); 0 for cells outside the radius-2 ball."""
    import torch

    world, inside = contracted_cell_centres(aabb, res)
    c = torch.as_tensor(scene.centers, device=device)
    inv2s2 = torch.as_tensor(1.0 / (2.0 * scene.scales**2), device=device)
    peaks = torch.as_tensor(scene.peaks, device=device)
    dens = torch.empty(world.shape[0], dtype=torch.float64, device=device)
    for s in range(0, world.shape[0], 1 << 16):
        x = torch.as_tensor(world[s : s + (1 << 16)], device=device)
        d2 = ((x[:, None, :] - c[None, :, :]) ** 2).sum(-1)
        dens[s : s + (1 << 16)] = torch.exp(-d2 * inv2s2[None, :]) @ peaks
    return dens * torch.as_tensor(inside, device=device)


def occupancy_bits_contracted(scene: BlobScene, aabb, res, thre=0.01, device="cpu") -> np.ndarray:
    """uint32 words of a contracted grid: bit = density(world point of the cell
    centre) > thre; cells outside the radius-2 ball are empty."""
    return pack_bits((density_at_contracted_centres(scene, aabb, res, device) > thre).cpu().numpy())


# ----------------------------------------------------------------------------
# Workload configurations (bounded/unbounded/batched/dynamic scenes)
# ----------------------------------------------------------------------------

SQRT3 = math.sqrt(3.0)


@dataclass
class Workload:
    """One batch of inputs for the marching + rendering path."""

    name: str
    rays_o: np.ndarray  # (R, 3) float32
    rays_d: np.ndarray  # (R, 3) float32
    bits: np.ndarray  # uint32 words
    res: tuple
    n_levels: int
    n_slots: int
    aabb: tuple
    near_plane: float
    far_plane: float
    dt_min: float
    dt_max: float
    cone: float
    max_steps: int
    early_stop_eps: float
    alpha_thre: float
    scenes: list = field(default_factory=list)
    ray_time: Optional[np.ndarray] = None  # (R,) float32
    ray_slot: Optional[np.ndarray] = None  # (R,) int32
    target_rgb: Optional[np.ndarray] = None  # (R, 3) float32
    backward: bool = True
    meta: dict = field(default_factory=dict)
    contraction: int = 0  # 1: contracted unbounded space (one level; see nacc_grid)
    field: Optional[np.ndarray] = None  # (G0, G1, G2) float32 density at lattice vertices (inference)
    field_box: Optional[tuple] = None  # box of the density lattice

    @property
    def n_rays(self) -> int:
        return int(self.rays_o.shape[0])


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tiny_config(seed: int = 0, device="cpu") -> Workload:
    """64x64 pinhole camera, 8 blobs, 64^3 grid (density > 0.01), dt = sqrt(3)*3/512, forward only."""
    scene = make_blob_scene(seed, 8)
    cam = sphere_cameras(seed, 1, 4.0)
    py, px = np.meshgrid(np.arange(64, dtype=np.float64), np.arange(64, dtype=np.float64), indexing="ij")
    px, py = px.reshape(-1), py.reshape(-1)
    pos = np.repeat(cam, px.size, axis=0)
    o, d = pinhole_rays(pos, np.zeros_like(pos), px, py, 80.0, 80.0, 32.0, 32.0)
    aabb = (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)
    bits = occupancy_bits(scene, aabb, (64, 64, 64), 1, 0.01, device=device)
    dt = SQRT3 * 3.0 / 512.0
    return Workload(
        "tiny-64x64-8blobs-grid64", _f32(o), _f32(d), bits, (64, 64, 64), 1, 1, aabb,
        0.0, 1e10, dt, dt, 0.0, 512, 0.0, 0.0, [scene], backward=False,
    )


def bounded_scene(seed: int = 0, device="cpu"):
    """Scene and grid of the bounded workload: 64 blobs, 128^3 bits over [-1.5, 1.5]^3 (density > 0.01)."""
    scene = make_blob_scene(seed, 64)
    aabb = (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)
    bits = occupancy_bits(scene, aabb, (128, 128, 128), 1, 0.01, device=device)
    return scene, aabb, bits


def bounded_rays(seed: int, n_rays: int, batch: int = 0, n_cams: int = 100):
    """Random (camera, pixel) rays of 100 cameras at 800x800 (fx = fy = 1111.1) on the r = 4
    sphere looking at the origin, and a seeded target colour per ray. ``batch`` selects an
    independent draw for the same cameras. Returns float32 (o, d, target)."""
    cams = sphere_cameras(seed, n_cams, 4.0)
    sb = 1000 + 16 * batch
    ci = rand_int(seed, sb + 1, n_rays, n_cams)
    pix = rand_int(seed, sb + 2, n_rays, 800 * 800)
    px, py = (pix % 800).astype(np.float64), (pix // 800).astype(np.float64)
    pos = cams[ci]
    o, d = pinhole_rays(pos, np.zeros_like(pos), px, py, 1111.1, 1111.1, 400.0, 400.0)
    target = rand_uniform(seed, sb + 3, 3 * n_rays).reshape(n_rays, 3)
    return _f32(o), _f32(d), _f32(target)


def bounded_config(seed: int = 0, n_rays: int = 1 << 18, n_cams: int = 100, device="cpu", batch: int = 0,
                   scene_grid=None) -> Workload:
    """Random rays of 100 cameras at 800x800 (fx = fy = 1111.1) on the r = 4 sphere,
    64 blobs, 128^3 grid over [-1.5, 1.5]^3, dt = sqrt(3)*3/1024 (<= 1024 steps),
    early stop 1e-4, alpha threshold 1e-2, seeded MSE target. ``batch`` selects
    an independent draw of rays for the same scene."""
    scene, aabb, bits = scene_grid if scene_grid is not None else bounded_scene(seed, device)
    o, d, target = bounded_rays(seed, n_rays, batch, n_cams)
    dt = SQRT3 * 3.0 / 1024.0
    name = ("bounded-2^%d-rays-64blobs-grid128" % int(round(math.log2(n_rays))) if n_rays & (n_rays - 1) == 0
            else "bounded-%d-rays-64blobs-grid128" % n_rays)
    return Workload(
        name, o, d, bits, (128, 128, 128), 1, 1, aabb,
        0.0, 1e10, dt, dt, 0.0, 1024, 1e-4, 1e-2, [scene], target_rgb=target,
    )


def inference_config(seed: int = 0, camera: int = 0, field_res: int = 129, device="cpu",
                     scene_grid=None) -> Workload:
    """One whole 800x800 image (fx = fy = 1111.1) of the bounded scene from camera
    ``camera`` of the bounded workload's 100 on the r = 4 sphere, pixel-major; the
    bounded workload's 128^3 occupancy grid and step; the scene's density baked
    at field_res^3 lattice vertices over the same box (the field the fused
    inference path evaluates). Early stop 1e-4, alpha threshold 1e-2."""
    scene, aabb, bits = scene_grid if scene_grid is not None else bounded_scene(seed, device)
    cam = sphere_cameras(seed, 100, 4.0)[camera % 100][None, :]
    py, px = np.meshgrid(np.arange(800, dtype=np.float64), np.arange(800, dtype=np.float64), indexing="ij")
    px, py = px.reshape(-1), py.reshape(-1)
    pos = np.repeat(cam, px.size, axis=0)
    o, d = pinhole_rays(pos, np.zeros_like(pos), px, py, 1111.1, 1111.1, 400.0, 400.0)
    dt = SQRT3 * 3.0 / 1024.0
    fr = (int(field_res),) * 3
    return Workload(
        "inference-800x800-grid128-field%d" % field_res, _f32(o), _f32(d), bits, (128, 128, 128),
        1, 1, aabb, 0.0, 1e10, dt, dt, 0.0, 1024, 1e-4, 1e-2, [scene], backward=False,
        field=density_at_vertices(scene, aabb, fr, device), field_box=tuple(aabb), meta={"camera": camera % 100},
    )


def unbounded_config(seed: int = 0, n_rays: int = 1 << 20, n_cams: int = 64, device="cpu", batch: int = 0) -> Workload:
    """2^20 rays from 64 cameras inside radius 100 of a radius-1000 scene of 256
    log-uniform-scale blobs (scale in [0.1, 100], peak U[10, 50] * 0.1/scale);
    4-level cascade of 128^3 (level-0 box [-125,125]^3); cone step
    dt = clamp(t/256, 1e-3, 10), t in [0.05, 1000]."""
    scene = make_blob_scene(seed, 256, center_radius=1000.0, scale_range=(0.1, 100.0), log_scale=True, ball=True,
                            peak_scale_ref=0.1)
    g = random_unit_vectors(seed, 200, n_cams)
    cams = g * (100.0 * rand_uniform(seed, 201, n_cams) ** (1.0 / 3.0))[:, None]
    sb = 2000 + 16 * batch
    ci = rand_int(seed, sb + 1, n_rays, n_cams)
    o = cams[ci]
    d = random_unit_vectors(seed, sb + 2, n_rays)
    aabb = (-125.0, -125.0, -125.0, 125.0, 125.0, 125.0)
    bits = occupancy_bits(scene, aabb, (128, 128, 128), 4, 0.01, device=device)
    target = rand_uniform(seed, sb + 3, 3 * n_rays).reshape(n_rays, 3)
    return Workload(
        "unbounded-cascade4x128-cone", _f32(o), _f32(d), bits, (128, 128, 128), 4, 1, aabb,
        0.05, 1000.0, 1e-3, 10.0, 1.0 / 256.0, 4096, 1e-4, 1e-2, [scene], target_rgb=_f32(target),
    )


def contracted_config(seed: int = 0, n_rays: int = 1 << 20, n_cams: int = 64, device="cpu", batch: int = 0,
                      res: int = 128) -> Workload:
    """The unbounded scene and rays of ``unbounded_config`` with the contracted grid
    instead of the cascade: one res^3 grid over the contraction of the space, the
    box [-125, 125]^3 normalising the unit ball, same cone steps and planes."""
    w = unbounded_config(seed, n_rays=n_rays, n_cams=n_cams, device=device, batch=batch)
    bits = occupancy_bits_contracted(w.scenes[0], w.aabb, (res, res, res), 0.01, device=device)
    w.name = "unbounded-contracted-grid%d-cone" % res
    w.bits, w.res, w.n_levels, w.contraction = bits, (res, res, res), 1, 1
    return w


def batched_config(seed: int = 0, n_scenes: int = 64, device="cpu", ray_scale: float = 1.0) -> Workload:
    """64 independent scenes (8..256 blobs), one 128^3 grid each, lognormal ray
    counts clamp(exp(N(ln 8000, 1)), 1024, 65536) per scene; rays ordered scene-major."""
    nb = 8 + rand_int(seed, 3000, n_scenes, 249)
    counts = np.exp(math.log(8000.0) + rand_normal(seed, 3001, n_scenes))
    counts = np.clip(np.round(counts * ray_scale), max(1, int(1024 * ray_scale)), int(65536 * ray_scale)).astype(np.int64)
    aabb = (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)
    os_, ds_, bits_, slots, targets, scenes = [], [], [], [], [], []
    for s in range(n_scenes):
        sc = make_blob_scene(seed + 7919 * (s + 1), int(nb[s]))
        scenes.append(sc)
        cams = sphere_cameras(seed + 7919 * (s + 1), 100, 4.0)
        n = int(counts[s])
        ci = rand_int(seed + 7919 * (s + 1), 3100, n, 100)
        pix = rand_int(seed + 7919 * (s + 1), 3101, n, 800 * 800)
        px, py = (pix % 800).astype(np.float64), (pix // 800).astype(np.float64)
        pos = cams[ci]
        o, d = pinhole_rays(pos, np.zeros_like(pos), px, py, 1111.1, 1111.1, 400.0, 400.0)
        os_.append(o)
        ds_.append(d)
        slots.append(np.full(n, s, dtype=np.int32))
        targets.append(rand_uniform(seed + 7919 * (s + 1), 3102, 3 * n).reshape(n, 3))
        dens = density_at_cell_centres(sc, aabb, (128, 128, 128), 1, None, device)
        bits_.append((dens > 0.01).cpu().numpy())
    bits = pack_bits(np.concatenate(bits_))
    dt = SQRT3 * 3.0 / 1024.0
    return Workload(
        "batched-%d-scenes-grid128" % n_scenes, _f32(np.concatenate(os_)), _f32(np.concatenate(ds_)), bits,
        (128, 128, 128), 1, n_scenes, aabb, 0.0, 1e10, dt, dt, 0.0, 1024, 1e-4, 1e-2, scenes,
        ray_slot=np.concatenate(slots), target_rgb=_f32(np.concatenate(targets)),
        meta={"rays_per_scene": counts.tolist()},
    )


def dynamic_config(seed: int = 0, n_rays: int = 1 << 19, n_bins: int = 16, device="cpu", batch: int = 0) -> Workload:
    """128 blobs moving linearly (v ~ U[-0.5, 0.5]^3) for t in [0, 1]; one 128^3
    grid per time bin (density at the bin-centre time > 0.01); 2^19 rays with
    times drawn unevenly over the bins (Dirichlet-like bin weights)."""
    scene = make_blob_scene(seed, 128, speed=0.5)
    cams = sphere_cameras(seed, 100, 4.0)
    sb = 4000 + 16 * batch
    wts = -np.log1p(-rand_uniform(seed, 4000, n_bins))  # Exp(1) -> Dirichlet(1,...,1)
    wts /= wts.sum()
    cdf = np.cumsum(wts)
    u = rand_uniform(seed, sb + 1, n_rays)
    b = np.minimum(np.searchsorted(cdf, u, side="right"), n_bins - 1)
    t = (b + rand_uniform(seed, sb + 2, n_rays)) / n_bins
    ci = rand_int(seed, sb + 3, n_rays, 100)
    pix = rand_int(seed, sb + 4, n_rays, 800 * 800)
    px, py = (pix % 800).astype(np.float64), (pix // 800).astype(np.float64)
    pos = cams[ci]
    o, d = pinhole_rays(pos, np.zeros_like(pos), px, py, 1111.1, 1111.1, 400.0, 400.0)
    aabb = (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)
    occ = []
    for k in range(n_bins):
        dens = density_at_cell_centres(scene, aabb, (128, 128, 128), 1, (k + 0.5) / n_bins, device)
        occ.append((dens > 0.01).cpu().numpy())
    bits = pack_bits(np.concatenate(occ))
    dt = SQRT3 * 3.0 / 1024.0
    target = rand_uniform(seed, sb + 5, 3 * n_rays).reshape(n_rays, 3)
    return Workload(
        "dynamic-%dbins-grid128" % n_bins, _f32(o), _f32(d), bits, (128, 128, 128), 1, n_bins, aabb,
        0.0, 1e10, dt, dt, 0.0, 1024, 1e-4, 1e-2, [scene], ray_time=_f32(t), target_rgb=_f32(target),
        meta={"bin_weights": wts.tolist()},
    )


def dynamic_shared_config(seed: int = 0, n_rays: int = 1 << 19, n_bins: int = 16, device="cpu",
                          batch: int = 0) -> Workload:
    """The dynamic scene and rays with one grid shared by all times (the paper's
    D-NeRF setting, Sec. 4: the grid holds the maximum over time): the bitwise OR
    of the per-bin grids of ``dynamic_config``."""
    w = dynamic_config(seed, n_rays=n_rays, n_bins=n_bins, device=device, batch=batch)
    w.bits = np.bitwise_or.reduce(w.bits.reshape(n_bins, -1), axis=0)
    w.n_slots = 1
    w.name = "dynamic-shared-grid128"
    return w


def grid_update_samples(seed: int, step: int, n: int, res, n_levels: int = 1, n_slots: int = 1):
    """Uniform random cells (with replacement) and float32 jitters in [0, 1)^3 for
    one grid update. Sample i takes draws 2i, 2i+1 of stream 50000 + 4*step for
    its cell: each 32-bit half h gives a coordinate (h * extent) >> 32 (x, y from
    the high and low halves of the first draw, z and the (slot, level) index from
    the second); and draws 2i, 2i+1 of stream 50001 + 4*step for its jitter: the
    24-bit fields at bits 40, 16 of the first and 40 of the second, times 2^-24.
    Flat cell = ((sl * rx + x) * ry + y) * rz + z, sl = slot * n_levels + level."""
    rx, ry, rz = (int(v) for v in res)
    m32 = np.uint64(0xFFFFFFFF)
    r = rand_u64(seed, 50000 + 4 * step, 2 * n).reshape(n, 2)
    with np.errstate(over="ignore"):
        ix = ((r[:, 0] >> np.uint64(32)) * np.uint64(rx)) >> np.uint64(32)
        iy = ((r[:, 0] & m32) * np.uint64(ry)) >> np.uint64(32)
        iz = ((r[:, 1] >> np.uint64(32)) * np.uint64(rz)) >> np.uint64(32)
        sl = ((r[:, 1] & m32) * np.uint64(n_levels * n_slots)) >> np.uint64(32)
    cells = (((sl.astype(np.int64) * rx + ix.astype(np.int64)) * ry + iy.astype(np.int64)) * rz
             + iz.astype(np.int64)).astype(np.int32)
    q = rand_u64(seed, 50001 + 4 * step, 2 * n).reshape(n, 2)
    m24 = np.uint64(0xFFFFFF)
    jit = np.stack([q[:, 0] >> np.uint64(40), (q[:, 0] >> np.uint64(16)) & m24, q[:, 1] >> np.uint64(40)], axis=1)
    return cells, jit.astype(np.float32) * np.float32(2.0 ** -24)


def level_boxes_f32(aabb: Sequence[float], n_levels: int):
    """float32 boxes of a cascade, formed as the marcher forms them: c = (lo + hi) / 2,
    h = (hi - lo) / 2, level l >= 1 = c -+ h * 2^l (each operation rounded to float32)."""
    lo = np.asarray(aabb[:3], dtype=np.float32)
    hi = np.asarray(aabb[3:], dtype=np.float32)
    c = (lo + hi) * np.float32(0.5)
    h = (hi - lo) * np.float32(0.5)
    out = []
    for lvl in range(n_levels):
        if lvl == 0:
            out.append((lo.copy(), hi.copy()))
        else:
            hl = h * np.float32(2.0**lvl)
            out.append((c - hl, c + hl))
    return out


def cell_positions(cells: np.ndarray, jitter: np.ndarray, aabb, res, n_levels=1, contraction=0) -> np.ndarray:
    """float32 points lo + (cell index + jitter) * cell size inside flat cells, every
    operation rounded to float32 (cell size = (hi - lo) / res of the cell's level;
    level = (cell / res^3) mod n_levels). With contraction the point is drawn in
    the contracted box [-2, 2]^3 and mapped back to the world (nacc_sample_grid_cells)."""
    if contraction:
        p = cell_positions(cells, jitter, (-2.0, -2.0, -2.0, 2.0, 2.0, 2.0), res, 1)
        r2 = (p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1]) + p[:, 2] * p[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.sqrt(r2)
            sc = np.where(r2 <= np.float32(1), np.float32(1),
                          np.where(r < np.float32(2), np.float32(1) / ((np.float32(2) - r) * r), np.float32(np.nan)))
        sc = sc.astype(np.float32)
        lo = np.asarray(aabb[:3], np.float32)
        hi = np.asarray(aabb[3:], np.float32)
        c = (lo + hi) * np.float32(0.5)
        h = (hi - lo) * np.float32(0.5)
        return (c + h * (p * sc[:, None])).astype(np.float32)
    rx, ry, rz = res
    per_level = rx * ry * rz
    cells = np.asarray(cells, dtype=np.int64)
    local = cells % per_level
    lvl = (cells // per_level) % n_levels
    ix, rem = local // (ry * rz), local % (ry * rz)
    iy, iz = rem // rz, rem % rz
    idx = np.stack([ix, iy, iz], axis=1).astype(np.float32)
    boxes = level_boxes_f32(aabb, n_levels)
    lo = np.stack([boxes[l][0] for l in range(n_levels)])[lvl]
    size = np.stack([(boxes[l][1] - boxes[l][0]) / np.asarray(res, dtype=np.float32) for l in range(n_levels)])[lvl]
    return lo + (idx + np.asarray(jitter, dtype=np.float32)) * size


def sample_field(scene: BlobScene, rays_o, rays_d, t_starts, t_ends, ray_indices, ray_time=None):
    """float32 (sigma, rgb) of the blob scene at sample midpoints o + d (t_s + t_e) / 2.

    The midpoint rule is the one in the paper's callbacks (Sec. 3 listing).
    Positions are formed in float64 from the float32 inputs.
    """
    ri = np.asarray(ray_indices, dtype=np.int64)
    o = np.asarray(rays_o, dtype=np.float64)[ri]
    d = np.asarray(rays_d, dtype=np.float64)[ri]
    mid = (np.asarray(t_starts, np.float64) + np.asarray(t_ends, np.float64)) * 0.5
    x = o + d * mid[:, None]
    if ray_time is not None and scene.velocities is not None:
        tt = np.asarray(ray_time, np.float64)[ri]
        sig = np.zeros(len(ri))
        inv2s2 = 1.0 / (2.0 * scene.scales**2)
        for s in range(0, len(ri), 1 << 15):
            c = scene.centers[None] + scene.velocities[None] * tt[s : s + (1 << 15), None, None]
            d2 = ((x[s : s + (1 << 15), None, :] - c) ** 2).sum(-1)
            sig[s : s + (1 << 15)] = (scene.peaks[None] * np.exp(-d2 * inv2s2[None])).sum(-1)
    else:
        sig = scene.density(x)
    rgb = scene.rgb(x)
    return np.ascontiguousarray(sig, np.float32), np.ascontiguousarray(rgb, np.float32)
