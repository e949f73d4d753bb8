"""Host-side checks of the C ABI (no GPU needed): the libraries load, export every
function the headers declare, and reject invalid arguments before touching the
device."""
import ctypes
import os
import re

import pytest

from paper_2210_04847_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs():
    build.build()
    return _lib.load(), _lib.load_field()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nacc_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(libs):
    lib, field = libs
    names = _declared("nacc.h")
    assert "nacc_march_rays" in names and "nacc_update_occupancy_grid" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    for n in _declared("nacc_field.h"):
        assert hasattr(field, n), n
    assert set(names) <= set(_lib.EXPORTS)


def test_version_and_error_strings(libs):
    lib, _ = libs
    assert lib.nacc_version() == 300
    assert lib.nacc_error_string(-1) == b"invalid argument"
    assert lib.nacc_error_string(12345) == b"unknown error code"


def test_invalid_arguments_rejected_on_host(libs):
    lib, _ = libs
    g = _lib.Grid()
    g.res[0] = g.res[1] = g.res[2] = 4
    g.n_levels, g.n_slots = 1, 1
    for k in range(3):
        g.aabb[k], g.aabb[3 + k] = -1.0, 1.0
    p = _lib.make_params(0.0, 1e10, 0.01, None, 0.0, 64)
    args = lambda n_rays=4, grid=g, params=p, cap=0, ws=None, wsb=0: (
        None, None, None, None, n_rays, ctypes.byref(grid), ctypes.byref(params), None, None, None, None, cap,
        ctypes.c_void_p(256), None, ws, wsb, None)
    assert lib.nacc_march_rays(*args(n_rays=-1)) == _lib.ERR_INVALID_ARG
    assert lib.nacc_march_rays(*args()) == _lib.ERR_INVALID_ARG  # null rays
    bad = _lib.make_params(0.0, 1e10, 0.0, None, 0.0, 64)
    assert lib.nacc_march_rays(*args(n_rays=0, params=bad)) == _lib.ERR_INVALID_ARG  # dt <= 0
    bad = _lib.make_params(0.0, 1e10, 0.01, None, 0.0, 40000)
    assert lib.nacc_march_rays(*args(n_rays=0, params=bad)) == _lib.ERR_INVALID_ARG  # max_steps
    g2 = _lib.Grid.from_buffer_copy(g)
    g2.n_levels = 17
    assert lib.nacc_march_rays(*args(n_rays=0, grid=g2)) == _lib.ERR_INVALID_ARG
    g2 = _lib.Grid.from_buffer_copy(g)
    g2.aabb[0] = 2.0  # lo > hi
    assert lib.nacc_march_rays(*args(n_rays=0, grid=g2)) == _lib.ERR_INVALID_ARG
    # workspace missing / misaligned
    assert lib.nacc_march_rays(*args(n_rays=0)) == _lib.ERR_INVALID_ARG
    assert lib.nacc_march_rays(*args(n_rays=0, ws=ctypes.c_void_p(4096 + 8), wsb=1 << 20)) == _lib.ERR_INVALID_ARG
    assert lib.nacc_prune_samples(None, -1, None, None, None, 0, 0.0, 0.0, None, None, None, None, 0,
                                  ctypes.c_void_p(8), None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_prune_samples(None, 0, None, None, None, 1 << 31, 0.0, 0.0, None, None, None, None, 0,
                                  ctypes.c_void_p(8), None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_render_fwd(None, 3, None, None, None, None, 0, None, None, None, None, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.nacc_render_bwd(None, -2, None, None, None, None, None, 0, None, None, None, None, None, None,
                               None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_accumulate_along_rays(None, 1, None, None, 0, 0, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_update_occupancy_grid(None, None, -1, None, None, 0, 0.9, 0.1, 0.0, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.nacc_update_occupancy_grid(None, None, 10, None, None, 0, 0.9, 0.1, 0.0, None, None) == \
        _lib.ERR_INVALID_ARG


def test_workspace_sizes(libs):
    lib, _ = libs
    p = _lib.make_params(0.0, 1e10, 0.01)
    assert lib.nacc_march_workspace_size(1 << 18, ctypes.byref(p)) >= (1 << 18) // 32 * 8
    assert lib.nacc_march_workspace_size(1 << 18, ctypes.byref(p)) % 256 == 0
    assert lib.nacc_prune_workspace_size(1000, 1 << 20) >= ((1 << 20) // 32 + 1000) * 4


def test_fused_and_density_field_arguments_rejected_on_host(libs):
    lib, _ = libs
    g = _lib.Grid()
    g.res[0] = g.res[1] = g.res[2] = 4
    g.n_levels, g.n_slots = 1, 1
    for k in range(3):
        g.aabb[k], g.aabb[3 + k] = -1.0, 1.0
    p = _lib.make_params(0.0, 1e10, 0.01, None, 0.0, 64)
    f = _lib.DensityField()
    f.sigma = 4096
    f.res[0] = f.res[1] = f.res[2] = 3
    for k in range(3):
        f.aabb[k], f.aabb[3 + k] = -1.0, 1.0
    ws = ctypes.c_void_p(1 << 20)  # never touched: every call below is rejected first

    def fused(field=f, grid=g, eps=1e-4, thre=1e-2, n_rays=0, n_samples=ctypes.c_void_p(256), wsb=1 << 16):
        return lib.nacc_march_fused(None, None, n_rays, ctypes.byref(grid), ctypes.byref(p),
                                    ctypes.byref(field) if field is not None else None, eps, thre, None, None, None,
                                    None, None, 0, n_samples, None, ws, wsb, None)

    assert fused(field=None) == _lib.ERR_INVALID_ARG
    bad = _lib.DensityField.from_buffer_copy(f)
    bad.res[2] = 1
    assert fused(field=bad) == _lib.ERR_INVALID_ARG
    bad = _lib.DensityField.from_buffer_copy(f)
    bad.aabb[1], bad.aabb[4] = 1.0, -1.0
    assert fused(field=bad) == _lib.ERR_INVALID_ARG
    bad = _lib.DensityField.from_buffer_copy(f)
    bad.sigma = None
    assert fused(field=bad) == _lib.ERR_INVALID_ARG
    assert fused(eps=float("nan")) == _lib.ERR_INVALID_ARG
    assert fused(thre=float("nan")) == _lib.ERR_INVALID_ARG
    assert fused(n_samples=None) == _lib.ERR_INVALID_ARG
    assert fused(n_rays=4) == _lib.ERR_INVALID_ARG  # rays and packed_info missing
    assert fused(wsb=0) == _lib.ERR_INVALID_ARG
    g2 = _lib.Grid.from_buffer_copy(g)
    g2.contraction, g2.n_levels = 1, 2  # contraction needs one level
    assert fused(grid=g2) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_query(None, None, 1, None, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_query(ctypes.byref(f), None, -1, None, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_query(ctypes.byref(f), None, 5, None, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_at_samples(ctypes.byref(f), None, None, 0, None, None, None, -1, None, None,
                                             None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_at_samples(ctypes.byref(f), None, None, 4, None, None, None, 3, None, None,
                                             None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_density_field_query(ctypes.byref(f), None, 0, None, None) == _lib.OK  # nothing to do


def test_lookback_test_hooks_validate_and_default(libs):
    lib, _ = libs
    assert lib.nacc_test_hook_get(0) == 1 << 22 and lib.nacc_test_hook_get(1) == 0
    assert lib.nacc_test_hook_get(2) == 0
    assert lib.nacc_test_hook_set(0, -1) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_set(0, (1 << 22) + 1) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_set(1, 2) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_set(2, 2) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_set(3, 0) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_get(7) == _lib.ERR_INVALID_ARG
    assert lib.nacc_test_hook_set(0, 17) == _lib.OK and lib.nacc_test_hook_get(0) == 17
    assert lib.nacc_test_hook_set(0, 1 << 22) == _lib.OK and lib.nacc_test_hook_get(0) == 1 << 22


def test_batched_march_arguments_rejected_on_host(libs):
    lib, _ = libs
    p = _lib.make_params(0.0, 1e10, 0.01, None, 0.0, 64)

    def desc(res=(8, 8, 8), n_levels=1, contraction=0, n_rays=2, aabb=(-1, -1, -1, 1, 1, 1), bits=4096):
        d = _lib.SceneDesc()
        d.bits = bits
        for k in range(3):
            d.res[k] = res[k]
        for k in range(6):
            d.aabb[k] = aabb[k]
        d.n_levels, d.contraction, d.n_rays = n_levels, contraction, n_rays
        return d

    def call(ds, n_rays=4, wsb=1 << 20):
        arr = (_lib.SceneDesc * len(ds))(*ds)
        # every call below is rejected before a pointer is touched
        return lib.nacc_march_rays_batched(arr, len(ds), ctypes.c_void_p(256), ctypes.c_void_p(512), n_rays,
                                           ctypes.byref(p), ctypes.c_void_p(1024), None, None, None, 0,
                                           ctypes.c_void_p(2048), None, ctypes.c_void_p(1 << 20), wsb, None)

    assert call([desc(), desc(n_rays=3)]) == _lib.ERR_INVALID_ARG  # counts sum to 5, not 4
    assert call([desc(), desc(res=(0, 8, 8))]) == _lib.ERR_INVALID_ARG
    assert call([desc(), desc(n_levels=17)]) == _lib.ERR_INVALID_ARG
    assert call([desc(), desc(contraction=1)]) == _lib.ERR_INVALID_ARG  # mixed contraction
    assert call([desc(), desc(aabb=(1, -1, -1, -1, 1, 1))]) == _lib.ERR_INVALID_ARG
    assert call([desc(), desc(bits=None)]) == _lib.ERR_INVALID_ARG  # rays but no grid
    assert call([desc(), desc(n_rays=-1), desc(n_rays=3)]) == _lib.ERR_INVALID_ARG
    assert call([desc(), desc()], wsb=16) == _lib.ERR_INVALID_ARG  # workspace too small
    assert call([]) == _lib.ERR_INVALID_ARG  # no scenes
    assert lib.nacc_march_batched_workspace_size(64, 1 << 18, ctypes.byref(p)) > \
        lib.nacc_march_workspace_size(1 << 18, ctypes.byref(p)) + 64 * 400


def test_grid_sat_sizes_and_rejections(libs):
    lib, _ = libs
    g = _lib.Grid()
    g.res[0], g.res[1], g.res[2] = 128, 96, 7
    g.n_levels, g.n_slots = 2, 3
    for k in range(3):
        g.aabb[k], g.aabb[3 + k] = -1.0, 1.0
    # the table's corners (a multiple of 8 entries here), then 2-bit states of the
    # 16 x 12 x 1 bricks of 8^3 cells, 8 per entry, for each of the 6 grids
    assert lib.nacc_grid_sat_bytes(ctypes.byref(g)) == (2 * 3 * 129 * 97 * 8 + 6 * (16 * 12 * 1 // 8)) * 2
    assert lib.nacc_build_grid_sat(ctypes.byref(g), ctypes.c_void_p(4096), None) == _lib.ERR_INVALID_ARG  # no bits
    g.bits = 4096
    assert lib.nacc_build_grid_sat(ctypes.byref(g), None, None) == _lib.ERR_INVALID_ARG  # no table
    g.res[0] = 0
    assert lib.nacc_grid_sat_bytes(ctypes.byref(g)) == 0
    assert lib.nacc_build_grid_sat(ctypes.byref(g), ctypes.c_void_p(4096), None) == _lib.ERR_INVALID_ARG
    g.res[0], g.res[1], g.res[2] = 1300, 1300, 1300  # corners over 2^31
    g.n_levels, g.n_slots = 1, 1
    assert lib.nacc_build_grid_sat(ctypes.byref(g), ctypes.c_void_p(4096), None) == _lib.ERR_INVALID_ARG
    # marching rejects a table that is misaligned or whose grid has too many corners
    p = _lib.make_params(0.0, 1e10, 0.01, None, 0.0, 64)
    g.res[0], g.res[1], g.res[2] = 8, 8, 8
    g.sat = 4097
    assert lib.nacc_march_rays(None, None, None, None, 0, ctypes.byref(g), ctypes.byref(p), None, None, None, None, 0,
                               ctypes.c_void_p(256), None, ctypes.c_void_p(1 << 20), 1 << 20, None) == \
        _lib.ERR_INVALID_ARG
