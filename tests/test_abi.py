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
    assert lib.nacc_version() == 100
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
    assert lib.nacc_update_occupancy_grid(None, None, -1, None, None, 0, 0.9, 0.1, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.nacc_update_occupancy_grid(None, None, 10, None, None, 0, 0.9, 0.1, None, None) == \
        _lib.ERR_INVALID_ARG


def test_workspace_sizes(libs):
    lib, _ = libs
    p = _lib.make_params(0.0, 1e10, 0.01)
    assert lib.nacc_march_workspace_size(1 << 18, ctypes.byref(p)) >= (1 << 18) // 32 * 8
    assert lib.nacc_march_workspace_size(1 << 18, ctypes.byref(p)) % 256 == 0
    assert lib.nacc_prune_workspace_size(1000, 1 << 20) >= ((1 << 20) // 32 + 1000) * 4
