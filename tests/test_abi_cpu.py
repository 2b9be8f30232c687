"""CPU-only checks of the C ABI: the library builds, loads and exports every
function include/mpm.h declares, and argument validation that needs no GPU
returns the documented status."""
import ctypes
import os
import subprocess

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2111_00699_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2111_00699_gb300 import _lib
    names = _lib.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a prototype for each one
    assert sorted(_lib._PROTOS) == names


def test_exports_are_c_symbols(lib):
    from paper_2111_00699_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in _lib.header_functions():
        assert n in syms, n                      # unmangled: extern "C"


def test_struct_layouts_match_header(lib):
    from paper_2111_00699_gb300 import _lib
    assert ctypes.sizeof(_lib.Material) == 4 * 12
    # res, dx, boundary, wall, gravity, padding, max_particles, five int32 knobs, transfer and the
    # three ASFLIP weights, the ASFLIP margin, reserved[1], padding to the 8-byte alignment of
    # max_particles
    assert ctypes.sizeof(_lib.Config) == 12 + 4 + 4 + 4 + 12 + 4 + 8 + 5 * 4 + 4 * 4 + 4 + 4 + 4
    assert ctypes.sizeof(_lib.Stats) == 6 * 8


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_2111_00699_gb300 import _lib
    ctx = ctypes.c_void_p()
    mat = _lib.material(_lib.ELASTIC)
    mats = (_lib.Material * 1)(mat)
    cfg = _lib.Config()
    cfg.res = (ctypes.c_int32 * 3)(64, 64, 64)
    cfg.dx = 1 / 64
    cfg.wall = 3
    assert lib.mpm_create(None, mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    assert lib.mpm_create(ctypes.byref(cfg), mats, 0, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    assert lib.mpm_create(ctypes.byref(cfg), mats, 9, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.res = (ctypes.c_int32 * 3)(64, 4, 64)
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.res = (ctypes.c_int32 * 3)(2048, 64, 64)
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.dx = 0.0
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.use_g2p2g = 2
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.resort_interval = -1
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.no_sort = 2
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    for transfer, alpha, bmin, bmax, fused in ((2, 0.0, 0.0, 0.0, 0), (_lib.ASFLIP, 1.5, 0.0, 1.0, 0),
                                                (_lib.ASFLIP, 0.9, -0.1, 1.0, 0), (_lib.ASFLIP, 0.9, 0.0, float("nan"), 0),
                                                (_lib.ASFLIP, 0.9, 0.0, 1.0, 1)):
        bad = _lib.Config.from_buffer_copy(cfg)
        bad.transfer, bad.flip_alpha, bad.flip_beta_min, bad.flip_beta_max, bad.use_g2p2g = (transfer, alpha, bmin,
                                                                                             bmax, fused)
        assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    for margin in (-1e-4, 1.0, float("nan")):
        bad = _lib.Config.from_buffer_copy(cfg)
        bad.transfer, bad.flip_alpha, bad.flip_beta_max, bad.flip_compress_margin = _lib.ASFLIP, 0.9, 1.0, margin
        assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.g2p_variant = 8
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad = _lib.Config.from_buffer_copy(cfg)
    bad.p2g_variant = 16
    assert lib.mpm_create(ctypes.byref(bad), mats, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad_mat = (_lib.Material * 1)(_lib.material(7))
    assert lib.mpm_create(ctypes.byref(cfg), bad_mat, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad_mat = (_lib.Material * 1)(_lib.material(_lib.ELASTIC, nu=0.5))
    assert lib.mpm_create(ctypes.byref(cfg), bad_mat, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad_mat = (_lib.Material * 1)(_lib.material(_lib.NACC, E=5e4, nu=0.3, friction_M=0.0))
    assert lib.mpm_create(ctypes.byref(cfg), bad_mat, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    bad_mat = (_lib.Material * 1)(_lib.material(6))
    assert lib.mpm_create(ctypes.byref(cfg), bad_mat, 1, None, None, ctypes.byref(ctx)) == _lib.MPM_EINVAL
    assert not ctx.value


def test_null_context_calls_are_safe(lib):
    from paper_2111_00699_gb300 import _lib
    assert lib.mpm_substep(None, 1e-4) == _lib.MPM_EINVAL
    assert lib.mpm_sync(None) == _lib.MPM_EINVAL
    assert lib.mpm_num_particles(None) == 0
    assert lib.mpm_last_error(None) == b"null context"
    lib.mpm_destroy(None)


def test_sort_scratch_query_is_host_only(lib):
    from paper_2111_00699_gb300 import _lib
    nb = ctypes.c_size_t()
    assert lib.mpm_radix_sort_pairs(None, None, None, None, 100000, 24, None, ctypes.byref(nb), None) == 0
    # two ping-pong buffers of n entries plus the digit histogram (256 per 2048-key tile)
    assert nb.value >= 2 * 4 * 100000 + 256 * 49 * 4
    assert lib.mpm_radix_sort_pairs(None, None, None, None, 10, 0, None, ctypes.byref(nb), None) == _lib.MPM_EINVAL
    assert lib.mpm_radix_sort_pairs(None, None, None, None, -1, 8, None, ctypes.byref(nb), None) == _lib.MPM_EINVAL


def test_scenes_are_deterministic_and_shaped():
    from paper_2111_00699_gb300 import scenes
    a, _ = scenes.snow_blocks()
    b, boxes = scenes.snow_blocks()
    np.testing.assert_array_equal(a, b)
    assert abs(len(a) - 1_330_000) <= 13_300
    assert len(boxes) == 6
    # 8 particles per cell, inside the walls
    assert a.min() > 3 / 256 and a.max() < 1 - 3 / 256
    cells = sum(int(np.prod(n)) for _, n in boxes)
    assert cells * 8 == len(a)
    x1, _ = scenes.fountain_batch(2, 7, 1e-4, (1 / 128) ** 3 / 8)
    x2, _ = scenes.fountain_batch(2, 7, 1e-4, (1 / 128) ** 3 / 8)
    x3, _ = scenes.fountain_batch(2, 8, 1e-4, (1 / 128) ** 3 / 8)
    np.testing.assert_array_equal(x1, x2)
    assert not np.array_equal(x1, x3)
    r = np.hypot(x1[:, 0] - 0.5, x1[:, 2] - 0.5)
    assert r.max() <= 0.05 + 1e-6


def test_splitmix64_reference_values():
    """splitmix64 outputs for seed-state 0 (Steele, Lea, Flood 2014;
    the values every published implementation reproduces)."""
    from paper_2111_00699_gb300 import scenes
    # state increments by the golden gamma before mixing: outputs for states 0, 1, 2 * gamma
    out = scenes.splitmix64(np.array([0, 0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF],
                                     dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_wait_timeout_check_rejects_bad_limit_without_the_gpu(lib):
    from paper_2111_00699_gb300 import _lib
    assert lib.mpm_debug_wait_timeout(0) == _lib.MPM_EINVAL
    assert lib.mpm_debug_wait_timeout(1 << 20) == _lib.MPM_EINVAL


def test_advance_rejects_a_null_context_without_the_gpu(lib):
    from paper_2111_00699_gb300 import _lib
    n = ctypes.c_int64(7)
    assert lib.mpm_advance(None, 0.01, 0.5, 1e-3, 100, None, ctypes.byref(n)) == _lib.MPM_EINVAL


def test_header_is_plain_c_and_layouts_match_the_binding(tmp_path):
    """include/mpm.h compiles as C11, and the sizes and field offsets a C
    compiler gives its structs are the ones the ctypes binding uses."""
    from paper_2111_00699_gb300 import _lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "mpm.h"
int main(void) {
    printf("%zu %zu %zu %zu\n", sizeof(mpm_config), sizeof(mpm_material), sizeof(mpm_stats), sizeof(mpm_scene_desc));
    printf("%zu %zu %zu %zu %zu\n", offsetof(mpm_config, max_particles), offsetof(mpm_config, transfer),
           offsetof(mpm_config, flip_beta_max), offsetof(mpm_config, flip_compress_margin),
           offsetof(mpm_material, alpha0));
    return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes, offs = [int(v) for v in out[:4]], [int(v) for v in out[4:]]
    assert sizes == [ctypes.sizeof(_lib.Config), ctypes.sizeof(_lib.Material), ctypes.sizeof(_lib.Stats),
                     ctypes.sizeof(_lib.SceneDesc)]
    assert offs == [_lib.Config.max_particles.offset, _lib.Config.transfer.offset, _lib.Config.flip_beta_max.offset,
                    _lib.Config.flip_compress_margin.offset, _lib.Material.alpha0.offset]


def test_red_rate_probe_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_2111_00699_gb300 import _lib
    V = ctypes.c_void_p
    assert lib.mpm_debug_red_rate(None, 64, 64, 1, 0, None) == _lib.MPM_EINVAL
    assert lib.mpm_debug_red_rate(V(256), 33, 64, 1, 0, None) == _lib.MPM_EINVAL       # nodes not a multiple of 32
    assert lib.mpm_debug_red_rate(V(256), 64, 48, 1, 0, None) == _lib.MPM_EINVAL       # threads not whole warps
    assert lib.mpm_debug_red_rate(V(256), 64, 64, 0, 0, None) == _lib.MPM_EINVAL       # no reductions
    assert lib.mpm_debug_red_rate(V(256), 64, 64, 5000, 0, None) == _lib.MPM_EINVAL
    assert lib.mpm_debug_red_rate(V(256), 64, 64, 1, 4, None) == _lib.MPM_EINVAL       # unknown pattern
    assert lib.mpm_debug_red_rate(V(264), 64, 64, 1, 0, None) == _lib.MPM_EINVAL       # not 16-byte aligned
