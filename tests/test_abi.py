"""The C-ABI library builds for sm_103a, loads, exports every entry point
that include/maskgs.h declares, and rejects bad arguments on the host
(no GPU needed: no call here reaches a kernel)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "maskgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_20522_gb300 import abi
    return abi.load()


def test_header_declares_the_pipeline():
    names = _declared()
    for n in ("mg_preprocess", "mg_bin", "mg_sort", "mg_render", "mg_render_backward",
              "mg_preprocess_backward", "mg_l1_loss_grad"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2412_20522_gb300 import abi
    assert sorted(abi.EXPORTED) == _declared()
    for n in _declared():
        if n not in ("mg_status_string", "mg_version", "mg_bin_workspace_bytes",
                     "mg_sort_workspace_bytes", "mg_tile_bits", "mg_total_tiles",
                     "mg_depth_order_workspace_bytes"):
            assert callable(getattr(abi, n))


def test_host_only_helpers(lib):
    from paper_2412_20522_gb300 import abi, scenes
    from paper_2412_20522_gb300.rasterize import RasterConfig, make_views
    assert abi.version().startswith("maskgs")
    assert abi.status_string(abi.MG_ERR_CAPACITY) == "instance capacity exceeded"
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 1557, 1038, 1150.0)
    views = make_views([cam, cam], [(0, 10), (0, 10)])
    cfg = RasterConfig().c()
    assert abi.mg_total_tiles(views, 2, cfg) == 2 * 98 * 65
    assert abi.mg_tile_bits(views, 2, cfg) == 14
    cfg.tile_w, cfg.tile_h = 8, 32
    assert abi.mg_total_tiles(views, 1, cfg) == 195 * 33
    cfg.tile_w = 12
    assert abi.mg_total_tiles(views, 1, cfg) == -1          # not a power of two
    cfg.tile_w, cfg.tile_h = 64, 4
    assert abi.mg_total_tiles(views, 1, cfg) == -1          # no 8x8 warp blocks
    assert abi.mg_bin_workspace_bytes(1_200_000) > 8 * (1_200_000 // 2048)
    # two look-back status arrays of 256 digits per partition of 5120 keys
    assert abi.mg_sort_workspace_bytes(10_000_000, 46) > 2 * 256 * 4 * (10_000_000 // 5120)


def test_bad_arguments_rejected_on_host(lib):
    from paper_2412_20522_gb300 import abi, scenes
    from paper_2412_20522_gb300.rasterize import RasterConfig, make_views
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64, 50.0)
    views = make_views([cam], [(0, 5)])
    cfg = RasterConfig().c()
    g = abi.mg_gaussians()
    g.n, g.sh_degree = 5, 7                                   # bad SH degree
    out = abi.mg_splats()
    st = lib.mg_preprocess(C.byref(g), views, 1, C.byref(cfg), C.byref(out), None, None)
    assert st == abi.MG_ERR_INVALID_ARG
    g.sh_degree = 3                                           # null arrays
    st = lib.mg_preprocess(C.byref(g), views, 1, C.byref(cfg), C.byref(out), None, None)
    assert st == abi.MG_ERR_INVALID_ARG
    st = lib.mg_render(C.byref(out), None, None, None, views, 1, C.byref(cfg), None, None, None,
                       None, None)
    assert st == abi.MG_ERR_INVALID_ARG
    st = lib.mg_render_l1(C.byref(out), None, None, None, views, 1, C.byref(cfg), None, None, None,
                          None, None, None, None)
    assert st == abi.MG_ERR_INVALID_ARG
    alt = C.c_int32(0)
    st = lib.mg_sort(None, None, None, None, None, 0, 20, None, 1, None, 0, C.byref(alt), None,
                     None, None)
    assert st == abi.MG_ERR_INVALID_ARG


def test_mask_pruning_and_inference_arguments_rejected_on_host(lib):
    """New entry points check their arguments before any launch."""
    from paper_2412_20522_gb300 import abi, scenes
    from paper_2412_20522_gb300.rasterize import RasterConfig, make_views
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 64, 50.0)
    views = make_views([cam], [(0, 5)])
    g = abi.mg_gaussians()
    g.n, g.sh_degree = 5, 3
    out = abi.mg_splats()
    for field, bad in (("mask_mode", 4), ("mask_apply", 2), ("mask_loss", 5)):
        cfg = RasterConfig().c()
        setattr(cfg, field, bad)
        assert lib.mg_preprocess(C.byref(g), views, 1, C.byref(cfg), C.byref(out), None,
                                 None) == abi.MG_ERR_INVALID_ARG
    cfg = RasterConfig(lambda_m=float("nan")).c()
    assert lib.mg_preprocess(C.byref(g), views, 1, C.byref(cfg), C.byref(out), None,
                             None) == abi.MG_ERR_INVALID_ARG
    # mask loss needs the per-view counts
    cfg = RasterConfig(lambda_m=0.1).c()
    assert lib.mg_mask_loss(C.byref(out), views, 1, C.byref(cfg), None, None) == abi.MG_ERR_INVALID_ARG
    # pruning: draw count and arrays
    assert lib.mg_prune_sample(C.byref(g), 1, 2, 0, None, None) == abi.MG_ERR_INVALID_ARG
    assert lib.mg_prune_sample(C.byref(g), 1, 2, 10, None, None) == abi.MG_ERR_INVALID_ARG
    dst = abi.mg_gaussian_arrays()
    assert lib.mg_compact(C.byref(g), None, C.byref(dst), None, None, None, 0, None,
                          None) == abi.MG_ERR_INVALID_ARG
    assert abi.mg_compact_workspace_bytes(1_000_000) >= 4 * 1_000_000
    assert lib.mg_render_inference(C.byref(out), None, None, None, views, 1, C.byref(cfg), None,
                                   None) == abi.MG_ERR_INVALID_ARG
    assert lib.mg_tile_order(None, 10, None, None) == abi.MG_ERR_INVALID_ARG
    assert lib.mg_selftest_wait_timeout(10, None, None) == abi.MG_ERR_INVALID_ARG
    assert lib.mg_selftest_warp_wait_timeout(10, None, None) == abi.MG_ERR_INVALID_ARG
    # the device-side iteration counter: a null or misaligned word
    assert lib.mg_advance_iteration(None, 1, None) == abi.MG_ERR_INVALID_ARG
    assert lib.mg_advance_iteration(C.c_void_p(4), 1, None) == abi.MG_ERR_INVALID_ARG
