"""Host-only checks of the C ABI: the library loads, exports every function that
include/imgs.h declares, and validates arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2407_01866_b300 import lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# each public header and the library that exports its declarations
HEADERS = {"imgs.h": "libimgs.so", "igs_peaks.h": "libigs_peaks.so"}


def declared_functions(header="imgs.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:int|void)\s+(igs_\w+)\s*\(", text, flags=re.M))


def test_every_header_is_mapped_to_its_library():
    assert sorted(h for h in os.listdir(os.path.join(ROOT, "include"))
                  if h.endswith(".h")) == sorted(HEADERS)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_2407_01866_b300 import build
        build.build()
    return L.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["igs_preprocess_bin", "igs_render_forward", "igs_render_backward",
                 "igs_fit_step", "igs_decode_points", "igs_workspace_size", "igs_read_stats"]:
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), f"{name} not exported by libimgs.so"
    assert names <= set(L.exported_names()), names - set(L.exported_names())


def test_peak_probe_library_exports_its_header(lib):
    from paper_2407_01866_b300 import peaks
    names = declared_functions("igs_peaks.h")
    assert names == {"igs_peak_probe"}
    plib = peaks.load()
    for name in names:
        assert hasattr(plib, name), f"{name} not exported by libigs_peaks.so"


def test_version_and_default_config(lib):
    assert L.version() == 10000
    c = L.default_config()
    assert c.K == 10 and c.tile == 16 and c.normalize == 1
    assert abs(c.lr_mu - 5e-4) < 1e-9 and abs(c.lr_color - 5e-3) < 1e-9
    assert abs(c.lr_inv_scale - 2e-3) < 1e-9 and abs(c.lr_theta - 2e-3) < 1e-9
    assert abs(c.theta_max - 3.14159265) < 1e-6


def test_workspace_size_grows_with_inputs_and_validates(lib):
    c = L.default_config()
    a = L.workspace_size(1000, 3, 256, 256, c, 10_000)
    b = L.workspace_size(2000, 3, 256, 256, c, 10_000)
    d = L.workspace_size(1000, 3, 256, 256, c, 20_000)
    assert 0 < a < b and a < d
    with pytest.raises(L.IgsError) as e:
        L.workspace_size(1000, 3, 256, 256, L.default_config(K=5), 10_000)
    assert e.value.code == L.IGS_ERR_INVALID_ARG
    with pytest.raises(L.IgsError):
        L.workspace_size(1000, 3, 256, 256, L.default_config(tile=12), 10_000)
    with pytest.raises(L.IgsError):
        L.workspace_size(1000, 0, 256, 256, c, 10_000)
    with pytest.raises(L.IgsError):
        L.workspace_size(1000, 3, 0, 256, c, 10_000)
    # the render grid has one CTA per tile and at most 65535 rows of tiles
    c8 = L.default_config(tile=8)
    assert L.workspace_size(1000, 3, 8 * 65535, 16, c8, 10_000) > 0
    with pytest.raises(L.IgsError) as e:
        L.workspace_size(1000, 3, 8 * 65535 + 1, 16, c8, 10_000)
    assert e.value.code == L.IGS_ERR_INVALID_ARG
    assert "65535" in str(e.value)


def test_entry_points_reject_bad_arguments_without_a_gpu(lib):
    c = L.default_config()
    bins = L.Bins()
    g = L.Gaussians()
    assert lib.igs_preprocess_bin(None, 16, 16, ctypes.byref(c), None, 0, 1,
                                  ctypes.byref(bins), None) == L.IGS_ERR_INVALID_ARG
    g.N, g.n, g.dtype = 4, 3, 0
    g.xy_stride, g.theta_stride, g.inv_scale_stride, g.color_stride = 2, 1, 2, 3
    g.xy = g.theta = g.inv_scale = g.color = 4096
    rc = lib.igs_preprocess_bin(ctypes.byref(g), 16, 16, ctypes.byref(c), ctypes.c_void_p(4096 + 16),
                                1 << 20, 100, ctypes.byref(bins), None)
    assert rc == L.IGS_ERR_ALIGN
    rc = lib.igs_preprocess_bin(ctypes.byref(g), 16, 16, ctypes.byref(c), ctypes.c_void_p(4096),
                                16, 100, ctypes.byref(bins), None)
    assert rc == L.IGS_ERR_INVALID_ARG
    buf = ctypes.create_string_buffer(256)
    assert lib.igs_last_error(buf, 256) > 0 and b"workspace" in buf.value
    g.dtype = 7
    rc = lib.igs_preprocess_bin(ctypes.byref(g), 16, 16, ctypes.byref(c), ctypes.c_void_p(4096),
                                1 << 20, 100, ctypes.byref(bins), None)
    assert rc == L.IGS_ERR_INVALID_ARG
    assert lib.igs_render_forward(ctypes.byref(bins), ctypes.byref(c), None, None) == \
        L.IGS_ERR_INVALID_ARG
    assert lib.igs_decode_points(None, ctypes.byref(c), None, 0, None, None) == \
        L.IGS_ERR_INVALID_ARG
    assert lib.igs_fit_step(None, None, 16, 16, ctypes.byref(c), None, 0, 1, None, None) == \
        L.IGS_ERR_INVALID_ARG
    st = L.FitState(4096, 8192, 12288, 16384, 20480, 4, 3)
    assert lib.igs_fit_step_half(ctypes.byref(st), ctypes.c_void_p(24576), 0, ctypes.c_void_p(28672),
                                 16, 16, ctypes.byref(c), None, 0, 1, None, None) == \
        L.IGS_ERR_INVALID_ARG   # float32 is not a half storage type
    assert lib.igs_fit_step_half(ctypes.byref(st), ctypes.c_void_p(24576 + 2), 1,
                                 ctypes.c_void_p(28672), 16, 16, ctypes.byref(c), None, 0, 1,
                                 None, None) == L.IGS_ERR_ALIGN
    assert lib.igs_image_loss(None, None, 0, 8, 8, ctypes.c_float(0.1), None, None, None, 0,
                              None) == L.IGS_ERR_INVALID_ARG
    assert lib.igs_image_loss(ctypes.c_void_p(4096), ctypes.c_void_p(8192), 3, 8, 8,
                              ctypes.c_float(0.1), ctypes.c_void_p(12288), None,
                              ctypes.c_void_p(16384 + 64), 1 << 20, None) == L.IGS_ERR_ALIGN
    bad = L.default_config(ssim_weight=-1.0)
    b = ctypes.c_size_t()
    assert lib.igs_workspace_size(10, 3, 16, 16, ctypes.byref(bad), 100, ctypes.byref(b)) == \
        L.IGS_ERR_INVALID_ARG
    on = L.default_config(ssim_weight=0.1)
    assert L.workspace_size(10, 3, 64, 64, on, 100) > L.workspace_size(10, 3, 64, 64, c, 100)
