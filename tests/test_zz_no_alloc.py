"""The no-allocation render entry point, igs_render_forward_static.

It exists for callers that cannot call cudaMalloc or pass the library a
workspace (a plug-in inside an application that owns all device memory, a
real-time thread that must not block on an allocation, code held to a fixed
memory budget). Its scratch is one static device array shared by every call.
The test renders through it twice in a row, with different Gaussians so that
contents left over by the first call would show, and compares each image
with the existing path (igs_preprocess_bin + igs_render_forward on a caller
workspace) at the pixel tolerance of the other parity tests. This file is
collected last so that a run stopping at its first failure has already run
every other test; it needs nothing from them.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2407_01866_b300 import lib as L  # noqa: E402
from paper_2407_01866_b300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PIX_TOL = 1e-5


def _params(N, n, seed):
    d = synth.gaussians(N, n, seed)
    return [torch.from_numpy(d[k]).cuda() for k in ("xy", "theta", "inv_scale", "color")]


def _existing_path(ts, H, W, cfg):
    view = L.gaussians_view(*ts)
    binner = L.Binner(view.N, view.n, H, W, cfg)
    bins = binner.bin(view)
    img = torch.empty((view.n, H, W), device="cuda")
    L.render_forward(bins, cfg, img)
    return img


def test_static_scratch_render_matches_workspace_render_twice_in_a_row():
    cfg = L.default_config()
    H, W, n = 256, 256, 3
    for N, seed in ((4096, 0), (3000, 1)):
        ts = _params(N, n, seed)
        img = torch.full((n, H, W), float("nan"), device="cuda")
        L.render_forward_static(L.gaussians_view(*ts), H, W, cfg, img)
        ref = _existing_path(ts, H, W, cfg)
        torch.cuda.synchronize()
        err = (img - ref).abs().max().item()
        assert err <= PIX_TOL, err


def test_static_scratch_rejects_oversized_problems():
    assert L.static_scratch_bytes() == 32 << 20
    cfg = L.default_config()
    g = L.Gaussians()
    g.N, g.n, g.dtype = 3_000_000, 3, L.IGS_F32       # parameters alone exceed 32 MiB
    g.xy_stride, g.theta_stride, g.inv_scale_stride, g.color_stride = 2, 1, 2, 3
    img = torch.empty(1, device="cuda")
    with pytest.raises(L.IgsError) as e:
        L.render_forward_static(g, 64, 64, cfg, img)
    assert e.value.code == L.IGS_ERR_CAPACITY
    buf = ctypes.create_string_buffer(512)
    L.load().igs_last_error(buf, 512)
    assert b"static scratch" in buf.value


def test_static_scratch_reports_too_many_intersections_then_recovers():
    """Large Gaussians on a 1024x1024 image hit more tiles than the static
    scratch's list holds: the GPU finds it out, the call returns
    IGS_ERR_CAPACITY with an incomplete image, and the next, smaller call
    still matches the workspace path."""
    cfg = L.default_config()
    H = W = 1024
    n = 3
    big = synth.gaussians(20000, n, seed=2, s_range=(50.0, 100.0))
    ts = [torch.from_numpy(big[k]).cuda() for k in ("xy", "theta", "inv_scale", "color")]
    img = torch.zeros((n, H, W), device="cuda")
    with pytest.raises(L.IgsError) as e:
        L.render_forward_static(L.gaussians_view(*ts), H, W, cfg, img)
    assert e.value.code == L.IGS_ERR_CAPACITY
    buf = ctypes.create_string_buffer(512)
    L.load().igs_last_error(buf, 512)
    assert b"static scratch" in buf.value
    ts = _params(4096, n, 3)
    img = torch.full((n, H, W), float("nan"), device="cuda")
    L.render_forward_static(L.gaussians_view(*ts), H, W, cfg, img)
    ref = _existing_path(ts, H, W, cfg)
    torch.cuda.synchronize()
    assert (img - ref).abs().max().item() <= PIX_TOL


@pytest.mark.parametrize("H,W,n,tile,ssim", [(1024, 1024, 3, 16, 0.1), (200, 136, 9, 8, 0.0)])
def test_static_scratch_other_shapes_match_workspace_render(H, W, n, tile, ssim):
    """An SSIM weight in the config leaves the scratch to the binning (a
    1024x1024 render fits), and a ragged 8x8-tile, 9-channel render matches."""
    cfg = L.default_config(tile=tile, ssim_weight=ssim)
    ts = _params(20000 if H == 1024 else 3000, n, 4)
    img = torch.full((n, H, W), float("nan"), device="cuda")
    L.render_forward_static(L.gaussians_view(*ts), H, W, cfg, img)
    ref = _existing_path(ts, H, W, cfg)
    torch.cuda.synchronize()
    assert (img - ref).abs().max().item() <= PIX_TOL
