"""The image-space fitting loss L1 + w (1 - SSIM) (Sec. 4.1) and the fit step
that uses it, through the C ABI, against the float64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import image_gs as O  # noqa: E402
from oracle import ssim as S  # noqa: E402
from paper_2407_01866_b300 import lib as L  # noqa: E402
from paper_2407_01866_b300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_harness import dev, grad_rel_error  # noqa: E402


def _pair(n, H, W, seed):
    """A target and a 'rendering' that differs from it by at least 1e-3 everywhere
    (one correct sign for the L1 term)."""
    y = synth.target_image(H, W, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    d = rng.normal(0, 0.08, y.shape)
    d = np.where(np.abs(d) < 1e-3, np.where(d >= 0, 1e-3, -1e-3), d)
    return (y + d).astype(np.float32), y


@pytest.mark.parametrize("n,H,W,w", [(3, 64, 48, 0.1), (1, 37, 53, 1.0), (9, 32, 40, 0.1),
                                     (3, 20, 20, 0.0), (2, 1, 30, 0.1), (3, 150, 97, 0.1)])
def test_image_loss_and_gradient_match_oracle(n, H, W, w):
    x, y = _pair(n, H, W, 3 + n)
    g = torch.empty((n, H, W), device="cuda")
    loss = torch.zeros(1, device="cuda")
    L.image_loss(dev(x), dev(y), w, g, loss)
    want_loss, want_g = S.image_loss(x.astype(np.float64), y.astype(np.float64), w)
    assert abs(loss.item() - want_loss) <= 2e-6 * max(1.0, want_loss)
    got = g.cpu().numpy().astype(np.float64)
    assert np.abs(got - want_g).max() <= 1e-3 * np.abs(want_g).max()


def test_fit_step_with_the_ssim_term_matches_oracle():
    H, W, N, n = 96, 80, 700, 3
    P = synth.packed(synth.gaussians(N, n, 11))
    g = O.Gaussians.from_packed(P)
    img = O.render_image(g, H, W)
    y = synth.target_image(H, W, n, seed=12).astype(np.float64)
    close = np.abs(img - y) < 1e-4
    y[close] = img[close] + np.where(y[close] >= img[close], 1e-4, -1e-4)
    y = y.astype(np.float32)
    cfg = L.default_config(ssim_weight=0.1)
    Pt = dev(P)
    G = torch.zeros_like(Pt)
    m = torch.zeros_like(Pt)
    v = torch.zeros_like(Pt)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.FitState(Pt.data_ptr(), G.data_ptr(), m.data_ptr(), v.data_ptr(), step.data_ptr(), N, n)
    ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, 8 * N))
    assert ws.numel() > L.workspace_size(N, n, H, W, L.default_config(), 8 * N)
    loss = torch.zeros(1, device="cuda")
    L.fit_step(st, dev(y), H, W, cfg, ws, 8 * N, loss)
    torch.cuda.synchronize()
    want_loss, dimg = S.image_loss(img, y.astype(np.float64), 0.1)
    assert abs(loss.item() - want_loss) <= 2e-6 * max(1.0, want_loss)
    ref = O.backward_image(g, dimg, H, W)
    errs = grad_rel_error(G.cpu().numpy().astype(np.float64), ref)
    assert max(errs.values()) <= 1e-3, errs
    # a workspace sized for L1 alone is refused
    small = L.alloc_workspace(L.workspace_size(N, n, H, W, L.default_config(), 8 * N))
    with pytest.raises(L.IgsError):
        L.fit_step(st, dev(y), H, W, cfg, small, 8 * N, loss)
