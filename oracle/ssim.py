"""Oracle of the image-space fitting loss L1 + w * L_SSIM (Sec. 3.3, Sec. 4.1).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU arms of `bench.py` may import this module. It shares no code with the
CUDA path.

Sec. 4.1 fits against L1 + 0.1 * L_SSIM. The paper does not define L_SSIM
further; the readings here (the same as the library header's) are the standard structural
similarity of Wang et al.:

* per channel, local statistics under an 11 x 11 Gaussian window with
  sigma = 1.5 (normalised to sum 1), applied as a zero-padded "same"
  correlation (pixels outside the image count as 0);
* SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 +
  s_y^2 + C2)) with C1 = 0.01^2, C2 = 0.03^2 (data range 1), s_x^2 =
  E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y;
* L_SSIM = 1 - mean of SSIM over channels and pixels; L1 is the mean
  absolute error over channels and pixels with d|z|/dz = sign(z), sign(0) = 0.

Everything is float64. The gradient with respect to the rendering x is the
closed form through the raw moments (mu_x, E[x^2], E[xy]) and the transposed
window (the window is symmetric, so the transpose of the zero-padded
correlation is the same correlation).
"""
import numpy as np
from scipy.ndimage import correlate1d

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window1d():
    i = np.arange(WIN, dtype=np.float64) - WIN // 2
    g = np.exp(-(i * i) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def blur(a):
    """Zero-padded separable window over the last two axes of a."""
    g = window1d()
    b = correlate1d(np.asarray(a, np.float64), g, axis=-1, mode="constant", cval=0.0)
    return correlate1d(b, g, axis=-2, mode="constant", cval=0.0)


def _terms(x, y):
    mx, my = blur(x), blur(y)
    exx, eyy, exy = blur(x * x), blur(y * y), blur(x * y)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    return mx, my, A1, A2, B1, B2


def ssim_map(x, y):
    """Per-pixel SSIM [n, H, W] of rendering x against target y."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    _, _, A1, A2, B1, B2 = _terms(x, y)
    return (A1 * A2) / (B1 * B2)


def image_loss(x, y, w_ssim):
    """L1 + w * (1 - mean SSIM) and its gradient with respect to x."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    M = x.size
    l1 = np.abs(x - y).mean()
    g = np.sign(x - y) / M
    if w_ssim == 0:
        return l1, g
    mx, my, A1, A2, B1, B2 = _terms(x, y)
    S = (A1 * A2) / (B1 * B2)
    # partials of S at fixed (mu_y, E[y^2]): through mu_x, E[x^2], E[xy]
    dS_dmx_direct = 2 * my * A2 / (B1 * B2) - S * 2 * mx / B1
    dS_dvx = -S / B2
    dS_dcxy = 2 * A1 / (B1 * B2)
    G1 = dS_dmx_direct - 2 * mx * dS_dvx - my * dS_dcxy   # d S / d mu_x
    G2 = dS_dvx                                            # d S / d E[x^2]
    G3 = dS_dcxy                                           # d S / d E[xy]
    dmean = (blur(G1) + 2 * x * blur(G2) + y * blur(G3)) / M
    return l1 + w_ssim * (1.0 - S.mean()), g - w_ssim * dmean
