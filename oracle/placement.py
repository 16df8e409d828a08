"""Oracle of Image-GS's content-adaptive placement (Sec. 3.3, Eq. 6 and Eq. 7).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU arms of `bench.py` may import this module. It shares no code with the
CUDA path.

What it computes:

* Eq. 6 (initial positions): a pixel centre is drawn with probability
  (1 - lambda) |grad I(x)|_2 / sum |grad I| + lambda / (H W); every Gaussian
  takes the target colour at its pixel, scale 5 px and rotation 0 (Sec. 4.1),
  stored as inverse scale t = 1/5.
* Eq. 7 (progressive addition): a pixel is drawn with probability
  |c_r(x) - c_t(x)| / sum |c_r - c_t|, and a Gaussian is initialised there
  the same way.

Readings where the paper is silent (the same as the library header's):

* grad I: per channel, central differences (I[x+1] - I[x-1]) / 2 inside the
  image and one-sided differences at the borders (zero along an axis of
  length 1); |grad I|_2 is the 2-norm over both directions and all channels.
* |c_r - c_t| for n channels is the sum of the channels' absolute errors.
* Draws are independent (with replacement). Eq. 6 is drawn as its mixture: a
  first uniform u1 picks the uniform part when u1 < lambda, a second uniform
  u2 picks the pixel. If every weight is zero the draw is uniform.
* The draws are decided exactly so that both sides pick the same pixels:
  weights are computed in binary32 with the sequence below, quantised to
  integers floor(min(w, 4096) * 2^24) (non-finite -> 0), and u = r / 2^53 for
  53-bit integers r given as inputs; the uniform part takes pixel
  floor(r2 * H W / 2^53), the weighted part the pixel whose integer
  cumulative weight interval contains floor(r2 * total / 2^53), and the
  branch test is r1 < floor(lambda * 2^53).
* mu = ((w + 1/2) / W, (h + 1/2) / H) rounded to binary32.
"""
import numpy as np

F32 = np.float32
SCALE_BITS = 24
W_CAP = F32(4096.0)
R_BITS = 53
S_INIT = 5.0  # px (Sec. 4.1)


def _diff(I, axis):
    """Per-channel binary32 difference along axis (1: x, 0: y) of I [H, W]."""
    L = I.shape[axis]
    g = np.zeros_like(I, dtype=F32)
    if L == 1:
        return g
    a = np.moveaxis(I, axis, 0)
    d = np.moveaxis(g, axis, 0)
    d[0] = a[1] - a[0]
    d[L - 1] = a[L - 1] - a[L - 2]
    if L > 2:
        d[1:L - 1] = (a[2:] - a[:-2]) * F32(0.5)
    return g


def gradient_magnitude(target):
    """|grad I|_2 per pixel in binary32, [H, W]: s += gx^2, s += gy^2 over channels, sqrt."""
    t = np.asarray(target, dtype=F32)
    s = np.zeros(t.shape[1:], dtype=F32)
    for c in range(t.shape[0]):
        gx = _diff(t[c], 1)
        gy = _diff(t[c], 0)
        s = s + gx * gx
        s = s + gy * gy
    return np.sqrt(s)


def error_magnitude(render, target):
    """sum over channels of |c_r - c_t| per pixel in binary32, [H, W]."""
    r = np.asarray(render, dtype=F32)
    t = np.asarray(target, dtype=F32)
    s = np.zeros(t.shape[1:], dtype=F32)
    for c in range(t.shape[0]):
        s = s + np.abs(r[c] - t[c])
    return s


def quantise(w):
    """floor(min(w, 4096) * 2^24) as Python ints (non-finite -> 0)."""
    w = np.asarray(w, dtype=F32).ravel()
    w = np.where(np.isfinite(w), np.minimum(w, W_CAP), F32(0.0))
    return [int(v) for v in np.floor(w.astype(np.float64) * 2.0 ** SCALE_BITS)]


def draw_pixels(weights_int, r1, r2, lam):
    """Pixel indices (row-major) of the mixture draws, exactly as specified."""
    P = len(weights_int)
    total = sum(weights_int)
    excl = np.zeros(P, dtype=object)
    run = 0
    for i, v in enumerate(weights_int):
        excl[i] = run
        run += v
    thr = int(np.floor(lam * 2.0 ** R_BITS))
    out = []
    for a, b in zip(r1, r2):
        a, b = int(a), int(b)
        if a < thr or total == 0:
            out.append((b * P) >> R_BITS)
        else:
            t = (b * total) >> R_BITS
            # the last pixel whose exclusive prefix is <= t
            lo, hi = 0, P - 1
            while lo < hi:
                mid = (lo + hi + 1) // 2
                if excl[mid] <= t:
                    lo = mid
                else:
                    hi = mid - 1
            out.append(lo)
    return np.asarray(out, dtype=np.int64)


def gaussians_at(pixels, target):
    """Packed [count, 5+n] rows for new Gaussians at the given pixels."""
    t = np.asarray(target, dtype=F32)
    n, H, W = t.shape
    h, w = pixels // W, pixels % W
    rows = np.zeros((len(pixels), 5 + n), dtype=F32)
    rows[:, 0] = (w.astype(F32) + F32(0.5)) / F32(W)
    rows[:, 1] = (h.astype(F32) + F32(0.5)) / F32(H)
    rows[:, 2] = F32(0.0)
    rows[:, 3] = rows[:, 4] = F32(1.0 / S_INIT)
    rows[:, 5:] = t[:, h, w].T
    return rows


def init_gaussians(target, r1, r2, lam=0.3):
    """Eq. 6: one Gaussian per (r1, r2) draw."""
    w = quantise(gradient_magnitude(target))
    return gaussians_at(draw_pixels(w, r1, r2, lam), target)


def add_gaussians(target, render, r2):
    """Eq. 7: one Gaussian per draw r2 (weighted part only)."""
    w = quantise(error_magnitude(render, target))
    r1 = [2 ** R_BITS - 1] * len(r2)   # never the uniform part
    return gaussians_at(draw_pixels(w, r1, r2, 0.0), target)
