"""Seeded synthetic inputs for the Image-GS rasteriser.

This module generates inputs only: targets, Gaussian parameter sets and
query points. It holds none of the method's arithmetic, and both the tests
(oracle side and CUDA side) and the benchmark draw their inputs from it.

The paper's own data (45 stylised 2K images, 19 texture stacks, CLIC2020) are
not available; these generators stand in for them at the paper's 2K x 2K scale
and its 3- and 9-channel shapes (Sec. 4.1).

Target generator, per channel: a sum of k random sinusoids (1-64 cycles per
image, random orientation and phase, amplitude 1/k), plus optional value noise
(bilinear random lattices at 8, 16, 32 cells per side with amplitudes 1/2,
1/4, 1/8), rescaled to [0, 1]; then R axis-aligned rectangles of uniform
colour are painted over it (sharp edges).

Gaussians: mu uniform in [0,1]^2, s1 and s2 independently log-uniform in
[0.5, 8] px (the inverse scale t = 1/s is what is stored), theta uniform in
[0, pi), colours uniform in [0, 1] (or a given range per channel).
"""
import numpy as np


def _sinusoids(rng, H, W, k):
    yy = (np.arange(H, dtype=np.float64) + 0.5) / H
    xx = (np.arange(W, dtype=np.float64) + 0.5) / W
    img = np.zeros((H, W), dtype=np.float64)
    for _ in range(k):
        f = rng.uniform(1.0, 64.0)
        ang = rng.uniform(0.0, np.pi)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        fx, fy = f * np.cos(ang), f * np.sin(ang)
        img += np.sin(2.0 * np.pi * (fy * yy[:, None] + fx * xx[None, :]) + ph) / k
    return img


def _value_noise(rng, H, W, octaves=3):
    img = np.zeros((H, W), dtype=np.float64)
    cells, amp = 8, 0.5
    for _ in range(octaves):
        lat = rng.uniform(0.0, 1.0, size=(cells + 1, cells + 1))
        gy = (np.arange(H) + 0.5) / H * cells
        gx = (np.arange(W) + 0.5) / W * cells
        iy = np.minimum(gy.astype(np.int64), cells - 1)
        ix = np.minimum(gx.astype(np.int64), cells - 1)
        fy = (gy - iy)[:, None]
        fx = (gx - ix)[None, :]
        a = lat[iy][:, ix]
        b = lat[iy][:, ix + 1]
        c = lat[iy + 1][:, ix]
        d = lat[iy + 1][:, ix + 1]
        img += amp * ((1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d))
        cells *= 2
        amp *= 0.5
    return img


def target_image(H, W, n=3, seed=0, n_sin=8, n_rect=20, noise_octaves=0):
    """Planar float32 target [n, H, W] in [0, 1]."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, H, W), dtype=np.float32)
    for ch in range(n):
        base = _sinusoids(rng, H, W, n_sin)
        if noise_octaves:
            base = base + _value_noise(rng, H, W, noise_octaves)
        lo, hi = base.min(), base.max()
        base = (base - lo) / (hi - lo) if hi > lo else np.zeros_like(base)
        out[ch] = base
    for _ in range(n_rect):
        x0, x1 = np.sort(rng.integers(0, W + 1, size=2))
        y0, y1 = np.sort(rng.integers(0, H + 1, size=2))
        col = rng.uniform(0.0, 1.0, size=n)
        out[:, y0:y1, x0:x1] = col[:, None, None].astype(np.float32)
    return out


def texture_stack(H, W, seed=0, n_sin=8, n_rect=20, noise_octaves=3):
    """9-channel float32 texture stack [9, H, W]: albedo RGB, normal XYZ in
    [-1, 1] renormalised to unit length, roughness, metallic, AO."""
    t = target_image(H, W, n=9, seed=seed, n_sin=n_sin, n_rect=n_rect,
                     noise_octaves=noise_octaves)
    nrm = t[3:6].astype(np.float64) * 2.0 - 1.0
    nrm[2] = np.abs(nrm[2]) + 0.25          # keep normals facing +z
    nrm /= np.linalg.norm(nrm, axis=0, keepdims=True)
    t[3:6] = nrm.astype(np.float32)
    return t


def gaussians(N, n=3, seed=0, s_range=(0.5, 8.0), color_lo=0.0, color_hi=1.0):
    """Random parameter set, float32 arrays: xy [N,2], theta [N], inv_scale [N,2], color [N,n].

    color_lo / color_hi may be scalars or per-channel sequences."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0.0, 1.0, size=(N, 2))
    ls = rng.uniform(np.log(s_range[0]), np.log(s_range[1]), size=(N, 2))
    theta = rng.uniform(0.0, np.pi, size=N)
    lo = np.broadcast_to(np.asarray(color_lo, dtype=np.float64), (n,))
    hi = np.broadcast_to(np.asarray(color_hi, dtype=np.float64), (n,))
    color = rng.uniform(0.0, 1.0, size=(N, n)) * (hi - lo) + lo
    return dict(xy=xy.astype(np.float32), theta=theta.astype(np.float32),
                inv_scale=np.exp(-ls).astype(np.float32), color=color.astype(np.float32))


def packed(g):
    """Pack a parameter dict into rows (mu_x, mu_y, theta, t1, t2, c...), float32 [N, 5+n]."""
    return np.concatenate([g["xy"], g["theta"][:, None], g["inv_scale"], g["color"]],
                          axis=1).astype(np.float32)


def query_points(Q, H, W, seed=0):
    """Q points uniform over [0, W) x [0, H), float32 [Q, 2] = (x, y) in pixels."""
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.uniform(0.0, W, size=Q), rng.uniform(0.0, H, size=Q)], axis=1)
    pts = np.minimum(pts.astype(np.float32), np.array([np.nextafter(np.float32(W), 0),
                                                      np.nextafter(np.float32(H), 0)],
                                                     dtype=np.float32))
    return pts


def sample_pixels(count, H, W, seed=0):
    """count distinct (h, w) pixel indices, int64 [count, 2]."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(H * W, size=min(count, H * W), replace=False)
    return np.stack([idx // W, idx % W], axis=1).astype(np.int64)


def batch_shapes(B=64, seed=0, side_range=(256, 2048), px_per_gaussian=28):
    """Ragged batch: list of (H, W, N) with sides log-uniform in side_range."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(side_range[0]), np.log(side_range[1])
    out = []
    for _ in range(B):
        H = int(round(np.exp(rng.uniform(lo, hi))))
        W = int(round(np.exp(rng.uniform(lo, hi))))
        out.append((H, W, max(1, int(round(H * W / px_per_gaussian)))))
    return out


# Named workloads (sizes from the statement of the problem; seeds 0..4).
CONFIGS = {
    "fit256_rgb": dict(H=256, W=256, n=3, N=4096, n_sin=8, n_rect=20, noise=0),
    "fit2048_rgb": dict(H=2048, W=2048, n=3, N=100_000, n_sin=8, n_rect=200, noise=3),
    "fit4096_tex9": dict(H=4096, W=4096, n=9, N=500_000, n_sin=8, n_rect=200, noise=3),
    "decode8192_rgb": dict(H=8192, W=8192, n=3, N=2_000_000, n_sin=8, n_rect=200, noise=3,
                           Q=1_000_000),
}
