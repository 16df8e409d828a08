"""Pins of the oracle's float64-key selection and of its near-tie report.

The kernels (and the oracle's main path) decide the top-K of Sec. 3.2 with
binary32 keys. selection_f64 ranks by float64 keys instead, and
selection_mismatches lists the points where the two selections differ; the
count on the benchmark workloads is what the float32 decision costs.
"""
import numpy as np

from oracle import image_gs as O
from paper_2407_01866_b300 import synth


def _q64_independent(g, H, W, px, py, idx):
    """d^T Sigma^-1 d with Sigma^-1 = inv(R S S^T R^T) from numpy.linalg."""
    mx = (g.xy[idx, 0].astype(np.float32) * np.float32(W)).astype(np.float64)
    my = (g.xy[idx, 1].astype(np.float32) * np.float32(H)).astype(np.float64)
    out = []
    for k, i in enumerate(idx):
        th = float(g.theta[i])
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        S = np.diag(1.0 / g.inv_scale[i].astype(np.float64))
        inv = np.linalg.inv(R @ S @ S.T @ R.T)
        d = np.array([px - mx[k], py - my[k]])
        out.append(d @ inv @ d)
    return np.array(out)


def test_selection_f64_is_the_sorted_float64_ranking():
    H, W, N = 64, 48, 300
    g = O.Gaussians.from_packed(synth.packed(synth.gaussians(N, 3, seed=3)))
    pts = synth.query_points(40, H, W, seed=4).astype(np.float64)
    for (x, y), got in zip(pts, O.selection_f64(g, pts, H, W, K=10)):
        tx, ty = min(int(x // 16), (W - 1) // 16), min(int(y // 16), (H - 1) // 16)
        member = np.nonzero(O.tile_members(g, tx, ty, 16, H, W))[0]
        q = _q64_independent(g, H, W, x, y, member)
        want = [i for _, i in sorted(zip(q.tolist(), member.tolist()))][:10]
        assert got.tolist() == want


def _twin_thetas():
    """Two binary32 angles one ulp apart whose cos and sin round to the same
    binary32 values (so the kernels' conics, and keys, are identical)."""
    th = np.float32(0.3)
    while True:
        t2 = np.nextafter(th, np.float32(1.0))
        same = (np.float32(np.cos(np.float64(th))) == np.float32(np.cos(np.float64(t2))) and
                np.float32(np.sin(np.float64(th))) == np.float32(np.sin(np.float64(t2))))
        if same:
            return th, t2
        th = t2


def test_mismatch_report_finds_a_constructed_near_tie():
    """Gaussians 0 and 1 share mu and scales and have twin angles: their
    binary32 keys tie at every pixel (the tie goes to index 0), while their
    float64 keys differ in a direction that flips across the long axis. With
    K = 1, exactly the pixels where Gaussian 1 is nearer in float64 differ."""
    H = W = 32
    th_a, th_b = _twin_thetas()
    xy = np.array([[0.5, 0.5], [0.5, 0.5], [0.05, 0.05]], np.float32)
    theta = np.array([th_a, th_b, 0.0], np.float32)
    inv_scale = np.array([[1.0, 0.05], [1.0, 0.05], [1.0, 1.0]], np.float32)
    color = np.eye(3, dtype=np.float32)
    g = O.Gaussians(xy, theta, inv_scale, color)
    pts = np.array([[16.5 + dx, 16.5 + dy] for dx in (-3, 3) for dy in (-2, 2)], np.float64)
    q = np.stack([_q64_independent(g, H, W, x, y, [0, 1]) for x, y in pts])
    want = [i for i in range(len(pts)) if q[i, 1] < q[i, 0]]
    assert 0 < len(want) < len(pts)       # the float64 order flips between pixels
    mx = np.float32(np.float32(0.5) * np.float32(W))
    A00, B, A11 = O.conic32(g)
    for x, y in pts:                      # the binary32 keys tie exactly
        k = O.rank_key32(x, y, mx, mx, A00[:2], B[:2], A11[:2])
        assert k[0] == k[1]
    assert O.selection_mismatches(g, pts, H, W, K=1) == want
    assert O.selection_mismatches(g, pts, H, W, K=2) == []


def test_near_tie_count_on_the_workloads():
    """Sampled pixels of the 256^2 and 2048^2 workloads (initial parameters):
    pixels whose binary32 selection differs from the float64 one."""
    for name, count in (("fit256_rgb", 2048), ("fit2048_rgb", 1024)):
        c = synth.CONFIGS[name]
        g = O.Gaussians.from_packed(synth.packed(synth.gaussians(c["N"], 3, seed=0)))
        pix = synth.sample_pixels(count, c["H"], c["W"], seed=9)
        bad = O.selection_mismatches(g, O.pixel_centres(pix), c["H"], c["W"])
        print(f"{name}: {len(bad)} of {count} sampled pixels select differently "
              "under float64 keys")
        assert len(bad) <= count // 200
