"""Pins of the image-loss oracle (L1 + w * L_SSIM): brute-force window sums,
closed-form cases and finite differences."""
import numpy as np

from oracle import ssim as S


def test_separable_blur_equals_brute_force_window_sum():
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, (2, 9, 13))
    g = S.window1d()
    w2 = np.outer(g, g)
    want = np.zeros_like(a)
    r = S.WIN // 2
    for c in range(2):
        for yy in range(9):
            for xx in range(13):
                s = 0.0
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        y2, x2 = yy + dy, xx + dx
                        if 0 <= y2 < 9 and 0 <= x2 < 13:
                            s += w2[dy + r, dx + r] * a[c, y2, x2]
                want[c, yy, xx] = s
    np.testing.assert_allclose(S.blur(a), want, rtol=1e-13, atol=1e-15)
    # the window: normalised Gaussian with sigma 1.5
    assert abs(g.sum() - 1.0) < 1e-15 and abs(g[6] / g[5] - np.exp(-1 / 4.5)) < 1e-15


def test_ssim_of_an_image_with_itself_is_one_and_has_no_gradient():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, 20, 17))
    np.testing.assert_allclose(S.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    loss, g = S.image_loss(x, x, 0.1)
    assert abs(loss) < 1e-12
    assert np.abs(g).max() < 1e-12


def test_constant_images_give_the_closed_form_inside():
    a, b = 0.3, 0.7
    x = np.full((1, 30, 30), a)
    y = np.full((1, 30, 30), b)
    m = S.ssim_map(x, y)
    want = (2 * a * b + S.C1) / (a * a + b * b + S.C1)   # zero variances
    np.testing.assert_allclose(m[0, 10:20, 10:20], want, rtol=1e-12)


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 1, (2, 12, 14))
    x = np.clip(y + rng.normal(0, 0.2, y.shape), 0, 1)
    w = 0.1
    _, g = S.image_loss(x, y, w)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (1, 5, 7), (0, 11, 13), (1, 3, 12), (0, 6, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (S.image_loss(xp, y, w)[0] - S.image_loss(xm, y, w)[0]) / (2 * h)
        assert abs(fd - g[c, i, j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (c, i, j, fd, g[c, i, j])


def test_zero_weight_is_plain_l1():
    rng = np.random.default_rng(3)
    x, y = rng.uniform(0, 1, (2, 3, 8, 8))
    loss, g = S.image_loss(x, y, 0.0)
    assert abs(loss - np.abs(x - y).mean()) < 1e-15
    np.testing.assert_array_equal(g, np.sign(x - y) / x.size)
