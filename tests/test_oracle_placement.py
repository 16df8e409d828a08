"""Pins of the placement oracle (Sec. 3.3, Eq. 6 and Eq. 7) against
references outside it: numpy's gradient operator, closed-form cases and the
empirical distribution of many draws."""
import numpy as np

from oracle import placement as PL

R53 = 2 ** 53


def _rand(count, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, R53, count, dtype=np.int64), rng.integers(0, R53, count, dtype=np.int64))


def test_gradient_magnitude_matches_numpy_gradient():
    rng = np.random.default_rng(0)
    t = rng.uniform(0, 1, (3, 17, 23)).astype(np.float32)
    got = PL.gradient_magnitude(t).astype(np.float64)
    want = np.zeros(t.shape[1:])
    for c in range(3):
        gy, gx = np.gradient(t[c].astype(np.float64))
        want += gx ** 2 + gy ** 2
    np.testing.assert_allclose(got, np.sqrt(want), rtol=2e-6, atol=1e-7)
    # an axis of length 1 has no gradient along it
    row = rng.uniform(0, 1, (1, 1, 9)).astype(np.float32)
    np.testing.assert_allclose(PL.gradient_magnitude(row)[0],
                               np.abs(np.gradient(row[0, 0].astype(np.float64))), rtol=2e-6)


def test_a_single_bright_pixel_puts_every_weighted_draw_on_its_four_neighbours():
    t = np.zeros((1, 9, 11), np.float32)
    t[0, 4, 6] = 1.0
    r1, r2 = _rand(4000, 1)
    P = PL.init_gaussians(t, r1, r2, lam=0.0)
    px = np.round(P[:, 0] * 11 - 0.5).astype(int)
    py = np.round(P[:, 1] * 9 - 0.5).astype(int)
    got = set(zip(py.tolist(), px.tolist()))
    assert got == {(4, 5), (4, 7), (3, 6), (5, 6)}
    # equal weights 1/2: close to a quarter each
    for cell in got:
        frac = np.mean((py == cell[0]) & (px == cell[1]))
        assert abs(frac - 0.25) < 0.03
    # the new Gaussians: scale 5 px, rotation 0, the target colour
    assert np.all(P[:, 2] == 0) and np.all(P[:, 3:5] == np.float32(0.2))
    assert np.all(P[:, 5] == 0.0)


def test_draws_follow_eq6_distribution():
    rng = np.random.default_rng(2)
    t = rng.uniform(0, 1, (3, 5, 6)).astype(np.float32)
    lam = 0.3
    g = np.zeros(t.shape[1:])
    for c in range(3):
        gy, gx = np.gradient(t[c].astype(np.float64))
        g += gx ** 2 + gy ** 2
    g = np.sqrt(g)
    p = (1 - lam) * g / g.sum() + lam / g.size       # Eq. 6 in float64
    r1, r2 = _rand(120_000, 3)
    w = PL.quantise(PL.gradient_magnitude(t))
    pix = PL.draw_pixels(w, r1, r2, lam)
    freq = np.bincount(pix, minlength=g.size) / len(pix)
    sigma = np.sqrt(p.ravel() * (1 - p.ravel()) / len(pix))
    assert np.all(np.abs(freq - p.ravel()) <= 5 * sigma + 1e-4)


def test_error_draws_land_only_where_the_error_is():
    rng = np.random.default_rng(4)
    t = rng.uniform(0, 1, (3, 8, 8)).astype(np.float32)
    r = t.copy()
    r[1, 2, 5] += 0.25
    r[0, 6, 1] -= 0.75
    _, r2 = _rand(3000, 5)
    P = PL.add_gaussians(t, r, r2)
    cells = list(zip(np.round(P[:, 1] * 8 - 0.5).astype(int).tolist(),
                     np.round(P[:, 0] * 8 - 0.5).astype(int).tolist()))
    assert set(cells) == {(2, 5), (6, 1)}
    frac = np.mean([c == (6, 1) for c in cells])
    assert abs(frac - 0.75) < 0.04          # Eq. 7: error 0.75 vs 0.25
    # a perfect render gives uniform draws
    P0 = PL.add_gaussians(t, t, r2[:2000])
    assert len(set(np.round(P0[:, 0] * 8 - 0.5).astype(int).tolist())) == 8


def test_lambda_one_is_uniform_over_pixels():
    t = np.zeros((1, 4, 4), np.float32)
    t[0, 1, 1] = 1.0
    r1, r2 = _rand(64_000, 6)
    pix = PL.draw_pixels(PL.quantise(PL.gradient_magnitude(t)), r1, r2, 1.0)
    freq = np.bincount(pix, minlength=16) / len(pix)
    assert np.all(np.abs(freq - 1 / 16) < 0.01)
