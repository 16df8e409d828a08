"""Pins of the FP64 oracle against closed forms, invariants, brute force and libraries.

Each test fixes something the paper and the mathematics determine without
reference to the oracle's own code (Eq. 1-5, Sec. 3.2-3.3, Sec. 4.1).
"""
import math

import numpy as np
import pytest

from oracle import image_gs as O
from paper_2407_01866_b300 import synth


def make(xy, theta, inv_scale, color):
    return O.Gaussians(np.asarray(xy, np.float32), np.asarray(theta, np.float32),
                       np.asarray(inv_scale, np.float32), np.asarray(color, np.float32))


def rand_set(N, n, seed, s_range=(0.5, 8.0)):
    d = synth.gaussians(N, n, seed, s_range=s_range)
    return O.Gaussians(d["xy"], d["theta"], d["inv_scale"], d["color"])


# ---------------------------------------------------------------- Eq. 1 / Eq. 2

def test_conic_equals_inverse_of_factored_covariance():
    """Sigma = R S S^T R^T (Eq. 2); the closed-form inverse equals numpy.linalg.inv."""
    g = rand_set(200, 3, 0)
    A00, A01, A11 = O.conic64(g)
    for i in range(g.N):
        th = float(g.theta[i])
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        S = np.diag(1.0 / g.inv_scale[i].astype(np.float64))
        inv = np.linalg.inv(R @ S @ S.T @ R.T)
        np.testing.assert_allclose([[A00[i], A01[i]], [A01[i], A11[i]]], inv,
                                   rtol=1e-10, atol=1e-12)


def test_binary32_conic_close_to_float64_conic():
    g = rand_set(500, 3, 1)
    A00, B, A11 = O.conic32(g)
    a00, a01, a11 = O.conic64(g)
    scale = np.maximum(np.abs(a00), np.abs(a11))
    assert np.max(np.abs(A00 - a00) / scale) < 1e-6
    assert np.max(np.abs(B / 2 - a01) / scale) < 1e-6
    assert np.max(np.abs(A11 - a11) / scale) < 1e-6


def test_single_axis_aligned_gaussian_closed_form_naive_mode():
    """Eq. 4 with one Gaussian at theta = 0 is c * exp(-((x-mx)^2 t1^2 + (y-my)^2 t2^2)/2)."""
    H, W = 40, 56
    g = make([[0.3, 0.6]], [0.0], [[0.4, 0.15]], [[0.7, -0.2]])
    mx = float(np.float32(np.float32(0.3) * np.float32(W)))
    my = float(np.float32(np.float32(0.6) * np.float32(H)))
    t1, t2 = float(np.float32(0.4)), float(np.float32(0.15))
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, [W, H], size=(300, 2))
    got = O.render_naive(g, pts, H, W)
    for (x, y), row in zip(pts, got):
        G = math.exp(-0.5 * (((x - mx) * t1) ** 2 + ((y - my) * t2) ** 2))
        assert abs(row[0] - float(np.float32(0.7)) * G) < 1e-14
        assert abs(row[1] - float(np.float32(-0.2)) * G) < 1e-14


# ---------------------------------------------------------------- Eq. 5 closed forms

def test_one_gaussian_is_constant_on_every_touched_tile_and_zero_elsewhere():
    H, W, T = 64, 48, 16
    g = make([[0.41, 0.37]], [0.6], [[0.5, 0.25]], [[0.2, 0.9, 0.5]])
    img = O.render_image(g, H, W, K=10, tile=T)
    mx, my = 0.41 * W, 0.37 * H
    r = 3.0 / 0.25
    for ty in range(H // T):
        for tx in range(W // T):
            # independent closed-rectangle distance in float64
            ex = max(tx * T - mx, mx - (tx + 1) * T, 0.0)
            ey = max(ty * T - my, my - (ty + 1) * T, 0.0)
            touched = math.hypot(ex, ey) <= r
            block = img[:, ty * T:(ty + 1) * T, tx * T:(tx + 1) * T]
            want = np.array([0.2, 0.9, 0.5], np.float32).astype(np.float64) if touched else np.zeros(3)
            np.testing.assert_allclose(block.reshape(3, -1).T, np.broadcast_to(want, (T * T, 3)),
                                       rtol=0, atol=1e-15)


def test_two_gaussians_give_a_logistic_blend():
    """Eq. 5 with two Gaussians: c = c2 + (c1 - c2) * sigmoid(-(q1 - q2)/2)."""
    H, W = 32, 32
    g = make([[0.4, 0.5], [0.6, 0.45]], [0.0, 0.0], [[0.3, 0.2], [0.25, 0.35]],
             [[1.0], [0.0]])
    pts = np.array([[x + 0.5, y + 0.5] for y in range(8, 24) for x in range(8, 24)])
    got = O.render_points(g, pts, H, W, K=10, tile=16)[:, 0]
    m = [(float(np.float32(np.float32(0.4) * 32)), float(np.float32(np.float32(0.5) * 32))),
         (float(np.float32(np.float32(0.6) * 32)), float(np.float32(np.float32(0.45) * 32)))]
    t = [(float(np.float32(0.3)), float(np.float32(0.2))), (float(np.float32(0.25)), float(np.float32(0.35)))]
    for (x, y), v in zip(pts, got):
        q1 = ((x - m[0][0]) * t[0][0]) ** 2 + ((y - m[0][1]) * t[0][1]) ** 2
        q2 = ((x - m[1][0]) * t[1][0]) ** 2 + ((y - m[1][1]) * t[1][1]) ** 2
        want = 1.0 / (1.0 + math.exp(0.5 * (q1 - q2)))
        assert abs(v - want) < 1e-13


def test_equal_colours_render_that_colour_and_blend_is_linear_in_colour():
    H, W = 48, 48
    g = rand_set(60, 2, 3)
    g.color[:] = np.float32([0.25, -0.75])
    img = O.render_image(g, H, W)
    covered = np.abs(img).sum(axis=0) > 0
    assert covered.mean() > 0.5
    np.testing.assert_allclose(img[0][covered], 0.25, atol=1e-13)
    np.testing.assert_allclose(img[1][covered], -0.75, atol=1e-13)
    ga, gb = rand_set(60, 2, 4), rand_set(60, 2, 4)
    gb.color = np.random.default_rng(9).uniform(-1, 1, gb.color.shape).astype(np.float32)
    gs = rand_set(60, 2, 4)
    gs.color = (ga.color.astype(np.float64) + gb.color).astype(np.float32)
    exact = (gs.color.astype(np.float64) == ga.color.astype(np.float64) + gb.color).all()
    if exact:
        np.testing.assert_allclose(O.render_image(gs, H, W),
                                   O.render_image(ga, H, W) + O.render_image(gb, H, W), atol=1e-12)


def test_normalised_weights_sum_to_one_and_match_unshifted_eq5():
    H, W = 32, 32
    g = rand_set(40, 3, 5, s_range=(2.0, 8.0))
    pts = O.pixel_centres(synth.sample_pixels(200, H, W, 0))
    for x, y in pts:
        tx, ty = int(x // 16), int(y // 16)
        out, aux = O._points_in_tile(g, np.array([[x, y]]), tx, ty, 16, H, W, 10, True, True)
        if aux["sel"].shape[1] == 0:
            continue
        w = aux["w"][0] / aux["Z"][0]
        assert abs(w.sum() - 1.0) < 1e-15
        G = np.exp(-0.5 * aux["q64"][0])
        if G.sum() > 1e-200:
            direct = (G[:, None] * g.color.astype(np.float64)[aux["sel"][0]]).sum(0) / G.sum()
            np.testing.assert_allclose(out[0], direct, rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- invariances

def test_rotation_by_pi_and_axis_swap_invariances():
    """theta -> theta + pi and (s1, s2, theta) -> (s2, s1, theta + pi/2) leave Sigma unchanged."""
    H, W = 48, 40
    g = rand_set(50, 3, 6)
    g.theta = (g.theta.astype(np.float64) * 0.5).astype(np.float32)   # keep theta + pi/2 < pi
    base = O.render_image(g, H, W, K=None)
    gp = rand_set(50, 3, 6)
    gp.theta = (g.theta.astype(np.float64) + np.pi).astype(np.float32)
    np.testing.assert_allclose(O.render_image(gp, H, W, K=None), base, atol=2e-5)
    gs = rand_set(50, 3, 6)
    gs.theta = (g.theta.astype(np.float64) + np.pi / 2).astype(np.float32)
    gs.inv_scale = g.inv_scale[:, ::-1].copy()
    np.testing.assert_allclose(O.render_image(gs, H, W, K=None), base, atol=2e-5)


def test_order_invariance_under_permutation():
    """The blend does not depend on the order in which Gaussians are given (Sec. 3.2)."""
    H, W = 48, 48
    g = rand_set(120, 3, 7)
    perm = np.random.default_rng(0).permutation(g.N)
    gp = O.Gaussians(g.xy[perm], g.theta[perm], g.inv_scale[perm], g.color[perm])
    np.testing.assert_allclose(O.render_image(gp, H, W), O.render_image(g, H, W), atol=1e-12)


# ---------------------------------------------------------------- top-K selection

def test_topk_selection_matches_python_sorted_brute_force():
    H, W = 40, 40
    g = rand_set(150, 1, 8)
    mx, my = O.means_px32(g, H, W)
    A00, B, A11 = O.conic32(g)
    pts = O.pixel_centres(synth.sample_pixels(150, H, W, 1))
    for K in (1, 3, 10):
        sel = O.selection(g, pts, H, W, K=K)
        for (x, y), s in zip(pts, sel):
            tx, ty = int(x // 16), int(y // 16)
            mem = np.nonzero(O.tile_members(g, tx, ty, 16, H, W))[0]
            keys = [(float(O.rank_key32(np.float32(x), np.float32(y), mx[i], my[i],
                                        A00[i], B[i], A11[i])), int(i)) for i in mem]
            want = [i for _, i in sorted(keys)[:K]]
            assert list(s) == want


def test_k_larger_than_hit_set_is_plain_normalised_sum_and_k1_is_nearest():
    H, W = 32, 48
    g = rand_set(80, 2, 9)
    pts = O.pixel_centres(synth.sample_pixels(120, H, W, 2))
    allK = O.render_points(g, pts, H, W, K=None)
    bigK = O.render_points(g, pts, H, W, K=10_000)
    np.testing.assert_array_equal(allK, bigK)
    k1 = O.render_points(g, pts, H, W, K=1)
    for (x, y), row, rowall in zip(pts, k1, allK):
        tx, ty = int(x // 16), int(y // 16)
        mem = np.nonzero(O.tile_members(g, tx, ty, 16, H, W))[0]
        if mem.size == 0:
            assert not row.any() and not rowall.any()
            continue
        # independent float64 Mahalanobis distances and plain normalised sum
        q = []
        for i in mem:
            th = float(g.theta[i])
            u = np.array([math.cos(th), math.sin(th)])
            v = np.array([-math.sin(th), math.cos(th)])
            d = np.array([x - float(np.float32(g.xy[i, 0] * np.float32(W))),
                          y - float(np.float32(g.xy[i, 1] * np.float32(H)))])
            q.append((float(g.inv_scale[i, 0]) * (u @ d)) ** 2 + (float(g.inv_scale[i, 1]) * (v @ d)) ** 2)
        q = np.array(q)
        np.testing.assert_array_equal(row, g.color[mem[np.argmin(q)]].astype(np.float64))
        w = np.exp(-0.5 * (q - q.min()))
        np.testing.assert_allclose(rowall, (w[:, None] * g.color[mem]).sum(0) / w.sum(),
                                   rtol=1e-12, atol=1e-13)


def test_empty_tiles_render_zero():
    H, W = 64, 64
    g = make([[0.1, 0.1]], [0.0], [[2.0, 2.0]], [[1.0]])          # r = 1.5 px
    img = O.render_image(g, H, W)
    assert img[0, :16, :16].min() == 1.0
    assert not img[0, 16:, :].any() and not img[0, :, 16:].any()


def test_ties_go_to_smaller_index():
    H, W = 16, 16
    # Two identical-shape Gaussians mirrored about the pixel (8.5, 8.5): equal q there.
    g = make([[4.5 / 16, 8.5 / 16], [12.5 / 16, 8.5 / 16], [8.5 / 16, 2.5 / 16]],
             [0.0, 0.0, 0.0], [[0.5, 0.5], [0.5, 0.5], [0.5, 0.5]], [[1.0], [2.0], [3.0]])
    sel = O.selection(g, [[8.5, 8.5]], H, W, K=1)[0]
    assert list(sel) == [0]
    g2 = make(g.xy[[1, 0, 2]], g.theta[[1, 0, 2]], g.inv_scale[[1, 0, 2]], g.color[[1, 0, 2]])
    assert list(O.selection(g2, [[8.5, 8.5]], H, W, K=1)[0]) == [0]
    # The selected colour follows the index, so it changes with the order.
    assert O.render_points(g, [[8.5, 8.5]], H, W, K=1)[0, 0] == 1.0
    assert O.render_points(g2, [[8.5, 8.5]], H, W, K=1)[0, 0] == 2.0


# ---------------------------------------------------------------- binning predicate

def _dense_min_distance(mx, my, X0, X1, Y0, Y1, steps=400):
    xs = np.linspace(X0, X1, steps)
    ys = np.linspace(Y0, Y1, steps)
    border = np.concatenate([
        np.stack([xs, np.full_like(xs, Y0)], 1), np.stack([xs, np.full_like(xs, Y1)], 1),
        np.stack([np.full_like(ys, X0), ys], 1), np.stack([np.full_like(ys, X1), ys], 1)])
    inside = X0 <= mx <= X1 and Y0 <= my <= Y1
    return 0.0 if inside else np.min(np.hypot(border[:, 0] - mx, border[:, 1] - my))


def test_tile_membership_matches_dense_sampled_distance_away_from_the_boundary():
    H, W, T = 80, 72, 16
    g = rand_set(300, 1, 10, s_range=(0.3, 6.0))
    mx, my = O.means_px32(g, H, W)
    r = 3.0 / np.minimum(g.inv_scale[:, 0], g.inv_scale[:, 1]).astype(np.float64)
    checked = 0
    for ty in range(-(-H // T)):
        for tx in range(-(-W // T)):
            mask = O.tile_members(g, tx, ty, T, H, W)
            X0, X1, Y0, Y1 = tx * T, min((tx + 1) * T, W), ty * T, min((ty + 1) * T, H)
            for i in range(0, g.N, 7):
                dist = _dense_min_distance(float(mx[i]), float(my[i]), X0, X1, Y0, Y1)
                step = 2.0 * max(X1 - X0, Y1 - Y0) / 400
                if abs(dist - r[i]) > step:
                    assert bool(mask[i]) == (dist <= r[i])
                    checked += 1
    assert checked > 1000


def test_tile_membership_hand_built_cases():
    H, W, T = 64, 64, 16
    # circle exactly tangent to the right edge x = 32 of tile (1, 1): t = 1 => r = 3
    g = make([[35.0 / 64, 24.0 / 64]], [0.0], [[1.0, 1.0]], [[1.0]])
    assert O.tile_members(g, 1, 1, T, H, W)[0]          # distance 3 == r: inclusive
    assert not O.tile_members(g, 0, 1, T, H, W)[0]
    g = make([[np.nextafter(np.float32(35.0 / 64), np.float32(1)), 24.0 / 64]], [0.0],
             [[1.0, 1.0]], [[1.0]])
    assert not O.tile_members(g, 1, 1, T, H, W)[0]      # a hair farther: excluded
    # centre outside the image still touches the border tiles it reaches
    g = make([[-0.05, 0.5]], [0.0], [[0.5, 0.5]], [[1.0]])   # mx = -3.2, r = 6
    assert O.tile_members(g, 0, 2, T, H, W)[0] and not O.tile_members(g, 1, 2, T, H, W)[0]
    # a huge radius covers every tile
    g = make([[0.5, 0.5]], [0.3], [[1e-3, 1e-3]], [[1.0]])
    assert all(O.tile_members(g, tx, ty, T, H, W)[0] for tx in range(4) for ty in range(4))
    # ragged last tile is clipped to the image: the rect ends at W = 40, not 48
    g = make([[42.5 / 40, 8.0 / 40]], [0.0], [[1.0, 1.0]], [[1.0]])  # mx = 42.5, r = 3
    assert O.tile_members(g, 2, 0, T, 40, 40)[0]
    g = make([[43.5 / 40, 8.0 / 40]], [0.0], [[1.0, 1.0]], [[1.0]])  # 3.5 past the clip
    assert not O.tile_members(g, 2, 0, T, 40, 40)[0]


def test_count_evals_equals_brute_force_pixel_sum():
    H, W = 40, 56
    g = rand_set(70, 1, 11)
    total = 0
    for h in range(H):
        for w in range(W):
            total += int(O.tile_members(g, w // 16, h // 16, 16, H, W).sum())
    assert O.count_evals(g, H, W) == total


# ---------------------------------------------------------------- gradients

def _fd_check(n, seed, K=3, normalize=True):
    H, W, T = 24, 24, 8
    g = rand_set(12, n, seed, s_range=(1.5, 6.0))
    rng = np.random.default_rng(seed)
    gout = rng.standard_normal((n, H, W))
    grad = O.backward_image(g, gout, H, W, K=K, tile=T, normalize=normalize)
    P0 = g.packed().astype(np.float64)
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    pix = np.stack([hh.ravel(), ww.ravel()], 1)
    pts = O.pixel_centres(pix)
    lists0 = O.tile_lists(g, H, W, T)
    sel0 = O.selection(g, pts, H, W, K=K, tile=T)

    def loss_at(P):
        gg = O.Gaussians.from_packed(P)
        if any(not np.array_equal(a, b) for a, b in zip(O.tile_lists(gg, H, W, T), lists0)):
            return None
        sel = O.selection(gg, pts, H, W, K=K, tile=T)
        if any(not np.array_equal(a, b) for a, b in zip(sel, sel0)):
            return None
        img = O.render_image(gg, H, W, K=K, tile=T, normalize=normalize)
        return float((img * gout).sum())

    checked = 0
    for i in range(g.N):
        for col in range(5 + n):
            base = float(P0[i, col])
            h = 1e-3 * max(abs(base), 1e-2) if col >= 5 else 2e-3 * max(abs(base), 1e-2)
            Pp, Pm = P0.copy(), P0.copy()
            Pp[i, col] = base + h
            Pm[i, col] = base - h
            # the oracle evaluates binary32 inputs: use the exactly representable step
            hp = float(np.float32(base + h)) - base
            hm = base - float(np.float32(base - h))
            lp, lm = loss_at(Pp.astype(np.float32)), loss_at(Pm.astype(np.float32))
            if lp is None or lm is None or hp <= 0 or hm <= 0:
                continue
            fd = (lp - lm) / (hp + hm)
            scale = max(np.abs(grad[:, col]).max(), 1e-12)
            assert abs(fd - grad[i, col]) <= 2e-3 * scale + 1e-9, (i, col, fd, grad[i, col])
            checked += 1
    return checked


@pytest.mark.parametrize("n,seed", [(1, 20), (3, 21)])
def test_gradients_match_central_finite_differences(n, seed):
    assert _fd_check(n, seed) > 5 * (5 + n)


@pytest.mark.parametrize("K,normalize", [(None, True), (3, False), (None, False)])
def test_ablation_mode_gradients_match_finite_differences(K, normalize):
    """All of S_j (K = infinity) and/or no normalisation (Eq. 4 over S_j)."""
    assert _fd_check(3, 23, K=K, normalize=normalize) > 3 * 8


def test_unnormalised_all_candidates_is_eq4_restricted_to_the_tile():
    """K = infinity without normalisation is Eq. 4 summed over S_j only."""
    H, W = 40, 40
    g = rand_set(30, 2, 24, s_range=(1.0, 4.0))
    pts = O.pixel_centres(synth.sample_pixels(100, H, W, 3))
    got = O.render_points(g, pts, H, W, K=None, normalize=False)
    for (x, y), row in zip(pts, got):
        mem = O.tile_members(g, int(x // 16), int(y // 16), 16, H, W)
        want = np.zeros(2)
        for i in np.nonzero(mem)[0]:
            th = float(g.theta[i])
            u = np.array([math.cos(th), math.sin(th)])
            v = np.array([-math.sin(th), math.cos(th)])
            d = np.array([x - float(np.float32(g.xy[i, 0] * np.float32(W))),
                          y - float(np.float32(g.xy[i, 1] * np.float32(H)))])
            q = (float(g.inv_scale[i, 0]) * (u @ d)) ** 2 + (float(g.inv_scale[i, 1]) * (v @ d)) ** 2
            want += math.exp(-0.5 * q) * g.color[i].astype(np.float64)
        np.testing.assert_allclose(row, want, rtol=1e-12, atol=1e-14)


def test_colour_gradient_is_exact_weight_sum():
    H, W = 32, 32
    g = rand_set(30, 1, 22)
    gout = np.ones((1, H, W))
    grad = O.backward_image(g, gout, H, W)
    # dL/dc_i = sum over pixels of w_i/Z (selection fixed); total weight is 1 per covered pixel
    img_cov = O.render_image(O.Gaussians(g.xy, g.theta, g.inv_scale, np.ones((g.N, 1))), H, W)
    assert abs(grad[:, 5].sum() - img_cov.sum()) < 1e-9


# ---------------------------------------------------------------- loss and Adam

def test_l1_matches_torch_autograd_including_sign_zero():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, (3, 5, 7))
    b = rng.uniform(0, 1, (3, 5, 7))
    b[0, 0, :3] = a[0, 0, :3]
    loss, grad = O.l1_loss(a, b)
    ta = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tl = torch.nn.functional.l1_loss(ta, torch.tensor(b, dtype=torch.float64))
    tl.backward()
    assert abs(loss - tl.item()) < 1e-15
    np.testing.assert_allclose(grad, ta.grad.numpy(), atol=1e-18)
    assert (grad[0, 0, :3] == 0).all()


def test_adam_matches_torch_optim_adam_then_clamps():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    N, n = 50, 3
    P = synth.packed(synth.gaussians(N, n, 5)).astype(np.float64)
    tP = [torch.tensor(P[:, 0:2].copy(), requires_grad=True),
          torch.tensor(P[:, 2:3].copy(), requires_grad=True),
          torch.tensor(P[:, 3:5].copy(), requires_grad=True),
          torch.tensor(P[:, 5:].copy(), requires_grad=True)]
    opt = torch.optim.Adam([dict(params=[tP[0]], lr=5e-4), dict(params=[tP[1]], lr=2e-3),
                            dict(params=[tP[2]], lr=2e-3), dict(params=[tP[3]], lr=5e-3)],
                           betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    big = dict(theta=(-1e9, 1e9), inv_scale=(-1e9, 1e9), mu=(-1e9, 1e9))
    for step in range(1, 6):
        G = rng.standard_normal(P.shape)
        for t, sl in zip(tP, [slice(0, 2), slice(2, 3), slice(3, 5), slice(5, None)]):
            t.grad = torch.tensor(G[:, sl].copy())
        opt.step()
        P, m, v = O.adam_update(P, G, m, v, step, bounds=big)
        got = np.concatenate([t.detach().numpy() for t in tP], axis=1)
        np.testing.assert_allclose(P, got, rtol=1e-12, atol=1e-14)
    # clamps: theta to [0, pi], t to [1e-3, 10], mu to [0, 1]
    Q = P.copy()
    Q[0, 2], Q[1, 2], Q[2, 3], Q[3, 4], Q[4, 0], Q[5, 1] = -0.1, 4.0, 1e-5, 50.0, -0.2, 1.3
    Q2, _, _ = O.adam_update(Q, np.zeros_like(Q), np.zeros_like(Q), np.zeros_like(Q), 1)
    assert Q2[0, 2] == 0.0 and Q2[1, 2] == np.pi and Q2[2, 3] == 1e-3 and Q2[3, 4] == 10.0
    assert Q2[4, 0] == 0.0 and Q2[5, 1] == 1.0
