"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: tile lists and top-K selections are integer results and must be
identical; pixels within 1e-5 max abs (FP32 path); gradients within 1e-3
normwise relative error per parameter group.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import image_gs as O  # noqa: E402
from paper_2407_01866_b300 import lib as L  # noqa: E402
from paper_2407_01866_b300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_harness import GpuSet, grad_elem_rel_error, grad_rel_error  # noqa: E402

PIX_TOL = 1e-5
GRAD_TOL = 1e-3


def oset(N, n, seed, s_range=(0.5, 8.0)):
    d = synth.gaussians(N, n, seed, s_range=s_range)
    return O.Gaussians(d["xy"], d["theta"], d["inv_scale"], d["color"])


CASES = [
    # (H, W, N, n, K, tile, seed, s_range)
    (256, 256, 4096, 3, 10, 16, 0, (0.5, 8.0)),     # the 256^2 RGB workload
    (37, 53, 300, 1, 3, 8, 1, (0.5, 8.0)),          # ragged tiles, 8x8 tiles
    (70, 45, 400, 4, 16, 16, 2, (0.5, 6.0)),
    (48, 64, 250, 9, 10, 16, 3, (0.5, 8.0)),
    (40, 40, 200, 5, 4, 8, 4, (0.5, 8.0)),          # generic channel count
    (64, 64, 1500, 2, 8, 16, 5, (8.0, 30.0)),       # |S_j| > shared-memory slots
    (33, 17, 60, 3, 1, 16, 6, (0.5, 8.0)),
    (16, 16, 1, 3, 10, 16, 7, (0.5, 8.0)),          # single Gaussian
    (1, 1, 5, 3, 2, 8, 8, (0.5, 8.0)),              # one pixel
    (32, 32, 9000, 1, 4, 16, 9, (12.0, 40.0)),      # lists > 4096: CTA sort with merges
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_N{c[2]}_n{c[3]}_K{c[4]}_t{c[5]}")
def test_tile_lists_equal_oracle_sets(case):
    H, W, N, n, K, tile, seed, sr = case
    g = oset(N, n, seed, sr)
    gs = GpuSet(g, H, W, K, tile)
    want = O.tile_lists(g, H, W, tile)
    got = gs.tile_lists()
    assert len(got) == len(want)
    for j, (a, b) in enumerate(zip(got, want)):
        # lists up to tile*tile entries come in no set order; longer ones ascending
        np.testing.assert_array_equal(a if len(a) > tile * tile else np.sort(a), b,
                                      err_msg=f"tile {j}")
    assert gs.stats.m_needed == sum(len(w) for w in want)
    assert gs.stats.evals == O.count_evals(g, H, W, tile)
    assert gs.stats.flags == 0


# Gaussians whose tile box exceeds 64 tiles are binned by a separate pass:
# tile blocks testing every such Gaussian (several rounds of 256 here), and
# beyond 16384 of them one CTA per Gaussian
WIDE_CASES = [
    (512, 512, 3000, 1, 16, 21, (10.0, 20.0)),
    (384, 320, 20000, 1, 16, 22, (20.0, 40.0)),
]


@pytest.mark.parametrize("case", WIDE_CASES, ids=lambda c: f"{c[0]}x{c[1]}_N{c[2]}")
def test_tile_lists_with_many_wide_gaussians(case):
    H, W, N, n, tile, seed, sr = case
    g = oset(N, n, seed, sr)
    want = O.tile_lists(g, H, W, tile)
    M = sum(len(w) for w in want)
    gs = GpuSet(g, H, W, 4, tile, m_capacity=M + 1024)
    got = gs.tile_lists()
    for j, (a, b) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(a if len(a) > tile * tile else np.sort(a), b,
                                      err_msg=f"tile {j}")
    assert gs.stats.m_needed == M
    assert gs.stats.flags == 0


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_N{c[2]}_n{c[3]}_K{c[4]}_t{c[5]}")
def test_forward_matches_oracle(case):
    H, W, N, n, K, tile, seed, sr = case
    g = oset(N, n, seed, sr)
    gs = GpuSet(g, H, W, K, tile)
    got = gs.forward()
    want = O.render_image(g, H, W, K=K, tile=tile)
    err = np.abs(got - want).max()
    print(f"forward {H}x{W} N={N} n={n} K={K} tile={tile}: max |pixel - oracle| {err:.2e}")
    assert err <= PIX_TOL, err


@pytest.mark.parametrize("case", CASES[:7], ids=lambda c: f"{c[0]}x{c[1]}_N{c[2]}_n{c[3]}_K{c[4]}_t{c[5]}")
def test_backward_with_upstream_gradient_matches_oracle(case):
    H, W, N, n, K, tile, seed, sr = case
    g = oset(N, n, seed, sr)
    gs = GpuSet(g, H, W, K, tile)
    gimg = np.random.default_rng(seed + 100).standard_normal((n, H, W)).astype(np.float32)
    got, _ = gs.backward(grad_img=gimg)
    want = O.backward_image(g, gimg, H, W, K=K, tile=tile)
    errs = grad_rel_error(got, want)
    assert max(errs.values()) <= GRAD_TOL, errs


def _unambiguous_target(g, H, W, K, tile, seed, margin=1e-4):
    """Synthetic target moved away from the oracle's image wherever |c_r - c_t|
    is within `margin`, so that sign(c_r - c_t) has one correct value."""
    t = synth.target_image(H, W, g.n, seed=seed).astype(np.float64)
    img = O.render_image(g, H, W, K=K, tile=tile)
    close = np.abs(img - t) < margin
    t[close] = img[close] + np.where(t[close] >= img[close], margin, -margin)
    t = t.astype(np.float32)
    assert np.abs(img - t.astype(np.float64)).min() >= margin * 0.5
    return t, img


# three small Gaussians leave most tiles empty: their pixels render 0 and
# still count in the mean L1 loss
UNCOVERED = (64, 64, 3, 3, 10, 16, 11, (0.5, 2.0))


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3], CASES[5], UNCOVERED],
                         ids=lambda c: f"{c[0]}x{c[1]}_N{c[2]}_n{c[3]}")
def test_fused_l1_loss_and_gradient_match_oracle(case):
    H, W, N, n, K, tile, seed, sr = case
    g = oset(N, n, seed, sr)
    target, img = _unambiguous_target(g, H, W, K, tile, seed)
    gs = GpuSet(g, H, W, K, tile)
    got, st = gs.backward(target=target)
    loss, dimg = O.l1_loss(img, target)
    want = O.backward_image(g, dimg, H, W, K=K, tile=tile)
    assert abs(st.loss_sum / (H * W * n) - loss) <= 1e-6
    errs = grad_rel_error(got, want)
    print(f"fused L1 {H}x{W} N={N} n={n}: loss {st.loss_sum / (H * W * n):.8f} vs {loss:.8f}, "
          f"gradient normwise {max(errs.values()):.2e}, per element "
          f"{max(grad_elem_rel_error(got, want).values()):.2e}")
    assert max(errs.values()) <= GRAD_TOL, errs


def test_decode_random_points_match_oracle():
    H, W, N, n = 256, 256, 4096, 3
    g = oset(N, n, 0)
    gs = GpuSet(g, H, W)
    pts = synth.query_points(5000, H, W, seed=3)
    pts = np.concatenate([pts, O.pixel_centres(synth.sample_pixels(500, H, W, 4)).astype(np.float32),
                          np.array([[0, 0], [W - 1e-3, H - 1e-3], [W - 1e-3, 0]], np.float32)])
    got = gs.decode(pts)
    want = O.render_points(g, pts.astype(np.float64), H, W)
    assert np.abs(got - want).max() <= PIX_TOL
    # decoding a pixel centre gives the rendered pixel (same winners; the
    # two kernels only sum the K terms in a different order)
    img = gs.forward()
    pix = synth.sample_pixels(300, H, W, 5)
    cen = O.pixel_centres(pix).astype(np.float32)
    np.testing.assert_allclose(gs.decode(cen), img[:, pix[:, 0], pix[:, 1]].T, rtol=0, atol=1e-6)


@pytest.mark.parametrize("dt", ["float16", "bfloat16"])
def test_half_precision_storage_forward_and_decode(dt):
    H, W, N, n = 128, 160, 2000, 3
    d = synth.gaussians(N, n, 11)
    tdt = getattr(torch, dt)
    # the oracle evaluates the exact upcast of the stored half values
    half = {k: torch.from_numpy(v).to(tdt).float().numpy() for k, v in d.items()}
    g = O.Gaussians(half["xy"], half["theta"], half["inv_scale"], half["color"])
    gs = GpuSet(g, H, W, dtype=tdt)
    got = gs.forward()
    want = O.render_image(g, H, W)
    err = np.abs(got - want).max()
    assert err <= 2e-3 and err <= PIX_TOL, err
    pts = synth.query_points(2000, H, W, seed=1)
    assert np.abs(gs.decode(pts) - O.render_points(g, pts.astype(np.float64), H, W)).max() <= PIX_TOL


def test_empty_set_and_empty_tiles_render_zero():
    g = O.Gaussians(np.zeros((0, 2)), np.zeros(0), np.zeros((0, 2)), np.zeros((0, 3)))
    gs = GpuSet(g, 40, 24)
    assert not gs.forward().any()
    assert gs.stats.m_needed == 0
    g1 = O.Gaussians([[0.1, 0.1]], [0.0], [[2.0, 2.0]], [[1.0, 2.0, 3.0]])
    gs1 = GpuSet(g1, 64, 64)
    img = gs1.forward()
    np.testing.assert_array_equal(img[:, 16:, :], 0)
    np.testing.assert_array_equal(img[:, :16, :16], np.broadcast_to(np.array([1.0, 2.0, 3.0])[:, None, None], (3, 16, 16)))


def test_capacity_overflow_is_flagged_and_recovered():
    H, W, N, n = 128, 128, 2000, 3
    g = oset(N, n, 12)
    gs = GpuSet(g, H, W, m_capacity=64)            # grows after the first binning
    assert gs.binner.m_capacity > 64
    np.testing.assert_allclose(gs.forward(), O.render_image(g, H, W), atol=PIX_TOL)
    v = gs.view
    small = L.preprocess_bin(v, H, W, gs.cfg, L.alloc_workspace(
        L.workspace_size(N, n, H, W, gs.cfg, 64)), 64)
    st = L.read_stats(small)
    assert st.flags & L.FLAG_CAPACITY and st.m_needed == gs.stats.m_needed


def test_nonfinite_parameters_are_flagged_and_skipped():
    H, W = 48, 48
    g = oset(50, 3, 13)
    g.inv_scale[3, 0] = -1.0
    g.xy[7, 1] = np.nan
    gs = GpuSet(g, H, W)
    assert gs.stats.flags & L.FLAG_NONFINITE
    lists = gs.tile_lists()
    assert all(3 not in l and 7 not in l for l in lists)
    keep = np.setdiff1d(np.arange(50), [3, 7])
    gk = O.Gaussians(g.xy[keep], g.theta[keep], g.inv_scale[keep], g.color[keep])
    want = O.render_image(gk, H, W)
    np.testing.assert_allclose(gs.forward(), want, atol=PIX_TOL)


ABLATION = [
    # (H, W, N, n, K, tile, normalize, seed)  K = 0: all of S_j
    (64, 48, 300, 3, 0, 16, 1, 30),
    (64, 48, 300, 3, 3, 16, 0, 31),
    (40, 56, 200, 1, 0, 8, 0, 32),
    (64, 64, 1200, 3, 0, 16, 1, 33),   # lists > 128 and > 256: staged chunks
]


@pytest.mark.parametrize("case", ABLATION, ids=lambda c: f"K{c[4]}_norm{c[6]}_t{c[5]}_N{c[2]}")
def test_ablation_modes_forward_adjoint_decode(case):
    """Table 1 ablations: all of S_j (K = 0) and/or no normalisation."""
    H, W, N, n, K, tile, norm, seed = case
    g = oset(N, n, seed, (1.0, 12.0) if N > 1000 else (0.5, 8.0))
    Ko = None if K == 0 else K
    gs = GpuSet(g, H, W, K, tile, normalize=norm)
    want = O.render_image(g, H, W, K=Ko, tile=tile, normalize=bool(norm))
    got = gs.forward()
    scale = max(1.0, np.abs(want).max())
    assert np.abs(got - want).max() <= PIX_TOL * scale
    gimg = np.random.default_rng(seed).standard_normal((n, H, W)).astype(np.float32)
    grad, _ = gs.backward(grad_img=gimg)
    ref = O.backward_image(g, gimg, H, W, K=Ko, tile=tile, normalize=bool(norm))
    errs = grad_rel_error(grad, ref)
    assert max(errs.values()) <= GRAD_TOL, errs
    pts = synth.query_points(500, H, W, seed=seed)
    dec = O.render_points(g, pts.astype(np.float64), H, W, K=Ko, tile=tile, normalize=bool(norm))
    assert np.abs(gs.decode(pts) - dec).max() <= PIX_TOL * scale


def dup_set(M, copies, n, seed, s_range=(0.5, 8.0)):
    """M Gaussians, each present `copies` times at scattered indices: equal
    parameters give bit-equal keys, so top-K boundaries fall inside groups of
    equal keys and the index order must decide (Sec. 3.2 ranking, ties to the
    smaller index)."""
    d = synth.gaussians(M, n, seed, s_range=s_range)
    idx = np.random.default_rng(seed + 50).permutation(np.repeat(np.arange(M), copies))
    return O.Gaussians(d["xy"][idx], d["theta"][idx], d["inv_scale"][idx], d["color"][idx])


def boundary_ties(g, H, W, K, tile):
    """Pixels whose K-th and (K+1)-th smallest keys are equal."""
    mx, my = O.means_px32(g, H, W)
    A00, B, A11 = O.conic32(g)
    count = 0
    for ty in range(-(-H // tile)):
        for tx in range(-(-W // tile)):
            mem = np.nonzero(O.tile_members(g, tx, ty, tile, H, W))[0]
            if len(mem) <= K:
                continue
            hh, ww = np.meshgrid(np.arange(ty * tile, min(H, ty * tile + tile)),
                                 np.arange(tx * tile, min(W, tx * tile + tile)), indexing="ij")
            px = (ww.ravel() + 0.5).astype(np.float32)[:, None]
            py = (hh.ravel() + 0.5).astype(np.float32)[:, None]
            q = np.sort(O.rank_key32(px, py, mx[mem][None], my[mem][None], A00[mem][None],
                                     B[mem][None], A11[mem][None]), axis=1)
            count += int((q[:, K - 1] == q[:, K]).sum())
    return count


TIES = [
    # (H, W, M, copies, n, K, tile, seed, s_range)
    (48, 40, 60, 3, 3, 4, 16, 11, (0.5, 8.0)),     # one-stage lists
    (32, 32, 40, 4, 1, 10, 8, 12, (0.5, 8.0)),     # 8x8 tiles
    (16, 16, 100, 3, 3, 10, 16, 13, (2.0, 20.0)),  # one tile of 300: chunked passes
]


@pytest.mark.parametrize("case", TIES, ids=lambda c: f"{c[0]}x{c[1]}_M{c[2]}x{c[3]}_K{c[5]}_t{c[6]}")
def test_equal_keys_at_the_kth_place_go_to_smaller_indices(case):
    H, W, M, copies, n, K, tile, seed, sr = case
    g = dup_set(M, copies, n, seed, sr)
    assert boundary_ties(g, H, W, K, tile) > 0
    gs = GpuSet(g, H, W, K, tile)
    assert np.abs(gs.forward() - O.render_image(g, H, W, K=K, tile=tile)).max() <= PIX_TOL
    gimg = np.random.default_rng(seed + 100).standard_normal((n, H, W)).astype(np.float32)
    got, _ = gs.backward(grad_img=gimg)
    want = O.backward_image(g, gimg, H, W, K=K, tile=tile)
    errs = grad_rel_error(got, want)
    assert max(errs.values()) <= GRAD_TOL, errs
    pix = np.stack(np.meshgrid(np.arange(H), np.arange(W), indexing="ij"), -1).reshape(-1, 2)
    cen = O.pixel_centres(pix)
    dec = gs.decode(cen.astype(np.float32))
    assert np.abs(dec - O.render_points(g, cen, H, W, K=K, tile=tile)).max() <= PIX_TOL


def test_autograd_render_matches_oracle_forward_and_adjoint():
    """lib.render is a torch.autograd.Function over the C ABI: its output is
    the forward render and its backward the adjoint of the upstream gradient."""
    H, W, N, n = 48, 40, 250, 3
    g = oset(N, n, 21)
    ts = [torch.from_numpy(a.copy()).cuda().requires_grad_(True)
          for a in (g.xy, g.theta, g.inv_scale, g.color)]
    img = L.render(*ts, H, W)
    np.testing.assert_allclose(img.detach().cpu().numpy(), O.render_image(g, H, W),
                               rtol=0, atol=PIX_TOL)
    weight = np.random.default_rng(22).standard_normal((n, H, W)).astype(np.float32)
    (img * torch.from_numpy(weight).cuda()).sum().backward()
    got = np.concatenate([ts[0].grad.cpu().numpy(), ts[1].grad.cpu().numpy()[:, None],
                          ts[2].grad.cpu().numpy(), ts[3].grad.cpu().numpy()], axis=1)
    want = O.backward_image(g, weight, H, W)
    errs = grad_rel_error(got.astype(np.float64), want)
    assert max(errs.values()) <= GRAD_TOL, errs


def test_autograd_render_reuses_its_workspace_and_runs_unchecked():
    """Repeated renders of one shape reuse a cached workspace (no allocation
    per call); check=False renders with no host synchronisation, and two
    interleaved forwards of the same shape keep their own adjoints."""
    H, W, N, n = 48, 40, 250, 3
    sets = [oset(N, n, 30 + k) for k in range(2)]
    tss = [[torch.from_numpy(a.copy()).cuda().requires_grad_(True)
            for a in (g.xy, g.theta, g.inv_scale, g.color)] for g in sets]
    L.render(*tss[0], H, W)   # a checked call sizes the cached workspace
    before = len(L._BINNERS)
    imgs = [L.render(*ts, H, W, check=False) for ts in tss]
    assert len(L._BINNERS) == before
    weight = np.random.default_rng(23).standard_normal((n, H, W)).astype(np.float32)
    wt = torch.from_numpy(weight).cuda()
    for g, ts, img in zip(sets, tss, imgs):
        np.testing.assert_allclose(img.detach().cpu().numpy(), O.render_image(g, H, W),
                                   rtol=0, atol=PIX_TOL)
    (imgs[0] * wt).sum().backward()
    (imgs[1] * wt).sum().backward()
    for g, ts in zip(sets, tss):
        got = np.concatenate([ts[0].grad.cpu().numpy(), ts[1].grad.cpu().numpy()[:, None],
                              ts[2].grad.cpu().numpy(), ts[3].grad.cpu().numpy()], axis=1)
        errs = grad_rel_error(got.astype(np.float64), O.backward_image(g, weight, H, W))
        assert max(errs.values()) <= GRAD_TOL, errs
