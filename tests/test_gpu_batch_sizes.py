"""Batched form at the batch workload's sizes, against the oracle.

The batch has images with sides of 256-2048 pixels (one 2048 wide), about one
Gaussian per 28 pixels, and a cluster of large Gaussians in one image, so that
some tile lists run past 256 entries and every stage of the persistent
adjoint (64, 128, 256) takes its chunked path somewhere. The batched forward
(igs_render_forward_batch) is compared with the oracle on sampled pixels of
three images (random pixels plus the cluster's centre tile), and the batched
adjoint of an upstream gradient that is non-zero only at those pixels
(igs_render_backward_batch) with the oracle's gradient over those pixels,
for every stage. The batched fit step with the SSIM term is compared with
single-image steps and, for one image, with the oracle.
"""
import functools

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

PIX_TOL = 1e-5
GRAD_TOL = 1e-3
CHECKED = (0, 1, 2)


@functools.lru_cache(maxsize=1)
def batch():
    shapes = [(h, w) for h, w, _ in synth.batch_shapes(5, seed=21)]
    shapes[0] = (1200, 2048)
    shapes[1] = (512, 640)
    n = 3
    Ps, gs = [], []
    for b, (H, W) in enumerate(shapes):
        N = max(1, round(H * W / 28))
        d = synth.gaussians(N, n, seed=30 + b)
        if b == 1:   # a cluster of large Gaussians at the image centre
            rng = np.random.default_rng(7)
            k = 400
            d["xy"][-k:] = (0.5 + 0.01 * rng.standard_normal((k, 2))).astype(np.float32)
            d["inv_scale"][-k:] = (1.0 / rng.uniform(10.0, 30.0, (k, 2))).astype(np.float32)
        P = synth.packed(d)
        Ps.append(P)
        gs.append(O.Gaussians.from_packed(P))
    Hs = [h for h, _ in shapes]
    Ws = [w for _, w in shapes]
    Ns = [P.shape[0] for P in Ps]
    # pixels checked per image: random ones, plus image 1's centre tile
    pix = {}
    for b in CHECKED:
        p = synth.sample_pixels(160, Hs[b], Ws[b], seed=40 + b)
        if b == 1:
            ty, tx = Hs[1] // 32, Ws[1] // 32
            hh, ww = np.meshgrid(np.arange(16 * ty, 16 * ty + 16), np.arange(16 * tx, 16 * tx + 16),
                                 indexing="ij")
            p = np.unique(np.concatenate([p, np.stack([hh.ravel(), ww.ravel()], 1)]), axis=0)
        pix[b] = p
    rng = np.random.default_rng(5)
    up = {b: rng.standard_normal((len(pix[b]), n)) for b in CHECKED}
    want_img = {b: O.render_pixels(gs[b], pix[b], Hs[b], Ws[b]) for b in CHECKED}
    want_grad = {b: O.backward_pixels(gs[b], pix[b], up[b], Hs[b], Ws[b]) for b in CHECKED}
    longest = len(np.nonzero(O.tile_members(gs[1], Ws[1] // 32, Hs[1] // 32, 16, Hs[1], Ws[1]))[0])
    return dict(Hs=Hs, Ws=Ws, Ns=Ns, Ps=Ps, gs=gs, pix=pix, up=up, want_img=want_img,
                want_grad=want_grad, longest=longest, n=n)


def _offsets(Hs, Ws, n):
    off = [0]
    for H, W in zip(Hs, Ws):
        off.append(off[-1] + n * H * W)
    return off


def _setup(B, cfg):
    shape = L.batch_shape(B["Hs"], B["Ws"], B["Ns"], B["n"])
    cap = 24 * sum(B["Ns"]) + 4096
    ws = L.alloc_workspace(L.batch_workspace_size(shape, cfg, cap))
    L.batch_setup(shape, cfg, ws, cap)
    return shape, cap, ws


def test_batch_has_lists_longer_than_every_stage():
    assert batch()["longest"] > 256


def test_batched_forward_matches_oracle_at_batch_sizes():
    B = batch()
    cfg = L.default_config()
    shape, cap, ws = _setup(B, cfg)
    P = dev(np.concatenate(B["Ps"]))
    off = _offsets(B["Hs"], B["Ws"], B["n"])
    imgs = torch.full((off[-1],), float("nan"), device="cuda")
    L.render_forward_batch(P, shape, cfg, ws, cap, imgs)
    torch.cuda.synchronize()
    for b in CHECKED:
        H, W, n = B["Hs"][b], B["Ws"][b], B["n"]
        img = imgs[off[b]:off[b + 1]].view(n, H, W)
        pt = torch.from_numpy(B["pix"][b]).cuda()
        got = img[:, pt[:, 0], pt[:, 1]].T.cpu().numpy()
        err = np.abs(got - B["want_img"][b]).max()
        assert err <= PIX_TOL, (b, err)
    assert torch.isfinite(imgs).all()


@pytest.mark.parametrize("stage", [64, 128, 256])
def test_batched_adjoint_of_a_sparse_gradient_matches_oracle(stage):
    B = batch()
    cfg = L.default_config()
    shape, cap, ws = _setup(B, cfg)
    P = dev(np.concatenate(B["Ps"]))
    off = _offsets(B["Hs"], B["Ws"], B["n"])
    gimgs = torch.zeros((off[-1],), device="cuda")
    for b in CHECKED:
        H, W, n = B["Hs"][b], B["Ws"][b], B["n"]
        gi = gimgs[off[b]:off[b + 1]].view(n, H, W)
        pt = torch.from_numpy(B["pix"][b]).cuda()
        gi[:, pt[:, 0], pt[:, 1]] = torch.from_numpy(B["up"][b].T.astype(np.float32).copy()).cuda()
    grad = torch.full_like(P, float("nan"))
    L.render_backward_batch(P, gimgs, shape, cfg, ws, cap, grad,
                            tuning=L.BatchTuning(4, stage, stage == 128))
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    o = np.concatenate([[0], np.cumsum(B["Ns"])])
    for b in range(len(B["Ns"])):
        gb = g[o[b]:o[b + 1]]
        if b in CHECKED:
            errs = grad_rel_error(gb, B["want_grad"][b])
            assert max(errs.values()) <= GRAD_TOL, (b, stage, errs)
        else:   # no upstream gradient reaches this image
            assert not np.any(gb), b


def test_batched_ssim_step_matches_single_image_steps_and_oracle():
    shapes = [(40, 57), (100, 33), (64, 64), (17, 90), (96, 80)]
    n = 3
    Ps, Ts = [], []
    for b, (H, W) in enumerate(shapes):
        Ps.append(synth.packed(synth.gaussians(max(1, round(H * W / 28)), n, 50 + b)))
        Ts.append(synth.target_image(H, W, n, seed=60 + b))
    # image 0's target moved away from the oracle image where the L1 sign is ambiguous
    g0 = O.Gaussians.from_packed(Ps[0])
    img0 = O.render_image(g0, *shapes[0])
    t0 = Ts[0].astype(np.float64)
    close = np.abs(img0 - t0) < 1e-4
    t0[close] = img0[close] + np.where(t0[close] >= img0[close], 1e-4, -1e-4)
    Ts[0] = t0.astype(np.float32)
    Hs = [h for h, _ in shapes]
    Ws = [w for _, w in shapes]
    Ns = [P.shape[0] for P in Ps]
    cfg = L.default_config(ssim_weight=0.1)
    shape = L.batch_shape(Hs, Ws, Ns, n)
    cap = 16 * sum(Ns) + 1024
    ws = L.alloc_workspace(L.batch_workspace_size(shape, cfg, cap))
    assert ws.numel() > L.batch_workspace_size(shape, L.default_config(), cap)
    L.batch_setup(shape, cfg, ws, cap)
    P = dev(np.concatenate(Ps))
    G = torch.zeros_like(P)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.FitState(P.data_ptr(), G.data_ptr(), m.data_ptr(), v.data_ptr(), step.data_ptr(),
                    P.shape[0], n)
    loss = torch.zeros(len(shapes), device="cuda")
    L.fit_batch_step(st, dev(np.concatenate([t.ravel() for t in Ts])), shape, cfg, ws, cap,
                     loss_out=loss)
    torch.cuda.synchronize()
    gb = G.cpu().numpy().astype(np.float64)
    lb = loss.cpu().numpy()
    o = np.concatenate([[0], np.cumsum(Ns)])
    for b in range(len(shapes)):
        Pb = dev(Ps[b])
        Gb, mb, vb = torch.zeros_like(Pb), torch.zeros_like(Pb), torch.zeros_like(Pb)
        sb = torch.zeros(1, dtype=torch.int32, device="cuda")
        s1 = L.FitState(Pb.data_ptr(), Gb.data_ptr(), mb.data_ptr(), vb.data_ptr(),
                        sb.data_ptr(), Ns[b], n)
        w1 = L.alloc_workspace(L.workspace_size(Ns[b], n, Hs[b], Ws[b], cfg, 16 * Ns[b] + 64))
        l1 = torch.zeros(1, device="cuda")
        L.fit_step(s1, dev(Ts[b]), Hs[b], Ws[b], cfg, w1, 16 * Ns[b] + 64, l1)
        torch.cuda.synchronize()
        assert abs(l1.item() - lb[b]) <= 1e-6 * max(1.0, abs(lb[b])), b
        errs = grad_rel_error(gb[o[b]:o[b + 1]], Gb.cpu().numpy().astype(np.float64))
        assert max(errs.values()) <= 1e-4, (b, errs)
    want_loss, dimg = S.image_loss(img0, Ts[0].astype(np.float64), 0.1)
    assert abs(lb[0] - want_loss) <= 2e-6 * max(1.0, want_loss)
    ref = O.backward_image(g0, dimg, *shapes[0])
    errs = grad_rel_error(gb[o[0]:o[1]], ref)
    assert max(errs.values()) <= GRAD_TOL, errs
