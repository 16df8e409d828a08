"""Fit-step parity: Adam kernel, fused step, graph capture (through the C ABI)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import image_gs as O  # noqa: E402
from paper_2407_01866_b300 import lib as L  # noqa: E402
from paper_2407_01866_b300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_harness import dev, grad_rel_error  # noqa: E402


class State:
    def __init__(self, P):
        self.P = dev(P)
        self.G = torch.zeros_like(self.P)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.step = torch.zeros(1, dtype=torch.int32, device="cuda")
        N, np_ = P.shape
        self.c = L.FitState(self.P.data_ptr(), self.G.data_ptr(), self.m.data_ptr(),
                            self.v.data_ptr(), self.step.data_ptr(), N, np_ - 5)


def lr_of(cfg, ncol):
    r = np.empty(ncol)
    r[0:2], r[2], r[3:5], r[5:] = cfg.lr_mu, cfg.lr_theta, cfg.lr_inv_scale, cfg.lr_color
    return r


def test_adam_update_matches_oracle_adam():
    rng = np.random.default_rng(0)
    P = synth.packed(synth.gaussians(3000, 3, 1))
    cfg = L.default_config()
    st = State(P)
    Pr, mr, vr = P.astype(np.float64), np.zeros(P.shape), np.zeros(P.shape)
    m_err = np.zeros(P.shape)   # running bound of the float32 error in m
    u = 2.0 ** -24
    for k in range(1, 7):
        G = (rng.standard_normal(P.shape) * 10.0 ** rng.uniform(-6, 0, P.shape)).astype(np.float32)
        st.G.copy_(dev(G))
        st.step.fill_(k - 1)
        L.adam_update(st.c, cfg)
        m_prev = mr
        Pr, mr, vr = O.adam_update(Pr, G, mr, vr, k)
        got = st.P.cpu().numpy()
        # float32 state vs float64: the update itself is ~lr, its float32 error ~1e-6 relative
        tol = 2e-6 * np.abs(Pr) + 1e-6 * lr_of(cfg, P.shape[1])[None, :] + 1e-7
        assert (np.abs(got - Pr) <= tol).all(), np.abs(got - Pr).max()
        # m = b1 m + (1 - b1) g may cancel, and earlier rounding carries over:
        # e_k <= b1 e_{k-1} + 4u (b1 |m_{k-1}| + (1 - b1) |g_k| + |m_k|)
        m_err = 0.9 * m_err + 4 * u * (0.9 * np.abs(m_prev) + 0.1 * np.abs(G) + np.abs(mr))
        assert (np.abs(st.m.cpu().numpy() - mr) <= m_err + 1e-30).all()
        np.testing.assert_allclose(st.v.cpu().numpy(), vr, rtol=1e-5, atol=1e-18)
    # clamps
    Q = P.copy()
    Q[0, 2], Q[1, 2], Q[2, 3], Q[3, 4], Q[4, 0], Q[5, 1] = -0.5, 4.0, 1e-6, 50.0, -0.2, 1.3
    sq = State(Q)
    L.adam_update(sq.c, cfg)
    q = sq.P.cpu().numpy()
    assert q[0, 2] == 0.0 and q[1, 2] == np.float32(np.pi) and q[2, 3] == np.float32(1e-3)
    assert q[3, 4] == 10.0 and q[4, 0] == 0.0 and q[5, 1] == 1.0


def _unambiguous_target(g, H, W, seed, margin=1e-4):
    t = synth.target_image(H, W, g.n, seed=seed).astype(np.float64)
    img = O.render_image(g, H, W)
    close = np.abs(img - t) < margin
    t[close] = img[close] + np.where(t[close] >= img[close], margin, -margin)
    return t.astype(np.float32), img


def test_fit_step_matches_oracle_step():
    H, W, N, n = 128, 96, 1200, 3
    d = synth.gaussians(N, n, 2)
    P = synth.packed(d)
    g = O.Gaussians.from_packed(P)
    target, img = _unambiguous_target(g, H, W, 3)
    cfg = L.default_config()
    st = State(P)
    ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, 8 * N))
    loss = torch.zeros(1, device="cuda")
    tt = dev(target)
    L.fit_step(st.c, tt, H, W, cfg, ws, 8 * N, loss)
    torch.cuda.synchronize()
    ref_loss, dimg = O.l1_loss(img, target)
    ref_grad = O.backward_image(g, dimg, H, W)
    assert abs(loss.item() - ref_loss) <= 1e-6
    assert int(st.step.item()) == 1
    errs = grad_rel_error(st.G.cpu().numpy().astype(np.float64), ref_grad)
    assert max(errs.values()) <= 1e-3, errs
    # Parameters after Adam step 1: u = lr * g / (|g| + eps). A gradient error
    # dg moves u by at most lr * eps * dg / (|g| + eps)^2 (and never by more than 2 lr).
    Pr, _, _ = O.adam_update(P, ref_grad, np.zeros(P.shape), np.zeros(P.shape), 1)
    lr = lr_of(cfg, P.shape[1])[None, :]
    gscale = np.abs(ref_grad).max(axis=0, keepdims=True)
    dg = 1e-3 * gscale
    eps = 1e-8
    bound = np.minimum(2 * lr, lr * eps * dg / (np.abs(ref_grad) + eps) ** 2 + 1e-6 * lr)
    bound = bound + 2e-6 * np.abs(Pr) + 1e-7
    got = st.P.cpu().numpy()
    assert (np.abs(got - Pr) <= bound).all()


def test_fit_step_counter_and_loss_without_gaussians():
    """The step counter and the mean loss are written by the Adam launch's last
    CTA, or by a separate kernel when there is nothing to update (N = 0); with
    no Gaussians every pixel renders 0 and the loss is mean |c_t|."""
    H, W, n = 40, 56, 3
    target = synth.target_image(H, W, n, seed=4)
    cfg = L.default_config()
    for N in (0, 500):
        P = synth.packed(synth.gaussians(max(N, 1), n, 5))
        st = State(P)
        st.c.N = N
        ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, 8 * max(N, 1)))
        loss = torch.zeros(1, device="cuda")
        tt = dev(target)
        for k in range(3):
            L.fit_step(st.c, tt, H, W, cfg, ws, 8 * max(N, 1), loss)
            torch.cuda.synchronize()
            assert int(st.step.item()) == k + 1
            if N == 0:
                assert abs(loss.item() - float(np.abs(target.astype(np.float64)).mean())) <= 1e-6
            else:
                assert 0.0 < loss.item() < 1.0


def test_fit_loss_decreases_and_graph_replay_matches_eager():
    H, W, N, n = 256, 256, 4096, 3
    d = synth.gaussians(N, n, 0)
    P = synth.packed(d)
    target = dev(synth.target_image(H, W, n, seed=0))
    cfg = L.default_config()
    cap = 8 * N
    ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, cap))

    def run_eager(steps):
        st = State(P)
        loss = torch.zeros(1, device="cuda")
        losses = []
        for _ in range(steps):
            L.fit_step(st.c, target, H, W, cfg, ws, cap, loss)
            losses.append(loss.item())
        return st, losses

    st_e, losses = run_eager(60)
    assert losses[-1] < 0.8 * losses[0]
    assert np.mean(losses[-10:]) < np.mean(losses[:10])

    st_g = State(P)
    loss = torch.zeros(1, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        L.fit_step(st_g.c, target, H, W, cfg, ws, cap, loss, stream=s)   # warm-up, step 1
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        L.fit_step(st_g.c, target, H, W, cfg, ws, cap, loss)
    glosses = [loss.item()]
    for _ in range(4):
        graph.replay()
        torch.cuda.synchronize()
        glosses.append(loss.item())
    # warm-up ran once, capture runs nothing, each replay runs one step
    assert int(st_g.step.item()) == 5
    np.testing.assert_allclose(glosses, losses[:5], rtol=1e-3)


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_half_storage_fit_step_matches_oracle_step(dt):
    """Sec. 4.1 half-precision storage: the step renders and differentiates the
    half-rounded parameters, and Adam updates the float32 master."""
    H, W, N, n = 96, 80, 800, 3
    P = synth.packed(synth.gaussians(N, n, 5))
    Pr16 = torch.from_numpy(P).to(dt).float().numpy()        # the stored values
    g = O.Gaussians.from_packed(Pr16)
    target, img = _unambiguous_target(g, H, W, 6)
    cfg = L.default_config()
    st = State(P)
    half = torch.zeros(P.shape, dtype=dt, device="cuda")
    ws = L.alloc_workspace(L.workspace_size(N, n, H, W, cfg, 8 * N))
    loss = torch.zeros(1, device="cuda")
    L.fit_step_half(st.c, half, dev(target), H, W, cfg, ws, 8 * N, loss)
    torch.cuda.synchronize()
    ref_loss, dimg = O.l1_loss(img, target)
    ref_grad = O.backward_image(g, dimg, H, W)
    assert abs(loss.item() - ref_loss) <= 1e-6
    assert int(st.step.item()) == 1
    errs = grad_rel_error(st.G.cpu().numpy().astype(np.float64), ref_grad)
    assert max(errs.values()) <= 1e-3, errs
    # the master moves by Adam step 1 from its own float32 values
    Pr, _, _ = O.adam_update(P, ref_grad, np.zeros(P.shape), np.zeros(P.shape), 1)
    lr = lr_of(cfg, P.shape[1])[None, :]
    dg = 1e-3 * np.abs(ref_grad).max(axis=0, keepdims=True)
    bound = np.minimum(2 * lr, lr * 1e-8 * dg / (np.abs(ref_grad) + 1e-8) ** 2 + 1e-6 * lr)
    bound = bound + 2e-6 * np.abs(Pr) + 1e-7
    got = st.P.cpu().numpy()
    assert (np.abs(got - Pr) <= bound).all()
    # the stored copy is the nearest-even rounding of the updated master
    assert torch.equal(half.cpu(), st.P.cpu().to(dt))
