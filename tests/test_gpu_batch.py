"""Batched form: many images of uneven size in one persistent launch.

The batched step must give each image what the single-image step gives it
(same binning, same selection, gradients up to float32 summation order), and
image gradients must match the oracle.
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

from gpu_harness import dev, grad_rel_error  # noqa: E402

SHAPES = [(40, 57), (100, 33), (64, 64), (17, 90), (128, 96), (5, 7)]


def make_batch(seed=0, n=3):
    Hs, Ws, Ns, Ps, Ts = [], [], [], [], []
    for b, (H, W) in enumerate(SHAPES):
        N = max(1, round(H * W / 28))
        P = synth.packed(synth.gaussians(N, n, seed + b))
        T = synth.target_image(H, W, n, seed=seed + 100 + b)
        Hs.append(H); Ws.append(W); Ns.append(N); Ps.append(P); Ts.append(T)
    return Hs, Ws, Ns, Ps, Ts


class State:
    def __init__(self, P):
        self.P = dev(P)
        self.G = torch.zeros_like(self.P)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.step = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.c = L.FitState(self.P.data_ptr(), self.G.data_ptr(), self.m.data_ptr(),
                            self.v.data_ptr(), self.step.data_ptr(), P.shape[0], P.shape[1] - 5)


def batched(Hs, Ws, Ns, Ps, Ts, n=3, tuning=None, cap_per_gauss=16):
    cfg = L.default_config()
    shape = L.batch_shape(Hs, Ws, Ns, n)
    cap = cap_per_gauss * sum(Ns) + 1024
    ws = L.alloc_workspace(L.batch_workspace_size(shape, cfg, cap))
    L.batch_setup(shape, cfg, ws, cap)
    st = State(np.concatenate(Ps))
    tg = dev(np.concatenate([t.ravel() for t in Ts]))
    loss = torch.zeros(len(Hs), device="cuda")
    return cfg, shape, cap, ws, st, tg, loss


def split(a, Ns):
    out, o = [], 0
    for N in Ns:
        out.append(a[o:o + N])
        o += N
    return out


def test_batched_step_equals_single_image_steps_and_oracle():
    Hs, Ws, Ns, Ps, Ts = make_batch()
    # image 0's target moved away from the oracle image where the L1 sign is ambiguous
    g0 = O.Gaussians.from_packed(Ps[0])
    img0 = O.render_image(g0, Hs[0], Ws[0])
    t0 = Ts[0].astype(np.float64)
    close = np.abs(img0 - t0) < 1e-4
    t0[close] = img0[close] + np.where(t0[close] >= img0[close], 1e-4, -1e-4)
    Ts[0] = t0.astype(np.float32)
    cfg, shape, cap, ws, st, tg, loss = batched(Hs, Ws, Ns, Ps, Ts)
    L.fit_batch_step(st.c, tg, shape, cfg, ws, cap, loss_out=loss)
    torch.cuda.synchronize()
    gb = split(st.G.cpu().numpy().astype(np.float64), Ns)
    pb = split(st.P.cpu().numpy(), Ns)
    lb = loss.cpu().numpy()
    assert int(st.step.item()) == 1
    for b in range(len(Hs)):
        s1 = State(Ps[b])
        w1 = L.alloc_workspace(L.workspace_size(Ns[b], 3, Hs[b], Ws[b], cfg, 16 * Ns[b] + 64))
        l1 = torch.zeros(1, device="cuda")
        L.fit_step(s1.c, dev(Ts[b]), Hs[b], Ws[b], cfg, w1, 16 * Ns[b] + 64, l1)
        torch.cuda.synchronize()
        assert abs(l1.item() - lb[b]) <= 1e-6 * max(1.0, abs(lb[b])), b
        errs = grad_rel_error(gb[b], s1.G.cpu().numpy().astype(np.float64))
        assert max(errs.values()) <= 1e-4, (b, errs)
    ref_loss, dimg = O.l1_loss(img0, Ts[0])
    assert abs(lb[0] - ref_loss) <= 1e-6
    ref = O.backward_image(g0, dimg, Hs[0], Ws[0])
    errs = grad_rel_error(gb[0], ref)
    assert max(errs.values()) <= 1e-3, errs


@pytest.mark.parametrize("tn", [(1, 64, 0), (2, 128, 1), (8, 256, 0), (3, 64, 1)])
def test_every_tuning_gives_the_same_gradients(tn):
    Hs, Ws, Ns, Ps, Ts = make_batch(seed=3)
    cfg, shape, cap, ws, st, tg, loss = batched(Hs, Ws, Ns, Ps, Ts)
    L.fit_batch_step(st.c, tg, shape, cfg, ws, cap)
    g_def = st.G.cpu().numpy().astype(np.float64)
    cfg, shape, cap, ws, st2, tg, loss = batched(Hs, Ws, Ns, Ps, Ts)
    L.fit_batch_step(st2.c, tg, shape, cfg, ws, cap, tuning=L.BatchTuning(*tn))
    errs = grad_rel_error(st2.G.cpu().numpy().astype(np.float64), g_def)
    assert max(errs.values()) <= 1e-4, errs


def test_autotune_and_graph_replay():
    Hs, Ws, Ns, Ps, Ts = make_batch(seed=5)
    cfg, shape, cap, ws, st, tg, loss = batched(Hs, Ws, Ns, Ps, Ts)
    best, ms = L.autotune_batch(st.c, tg, shape, cfg, ws, cap, reps=2)
    assert best.ctas_per_sm in (2, 3, 4, 6, 8) and best.stage in (64, 128, 256)
    assert best.order in (0, 1) and ms > 0
    assert int(st.step.item()) == 0 and np.array_equal(st.P.cpu().numpy(), np.concatenate(Ps))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        L.fit_batch_step(st.c, tg, shape, cfg, ws, cap, tuning=best, loss_out=loss, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    first = loss.cpu().numpy().copy()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        L.fit_batch_step(st.c, tg, shape, cfg, ws, cap, tuning=best, loss_out=loss)
    for _ in range(40):
        graph.replay()
    torch.cuda.synchronize()
    assert int(st.step.item()) == 41
    last = loss.cpu().numpy()
    assert (last < first).all(), (first, last)


@pytest.mark.parametrize("K,normalize", [(3, 1), (0, 0), (16, 1)])
def test_batched_step_equals_single_image_steps_in_other_modes(K, normalize):
    Hs, Ws, Ns, Ps, Ts = make_batch(seed=9)
    cfg = L.default_config(K=K, normalize=normalize)
    shape = L.batch_shape(Hs, Ws, Ns, 3)
    cap = 16 * sum(Ns) + 1024
    ws = L.alloc_workspace(L.batch_workspace_size(shape, cfg, cap))
    L.batch_setup(shape, cfg, ws, cap)
    st = State(np.concatenate(Ps))
    tg = dev(np.concatenate([t.ravel() for t in Ts]))
    loss = torch.zeros(len(Hs), device="cuda")
    L.fit_batch_step(st.c, tg, shape, cfg, ws, cap, loss_out=loss)
    torch.cuda.synchronize()
    gb = split(st.G.cpu().numpy().astype(np.float64), Ns)
    lb = loss.cpu().numpy()
    for b in range(len(Hs)):
        s1 = State(Ps[b])
        w1 = L.alloc_workspace(L.workspace_size(Ns[b], 3, Hs[b], Ws[b], cfg, 16 * Ns[b] + 64))
        l1 = torch.zeros(1, device="cuda")
        L.fit_step(s1.c, dev(Ts[b]), Hs[b], Ws[b], cfg, w1, 16 * Ns[b] + 64, l1)
        torch.cuda.synchronize()
        assert abs(l1.item() - lb[b]) <= 1e-6 * max(1.0, abs(lb[b])), b
        errs = grad_rel_error(gb[b], s1.G.cpu().numpy().astype(np.float64))
        assert max(errs.values()) <= 1e-4, (b, errs)
