"""Helpers that run the CUDA path through the C ABI on numpy inputs (tests only)."""
import numpy as np
import torch

from paper_2407_01866_b300 import lib as L

DEV = "cuda"


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


class GpuSet:
    """Device copies of a parameter set plus its binning."""

    def __init__(self, g, H, W, K=10, tile=16, dtype=torch.float32, m_capacity=None,
                 normalize=1):
        self.H, self.W, self.n, self.N = H, W, g.n, g.N
        self.cfg = L.default_config(K=K, tile=tile, normalize=normalize)
        self.xy = dev(g.xy, dtype)
        self.theta = dev(g.theta, dtype)
        self.inv_scale = dev(g.inv_scale, dtype)
        self.color = dev(g.color, dtype)
        self.view = L.gaussians_view(self.xy, self.theta, self.inv_scale, self.color)
        self.binner = L.Binner(g.N, g.n, H, W, self.cfg, m_capacity=m_capacity)
        self.bins = self.binner.bin(self.view)
        self.stats = L.read_stats(self.bins)

    def ws_array(self, ptr, count, dtype):
        ws = self.binner.ws
        off = ptr - ws.data_ptr()
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return ws[off:off + nbytes].view(dtype)

    def tile_lists(self):
        T = self.bins.tiles_x * self.bins.tiles_y
        rng = self.ws_array(self.bins.tile_range, 2 * T, torch.int32).cpu().numpy().reshape(T, 2)
        lst = self.ws_array(self.bins.list, max(int(self.stats.m_needed), 1),
                            torch.int32).cpu().numpy()
        return [lst[a:b] for a, b in rng]

    def forward(self):
        img = torch.empty((self.n, self.H, self.W), device=DEV)
        L.render_forward(self.bins, self.cfg, img)
        return img.cpu().numpy()

    def backward(self, grad_img=None, target=None):
        grad = torch.empty((self.N, 5 + self.n), device=DEV)
        gi = dev(grad_img) if grad_img is not None else None
        tg = dev(target) if target is not None else None
        L.render_backward(self.view, self.bins, self.cfg, gi, tg, grad)
        st = L.read_stats(self.bins)
        return grad.cpu().numpy().astype(np.float64), st

    def decode(self, pts):
        q = dev(pts)
        out = torch.empty((pts.shape[0], self.n), device=DEV)
        L.decode_points(self.bins, self.cfg, q, out)
        return out.cpu().numpy()


GROUPS = [("mu", slice(0, 2)), ("theta", slice(2, 3)), ("inv_scale", slice(3, 5)),
          ("color", slice(5, None))]


def grad_rel_error(got, ref):
    """Normwise relative error per parameter group: max|d| / max|ref|."""
    out = {}
    for name, sl in GROUPS:
        r = ref[:, sl]
        d = np.abs(got[:, sl] - r).max() if r.size else 0.0
        s = np.abs(r).max() if r.size else 0.0
        out[name] = d / s if s > 0 else d
    return out


def grad_elem_rel_error(got, ref, floor=1e-6):
    """Per-element relative error per parameter group: the largest
    |got - ref| / max(|ref|, floor * max|ref| over the group)."""
    out = {}
    for name, sl in GROUPS:
        r = ref[:, sl]
        if not r.size:
            out[name] = 0.0
            continue
        s = np.abs(r).max()
        den = np.maximum(np.abs(r), floor * s) if s > 0 else np.ones_like(r)
        out[name] = float((np.abs(got[:, sl] - r) / den).max())
    return out
