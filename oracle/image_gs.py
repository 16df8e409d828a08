"""Plain, slow CPU oracle of the Image-GS rasteriser (forward, adjoint, fit step).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this module. It shares no code with
the CUDA path and imports nothing from the package.

What it computes (Image-GS, Sec. 3.1-3.3 and Sec. 4.1):

* A Gaussian i has parameters p_i = (mu_i, theta_i, s_i, c_i) in R^(5+n)
  (Eq. 3), with the image domain mapped to [0,1]^2 (Sec. 4.1). The trainable
  scale is the inverse scale t = 1/s (Sec. 3.3 footnote, Sec. 4.1).
* Its value at x is G_i(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)) (Eq. 1) with
  Sigma = R S S^T R^T (Eq. 2), R the rotation by theta, S = diag(s1, s2). Hence
  Sigma^-1 = R diag(t1^2, t2^2) R^T, used here in closed form.
* The image is cut into tiles (16x16 in Sec. 4.1). S_j is the set of Gaussians
  whose minimum enclosing circle of the 3-sigma ellipse, radius 3*max(s1,s2),
  intersects tile j (Sec. 3.2).
* A pixel x in tile j ranks the members of S_j by their value at x, keeps the
  top K (K = 10, Sec. 4.1) and renders the normalised blend of Eq. 5. Eq. 4
  (the unnormalised sum over all N) is kept as a mode for closed-form checks.
* Fitting minimises the L1 loss (Sec. 3.3, Sec. 4.1; the SSIM term is not part
  of this path) with Adam and the per-group learning rates of Sec. 4.1,
  clipping theta and the scales to valid ranges after each update (Sec. 3.1).
  Gradients pass through the K retained Gaussians only (Sec. 3.3).

Readings where the paper is silent (the same as the library header's): pixel (h, w) is
evaluated at its centre (w + 1/2, h + 1/2) in pixels, x along the width, y
down the rows; mu in pixels is mu_px = (fl32(mu_x * W), fl32(mu_y * H)) -- the
binary32 product is the input's rounding point; tile j is the closed rectangle
clipped to the image and "intersects" means distance <= r; ranking is by the
quadratic form q = (x-mu)^T Sigma^-1 (x-mu) ascending (equivalently G
descending), ties to the smaller Gaussian index; the blend is evaluated with
weights exp(-(q - q_min)/2), equal to Eq. 5 in exact arithmetic; an empty S_j
renders 0; the loss is the mean over H*W*n with d|z|/dz = sign(z), sign(0)=0;
Adam uses beta = (0.9, 0.999), eps = 1e-8 with bias correction; theta is clamped
to [0, pi], t to [t_min, t_max], mu to [0, 1]^2.

Precision: every value is float64. The two integer decisions that floating
point makes -- tile membership and the top-K ranking -- are taken in binary32
with the operation sequence the library's header fixes (see `fp32.py`), so the
oracle and the CUDA path select identical sets.

Parity pins for every function here live in tests/test_oracle_*.py.
"""
import numpy as np

from .fp32 import F32, F64, fma32

# Column order of a packed parameter / gradient row: mu_x, mu_y, theta, t1, t2, c...
COL_MUX, COL_MUY, COL_THETA, COL_T1, COL_T2, COL_C0 = range(6)


class Gaussians:
    """Parameter set p_i = (mu, theta, t = 1/s, c), Eq. 3 with inverse scales.

    Arrays are copied to binary32 (or taken as given when already binary32):
    the oracle evaluates exactly the numbers the device stores. Half-precision
    inputs are passed as their exact binary32 upcasts.
    """

    def __init__(self, xy, theta, inv_scale, color):
        self.xy = np.ascontiguousarray(np.asarray(xy, dtype=F32).reshape(-1, 2))
        self.theta = np.ascontiguousarray(np.asarray(theta, dtype=F32).reshape(-1))
        self.inv_scale = np.ascontiguousarray(np.asarray(inv_scale, dtype=F32).reshape(-1, 2))
        c = np.asarray(color, dtype=F32)
        self.color = np.ascontiguousarray(c.reshape(c.shape[0], c.shape[1] if c.ndim > 1 else 1))
        self.N = self.xy.shape[0]
        self.n = self.color.shape[1]
        assert self.theta.shape[0] == self.N and self.inv_scale.shape[0] == self.N
        assert self.color.shape[0] == self.N

    @staticmethod
    def from_packed(P):
        """From a packed [N, 5+n] row array (mu_x, mu_y, theta, t1, t2, c...)."""
        P = np.asarray(P)
        return Gaussians(P[:, 0:2], P[:, 2], P[:, 3:5], P[:, 5:])

    def packed(self):
        return np.concatenate([self.xy, self.theta[:, None], self.inv_scale,
                               self.color], axis=1)


# ---------------------------------------------------------------------------
# Binary32 decision quantities (tile membership, ranking key).
# ---------------------------------------------------------------------------

def means_px32(g, H, W):
    """mu in pixels, binary32: (fl32(mu_x * W), fl32(mu_y * H)) (Sec. 4.1 [0,1]^2 map)."""
    return g.xy[:, 0] * F32(W), g.xy[:, 1] * F32(H)


def trig32(g):
    """cos(theta), sin(theta) evaluated in float64, each rounded once to binary32."""
    th = g.theta.astype(F64)
    return np.cos(th).astype(F32), np.sin(th).astype(F32)


def conic32(g):
    """Sigma^-1 = R diag(t1^2, t2^2) R^T (Eq. 2 inverted) in binary32.

    Returns (A00, B, A11) with B = 2*A01, each product and sum rounded once:
    A00 = T1*cc + T2*ss, A11 = T1*ss + T2*cc, A01 = (T1 - T2)*cs,
    T1 = t1*t1, T2 = t2*t2, cc = c*c, ss = s*s, cs = c*s.
    """
    c, s = trig32(g)
    t1, t2 = g.inv_scale[:, 0], g.inv_scale[:, 1]
    T1, T2 = t1 * t1, t2 * t2
    cc, ss, cs = c * c, s * s, c * s
    A00 = (T1 * cc) + (T2 * ss)
    A11 = (T1 * ss) + (T2 * cc)
    A01 = (T1 - T2) * cs
    B = A01 + A01
    return A00, B, A11


def radius32(g):
    """Radius of the minimum enclosing circle of the 3-sigma ellipse (Sec. 3.2).

    r = 3 * max(s1, s2) = 3 / min(t1, t2), one binary32 division.
    """
    return F32(3.0) / np.minimum(g.inv_scale[:, 0], g.inv_scale[:, 1])


def tile_rect(tx, ty, tile, H, W):
    """Closed pixel rectangle [X0, X1] x [Y0, Y1] of tile (tx, ty), clipped to the image."""
    X0 = F32(tx * tile)
    Y0 = F32(ty * tile)
    X1 = F32(min((tx + 1) * tile, W))
    Y1 = F32(min((ty + 1) * tile, H))
    return X0, X1, Y0, Y1


def tile_members(g, tx, ty, tile, H, W):
    """Boolean mask over all N Gaussians: i in S_j for tile j = (tx, ty) (Sec. 3.2).

    Circle-rectangle test in binary32: ex = max(X0 - mx, mx - X1, 0),
    ey likewise, member iff ex*ex + ey*ey <= r*r.
    """
    mx, my = means_px32(g, H, W)
    r = radius32(g)
    X0, X1, Y0, Y1 = tile_rect(tx, ty, tile, H, W)
    ex = np.maximum(np.maximum(X0 - mx, mx - X1), F32(0.0))
    ey = np.maximum(np.maximum(Y0 - my, my - Y1), F32(0.0))
    d2 = (ex * ex) + (ey * ey)
    return d2 <= (r * r)


def rank_key32(px, py, mx, my, A00, B, A11):
    """Ranking key q at (px, py) in binary32 (order fixed by the library header).

    dx = px - mx, dy = py - my, h = fma(B, dy, A00*dx),
    q = fma(h, dx, (A11*dy)*dy)  ==  A00 dx^2 + 2 A01 dx dy + A11 dy^2.
    Broadcasts over any matching shapes.
    """
    px = np.asarray(px, dtype=F32)
    py = np.asarray(py, dtype=F32)
    dx = px - mx
    dy = py - my
    h = fma32(B, dy, A00 * dx)
    e = (A11 * dy) * dy
    return fma32(h, dx, e)


# ---------------------------------------------------------------------------
# Float64 values.
# ---------------------------------------------------------------------------

def frame64(g):
    """Float64 rotation frame: u = (cos, sin), v = (-sin, cos) (columns of R, Eq. 2)."""
    th = g.theta.astype(F64)
    return np.cos(th), np.sin(th)


def conic64(g):
    """Sigma^-1 = t1^2 u u^T + t2^2 v v^T in float64 as (A00, A01, A11)."""
    c, s = frame64(g)
    T1 = g.inv_scale[:, 0].astype(F64) ** 2
    T2 = g.inv_scale[:, 1].astype(F64) ** 2
    return T1 * c * c + T2 * s * s, (T1 - T2) * c * s, T1 * s * s + T2 * c * c


def quad_form64(px, py, g, H, W, idx=None):
    """q = d^T Sigma^-1 d with d = x - mu_px in float64 (Eq. 1 exponent times -2).

    mu_px enters as its binary32 value (the rounding point); everything else
    is float64: q = t1^2 (u.d)^2 + t2^2 (v.d)^2.
    """
    mx32, my32 = means_px32(g, H, W)
    c, s = frame64(g)
    t1 = g.inv_scale[:, 0].astype(F64)
    t2 = g.inv_scale[:, 1].astype(F64)
    if idx is not None:
        mx32, my32, c, s, t1, t2 = mx32[idx], my32[idx], c[idx], s[idx], t1[idx], t2[idx]
    dx = np.asarray(px, dtype=F64) - mx32.astype(F64)
    dy = np.asarray(py, dtype=F64) - my32.astype(F64)
    a = c * dx + s * dy
    b = -s * dx + c * dy
    return (t1 * a) ** 2 + (t2 * b) ** 2


# ---------------------------------------------------------------------------
# Forward: Eq. 5 (top-K normalised) and Eq. 4 (naive sum).
# ---------------------------------------------------------------------------

def _tile_of(px, py, tile, H, W):
    tiles_x = -(-W // tile)
    tiles_y = -(-H // tile)
    tx = min(max(int(np.floor(px / tile)), 0), tiles_x - 1)
    ty = min(max(int(np.floor(py / tile)), 0), tiles_y - 1)
    return tx, ty


def _select_topk(q32, gids, K):
    """Rows of q32 [P, M]: column order of the K smallest (q32, gid) per row."""
    M = q32.shape[1]
    gid_b = np.broadcast_to(gids[None, :], q32.shape)
    order = np.lexsort((gid_b, q32), axis=-1)
    keep = M if K is None else min(K, M)
    return order[:, :keep]


def _points_in_tile(g, pts, tx, ty, tile, H, W, K, normalize, want_aux):
    """Evaluate Eq. 5 at the points pts [P,2] (pixels) that all lie in tile (tx, ty)."""
    n = g.n
    P = pts.shape[0]
    member = np.nonzero(tile_members(g, tx, ty, tile, H, W))[0]
    out = np.zeros((P, n), dtype=F64)
    aux = None
    if member.size == 0:
        if want_aux:
            aux = dict(sel=np.zeros((P, 0), np.int64), w=np.zeros((P, 0)), Z=np.zeros(P))
        return out, aux
    mx, my = means_px32(g, H, W)
    A00, B, A11 = conic32(g)
    px32 = pts[:, 0].astype(F32)[:, None]
    py32 = pts[:, 1].astype(F32)[:, None]
    q32 = rank_key32(px32, py32, mx[member][None, :], my[member][None, :],
                     A00[member][None, :], B[member][None, :], A11[member][None, :])
    cols = _select_topk(q32, member, K)
    sel = member[cols]                                   # [P, K'] gids, ranked
    q64 = quad_form64(pts[:, 0:1], pts[:, 1:2], g, H, W, idx=sel)
    csel = g.color.astype(F64)[sel]                      # [P, K', n]
    if normalize:
        w = np.exp(-0.5 * (q64 - q64.min(axis=1, keepdims=True)))
        Z = w.sum(axis=1)
        out = (w[:, :, None] * csel).sum(axis=1) / Z[:, None]
    else:
        w = np.exp(-0.5 * q64)
        Z = np.ones(P)
        out = (w[:, :, None] * csel).sum(axis=1)
    if want_aux:
        aux = dict(sel=sel, w=w, Z=Z, q64=q64)
    return out, aux


def render_points(g, pts, H, W, K=10, tile=16, normalize=True):
    """Colours c_r at arbitrary points pts [P,2] = (x, y) in pixels (Eq. 5).

    The point's tile is (floor(x/tile), floor(y/tile)) clamped to the grid;
    K=None keeps all of S_j. Returns float64 [P, n].
    """
    pts = np.asarray(pts, dtype=F64).reshape(-1, 2)
    out = np.zeros((pts.shape[0], g.n), dtype=F64)
    keys = [_tile_of(x, y, tile, H, W) for x, y in pts]
    groups = {}
    for i, k in enumerate(keys):
        groups.setdefault(k, []).append(i)
    for (tx, ty), rows in groups.items():
        rows = np.asarray(rows)
        o, _ = _points_in_tile(g, pts[rows], tx, ty, tile, H, W, K, normalize, False)
        out[rows] = o
    return out


def pixel_centres(pixels):
    """(h, w) integer pixel indices -> their centres (w + 1/2, h + 1/2)."""
    pixels = np.asarray(pixels).reshape(-1, 2)
    return np.stack([pixels[:, 1] + 0.5, pixels[:, 0] + 0.5], axis=1).astype(F64)


def render_pixels(g, pixels, H, W, K=10, tile=16, normalize=True):
    """c_r at integer pixels [P,2] = (h, w); float64 [P, n]."""
    return render_points(g, pixel_centres(pixels), H, W, K, tile, normalize)


def render_image(g, H, W, K=10, tile=16, normalize=True):
    """Full image, planar float64 [n, H, W] (small images only)."""
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    pix = np.stack([hh.ravel(), ww.ravel()], axis=1)
    out = render_pixels(g, pix, H, W, K, tile, normalize)
    return out.T.reshape(g.n, H, W)


def render_naive(g, pts, H, W):
    """Eq. 4: c_r(x) = sum over ALL N of G_i(x) c_i, no tiles, no normalisation."""
    pts = np.asarray(pts, dtype=F64).reshape(-1, 2)
    q = quad_form64(pts[:, 0:1], pts[:, 1:2], g, H, W, idx=np.arange(g.N)[None, :])
    G = np.exp(-0.5 * q)
    return G @ g.color.astype(F64)


def selection(g, pts, H, W, K=10, tile=16):
    """Selected Gaussian indices per point, ranked (list of int arrays)."""
    pts = np.asarray(pts, dtype=F64).reshape(-1, 2)
    res = []
    for x, y in pts:
        tx, ty = _tile_of(x, y, tile, H, W)
        _, aux = _points_in_tile(g, np.array([[x, y]]), tx, ty, tile, H, W, K, True, True)
        res.append(aux["sel"][0])
    return res


def selection_f64(g, pts, H, W, K=10, tile=16):
    """Per point, the indices the top-K of Sec. 3.2 keeps when it ranks by
    float64 keys (quad_form64, the binary32 rounding of the key evaluation
    removed; ties to the smaller index) instead of the binary32 keys. The
    candidates are the same S_j. List of index arrays, ranked."""
    pts = np.asarray(pts, dtype=F64).reshape(-1, 2)
    res = []
    for x, y in pts:
        tx, ty = _tile_of(x, y, tile, H, W)
        member = np.nonzero(tile_members(g, tx, ty, tile, H, W))[0]
        if member.size == 0:
            res.append(member)
            continue
        q64 = quad_form64(np.array([[x]]), np.array([[y]]), g, H, W, idx=member[None, :])
        cols = _select_topk(q64, member, K)
        res.append(member[cols[0]])
    return res


def selection_mismatches(g, pts, H, W, K=10, tile=16):
    """Points whose selected set under binary32 keys (the decision the kernels
    take) differs from the set under float64 keys: the pixels where rounding
    of the key decides which Gaussians are kept (near-ties at the K-th place).
    Returns the indices of those points."""
    a = selection(g, pts, H, W, K, tile)
    b = selection_f64(g, pts, H, W, K, tile)
    return [i for i, (u, v) in enumerate(zip(a, b)) if set(u.tolist()) != set(v.tolist())]


# ---------------------------------------------------------------------------
# Adjoint: gradients through the K retained Gaussians (Sec. 3.3).
# ---------------------------------------------------------------------------

def backward_points(g, pts, grad_out, H, W, K=10, tile=16, normalize=True):
    """dL/dp for L with dL/dc_r(x) = grad_out[x] at the points pts, selection fixed.

    Returns float64 [N, 5+n] in the packed column order
    (mu_x, mu_y, theta, t1, t2, c...). Closed forms, with a = u.d, b = v.d,
    w_k = exp(-(q_k - q_min)/2), Z = sum w_k, G_k = dL/dq_k:
      dL/dc_k = g w_k / Z
      G_k = -(w_k / (2Z)) sum_ch g_ch (c_k,ch - c_r,ch)
      dq/dt1 = 2 t1 a^2, dq/dt2 = 2 t2 b^2, dq/dtheta = 2ab(t1^2 - t2^2)
      dq/dmu_px = -2 (t1^2 a u + t2^2 b v), dmu_px/dmu = (W, H).
    Without normalisation (c_r = sum G_k c_k, G_k = exp(-q_k/2), the
    ablation of Table 1): dL/dc_k = g G_k and G_k' = -(G_k/2) sum_ch g_ch c_k,ch.
    """
    pts = np.asarray(pts, dtype=F64).reshape(-1, 2)
    go = np.asarray(grad_out, dtype=F64).reshape(pts.shape[0], g.n)
    grad = np.zeros((g.N, 5 + g.n), dtype=F64)
    c64, s64 = frame64(g)
    t1 = g.inv_scale[:, 0].astype(F64)
    t2 = g.inv_scale[:, 1].astype(F64)
    mx32, my32 = means_px32(g, H, W)
    col = g.color.astype(F64)
    keys = [_tile_of(x, y, tile, H, W) for x, y in pts]
    groups = {}
    for i, k in enumerate(keys):
        groups.setdefault(k, []).append(i)
    for (tx, ty), rows in groups.items():
        rows = np.asarray(rows)
        P = pts[rows]
        cr, aux = _points_in_tile(g, P, tx, ty, tile, H, W, K, normalize, True)
        sel, w, Z = aux["sel"], aux["w"], aux["Z"]
        if sel.shape[1] == 0:
            continue
        gp = go[rows]                                          # [P, n]
        wz = w / Z[:, None]                                    # [P, K']
        ck = col[sel]                                          # [P, K', n]
        if normalize:
            Gq = -0.5 * wz * ((ck - cr[:, None, :]) * gp[:, None, :]).sum(axis=2)
        else:
            Gq = -0.5 * w * (ck * gp[:, None, :]).sum(axis=2)
        dx = P[:, 0:1] - mx32[sel].astype(F64)
        dy = P[:, 1:2] - my32[sel].astype(F64)
        c, s, a1, a2 = c64[sel], s64[sel], t1[sel], t2[sel]
        a = c * dx + s * dy
        b = -s * dx + c * dy
        d_mx = -2.0 * (a1 * a1 * a * c - a2 * a2 * b * s)
        d_my = -2.0 * (a1 * a1 * a * s + a2 * a2 * b * c)
        d_th = 2.0 * a * b * (a1 * a1 - a2 * a2)
        d_t1 = 2.0 * a1 * a * a
        d_t2 = 2.0 * a2 * b * b
        flat = sel.ravel()
        np.add.at(grad[:, COL_MUX], flat, (Gq * d_mx * W).ravel())
        np.add.at(grad[:, COL_MUY], flat, (Gq * d_my * H).ravel())
        np.add.at(grad[:, COL_THETA], flat, (Gq * d_th).ravel())
        np.add.at(grad[:, COL_T1], flat, (Gq * d_t1).ravel())
        np.add.at(grad[:, COL_T2], flat, (Gq * d_t2).ravel())
        dc = wz[:, :, None] * gp[:, None, :]                   # [P, K', n]
        for ch in range(g.n):
            np.add.at(grad[:, COL_C0 + ch], flat, dc[:, :, ch].ravel())
    return grad


def backward_pixels(g, pixels, grad_out, H, W, K=10, tile=16, normalize=True):
    """backward_points at integer pixels (h, w)."""
    return backward_points(g, pixel_centres(pixels), grad_out, H, W, K, tile, normalize)


def backward_image(g, grad_img, H, W, K=10, tile=16, normalize=True):
    """Adjoint of render_image for a planar upstream gradient [n, H, W]."""
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    pix = np.stack([hh.ravel(), ww.ravel()], axis=1)
    go = np.asarray(grad_img, dtype=F64).reshape(g.n, H * W).T
    return backward_pixels(g, pix, go, H, W, K, tile, normalize)


# ---------------------------------------------------------------------------
# Loss and fit step (Sec. 3.3, Sec. 4.1).
# ---------------------------------------------------------------------------

def l1_loss(img, target):
    """Mean absolute error over every element and its gradient sign(img-target)/count."""
    img = np.asarray(img, dtype=F64)
    target = np.asarray(target, dtype=F64)
    diff = img - target
    return np.abs(diff).mean(), np.sign(diff) / diff.size


DEFAULT_LR = dict(mu=5e-4, color=5e-3, inv_scale=2e-3, theta=2e-3)   # Sec. 4.1
DEFAULT_BOUNDS = dict(theta=(0.0, np.pi), inv_scale=(1e-3, 10.0), mu=(0.0, 1.0))


def adam_update(P, G, m, v, step, lr=None, betas=(0.9, 0.999), eps=1e-8, bounds=None):
    """One Adam update of packed parameters P [N, 5+n] with gradient G, then clamps.

    Adam (Kingma and Ba) with bias correction, step >= 1; learning rate per
    column group from Sec. 4.1; afterwards theta in [0, pi], t in bounds,
    mu in [0, 1]^2 (Sec. 3.1 "clipped to the valid ranges"). Returns new
    (P, m, v) in float64.
    """
    lr = dict(DEFAULT_LR if lr is None else lr)
    bounds = dict(DEFAULT_BOUNDS if bounds is None else bounds)
    P = np.asarray(P, dtype=F64).copy()
    G = np.asarray(G, dtype=F64)
    b1, b2 = betas
    m = b1 * np.asarray(m, dtype=F64) + (1 - b1) * G
    v = b2 * np.asarray(v, dtype=F64) + (1 - b2) * G * G
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    ncol = P.shape[1]
    rate = np.empty(ncol)
    rate[[COL_MUX, COL_MUY]] = lr["mu"]
    rate[COL_THETA] = lr["theta"]
    rate[[COL_T1, COL_T2]] = lr["inv_scale"]
    rate[COL_C0:] = lr["color"]
    P -= rate[None, :] * mhat / (np.sqrt(vhat) + eps)
    P[:, COL_MUX:COL_MUY + 1] = np.clip(P[:, COL_MUX:COL_MUY + 1], *bounds["mu"])
    P[:, COL_THETA] = np.clip(P[:, COL_THETA], *bounds["theta"])
    P[:, COL_T1:COL_T2 + 1] = np.clip(P[:, COL_T1:COL_T2 + 1], *bounds["inv_scale"])
    return P, m, v


def count_evals(g, H, W, tile=16):
    """Gaussian-pixel evaluations of one forward: sum over tiles of |S_j| * |tile pixels|."""
    tiles_x = -(-W // tile)
    tiles_y = -(-H // tile)
    total = 0
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            X0, X1, Y0, Y1 = tile_rect(tx, ty, tile, H, W)
            npx = int(X1 - X0) * int(Y1 - Y0)
            total += int(tile_members(g, tx, ty, tile, H, W).sum()) * npx
    return total


def tile_lists(g, H, W, tile=16):
    """S_j for every tile as sorted index arrays (row-major tile order); small cases only."""
    tiles_x = -(-W // tile)
    tiles_y = -(-H // tile)
    return [np.nonzero(tile_members(g, tx, ty, tile, H, W))[0]
            for ty in range(tiles_y) for tx in range(tiles_x)]
