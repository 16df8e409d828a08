"""ctypes binding of libimgs.so (include/imgs.h), with a torch.autograd wrapper.

Argument marshalling only: every step of the rasteriser runs in the CUDA
library. PyTorch supplies device memory and the current stream. There is no
CPU fallback: if the library is missing or cannot be loaded, every call raises.
"""
import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libimgs.so")

IGS_OK, IGS_ERR_INVALID_ARG, IGS_ERR_ALIGN, IGS_ERR_CAPACITY, IGS_ERR_CUDA, \
    IGS_ERR_TIMEOUT, IGS_ERR_NONFINITE = range(7)
IGS_F32, IGS_F16, IGS_BF16 = 0, 1, 2
FLAG_CAPACITY, FLAG_NONFINITE, FLAG_TIMEOUT = 1, 2, 4

_DTYPE = {torch.float32: IGS_F32, torch.float16: IGS_F16, torch.bfloat16: IGS_BF16}


class IgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libimgs error {code}: {msg}")
        self.code = code


class Gaussians(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("inv_scale", ctypes.c_void_p), ("color", ctypes.c_void_p),
                ("xy_stride", ctypes.c_int64), ("theta_stride", ctypes.c_int64),
                ("inv_scale_stride", ctypes.c_int64), ("color_stride", ctypes.c_int64),
                ("N", ctypes.c_int64), ("n", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("tile", ctypes.c_int32), ("normalize", ctypes.c_int32),
                ("lr_mu", ctypes.c_float), ("lr_theta", ctypes.c_float),
                ("lr_inv_scale", ctypes.c_float), ("lr_color", ctypes.c_float),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_float),
                ("theta_min", ctypes.c_float), ("theta_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("t_max", ctypes.c_float),
                ("mu_min", ctypes.c_float), ("mu_max", ctypes.c_float),
                ("ssim_weight", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("m_needed", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("loss_sum", ctypes.c_double)]


class Bins(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32), ("n", ctypes.c_int32),
                ("N", ctypes.c_int64), ("m_capacity", ctypes.c_int64),
                ("tile_range", ctypes.c_void_p), ("list", ctypes.c_void_p),
                ("rec", ctypes.c_void_p), ("trig", ctypes.c_void_p),
                ("color", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("rec16", ctypes.c_void_p),
                ("color16", ctypes.c_void_p)]


class FitState(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("step", ctypes.c_void_p), ("N", ctypes.c_int64), ("n", ctypes.c_int32)]


class BatchShape(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("n", ctypes.c_int32),
                ("H", ctypes.POINTER(ctypes.c_int32)), ("W", ctypes.POINTER(ctypes.c_int32)),
                ("N", ctypes.POINTER(ctypes.c_int64))]


class BatchTuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("order", ctypes.c_int32)]

    def __repr__(self):
        return f"BatchTuning(ctas_per_sm={self.ctas_per_sm}, stage={self.stage}, order={self.order})"


_P = ctypes.c_void_p
_SIGNATURES = {
    "igs_version": ([], ctypes.c_int),
    "igs_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
    "igs_default_config": ([ctypes.POINTER(Config)], None),
    "igs_workspace_size": ([ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                            ctypes.POINTER(Config), ctypes.c_int64,
                            ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "igs_preprocess_bin": ([ctypes.POINTER(Gaussians), ctypes.c_int32, ctypes.c_int32,
                            ctypes.POINTER(Config), _P, ctypes.c_size_t, ctypes.c_int64,
                            ctypes.POINTER(Bins), _P], ctypes.c_int),
    "igs_render_forward": ([ctypes.POINTER(Bins), ctypes.POINTER(Config), _P, _P], ctypes.c_int),
    "igs_render_backward": ([ctypes.POINTER(Gaussians), ctypes.POINTER(Bins),
                             ctypes.POINTER(Config), _P, _P, _P, _P], ctypes.c_int),
    "igs_fit_step": ([ctypes.POINTER(FitState), _P, ctypes.c_int32, ctypes.c_int32,
                      ctypes.POINTER(Config), _P, ctypes.c_size_t, ctypes.c_int64, _P, _P],
                     ctypes.c_int),
    "igs_fit_step_half": ([ctypes.POINTER(FitState), _P, ctypes.c_int32, _P, ctypes.c_int32,
                           ctypes.c_int32, ctypes.POINTER(Config), _P, ctypes.c_size_t,
                           ctypes.c_int64, _P, _P], ctypes.c_int),
    "igs_adam_update": ([ctypes.POINTER(FitState), ctypes.POINTER(Config), _P], ctypes.c_int),
    "igs_image_loss_workspace_size": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "igs_image_loss": ([_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                        _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "igs_placement_workspace_size": ([ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "igs_init_gaussians": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                            ctypes.c_double, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "igs_add_gaussians": ([_P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64,
                           ctypes.POINTER(FitState), _P, ctypes.c_size_t, _P], ctypes.c_int),
    "igs_decode_points": ([ctypes.POINTER(Bins), ctypes.POINTER(Config), _P, ctypes.c_int64,
                           _P, _P], ctypes.c_int),
    "igs_read_stats": ([ctypes.POINTER(Bins), ctypes.POINTER(Stats), _P], ctypes.c_int),
    "igs_render_forward_static": ([ctypes.POINTER(Gaussians), ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(Config), _P, _P], ctypes.c_int),
    "igs_static_scratch_bytes": ([ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "igs_batch_workspace_size": ([ctypes.POINTER(BatchShape), ctypes.POINTER(Config),
                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "igs_render_forward_batch": ([_P, ctypes.c_int64, ctypes.POINTER(BatchShape),
                                  ctypes.POINTER(Config), _P, ctypes.c_size_t, ctypes.c_int64,
                                  _P, _P], ctypes.c_int),
    "igs_render_backward_batch": ([_P, ctypes.c_int64, _P, ctypes.POINTER(BatchShape),
                                   ctypes.POINTER(Config), ctypes.POINTER(BatchTuning), _P,
                                   ctypes.c_size_t, ctypes.c_int64, _P, _P], ctypes.c_int),
    "igs_batch_setup": ([ctypes.POINTER(BatchShape), ctypes.POINTER(Config), _P, ctypes.c_size_t,
                         ctypes.c_int64, _P], ctypes.c_int),
    "igs_fit_batch_step": ([ctypes.POINTER(FitState), _P, ctypes.POINTER(BatchShape),
                            ctypes.POINTER(Config), ctypes.POINTER(BatchTuning), _P,
                            ctypes.c_size_t, ctypes.c_int64, _P, _P], ctypes.c_int),
    "igs_autotune_batch": ([ctypes.POINTER(FitState), _P, ctypes.POINTER(BatchShape),
                            ctypes.POINTER(Config), _P, ctypes.c_size_t, ctypes.c_int64,
                            ctypes.c_int32, ctypes.POINTER(BatchTuning),
                            ctypes.POINTER(ctypes.c_float), _P], ctypes.c_int),
}

_lib = None


def load():
    """Load libimgs.so once; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2407_01866_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def exported_names():
    return list(_SIGNATURES)


def _check(code):
    if code != IGS_OK:
        buf = ctypes.create_string_buffer(1024)
        load().igs_last_error(buf, 1024)
        raise IgsError(code, buf.value.decode())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def default_config(**overrides):
    c = Config()
    load().igs_default_config(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def version():
    return load().igs_version()


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors")


def gaussians_view(xy, theta, inv_scale, color):
    """igs_gaussians over four tensors of one dtype (rows may be strided views)."""
    _require_cuda(xy, theta, inv_scale, color)
    dt = _DTYPE[xy.dtype]
    for t in (theta, inv_scale, color):
        if t.dtype != xy.dtype:
            raise ValueError("all parameter tensors must share one dtype")
    N = xy.shape[0]
    n = color.shape[1]
    if N > 0 and (xy.stride(1) != 1 or inv_scale.stride(1) != 1 or color.stride(1) != 1):
        raise ValueError("parameter rows must be contiguous")
    g = Gaussians(xy.data_ptr(), theta.data_ptr(), inv_scale.data_ptr(), color.data_ptr(),
                  xy.stride(0), theta.stride(0), inv_scale.stride(0), color.stride(0), N, n, dt)
    return g


def packed_view(P, n):
    """igs_gaussians over a packed [N, 5+n] tensor (mu_x, mu_y, theta, t1, t2, c...)."""
    return gaussians_view(P[:, 0:2], P[:, 2], P[:, 3:5], P[:, 5:5 + n])


def workspace_size(N, n, H, W, cfg, m_capacity):
    b = ctypes.c_size_t(0)
    _check(load().igs_workspace_size(N, n, H, W, ctypes.byref(cfg), m_capacity, ctypes.byref(b)))
    return b.value


def alloc_workspace(nbytes, device=None):
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(nbytes, 256), dtype=torch.uint8,
                       device=device or torch.device("cuda"))


def preprocess_bin(g, H, W, cfg, ws, m_capacity, stream=None):
    bins = Bins()
    _check(load().igs_preprocess_bin(ctypes.byref(g), H, W, ctypes.byref(cfg), _ptr(ws),
                                     ws.numel(), m_capacity, ctypes.byref(bins), _stream(stream)))
    bins._workspace = ws   # the bins point into ws: keep it alive with them
    return bins


def render_forward(bins, cfg, img, stream=None):
    _check(load().igs_render_forward(ctypes.byref(bins), ctypes.byref(cfg), _ptr(img),
                                     _stream(stream)))


def render_backward(g, bins, cfg, grad_img, target, grad, stream=None):
    _check(load().igs_render_backward(ctypes.byref(g), ctypes.byref(bins), ctypes.byref(cfg),
                                      _ptr(grad_img), _ptr(target), _ptr(grad), _stream(stream)))


def fit_step(state, target, H, W, cfg, ws, m_capacity, loss_out=None, stream=None):
    _check(load().igs_fit_step(ctypes.byref(state), _ptr(target), H, W, ctypes.byref(cfg),
                               _ptr(ws), ws.numel(), m_capacity, _ptr(loss_out), _stream(stream)))


def fit_step_half(state, params_half, target, H, W, cfg, ws, m_capacity, loss_out=None,
                  stream=None):
    """One fit step with half-precision storage: params_half is a [N, 5+n]
    torch.float16 or torch.bfloat16 tensor that receives the rounded master."""
    dt = _DTYPE.get(params_half.dtype)
    if dt not in (IGS_F16, IGS_BF16):
        raise IgsError(IGS_ERR_INVALID_ARG, "params_half must be float16 or bfloat16")
    _check(load().igs_fit_step_half(ctypes.byref(state), _ptr(params_half), dt, _ptr(target),
                                    H, W, ctypes.byref(cfg), _ptr(ws), ws.numel(), m_capacity,
                                    _ptr(loss_out), _stream(stream)))


def image_loss(render, target, ssim_weight, grad_img, loss_out=None, ws=None, stream=None):
    """L1 + ssim_weight * (1 - SSIM) of render against target ([n, H, W] each) and
    its image-space gradient (Sec. 4.1)."""
    n, H, W = target.shape
    if ws is None:
        b = ctypes.c_size_t()
        _check(load().igs_image_loss_workspace_size(n, H, W, ctypes.byref(b)))
        ws = alloc_workspace(b.value, target.device)
    _check(load().igs_image_loss(_ptr(render), _ptr(target), n, H, W, ssim_weight,
                                 _ptr(grad_img), _ptr(loss_out), _ptr(ws), ws.numel(),
                                 _stream(stream)))


def placement_workspace_size(H, W):
    b = ctypes.c_size_t()
    _check(load().igs_placement_workspace_size(H, W, ctypes.byref(b)))
    return b.value


def init_gaussians(target, N, rand, params, ws, lam=0.3, stream=None):
    """Eq. 6 placement: target [n, H, W] float32, rand [N, 2] int64 (53-bit
    values), params [N, 5+n] float32 output."""
    n, H, W = target.shape
    _check(load().igs_init_gaussians(_ptr(target), H, W, n, N, lam, _ptr(rand), _ptr(params),
                                     _ptr(ws), ws.numel(), _stream(stream)))


def add_gaussians(target, render, rand, count, state, ws, stream=None):
    """Eq. 7 placement of `count` Gaussians after row state.N (the caller raises
    state.N afterwards)."""
    n, H, W = target.shape
    _check(load().igs_add_gaussians(_ptr(target), _ptr(render), H, W, _ptr(rand), count,
                                    ctypes.byref(state), _ptr(ws), ws.numel(), _stream(stream)))


def adam_update(state, cfg, stream=None):
    _check(load().igs_adam_update(ctypes.byref(state), ctypes.byref(cfg), _stream(stream)))


def decode_points(bins, cfg, xy, out, stream=None):
    _check(load().igs_decode_points(ctypes.byref(bins), ctypes.byref(cfg), _ptr(xy),
                                    xy.shape[0], _ptr(out), _stream(stream)))


def render_forward_static(g, H, W, cfg, img, stream=None):
    """Bin and render with the library's fixed static scratch (no workspace,
    no allocation); synchronises the stream. See igs_render_forward_static."""
    _check(load().igs_render_forward_static(ctypes.byref(g), H, W, ctypes.byref(cfg), _ptr(img),
                                            _stream(stream)))


def static_scratch_bytes():
    b = ctypes.c_size_t(0)
    _check(load().igs_static_scratch_bytes(ctypes.byref(b)))
    return b.value


def batch_shape(Hs, Ws, Ns, n):
    """igs_batch_shape over host arrays (kept alive on the returned struct)."""
    B = len(Hs)
    h = (ctypes.c_int32 * B)(*[int(v) for v in Hs])
    w = (ctypes.c_int32 * B)(*[int(v) for v in Ws])
    m = (ctypes.c_int64 * B)(*[int(v) for v in Ns])
    sh = BatchShape(B, n, h, w, m)
    sh._keep = (h, w, m)
    return sh


def batch_workspace_size(shape, cfg, m_capacity):
    b = ctypes.c_size_t(0)
    _check(load().igs_batch_workspace_size(ctypes.byref(shape), ctypes.byref(cfg), m_capacity,
                                           ctypes.byref(b)))
    return b.value


def batch_setup(shape, cfg, ws, m_capacity, stream=None):
    _check(load().igs_batch_setup(ctypes.byref(shape), ctypes.byref(cfg), _ptr(ws), ws.numel(),
                                  m_capacity, _stream(stream)))


def fit_batch_step(state, targets, shape, cfg, ws, m_capacity, tuning=None, loss_out=None,
                   stream=None):
    tp = ctypes.byref(tuning) if tuning is not None else None
    _check(load().igs_fit_batch_step(ctypes.byref(state), _ptr(targets), ctypes.byref(shape),
                                     ctypes.byref(cfg), tp, _ptr(ws), ws.numel(), m_capacity,
                                     _ptr(loss_out), _stream(stream)))


def render_forward_batch(params, shape, cfg, ws, m_capacity, imgs, stream=None):
    """Renders every image of the batch (packed params [N, 5+n]) into imgs,
    the concatenated planar images."""
    _check(load().igs_render_forward_batch(_ptr(params), params.shape[0], ctypes.byref(shape),
                                           ctypes.byref(cfg), _ptr(ws), ws.numel(), m_capacity,
                                           _ptr(imgs), _stream(stream)))


def render_backward_batch(params, grad_imgs, shape, cfg, ws, m_capacity, grad, tuning=None,
                          stream=None):
    """Adjoint of every image of the batch for the upstream gradient
    grad_imgs (laid out like the rendered images); grad [N, 5+n] receives dL/dp."""
    tp = ctypes.byref(tuning) if tuning is not None else None
    _check(load().igs_render_backward_batch(_ptr(params), params.shape[0], _ptr(grad_imgs),
                                            ctypes.byref(shape), ctypes.byref(cfg), tp,
                                            _ptr(ws), ws.numel(), m_capacity, _ptr(grad),
                                            _stream(stream)))


def autotune_batch(state, targets, shape, cfg, ws, m_capacity, reps=3, stream=None):
    """Times every persistent-adjoint mapping on this batch; returns (tuning, ms)."""
    best = BatchTuning()
    ms = ctypes.c_float(0)
    _check(load().igs_autotune_batch(ctypes.byref(state), _ptr(targets), ctypes.byref(shape),
                                     ctypes.byref(cfg), _ptr(ws), ws.numel(), m_capacity, reps,
                                     ctypes.byref(best), ctypes.byref(ms), _stream(stream)))
    return best, ms.value


def read_stats(bins, stream=None):
    st = Stats()
    _check(load().igs_read_stats(ctypes.byref(bins), ctypes.byref(st), _stream(stream)))
    return st


# ---------------------------------------------------------------------------
# Convenience layer: sized workspaces and an autograd function.
# ---------------------------------------------------------------------------

class Binner:
    """Owns a workspace sized for (N, n, H, W) and grows its intersection
    capacity when a binning reports that it overflowed."""

    def __init__(self, N, n, H, W, cfg=None, m_capacity=None, headroom=1.5):
        self.N, self.n, self.H, self.W = N, n, H, W
        self.cfg = cfg or default_config()
        self.headroom = headroom
        self.m_capacity = int(m_capacity or max(1024, 8 * N))
        self._alloc()

    def _alloc(self):
        self.ws = alloc_workspace(workspace_size(self.N, self.n, self.H, self.W, self.cfg,
                                                 self.m_capacity))

    def bin(self, g, stream=None, check=True):
        """Bin g; with check=True, synchronises and re-bins with a larger
        capacity if the intersections did not fit."""
        bins = preprocess_bin(g, self.H, self.W, self.cfg, self.ws, self.m_capacity, stream)
        if check:
            st = read_stats(bins, stream)
            if st.flags & FLAG_CAPACITY:
                self.m_capacity = int(st.m_needed * self.headroom) + 1024
                self._alloc()
                bins = preprocess_bin(g, self.H, self.W, self.cfg, self.ws, self.m_capacity,
                                      stream)
        return bins


# Binners of the autograd path, one per (shape, config, device): their
# workspaces are allocated once and reused by every call of that shape.
_BINNERS = {}


def _binner_for(N, n, H, W, cfg, device):
    key = (N, n, H, W, cfg.K, cfg.tile, cfg.normalize, device.index)
    b = _BINNERS.get(key)
    if b is None:
        with torch.cuda.device(device):
            b = _BINNERS[key] = Binner(N, n, H, W, cfg)
    return b


class _RenderFn(torch.autograd.Function):
    """Forward render and its adjoint. The binning workspace is cached per
    shape; the backward bins the saved parameters again (into that cached
    workspace), so interleaved forwards of the same shape cannot disturb it.
    With check=False no call synchronises the host and an intersection
    overflow goes undetected (that call's lists are truncated): make a first
    checked call of the shape to size the cached workspace."""

    @staticmethod
    def forward(ctx, xy, theta, inv_scale, color, H, W, cfg, check):
        g = gaussians_view(xy, theta, inv_scale, color)
        binner = _binner_for(g.N, g.n, H, W, cfg, xy.device)
        bins = binner.bin(g, check=check)
        img = torch.empty((g.n, H, W), dtype=torch.float32, device=xy.device)
        render_forward(bins, cfg, img)
        ctx.save_for_backward(xy, theta, inv_scale, color)
        ctx.keep = (cfg, H, W, check)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        xy, theta, inv_scale, color = ctx.saved_tensors
        cfg, H, W, check = ctx.keep
        g = gaussians_view(xy, theta, inv_scale, color)
        binner = _binner_for(g.N, g.n, H, W, cfg, xy.device)
        bins = binner.bin(g, check=check)
        n = color.shape[1]
        grad = torch.empty((xy.shape[0], 5 + n), dtype=torch.float32, device=xy.device)
        render_backward(g, bins, cfg, grad_img.contiguous().float(), None, grad)
        return (grad[:, 0:2], grad[:, 2], grad[:, 3:5], grad[:, 5:], None, None, None, None)


def render(xy, theta, inv_scale, color, H, W, cfg=None, check=True):
    """Differentiable render (Eq. 5) -> planar float32 [n, H, W].

    check=True (default) synchronises once per call to re-bin with a larger
    capacity if the intersections overflowed; check=False keeps every call
    stream-ordered (graph-capturable after a first checked call has sized
    the cached workspace)."""
    return _RenderFn.apply(xy, theta, inv_scale, color, H, W, cfg or default_config(), check)


class Fitter:
    """The fitting schedule of Sec. 4.1 on one target, through the C ABI.

    It starts with N/2 Gaussians placed by Eq. 6 (gradient-guided, uniform
    share `lam`), then runs fit steps (`igs_fit_step`, or `igs_fit_step_half`
    with `storage` 'f16'/'bf16'). Every `add_every` steps it adds N/8
    Gaussians placed by Eq. 7 on the current rendering, until the budget N is
    reached. Buffers are sized for N up front. `graphs=True` replays each step
    from a CUDA graph captured per Gaussian count. The random numbers of the
    draws come from numpy's generator seeded with `seed`.
    """

    R53 = 1 << 53

    def __init__(self, target, N, cfg=None, lam=0.3, seed=0, start_frac=0.5, add_frac=0.125,
                 add_every=500, storage="f32", graphs=False, m_capacity=None):
        self.target = target.contiguous().float()
        self.n, self.H, self.W = self.target.shape
        self.budget = int(N)
        self.cfg = cfg or default_config()
        self.add_n = max(1, int(round(add_frac * N)))
        self.add_every = int(add_every)
        self.rng = np.random.default_rng(seed)
        dev = self.target.device
        np_ = 5 + self.n
        self.P = torch.zeros((N, np_), device=dev)
        self.G = torch.zeros_like(self.P)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.step_ctr = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.half = None
        if storage != "f32":
            self.half = torch.zeros((N, np_), dtype={"f16": torch.float16,
                                                      "bf16": torch.bfloat16}[storage],
                                    device=dev)
        self.m_capacity = int(m_capacity or 16 * N + 4096)
        self.ws = alloc_workspace(workspace_size(N, self.n, self.H, self.W, self.cfg,
                                                 self.m_capacity), dev)
        self.pws = alloc_workspace(placement_workspace_size(self.H, self.W), dev)
        n0 = max(1, int(round(start_frac * N)))
        init_gaussians(self.target, n0, self._rand(n0), self.P, self.pws, lam=lam)
        self.state = FitState(self.P.data_ptr(), self.G.data_ptr(), self.m.data_ptr(),
                              self.v.data_ptr(), self.step_ctr.data_ptr(), n0, self.n)
        self.steps = 0
        self.graphs = graphs
        self._graph = None
        self._graph_n = -1

    def _rand(self, count):
        r = self.rng.integers(0, self.R53, (count, 2), dtype=np.int64)
        return torch.from_numpy(r).to(self.target.device)

    @property
    def N(self):
        return int(self.state.N)

    @property
    def params(self):
        return self.P[:self.N]

    def _one_step(self, stream=None):
        if self.half is None:
            fit_step(self.state, self.target, self.H, self.W, self.cfg, self.ws, self.m_capacity,
                     self.loss, stream=stream)
        else:
            fit_step_half(self.state, self.half, self.target, self.H, self.W, self.cfg, self.ws,
                          self.m_capacity, self.loss, stream=stream)

    def step(self):
        """One fit step (and the scheduled addition after it); returns the loss tensor."""
        if self.graphs:
            if self._graph_n != self.N:
                s = torch.cuda.Stream(device=self.target.device)
                s.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(s):
                    self._one_step(stream=s)     # this is the step itself
                torch.cuda.current_stream().wait_stream(s)
                self._graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self._graph):   # recorded, not run
                    self._one_step()
                self._graph_n = self.N
            else:
                self._graph.replay()
        else:
            self._one_step()
        self.steps += 1
        if self.add_every > 0 and self.steps % self.add_every == 0 and self.N < self.budget:
            self.add()
        return self.loss

    def render(self):
        """The current image [n, H, W] (from the stored parameters)."""
        src = self.params if self.half is None else self.half[:self.N]
        view = packed_view(src, self.n)
        bins = preprocess_bin(view, self.H, self.W, self.cfg, self.ws, self.m_capacity)
        img = torch.empty((self.n, self.H, self.W), device=self.target.device)
        render_forward(bins, self.cfg, img)
        return img

    def add(self):
        """Eq. 7: add min(N/8, room) Gaussians where the rendering errs most."""
        count = min(self.add_n, self.budget - self.N)
        if count <= 0:
            return
        img = self.render()
        add_gaussians(self.target, img, self._rand(count), count, self.state, self.pws)
        self.state.N = self.N + count
