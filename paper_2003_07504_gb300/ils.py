"""PyTorch-facing binding of libils.so: plans over device tensors.

PyTorch provides device memory and streams only; every arithmetic step of the
smoothing runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


def _stream_ptr(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _check_image(t: torch.Tensor, shape, name: str) -> None:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Plan:
    """An ILS plan for C x H x W float32 images (ils_plan_create).  penalty="welsch": ILS with
    the Welsch penalty of scale gamma (ils_plan_create_welsch); penalty="hqs": the
    half-quadratic-splitting comparison method with phi = |x|, weights beta0 kappa^n
    (ils_plan_create_hqs; beta0=None means 2 lam).  p and eps are unused by both."""

    def __init__(self, H: int, W: int, C: int = 1, lam: float = 1.0, p: float = 0.8,
                 eps: float = 1e-4, N: int = 4, penalty: str = "lp", gamma: float | None = None,
                 beta0: float | None = None, kappa: float = 2.0):
        self.H, self.W, self.C, self.N = int(H), int(W), int(C), int(N)
        self.lam, self.p, self.eps = float(lam), float(p), float(eps)
        self.penalty = penalty
        L = _lib.lib()
        h = ctypes.c_void_p()
        if penalty == "welsch":
            if gamma is None:
                raise ValueError("the Welsch penalty needs gamma")
            self.gamma = float(gamma)
            _lib.check(L.ils_plan_create_welsch(self.H, self.W, self.C, self.lam, self.gamma, self.N,
                                                ctypes.byref(h)), "ils_plan_create_welsch")
        elif penalty == "hqs":
            _lib.check(L.ils_plan_create_hqs(self.H, self.W, self.C, self.lam,
                                             0.0 if beta0 is None else float(beta0), float(kappa), self.N,
                                             ctypes.byref(h)), "ils_plan_create_hqs")
        elif penalty == "lp":
            _lib.check(L.ils_plan_create(self.H, self.W, self.C, self.lam, self.p, self.eps, self.N,
                                         ctypes.byref(h)), "ils_plan_create")
        else:
            raise ValueError(f"unknown penalty {penalty!r}")
        self._h = h

    @property
    def shape(self):
        return (self.C, self.H, self.W)

    @property
    def c(self) -> float:
        return float(_lib.lib().ils_plan_c(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ils_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _as3d(self, t):
        return t.view(self.shape) if t.dim() == 2 and self.C == 1 else t

    def smooth(self, f: torch.Tensor, out: torch.Tensor | None = None, u0: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        """u = ILS(f) (Algorithm 1), optionally started from u0 (warm start)."""
        f3 = self._as3d(f)
        _check_image(f3, self.shape, "f")
        if out is None:
            out = torch.empty_like(f)
        _check_image(self._as3d(out), self.shape, "out")
        L = _lib.lib()
        if u0 is None:
            st = L.ils_smooth(self._h, f.data_ptr(), out.data_ptr(), _stream_ptr(stream))
            _lib.check(st, "ils_smooth")
        else:
            _check_image(self._as3d(u0), self.shape, "u0")
            st = L.ils_smooth_from(self._h, f.data_ptr(), u0.data_ptr(), out.data_ptr(), _stream_ptr(stream))
            _lib.check(st, "ils_smooth_from")
        return out

    def enhance(self, f: torch.Tensor, k: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Detail enhancement u + k (f - u), u = ILS(f), in the final inverse pass."""
        _check_image(self._as3d(f), self.shape, "f")
        if out is None:
            out = torch.empty_like(f)
        _check_image(self._as3d(out), self.shape, "out")
        _lib.check(_lib.lib().ils_smooth_enhance(self._h, f.data_ptr(), out.data_ptr(), float(k),
                                                 _stream_ptr(stream)), "ils_smooth_enhance")
        return out

    def smooth_luma(self, rgb: torch.Tensor, k: float = 0.0, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
        """Luminance-only smoothing of a 3 x H x W RGB image (plan made with C = 1): every channel
        changes by the change of Y = 0.299 R + 0.587 G + 0.114 B; k > 0 boosts Y's details."""
        if self.C != 1:
            raise ValueError("smooth_luma needs a plan with C = 1")
        _check_image(rgb, (3, self.H, self.W), "rgb")
        if out is None:
            out = torch.empty_like(rgb)
        _check_image(out, (3, self.H, self.W), "out")
        _lib.check(_lib.lib().ils_smooth_luma(self._h, rgb.data_ptr(), out.data_ptr(), float(k),
                                              _stream_ptr(stream)), "ils_smooth_luma")
        return out

    def smooth_hwc(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """u = ILS(f) for a pixel-interleaved H x W x C image (the planar copy Algorithm 1 re-reads
        is made by a gather kernel; the final inverse pass writes u interleaved)."""
        _check_image(f, (self.H, self.W, self.C), "f")
        if out is None:
            out = torch.empty_like(f)
        _check_image(out, (self.H, self.W, self.C), "out")
        _lib.check(_lib.lib().ils_smooth_hwc(self._h, f.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
                   "ils_smooth_hwc")
        return out

    def smooth_presmoothed(self, f: torch.Tensor, sigma: float = 1.0, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
        """Texture smoothing (Sec. 5): ILS of the input pre-smoothed by a periodic Gaussian of
        standard deviation sigma (<= 5 pixels); the paper pairs it with a Welsch plan, N = 15."""
        _check_image(self._as3d(f), self.shape, "f")
        if out is None:
            out = torch.empty_like(f)
        _check_image(self._as3d(out), self.shape, "out")
        _lib.check(_lib.lib().ils_smooth_presmoothed(self._h, f.data_ptr(), out.data_ptr(), float(sigma),
                                                     _stream_ptr(stream)), "ils_smooth_presmoothed")
        return out

    def tonemap(self, rgb: torch.Tensor, s: float, k: float = 1.0, o: float = 0.0,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Single-scale HDR tone mapping of a 3 x H x W linear-radiance image (plan made with C = 1):
        b = ILS(l) of l = ln Y, l' = s b + k (l - b), out_c = rgb_c exp(l' - l + o)."""
        if self.C != 1:
            raise ValueError("tonemap needs a plan with C = 1")
        _check_image(rgb, (3, self.H, self.W), "rgb")
        if out is None:
            out = torch.empty_like(rgb)
        _check_image(out, (3, self.H, self.W), "out")
        _lib.check(_lib.lib().ils_tonemap_log(self._h, rgb.data_ptr(), out.data_ptr(), float(s), float(k), float(o),
                                              _stream_ptr(stream)), "ils_tonemap_log")
        return out

    def smooth_checkpointed(self, f: torch.Tensor, out: torch.Tensor | None = None,
                            u0: torch.Tensor | None = None, stream=None):
        """Forward pass that also returns the iterates u^0..u^{N-1} (N x C x H x W, caller-owned)
        for backward_ckpt()."""
        f3 = self._as3d(f)
        _check_image(f3, self.shape, "f")
        if out is None:
            out = torch.empty_like(f)
        _check_image(self._as3d(out), self.shape, "out")
        if u0 is not None:
            _check_image(self._as3d(u0), self.shape, "u0")
        ckpt = torch.empty((max(self.N, 1),) + self.shape, dtype=torch.float32, device=f.device)
        st = _lib.lib().ils_smooth_checkpointed(self._h, f.data_ptr(), 0 if u0 is None else u0.data_ptr(),
                                                out.data_ptr(), ckpt.data_ptr(), _stream_ptr(stream))
        _lib.check(st, "ils_smooth_checkpointed")
        return out, ckpt

    def backward_ckpt(self, ckpt: torch.Tensor, grad_u: torch.Tensor, separate_u0: bool = False, stream=None):
        """dL/df (and dL/du^0 if separate_u0) from dL/du^N and caller-owned checkpoints
        (ils_backward_ckpt)."""
        _check_image(self._as3d(grad_u), self.shape, "grad_u")
        if ckpt.dtype != torch.float32 or not ckpt.is_cuda or not ckpt.is_contiguous() or \
                tuple(ckpt.shape) != (max(self.N, 1),) + self.shape:
            raise ValueError("ckpt must come from smooth_checkpointed of this plan")
        grad_f = torch.empty_like(grad_u)
        grad_u0 = torch.empty_like(grad_u) if separate_u0 else None
        st = _lib.lib().ils_backward_ckpt(self._h, ckpt.data_ptr(), grad_u.data_ptr(), grad_f.data_ptr(),
                                          0 if grad_u0 is None else grad_u0.data_ptr(), _stream_ptr(stream))
        _lib.check(st, "ils_backward_ckpt")
        return (grad_f, grad_u0) if separate_u0 else grad_f

    def set_checkpointing(self, on: bool) -> None:
        """Plan-owned checkpoints (ils_set_checkpointing): later smooth() calls keep their
        iterates for backward()."""
        _lib.check(_lib.lib().ils_set_checkpointing(self._h, 1 if on else 0), "ils_set_checkpointing")

    def backward(self, f: torch.Tensor, grad_u: torch.Tensor, grad_f: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
        """dL/df through the last smooth() of this f made with checkpointing on (ils_backward)."""
        _check_image(self._as3d(f), self.shape, "f")
        _check_image(self._as3d(grad_u), self.shape, "grad_u")
        if grad_f is None:
            grad_f = torch.empty_like(grad_u)
        _check_image(self._as3d(grad_f), self.shape, "grad_f")
        st = _lib.lib().ils_backward(self._h, f.data_ptr(), grad_u.data_ptr(), grad_f.data_ptr(),
                                     _stream_ptr(stream))
        _lib.check(st, "ils_backward")
        return grad_f

    def set_profiling(self, on: bool) -> None:
        _lib.check(_lib.lib().ils_set_profiling(self._h, 1 if on else 0), "ils_set_profiling")

    def profile(self) -> dict:
        """{kind: (total_ms, launches)} accumulated since profiling was turned on."""
        n = len(_lib.KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _lib.check(_lib.lib().ils_get_profile(self._h, ms, cnt), "ils_get_profile")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_lib.KERNEL_KINDS)}

    def smooth_host(self, f_host: torch.Tensor, out_host: torch.Tensor, stream=None) -> torch.Tensor:
        """ILS on host (CPU) tensors; copies in and out inside the call and synchronizes."""
        for t, n in ((f_host, "f_host"), (out_host, "out_host")):
            if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != self.C * self.H * self.W:
                raise ValueError(f"{n} must be a contiguous float32 CPU tensor of {self.shape}")
        st = _lib.lib().ils_smooth_host(self._h, f_host.data_ptr(), out_host.data_ptr(), _stream_ptr(stream))
        _lib.check(st, "ils_smooth_host")
        return out_host


class Batch:
    """Frames of uneven size smoothed by one CUDA-graph launch (ils_batch_create / ils_batch_run).

    frames: sequence of (f, u, lam, p, eps, N) with f, u contiguous float32 CUDA tensors of
    shape (C, H, W) (or (H, W)).  The tensors must stay alive while the batch is used.
    """

    def __init__(self, frames, autotune: bool = False):
        arr = (_lib.Frame * len(frames))()
        self._keep = []
        for i, (f, u, lam, p, eps, N) in enumerate(frames):
            shape = (1, *f.shape) if f.dim() == 2 else tuple(f.shape)
            _check_image(f.view(shape), shape, "f")
            _check_image(u.view(shape), shape, "u")
            C, H, W = shape
            arr[i] = _lib.Frame(H, W, C, int(N), float(lam), float(p), float(eps), f.data_ptr(), u.data_ptr())
            self._keep.append((f, u))
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().ils_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(frames),
                                               1 if autotune else 0, ctypes.byref(h)), "ils_batch_create")
        self._h = h
        self.count = len(frames)

    def run(self, stream=None) -> None:
        _lib.check(_lib.lib().ils_batch_run(self._h, _stream_ptr(stream)), "ils_batch_run")

    def choice(self, i: int):
        """(branch, row kernel variant, column kernel variant) of frame i (-1 = generic kernels)."""
        r, c = ctypes.c_int(), ctypes.c_int()
        br = _lib.lib().ils_batch_kernel_choice(self._h, i, ctypes.byref(r), ctypes.byref(c))
        return br, r.value, c.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ils_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def smooth_batched(frames, stream=None) -> None:
    """One-shot batch: create, run, wait, destroy (ils_smooth_batched)."""
    arr = (_lib.Frame * len(frames))()
    for i, (f, u, lam, p, eps, N) in enumerate(frames):
        shape = (1, *f.shape) if f.dim() == 2 else tuple(f.shape)
        _check_image(f.view(shape), shape, "f")
        _check_image(u.view(shape), shape, "u")
        C, H, W = shape
        arr[i] = _lib.Frame(H, W, C, int(N), float(lam), float(p), float(eps), f.data_ptr(), u.data_ptr())
    _lib.check(_lib.lib().ils_smooth_batched(ctypes.cast(arr, ctypes.c_void_p), len(frames), _stream_ptr(stream)),
               "ils_smooth_batched")


class ILSFunction(torch.autograd.Function):
    """u = ILS(f) (optionally from a warm start u0) as a differentiable op.

    Forward keeps the iterates u^0..u^{N-1} (caller-owned checkpoints, one N x C x H x W
    tensor per call) and backward runs the library's hand-written adjoint on them.
    """

    @staticmethod
    def forward(ctx, f, plan, u0=None):
        fc = f.contiguous()
        u0c = None if u0 is None else u0.contiguous()
        u, ckpt = plan.smooth_checkpointed(fc, u0=u0c)
        ctx.plan = plan
        ctx.has_u0 = u0 is not None
        ctx.save_for_backward(ckpt)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (ckpt,) = ctx.saved_tensors
        g = grad_u.contiguous()
        if ctx.has_u0:
            gf, gu0 = ctx.plan.backward_ckpt(ckpt, g, separate_u0=True)
            return gf, None, gu0
        return ctx.plan.backward_ckpt(ckpt, g), None, None


def ils_function(f: torch.Tensor, plan: Plan, u0: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable ILS (see ILSFunction)."""
    return ILSFunction.apply(f, plan, u0)


_plans: dict = {}


def smooth(f: torch.Tensor, lam: float = 1.0, p: float = 0.8, eps: float = 1e-4, N: int = 4,
           u0: torch.Tensor | None = None) -> torch.Tensor:
    """ILS-smooth a (C,H,W) or (H,W) float32 CUDA tensor; plans are cached by shape and parameters."""
    shape = tuple(f.shape)
    C, H, W = (1, *shape) if len(shape) == 2 else shape
    key = (C, H, W, float(lam), float(p), float(eps), int(N), f.device.index)
    plan = _plans.get(key)
    if plan is None:
        with torch.cuda.device(f.device):
            plan = Plan(H, W, C, lam, p, eps, N)
        _plans[key] = plan
    return plan.smooth(f, u0=u0)


def log_luma(rgb: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """l = ln max(Y, 1e-12), Y = 0.299 R + 0.587 G + 0.114 B, of a 3 x H x W CUDA tensor: the
    log-luminance whose smoothing b = ILS(l) splits an HDR image into base b and detail l - b."""
    if rgb.dim() != 3 or rgb.shape[0] != 3:
        raise ValueError(f"rgb: expected shape (3, H, W), got {tuple(rgb.shape)}")
    H, W = int(rgb.shape[1]), int(rgb.shape[2])
    _check_image(rgb, (3, H, W), "rgb")
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=rgb.device)
    _check_image(out, (H, W), "out")
    _lib.check(_lib.lib().ils_log_luma(rgb.data_ptr(), out.data_ptr(), H, W, _stream_ptr(stream)), "ils_log_luma")
    return out


def gaussian_blur(f: torch.Tensor, sigma: float, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Separable periodic Gaussian blur (taps r = ceil(3 sigma), normalized) of a (C, H, W) or
    (H, W) float32 CUDA tensor; 0 <= sigma <= 5."""
    shape = tuple(f.shape)
    C, H, W = (1, *shape) if len(shape) == 2 else shape
    _check_image(f, shape, "f")
    if out is None:
        out = torch.empty_like(f)
    _check_image(out, shape, "out")
    _lib.check(_lib.lib().ils_gaussian_blur(f.data_ptr(), out.data_ptr(), H, W, C, float(sigma), _stream_ptr(stream)),
               "ils_gaussian_blur")
    return out
