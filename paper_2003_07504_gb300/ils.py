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
    """An ILS plan for C x H x W float32 images (ils_plan_create)."""

    def __init__(self, H: int, W: int, C: int = 1, lam: float = 1.0, p: float = 0.8,
                 eps: float = 1e-4, N: int = 4):
        self.H, self.W, self.C, self.N = int(H), int(W), int(C), int(N)
        self.lam, self.p, self.eps = float(lam), float(p), float(eps)
        L = _lib.lib()
        h = ctypes.c_void_p()
        _lib.check(L.ils_plan_create(self.H, self.W, self.C, self.lam, self.p, self.eps, self.N,
                                     ctypes.byref(h)), "ils_plan_create")
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
