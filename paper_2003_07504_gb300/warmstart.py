"""Learned warm start for ILS (not in the paper): u^0 = f + net(f), trained on the GPU by
the library's own tensor-core forward/backward kernels to predict plain ILS N=4 output,
then 1-2 ILS iterations from u^0, with plain ILS as the fallback (ils_warm_*).

PyTorch is used for device memory and streams only; every arithmetic step of the network,
the loss, the optimizer and the smoothing runs in libils.so.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _lib, synth
from .ils import Plan, _stream_ptr

LAYERS = [(3, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 3)]
WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_WEIGHTS = os.path.join(WEIGHTS_DIR, "warmstart_lam1_p08_N4.npy")
# Fallback threshold on the last iterate change max|u^k - u^{k-1}|: about twice the largest
# change seen after one warm iteration on held-out synthetic frames (0.024), so only inputs
# on which the network is far off its training distribution fall back to plain ILS.
DEFAULT_TAU = 0.05


def param_count() -> int:
    return int(_lib.lib().ils_cnn_param_count())


def init_params(seed: int = 0, last_scale: float = 1e-3) -> np.ndarray:
    """He-normal weights, zero biases; the last layer starts near zero so u^0 starts near f."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (ci * 9)) * (last_scale if i == len(LAYERS) - 1 else 1.0)
        parts.append(rng.normal(0.0, std, size=(co, ci, 3, 3)).ravel())
        parts.append(np.zeros(co))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == param_count()
    return p


def unpack_params(p: np.ndarray):
    """Flat parameter vector -> ([W per layer], [b per layer]) (PyTorch conv layouts)."""
    ws, bs, off = [], [], 0
    for ci, co in LAYERS:
        n = co * ci * 9
        ws.append(p[off:off + n].reshape(co, ci, 3, 3))
        off += n
        bs.append(p[off:off + co])
        off += co
    return ws, bs


class WarmStartNet:
    """The network (ils_cnn): batches of RGB frames, B x 3 x H x W FP32 on the device."""

    def __init__(self, max_pixels: int, params: np.ndarray | None = None):
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().ils_cnn_create(int(max_pixels), ctypes.byref(h)), "ils_cnn_create")
        self._h = h
        self.set_params(init_params() if params is None else params)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ils_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: np.ndarray) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        _lib.check(_lib.lib().ils_cnn_set_weights(self._h, p.ctypes.data, p.size), "ils_cnn_set_weights")

    def get_params(self) -> np.ndarray:
        p = np.empty(param_count(), np.float32)
        _lib.check(_lib.lib().ils_cnn_get_weights(self._h, p.ctypes.data, p.size), "ils_cnn_get_weights")
        return p

    def get_grads(self) -> np.ndarray:
        g = np.empty(param_count(), np.float32)
        _lib.check(_lib.lib().ils_cnn_get_grads(self._h, g.ctypes.data, g.size), "ils_cnn_get_grads")
        return g

    def get_adam(self):
        """(m, v, step): Adam moments in parameter order and the bias-correction step count."""
        m = np.empty(param_count(), np.float32)
        v = np.empty(param_count(), np.float32)
        step = ctypes.c_longlong(0)
        _lib.check(_lib.lib().ils_cnn_get_adam(self._h, m.ctypes.data, v.ctypes.data, m.size, ctypes.byref(step)),
                   "ils_cnn_get_adam")
        return m, v, int(step.value)

    def set_adam(self, m: np.ndarray, v: np.ndarray, step: int) -> None:
        """Restore Adam state (after set_params, which resets it)."""
        m = np.ascontiguousarray(m, dtype=np.float32)
        v = np.ascontiguousarray(v, dtype=np.float32)
        _lib.check(_lib.lib().ils_cnn_set_adam(self._h, m.ctypes.data, v.ctypes.data, m.size, int(step)),
                   "ils_cnn_set_adam")

    @staticmethod
    def _shape(f):
        if f.dim() != 4 or f.shape[1] != 3 or f.dtype != torch.float32 or not f.is_cuda or not f.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor of shape (B, 3, H, W)")
        return f.shape[0], f.shape[2], f.shape[3]

    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        B, H, W = self._shape(f)
        out = torch.empty_like(f) if out is None else out
        _lib.check(_lib.lib().ils_cnn_forward(self._h, B, H, W, f.data_ptr(), out.data_ptr(), _stream_ptr()),
                   "ils_cnn_forward")
        return out

    def infer(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """u0 = f + net(f) without keeping activations (two fused tensor-core kernels)."""
        B, H, W = self._shape(f)
        out = torch.empty_like(f) if out is None else out
        _lib.check(_lib.lib().ils_cnn_infer(self._h, B, H, W, f.data_ptr(), out.data_ptr(), _stream_ptr()),
                   "ils_cnn_infer")
        return out

    def backward(self, f: torch.Tensor, grad_u0: torch.Tensor) -> None:
        B, H, W = self._shape(f)
        self._shape(grad_u0)
        _lib.check(_lib.lib().ils_cnn_backward(self._h, B, H, W, f.data_ptr(), grad_u0.data_ptr(), _stream_ptr()),
                   "ils_cnn_backward")

    @property
    def uses_tcgen05(self) -> bool:
        return bool(_lib.lib().ils_cnn_uses_tcgen05(self._h))

    def check(self) -> None:
        """Raise if a tensor-core kernel's bounded wait gave up (ILS_ERR_TIMEOUT)."""
        _lib.check(_lib.lib().ils_cnn_check(self._h), "ils_cnn_check")

    def zero_grad(self) -> None:
        _lib.check(_lib.lib().ils_cnn_zero_grad(self._h, _stream_ptr()), "ils_cnn_zero_grad")

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
        _lib.check(_lib.lib().ils_cnn_adam_step(self._h, lr, beta1, beta2, eps, _stream_ptr()), "ils_cnn_adam_step")


def mse(u0: torch.Tensor, target: torch.Tensor, grad: torch.Tensor, loss: torch.Tensor) -> None:
    """grad = 2 (u0 - target)/n; loss (1-element FP32 device tensor) += mean squared error."""
    _lib.check(_lib.lib().ils_mse(u0.data_ptr(), target.data_ptr(), grad.data_ptr(), u0.numel(), loss.data_ptr(),
                                  _stream_ptr()), "ils_mse")


class WarmSmoother:
    """u = ILS_iters(f; u^0 = f + net(f)), or plain ILS N=n_plain when the last change > tau."""

    def __init__(self, net: WarmStartNet, H: int, W: int, C: int = 3, lam: float = 1.0, p: float = 0.8,
                 eps: float = 1e-4, iters: int = 1, n_plain: int = 4, tau: float = DEFAULT_TAU):
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().ils_warm_create(H, W, C, lam, p, eps, iters, n_plain, tau, net._h, ctypes.byref(h)),
                   "ils_warm_create")
        self._h = h
        self.net = net
        self.shape = (C, H, W)

    def smooth(self, f: torch.Tensor, out: torch.Tensor | None = None):
        """(u, fallback taken, delta): waits for the call's stream to report the decision."""
        out = torch.empty_like(f) if out is None else out
        fb = ctypes.c_int()
        d = ctypes.c_float()
        _lib.check(_lib.lib().ils_warm_smooth(self._h, f.data_ptr(), out.data_ptr(), ctypes.byref(fb), ctypes.byref(d),
                                              _stream_ptr()), "ils_warm_smooth")
        return out, fb.value == _lib.ILS_ERR_FALLBACK_TAKEN, float(d.value)

    def smooth_async(self, f: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """u without waiting: the fallback decision is taken on the device; result() reads it
        once the stream has been synchronized."""
        out = torch.empty_like(f) if out is None else out
        _lib.check(_lib.lib().ils_warm_smooth(self._h, f.data_ptr(), out.data_ptr(), None, None, _stream_ptr()),
                   "ils_warm_smooth")
        return out

    def result(self):
        """(fallback taken, delta) of the last call (after its stream has been synchronized)."""
        fb = ctypes.c_int()
        d = ctypes.c_float()
        _lib.check(_lib.lib().ils_warm_result(self._h, ctypes.byref(fb), ctypes.byref(d)), "ils_warm_result")
        return fb.value == _lib.ILS_ERR_FALLBACK_TAKEN, float(d.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().ils_warm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- training

def crop_pool(n_images: int, size: int, seed: int) -> np.ndarray:
    """Source images for training crops: the small-image generator (12 regions per 256 x 256
    area, texture period 4-8 px, noise 0.02) at size x size, RGB."""
    K = max(12, int(12 * (size / 256) ** 2))
    return np.stack([synth.voronoi_texture(size, size, 3, K=K, A=0.05, Tmin=4, Tmax=8, sigma=0.02,
                                           seed=seed + i) for i in range(n_images)])


def save_checkpoint(path: str, net: "WarmStartNet", step: int, losses, best) -> None:
    """Training state after `step` steps: weights, Adam moments and step count, the loss log
    and the best snapshot (npz; the data order and learning-rate schedule follow from step)."""
    m, v, t = net.get_adam()
    tmp = path + ".tmp.npz"
    np.savez(tmp, params=net.get_params(), adam_m=m, adam_v=v, adam_t=t, step=step,
             losses=np.asarray(losses, dtype=np.float64).reshape(-1, 2),
             best_loss=np.inf if best is None else best[0],
             best_params=net.get_params() if best is None else best[1])
    os.replace(tmp, path)


def train(steps: int = 600, batch: int = 16, crop: int = 256, lr: float = 1e-3, lam: float = 1.0, p: float = 0.8,
          eps: float = 1e-4, N: int = 4, n_crops: int = 20000, seed: int = 0, log_every: int = 50,
          params: np.ndarray | None = None, pool_images: int = 24, pool_size: int = 1024, verbose: bool = True,
          warmup: int = 200, checkpoint: str | None = None, checkpoint_every: int = 500, resume: str | None = None,
          stop_after: int | None = None):
    """Train the network on (f, ILS_N(f)) pairs of random crops; returns (params, losses).

    The crops are the first n_crops of a seeded sequence of (image, offset) draws from a pool
    of generated images; targets are computed on the GPU by plain ILS N=N (this library).
    Learning rate: linear warm-up over `warmup` steps, then cosine decay.  The returned
    parameters are those at the lowest logged loss (a ReLU network can collapse to a
    constant output after one large step; the snapshot keeps the last good state).
    checkpoint: file written every `checkpoint_every` steps and at the end (save_checkpoint);
    resume: such a file to continue from (same seed, batch and schedule arguments);
    stop_after: end after that many steps of the `steps`-long schedule (an interrupted run;
    the checkpoint, if any, is written there).
    """
    dev = torch.device("cuda")
    pool = torch.from_numpy(crop_pool(pool_images, pool_size, seed=7000 + seed)).to(dev)
    rng = np.random.default_rng(seed)
    draws = np.stack([rng.integers(0, pool_images, n_crops), rng.integers(0, pool_size - crop + 1, n_crops),
                      rng.integers(0, pool_size - crop + 1, n_crops)], axis=1)
    net = WarmStartNet(batch * crop * crop, params)
    plan = Plan(crop, crop, 3 * batch, lam, p, eps, N)
    f = torch.empty(batch, 3, crop, crop, device=dev)
    target = torch.empty_like(f)
    grad = torch.empty_like(f)
    loss = torch.zeros(1, device=dev)
    losses = []
    best = None
    start = 0
    if resume is not None:
        ck = np.load(resume)
        net.set_params(ck["params"])
        net.set_adam(ck["adam_m"], ck["adam_v"], int(ck["adam_t"]))
        start = int(ck["step"])
        losses = [(int(a), float(b)) for a, b in ck["losses"]]
        if np.isfinite(float(ck["best_loss"])):
            best = (float(ck["best_loss"]), ck["best_params"].astype(np.float32))
    cursor = start * batch
    end = steps if stop_after is None else min(steps, stop_after)
    for step in range(start, end):
        for i in range(batch):
            k, y, x = draws[cursor % n_crops]
            cursor += 1
            f[i] = pool[k, :, y:y + crop, x:x + crop]
        plan.smooth(f.view(3 * batch, crop, crop), out=target.view(3 * batch, crop, crop))
        loss.zero_()
        u0 = net.forward(f)
        mse(u0, target, grad, loss)
        net.zero_grad()
        net.backward(f, grad)
        scale = min(1.0, (step + 1) / max(1, warmup)) * 0.5 * (1 + np.cos(np.pi * step / steps))
        net.adam_step(lr * scale)
        if step % log_every == 0 or step == steps - 1:
            losses.append((step, float(loss.item())))
            if best is None or losses[-1][1] < best[0]:
                best = (losses[-1][1], net.get_params())
            if verbose:
                print(f"step {step:5d}  mse {losses[-1][1]:.3e}", flush=True)
        if checkpoint is not None and ((step + 1) % checkpoint_every == 0 or step == end - 1):
            save_checkpoint(checkpoint, net, step + 1, losses, best)
    if best is None:   # resumed at the end: nothing left to run
        best = (float("inf"), net.get_params())
    params = best[1]
    plan.close()
    net.close()
    return params, losses


def load_params(path: str = DEFAULT_WEIGHTS) -> np.ndarray:
    return np.load(path).astype(np.float32)


def converged_ils(plan_factory, f: torch.Tensor, max_iters: int = 20000, tol: float = 1e-6, chunk: int = 50):
    """ILS from f iterated until max|u^{n+1} - u^n| < tol (or max_iters): the 'converged ILS'
    reference of the equal-error comparison.  Runs in chunks of `chunk` iterations.
    Returns (u, iterations, last change max|u^{n+1} - u^n|)."""
    C, H, W = f.shape
    with plan_factory(H, W, C, chunk) as big, plan_factory(H, W, C, 1) as one:
        u = f.clone()
        done = 0
        change = float("inf")
        while done < max_iters:
            u = big.smooth(f, u0=u)
            done += chunk
            nxt = one.smooth(f, u0=u)
            change = float((nxt - u).abs().max())
            done += 1
            u = nxt
            if change < tol:
                break
        return u, done, change


def stationarity_residual(u: torch.Tensor, f: torch.Tensor, lam: float, p: float, eps: float) -> float:
    """max |(u - f) + (lambda/2) sum_* grad_*^T phi_p'(grad_* u)| over the image, in FP64 on the host:
    half the gradient of Eq. 1 (periodic forward differences), zero at a stationary point."""
    uu = u.detach().double().cpu().numpy()
    ff = f.detach().double().cpu().numpy()
    res = uu - ff
    for ax in (-1, -2):
        g = np.roll(uu, -1, axis=ax) - uu
        d = p * g * (g * g + eps) ** (p / 2.0 - 1.0)
        res += 0.5 * lam * (np.roll(d, 1, axis=ax) - d)
    return float(np.abs(res).max())


def main(argv=None):
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description="train the ILS warm-start network on the GPU")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--crop", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--n-crops", type=int, default=20000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--checkpoint", default=None, help="training-state file, written every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", default=None, help="continue training from a --checkpoint file")
    ap.add_argument("--smooth", metavar="HxW", default=None,
                    help="instead of training: warm-started smoothing (1 ILS iteration) of a synthetic RGB "
                         "frame of this size with the weights in --out, repeated --repeat times")
    ap.add_argument("--repeat", type=int, default=3)
    a = ap.parse_args(argv)
    if a.smooth is not None:
        from . import synth
        H, W = (int(v) for v in a.smooth.lower().split("x"))
        f = torch.from_numpy(synth.preset_image(H, W, 3, "hd", a.seed)).cuda()
        net = WarmStartNet(H * W, load_params(a.out))
        sm = WarmSmoother(net, H, W, 3, iters=1)
        times = []
        for _ in range(a.repeat):
            torch.cuda.synchronize()
            t = time.perf_counter()
            u, fb, d = sm.smooth(f)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        net.check()
        print(json.dumps({"frame": [3, H, W], "fallback": fb, "last_change": d, "seconds": times}))
        sm.close()
        net.close()
        return
    t0 = time.time()
    params, losses = train(steps=a.steps, batch=a.batch, crop=a.crop, lr=a.lr, n_crops=a.n_crops, seed=a.seed,
                           checkpoint=a.checkpoint, checkpoint_every=a.checkpoint_every, resume=a.resume)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, params)
    print(json.dumps({"out": a.out, "seconds": time.time() - t0, "losses": losses}))


if __name__ == "__main__":
    main()
