"""FP64 CPU oracle for Iterative Least Squares (ILS) smoothing.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The product library never does, and this module imports nothing from
the product package: the two share no kernels, tables, helpers or constants.

Everything here follows Liu et al., "Real-time Image Smoothing via Iterative
Least Squares" (arXiv 2003.07504).  Equations are numbered in the order the
paper's LaTeX source numbers them:

  Eq. 1  objective  E(u,f) = sum_s (u_s-f_s)^2 + lam * sum_{*=x,y} phi_p(grad_* u_s)   (Sec. 3)
  Eq. 2  generalized Charbonnier penalty  phi_p(x) = (x^2+eps)^(p/2)                  (Sec. 3)
  Eq. 7  half-quadratic auxiliary update  mu = c*grad u - phi_p'(grad u)              (Sec. 3.1)
  Eq. 8  the per-iteration least-squares problem (ILS)                                (Sec. 3.2)
  Eq. 9  its periodic-boundary FFT solution                                           (Sec. 3.2)
  Eq. 11 c >= c0 = p*eps^(p/2-1), with c = c0 used throughout                         (Sec. 3.3, App. B)
  Eq. 12-14 half-quadratic splitting (the comparison method), Eq. 15-17 its Huber view  (Sec. 3.5)
  Eq. 18 Welsch penalty phi_W;  Eq. 19 its mu update;  Eq. 20 its c0 = 2              (Sec. 3.5, Sec. 5)
  Algorithm 1: u^0 = f; for n = 0..N-1: mu^n from u^n (Eq. 7), u^{n+1} from Eq. 9.
  Sec. 3.4: colour images are smoothed one RGB channel at a time (option II), or the
            luminance only (option I).
  Sec. 4.2: HDR tone mapping smooths the logarithm of the luminance (base / detail split).
  Sec. 5:   texture smoothing pre-smooths the input with a small Gaussian before the Welsch ILS.

Arithmetic is float64 throughout.  The 2-D DFT is the naive separable DFT: an
explicit n x n DFT matrix applied along rows and then columns (a matrix product
is the only library primitive used).  No blocking, fusion or reordering beyond
what the equations state.

Readings of points the paper leaves open (each is also listed with the design
notes of the repository):
  * gradients are forward differences with periodic wrap,
      (grad_x u)[y,x] = u[y,(x+1)%W] - u[y,x],  (grad_y u)[y,x] = u[(y+1)%H,x] - u[y,x];
    the "inverse direction" derivative of Sec. 3.2 is the transpose,
      (grad_x^T m)[y,x] = m[y,(x-1)%W] - m[y,x]   (likewise for y);
  * forward DFT uses exp(-2*pi*i*jk/n), the inverse exp(+...)/n; the real part of
    the inverse is the result (the exact result is real);
  * u^0 = f unless a warm start u0 is given; no clipping of u;
  * c = c0 exactly;
  * the applications' unstated choices (BT.601 luma, natural log with a 1e-12 floor, the
    linear base compression of the tone mapping, the Gaussian's 3-sigma truncation and
    periodic boundary, sigma = 1) are stated in the docstrings of the functions that make them.
Every function is pinned by tests/test_oracle_pins.py against facts the paper or the
mathematics fix; the paper's energy-decrease percentages (74-90 % at N = 4, measured on its
photographs) are the one statement left unpinned ("parity unpinned"), the tests check the
monotone decrease instead.
"""
from __future__ import annotations

import functools

import numpy as np

__all__ = [
    "c0", "phi_p", "dphi_p", "d2phi_p", "g2", "mu_update",
    "grad_x", "grad_y", "grad_x_T", "grad_y_T",
    "dft_matrix", "dft2", "idft2", "gradient_transfer_functions", "denominator",
    "solve_eq9", "ils_iteration", "ils_smooth", "ils_channel", "energy", "ils_backward",
    "conv3x3", "warmstart_cnn_forward", "bf16_round", "warmstart_forward_bf16", "warmstart_backward_bf16",
    "adam_step",
    "C0_WELSCH", "phi_welsch", "dphi_welsch", "d2phi_welsch", "g2_welsch", "mu_welsch",
    "ils_channel_welsch", "ils_smooth_welsch", "energy_welsch", "ils_backward_welsch",
    "LUMA_BT601", "luma", "detail_enhance", "ils_smooth_luma",
    "LUMA_FLOOR", "log_luma", "tonemap_log", "hwc_to_planar", "planar_to_hwc", "ils_smooth_hwc",
    "gaussian_weights", "gaussian_blur_periodic", "texture_smooth",
    "hqs_shrink_l1", "hqs_channel", "hqs_smooth",
]


# ----------------------------------------------------------------------------
# Penalty and half-quadratic pieces (Eq. 2, Eq. 7, Eq. 11, Appendix B)
# ----------------------------------------------------------------------------

def c0(p: float, eps: float) -> float:
    """Smallest constant keeping g(x) = c/2 x^2 - phi_p(x) convex: c0 = p*eps^(p/2-1).

    Eq. 11 (Sec. 3.3) and Appendix B (h(0) = p*eps^(p/2-1)).
    """
    return float(p) * float(eps) ** (float(p) / 2.0 - 1.0)


def phi_p(x, p, eps):
    """Generalized Charbonnier penalty, Eq. 2: (x^2 + eps)^(p/2)."""
    x = np.asarray(x, dtype=np.float64)
    return (x * x + eps) ** (p / 2.0)


def dphi_p(x, p, eps):
    """phi_p'(x) = p * x * (x^2 + eps)^(p/2 - 1), the derivative written out in Eq. 7."""
    x = np.asarray(x, dtype=np.float64)
    return p * x * (x * x + eps) ** (p / 2.0 - 1.0)


def d2phi_p(x, p, eps):
    """phi_p''(x) = p (x^2+eps)^(p/2-2) [(p-1) x^2 + eps]: the h(x) of Appendix B."""
    x = np.asarray(x, dtype=np.float64)
    return p * (x * x + eps) ** (p / 2.0 - 2.0) * ((p - 1.0) * x * x + eps)


def g2(x, p, eps, c):
    """g''(x) = c - p (x^2+eps)^(p/2-2) [(p-1) x^2 + eps]  (Appendix B).

    This is also d mu / d x for the mu of Eq. 7, which the adjoint needs.
    """
    return c - d2phi_p(x, p, eps)


def mu_update(x, p, eps, c):
    """Eq. 7: mu = c*x - p*x*(x^2+eps)^(p/2-1), elementwise on a gradient field x."""
    x = np.asarray(x, dtype=np.float64)
    return c * x - p * x * (x * x + eps) ** (p / 2.0 - 1.0)


# ----------------------------------------------------------------------------
# Discrete differential operators (Sec. 3: [1,-1] and [1,-1]^T; Sec. 3.2: the
# inverse-direction derivative).  Periodic boundary, as the FFT solve assumes.
# ----------------------------------------------------------------------------

def grad_x(u):
    """(grad_x u)[y,x] = u[y,x+1] - u[y,x], periodic in x."""
    return np.roll(u, -1, axis=-1) - u


def grad_y(u):
    """(grad_y u)[y,x] = u[y+1,x] - u[y,x], periodic in y."""
    return np.roll(u, -1, axis=-2) - u


def grad_x_T(m):
    """Transpose of grad_x (the 'inverse direction' derivative of Sec. 3.2)."""
    return np.roll(m, 1, axis=-1) - m


def grad_y_T(m):
    """Transpose of grad_y."""
    return np.roll(m, 1, axis=-2) - m


# ----------------------------------------------------------------------------
# Naive separable DFT (the F and F^{-1} of Eq. 9)
# ----------------------------------------------------------------------------

@functools.lru_cache(maxsize=16)
def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    """Explicit n x n DFT matrix  F[j,k] = exp(sign * 2*pi*i * j*k / n).

    The product j*k is reduced mod n before the angle is formed so the twiddle
    keeps full float64 accuracy for large n.
    """
    j = np.arange(n, dtype=np.int64)
    m = np.outer(j, j) % n
    F = np.exp(sign * 2j * np.pi * m.astype(np.float64) / n)
    F.setflags(write=False)
    return F


def dft2(x: np.ndarray) -> np.ndarray:
    """Forward 2-D DFT of an H x W array: the row DFT, then the column DFT."""
    H, W = x.shape
    rows = np.asarray(x, dtype=np.complex128) @ dft_matrix(W, -1)   # DFT along x (F symmetric)
    return dft_matrix(H, -1) @ rows                                 # DFT along y


def idft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2-D DFT (sign +, scaled by 1/(H*W))."""
    H, W = X.shape
    rows = np.asarray(X, dtype=np.complex128) @ dft_matrix(W, +1)
    return (dft_matrix(H, +1) @ rows) / (H * W)


def gradient_transfer_functions(H: int, W: int):
    """F(grad_x) and F(grad_y): the DFT of the impulse responses of the two
    difference operators, as Eq. 9 writes them.

    grad_x u = u (*) h_x (circular convolution) with h_x[0,0] = -1, h_x[0,-1] = +1;
    grad_y likewise along y.
    """
    hx = np.zeros((H, W))
    hx[0, 0] = -1.0
    hx[0, (W - 1) % W] += 1.0
    hy = np.zeros((H, W))
    hy[0, 0] = -1.0
    hy[(H - 1) % H, 0] += 1.0
    return dft2(hx), dft2(hy)


def denominator(H: int, W: int, lam: float, c: float, Fdx=None, Fdy=None) -> np.ndarray:
    """Eq. 9 denominator: F(1) + (c/2) lam (conj(F grad_x) F grad_x + conj(F grad_y) F grad_y).

    F(1) is the DFT of the unit impulse, i.e. all ones.
    """
    if Fdx is None or Fdy is None:
        Fdx, Fdy = gradient_transfer_functions(H, W)
    delta = np.zeros((H, W))
    delta[0, 0] = 1.0
    F1 = dft2(delta)
    return F1 + (c / 2.0) * lam * (np.conj(Fdx) * Fdx + np.conj(Fdy) * Fdy)


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------

def solve_eq9(Ff, mu_x, mu_y, lam, den, Fdx, Fdy):
    """Eq. 9: F^{-1}[(F(f) + lam/2 (conj(F grad_x) F(mu_x) + conj(F grad_y) F(mu_y))) / den],
    the minimizer of the Eq. 8 least-squares problem for fixed mu (real part taken)."""
    num = Ff + (lam / 2.0) * (np.conj(Fdx) * dft2(mu_x) + np.conj(Fdy) * dft2(mu_y))
    return np.real(idft2(num / den))


def ils_iteration(u, f, lam, p, eps, c, Ff, den, Fdx, Fdy):
    """One pass of Algorithm 1's loop body on one channel.

    Step 1: mu^n_* from grad_* u^n by Eq. 7.
    Step 2: u^{n+1} by Eq. 9 (solve_eq9).
    """
    mu_x = mu_update(grad_x(u), p, eps, c)
    mu_y = mu_update(grad_y(u), p, eps, c)
    return solve_eq9(Ff, mu_x, mu_y, lam, den, Fdx, Fdy)


def ils_channel(f, lam, p, eps, N, u0=None, c=None, return_iterates=False):
    """Algorithm 1 on one H x W channel (float64).  Returns u^N (and u^0..u^N)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    if c is None:
        c = c0(p, eps)
    Fdx, Fdy = gradient_transfer_functions(H, W)
    den = denominator(H, W, lam, c, Fdx, Fdy)   # pre-computed once (Algorithm 1, input line)
    Ff = dft2(f)                                 # pre-computed once
    u = f.copy() if u0 is None else np.asarray(u0, dtype=np.float64).copy()
    iterates = [u.copy()]
    for _ in range(int(N)):
        u = ils_iteration(u, f, lam, p, eps, c, Ff, den, Fdx, Fdy)
        if return_iterates:
            iterates.append(u.copy())
    return (u, iterates) if return_iterates else u


def ils_smooth(f, lam=1.0, p=0.8, eps=1e-4, N=4, u0=None, c=None):
    """ILS on a C x H x W (or H x W) image, channels independent (Sec. 3.4)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        return ils_channel(f, lam, p, eps, N, u0, c)
    out = np.empty_like(f)
    for ch in range(f.shape[0]):
        out[ch] = ils_channel(f[ch], lam, p, eps, N, None if u0 is None else u0[ch], c)
    return out


def energy(u, f, lam, p, eps):
    """Eq. 1 with the penalty of Eq. 2, periodic forward differences."""
    u = np.asarray(u, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    return float(np.sum((u - f) ** 2)
                 + lam * np.sum(phi_p(grad_x(u), p, eps))
                 + lam * np.sum(phi_p(grad_y(u), p, eps)))


# ----------------------------------------------------------------------------
# ILS with the Welsch penalty (Sec. 5): the same additive half-quadratic procedure
# with phi_W in place of phi_p, the mu update of Eq. 19 and c0 = 2 (Eq. 20).
# ----------------------------------------------------------------------------

C0_WELSCH = 2.0  # Eq. 20 (proof: Appendix B, Eq. 24): c >= h(0) = 2


def phi_welsch(x, gamma):
    """Welsch penalty of Eq. 18, phi_W(x) = 2 gamma^2 (1 - exp(-x^2 / (2 gamma^2))).

    Reading: the exponent is printed without its minus sign in Eq. 18; the derivative the
    paper uses in Eq. 19, 2 x exp(-x^2/(2 gamma^2)), and the bounded penalty the text
    describes both fix it as exp(-x^2/(2 gamma^2)).
    """
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * gamma * gamma * (1.0 - np.exp(-x * x / (2.0 * gamma * gamma)))


def dphi_welsch(x, gamma):
    """phi_W'(x) = 2 x exp(-x^2 / (2 gamma^2)), as written out in Eq. 19."""
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * x * np.exp(-x * x / (2.0 * gamma * gamma))


def d2phi_welsch(x, gamma):
    """phi_W''(x) = 2 exp(-x^2/(2 gamma^2)) (1 - x^2/gamma^2): the h(x) of Appendix B
    (written there with kappa for gamma)."""
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * np.exp(-x * x / (2.0 * gamma * gamma)) * (1.0 - x * x / (gamma * gamma))


def g2_welsch(x, gamma, c):
    """g''(x) = c - phi_W''(x) (Appendix B), the derivative of the Eq. 19 mu."""
    return c - d2phi_welsch(x, gamma)


def mu_welsch(x, gamma, c):
    """Eq. 19: mu = c*x - 2 x exp(-x^2 / (2 gamma^2))."""
    x = np.asarray(x, dtype=np.float64)
    return c * x - dphi_welsch(x, gamma)


def ils_channel_welsch(f, lam, gamma, N, u0=None, c=None, return_iterates=False):
    """Algorithm 1 with the Welsch penalty on one H x W channel (float64): mu^n by Eq. 19,
    u^{n+1} by Eq. 9 with c = c0 = 2 (Eq. 20) in the denominator."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    if c is None:
        c = C0_WELSCH
    Fdx, Fdy = gradient_transfer_functions(H, W)
    den = denominator(H, W, lam, c, Fdx, Fdy)
    Ff = dft2(f)
    u = f.copy() if u0 is None else np.asarray(u0, dtype=np.float64).copy()
    iterates = [u.copy()]
    for _ in range(int(N)):
        mu_x = mu_welsch(grad_x(u), gamma, c)
        mu_y = mu_welsch(grad_y(u), gamma, c)
        u = solve_eq9(Ff, mu_x, mu_y, lam, den, Fdx, Fdy)
        if return_iterates:
            iterates.append(u.copy())
    return (u, iterates) if return_iterates else u


def ils_smooth_welsch(f, lam=20.0, gamma=10.0 / 255.0, N=10, u0=None, c=None):
    """Welsch-penalty ILS on a C x H x W (or H x W) image, channels independent (Sec. 3.4)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        return ils_channel_welsch(f, lam, gamma, N, u0, c)
    out = np.empty_like(f)
    for ch in range(f.shape[0]):
        out[ch] = ils_channel_welsch(f[ch], lam, gamma, N, None if u0 is None else u0[ch], c)
    return out


def energy_welsch(u, f, lam, gamma):
    """Eq. 1 with the Welsch penalty phi_W of Eq. 18."""
    u = np.asarray(u, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    return float(np.sum((u - f) ** 2)
                 + lam * np.sum(phi_welsch(grad_x(u), gamma))
                 + lam * np.sum(phi_welsch(grad_y(u), gamma)))


def ils_backward_welsch(f, grad_u, lam, gamma, N, c=None, u0=None, split=False):
    """Gradient of <grad_u, u^N(f)> for the Welsch ILS: the chain rule of ils_backward with
    g'' = c - phi_W'' (Appendix B)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    if c is None:
        c = C0_WELSCH
    _, iterates = ils_channel_welsch(f, lam, gamma, N, u0=u0, c=c, return_iterates=True)
    den = denominator(H, W, lam, c)
    g = np.asarray(grad_u, dtype=np.float64).copy()
    gf = np.zeros_like(f)
    for n in range(int(N) - 1, -1, -1):
        r = np.real(idft2(dft2(g) / den))
        gf += r
        un = iterates[n]
        g = (lam / 2.0) * (grad_x_T(g2_welsch(grad_x(un), gamma, c) * grad_x(r))
                           + grad_y_T(g2_welsch(grad_y(un), gamma, c) * grad_y(r)))
    return (gf, g) if split else gf + g


# ----------------------------------------------------------------------------
# Half-quadratic splitting (Sec. 3.5, Eq. 12-14): the comparison method.  With the L1
# penalty phi(x) = |x| (anisotropic total variation, the case Sec. 3.5 analyses), Q1 is the
# soft threshold of grad u at lam / (2 beta_n) (Eq. 15-17, Appendix C) and Q2 is Eq. 9's FFT
# solve with weight beta_n in place of lam c / 2; beta_n = kappa beta_{n-1}.
# ----------------------------------------------------------------------------

def hqs_shrink_l1(x, lam, beta):
    """Q1 of Eq. 14 for phi = |x|: argmin_mu beta (x - mu)^2 + lam |mu| = soft threshold at lam/(2 beta)."""
    x = np.asarray(x, dtype=np.float64)
    t = lam / (2.0 * beta)
    return np.sign(x) * np.maximum(np.abs(x) - t, 0.0)


def hqs_channel(f, lam, N, beta0=None, kappa=2.0, u0=None, return_iterates=False):
    """Eq. 14 on one H x W channel (float64), phi = |x|: u^0 = f; for n = 0..N-1:
    mu^n = shrink(grad u^n, lam / (2 beta_n)), u^{n+1} = argmin (u - f)^2 + beta_n (grad u - mu^n)^2
    (Q2, solved by the periodic FFT as Eq. 9), beta_{n+1} = kappa beta_n.  beta0 defaults to 2 lam
    (the setting the paper uses in Fig. 11); kappa = 2 is a reading (the paper only requires kappa > 1)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    beta = 2.0 * lam if beta0 is None else float(beta0)
    Fdx, Fdy = gradient_transfer_functions(H, W)
    Ff = dft2(f)
    u = f.copy() if u0 is None else np.asarray(u0, dtype=np.float64).copy()
    iterates = [u.copy()]
    for _ in range(int(N)):
        mu_x = hqs_shrink_l1(grad_x(u), lam, beta)
        mu_y = hqs_shrink_l1(grad_y(u), lam, beta)
        den = 1.0 + beta * (np.abs(Fdx) ** 2 + np.abs(Fdy) ** 2)
        num = Ff + beta * (np.conj(Fdx) * dft2(mu_x) + np.conj(Fdy) * dft2(mu_y))
        u = np.real(idft2(num / den))
        beta *= kappa
        if return_iterates:
            iterates.append(u.copy())
    return (u, iterates) if return_iterates else u


def hqs_smooth(f, lam=0.25, N=4, beta0=None, kappa=2.0):
    """Half-quadratic splitting (phi = |x|) on a C x H x W (or H x W) image, channels independent."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        return hqs_channel(f, lam, N, beta0, kappa)
    return np.stack([hqs_channel(f[c], lam, N, beta0, kappa) for c in range(f.shape[0])])


# ----------------------------------------------------------------------------
# Colour option (I) of Sec. 3.4 and detail enhancement (the paper's figures: details
# boosted k = 3 times)
# ----------------------------------------------------------------------------

LUMA_BT601 = (0.299, 0.587, 0.114)


def luma(f_rgb):
    """Y of an RGB image (3 x H x W): the BT.601 luma weights.  Reading: Sec. 3.4 names the
    YUV luminance without a matrix."""
    f = np.asarray(f_rgb, dtype=np.float64)
    return LUMA_BT601[0] * f[0] + LUMA_BT601[1] * f[1] + LUMA_BT601[2] * f[2]


def detail_enhance(f, u, k):
    """Base u plus k times the detail layer f - u (k = 0: the smoothed image, k = 1: f)."""
    f = np.asarray(f, dtype=np.float64)
    return np.asarray(u, dtype=np.float64) + k * (f - np.asarray(u, dtype=np.float64))


def ils_smooth_luma(f_rgb, lam=1.0, p=0.8, eps=1e-4, N=4, k=0.0):
    """Option (I) of Sec. 3.4: ILS on the luminance only.  Y = luma(f); u_Y = ILS(Y), detail
    enhanced by k; the chroma (colour differences) is kept, so every RGB channel changes by
    the change of Y:  out_c = f_c + (Y' - Y),  Y' = u_Y + k (Y - u_Y)."""
    f = np.asarray(f_rgb, dtype=np.float64)
    Y = luma(f)
    uY = ils_channel(Y, lam, p, eps, N)
    Yp = detail_enhance(Y, uY, k)
    return f + (Yp - Y)[None, :, :]


LUMA_FLOOR = 1e-12  # reading: the log of a black pixel is taken at this luminance


def log_luma(f_rgb):
    """l = ln max(Y, LUMA_FLOOR) of a linear-radiance RGB image: Sec. 4.2 compresses only the
    luminance of an HDR image and smooths its logarithm.  Readings: natural log, BT.601 luma."""
    return np.log(np.maximum(luma(f_rgb), LUMA_FLOOR))


def tonemap_log(f_rgb, s, k=1.0, o=0.0, lam=10.0, p=1.0, eps=1e-4, N=4):
    """Single-scale HDR tone mapping in the base / detail form of Sec. 4.2 (the paper's
    single-scale setting: p = 1, lambda = 10).  The log-luminance l is split into the base
    layer b = ILS(l) and the detail d = l - b; the new log-luminance is l' = s b + k d (s < 1
    compresses the base, k boosts details) and every colour channel is scaled by the change of
    luminance, exp(l' - l), times exp(o) (exposure).  Returns (out, b, d).  Readings: the
    paper runs these steps inside a third-party framework whose compression is not stated;
    this is the linear base compression with colour ratios kept."""
    f = np.asarray(f_rgb, dtype=np.float64)
    l = log_luma(f)
    b = ils_channel(l, lam, p, eps, N)
    d = l - b
    lp = s * b + k * d
    return f * np.exp(lp - l + o)[None, :, :], b, d


def hwc_to_planar(x):
    """H x W x C (channels of a pixel adjacent) to C x H x W."""
    return np.ascontiguousarray(np.transpose(np.asarray(x), (2, 0, 1)))


def planar_to_hwc(x):
    """C x H x W to H x W x C."""
    return np.ascontiguousarray(np.transpose(np.asarray(x), (1, 2, 0)))


def ils_smooth_hwc(f_hwc, lam=1.0, p=0.8, eps=1e-4, N=4):
    """ILS of a pixel-interleaved image: the channels are independent (Sec. 3.4, option II),
    so it is ILS of each channel plane, stored back interleaved."""
    return planar_to_hwc(ils_smooth(hwc_to_planar(f_hwc), lam, p, eps, N))


def gaussian_weights(sigma):
    """Taps w_k, k = -r..r, of the truncated, normalized Gaussian: r = ceil(3 sigma),
    w_k = exp(-k^2 / (2 sigma^2)) / sum_j exp(-j^2 / (2 sigma^2)); sigma = 0 gives [1].
    Reading: the paper pre-smooths with 'a Gaussian filter of a small variation' (Sec. 5)
    and states neither the truncation nor the boundary."""
    if sigma <= 0:
        return np.ones(1)
    r = int(np.ceil(3.0 * sigma))
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    return w / w.sum()


def gaussian_blur_periodic(f, sigma):
    """Separable Gaussian blur of each H x W channel with periodic wrap (the boundary model of
    Eq. 9's solve): rows, then columns, each a sum of shifted copies."""
    f = np.asarray(f, dtype=np.float64)
    w = gaussian_weights(sigma)
    r = (len(w) - 1) // 2
    tmp = np.zeros_like(f)
    for i, k in enumerate(range(-r, r + 1)):
        tmp += w[i] * np.roll(f, -k, axis=-1)      # out[x] += w_k f[x + k]
    out = np.zeros_like(f)
    for i, k in enumerate(range(-r, r + 1)):
        out += w[i] * np.roll(tmp, -k, axis=-2)
    return out


def texture_smooth(f, sigma=1.0, lam=30.0, gamma=10.0 / 255.0, N=15):
    """Texture smoothing of Sec. 5: the input is pre-smoothed by a small Gaussian (so that
    the Welsch penalty, which barely penalizes large gradients, also flattens high-contrast
    texture), then smoothed by Welsch-penalty ILS with the paper's lambda = 30, gamma = 10/255,
    N = 15.  Reading: sigma = 1 pixel by default (the paper gives no value)."""
    g = gaussian_blur_periodic(f, sigma)
    return ils_smooth_welsch(g, lam, gamma, N)


# ----------------------------------------------------------------------------
# Adjoint of Algorithm 1 with respect to f
# ----------------------------------------------------------------------------

def ils_backward(f, grad_u, lam, p, eps, N, c=None, u0=None, split=False):
    """Gradient of <grad_u, u^N(f)> with respect to f, on one H x W channel (float64).

    The paper has no adjoint; this is the chain rule through Algorithm 1.
    Write A for the Eq. 9 operator (I + (lam c/2)(grad_x^T grad_x + grad_y^T grad_y)),
    diagonal in Fourier space with the real, even eigenvalues `den`, hence symmetric.
    u^{n+1} = A^{-1} (f + lam/2 sum_* grad_*^T mu(grad_* u^n)), u^0 = f, so with
    g = dL/du^{n+1}:
        r = A^{-1} g;   dL/df += r;   dL/du^n = lam/2 sum_* grad_*^T [ g''(grad_* u^n) * grad_* r ],
    where g'' = d mu / dx is the Appendix B second derivative.  Finally dL/df += dL/du^0
    (u^0 = f).  With a warm start u0 the iterates start from u0 and, if split, the pair
    (dL/df through Eq. 9 only, dL/du^0) is returned instead of their sum.
    """
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    if c is None:
        c = c0(p, eps)
    _, iterates = ils_channel(f, lam, p, eps, N, u0=u0, c=c, return_iterates=True)
    den = denominator(H, W, lam, c)
    g = np.asarray(grad_u, dtype=np.float64).copy()
    gf = np.zeros_like(f)
    for n in range(int(N) - 1, -1, -1):
        r = np.real(idft2(dft2(g) / den))
        gf += r
        un = iterates[n]
        g = (lam / 2.0) * (grad_x_T(g2(grad_x(un), p, eps, c) * grad_x(r))
                           + grad_y_T(g2(grad_y(un), p, eps, c) * grad_y(r)))
    return (gf, g) if split else gf + g


# ----------------------------------------------------------------------------
# Warm-start network (not in the paper): 3x3 convolutions, ReLU, residual output.
# ----------------------------------------------------------------------------

def conv3x3(x, w, b):
    """Zero-padded 3x3 cross-correlation, NCHW: out[o] = b[o] + sum_{i,dy,dx} w[o,i,dy,dx] x[i, y+dy-1, x+dx-1].

    Plain torch.nn.functional.conv2d in float64 (a library primitive).
    """
    import torch
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    wt = torch.as_tensor(np.asarray(w, dtype=np.float64))
    bt = torch.as_tensor(np.asarray(b, dtype=np.float64))
    squeeze = xt.ndim == 3
    if squeeze:
        xt = xt[None]
    y = torch.nn.functional.conv2d(xt, wt, bt, padding=1)
    return (y[0] if squeeze else y).numpy()


def warmstart_cnn_forward(f, weights, biases):
    """u0 = f + net(f): conv3x3 layers with ReLU between them, none after the last."""
    x = np.asarray(f, dtype=np.float64)
    h = x
    L = len(weights)
    for i, (w, b) in enumerate(zip(weights, biases)):
        h = conv3x3(h, w, b)
        if i < L - 1:
            h = np.maximum(h, 0.0)
    return x + h


# ----------------------------------------------------------------------------
# The warm-start network with the rounding points of a BF16 implementation.
#
# The tensor-core kernels hold weights, the network input and every hidden activation
# (and every hidden gradient) in BF16 and accumulate in FP32.  Where a value is stored
# as BF16 the oracle rounds it the same way (round to nearest even on the top 16 bits
# of the IEEE binary32 value); everything else is float64.
# ----------------------------------------------------------------------------

def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float64).astype(np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def _conv_fwd_bwd(x, w, g=None):
    """y = conv3x3(x, w) (zero padding, no bias), and with g = dL/dy also (dL/dx, dL/dw): float64 autograd."""
    import torch
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64)).requires_grad_(g is not None)
    wt = torch.as_tensor(np.asarray(w, dtype=np.float64)).requires_grad_(g is not None)
    y = torch.nn.functional.conv2d(xt, wt, padding=1)
    if g is None:
        return y.detach().numpy()
    y.backward(torch.as_tensor(np.asarray(g, dtype=np.float64)))
    return y.detach().numpy(), xt.grad.numpy(), wt.grad.numpy()


def warmstart_forward_bf16(f, weights, biases, rounding=True):
    """u0 = f + net(f) for a batch f (B x 3 x H x W) with the BF16 rounding points
    (rounding=False: plain float64, for checking the chain itself).

    Returns (u0, hidden) where hidden[l] is the stored (post-ReLU) output of layer l.
    """
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    f = np.asarray(f, dtype=np.float64)
    h = rnd(f)
    hidden = []
    L = len(weights)
    for l in range(L):
        y = _conv_fwd_bwd(h, rnd(weights[l])) + np.asarray(biases[l], dtype=np.float64)[None, :, None, None]
        if l < L - 1:
            h = rnd(np.maximum(y, 0.0))
            hidden.append(h)
        else:
            return f + y, hidden


def warmstart_backward_bf16(f, weights, biases, grad_u0, rounding=True):
    """dL/dW, dL/db of the network given dL/du0, with the BF16 rounding points of the kernels:
    each layer's output gradient is rounded to BF16 where it is stored, and the ReLU mask is
    taken from the stored activation (rounding=False: plain float64 reverse mode)."""
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    f = np.asarray(f, dtype=np.float64)
    _, hidden = warmstart_forward_bf16(f, weights, biases, rounding)
    L = len(weights)
    inputs = [rnd(f)] + hidden                   # input of layer l
    g = rnd(grad_u0)                             # gradient at the last layer's output
    dW, db = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        _, gx, gw = _conv_fwd_bwd(inputs[l], rnd(weights[l]), g)
        dW[l] = gw
        db[l] = g.sum(axis=(0, 2, 3))
        if l > 0:
            g = rnd(gx * (inputs[l] > 0))        # ReLU of layer l-1, stored as BF16
    return dW, db


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma and Ba); returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
