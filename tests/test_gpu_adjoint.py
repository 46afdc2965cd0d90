"""The hand-written adjoint (ils_backward through the C ABI, and ILSFunction in autograd)
against the FP64 oracle's reverse-mode gradient and finite differences of the oracle.

Bar: relative max-norm error <= 1e-4 against the FP64 gradient.  FP32 forward errors are
~1e-6 of a [0,1] image; g'' = c - h(x) cancels to O(x^2) near x = 0 with c ~ 200, so its
absolute FP32 error is ~1e-5 c-relative, which bounds the gradient error well below 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_2003_07504_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4


@pytest.fixture(scope="module")
def ils():
    import torch
    from paper_2003_07504_gb300 import build
    build.build()
    from paper_2003_07504_gb300 import ils as mod
    assert torch.cuda.is_available()
    return mod


def rel_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(1e-30, np.abs(b).max()))


def gpu_grad(ils, f, w, lam=1.0, p=0.8, N=4, u0=None, separate=False):
    import torch
    C, H, W = f.shape
    with ils.Plan(H, W, C, lam, p, 1e-4, N) as plan:
        ft = torch.from_numpy(f).cuda()
        u0t = None if u0 is None else torch.from_numpy(u0).cuda()
        u, ck = plan.smooth_checkpointed(ft, u0=u0t)
        plain = plan.smooth(ft, u0=u0t)
        torch.cuda.synchronize()
        assert torch.equal(u, plain)   # checkpointing does not change the forward
        out = plan.backward_ckpt(ck, torch.from_numpy(w).cuda(), separate_u0=separate)
        torch.cuda.synchronize()
        if separate:
            return out[0].cpu().numpy(), out[1].cpu().numpy()
        return out.cpu().numpy()


@pytest.mark.parametrize("H,W,C,lam,p,N", [
    (32, 40, 1, 1.0, 0.8, 4), (45, 64, 2, 2.0, 1.0, 3), (64, 64, 1, 0.5, 0.5, 2), (30, 48, 3, 1.0, 0.8, 1),
    (256, 256, 1, 1.0, 0.8, 4), (75, 30, 1, 3.5, 0.8, 4),
    # warp-per-row adjoint kernels: L = 8, 10, 20, 30, 32 (ragged last strip: H not a multiple of 6)
    (20, 512, 1, 1.0, 0.8, 3), (15, 640, 2, 1.0, 0.8, 2), (16, 1280, 1, 2.0, 0.8, 2), (25, 1920, 1, 1.0, 0.8, 2),
    (9, 2048, 1, 1.0, 1.0, 2),
    # 3840-wide rows: warp-pair forward kernels, generic adjoint row kernel
    (9, 3840, 1, 1.0, 0.8, 2),
])
def test_adjoint_matches_fp64_reverse_mode(ils, H, W, C, lam, p, N):
    f = synth.preset_image(H, W, C, "small", H + W + C)
    w = synth.random_field(f.shape, seed=7)
    g = gpu_grad(ils, f, w, lam, p, N)
    for ch in range(C):
        want = O.ils_backward(f[ch].astype(np.float64), w[ch].astype(np.float64), lam, p, 1e-4, N)
        assert rel_err(g[ch], want) <= REL_TOL


def test_adjoint_against_finite_differences_of_the_fp64_forward(ils):
    # <dL/df, v> against central differences of the FP64 forward.  h = 1e-5: with
    # sqrt(eps) = 0.01 the curvature scale, h = 1e-3 leaves O(1e-2) truncation error.
    H, W = 48, 64
    f = synth.preset_image(H, W, 1, "small", 3)
    w = synth.random_field(f.shape, seed=8)
    g = gpu_grad(ils, f, w)[0].astype(np.float64)
    f64, w64 = f[0].astype(np.float64), w[0].astype(np.float64)
    rng = np.random.default_rng(2)
    for trial in range(3):
        v = rng.normal(size=(H, W))
        h = 1e-5
        fd = (np.sum(w64 * O.ils_channel(f64 + h * v, 1.0, 0.8, 1e-4, 4)) -
              np.sum(w64 * O.ils_channel(f64 - h * v, 1.0, 0.8, 1e-4, 4))) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-4)
    # the h = 1e-3 difference named for this check agrees only to its truncation error
    v = rng.normal(size=(H, W))
    h = 1e-3
    fd3 = (np.sum(w64 * O.ils_channel(f64 + h * v, 1.0, 0.8, 1e-4, 4)) -
           np.sum(w64 * O.ils_channel(f64 - h * v, 1.0, 0.8, 1e-4, 4))) / (2 * h)
    assert np.sum(g * v) == pytest.approx(fd3, rel=0.15)


def test_adjoint_warm_start_split(ils):
    H, W = 40, 48
    f = synth.preset_image(H, W, 1, "small", 11)
    u0 = synth.random_field(f.shape, seed=12, lo=0.0, hi=1.0)
    w = synth.random_field(f.shape, seed=13)
    gf, gu0 = gpu_grad(ils, f, w, u0=u0, separate=True)
    want_f, want_u0 = O.ils_backward(f[0].astype(np.float64), w[0].astype(np.float64), 1.0, 0.8, 1e-4, 4,
                                     u0=u0[0].astype(np.float64), split=True)
    assert rel_err(gf[0], want_f) <= REL_TOL
    assert rel_err(gu0[0], want_u0) <= REL_TOL


def test_adjoint_n0_and_lambda0(ils):
    f = synth.preset_image(16, 24, 1, "small", 1)
    w = synth.random_field(f.shape, seed=2)
    np.testing.assert_array_equal(gpu_grad(ils, f, w, N=0), w)      # u = f
    g = gpu_grad(ils, f, w, lam=0.0)                                   # u = f for every N
    assert np.abs(g - w).max() < 1e-5


def test_autograd_function(ils):
    import torch
    H, W = 36, 60
    f = synth.preset_image(H, W, 2, "small", 21)
    w = synth.random_field(f.shape, seed=22)
    with ils.Plan(H, W, 2) as plan:
        ft = torch.from_numpy(f).cuda().requires_grad_(True)
        u = ils.ils_function(ft, plan)
        loss = (u * torch.from_numpy(w).cuda()).sum()
        loss.backward()
        g = ft.grad.cpu().numpy()
    for ch in range(2):
        want = O.ils_backward(f[ch].astype(np.float64), w[ch].astype(np.float64), 1.0, 0.8, 1e-4, 4)
        assert rel_err(g[ch], want) <= REL_TOL


def test_adjoint_batch_of_512_images_against_fp64_samples(ils):
    # 16 gray 512 x 512 images as one 16-channel plan; two channels checked against the
    # FP64 reverse mode element by element, the rest by channel independence.
    import torch
    C, H, W = 16, 512, 512
    f = synth.preset_image(H, W, C, "small", 512)
    w = synth.random_field(f.shape, seed=513)
    g = gpu_grad(ils, f, w)
    for ch in (0, 11):
        want = O.ils_backward(f[ch].astype(np.float64), w[ch].astype(np.float64), 1.0, 0.8, 1e-4, 4)
        assert rel_err(g[ch], want) <= REL_TOL
    np.testing.assert_array_equal(gpu_grad(ils, f[5:6].copy(), w[5:6].copy()), g[5:6])


@pytest.mark.parametrize("H,W,lam,gamma,N", [(32, 40, 20.0, 10 / 255, 3), (48, 64, 5.0, 0.1, 4),
                                             (20, 512, 20.0, 10 / 255, 3), (12, 1920, 5.0, 0.1, 2)])
def test_welsch_adjoint_matches_fp64_reverse_mode(ils, H, W, lam, gamma, N):
    # Welsch g'' (Appendix B) in the adjoint row kernel; c = 2, so FP32 cancellation is mild
    import torch
    f = synth.preset_image(H, W, 1, "small", H * W)
    w = synth.random_field(f.shape, seed=9)
    with ils.Plan(H, W, 1, lam, N=N, penalty="welsch", gamma=gamma) as plan:
        u, ck = plan.smooth_checkpointed(torch.from_numpy(f).cuda())
        g = plan.backward_ckpt(ck, torch.from_numpy(w).cuda()).cpu().numpy()
    want = O.ils_backward_welsch(f[0].astype(np.float64), w[0].astype(np.float64), lam, gamma, N)
    assert rel_err(g[0], want) <= REL_TOL


def test_plan_owned_checkpoints_and_backward_by_f(ils):
    """ils_set_checkpointing + ils_smooth + ils_backward(plan, f, grad_u, grad_f): the gradient
    of the last checkpointed call, checked against the FP64 reverse mode."""
    import torch
    from paper_2003_07504_gb300 import _lib
    C, H, W, lam, p, N = 2, 45, 64, 1.0, 0.8, 4
    f = synth.preset_image(H, W, C, "small", 5)
    w = synth.random_field(f.shape, seed=8)
    want = np.stack([O.ils_backward(f[c].astype(np.float64), w[c].astype(np.float64), lam, p, 1e-4, N)
                     for c in range(C)])
    with ils.Plan(H, W, C, lam, p, 1e-4, N) as plan:
        ft = torch.from_numpy(f).cuda()
        other = ft.clone()
        wt = torch.from_numpy(w).cuda()
        with pytest.raises(_lib.ILSError):     # no checkpoints yet
            plan.backward(ft, wt)
        plan.set_checkpointing(True)
        plan.smooth(other)
        u = plan.smooth(ft)                     # the last checkpointed call: f
        ref = ils.Plan(H, W, C, lam, p, 1e-4, N).smooth(ft)
        torch.cuda.synchronize()
        assert torch.equal(u, ref)              # checkpointing does not change the forward
        g = plan.backward(ft, wt).cpu().numpy()
        with pytest.raises(_lib.ILSError):     # another f than the last checkpointed call
            plan.backward(other, wt)
        plan.set_checkpointing(False)
        with pytest.raises(_lib.ILSError):
            plan.backward(ft, wt)
    assert rel_err(g, want) <= 1e-4


def test_c99_program_backward_through_the_abi(ils, tmp_path):
    """A C99 program (CUDA runtime API for device memory, no torch) calls ils_set_checkpointing,
    ils_smooth and ils_backward through libils.so; its dL/df matches the FP64 reverse mode."""
    import os
    import shutil
    import subprocess
    from paper_2003_07504_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    C, H, W, lam, p, N = 1, 30, 48, 1.0, 0.8, 3
    f = synth.preset_image(H, W, C, "small", 11)
    w = synth.random_field(f.shape, seed=12)
    f.astype(np.float32).tofile(tmp_path / "f.bin")
    w.astype(np.float32).tofile(tmp_path / "g.bin")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib_dir = os.path.dirname(_lib.LIB_PATH)
    src = tmp_path / "bwd.c"
    src.write_text(r'''
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime_api.h>
#include "ils.h"
#define CK(x) do { if ((x) != 0) { fprintf(stderr, "failed: %s\n", #x); return 1; } } while (0)
int main(int argc, char** argv) {
  (void)argc;
  const int H = atoi(argv[1]), W = atoi(argv[2]), C = atoi(argv[3]), N = atoi(argv[4]);
  const float lam = (float)atof(argv[5]), p = (float)atof(argv[6]);
  const size_t n = (size_t)C * H * W;
  float* hf = malloc(n * sizeof(float));
  float* hg = malloc(n * sizeof(float));
  FILE* fp = fopen(argv[7], "rb"); if (!fp || fread(hf, sizeof(float), n, fp) != n) return 2; fclose(fp);
  fp = fopen(argv[8], "rb"); if (!fp || fread(hg, sizeof(float), n, fp) != n) return 3; fclose(fp);
  float *f, *u, *g, *gf;
  CK(cudaMalloc((void**)&f, n * 4)); CK(cudaMalloc((void**)&u, n * 4));
  CK(cudaMalloc((void**)&g, n * 4)); CK(cudaMalloc((void**)&gf, n * 4));
  CK(cudaMemcpy(f, hf, n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(g, hg, n * 4, cudaMemcpyHostToDevice));
  ils_plan* plan = NULL;
  CK(ils_plan_create(H, W, C, lam, p, 1e-4f, N, &plan));
  if (ils_backward(plan, f, g, gf, NULL) != ILS_ERR_INVALID_ARG) return 4;  /* no checkpoints */
  CK(ils_set_checkpointing(plan, 1));
  CK(ils_smooth(plan, f, u, NULL));
  CK(ils_backward(plan, f, g, gf, NULL));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(hg, gf, n * 4, cudaMemcpyDeviceToHost));
  CK(ils_plan_destroy(plan));
  fp = fopen(argv[9], "wb"); if (!fp || fwrite(hg, sizeof(float), n, fp) != n) return 5; fclose(fp);
  cudaFree(f); cudaFree(u); cudaFree(g); cudaFree(gf);
  free(hf); free(hg);
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "bwd"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                    "-I", os.path.join(cuda, "include"), str(src), "-o", str(exe), "-L", lib_dir, "-lils",
                    f"-Wl,-rpath,{lib_dir}", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"], check=True)
    r = subprocess.run([str(exe), str(H), str(W), str(C), str(N), str(lam), str(p), str(tmp_path / "f.bin"),
                        str(tmp_path / "g.bin"), str(tmp_path / "gf.bin")], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
    got = np.fromfile(tmp_path / "gf.bin", dtype=np.float32).reshape(f.shape)
    want = np.stack([O.ils_backward(f[c].astype(np.float64), w[c].astype(np.float64), lam, p, 1e-4, N)
                     for c in range(C)])
    assert rel_err(got, want) <= 1e-4
