"""Batches of frames of uneven size in one CUDA-graph launch (ils_batch_* through the C ABI)."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07504_gb300 import synth
from tests._util import MAX_ABS_TOL, RMS_TOL, err_stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ils():
    import torch
    from paper_2003_07504_gb300 import build
    build.build()
    from paper_2003_07504_gb300 import ils as mod
    assert torch.cuda.is_available()
    return mod


def make_frames(specs, seed0=0):
    import torch
    frames = []
    for k, (C, H, W, lam, p, N) in enumerate(specs):
        f = torch.from_numpy(synth.preset_image(H, W, C, "small", seed0 + k)).cuda()
        u = torch.full_like(f, float("nan"))
        frames.append((f, u, lam, p, 1e-4, N))
    return frames


def plan_result(ils, f, lam, p, N):
    C, H, W = f.shape
    with ils.Plan(H, W, C, lam, p, 1e-4, N) as plan:
        return plan.smooth(f)


SMALL = [(3, 48, 64, 1.0, 0.8, 4), (1, 30, 40, 0.5, 1.0, 4), (3, 64, 96, 2.0, 0.8, 2), (1, 48, 64, 1.5, 0.8, 1),
         (2, 75, 30, 1.0, 1.0, 3), (3, 48, 64, 0.7, 0.8, 4), (1, 16, 16, 1.0, 0.8, 0), (1, 256, 256, 1.0, 0.8, 4)]


def test_batch_matches_oracle_and_plan_path(ils):
    import torch
    frames = make_frames(SMALL)
    with ils.Batch(frames) as b:
        for rep in range(2):                          # the graph can be launched again
            for _, u, *_ in frames:
                u.fill_(float("nan"))
            b.run()
            torch.cuda.synchronize()
            for (f, u, lam, p, eps, N) in frames:
                got = u.cpu().numpy()
                want = O.ils_smooth(f.cpu().numpy().astype(np.float64), lam, p, eps, N)
                mx, rms = err_stats(got, want)
                assert mx <= MAX_ABS_TOL and rms <= RMS_TOL, (f.shape, lam, p, N, mx, rms)
                # default kernel choice = the plan path's: same bits
                assert torch.equal(u, plan_result(ils, f, lam, p, N))


def test_one_shot_call_equals_batch(ils):
    import torch
    frames = make_frames(SMALL[:5], seed0=50)
    ils.smooth_batched(frames)
    outs = [u.clone() for _, u, *_ in frames]
    with ils.Batch(frames) as b:
        b.run()
        torch.cuda.synchronize()
    for (_, u, *_), o in zip(frames, outs):
        assert torch.equal(u, o)


def test_autotuned_batch_at_the_serving_sizes(ils, tmp_path, monkeypatch):
    # one RGB frame of each size of the uneven-frame workload, per-frame lambda and p
    import torch
    specs = [(3, 480, 640, 0.6, 0.8, 4), (3, 720, 1280, 1.9, 1.0, 4), (3, 1080, 1920, 1.2, 0.8, 4),
             (3, 1536, 2048, 0.9, 1.0, 4)]
    frames = make_frames(specs, seed0=100)
    cache = tmp_path / "autotune.txt"
    monkeypatch.setenv("ILS_AUTOTUNE_CACHE", str(cache))
    with ils.Batch(frames, autotune=True) as b:
        b.run()
        torch.cuda.synchronize()
        choices = [b.choice(i) for i in range(len(frames))]
    assert cache.exists() and len(cache.read_text().splitlines()) == len(specs)
    for (f, u, lam, p, eps, N) in frames:
        ref = plan_result(ils, f, lam, p, N)
        mx, rms = err_stats(u.cpu().numpy(), ref.cpu().numpy())
        assert mx <= MAX_ABS_TOL and rms <= RMS_TOL
    # a second batch reads the cached choices
    with ils.Batch(frames, autotune=True) as b2:
        assert [b2.choice(i)[1:] for i in range(len(frames))] == [c[1:] for c in choices]


def energy64(u, f, lam, p, eps):
    """Eq. 1 with the Eq. 2 penalty, periodic forward differences, float64 (test-side)."""
    gx = np.roll(u, -1, axis=-1) - u
    gy = np.roll(u, -1, axis=-2) - u
    return float(((u - f) ** 2).sum() + lam * (((gx ** 2 + eps) ** (p / 2)).sum() + ((gy ** 2 + eps) ** (p / 2)).sum()))


def test_batch_of_4k_frames_with_large_iteration_counts(ils):
    # 3840 x 2160 frames with N = 10 and 15 in one graph launch: the same bits as the plan path,
    # the mean of every channel kept (the DC denominator is 1), and Eq. 1's energy below that
    # of fewer iterations (Appendix A: it decreases monotonically)
    import torch
    specs = [(3, 2160, 3840, 1.0, 0.8, 10), (3, 2160, 3840, 2.0, 1.0, 15), (1, 2160, 3840, 0.5, 0.8, 15),
             (3, 1080, 1920, 1.5, 0.8, 10)]
    frames = make_frames(specs, seed0=300)
    with ils.Batch(frames) as b:
        b.run()
        torch.cuda.synchronize()
    for (f, u, lam, p, eps, N) in frames:
        assert bool(torch.isfinite(u).all())
        assert torch.equal(u, plan_result(ils, f, lam, p, N))
        dm = (u.double().mean(dim=(1, 2)) - f.double().mean(dim=(1, 2))).abs().max().item()
        assert dm <= 1e-5, dm
        f64 = f.cpu().numpy().astype(np.float64)
        e_n = energy64(u.cpu().numpy().astype(np.float64), f64, lam, p, eps)
        e_fewer = energy64(plan_result(ils, f, lam, p, N - 6).cpu().numpy().astype(np.float64), f64, lam, p, eps)
        assert e_n < e_fewer, (f.shape, N, e_n, e_fewer)


def test_batch_rejects_bad_frames(ils):
    import torch
    from paper_2003_07504_gb300._lib import ILSError
    f = torch.rand(1, 32, 32, device="cuda")
    u = torch.empty_like(f)
    with pytest.raises(ILSError) as e:
        ils.Batch([(f, u, 1.0, 0.8, 1e-4, 4), (f, u, 1.0, 0.8, 1e-4, 4)])   # two frames share an output
    assert e.value.name == "ILS_ERR_INVALID_ARG"
    g = torch.rand(1, 14, 32, device="cuda")
    with pytest.raises(ILSError) as e:
        ils.Batch([(g, torch.empty_like(g), 1.0, 0.8, 1e-4, 4)])
    assert e.value.name == "ILS_ERR_UNSUPPORTED_SIZE"
