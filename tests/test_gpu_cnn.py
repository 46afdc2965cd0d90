"""The warm-start network's tensor-core kernels against the FP64 oracle with BF16 rounding
points, its training, and the warm-started smoothing with its fallback.

Bars: the forward and every parameter gradient agree with the oracle that rounds to BF16
where the kernels store BF16; the remaining difference is FP32 vs FP64 accumulation, which
can move a value across a BF16 rounding boundary (one BF16 step, 2^-8 relative) and
propagate, so the bar is 2% of each tensor's largest magnitude (max-norm) and 0.5% in RMS.
"""
import numpy as np
import pytest

import oracle as O
from paper_2003_07504_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2003_07504_gb300 import build
    build.build()
    from paper_2003_07504_gb300 import warmstart as mod
    assert torch.cuda.is_available()
    return mod


def rel_max(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(1e-30, np.abs(b).max()))


def rel_rms(a, b):
    d = np.asarray(a, np.float64) - b
    return float(np.sqrt((d * d).mean()) / max(1e-30, np.sqrt((np.asarray(b) ** 2).mean())))


def random_params(ws, seed, last_scale=0.3):
    return ws.init_params(seed=seed, last_scale=last_scale)


@pytest.mark.parametrize("B,H,W", [(1, 8, 16), (2, 20, 36), (1, 33, 47)])
def test_forward_matches_oracle(ws, B, H, W):
    import torch
    p = random_params(ws, 1)
    f = synth.preset_image(H, W, 3 * B, "small", H + W).reshape(B, 3, H, W)
    net = ws.WarmStartNet(B * H * W, p)
    u0 = net.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    wts, bs = ws.unpack_params(p)
    want, _ = O.warmstart_forward_bf16(f, wts, bs)
    assert rel_max(u0 - f, want - f) <= 2e-2 and rel_rms(u0 - f, want - f) <= 5e-3
    net.close()


@pytest.mark.parametrize("B,H,W", [(2, 16, 32), (1, 27, 45)])
def test_backward_matches_oracle(ws, B, H, W):
    import torch
    p = random_params(ws, 2)
    f = synth.preset_image(H, W, 3 * B, "small", 5 + H).reshape(B, 3, H, W)
    g = synth.random_field((B, 3, H, W), seed=6)
    net = ws.WarmStartNet(B * H * W, p)
    ft = torch.from_numpy(f).cuda()
    net.forward(ft)
    net.zero_grad()
    net.backward(ft, torch.from_numpy(g).cuda())
    grads = net.get_grads()
    wts, bs = ws.unpack_params(p)
    dW, db = O.warmstart_backward_bf16(f, wts, bs, g)
    gw, gb = ws.unpack_params(grads)
    for l in range(len(wts)):
        assert rel_max(gw[l], dW[l]) <= 2e-2 and rel_rms(gw[l], dW[l]) <= 5e-3, l
        assert rel_max(gb[l], db[l]) <= 2e-2, l
    # gradients accumulate until zero_grad
    net.backward(ft, torch.from_numpy(g).cuda())
    np.testing.assert_allclose(net.get_grads(), 2 * grads, rtol=1e-5, atol=1e-6 * np.abs(grads).max())
    net.close()


def test_adam_step_matches_oracle(ws):
    import torch
    p = random_params(ws, 3)
    H, W = 16, 16
    f = synth.preset_image(H, W, 3, "small", 9).reshape(1, 3, H, W)
    net = ws.WarmStartNet(H * W, p)
    ft = torch.from_numpy(f).cuda()
    net.forward(ft)
    net.zero_grad()
    net.backward(ft, torch.from_numpy(synth.random_field((1, 3, H, W), seed=1)).cuda())
    g = net.get_grads().astype(np.float64)
    net.adam_step(1e-3)
    want, _, _ = O.adam_step(p.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    np.testing.assert_allclose(net.get_params(), want, rtol=1e-5, atol=1e-7)
    net.close()


def test_adam_state_round_trip_and_restored_step(ws):
    # checkpointed Adam state restores the next update: two steps on one network against one
    # step, a checkpoint (weights, moments, step count) into a second network, and its step
    import torch
    p = random_params(ws, 5)
    H, W = 16, 16
    ft = torch.from_numpy(synth.preset_image(H, W, 3, "small", 11).reshape(1, 3, H, W)).cuda()
    gu = torch.from_numpy(synth.random_field((1, 3, H, W), seed=3)).cuda()

    def grad_step(net):
        net.forward(ft)
        net.zero_grad()
        net.backward(ft, gu)
        g = net.get_grads().astype(np.float64)
        net.adam_step(1e-3)
        return g

    a = ws.WarmStartNet(H * W, p)
    grad_step(a)
    m, v, t = a.get_adam()
    assert t == 1 and np.abs(m).max() > 0 and np.abs(v).max() > 0
    b = ws.WarmStartNet(H * W, a.get_params())
    b.set_adam(m, v, t)
    m2, v2, t2 = b.get_adam()
    np.testing.assert_array_equal(m2, m)
    np.testing.assert_array_equal(v2, v)
    assert t2 == t
    w1 = a.get_params().astype(np.float64)
    g = grad_step(b)
    # the second Adam step from the restored state, in FP64
    want, _, _ = O.adam_step(w1, g, m.astype(np.float64), v.astype(np.float64), 2, lr=1e-3)
    np.testing.assert_allclose(b.get_params(), want, rtol=1e-5, atol=1e-7)
    a.close()
    b.close()


def test_training_resumes_from_a_checkpoint(ws, tmp_path):
    # a 6-step run against the same run stopped after 3 steps (checkpoint written) and resumed:
    # the same data order, schedule and optimizer state, so the same loss trajectory and
    # weights up to the FP32 atomic order of the weight gradients
    kw = dict(steps=6, batch=2, crop=64, lr=3e-3, n_crops=16, pool_images=2, pool_size=128, log_every=1,
              verbose=False, warmup=2)
    full, full_losses = ws.train(**kw)
    ck = str(tmp_path / "ck.npz")
    ws.train(stop_after=3, checkpoint=ck, checkpoint_every=1000, **kw)
    assert int(np.load(ck)["step"]) == 3
    resumed, resumed_losses = ws.train(resume=ck, **kw)
    assert [st for st, _ in resumed_losses] == [st for st, _ in full_losses] == list(range(6))
    np.testing.assert_allclose([v for _, v in resumed_losses], [v for _, v in full_losses], rtol=1e-3)
    np.testing.assert_allclose(resumed, full, rtol=1e-3, atol=1e-5)


def test_mse_kernel(ws):
    import torch
    a = torch.from_numpy(synth.random_field((2, 3, 10, 12), seed=1)).cuda()
    b = torch.from_numpy(synth.random_field((2, 3, 10, 12), seed=2)).cuda()
    grad = torch.empty_like(a)
    loss = torch.zeros(1, device="cuda")
    ws.mse(a, b, grad, loss)
    d = (a - b).double().cpu().numpy()
    assert float(loss.item()) == pytest.approx((d * d).mean(), rel=1e-5)
    np.testing.assert_allclose(grad.cpu().numpy(), 2 * d / d.size, rtol=1e-5, atol=1e-9)


def test_training_fits_a_fixed_batch(ws):
    # the same 4 crops every step: the loss (u0 vs the ILS N=4 target) must fall well below
    # its starting value u0 = f
    params, losses = ws.train(steps=200, batch=4, crop=64, lr=3e-3, n_crops=4, pool_images=2, pool_size=128,
                              log_every=25, verbose=False)
    first, last = losses[0][1], losses[-1][1]
    assert np.isfinite(params).all() and last < 0.6 * first, losses


def test_warm_smoother_paths(ws):
    # tau = inf: never falls back -> equals ILS_iters from u0 = net(f); tau = 0: always plain ILS N=4
    import torch
    from paper_2003_07504_gb300 import ils
    H, W = 48, 64
    p = random_params(ws, 4, last_scale=1e-2)
    f = torch.from_numpy(synth.preset_image(H, W, 3, "small", 12)).cuda()
    net = ws.WarmStartNet(H * W, p)
    u0 = net.infer(f.view(1, 3, H, W)).view(3, H, W)  # the smoother's own network call
    for iters in (1, 2):
        sm = ws.WarmSmoother(net, H, W, 3, iters=iters, tau=float("inf"))
        u, fb, d = sm.smooth(f)
        with ils.Plan(H, W, 3, 1.0, 0.8, 1e-4, iters) as plan:
            ref = plan.smooth(f, u0=u0)
        assert not fb and torch.equal(u, ref) and d > 0
        sm.close()
    sm = ws.WarmSmoother(net, H, W, 3, iters=1, tau=0.0)
    u, fb, d = sm.smooth(f)
    with ils.Plan(H, W, 3, 1.0, 0.8, 1e-4, 4) as plan:
        assert fb and torch.equal(u, plan.smooth(f))
    sm.close()
    net.close()


@pytest.mark.parametrize("B,H,W", [(1, 12, 128), (2, 9, 200), (1, 40, 384)])
def test_tcgen05_layers_match_the_mma_sync_kernels(ws, monkeypatch, B, H, W):
    # the tcgen05 kernels (TMA + tensor memory: every convolution but the last layer's forward,
    # every weight gradient) against the mma.sync kernels: same BF16 inputs, FP32 accumulation
    # in a different order -> BF16-rounding-level agreement
    import torch
    p = random_params(ws, 7)
    f = torch.from_numpy(synth.preset_image(H, W, 3 * B, "small", 3 + W).reshape(B, 3, H, W)).cuda()
    g = torch.from_numpy(synth.random_field((B, 3, H, W), seed=4)).cuda()
    tc = ws.WarmStartNet(B * H * W, p)
    monkeypatch.setenv("ILS_CNN_TC", "0")
    ref = ws.WarmStartNet(B * H * W, p)
    monkeypatch.delenv("ILS_CNN_TC")
    assert tc.uses_tcgen05 and not ref.uses_tcgen05
    outs = []
    for net in (tc, ref):
        u0 = net.forward(f)
        net.zero_grad()
        net.backward(f, g)
        net.check()
        outs.append((u0.cpu().numpy(), net.get_grads()))
    assert rel_max(outs[0][0] - f.cpu().numpy(), outs[1][0] - f.cpu().numpy()) <= 2e-2
    assert rel_max(outs[0][1], outs[1][1]) <= 2e-2 and rel_rms(outs[0][1], outs[1][1]) <= 5e-3
    tc.close()
    ref.close()


def test_tcgen05_bounded_wait_reports_timeout(ws, monkeypatch):
    # a poll limit of 1 makes the per-tile waits give up: the kernel must raise its flag,
    # wait for its own copies, free tensor memory and return; the next call works normally
    import torch
    H, W = 16, 256
    p = random_params(ws, 8)
    f = torch.from_numpy(synth.preset_image(H, W, 3, "small", 1).reshape(1, 3, H, W)).cuda()
    net = ws.WarmStartNet(H * W, p)
    if not net.uses_tcgen05:
        pytest.skip("tcgen05 path not available")
    monkeypatch.setenv("ILS_TEST_TC_SPIN", "1")
    net.forward(f)
    from paper_2003_07504_gb300._lib import ILSError
    with pytest.raises(ILSError) as e:
        net.check()
    assert e.value.name == "ILS_ERR_TIMEOUT"
    monkeypatch.delenv("ILS_TEST_TC_SPIN")
    u0 = net.forward(f)
    net.check()
    wts, bs = ws.unpack_params(p)
    want, _ = O.warmstart_forward_bf16(f.cpu().numpy(), wts, bs)
    assert rel_max(u0.cpu().numpy() - f.cpu().numpy(), want - f.cpu().numpy()) <= 2e-2
    net.close()


@pytest.mark.parametrize("B,H,W", [(1, 12, 122), (1, 25, 250), (2, 40, 300), (1, 13, 5), (1, 1, 130)])
def test_fused_inference_matches_oracle(ws, monkeypatch, B, H, W):
    # two fused tcgen05 kernels (layers 1-3, 4-6): one tile, ragged tiles in x and y, several
    # images, a single narrow tile, a single row
    import torch
    monkeypatch.setenv("ILS_CNN_FUSED", "1")
    p = random_params(ws, 11)
    f = synth.preset_image(H, W, 3 * B, "small", 7 * H + W).reshape(B, 3, H, W)
    net = ws.WarmStartNet(B * H * W, p)
    u0 = net.infer(torch.from_numpy(f).cuda()).cpu().numpy()
    net.check()
    wts, bs = ws.unpack_params(p)
    want, _ = O.warmstart_forward_bf16(f, wts, bs)
    assert rel_max(u0 - f, want - f) <= 2e-2 and rel_rms(u0 - f, want - f) <= 5e-3
    net.close()


def test_fused_inference_matches_layer_kernels_at_1080p(ws, monkeypatch):
    # full-size frame: fused inference against the layer-by-layer forward (same BF16 rounding
    # points, FP32 accumulation in another order) with the trained weights when present
    import os
    import torch
    monkeypatch.setenv("ILS_CNN_FUSED", "1")
    H, W = 1080, 1920
    p = ws.load_params(ws.DEFAULT_WEIGHTS) if os.path.exists(ws.DEFAULT_WEIGHTS) else random_params(ws, 12)
    f = torch.from_numpy(synth.preset_image(H, W, 3, "hd", 31).reshape(1, 3, H, W)).cuda()
    net = ws.WarmStartNet(H * W, p)
    a = net.infer(f)
    b = net.forward(f)
    net.check()
    d = (a - f).double().cpu().numpy(), (b - f).double().cpu().numpy()
    assert rel_max(d[0], d[1]) <= 2e-2 and rel_rms(d[0], d[1]) <= 5e-3
    # sampled pixels against the oracle on 20 x 20 windows (the receptive field is 13 x 13)
    wts, bs = ws.unpack_params(p)
    fh = f.cpu().numpy()
    for (y, x) in [(0, 0), (500, 960), (1060, 1900), (37, 1911), (1075, 3)]:
        y0, x0 = max(0, y - 6), max(0, x - 6)
        win = fh[:, :, y0:y0 + 20, x0:x0 + 20]
        want, _ = O.warmstart_forward_bf16(win, wts, bs)
        yy, xx = y - y0, x - x0
        got = a[0, :, y, x].cpu().numpy()
        # only pixels whose 13 x 13 receptive field lies inside the window or the image edge
        ok_y = (y < 6 or yy >= 6) and (y >= H - 6 or yy + 6 < win.shape[2])
        ok_x = (x < 6 or xx >= 6) and (x >= W - 6 or xx + 6 < win.shape[3])
        if ok_y and ok_x:
            scale = max(1e-6, float(np.abs(want - win).max()))
            assert float(np.abs(got - want[0, :, yy, xx]).max()) <= 2e-2 * scale, (y, x)
    net.close()


def test_fused_inference_bounded_wait_reports_timeout(ws, monkeypatch):
    import torch
    monkeypatch.setenv("ILS_CNN_FUSED", "1")
    H, W = 30, 260
    p = random_params(ws, 13)
    f = torch.from_numpy(synth.preset_image(H, W, 3, "small", 2).reshape(1, 3, H, W)).cuda()
    net = ws.WarmStartNet(H * W, p)
    if not net.uses_tcgen05:
        pytest.skip("tcgen05 path not available")
    monkeypatch.setenv("ILS_TEST_TC_SPIN", "1")
    net.infer(f)
    from paper_2003_07504_gb300._lib import ILSError
    with pytest.raises(ILSError) as e:
        net.check()
    assert e.value.name == "ILS_ERR_TIMEOUT"
    monkeypatch.delenv("ILS_TEST_TC_SPIN")
    u0 = net.infer(f)
    net.check()
    wts, bs = ws.unpack_params(p)
    want, _ = O.warmstart_forward_bf16(f.cpu().numpy(), wts, bs)
    assert rel_max(u0.cpu().numpy() - f.cpu().numpy(), want - f.cpu().numpy()) <= 2e-2
    net.close()
