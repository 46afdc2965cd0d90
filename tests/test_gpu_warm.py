"""The warm-started smoother: the iterate change delta that decides the fallback, checked
against the FP64 oracle, the threshold tau on both sides of it, and what the trained
network gains over plain ILS at equal iteration budgets (the learned warm start's purpose)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2003_07504_gb300 import synth
from tests._util import MAX_ABS_TOL, RMS_TOL, err_stats

pytestmark = pytest.mark.gpu

LAM, P, EPS = 1.0, 0.8, 1e-4


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_2003_07504_gb300 import build
    build.build()
    from paper_2003_07504_gb300 import warmstart
    assert torch.cuda.is_available()
    return warmstart


def _params(ws):
    if os.path.exists(ws.DEFAULT_WEIGHTS):
        return ws.load_params(ws.DEFAULT_WEIGHTS)
    rng = np.random.default_rng(5)
    return (rng.standard_normal(ws.param_count()) * 1e-2).astype(np.float32)


@pytest.mark.parametrize("iters", [1, 2])
def test_delta_matches_oracle_and_tau_decides(ws, iters):
    import torch
    from paper_2003_07504_gb300 import ils
    H, W = 48, 64
    f = synth.preset_image(H, W, 3, "small", 21 + iters)
    ft = torch.from_numpy(f).cuda()
    net = ws.WarmStartNet(H * W, _params(ws))
    u0 = net.infer(ft.view(1, 3, H, W)).view(3, H, W).cpu().numpy().astype(np.float64)
    # the oracle's iterates from the network's own u^0 (Algorithm 1 with u^0 given)
    its = [O.ils_channel(f[c].astype(np.float64), LAM, P, EPS, iters, u0=u0[c], return_iterates=True)
           for c in range(3)]
    u_k = np.stack([it[1][iters] for it in its])
    u_km1 = np.stack([it[1][iters - 1] for it in its])
    delta_o = float(np.abs(u_k - u_km1).max())
    sm = ws.WarmSmoother(net, H, W, 3, LAM, P, EPS, iters=iters, tau=float("inf"))
    u, fb, d = sm.smooth(ft)
    sm.close()
    assert not fb
    assert abs(d - delta_o) <= MAX_ABS_TOL, (d, delta_o)
    mx, rms = err_stats(u.cpu().numpy(), u_k)
    assert mx <= MAX_ABS_TOL and rms <= RMS_TOL, (mx, rms)
    with ils.Plan(H, W, 3, LAM, P, EPS, 4) as plan:
        plain = plan.smooth(ft)
    for tau, expect in ((delta_o + 1e-3, False), (delta_o - 1e-3, True)):
        sm = ws.WarmSmoother(net, H, W, 3, LAM, P, EPS, iters=iters, n_plain=4, tau=tau)
        for _ in range(2):                     # first call captures the call's graph, second replays it
            u, fb, d = sm.smooth(ft)
            assert fb == expect and abs(d - delta_o) <= MAX_ABS_TOL
            if expect:
                assert torch.equal(u, plain)   # the fallback is plain ILS N=4 from f
            else:
                mx, rms = err_stats(u.cpu().numpy(), u_k)
                assert mx <= MAX_ABS_TOL and rms <= RMS_TOL
        # asynchronous form: the device decides, the host reads the decision after a sync
        u2 = sm.smooth_async(ft)
        torch.cuda.synchronize()
        fb2, d2 = sm.result()
        assert fb2 == expect and d2 == d and torch.equal(u2, u)
        sm.close()
    net.close()


@pytest.mark.parametrize("H,W,preset,seed", [(256, 256, "small", 7101), (1080, 1920, "hd", 7102)])
def test_trained_network_gains_over_plain_ils(ws, H, W, preset, seed):
    """With the trained weights, one ILS iteration from the network's u^0 is closer to converged
    ILS (from f) than plain ILS N=4, and than one plain iteration from f."""
    import torch
    from paper_2003_07504_gb300 import ils
    if not os.path.exists(ws.DEFAULT_WEIGHTS):
        pytest.skip("no trained weights file")
    ft = torch.from_numpy(synth.preset_image(H, W, 3, preset, seed)).cuda()
    ref, iters, change = ws.converged_ils(lambda h, w, c, n: ils.Plan(h, w, c, LAM, P, EPS, n), ft, max_iters=20000)
    assert change < 1e-6, (iters, change)   # the reference is converged to the FP32 floor
    rms = lambda u: float(((u - ref) ** 2).mean().sqrt())
    net = ws.WarmStartNet(H * W, ws.load_params(ws.DEFAULT_WEIGHTS))
    sm = ws.WarmSmoother(net, H, W, 3, LAM, P, EPS, iters=1, tau=float("inf"))
    warm1, fb, _ = sm.smooth(ft)
    assert not fb
    with ils.Plan(H, W, 3, LAM, P, EPS, 4) as p4, ils.Plan(H, W, 3, LAM, P, EPS, 1) as p1:
        plain4, plain1 = p4.smooth(ft), p1.smooth(ft)
    e_warm, e4, e1 = rms(warm1), rms(plain4), rms(plain1)
    assert e_warm <= e4 and e_warm < e1, (e_warm, e4, e1)
    sm.close()
    net.close()
