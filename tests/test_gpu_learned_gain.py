"""What the trained proposal network gains over the method without it.

A network is trained on the GPU (the library's forward, backward and Adam kernels) on three seeded
scenes, its fallback threshold is calibrated on a fourth, and on a fifth scene the learned fusion
must (a) evaluate far fewer patch-cost directions than the plain fusion and (b) stay within the
accuracy bounds against the FP64 oracle (median <= 2 deg, p95 <= 8 deg).  The fallback fraction
and both timings are recorded in the test's output."""
import time

import numpy as np
import pytest

import oracle
import scenegen
from helpers import angle_deg

pytestmark = pytest.mark.gpu

H, T, T_SHORT, ALPHA = 64, 8, 2, 0.24
SHAPE = dict(n_strands=4000)   # the full preset (64 views of 1920 x 1080) with 200,000 points


def _scene(seed):
    return scenegen.make_scene("full", seed=seed, **SHAPE)


def test_learned_path_gain():
    import torch

    import paper_2604_05794_b300 as hf
    from paper_2604_05794_b300 import learned as L
    dev = torch.device("cuda", 0)
    X, Tg = L.training_set(_scene, [500, 501, 502], 200000, H, T, dev)
    net, losses = L.train(X, Tg, steps=4000, batch=4096, lr=1e-3)
    del X, Tg
    assert np.mean(losses[-100:]) < 0.5 * np.mean(losses[:20])
    tau, _ = L.calibrate_tau(_scene(503), net, H, T, T_SHORT, ALPHA, dev, median_deg=1.8, p95_deg=7.5)

    sc = _scene(504)
    N = sc["N"]
    t = L.scene_tensors(sc, dev)
    mk = lambda: (torch.empty((N, 3), device=dev), torch.empty(N, device=dev),
                  torch.empty(N, dtype=torch.int32, device=dev), torch.empty(N, dtype=torch.uint8, device=dev))
    o_l, o_p = mk(), mk()
    with hf.HairFuse(H, sc["k"], T) as f:
        f.upload_views(t["cams"], t["angle"], t["conf"])
        f.upload_points(t["points"], t["nbr"])
        n_fb = f.fuse_learned(net, *o_l, T_short=T_SHORT, alpha_short=ALPHA, tau=tau)
        work = f.learned_work()
        pv = f.work()
        f.fuse(*o_p)
        f.sync()

        def timed(step, reps=5):
            step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                step()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps

        ms_l = 1e3 * timed(lambda: f.fuse_learned(net, *o_l, T_short=T_SHORT, alpha_short=ALPHA, tau=tau,
                                                  count_fallback=False))
        ms_p = 1e3 * timed(lambda: f.fuse(*o_p))
    # directions whose patch cost each path evaluates per (point, view): the plain fusion H hypotheses
    # and 6 T rotations (+ its start); the learned path the proposal, then 6 T_short rotations (+ start)
    # for accepted points and the plain fusion's work for fallback points
    plain_evals = pv * (H + 6 * T + 1)
    learned_evals = (pv + work["accepted_point_views"] * (6 * T_SHORT + 1) +
                     work["fallback_point_views"] * (H + 6 * T + 1))
    frac_fb = n_fb / N
    print(f"\nlearned gain: fallback {frac_fb:.3f}, evaluations {learned_evals / plain_evals:.3f} of plain, "
          f"time {ms_l:.3f} ms vs plain {ms_p:.3f} ms, tau {tau:.4f}")
    assert 0.0 < frac_fb < 0.65
    assert learned_evals < 0.7 * plain_evals
    # accuracy of the learned path against the FP64 oracle on a sample of points
    osc = oracle.Scene.from_dict(sc)
    sel = np.linspace(0, N - 1, 400).astype(np.int64)
    hyps = hf.fibonacci_hemisphere(H)
    orc = oracle.fuse(osc, hyps, T, idx=sel)   # rows follow sel
    ok = orc["status"] == 0
    ang = angle_deg(o_l[0].cpu().numpy()[sel], orc["dir"])[ok]
    assert np.median(ang) <= 2.0, np.median(ang)
    assert np.percentile(ang, 95) <= 8.0, np.percentile(ang, 95)
