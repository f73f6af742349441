"""Batched serving: several scenes of uneven size fused in one submission give, scene by scene,
exactly the results of the same scene fused alone (plain and learned paths), whatever launch shape
the batch runs with, eagerly or as a replayed CUDA graph; spot checks against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import oracle.mlp as om
import scenegen
from helpers import compare

pytestmark = pytest.mark.gpu


def _scenes():
    """Five small scenes that differ in point count, views, map size and dtype, k, H, T, top-K; the
    last has 150 views, more than one group of 32 lanes holds, so its refinement gathers the patch
    in several chunks."""
    return [
        (scenegen.make_scene("tiny"), dict(H=32, T=4, top_k=0)),
        (scenegen.make_scene("mid", seed=11, n_strands=150, width=512, height=512, f=600.0), dict(H=64, T=8, top_k=0)),
        (scenegen.make_scene("full", seed=12, n_strands=120, V=16, width=640, height=360, f=433.0),
         dict(H=48, T=6, top_k=5)),
        (scenegen.make_scene("mid", seed=13, n_strands=40, V=24, width=512, height=512, f=600.0),
         dict(H=64, T=8, top_k=0)),
        (scenegen.make_scene("mid", seed=14, n_strands=12, V=150, width=256, height=256, f=300.0),
         dict(H=32, T=4, top_k=0)),
    ]


@pytest.fixture(scope="module")
def scenes():
    return _scenes()


def _ctx(sc, o):
    import paper_2604_05794_b300 as hf
    f = hf.HairFuse(o["H"], sc["k"], o["T"], top_k_views=o["top_k"])
    f.upload_views(sc["cams"], sc["angle"], sc["conf"])
    f.upload_points(sc["points"], sc["nbr"])
    return f


def _outs(N):
    import torch
    return (torch.empty((N, 3), device="cuda"), torch.empty(N, device="cuda"),
            torch.empty(N, dtype=torch.int32, device="cuda"), torch.empty(N, dtype=torch.uint8, device="cuda"))


def _host(o):
    return [x.cpu().numpy() for x in o]


def _alone_plain(ctxs, scenes):
    res = []
    for f, (sc, _) in zip(ctxs, scenes):
        o = _outs(sc["N"])
        f.fuse(*o)
        f.sync()
        res.append(_host(o))
    return res


def _equal(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("shape", [dict(autotune=True), dict(autotune=False, cta_threads=64, order=2),
                                   dict(autotune=False, cta_threads=256, order=3),
                                   dict(autotune=False, cta_threads=128, order=1),
                                   dict(autotune=False, cta_threads=128, order=0)])
def test_plain_batch_equals_alone(scenes, shape):
    import torch

    import paper_2604_05794_b300 as hf
    ctxs = [_ctx(sc, o) for sc, o in scenes]
    want = _alone_plain(ctxs, scenes)
    outs = [_outs(sc["N"]) for sc, _ in scenes]
    with hf.Batch(ctxs, **shape) as b:
        for s, o in enumerate(outs):
            b.set_outputs(s, *o)
        for use_graph in (False, True, True):
            for o in outs:
                for x in o:
                    x.zero_()
            b.run(use_graph=use_graph)
            b.sync()
            for s in range(len(scenes)):
                _equal(_host(outs[s]), want[s])
        lat = b.latency_ms()
        assert np.all(lat > 0) and np.all(np.isfinite(lat))
        assert np.all(b.fallbacks() == 0)
        t = b.tuning()
        assert t["cta_threads"] in (64, 128, 256)
        if not shape["autotune"]:
            assert t["cta_threads"] == shape["cta_threads"]
    torch.cuda.synchronize()
    for f in ctxs:
        f.close()


def test_autotune_result_cached_per_shape_class(scenes):
    """A second batch of the same shape class takes the first one's tuned launch shape without
    timing, and its results are still those of each scene fused alone."""
    import torch

    import paper_2604_05794_b300 as hf
    ctxs = [_ctx(sc, o) for sc, o in scenes]
    want = _alone_plain(ctxs, scenes)
    shapes = []
    for rep in range(2):
        outs = [_outs(sc["N"]) for sc, _ in scenes]
        with hf.Batch(ctxs, autotune=True) as b:
            for s, o in enumerate(outs):
                b.set_outputs(s, *o)
            b.run(use_graph=True)
            b.sync()
            for s in range(len(scenes)):
                _equal(_host(outs[s]), want[s])
            shapes.append(b.tuning())
    assert shapes[1]["cached"]
    assert (shapes[0]["cta_threads"], shapes[0]["order"]) == (shapes[1]["cta_threads"], shapes[1]["order"])
    torch.cuda.synchronize()
    for f in ctxs:
        f.close()


@pytest.mark.parametrize("Ts", [2, 4])
def test_learned_batch_equals_alone(scenes, Ts):
    import paper_2604_05794_b300 as hf
    net = hf.ProposalNet(1024)
    net.set_params(om.init(5).astype(np.float32))
    al, tau = 0.05, 0.3
    ctxs = [_ctx(sc, o) for sc, o in scenes]
    want, nf_want = [], []
    for f, (sc, _) in zip(ctxs, scenes):
        o = _outs(sc["N"])
        nf_want.append(f.fuse_learned(net, *o, T_short=Ts, alpha_short=al, tau=tau))
        want.append(_host(o))
    assert sum(nf_want) > 0 and sum(nf_want) < sum(sc["N"] for sc, _ in scenes)
    outs = [_outs(sc["N"]) for sc, _ in scenes]
    with hf.Batch(ctxs, net=net, T_short=Ts, alpha_short=al, tau=tau, autotune=True) as b:
        for s, o in enumerate(outs):
            b.set_outputs(s, *o)
        for use_graph in (False, True, True):
            for o in outs:
                for x in o:
                    x.zero_()
            b.run(use_graph=use_graph)
            b.sync()
            for s in range(len(scenes)):
                _equal(_host(outs[s]), want[s])
            assert list(b.fallbacks()) == nf_want
        assert np.all(b.latency_ms() > 0)
    for f in ctxs:
        f.close()


def test_batch_matches_oracle_sample(scenes):
    """A sample of the batched plain result of every scene against the FP64 oracle."""
    import paper_2604_05794_b300 as hf
    ctxs = [_ctx(sc, o) for sc, o in scenes]
    outs = [_outs(sc["N"]) for sc, _ in scenes]
    with hf.Batch(ctxs, autotune=False) as b:
        for s, o in enumerate(outs):
            b.set_outputs(s, *o)
        b.run(use_graph=True)
        b.sync()
        for s, (sc, o) in enumerate(scenes):
            osc = oracle.Scene.from_dict(sc)
            sel = np.linspace(0, sc["N"] - 1, 60).astype(np.int64)
            hyps = hf.fibonacci_hemisphere(o["H"])
            orc = oracle.fuse(osc, hyps, o["T"], idx=sel, top_k=o["top_k"])
            d, c, i, st = _host(outs[s])
            compare(dict(dir=d, cost=c, idx=i, status=st), orc, sel, osc, hyps, o["H"], top_k=o["top_k"],
                    strict_frac=0.95)
    for f in ctxs:
        f.close()


def test_batch_rejects_bad_arguments(scenes):
    import paper_2604_05794_b300 as hf
    sc, o = scenes[0]
    f = _ctx(sc, o)
    with pytest.raises(hf.HairFuseError):
        hf.Batch([])
    with pytest.raises(hf.HairFuseError):
        hf.Batch([f, f])
    empty = hf.HairFuse(32, 5, 4)
    with pytest.raises(hf.HairFuseError):
        hf.Batch([f, empty])
    net = hf.ProposalNet(1024)
    with pytest.raises(hf.HairFuseError):
        hf.Batch([f], net=net, T_short=0)
    with hf.Batch([f]) as b:
        with pytest.raises(hf.HairFuseError):
            b.run()   # outputs not set
        with pytest.raises(hf.HairFuseError):
            b.set_outputs(3, *_outs(sc["N"]))
    empty.close()
    f.close()


def test_asynchronous_uploads_two_streams():
    """HF_HOST_ASYNC: pinned uploads queued without waiting, two contexts on two streams taking
    turns (the serving pipeline), give the same bits as the synchronous upload; pageable arrays
    are refused."""
    import torch

    import paper_2604_05794_b300 as hf
    sc = scenegen.make_scene("mid", seed=21, n_strands=60, V=12, width=512, height=512, f=600.0)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h = [pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr")]
    N = sc["N"]
    ref = np.empty((N, 3), np.float32)
    with hf.HairFuse(32, sc["k"], 4) as f:
        f.upload_views(sc["cams"], sc["angle"], sc["conf"])
        f.upload_points(sc["points"], sc["nbr"])
        f.fuse(ref)
        with pytest.raises(ValueError):
            f.upload_views(sc["cams"], sc["angle"], sc["conf"], asynchronous=True)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctxs = [hf.HairFuse(32, sc["k"], 4, stream=s.cuda_stream) for s in streams]
    outs = [torch.empty((N, 3), device="cuda") for _ in streams]
    try:
        for rep in range(3):
            for f, o in zip(ctxs, outs):
                f.upload_views(h[0], h[1], h[2], asynchronous=True)
                f.upload_points(h[3], h[4])
                f.fuse(o)
        torch.cuda.synchronize()
        for o in outs:
            assert np.array_equal(o.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    finally:
        for f in ctxs:
            f.close()
