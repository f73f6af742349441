"""The allocation-free fusion entry point (for callers that may not call cudaMalloc).

Callers such as plugin hosts whose enqueue hooks forbid allocation, or processes whose device
memory belongs to a framework's caching allocator, use hair_fuse_fuse_directions_noalloc: its
scratch is a fixed static device array inside the library.  These tests call it through the C
ABI and check that it gives, bit for bit, what the context-based entry point gives (the two run the
same kernels), also when a call reuses the array after a call of another shape; this file is
collected last.
"""
import ctypes

import numpy as np
import pytest

import scenegen


def _ptr(x):
    return None if x is None else x.data_ptr()


def _call(hf, cfg, sc, d, out, stream, hyps=None):
    return hf.hair_fuse_fuse_directions_noalloc(
        ctypes.byref(cfg), sc["N"], sc["V"], sc["W"], sc["H"], d["cams"].data_ptr(), d["angle"].data_ptr(),
        d["conf"].data_ptr(), hf.HF_F16 if sc["conf"].dtype == np.float16 else hf.HF_F32, d["points"].data_ptr(),
        d["nbr"].data_ptr(), _ptr(hyps), out["dir"].data_ptr(), _ptr(out["cost"]), _ptr(out["idx"]),
        _ptr(out["status"]), stream)


def test_rejects_inputs_beyond_the_static_scratch():
    import paper_2604_05794_b300 as hf
    cfg = hf.hf_config(64, 8, 8, 0, 0.0, 0)
    # N * V = 2,000,000 > 1,048,576: rejected before any CUDA call, so no device is needed
    rc = hf.hair_fuse_fuse_directions_noalloc(ctypes.byref(cfg), 1000000, 2, 64, 64, 1, 1, 1, hf.HF_F32, 1, 1,
                                              None, 1, None, None, None, None)
    assert rc == hf.HF_ERR_SHAPE
    assert b"1048576" in hf.hair_fuse_last_error(None)


def test_rejects_each_shape_limit():
    import paper_2604_05794_b300 as hf
    # rejected before any CUDA call, so no device is needed: N > 262,144; V > 1024; V * Hq > 65,536
    for H, N, V in ((64, 300000, 2), (64, 100, 1025), (1024, 100, 65)):
        cfg = hf.hf_config(H, 8, 8, 0, 0.0, 0)
        rc = hf.hair_fuse_fuse_directions_noalloc(ctypes.byref(cfg), N, V, 64, 64, 1, 1, 1, hf.HF_F32, 1, 1, None, 1,
                                                  None, None, None, None, None)
        assert rc == hf.HF_ERR_SHAPE, (H, N, V)


def _scene(kind):
    if kind == "tiny":
        return scenegen.make_scene("tiny")
    if kind == "tiny_f16":
        return scenegen.make_scene("tiny", conf_f16=True, seed=11)
    if kind == "odd":   # an odd view count: the last view pair's second half is padding
        return scenegen.make_scene("mid", seed=13, n_strands=30, V=13, width=384, height=384, f=450.0)
    # more points and views than the tiny scene, to reuse the shared array with another shape
    return scenegen.make_scene("mid", seed=12, n_strands=60, V=20, width=512, height=512, f=600.0)


def _reference(hf, sc, H, T, top_k, d, hyps, mk):
    ref = mk()
    with hf.HairFuse(H, sc["k"], T, top_k_views=top_k) as f:
        f.upload_views(d["cams"], d["angle"], d["conf"])
        f.upload_points(d["points"], d["nbr"])
        f.fuse(ref["dir"], ref["cost"], ref["idx"], ref["status"], hyps=hyps)
        f.sync()
    return ref


# (scene, H, T, top-K, caller hypotheses, outputs other than dir given)
CASES = [("tiny", 32, 4, 0, False, True), ("tiny_f16", 32, 4, 0, False, True), ("tiny", 64, 4, 0, True, True),
         ("tiny", 32, 4, 3, False, True), ("tiny", 32, 4, 0, False, False), ("larger", 48, 6, 0, False, True),
         ("odd", 32, 4, 0, False, True)]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-H{c[1]}-top{c[3]}-hyps{int(c[4])}-outs{int(c[5])}" for c in CASES])
def test_bit_identical_to_context_entry_point(case):
    """Two calls in a row, then (for the larger scene) a call on the tiny scene after it: every output
    equals the context-based entry point's bit for bit (both run the same kernels)."""
    import torch

    import paper_2604_05794_b300 as hf
    kind, H, T, top_k, own_hyps, all_outs = case
    dev = torch.device("cuda")
    scenes = [_scene(kind)] + ([_scene("tiny")] if kind == "larger" else [])
    for sc in scenes:
        N = sc["N"]
        d = {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr")}
        hyps = torch.from_numpy(hf.fibonacci_hemisphere(H)[::-1].copy()).to(dev) if own_hyps else None
        mk = lambda: dict(dir=torch.empty((N, 3), device=dev), cost=torch.empty(N, device=dev),
                          idx=torch.empty(N, dtype=torch.int32, device=dev),
                          status=torch.empty(N, dtype=torch.uint8, device=dev))
        ref = _reference(hf, sc, H, T, top_k, d, hyps, mk)
        cfg = hf.hf_config(H, sc["k"], T, top_k, 0.0, 0)
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = mk()
            if not all_outs:
                out["cost"] = out["idx"] = out["status"] = None
            rc = _call(hf, cfg, sc, d, out, stream, hyps)
            assert rc == hf.HF_OK, hf.hair_fuse_last_error(None)
            torch.cuda.synchronize()
            for key in ("dir", "cost", "idx", "status"):
                if out[key] is not None:
                    assert torch.equal(out[key].view(torch.uint8), ref[key].view(torch.uint8)), (call, key)


@pytest.mark.gpu
def test_non_unit_hypothesis_is_reported():
    import torch

    import paper_2604_05794_b300 as hf
    sc = scenegen.make_scene("tiny")
    dev = torch.device("cuda")
    d = {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr")}
    hyps = torch.from_numpy(hf.fibonacci_hemisphere(32)).to(dev)
    hyps[5] *= 1.5
    N = sc["N"]
    out = dict(dir=torch.empty((N, 3), device=dev), cost=None, idx=None, status=None)
    cfg = hf.hf_config(32, sc["k"], 4, 0, 0.0, 0)
    rc = _call(hf, cfg, sc, d, out, torch.cuda.current_stream().cuda_stream, hyps)
    assert rc == hf.HF_ERR_INVALID_ARG
    assert b"unit length" in hf.hair_fuse_last_error(None)


@pytest.mark.gpu
def test_rejects_bad_neighbour_index_without_reading_through_it():
    import torch

    import paper_2604_05794_b300 as hf
    sc = scenegen.make_scene("tiny")
    dev = torch.device("cuda")
    d = {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr")}
    d["nbr"][17, 3] = sc["N"] + 5
    N = sc["N"]
    out = dict(dir=torch.empty((N, 3), device=dev), cost=torch.empty(N, device=dev),
               idx=torch.empty(N, dtype=torch.int32, device=dev), status=torch.empty(N, dtype=torch.uint8, device=dev))
    cfg = hf.hf_config(32, sc["k"], 4, 0, 0.0, 0)
    rc = _call(hf, cfg, sc, d, out, torch.cuda.current_stream().cuda_stream)
    assert rc == hf.HF_ERR_INVALID_ARG
