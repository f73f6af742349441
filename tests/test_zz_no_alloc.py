"""The allocation-free fusion entry point (for callers that may not call cudaMalloc).

Callers such as plugin hosts whose enqueue hooks forbid allocation, or processes whose device
memory belongs to a framework's caching allocator, use hair_fuse_fuse_directions_noalloc: its
scratch is a fixed static device array inside the library.  These tests call it through the C
ABI and check it against the context-based entry point; this file is collected last.
"""
import ctypes

import numpy as np
import pytest

import scenegen

TOL_COST_RTOL, TOL_COST_ATOL = 1e-4, 1e-6


def _call(hf, cfg, sc, d, out, stream):
    return hf.hair_fuse_fuse_directions_noalloc(
        ctypes.byref(cfg), sc["N"], sc["V"], sc["W"], sc["H"], d["cams"].data_ptr(), d["angle"].data_ptr(),
        d["conf"].data_ptr(), hf.HF_F16 if sc["conf"].dtype == np.float16 else hf.HF_F32, d["points"].data_ptr(),
        d["nbr"].data_ptr(), None, out["dir"].data_ptr(), out["cost"].data_ptr(), out["idx"].data_ptr(),
        out["status"].data_ptr(), stream)


def test_rejects_inputs_beyond_the_static_scratch():
    import paper_2604_05794_b300 as hf
    cfg = hf.hf_config(64, 8, 8, 0, 0.0, 0)
    # N * V = 2,000,000 > 1,048,576: rejected before any CUDA call, so no device is needed
    rc = hf.hair_fuse_fuse_directions_noalloc(ctypes.byref(cfg), 1000000, 2, 64, 64, 1, 1, 1, hf.HF_F32, 1, 1,
                                              None, 1, None, None, None, None)
    assert rc == hf.HF_ERR_SHAPE
    assert b"1048576" in hf.hair_fuse_last_error(None)


@pytest.mark.gpu
def test_matches_context_entry_point_on_two_calls_in_a_row():
    import torch

    import paper_2604_05794_b300 as hf
    dev = torch.device("cuda")
    for preset, kw in (("tiny", {}), ("tiny", dict(conf_f16=True, seed=11))):
        sc = scenegen.make_scene(preset, **kw)
        N, H, T, k = sc["N"], 32, 4, sc["k"]
        d = {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr")}
        mk = lambda: dict(dir=torch.empty((N, 3), device=dev), cost=torch.empty(N, device=dev),
                          idx=torch.empty(N, dtype=torch.int32, device=dev),
                          status=torch.empty(N, dtype=torch.uint8, device=dev))
        ref = mk()
        with hf.HairFuse(H, k, T) as f:
            f.upload_views(d["cams"], d["angle"], d["conf"])
            f.upload_points(d["points"], d["nbr"])
            f.fuse(ref["dir"], ref["cost"], ref["idx"], ref["status"])
            f.sync()
        cfg = hf.hf_config(H, k, T, 0, 0.0, 0)
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            out = mk()
            rc = _call(hf, cfg, sc, d, out, stream)
            assert rc == hf.HF_OK, hf.hair_fuse_last_error(None)
            torch.cuda.synchronize()
            assert torch.equal(out["status"], ref["status"])
            assert torch.equal(out["idx"], ref["idx"])
            g, r = out["cost"].cpu().numpy(), ref["cost"].cpu().numpy()
            assert np.all(np.abs(g - r) <= TOL_COST_RTOL * np.abs(r) + TOL_COST_ATOL)
            a, b = out["dir"].cpu().numpy().astype(np.float64), ref["dir"].cpu().numpy().astype(np.float64)
            ang = np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1))))
            assert np.max(ang) <= 0.1, (call, np.max(ang))


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
