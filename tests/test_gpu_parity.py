"""GPU parity of the fusion path against the FP64 oracle (needs a B300 and the built library).

Every comparison runs the CUDA library through its C ABI (ctypes binding) and the oracle on the
same seeded inputs; see helpers.py for the tolerances and the exemptions."""
import numpy as np
import pytest

import oracle
import scenegen
from helpers import angle_deg, compare, library_eval_costs, run_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    return scenegen.make_scene("tiny")


def lib_hyps(H):
    import paper_2604_05794_b300 as hf
    return hf.fibonacci_hemisphere(H)


def test_builtin_hypotheses_are_the_fibonacci_hemisphere():
    for H in (8, 32, 64, 100):
        got = lib_hyps(H).astype(np.float64)
        want = oracle.fibonacci_hemisphere(H)
        assert np.max(np.abs(got - want)) <= 2 ** -23


def test_tiny_scene_all_points(tiny):
    H, T = 32, 4
    hyps = lib_hyps(H)
    gpu = run_library(tiny, H, T)                    # built-in hypotheses
    osc = oracle.Scene.from_dict(tiny)
    orc = oracle.fuse(osc, hyps, T)
    st = compare(gpu, orc, np.arange(tiny["N"]), osc, hyps, H)
    print("tiny", st)
    assert st["boundary"] <= 2


def test_cost_table_elementwise(tiny):
    """c_i(h_m) for every point and hypothesis plus random directions, element by element."""
    H = 32
    hyps = lib_hyps(H)
    rng = np.random.default_rng(3)
    rnd = rng.normal(size=(tiny["N"], 8, 3)).astype(np.float32)
    dirs = np.concatenate([np.broadcast_to(hyps, (tiny["N"], H, 3)), rnd], axis=1).astype(np.float32)
    got = library_eval_costs(tiny, dirs)
    osc = oracle.Scene.from_dict(tiny)
    want = oracle.eval_costs(osc, dirs.astype(np.float64))
    flags = oracle.fuse(osc, hyps, 0)["flags"]
    keep = (flags & oracle.FLAG_BOUNDARY) == 0
    err = np.abs(got - want)
    assert np.all((err <= 1e-4 * np.abs(want) + 1e-6)[keep]), np.max(err[keep])


def test_explicit_hypotheses_equal_builtin(tiny):
    H, T = 32, 4
    a = run_library(tiny, H, T)
    b = run_library(tiny, H, T, hyps=lib_hyps(H))
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_host_and_device_calls_agree_bitwise(tiny):
    H, T = 32, 4
    a = run_library(tiny, H, T, device=True)
    b = run_library(tiny, H, T, device=False)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_deterministic(tiny):
    a = run_library(tiny, 32, 4)
    b = run_library(tiny, 32, 4)
    for key in a:
        assert np.array_equal(a[key], b[key]), key


def test_neighbour_order_does_not_matter(tiny):
    """The patch maximum is over a set (Eq. patch_min): permuting each point's neighbour list (the
    library reorders it for its gathers) gives the same outputs bit for bit, k = 8 and k = 16."""
    rng = np.random.default_rng(11)
    for k in (8, 16):
        sc = dict(tiny)
        sc["nbr"] = scenegen.knn_of(tiny["points"], k)
        a = run_library(sc, 32, 4)
        sc["nbr"] = np.ascontiguousarray(rng.permuted(sc["nbr"], axis=1))
        b = run_library(sc, 32, 4)
        for key in a:
            assert np.array_equal(a[key], b[key]), (k, key)


@pytest.mark.parametrize("V", [1, 7, 21])
def test_odd_view_counts(V):
    """Samples and ratios are stored in view pairs: with an odd V the last pair's second half is
    padding that no kernel may read as a view (one view, and the point-per-thread and lanes layouts)."""
    sc = scenegen.make_scene("mid", seed=30 + V, n_strands=40, V=V, width=384, height=384, f=450.0)
    H, T = 32, 4
    hyps = lib_hyps(H)
    gpu = run_library(sc, H, T)
    osc = oracle.Scene.from_dict(sc)
    orc = oracle.fuse(osc, hyps, T)
    compare(gpu, orc, np.arange(sc["N"]), osc, hyps, H, strict_frac=0.9)


@pytest.mark.parametrize("n", [1, 2, 7, 127, 128, 129, 300])
def test_ragged_sizes(tiny, n):
    sub = scenegen.subset_scene(tiny, np.arange(0, tiny["N"], tiny["N"] // n)[:n])   # k = min(5, n - 1)
    H, T = 32, 4
    hyps = lib_hyps(H)
    gpu = run_library(sub, H, T)
    osc = oracle.Scene.from_dict(sub)
    orc = oracle.fuse(osc, hyps, T)
    compare(gpu, orc, np.arange(n), osc, hyps, H, strict_frac=0.9 if n >= 10 else 0.0)


@pytest.mark.parametrize("H,T", [(8, 0), (16, 2), (64, 6), (100, 3)])
def test_other_hypothesis_counts_and_rounds(tiny, H, T):
    hyps = lib_hyps(H)
    gpu = run_library(tiny, H, T)
    osc = oracle.Scene.from_dict(tiny)
    orc = oracle.fuse(osc, hyps, T)
    compare(gpu, orc, np.arange(tiny["N"]), osc, hyps, H)


@pytest.mark.parametrize("K", [1, 3, 5])
def test_top_k_views(tiny, K):
    H, T = 32, 4
    hyps = lib_hyps(H)
    gpu = run_library(tiny, H, T, top_k=K)
    osc = oracle.Scene.from_dict(tiny)
    orc = oracle.fuse(osc, hyps, T, top_k=K)
    st = compare(gpu, orc, np.arange(tiny["N"]), osc, hyps, H, top_k=K)
    print("top", K, st)


def test_fp16_confidence():
    sc = scenegen.make_scene("tiny", conf_f16=True)
    H, T = 32, 4
    hyps = lib_hyps(H)
    gpu = run_library(sc, H, T)
    osc = oracle.Scene.from_dict(sc)
    orc = oracle.fuse(osc, hyps, T)
    compare(gpu, orc, np.arange(sc["N"]), osc, hyps, H)


def test_patch_sizes(tiny):
    for k in (0, 1, 3, 8, 11, 16):
        sc = dict(tiny)
        sc["nbr"] = scenegen.knn_of(tiny["points"], k) if k else np.zeros((tiny["N"], 0), np.int32)
        hyps = lib_hyps(16)
        gpu = run_library(sc, 16, 2)
        osc = oracle.Scene.from_dict(sc)
        orc = oracle.fuse(osc, hyps, 2)
        compare(gpu, orc, np.arange(tiny["N"]), osc, hyps, 16)


def test_bad_and_invisible_points(tiny):
    pts = tiny["points"].copy()
    pts[5] = [np.nan, 0.0, 0.0]
    pts[6] = [np.inf, 1.0, 0.0]
    pts[7] = [0.0, 40.0, 0.0]       # far above: outside every view
    gpu = run_library(tiny, 32, 4, points=pts)
    assert gpu["status"][5] == 2 and gpu["status"][6] == 2 and gpu["status"][7] == 1
    assert gpu["cost"][7] == 1.0 and gpu["idx"][5] == -1
    osc = oracle.Scene(pts, tiny["cams"], tiny["angle"], tiny["conf"], tiny["nbr"])
    orc = oracle.fuse(osc, lib_hyps(32), 4)
    compare(gpu, orc, np.arange(tiny["N"]), osc, lib_hyps(32), 32)


def test_invalid_arguments(tiny):
    import torch

    import paper_2604_05794_b300 as hf
    f = hf.HairFuse(32, 5, 4)
    out = torch.empty((tiny["N"], 3), device="cuda")
    with pytest.raises(hf.HairFuseError) as e:
        f.fuse(out)
    assert e.value.code == hf.HF_ERR_NOT_UPLOADED
    f.upload_views(tiny["cams"], tiny["angle"], tiny["conf"])
    bad = tiny["nbr"].copy()
    bad[3, 2] = tiny["N"]
    with pytest.raises(hf.HairFuseError) as e:
        f.upload_points(tiny["points"], bad)
    assert e.value.code == hf.HF_ERR_INVALID_ARG
    bad_dev = torch.from_numpy(tiny["nbr"].copy()).cuda()
    bad_dev[9, 0] = -1
    with pytest.raises(hf.HairFuseError):
        f.upload_points(torch.from_numpy(tiny["points"]).cuda(), bad_dev)
    with pytest.raises(hf.HairFuseError):
        f.upload_points(tiny["points"][:5], tiny["nbr"][:5])          # k = 5 >= N = 5
    f.upload_points(tiny["points"], tiny["nbr"])
    hy = lib_hyps(32) * 1.01
    with pytest.raises(hf.HairFuseError) as e:
        f.fuse(np.empty((tiny["N"], 3), np.float32), hyps=hy)
    assert e.value.code == hf.HF_ERR_INVALID_ARG
    # a device-side bad hypothesis is latched and reported by the next synchronising call
    hy_dev = torch.from_numpy(hy).cuda()       # kept alive until the stream has read it
    f.fuse(out, hyps=hy_dev)
    with pytest.raises(hf.HairFuseError):
        f.sync()
    f.sync()   # cleared
    # a map side above 2^22 pixels is refused before anything is copied
    wide = np.zeros((1, 1, (1 << 22) + 1), np.float32)
    with pytest.raises(hf.HairFuseError) as e:
        f.upload_views(tiny["cams"][:1], wide, wide)
    assert e.value.code == hf.HF_ERR_SHAPE
    f.close()


def _sampled(scene, step, H, T):
    sel = np.unique(np.concatenate([np.arange(0, scene["N"], step), np.arange(scene["N"] - 5, scene["N"])]))
    hyps = lib_hyps(H)
    gpu = run_library(scene, H, T)
    osc = oracle.Scene.from_dict(scene)
    orc = oracle.fuse(osc, hyps, T, idx=sel)
    return compare(gpu, orc, sel, osc, hyps, H)


def test_mid_scene_sampled():
    sc = scenegen.make_scene("mid")
    st = _sampled(sc, 97, 64, 8)
    print("mid", st)


def test_full_scene_sampled():
    """1M points, 64 views of 1920x1080 (fp16 confidence): the whole scene on the GPU in the
    benchmark's launch configuration, ~2,000 sampled points on the oracle."""
    sc = scenegen.make_scene("full")
    st = _sampled(sc, 499, 64, 8)
    print("full", st)
    assert st["median_deg"] <= 2.0
