"""Synthetic scene generator: determinism, shapes, kNN by brute force, fp16 rounding (no GPU)."""
import numpy as np

import scenegen


def test_deterministic_and_seed_dependent():
    a = scenegen.make_scene("tiny")
    b = scenegen.make_scene("tiny")
    c = scenegen.make_scene("tiny", seed=7)
    for key in ("points", "tangents", "cams", "angle", "conf", "nbr"):
        assert np.array_equal(a[key], b[key]), key
    assert not np.array_equal(a["points"], c["points"])


def test_shapes_and_ranges():
    s = scenegen.make_scene("tiny")
    N, V, H, W, k = s["N"], s["V"], s["H"], s["W"], s["k"]
    assert (N, V, H, W, k) == (2000, 8, 256, 256, 5)
    assert s["points"].shape == (N, 3) and s["cams"].shape == (V, 16)
    assert s["angle"].shape == (V, H, W) and s["conf"].shape == (V, H, W)
    assert s["angle"].min() >= 0 and s["angle"].max() < np.pi
    assert s["conf"].min() >= 0 and s["conf"].max() <= 1
    assert np.allclose(np.linalg.norm(s["tangents"], axis=1), 1, atol=1e-6)
    # roots lie on the unit sphere cap, strands grow outward
    r = np.linalg.norm(s["points"], axis=1)
    assert r.min() > 0.95 and r.max() < 1.5
    # rotations in the camera records are orthonormal
    for cam in s["cams"]:
        R = cam[4:13].reshape(3, 3).astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)


def test_mid_outliers_and_point_count():
    s = scenegen.make_scene("mid", knn=False, n_strands=300, width=256, height=256, V=4)
    assert s["N"] == 300 * 40
    low = (s["conf"] < 0.3) & (s["conf"] > 0)
    # about 10 % of pixels are outliers with confidence below 0.3
    assert 0.07 < low.mean() < 0.13


def test_knn_matches_brute_force():
    s = scenegen.make_scene("tiny", n_strands=60)
    p = s["points"].astype(np.float64)
    d = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d, np.inf)
    idx = np.broadcast_to(np.arange(len(p)), d.shape)
    want = np.lexsort((idx, d), axis=1)[:, :5]
    assert np.array_equal(want, s["nbr"])


def test_knn_ties_go_to_lower_index():
    pts = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, 5]], np.float32)
    nbr = scenegen.knn_of(pts, 3)
    assert nbr[0].tolist() == [1, 2, 3]


def test_fp16_confidence_rounds_like_numpy():
    a = scenegen.make_scene("tiny", conf_f16=False)
    b = scenegen.make_scene("tiny", conf_f16=True)
    assert b["conf"].dtype == np.float16
    assert np.array_equal(a["conf"].astype(np.float16), b["conf"])


def test_exact_maps_owner_semantics():
    s = scenegen.make_scene("tiny", exact_maps=True, strand_maps=False)
    assert s["owner"].shape == (s["V"], s["N"])
    # each covered pixel has exactly one owner, so owners per view == covered pixels per view
    for v in range(s["V"]):
        assert s["owner"][v].sum() == int((s["exact_conf"][v] == 1).sum())
