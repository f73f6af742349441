"""Pins of the FP64 oracle of the paper's FPMVO step (candidate generation, medoid fusion, P x P
patch consistency; no GPU): the inverse projection against the projection, planted medoids,
exact recovery of a straight strand from maps the test renders itself, rigid invariance, and the
degenerate cases."""
import numpy as np
import pytest

import oracle
import scenegen

RNG = np.random.default_rng(7)


def look_at_cam(center, f=600.0, W=512, H=512):
    c = np.asarray(center, np.float64)
    fwd = -c / np.linalg.norm(c)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    return np.concatenate([[f, f, W / 2.0, H / 2.0], R.ravel(), -R @ c])


def test_backprojection_inverts_projection():
    for q in range(50):
        cam = look_at_cam(RNG.normal(size=3) * 3 + [0, 0, 0.1])
        if q % 2:
            # a matrix that is not orthonormal (a rotation stored in single precision is not exactly
            # either): the inverse projection must still land on the point, so R^T will not do
            cam[4:13] = (cam[4:13].reshape(3, 3) @ np.diag([1.01, 0.98, 1.0])).ravel()
        p = RNG.normal(size=3) * 0.3
        u, v = oracle.project(cam, p, 512, 512)[1:3]
        R = cam[4:13].reshape(3, 3)
        Z = (R @ p + cam[13:16])[2]
        assert np.allclose(oracle.backproject(cam, u, v, Z), p, atol=1e-12)


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_medoid_planted():
    d = _unit([1.0, 0.2, 0.1])
    # four copies (two sign-flipped) and an outlier: a copy wins, scoring 4/5 of the weight
    dirs = np.stack([d, -d, _unit([0.1, 1.0, 0.0]), d, -d])
    i, best, second = oracle.medoid(dirs, np.ones(5))
    assert i == 0                                      # the first of the tied copies
    assert best == pytest.approx((4 + abs(np.dot(d, dirs[2]))) / 5, abs=1e-15)
    # all identical up to sign: every score is 1, the first is taken
    i, best, second = oracle.medoid(np.stack([d, -d, d]), np.array([0.2, 0.5, 0.3]))
    assert i == 0 and best == pytest.approx(1.0) and second == pytest.approx(1.0)
    # weights decide between two clusters: two heavy candidates beat three light ones
    a, b = _unit([1.0, 0.0, 0.0]), _unit([0.0, 1.0, 0.0])
    i, _, _ = oracle.medoid(np.stack([b, a, b, a, b]), np.array([1.0, 10.0, 1.0, 10.0, 1.0]))
    assert i == 1
    # one candidate
    assert oracle.medoid(d[None], np.ones(1))[0] == 0


def _render_line(cams, a, b, W, H, n=40000):
    """Angle, confidence and depth maps of the segment a-b: dense samples projected to their nearest
    pixel, nearest depth wins; angle = the projected segment direction mod pi, confidence 1."""
    V = len(cams)
    ang = np.zeros((V, H, W), np.float32)
    conf = np.zeros((V, H, W), np.float32)
    dep = np.full((V, H, W), np.inf, np.float32)
    t = np.linspace(0.0, 1.0, n)[:, None]
    P = a + t * (b - a)
    for v, cam in enumerate(cams):
        R = cam[4:13].reshape(3, 3)
        X = P @ R.T + cam[13:16]
        u = cam[0] * X[:, 0] / X[:, 2] + cam[2]
        w = cam[1] * X[:, 1] / X[:, 2] + cam[3]
        du, dw = u[-1] - u[0], w[-1] - w[0]
        th = np.arctan2(dw, du) % np.pi
        x, y = np.floor(u).astype(int), np.floor(w).astype(int)
        inside = (x >= 0) & (x < W) & (y >= 0) & (y < H)
        for xi, yi, zi in zip(x[inside], y[inside], X[inside, 2]):
            if zi < dep[v, yi, xi]:
                dep[v, yi, xi] = zi
        cov = np.isfinite(dep[v])
        ang[v][cov] = th
        conf[v][cov] = 1.0
    return ang, conf, dep


def _line_scene(Q=np.eye(3), s=np.zeros(3)):
    """A vertical straight strand seen by six cameras on a ring in the y = 0 plane: the strand keeps
    one depth per view, so the undisturbed depth sample lands on it exactly."""
    W = H = 512
    cams = [look_at_cam(3.0 * np.array([np.cos(t), 0.0, np.sin(t)])) for t in np.linspace(0, 2 * np.pi, 6, endpoint=False)]
    a, b = np.array([0.01, -0.3, 0.02]), np.array([0.01, 0.3, 0.02])
    ang, conf, dep = _render_line(cams, a, b, W, H)
    pts = a + np.linspace(0.3, 0.7, 41)[:, None] * (b - a)
    # rigid motion of the world: p' = Q p + s, R' = R Q^T, t' = t - R' s (maps unchanged)
    cams2 = []
    for cam in cams:
        R2 = cam[4:13].reshape(3, 3) @ Q.T
        cams2.append(np.concatenate([cam[:4], R2.ravel(), cam[13:16] - R2 @ s]))
    # float64 geometry: the rigid motion stays exact up to double rounding
    sc = dict(N=len(pts), V=len(cams), W=W, H=H, k=0, points=pts @ Q.T + s,
              cams=np.array(cams2, np.float64), angle=ang, conf=conf, nbr=np.zeros((len(pts), 0), np.int32))
    return sc, dep, _unit(Q @ (b - a))


def test_straight_strand_recovered_exactly():
    sc, dep, t = _line_scene()
    r = oracle.fpmvo(oracle.Scene.from_dict(sc), dep, K=5, S=5, P=5, lambda_px=4.0, delta=0.01, eps_vis=0.02)
    assert np.all(r["status"] == oracle.OK)
    err = np.degrees(np.arccos(np.clip(np.abs(r["dir"] @ t), 0, 1)))
    assert np.max(err) < 1e-3, np.max(err)
    assert np.all(r["sel"] == 2)                       # the undisturbed depth sample
    assert np.all(r["cost"] < 1e-6)                    # every patch holds the exact orientation


def test_rigid_invariance():
    Q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
    s = np.array([0.05, -0.02, 0.03])
    sc0, dep, _ = _line_scene()
    sc1, _, _ = _line_scene(Q, s)
    # perturb the maps so the answer is not the exact strand
    noise = RNG.normal(size=sc0["angle"].shape).astype(np.float32) * 0.05
    for sc in (sc0, sc1):
        sc["angle"] = np.mod(sc["angle"] + noise, np.pi).astype(np.float32)
    r0 = oracle.fpmvo(oracle.Scene.from_dict(sc0), dep, delta=0.01)
    r1 = oracle.fpmvo(oracle.Scene.from_dict(sc1), dep, delta=0.01)
    ok = (r0["flags"] == 0) & (r1["flags"] == 0)
    assert ok.mean() > 0.8
    assert np.array_equal(r0["sel"][ok], r1["sel"][ok])
    assert np.allclose(r0["cost"][ok], r1["cost"][ok], atol=1e-9)
    d0 = r0["dir"][ok] @ Q.T
    assert np.allclose(np.abs(np.sum(d0 * r1["dir"][ok], axis=1)), 1.0, atol=1e-9)


def test_degenerate_points():
    sc, dep, _ = _line_scene()
    sc["points"] = sc["points"].copy()
    sc["points"][0] = np.nan                           # non-finite input
    sc["points"][1] = [0.0, 0.0, 50.0]                 # outside every view
    r = oracle.fpmvo(oracle.Scene.from_dict(sc), dep, delta=0.01)
    assert r["status"][0] == oracle.BAD_INPUT and np.isnan(r["cost"][0])
    assert r["status"][1] == oracle.NO_VIEWS and r["cost"][1] == 1.0 and r["sel"][1] == -1
    # a point behind the depth maps everywhere is seen by no view
    far = dep.copy()
    far[np.isinf(far)] = 0.5
    r = oracle.fpmvo(oracle.Scene.from_dict(sc), np.minimum(far, 0.5), delta=0.01)
    assert np.all(r["status"][1:] == oracle.NO_VIEWS)


def test_layer_outputs():
    """Per-layer results: the best layer is the output, and the depth samples are laid out evenly
    over [-Delta, Delta], so 3 samples are the first, middle and last of 5 and 1 is the middle."""
    sc = scenegen.make_scene("tiny", depth=True)
    scene = oracle.Scene.from_dict(sc)
    r5 = oracle.fpmvo(scene, sc["depth"], S=5, delta=0.02, layers=True)
    r3 = oracle.fpmvo(scene, sc["depth"], S=3, delta=0.02, layers=True)
    r1 = oracle.fpmvo(scene, sc["depth"], S=1, delta=0.02, layers=True)
    ok = r5["status"] == oracle.OK
    assert ok.mean() > 0.8
    assert np.array_equal(np.max(r5["layer_L"][ok], axis=1), 1.0 - r5["cost"][ok])
    assert np.array_equal(r5["layer_dir"][ok, r5["sel"][ok]], r5["dir"][ok])
    assert np.array_equal(r3["layer_L"], r5["layer_L"][:, [0, 2, 4]])
    assert np.array_equal(r1["layer_L"][:, 0], r5["layer_L"][:, 2])
    assert np.array_equal(r3["layer_dir"], r5["layer_dir"][:, [0, 2, 4]])


def test_scene_runs_and_flags_are_rare():
    sc = scenegen.make_scene("tiny", depth=True)
    r = oracle.fpmvo(oracle.Scene.from_dict(sc), sc["depth"], delta=0.02)
    assert np.mean(r["status"] == oracle.OK) > 0.8
    assert np.all(np.isfinite(r["cost"][r["status"] == oracle.OK]))
    assert np.mean(r["flags"] != 0) < 0.1
