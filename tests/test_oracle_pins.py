"""Pins of the FP64 oracle against facts fixed by the paper and by geometry (no GPU).

Each test ties a part of the oracle to something other than itself: hand-computed
projections, finite differences of the projection, closed forms for one and two views,
constructed patches, invariances (direction sign, rigid motion), brute force over the
hypothesis set, and independent library routines (numpy's half decoding).
"""
import numpy as np
import pytest

import oracle
import scenegen

RNG = np.random.default_rng(12345)


# ----------------------------------------------------------------------------- helpers

def look_at_cam(center, f=300.0, W=256, H=256):
    """16-float camera looking at the origin from `center`, world up +y (x right, y down)."""
    c = np.asarray(center, np.float64)
    fwd = -c / np.linalg.norm(c)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ c
    return np.concatenate([[f, f, W / 2.0, H / 2.0], R.ravel(), t])


def const_maps(V, W, H, theta, conf):
    ang = np.empty((V, H, W), np.float32)
    cf = np.empty((V, H, W), np.float32)
    for v in range(V):
        ang[v] = theta[v]
        cf[v] = conf[v]
    return ang, cf


def pinhole(cam, p):
    """Textbook pinhole u = fx X/Z + cx, v = fy Y/Z + cy with X = R p + t (test's own)."""
    R = np.asarray(cam[4:13]).reshape(3, 3)
    X = R @ p + cam[13:16]
    return np.array([cam[0] * X[0] / X[2] + cam[2], cam[1] * X[1] / X[2] + cam[3]])


def image_angle_finite(cam, p, d, eps=1e-7):
    """Angle of the image of the short segment p -> p + eps d (Eq. proj_r with a finite offset)."""
    r = pinhole(cam, p + eps * d) - pinhole(cam, p)
    return np.arctan2(r[1], r[0])


def rand_unit(n):
    v = RNG.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.fixture(scope="module")
def tiny():
    return scenegen.make_scene("tiny", exact_maps=True)


# ----------------------------------------------------------------------------- projection

def test_projection_hand_values():
    cam = np.array([300, 300, 128, 128, 1, 0, 0, 0, -1, 0, 0, 0, -1, 0, 0, 3], np.float64)
    vis, u, v, a, b = oracle.project(cam, [0.3, 0.6, 0.0], 256, 256)
    assert vis == 1 and u == pytest.approx(158.0, abs=1e-12) and v == pytest.approx(68.0, abs=1e-12)
    assert a == pytest.approx(0.1) and b == pytest.approx(-0.2)
    assert oracle.project(cam, [0.0, 0.0, 3.5], 256, 256)[0] == 0          # behind the camera
    assert oracle.project(cam, [5.0, 0.0, 0.0], 256, 256)[0] == 0          # right of the frame
    # u = 0 is inside, u = W is outside (pixel (floor u, floor v), 0 <= u < W)
    assert oracle.project(cam, [-128.0 / 100.0, 0.0, 0.0], 256, 256)[0] == 1
    assert oracle.project(cam, [128.0 / 100.0, 0.0, 0.0], 256, 256)[0] == 0


def test_jacobian_matches_central_difference():
    for _ in range(50):
        cam = look_at_cam(rand_unit(1)[0] * 3.0)
        p = RNG.uniform(-0.5, 0.5, 3)
        d = rand_unit(1)[0]
        r = oracle.reproject_dir(cam, p, d)
        for eps in (1e-4, 1e-5):
            up = oracle.project(cam, p + eps * d, 256, 256)
            um = oracle.project(cam, p - eps * d, 256, 256)
            fd = np.array([up[1] - um[1], up[2] - um[2]]) / (2 * eps)
            assert np.linalg.norm(fd - r) <= 1e-7 * np.linalg.norm(r) + 1e-9


# ----------------------------------------------------------------------------- closed forms

def test_single_view_closed_form():
    """V = 1, k = 0, C = 1: c(d) = 1 - |cos(psi(d) - theta)|, psi the image angle of d."""
    W = H = 256
    cam = look_at_cam([0.7, 0.4, 2.9], W=W, H=H)
    theta = 0.7
    ang, cf = const_maps(1, W, H, [theta], [1.0])
    pts = RNG.uniform(-0.3, 0.3, (20, 3))
    sc = oracle.Scene(pts, cam[None], ang, cf, None)
    dirs = rand_unit(20 * 16).reshape(20, 16, 3)
    got = oracle.eval_costs(sc, dirs)
    for i in range(20):
        for m in range(16):
            psi = image_angle_finite(cam, pts[i], dirs[i, m])
            want = 1.0 - abs(np.cos(psi - theta))
            assert got[i, m] == pytest.approx(want, abs=2e-6)
    # the zero set: any direction in the plane of the viewing ray and the back-projected image line
    R = cam[4:13].reshape(3, 3)
    centre = -R.T @ cam[13:16]
    for i in range(20):
        Z = (R @ pts[i] + cam[13:16])[2]
        w = R.T @ np.array([np.cos(theta) * Z / cam[0], np.sin(theta) * Z / cam[1], 0.0])
        ray = pts[i] - centre
        for beta in np.linspace(0, np.pi, 7):
            d = np.cos(beta) * ray / np.linalg.norm(ray) + np.sin(beta) * w / np.linalg.norm(w)
            if np.linalg.norm(np.cross(d, ray)) < 1e-3 * np.linalg.norm(ray):
                continue  # along the ray itself the image offset vanishes
            assert oracle.eval_costs(sc, d[None, None], idx=[i])[0, 0] < 1e-12
    # a direction along the viewing ray has no image offset: the view contributes L = 0
    d = (pts[0] - centre) / np.linalg.norm(pts[0] - centre)
    assert oracle.eval_costs(sc, d[None, None], idx=[0])[0, 0] == pytest.approx(1.0, abs=1e-9)


def _two_view_scene(t, conf=(1.0, 1.0), k=0):
    W = H = 256
    cams = np.stack([look_at_cam([0.0, 0.3, 3.0]), look_at_cam([2.6, -0.2, 1.5])])
    p = np.array([0.05, -0.02, 0.1])
    thetas = [image_angle_finite(cams[v], p, t) % np.pi for v in range(2)]
    ang, cf = const_maps(2, W, H, thetas, conf)
    return oracle.Scene(p[None], cams, ang, cf, None), cams, p


def test_two_view_recovers_planted_direction():
    """Two views with exact orientation at the point: the zero-cost direction is the
    intersection of the two back-projected line planes, i.e. the planted tangent."""
    for _ in range(5):
        t = rand_unit(1)[0]
        sc, cams, p = _two_view_scene(t)
        assert oracle.eval_costs(sc, t[None, None])[0, 0] < 1e-10
        # plane normals n_v = ray_v x w_v; n_1 x n_2 is parallel to t
        ns = []
        for v in range(2):
            R = cams[v][4:13].reshape(3, 3)
            centre = -R.T @ cams[v][13:16]
            th = float(sc.angle[v, 0, 0])
            Z = (R @ p + cams[v][13:16])[2]
            w = R.T @ np.array([np.cos(th) * Z / cams[v][0], np.sin(th) * Z / cams[v][1], 0.0])
            ns.append(np.cross(p - centre, w))
        n12 = np.cross(ns[0], ns[1])
        n12 /= np.linalg.norm(n12)
        assert abs(abs(n12 @ t) - 1.0) < 1e-9
        hyps = oracle.fibonacci_hemisphere(64)
        res = oracle.fuse(sc, hyps, T=22)
        ang_err = np.arccos(min(1.0, abs(res["dir"][0] @ t)))
        assert ang_err < 1e-4, ang_err
        assert res["cost"][0] < 1e-8


def test_view_aggregation_is_unweighted_mean():
    """c = 1 - (L_1 + L_2)/2 with L_v = C_v |cos(psi_v - theta_v)| (Eqs. patchloss, final_dout)."""
    t = rand_unit(1)[0]
    sc, cams, p = _two_view_scene(t, conf=(1.0, 0.5))
    assert oracle.eval_costs(sc, t[None, None])[0, 0] == pytest.approx(1 - (1.0 + 0.5) / 2, abs=1e-10)
    for d in rand_unit(10):
        L = [c * abs(np.cos(image_angle_finite(cams[v], p, d) - sc.angle[v, 0, 0]))
             for v, c in enumerate((1.0, 0.5))]
        assert oracle.eval_costs(sc, d[None, None])[0, 0] == pytest.approx(1 - np.mean(L), abs=2e-6)


def test_patch_max_closed_form():
    """Patch = point + neighbour, each sampled at its own pixel: L = max_j C_j |cos(psi - theta_j)|."""
    W = H = 64
    cam = look_at_cam([0.0, 0.0, 3.0], f=100.0, W=W, H=H)
    pts = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.1]])
    ang = np.zeros((1, H, W), np.float32)
    cf = np.zeros((1, H, W), np.float32)
    th, C = [0.4, 2.1], [0.3, 0.8]
    for j in range(2):
        u, v = pinhole(cam, pts[j])
        ang[0, int(np.floor(v)), int(np.floor(u))] = th[j]
        cf[0, int(np.floor(v)), int(np.floor(u))] = C[j]
    nbr = np.array([[1], [0]], np.int32)
    sc = oracle.Scene(pts, cam[None], ang, cf, nbr)
    for d in rand_unit(40):
        psi = image_angle_finite(cam, pts[0], d)
        L = max(C[0] * abs(np.cos(psi - th[0])), C[1] * abs(np.cos(psi - th[1])))
        assert oracle.eval_costs(sc, d[None, None], idx=[0])[0, 0] == pytest.approx(1 - L, abs=2e-6)
    # a neighbour outside the frame contributes nothing
    pts2 = pts.copy()
    pts2[1] = [50.0, 0.0, 0.0]
    sc2 = oracle.Scene(pts2, cam[None], ang, cf, nbr)
    for d in rand_unit(10):
        psi = image_angle_finite(cam, pts[0], d)
        L = C[0] * abs(np.cos(psi - th[0]))
        assert oracle.eval_costs(sc2, d[None, None], idx=[0])[0, 0] == pytest.approx(1 - L, abs=2e-6)


# ----------------------------------------------------------------------------- invariances

def test_sign_invariance_bitwise(tiny):
    sc = oracle.Scene.from_dict(tiny)
    d = rand_unit(tiny["N"] * 4).reshape(tiny["N"], 4, 3)
    a = oracle.eval_costs(sc, d)
    b = oracle.eval_costs(sc, -d)
    assert np.array_equal(a, b)


def _rigid(sc_dict, Q, s):
    pts = sc_dict["points"].astype(np.float64) @ Q.T + s
    cams = sc_dict["cams"].astype(np.float64).copy()
    for v in range(len(cams)):
        R = cams[v, 4:13].reshape(3, 3)
        R2 = R @ Q.T
        cams[v, 4:13] = R2.ravel()
        cams[v, 13:16] = cams[v, 13:16] - R2 @ s
    return oracle.Scene(pts, cams, sc_dict["angle"], sc_dict["conf"], sc_dict["nbr"])


def _rand_rotation():
    q = RNG.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def test_rigid_invariance_of_cost(tiny):
    sc = oracle.Scene.from_dict(tiny)
    Q, s = _rand_rotation(), RNG.normal(size=3)
    sc2 = _rigid(tiny, Q, s)
    d = rand_unit(tiny["N"] * 3).reshape(tiny["N"], 3, 3)
    a = oracle.eval_costs(sc, d)
    b = oracle.eval_costs(sc2, d @ Q.T)
    flags = oracle.fuse(sc, oracle.fibonacci_hemisphere(8), T=0)["flags"]
    ok = (flags & oracle.FLAG_BOUNDARY) == 0
    assert ok.mean() > 0.95
    assert np.max(np.abs(a - b)[ok]) < 1e-12


def test_rigid_equivariance_of_fusion(tiny):
    """Under a signed axis permutation Q (which maps the refinement's rotation axes onto
    themselves) and any translation, fused directions map by Q and costs are unchanged."""
    sc = oracle.Scene.from_dict(tiny)
    Q = np.array([[0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    s = np.array([0.37, -1.2, 0.55])
    sc2 = _rigid(tiny, Q, s)
    hyps = oracle.fibonacci_hemisphere(32)
    r1 = oracle.fuse(sc, hyps, T=4)
    r2 = oracle.fuse(sc2, hyps @ Q.T, T=4)
    ok = (r1["flags"] == 0) & (r2["flags"] == 0)
    assert ok.mean() > 0.9
    assert np.array_equal(r1["idx"][ok], r2["idx"][ok])
    assert np.max(np.abs(r1["cost"] - r2["cost"])[ok]) < 1e-12
    a, b = r1["dir"] @ Q.T, r2["dir"]
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1)))
    assert np.max(np.degrees(ang[ok])) < 1e-6


# ----------------------------------------------------------------------------- argmin, refine, exact maps

def test_argmin_matches_exhaustive_evaluation(tiny):
    sc = oracle.Scene.from_dict(tiny)
    hyps = oracle.fibonacci_hemisphere(32)
    idx = np.arange(0, tiny["N"], 40)
    costs = oracle.eval_costs(sc, np.broadcast_to(hyps, (len(idx), 32, 3)), idx=idx)
    res = oracle.fuse(sc, hyps, T=0, idx=idx)
    assert np.array_equal(res["idx"], np.argmin(costs, axis=1))
    assert np.array_equal(res["cost"], costs.min(axis=1))
    h = hyps[res["idx"]]
    sgn = np.where(np.abs(h[:, 2]) > 1e-12, np.sign(h[:, 2]), 1.0)
    assert np.allclose(res["dir"], h * sgn[:, None], atol=1e-15)


def test_refinement_descends_and_reports_own_cost(tiny):
    sc = oracle.Scene.from_dict(tiny)
    hyps = oracle.fibonacci_hemisphere(32)
    r0 = oracle.fuse(sc, hyps, T=0)
    r4 = oracle.fuse(sc, hyps, T=4)
    assert np.all(r4["cost"] <= r0["cost"])
    assert np.array_equal(r4["idx"], r0["idx"])
    again = oracle.eval_costs(sc, r4["dir"][:, None, :])[:, 0]
    assert np.max(np.abs(again - r4["cost"])) < 1e-12
    # canonical sign: first of z, y, x with |.| > 1e-12 is positive
    d = r4["dir"]
    first = np.where(np.abs(d[:, 2]) > 1e-12, d[:, 2], np.where(np.abs(d[:, 1]) > 1e-12, d[:, 1], d[:, 0]))
    assert np.all(first > 0)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)


def test_refine_from_start_keeps_the_exact_tangent(tiny):
    """Learned-path refinement from a given start: on point-splatted exact maps the true tangent
    costs 0 and nothing is strictly lower, so a start at the tangent stays there (up to the
    canonical sign) with cost 0, for any step size; a start rotated away by a few degrees is
    pulled back to within the last step of the tangent."""
    se = oracle.Scene.from_dict(tiny, exact=True)
    N, V = tiny["N"], tiny["V"]
    vis = np.array([[oracle.project(tiny["cams"][v], tiny["points"][i], tiny["W"], tiny["H"])[0]
                     for v in range(V)] for i in range(N)])
    owns = np.nonzero(np.all((tiny["owner"].T == 1) | (vis == 0), axis=1) & (vis.sum(1) >= 2))[0][:200]
    t = tiny["tangents"][owns].astype(np.float64)
    for alpha in (0.02, 0.2):
        r = oracle.refine(se, t, 4, alpha, idx=owns)
        assert np.all(r["cost"] <= 1e-12)
        assert np.allclose(np.abs(np.sum(r["dir"] * t, axis=1)), 1.0, atol=1e-12)
    # a small rotation about a random axis perpendicular to the tangent
    ax = np.cross(t, rand_unit(len(t)))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = np.radians(3.0)
    start = t * np.cos(ang) + np.cross(ax, t) * np.sin(ang)
    r = oracle.refine(se, start, 8, np.radians(4.0), idx=owns)
    c0 = oracle.eval_costs(se, start[:, None, :], idx=owns)[:, 0]
    assert np.all(r["cost"] <= c0)
    err = np.degrees(np.arccos(np.clip(np.abs(np.sum(r["dir"] * t, axis=1)), 0, 1)))
    assert np.median(err) < 4.0 * 2.0 ** -7 * 2


def test_refine_from_argmin_hypothesis_is_the_fused_refinement(tiny):
    """Started at the argmin hypothesis with the hypothesis-derived first step 1/2 sqrt(2 pi / H),
    the learned-path refinement reproduces the plain fusion's refinement exactly (same rotation
    order, halving and sign rule)."""
    sc = oracle.Scene.from_dict(tiny)
    H = 32
    hyps = oracle.fibonacci_hemisphere(H)
    idx = np.arange(0, tiny["N"], 7)
    fused = oracle.fuse(sc, hyps, T=4, idx=idx)
    start = oracle.fuse(sc, hyps, T=0, idx=idx)
    r = oracle.refine(sc, hyps[start["idx"]], 4, 0.5 * np.sqrt(2 * np.pi / H), idx=idx)
    ok = fused["status"] == oracle.OK
    assert np.array_equal(r["dir"][ok], fused["dir"][ok])
    assert np.array_equal(r["cost"][ok], fused["cost"][ok])


def test_dense_sphere_bounds_the_fused_cost(tiny):
    """Brute force over a 20,000-direction Fibonacci hemisphere on a 50-point slice: no fused
    cost lies below the dense minimum by more than the cost change over one grid spacing, and
    on most points the fused direction reaches that minimum closely."""
    sc = oracle.Scene.from_dict(tiny)
    idx = np.arange(0, tiny["N"], 40)[:50]
    dense = oracle.fibonacci_hemisphere(20000)
    c_dense = oracle.eval_costs(sc, np.broadcast_to(dense, (len(idx), 20000, 3)), idx=idx)
    res = oracle.fuse(sc, oracle.fibonacci_hemisphere(32), T=4, idx=idx)
    spacing = np.sqrt(2 * np.pi / 20000)
    lip = 2.0 * 64.0  # |dc/dangle| <= sum over views of the image-angle rate, bounded loosely
    assert np.all(res["cost"] >= c_dense.min(axis=1) - lip * spacing)
    close = res["cost"] <= c_dense.min(axis=1) + 0.05
    assert close.mean() > 0.5


def test_true_tangent_is_zero_cost_on_exact_maps(tiny):
    """Point-splatted maps of the true tangents (C = 1 at owned pixels, 0 elsewhere): for every
    point owning its pixel in each view that sees it, the true tangent has cost 0, and costs
    are never negative, so it is a minimiser."""
    se = oracle.Scene.from_dict(tiny, exact=True)
    N, V = tiny["N"], tiny["V"]
    vis = np.array([[oracle.project(tiny["cams"][v], tiny["points"][i], tiny["W"], tiny["H"])[0]
                     for v in range(V)] for i in range(N)])
    owns = np.all((tiny["owner"].T == 1) | (vis == 0), axis=1) & (vis.sum(1) > 0)
    assert owns.mean() > 0.4
    c_true = oracle.eval_costs(se, tiny["tangents"][:, None, :])[:, 0]
    assert np.all(c_true[owns] <= 1e-12)
    hyps = oracle.fibonacci_hemisphere(32)
    c_h = oracle.eval_costs(se, np.broadcast_to(hyps, (N, 32, 3)))
    assert c_h.min() >= 0.0 and c_true.min() >= 0.0
    assert np.all(c_true[owns][:, None] <= c_h[owns])


# ----------------------------------------------------------------------------- views, statuses, inputs

def test_top_k_selection_brute_force(tiny):
    sc = oracle.Scene.from_dict(tiny)
    se = oracle.Scene.from_dict(tiny, exact=True)   # C = 1 at many pixels: exact ties
    for scene in (sc, se):
        for i in range(0, tiny["N"], 97):
            confs = []
            for v in range(tiny["V"]):
                vis, u, vv, _, _ = oracle.project(tiny["cams"][v], tiny["points"][i], tiny["W"], tiny["H"])
                if vis:
                    confs.append((-float(scene.conf[v, int(np.floor(vv)), int(np.floor(u))]), v))
            for K in (1, 3, 5):
                want = sorted(confs)[:K]
                n, mask = oracle.view_set(scene, i, K)
                assert n == min(K, len(confs))
                assert set(np.nonzero(mask)[0]) == {v for _, v in want}
            # the cost with top-K uses exactly those views
            n, mask = oracle.view_set(scene, i, 3)
            d = rand_unit(1)[0]
            terms = [oracle.view_term(scene, i, v, d) for v in np.nonzero(mask)[0]]
            assert oracle.eval_costs(scene, d[None, None], idx=[i], top_k=3)[0, 0] == \
                pytest.approx(1 - np.mean(terms), abs=1e-15)


def test_no_views_and_bad_input():
    cam = look_at_cam([0.0, 0.0, 3.0])
    ang, cf = const_maps(1, 256, 256, [0.3], [1.0])
    pts = np.array([[0.0, 0.0, 4.0], [np.nan, 0.0, 0.0], [0.1, 0.1, 0.1]])
    nbr = np.array([[2], [2], [0]], np.int32)
    sc = oracle.Scene(pts, cam[None], ang, cf, nbr)
    res = oracle.fuse(sc, oracle.fibonacci_hemisphere(16), T=2)
    assert res["status"][0] == oracle.NO_VIEWS and res["cost"][0] == 1.0
    assert res["status"][1] == oracle.BAD_INPUT and np.isnan(res["cost"][1]) and res["idx"][1] == -1
    assert res["status"][2] == oracle.OK


def test_half_confidence_decoding(tiny):
    """fp16 confidence maps give exactly the costs of their float32 widening (numpy's decoder)."""
    sc16 = scenegen.make_scene("tiny", conf_f16=True)
    a = oracle.Scene.from_dict(sc16)
    b = oracle.Scene(sc16["points"], sc16["cams"], sc16["angle"], sc16["conf"].astype(np.float32), sc16["nbr"])
    d = rand_unit(200 * 2).reshape(200, 2, 3)
    idx = np.arange(200)
    assert np.array_equal(oracle.eval_costs(a, d, idx=idx), oracle.eval_costs(b, d, idx=idx))
    special = np.array([0.0, 6e-8, 6.1e-5, 0.3, 1.0, 65504.0], np.float16)
    sc16["conf"][0, 0, :6] = special
    c = oracle.Scene.from_dict(sc16)
    assert c.conf[0, 0, :6].astype(np.float64).tolist() == special.astype(np.float64).tolist()


def test_fibonacci_hemisphere_closed_form():
    for H in (32, 64, 257):
        h = oracle.fibonacci_hemisphere(H)
        assert np.allclose(np.linalg.norm(h, axis=1), 1.0, atol=1e-15)
        assert np.allclose(np.diff(h[:, 2]), -1.0 / H, atol=1e-14)
        assert h[0, 2] == pytest.approx(1 - 0.5 / H) and np.all(h[:, 2] > 0)
        az = np.unwrap(np.arctan2(h[:, 1], h[:, 0]))
        golden = np.pi * (3 - np.sqrt(5))   # 137.5077... degrees
        assert np.allclose(np.mod(np.diff(az), 2 * np.pi), golden, atol=1e-9)
