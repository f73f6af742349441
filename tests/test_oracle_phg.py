"""Pins of the CPU oracle of the Parallel Hair Growing consumer (Sec. 3.2; no GPU): voxel indexing
against numpy, the voxel orientation against an FP64 eigendecomposition and closed forms, strands
traced through planted fields (straight runs, sign alignment, sharp turns, the root walk, deferred
occupancy between batches), segments seeded from the voxels no strand reached, and the linking of
Eq. segment_connection against planted gaps and a graph library's connected components."""
import networkx as nx
import numpy as np

import oracle

RNG = np.random.default_rng(11)


def cfg(origin=(0.0, 0.0, 0.0), voxel=0.1, dims=(20, 20, 20), step=0.05, max_steps=40, root_steps=4,
        cos_turn=0.5, occ_cap=1000, batch=1024, link_dist=0.15, link_cos=0.9):
    return oracle.phg_cfg(origin, voxel, dims, step, max_steps, root_steps, cos_turn, occ_cap, batch, link_dist,
                          link_cos)


def line_points(a, b, n):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    t = np.linspace(0.0, 1.0, n)[:, None]
    d = (b - a) / np.linalg.norm(b - a)
    return (a + t * (b - a)).astype(np.float32), np.repeat(d[None], n, 0).astype(np.float32)


def test_voxel_index_against_numpy():
    c = cfg(origin=(-1.0, -0.5, 0.25), voxel=0.07, dims=(30, 17, 23))
    p = (RNG.uniform(-1.2, 1.4, size=(4000, 3))).astype(np.float32)
    p[:50] = np.float32(-1.0) + np.float32(0.07) * np.arange(50, dtype=np.float32)[:, None]   # on voxel faces
    o = np.array([-1.0, -0.5, 0.25], np.float32)
    q = ((p - o) / np.float32(0.07)).astype(np.float32)
    n = np.array([30, 17, 23])
    inside = np.all((q >= 0) & (q < n), axis=1)
    ci = np.floor(q).astype(np.int64)
    want = np.where(inside, (ci[:, 2] * 17 + ci[:, 1]) * 30 + ci[:, 0], -1)
    got = np.array([oracle.phg_voxel(c, x) for x in p])
    assert np.array_equal(got, want)


def test_orientation_closed_forms_and_eigh():
    d = np.array([0.3, -0.5, 0.8], np.float32)
    d /= np.linalg.norm(d)
    # copies and sign flips: the direction itself, canonical sign (z > 0)
    c = cfg(voxel=1.0, dims=(1, 1, 1))
    occ, T = oracle.phg_splat(c, np.full((5, 3), 0.5, np.float32), np.stack([d, -d, d, d, -d]))
    o = oracle.phg_orient_one(T[0], occ[0])
    assert occ[0] == 5 and np.allclose(o, d, atol=1e-6)
    # two orthogonal directions weighted 3:1 - the heavier one
    a, b = np.array([1, 0, 0], np.float32), np.array([0, 1, 0], np.float32)
    occ, T = oracle.phg_splat(c, np.full((4, 3), 0.5, np.float32), np.stack([b, -b, a, b]))
    assert np.allclose(oracle.phg_orient_one(T[0], occ[0]), b, atol=1e-6)
    # random bundles around an axis: the dominant eigenvector of sum d d^T (FP64 eigh) to 1e-4
    for _ in range(40):
        axis = RNG.normal(size=3)
        axis /= np.linalg.norm(axis)
        dirs = axis + RNG.normal(size=(12, 3)) * 0.3
        dirs = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * RNG.choice([-1, 1], size=(12, 1)))
        dirs = dirs.astype(np.float32)
        occ, T = oracle.phg_splat(c, np.full((12, 3), 0.5, np.float32), dirs)
        w, v = np.linalg.eigh(dirs.astype(np.float64).T @ dirs.astype(np.float64))
        e = v[:, -1] * np.sign(v[2, -1])
        assert abs(abs(np.dot(oracle.phg_orient_one(T[0], occ[0]), e)) - 1.0) < 1e-8 + 1e-4
    # an empty voxel has no orientation
    assert np.all(oracle.phg_orient_one(np.zeros(6, np.int64), 0) == 0)


def test_splat_counts_every_valid_point_inside():
    c = cfg()
    p = RNG.uniform(-0.5, 2.5, size=(3000, 3)).astype(np.float32)
    d = RNG.normal(size=(3000, 3)).astype(np.float32)
    d[7] = np.nan
    valid = np.ones(3000, np.uint8)
    valid[::10] = 0
    occ, T = oracle.phg_splat(c, p, d, valid)
    inside = np.all((p >= 0) & (p < 2.0), axis=1) & (valid == 1) & np.all(np.isfinite(d), axis=1)
    assert occ.sum() == inside.sum()
    h, _ = np.histogramdd(p[inside], bins=(20, 20, 20), range=[(0, 2)] * 3)
    assert np.array_equal(occ.reshape(20, 20, 20).transpose(2, 1, 0), h.astype(np.int32))


def run(c, pts, dirs, seeds, normals, **kw):
    return oracle.phg(c, pts, dirs, np.asarray(seeds, np.float32), np.asarray(normals, np.float32), **kw)


def test_straight_run_sign_and_length():
    c = cfg(max_steps=100)
    pts, dirs = line_points([0.15, 1.05, 1.05], [1.75, 1.05, 1.05], 200)
    r = run(c, pts, dirs, [[0.12, 1.05, 1.05]], [[1.0, 0.0, 0.0]])
    # the strand walks +x along the line until it leaves the occupied voxels (x >= 1.8)
    n = r["glen"][0]
    v = r["gverts"][0, :n]
    assert r["gstop"][0] == oracle.PHG_EMPTY
    assert np.allclose(v[:, 1:], [1.05, 1.05]) and np.all(np.diff(v[:, 0]) > 0)
    assert np.allclose(np.diff(v[:, 0]), 0.05, atol=1e-6)
    assert 1.8 <= v[-1, 0] < 1.85 + 1e-6
    # a normal pointing the other way is turned by the field's sign-free orientation... and walks -x
    r2 = run(c, pts, dirs, [[1.0, 1.05, 1.05]], [[-1.0, 0.0, 0.0]])
    v2 = r2["gverts"][0, :r2["glen"][0]]
    assert np.all(np.diff(v2[:, 0]) < 0) and v2[-1, 0] < 0.1 + 1e-6
    assert np.allclose(r2["gtan"][0], [-1, 0, 0])


def test_turn_root_walk_and_maxlen():
    c = cfg(max_steps=100, cos_turn=0.5)
    a, da = line_points([0.15, 0.55, 1.05], [1.05, 0.55, 1.05], 90)
    b, db = line_points([1.15, 0.65, 1.05], [1.15, 1.75, 1.05], 110)   # perpendicular continuation
    pts, dirs = np.concatenate([a, b]), np.concatenate([da, db])
    r = run(c, pts, dirs, [[0.12, 0.55, 1.05]], [[1, 0, 0]])
    assert r["gstop"][0] in (oracle.PHG_TURN, oracle.PHG_EMPTY)
    assert r["gverts"][0, r["glen"][0] - 1, 0] < 1.25
    # the root walk: from x = -0.3 the line's first voxel [0.1, 0.2) is 8 steps of 0.05 away; 10 allowed
    # steps reach it (the walk is part of the strand), 5 do not
    wide = dict(max_steps=100, origin=(-1.0, 0.0, 0.0), dims=(30, 20, 20))
    r = run(cfg(root_steps=10, **wide), a, da, [[-0.3, 0.55, 1.05]], [[1, 0, 0]])
    v = r["gverts"][0, :r["glen"][0]]
    assert r["glen"][0] > 20 and v[0, 0] == np.float32(-0.3) and v[-1, 0] > 1.0
    r = run(cfg(root_steps=5, **wide), a, da, [[-0.3, 0.55, 1.05]], [[1, 0, 0]])
    assert r["glen"][0] == 0 and r["gstop"][0] == oracle.PHG_NO_ROOT
    # max_steps caps the strand
    r = run(cfg(max_steps=7), a, da, [[0.12, 0.55, 1.05]], [[1, 0, 0]])
    assert r["glen"][0] == 8 and r["gstop"][0] == oracle.PHG_MAXLEN


def test_deferred_occupancy_between_batches():
    pts, dirs = line_points([0.15, 1.05, 1.05], [1.75, 1.05, 1.05], 200)
    seeds = [[0.12, 1.05, 1.05]] * 3
    normals = [[1, 0, 0]] * 3
    # one batch: every strand traces against the empty occupancy and all three grow
    r = run(cfg(occ_cap=1, batch=8), pts, dirs, seeds, normals)
    assert np.all(r["glen"] == r["glen"][0]) and r["glen"][0] > 20
    # batches of one: the second and third stop at their first occupied voxel
    r = run(cfg(occ_cap=1, batch=1), pts, dirs, seeds, normals)
    assert r["glen"][0] > 20 and np.all(r["gstop"][1:] == oracle.PHG_CROWDED)
    # a cap of two lets the second through
    r = run(cfg(occ_cap=2, batch=1), pts, dirs, seeds, normals)
    assert r["glen"][1] == r["glen"][0] and r["gstop"][2] == oracle.PHG_CROWDED
    # every voxel on the line counts the strands that entered it
    line_vox = np.unique([oracle.phg_voxel(cfg(), x) for x in pts])
    r = run(cfg(occ_cap=1000, batch=1), pts, dirs, seeds, normals)
    assert np.all(r["crowd"][line_vox] == 3)


def test_segments_cover_the_unreached_voxels():
    # no seeds at all: the lowest occupied voxel seeds a segment that runs both ways along the line
    pts, dirs = line_points([0.15, 1.05, 1.05], [1.75, 1.05, 1.05], 200)
    r = run(cfg(batch=1, max_steps=100), pts, dirs, np.zeros((0, 3)), np.zeros((0, 3)))
    assert len(r["slen"]) == 17 and r["slen"][0] > 30 and np.all(r["slen"][1:] == 0)
    v = r["sverts"][0, :r["slen"][0]]
    assert np.all(np.diff(v[:, 0]) > 0)           # start at -x, end at +x (the field's canonical +x)
    assert np.allclose(r["stan"][0, 0], [-1, 0, 0]) and np.allclose(r["stan"][0, 1], [1, 0, 0])
    # in one batch every seed grows (deferred occupancy)
    r = run(cfg(batch=1000, max_steps=100), pts, dirs, np.zeros((0, 3)), np.zeros((0, 3)))
    assert np.all(r["slen"] > 0)


def test_linking_planted_gap_and_angle():
    a, da = line_points([0.15, 1.05, 1.05], [0.95, 1.05, 1.05], 80)
    b, db = line_points([1.25, 1.05, 1.05], [1.85, 1.05, 1.05], 60)     # collinear, two empty voxels later
    pts, dirs = np.concatenate([a, b]), np.concatenate([da, db])
    seeds, normals = [[0.12, 1.05, 1.05]], [[1, 0, 0]]
    r = run(cfg(link_dist=0.35, max_steps=100), pts, dirs, seeds, normals)
    assert r["glen"][0] > 0 and r["gstop"][0] == oracle.PHG_EMPTY
    seg = np.nonzero(r["slen"] > 0)[0]
    assert len(seg) >= 1
    first_b = [k for k in seg if r["sverts"][k, 0, 0] > 1.1]
    assert first_b and r["label"][1 + first_b[0]] == 0      # the guide strand's tip joined segment b
    # a gap beyond delta_d (the tip stops in the first empty voxel, x in [1.0, 1.05); b's segment
    # starts in its last empty one, x in [1.15, 1.2)), or a perpendicular continuation, joins nothing
    r = run(cfg(link_dist=0.09, max_steps=100), pts, dirs, seeds, normals)
    assert np.all(r["label"][1:] != 0)
    c, dc = line_points([1.05, 1.35, 1.05], [1.05, 1.95, 1.05], 60)
    r = run(cfg(link_dist=0.6, max_steps=100), np.concatenate([a, c]), np.concatenate([da, dc]), seeds, normals)
    assert np.all(r["label"][1:] != 0)


def brute_labels(r, link_dist, link_cos):
    """The components of the nearest-compatible-end graph, recomputed here from the traced strands with
    numpy and networkx."""
    S, K = len(r["glen"]), len(r["slen"])
    ends = []
    for g in range(S):
        if r["glen"][g] > 0:
            ends.append((g, r["gverts"][g, r["glen"][g] - 1], r["gtan"][g], -1))
    cand = []
    for k in range(K):
        if r["slen"][k] > 0:
            for side in (0, 1):
                pos = r["sverts"][k, 0 if side == 0 else r["slen"][k] - 1]
                item = (S + k, pos, r["stan"][k, side], 2 * k + side)
                ends.append(item)
                cand.append(item)
    G = nx.Graph()
    G.add_nodes_from(range(S + K))
    L2 = np.float32(link_dist) * np.float32(link_dist)
    for se, pe, te, _ in ends:
        best = None
        for sq, pq, tq, q in cand:
            if sq == se:
                continue
            dd = (pe - pq).astype(np.float32)
            d2 = np.float32(dd[0] * dd[0] + np.float32(dd[1] * dd[1] + np.float32(dd[2] * dd[2])))
            dt = float(np.dot(te.astype(np.float64), tq.astype(np.float64)))
            if d2 < L2 and -dt > link_cos and (best is None or d2 < best[0]):
                best = (d2, sq)
        if best is not None:
            G.add_edge(se, best[1])
    lab = np.arange(S + K)
    for comp in nx.connected_components(G):
        m = min(comp)
        for x in comp:
            lab[x] = m
    return lab


def test_labels_match_graph_components_on_a_scene():
    import scenegen
    sc = scenegen.make_scene("tiny", strand_maps=False, knn=False)
    noise = RNG.normal(size=sc["tangents"].shape).astype(np.float32) * 0.1
    d = sc["tangents"] + noise
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    roots = sc["verts"][:, 0]
    c = cfg(origin=(-1.2, -0.5, -1.2), voxel=0.05, dims=(48, 40, 48), step=0.025, max_steps=24, root_steps=3,
            cos_turn=0.3, occ_cap=3, batch=16, link_dist=0.08, link_cos=0.8)
    r = run(c, sc["points"], d, roots, roots / np.linalg.norm(roots, axis=1, keepdims=True))
    assert np.mean(r["glen"] > 1) > 0.5 and len(r["slen"]) > 0
    assert np.array_equal(r["label"], brute_labels(r, 0.08, 0.8))
    assert len(np.unique(r["label"])) < len(r["label"])     # some strands were joined
