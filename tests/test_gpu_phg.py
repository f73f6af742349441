"""GPU parity of the Parallel Hair Growing consumer (hair_fuse_phg) against the CPU oracle on the
same seeded inputs: the single-precision steps replay the same operations, so every output is
compared bit for bit (volumes, guide strands, segments, component labels)."""
import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(5)


def scene_inputs(preset, n_strands=None, noise=0.1, seed=3):
    over = {} if n_strands is None else dict(n_strands=n_strands)
    sc = scenegen.make_scene(preset, seed=seed, strand_maps=False, knn=False, **over)
    rng = np.random.default_rng(seed)
    d = sc["tangents"] + rng.normal(size=sc["tangents"].shape).astype(np.float32) * np.float32(noise)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    roots = np.ascontiguousarray(sc["verts"][:, 0], np.float32)
    normals = (roots / np.linalg.norm(roots, axis=1, keepdims=True)).astype(np.float32)
    return np.ascontiguousarray(sc["points"], np.float32), d, roots, normals


def grid_for(pts, voxel):
    fin = pts[np.all(np.isfinite(pts), axis=1)]
    lo = fin.min(0) - 2 * voxel
    hi = fin.max(0) + 2 * voxel
    dims = np.ceil((hi - lo) / voxel).astype(int)
    return lo.astype(np.float32), dims


def both(pts, dirs, seeds, normals, voxel, step, max_steps, root_steps, cos_turn, occ_cap, batch, link_dist, link_cos,
         valid=None, device=True):
    import torch

    import paper_2604_05794_b300 as hf
    o, dims = grid_for(pts, voxel)
    oc = oracle.phg_cfg(o, voxel, dims, step, max_steps, root_steps, cos_turn, occ_cap, batch, link_dist, link_cos)
    gc = hf.hf_phg_cfg((ctypes_floats(o)), voxel, *[int(x) for x in dims], step, max_steps, root_steps, cos_turn,
                       occ_cap, batch, link_dist, link_cos)
    want = oracle.phg(oc, pts, dirs, seeds, normals, valid=valid)
    with hf.HairFuse(8, 0, 0) as f:
        if device:
            t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
            got = f.phg(gc, t(pts), t(dirs), t(seeds), t(normals), valid=t(valid))
            got = {k: v.cpu().numpy() for k, v in got.items()}
        else:
            got = f.phg(gc, pts, dirs, seeds, normals, valid=valid)
    return want, got


def ctypes_floats(o):
    import ctypes
    return (ctypes.c_float * 3)(*[float(x) for x in o])


def assert_same(want, got):
    for k in ("occ", "ori", "crowd", "glen", "gstop", "slen", "svox", "label"):
        assert np.array_equal(want[k].view(np.uint8), got[k].view(np.uint8)), k
    assert int(got["n_seg"][0]) == len(want["slen"])
    for i, n in enumerate(want["glen"]):
        assert np.array_equal(want["gverts"][i, :n].view(np.uint32), got["gverts"][i, :n].view(np.uint32)), i
        if n:
            assert np.array_equal(want["gtan"][i].view(np.uint32), got["gtan"][i].view(np.uint32)), i
    for k, n in enumerate(want["slen"]):
        assert np.array_equal(want["sverts"][k, :n].view(np.uint32), got["sverts"][k, :n].view(np.uint32)), k
        if n:
            assert np.array_equal(want["stan"][k].view(np.uint32), got["stan"][k].view(np.uint32)), k


def test_tiny_scene_bit_exact():
    pts, d, roots, normals = scene_inputs("tiny")
    want, got = both(pts, d, roots, normals, voxel=0.05, step=0.025, max_steps=24, root_steps=3, cos_turn=0.3,
                     occ_cap=3, batch=16, link_dist=0.08, link_cos=0.8)
    assert np.mean(want["glen"] > 1) > 0.5 and len(want["slen"]) > 100
    assert len(np.unique(want["label"])) < len(want["label"])
    assert_same(want, got)


def test_mid_subset_options_and_ragged_batches():
    pts, d, roots, normals = scene_inputs("mid", n_strands=600, seed=4)
    valid = (RNG.random(len(pts)) > 0.05).astype(np.uint8)
    for kw in (dict(voxel=0.02, step=0.01, max_steps=64, root_steps=4, cos_turn=0.5, occ_cap=2, batch=37,
                    link_dist=0.03, link_cos=0.7),
               dict(voxel=0.03, step=0.03, max_steps=20, root_steps=0, cos_turn=-1.0, occ_cap=1, batch=1,
                    link_dist=0.09, link_cos=0.0),
               dict(voxel=0.015, step=0.005, max_steps=128, root_steps=10, cos_turn=0.9, occ_cap=1000,
                    batch=100000, link_dist=0.0, link_cos=0.5)):
        want, got = both(pts, d, roots, normals, valid=valid, **kw)
        assert_same(want, got)


def test_host_and_device_agree_and_degenerate_inputs():
    pts, d, roots, normals = scene_inputs("tiny")
    pts = pts.copy()
    d = d.copy()
    pts[3] = np.nan
    d[5] = np.inf
    roots = np.concatenate([roots, [[50.0, 50.0, 50.0]]]).astype(np.float32)   # a seed outside the grid
    normals = np.concatenate([normals, [[0.0, 0.0, 1.0]]]).astype(np.float32)
    kw = dict(voxel=0.05, step=0.025, max_steps=24, root_steps=3, cos_turn=0.3, occ_cap=3, batch=16, link_dist=0.08,
              link_cos=0.8)
    want, got_d = both(pts, d, roots, normals, device=True, **kw)
    _, got_h = both(pts, d, roots, normals, device=False, **kw)
    assert_same(want, got_d)
    assert_same(want, got_h)
    assert got_h["glen"][-1] == 0 and got_h["gstop"][-1] == oracle.PHG_NO_ROOT


def test_phg_arguments():
    import paper_2604_05794_b300 as hf
    pts, d, roots, normals = scene_inputs("tiny")
    o, dims = grid_for(pts, 0.05)
    base = dict(voxel=0.05, step=0.025, max_steps=24, root_steps=3, cos_turn=0.3, occ_cap=3, batch=16, link_dist=0.08,
                link_cos=0.8)
    with hf.HairFuse(8, 0, 0) as f:
        for bad in (dict(step=0.06), dict(step=0.0), dict(max_steps=0), dict(occ_cap=0), dict(batch=0),
                    dict(link_dist=0.5), dict(cos_turn=1.5), dict(voxel=0.0)):
            kw = dict(base, **bad)
            gc = hf.hf_phg_cfg(ctypes_floats(o), kw["voxel"], *[int(x) for x in dims], kw["step"], kw["max_steps"],
                               kw["root_steps"], kw["cos_turn"], kw["occ_cap"], kw["batch"], kw["link_dist"],
                               kw["link_cos"])
            with pytest.raises(hf.HairFuseError):
                f.phg(gc, pts, d, roots, normals)
        gc = hf.hf_phg_cfg(ctypes_floats(o), 0.05, *[int(x) for x in dims], 0.025, 24, 3, 0.3, 3, 16, 0.08, 0.8)
        with pytest.raises(hf.HairFuseError):
            f.phg(gc, pts, d, roots, normals, seg_cap=3)   # more segment seeds than room
