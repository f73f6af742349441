"""The partition hook (hair_fuse_fuse_range): fusing a scene range by range, as ranks of a
multi-GPU split would, gives exactly the rows of fusing it whole."""
import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    return scenegen.make_scene("mid", seed=21, n_strands=300, width=512, height=512, f=600.0)


def _outs(n, dev=True):
    import torch
    if dev:
        return (torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
                torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"))
    return (np.empty((n, 3), np.float32), np.empty(n, np.float32), np.empty(n, np.int32), np.empty(n, np.uint8))


def _host(o):
    return [x.cpu().numpy() if hasattr(x, "cpu") else x for x in o]


def test_ranges_tile_the_whole_scene(scene):
    import bench
    import paper_2604_05794_b300 as hf
    N = scene["N"]
    with hf.HairFuse(64, scene["k"], 8) as f:
        f.upload_views(scene["cams"], scene["angle"], scene["conf"])
        f.upload_points(scene["points"], scene["nbr"])
        whole = _outs(N)
        f.fuse(*whole)
        want = _host(whole)
        for world in (2, 3, 7):
            got = [[], [], [], []]
            for rank in range(world):
                lo, hi = bench.rank_range(N, rank, world)
                o = _outs(hi - lo, dev=(rank % 2 == 0))   # device and host outputs alike
                f.fuse_range(lo, hi - lo, *o)
                for q, x in enumerate(_host(o)):
                    got[q].append(x)
            for q in range(4):
                g = np.concatenate(got[q])
                assert g.dtype == want[q].dtype and np.array_equal(g.view(np.uint8), want[q].view(np.uint8))


def test_range_arguments(scene):
    import paper_2604_05794_b300 as hf
    N = scene["N"]
    with hf.HairFuse(64, scene["k"], 8) as f:
        f.upload_views(scene["cams"], scene["angle"], scene["conf"])
        f.upload_points(scene["points"], scene["nbr"])
        f.fuse_range(5, 0, *_outs(1))   # empty range: nothing to do
        for first, count in ((-1, 4), (N - 2, 3), (0, N + 1)):
            with pytest.raises(hf.HairFuseError):
                f.fuse_range(first, count, *_outs(max(count, 1)))
