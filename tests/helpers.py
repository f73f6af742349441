"""Shared helpers of the GPU parity tests: run the library on a scene, compare with the oracle.

Tolerances (from the fusion step's accuracy targets):
  cost          |c_gpu - c_oracle| <= 1e-4 |c_oracle| + 1e-6
  index         identical, except where the oracle's two best hypothesis costs are within 1e-5
                relative (+1e-6): then the GPU's pick must cost no more than that tie margin
  direction     within 0.1 deg; where the oracle's refinement meets a near-tie (two best of the
                seven costs of a round within 2e-6, the order FP32 cannot fix) at round t*, the
                two trajectories agree before t* and each moves by < 2 alpha_t* afterwards, so the
                bound is max(0.1 deg, 4 alpha_t*)
  boundary      points whose samples lie within 1e-6 px of a pixel edge are counted, not compared
"""
import numpy as np

import oracle

COST_RTOL, COST_ATOL = 1e-4, 1e-6


def angle_deg(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    dt = np.abs(np.sum(a * b, axis=-1))
    return np.degrees(np.arctan2(cr, dt))


def run_library(scene, H, T, top_k=0, hyps=None, device=True, conf=None, points=None, nbr=None):
    """Fuse a scene with the CUDA library; returns numpy dir/cost/idx/status."""
    import torch

    import paper_2604_05794_b300 as hf
    conf = scene["conf"] if conf is None else conf
    points = scene["points"] if points is None else points
    nbr = scene["nbr"] if nbr is None else nbr
    N, k = points.shape[0], nbr.shape[1]
    with hf.HairFuse(H, k, T, top_k) as f:
        if device:
            dev = torch.device("cuda")
            f.upload_views(torch.from_numpy(scene["cams"]).to(dev), torch.from_numpy(scene["angle"]).to(dev),
                           torch.from_numpy(conf).to(dev))
            f.upload_points(torch.from_numpy(points).to(dev), torch.from_numpy(nbr).to(dev))
            out = dict(dir=torch.empty((N, 3), device=dev), cost=torch.empty(N, device=dev),
                       idx=torch.empty(N, dtype=torch.int32, device=dev),
                       status=torch.empty(N, dtype=torch.uint8, device=dev))
            hy = None if hyps is None else torch.from_numpy(np.ascontiguousarray(hyps, np.float32)).to(dev)
            f.fuse(out["dir"], out["cost"], out["idx"], out["status"], hyps=hy)
            f.sync()
            return {k_: v.cpu().numpy() for k_, v in out.items()}
        f.upload_views(scene["cams"], scene["angle"], conf)
        f.upload_points(points, nbr)
        out = dict(dir=np.empty((N, 3), np.float32), cost=np.empty(N, np.float32), idx=np.empty(N, np.int32),
                   status=np.empty(N, np.uint8))
        f.fuse(out["dir"], out["cost"], out["idx"], out["status"],
               hyps=None if hyps is None else np.ascontiguousarray(hyps, np.float32))
        return out


def library_eval_costs(scene, dirs, conf=None):
    import torch

    import paper_2604_05794_b300 as hf
    conf = scene["conf"] if conf is None else conf
    dev = torch.device("cuda")
    N = scene["points"].shape[0]
    with hf.HairFuse(8, scene["nbr"].shape[1], 0, 0) as f:
        f.upload_views(torch.from_numpy(scene["cams"]).to(dev), torch.from_numpy(scene["angle"]).to(dev),
                       torch.from_numpy(conf).to(dev))
        f.upload_points(torch.from_numpy(scene["points"]).to(dev), torch.from_numpy(scene["nbr"]).to(dev))
        d = torch.from_numpy(np.ascontiguousarray(dirs, np.float32)).to(dev)
        c = torch.empty((N, dirs.shape[1]), device=dev)
        f.eval_costs(d, c)
        f.sync()
        return c.cpu().numpy()


def compare(gpu, orc, sel, osc, hyps, H, top_k=0, strict_frac=0.95):
    """Check GPU outputs (restricted to the point indices sel) against oracle results on sel.

    Returns a dict of statistics; raises AssertionError on any violation."""
    g = {k_: v[sel] for k_, v in gpu.items()}
    n = len(sel)
    assert np.array_equal(g["status"], orc["status"]), "status differs"
    ok = orc["status"] == oracle.OK
    bad = orc["status"] == oracle.BAD_INPUT
    assert np.all(g["idx"][bad] == -1) and np.all(np.isnan(g["cost"][bad])) and np.all(g["dir"][bad] == 0)
    boundary = (orc["flags"] & oracle.FLAG_BOUNDARY) > 0
    idx_tie = (orc["flags"] & oracle.FLAG_IDX_TIE) > 0
    cmp = ~boundary & ~bad
    # hypothesis index
    same_idx = g["idx"] == orc["idx"]
    assert np.all(same_idx[cmp & ~idx_tie]), f"index differs at {np.nonzero(~same_idx & cmp & ~idx_tie)[0][:10]}"
    if np.any(cmp & idx_tie & ~same_idx):
        q = np.nonzero(cmp & idx_tie & ~same_idx)[0]
        hc = oracle.eval_costs(osc, np.broadcast_to(hyps, (len(q), H, 3)), idx=sel[q], top_k=top_k)
        picked = hc[np.arange(len(q)), g["idx"][q]]
        best = hc.min(axis=1)
        assert np.all(picked <= best + 1e-5 * np.abs(best) + 1e-6)
    # cost of the returned direction, evaluated by the oracle at the GPU's direction
    c_at_gpu = oracle.eval_costs(osc, g["dir"][:, None, :].astype(np.float64), idx=sel, top_k=top_k)[:, 0]
    err_self = np.abs(g["cost"] - c_at_gpu)
    assert np.all((err_self <= COST_RTOL * np.abs(c_at_gpu) + COST_ATOL)[cmp]), \
        f"cost at own direction: max err {np.max(err_self[cmp])}"
    # cost against the oracle's own refined cost where the trajectories are determined
    no_tie = cmp & ~idx_tie & (orc["tie_step"] < 0)
    err = np.abs(g["cost"] - orc["cost"])
    assert np.all((err <= COST_RTOL * np.abs(orc["cost"]) + COST_ATOL)[no_tie]), \
        f"cost vs oracle: max err {np.max(err[no_tie])}"
    # direction
    ang = angle_deg(g["dir"], orc["dir"])
    al0 = np.degrees(0.5 * np.sqrt(2 * np.pi / H))
    bound = np.where(orc["tie_step"] < 0, 0.1, np.maximum(0.1, 4 * al0 / 2.0 ** np.maximum(orc["tie_step"], 0)))
    chk = cmp & ~idx_tie & ok
    viol = chk & (ang > bound + 1e-3)
    assert not np.any(viol), f"direction beyond bound at {np.nonzero(viol)[0][:10]}: {ang[viol][:10]}"
    within = np.mean(ang[chk] <= 0.1) if np.any(chk) else 1.0
    assert within >= strict_frac, f"only {within:.4f} of points within 0.1 deg"
    return dict(n=n, boundary=int(boundary.sum()), idx_tie=int(idx_tie.sum()),
                refine_tie=int((orc["tie_step"] >= 0).sum()), within_0p1=float(within),
                median_deg=float(np.median(ang[chk])) if np.any(chk) else 0.0,
                p95_deg=float(np.percentile(ang[chk], 95)) if np.any(chk) else 0.0,
                max_cost_err=float(np.max(err_self[cmp])) if np.any(cmp) else 0.0)
