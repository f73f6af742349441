"""Training and calibration of the learned proposal network (orchestration of library calls).

The network is trained on directions the plain fusion itself produces: for each training scene the
plain GPU fusion gives the targets and the library computes the features; a seeded subset of the
points forms the training set.  The fallback threshold tau is calibrated on held-out scenes so that
the points it accepts (proposal cost at most tau, then refined) stay close to the plain result.
"""
import numpy as np

from . import HairFuse, ProposalNet


def scene_tensors(sc, dev):
    import torch
    return {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr")}


def plain_and_features(sc, H, T, dev):
    """(plain directions (N, 3), plain costs (N,), features (N, 64) bf16 bits as int16) of a scene."""
    import torch
    t = scene_tensors(sc, dev)
    N = sc["N"]
    with HairFuse(H, sc["k"], T) as f:
        f.upload_views(t["cams"], t["angle"], t["conf"])
        f.upload_points(t["points"], t["nbr"])
        d = torch.empty((N, 3), device=dev)
        c = torch.empty(N, device=dev)
        f.fuse(d, c)
        x = f.features(torch.empty((N, 64), dtype=torch.int16, device=dev))
        f.sync()
    return d, c, x


def training_set(scene_fn, seeds, samples_per_scene, H, T, dev, seed=0):
    """Concatenated (features, targets) of `samples_per_scene` seeded points from each scene."""
    import torch
    xs, ts = [], []
    rng = np.random.default_rng(seed)
    for s in seeds:
        sc = scene_fn(s)
        d, _, x = plain_and_features(sc, H, T, dev)
        sel = torch.from_numpy(rng.choice(sc["N"], size=min(samples_per_scene, sc["N"]), replace=False)).to(dev)
        xs.append(x[sel])
        ts.append(d[sel])
        del sc
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def train(X, Tg, steps=20000, batch=8192, lr=1e-3, seed=0, init_seed=1, net=None):
    """Train (or continue training) a ProposalNet; returns (net, per-step losses)."""
    if net is None:
        net = ProposalNet(batch)
        net.init(init_seed)
    losses = net.train(X, Tg, batch, steps, lr, seed, use_graph=True)
    return net, losses


def angle_deg(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1))))


def learned_no_fallback(sc, net, H, T, T_short, alpha_short, dev):
    """Directions and costs of the learned path with fallback disabled (tau = +inf)."""
    import torch
    t = scene_tensors(sc, dev)
    N = sc["N"]
    with HairFuse(H, sc["k"], T) as f:
        f.upload_views(t["cams"], t["angle"], t["conf"])
        f.upload_points(t["points"], t["nbr"])
        d = torch.empty((N, 3), device=dev)
        c = torch.empty(N, device=dev)
        f.fuse_learned(net, d, c, T_short=T_short, alpha_short=alpha_short, tau=float("inf"))
        f.sync()
    return d, c


def proposal_costs(sc, net, H, T, dev):
    """(proposals (N, 3), their costs (N,)) of a scene: the quantity the fallback threshold applies to."""
    import torch
    t = scene_tensors(sc, dev)
    N = sc["N"]
    with HairFuse(H, sc["k"], T) as f:
        f.upload_views(t["cams"], t["angle"], t["conf"])
        f.upload_points(t["points"], t["nbr"])
        x = f.features(torch.empty((N, 64), dtype=torch.int16, device=dev))
        prop = net.forward(x)
        c0 = torch.empty((N, 1), device=dev)
        f.eval_costs(prop.view(N, 1, 3).contiguous(), c0)
        f.sync()
    return prop, c0[:, 0]


def calibrate_tau_batch(scenes, net, H, T, T_short, alpha_short, dev, median_deg=1.8, p95_deg=7.5):
    """Largest tau on the proposal cost for which, pooled over the points of all `scenes`, the
    accepted points refined from their proposals (fallback points counted as exact) keep the angular
    error against the plain fusion within median_deg and p95_deg.  Returns (tau, info) with the
    fallback fraction at that tau."""
    errs, costs = [], []
    for sc in scenes:
        plain, _, _ = plain_and_features(sc, H, T, dev)
        d, _ = learned_no_fallback(sc, net, H, T, T_short, alpha_short, dev)
        _, c0 = proposal_costs(sc, net, H, T, dev)
        errs.append(angle_deg(d.cpu().numpy(), plain.cpu().numpy()))
        costs.append(c0.cpu().numpy())
    err, cost = np.concatenate(errs), np.concatenate(costs)
    best = float(np.min(cost)) - 1e-6
    for q in np.linspace(1.0, 0.0, 801):
        tau = float(np.quantile(cost, q))
        e = np.where(cost <= tau, err, 0.0)
        if np.median(e) <= median_deg and np.percentile(e, 95) <= p95_deg:
            best = tau
            break
    return best, dict(err=err, cost=cost, fallback_frac=float(np.mean(cost > best)))


def calibrate_tau(sc, net, H, T, T_short, alpha_short, dev, median_deg=1.0, p95_deg=5.0):
    """Largest tau on the proposal cost (fewest fallbacks) for which the accepted points, refined
    from their proposals, with fallback points counted as exact, keep the angular error against the
    plain fusion within median_deg and p95_deg."""
    plain, plain_cost, _ = plain_and_features(sc, H, T, dev)
    d, _ = learned_no_fallback(sc, net, H, T, T_short, alpha_short, dev)
    _, c0 = proposal_costs(sc, net, H, T, dev)
    err = angle_deg(d.cpu().numpy(), plain.cpu().numpy())
    cost = c0.cpu().numpy()
    best = float(np.min(cost)) - 1e-6
    for q in np.linspace(1.0, 0.0, 401):
        tau = float(np.quantile(cost, q))
        e = np.where(cost <= tau, err, 0.0)
        if np.median(e) <= median_deg and np.percentile(e, 95) <= p95_deg:
            best = tau
            break
    return best, dict(err=err, cost=cost, plain_cost=plain_cost.cpu().numpy())
