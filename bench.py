"""Benchmark of the multi-view hair direction fusion on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload serving16|full|mid|tiny]

Default workload (serving16): the learned + batched form against the plain form on an uneven batch
of 16 synthetic scenes (50k-1M points, 16-64 views, 512x512 to 1920x1080 maps, H = 64, k = 8,
T = 8).  One step = one fusion of every point of every scene: for the learned + batched form, one
replay of the batch's CUDA graph (per-stage persistent launches over all scenes: constants,
projection + gather (which also writes the features' view part), the features' position part,
proposal network, proposal cost with fallback selection and short refinement, argmin and
refinement of the fallback points); for the plain form, the plain fusion of the scenes one after
another.  The proposal network is trained on the GPU first (library kernels, four scenes shaped like
the full workload) and its fallback threshold calibrated on eight held-out serving-shaped scenes.

--workload full|mid|tiny: the plain fusion of one resident scene (full: 1,000,000 points, 64 views
of 1920x1080).

Rank 0 prints one JSON line.  Under torchrun each rank fuses its own scenes (independent problems,
weak scaling, no data-path collective); timing is the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (the paper publishes no code and no fusion throughput to compare with).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused points/s at median angle err ≤2° vs FP64 oracle; learned+batched vs plain"
WORKLOADS = {
    "serving16": "batched serving: 16 scenes (seeds 200-215), points log-uniform in [50k, 1M], views uniform in "
                 "{16..64}, maps from {512x512, 1024x1024, 1920x1080}, full-preset geometry (orbit, 0.5 deg pose "
                 "noise), H=64, k=8, T=8; learned proposal (trained on 4 full-like scenes, 2M samples, 20k Adam "
                 "steps, batch 8192, lr 1e-3) + 2 refinement rounds + plain fallback, against the plain fusion "
                 "of the scenes one by one",
    "learned": "learned proposal on one full-workload scene (seed 104: 1,000,000 points, 64 views 1920x1080, "
               "fp16 confidence): network trained on 4 full-like scenes (2M samples, 20k Adam steps, batch 8192, "
               "lr 1e-3), proposal cost against a calibrated tau, 2 refinement rounds for accepted proposals, "
               "the plain fusion (H=64, T=8) for the others; against the plain fusion of the same scene",
    "full": "plain fusion, full: 1,000,000 points (20,000 strands x 50 segments), 64 views 1920x1080, "
            "f32 angle + fp16 confidence, 0.5 deg pose noise, H=64, k=8, T=8",
    "mid": "plain fusion, mid: 200,000 points, 32 views 1024x1024 with 10% outlier pixels, H=64, k=8, T=8",
    "tiny": "plain fusion, tiny: 2,000 points, 8 views 256x256, H=32, k=5, T=4",
    "phg": "the paper's Parallel Hair Growing consumer on the full scene's strands (seed 2: 1,000,000 points, "
           "tangents with N(0, 0.1) noise renormalised; 20,000 scalp seeds at the strand roots): voxel 0.02, step "
           "0.01, 64 steps, 4 root steps, turn cos 0.5, 4 strands per voxel, batches of 32768 seeds, link 0.03 / "
           "cos 0.7",
    "gabor": "orientation and confidence maps of the full scene's 64 views (1920x1080 grayscale strand images, "
             "seed 2: rendered coverage blurred by 0.8 px plus N(0, 0.02) noise) with a 64-orientation even/odd "
             "Gabor bank, 15x15 window, sigma 2.5 / 1.5 px, wavelength 4 px; bf16 tensor-core correlations",
    "fpmvo": "the paper's FPMVO step on the full scene (seed 2: 1,000,000 points, 64 views 1920x1080, f32 angle + "
             "fp16 confidence, depth maps from the renderer's z-buffer): K=5 top views, S=5 depth samples over "
             "[-0.0046, 0.0046], P=5 patch, lambda=4 px, depth-test tolerance 0.02",
}
FPMVO_CFG = dict(K=5, S=5, P=5, lambda_px=4.0, delta=0.0046, eps_vis=0.02)
PHG_CFG = dict(voxel=0.02, step=0.01, max_steps=64, root_steps=4, cos_turn=0.5, occ_cap=4, batch=32768, link_dist=0.03,
               link_cos=0.7)
SM_COUNT, FP32_LANES_PER_SM = 148, 128


def s8d_ops(k):
    """FP32 operations per (direction, view) of the cost's reference count: 3 per patch member
    (multiply, multiply-add, maximum) + 12 per (hypothesis, view), + 9 more per refinement candidate
    (its rotation into the view)."""
    per_hyp = 3 * (k + 1) + 12
    return per_hyp, per_hyp + 9


def issued_per_dir_view(k):
    """Instructions the cost kernels issue per (direction, view), counted from their source: 6 for
    r = J d, 2 for |r|^2, 2 to broadcast r, 3 per member pair (packed multiply, packed multiply-add,
    three-input max of |x|), 3 for an odd last member, 4 for the threshold test, reciprocal square
    root, scale and sum."""
    kp = k + 1
    for cand in (1, 4, 6, 9, 12, 17):   # the compiled patch widths
        if kp <= cand:
            kp = cand
            break
    return 14 + 3 * (kp // 2) + 3 * (kp & 1)


_ALU_PEAK = None


def alu_peak(reps=5):
    """Measured FP32 peak for the cost kernels (hair_fuse_issue_rate, CUDA events, full-occupancy grid):
    the best rate of the patch term's inner step (packed multiply / multiply-add and the three-input
    max of absolute values), in operations/s at 3 operations per evaluation (the reference count of a
    patch member); scalar fma, packed fma and the three-input max are measured beside it.  Cached per
    run."""
    global _ALU_PEAK
    if _ALU_PEAK is None:
        import paper_2604_05794_b300 as hf
        rates = {}
        for kind in ("ffma", "ffma2", "fmax3_abs", "patch", "patch3"):
            rates[kind] = max(hf.issue_rate(kind, iters=4096)["ops_per_s"] for _ in range(reps))
        _ALU_PEAK = {"peak": rates["patch3"], "rates_ops_per_s": rates,
                     "source": "measured: hair_fuse_issue_rate HF_ISSUE_PATCH3 (2 mul.f32x2 + 2 fma.f32x2 + 2 "
                               "three-input max of |x| per 4 patch-term evaluations, 3 ops each), best of "
                               f"{reps} launches"}
    return _ALU_PEAK


# DRAM bytes (read + write) per work unit of a kernel from one ncu capture, valid only for the kernel
# sources it was taken on: the first 12 hex digits of the SHA-256 of every csrc/*.cu and *.cuh file
# (in name order).  After any source change every kernel reports traffic null until captured again.
TRAFFIC = {
    "k_project_batch": (27.82, "point-view (N V)", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_featpos_batch": (37.50, "point", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_mlp": (137.58, "point (feature row)", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_select_batch": (32.91, "point-view (N V)", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_refine_short_batch": (74.16, "accepted point-view", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_argmin_batch": (76.47, "fallback point-view", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_refine_batch": (305.76, "fallback point-view", "b73f0f2b1272", "ncu --set full, 4-scene serving batch (seeds 200-203, 1,979,650 points), scaled by units"),
    "k_project": (34.87, "point-view (N V)", "b73f0f2b1272", "ncu --set full, mid workload (200,000 points, 32 views 1024x1024), scaled by units"),
    "k_argmin": (19.50, "point-view in V_i", "b73f0f2b1272", "ncu --set full, mid workload (200,000 points, 32 views 1024x1024), scaled by units"),
    "k_refine": (20.70, "point-view in V_i", "b73f0f2b1272", "ncu --set full, mid workload (200,000 points, 32 views 1024x1024), scaled by units"),
}


def kernels_source_sha():
    import glob
    import hashlib
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2604_05794_b300", "csrc", "*.cu*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def kernel_traffic(name, units):
    """(traffic bytes of a launch, source note) from TRAFFIC, or (None, why)."""
    t = TRAFFIC.get(name)
    if t is None:
        return None, "no ncu capture of this kernel"
    bpu, unit, sha, how = t
    if sha != kernels_source_sha():
        return None, f"stale: captured on kernel source {sha}, now {kernels_source_sha()}"
    return bpu * units, f"{bpu:.2f} DRAM bytes per {unit} ({how}) x {units} units of this launch"


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0   # fallback B300 copy bandwidth when the measured file is absent


HBM_GBS = _hbm_peak()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="serving16", choices=list(WORKLOADS))
    ap.add_argument("--partition", action="store_true", help="full/mid/tiny under torchrun: every rank uploads "
                    "the same scene and fuses its own point range (strong scaling) instead of its own scene")
    ap.add_argument("--phg-strands", type=int, default=0, help="phg: strands of the scene (0: the full preset's)")
    ap.add_argument("--gabor-views", type=int, default=64, help="gabor: views of the full scene (the small case "
                    "for profiler captures: 4)")
    ap.add_argument("--fpmvo-scene", default="full", choices=["full", "mid"],
                    help="fpmvo: the scene preset (mid: the small case for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--net", default=None, help="serving16: load the proposal network from this file instead of "
                    "training it (profiling runs)")
    ap.add_argument("--save-net", default=None, help="serving16: save the trained proposal network here")
    ap.add_argument("--tau", type=float, default=None, help="serving16 with --net: fallback threshold (skips "
                    "the calibration)")
    ap.add_argument("--scenes", default="16", help="serving16: number of scenes of the batch, or a comma list of "
                    "their indices (profiling runs)")
    ap.add_argument("--only-learned", action="store_true", help="serving16: skip the plain comparison runs")
    ap.add_argument("--accuracy-sample", type=int, default=0,
                    help="oracle sample for the accuracy check (default 400 points; 50,000 across the serving batch)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(x, pg, dev, op="max"):
    """x combined over the ranks of the process group (max for times, sum for work); x itself
    without one.  dev: the device of the collective's tensor (cuda for NCCL, cpu for gloo)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX if op == "max" else pg.ReduceOp.SUM)
    return float(t.item())


def rank_range(n, rank, world):
    """Contiguous point range [lo, hi) of a rank when one scene is split over the ranks (sizes differ
    by at most one; the ranges tile [0, n) in rank order)."""
    lo = n * rank // world
    return lo, n * (rank + 1) // world


def rank_first_seed(rank):
    """First seed of the serving batch of a rank: every rank fuses its own independent scenes."""
    return 200 + 1000 * rank


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def make_workload(name, seed_offset=0):
    import scenegen
    seed = scenegen.PRESET_SEEDS[name] + seed_offset
    sc = scenegen.make_scene(name, seed=seed)
    return sc


def cpu_baseline(sc, H, T, budget_s=15.0):
    """The FP64 oracle on the host cores over a bounded sample of points (stratified, every n-th)."""
    import oracle
    osc = oracle.Scene.from_dict(sc)
    hyps = oracle.fibonacci_hemisphere(H)
    probe = np.arange(0, sc["N"], max(1, sc["N"] // 512))
    oracle.fuse(osc, hyps, T, idx=probe[:64])             # thread start-up
    t0 = time.perf_counter()
    oracle.fuse(osc, hyps, T, idx=probe)
    per_pt = (time.perf_counter() - t0) / len(probe)
    n = int(min(sc["N"], max(len(probe), budget_s / max(per_pt, 1e-9))))
    sel = np.linspace(0, sc["N"] - 1, n).astype(np.int64)
    t0 = time.perf_counter()
    oracle.fuse(osc, hyps, T, idx=sel)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} of {sc['N']} points, evenly spaced (every ~{sc['N'] // n}th), FP64 C + OpenMP, "
                      f"{dt:.1f} s"}


def accuracy(sc, H, T, gpu_dir, n_sample, lo=0, hi=None):
    """Angular error of the GPU directions against the FP64 oracle on a stratified sample of the
    points lo .. hi - 1."""
    import oracle
    osc = oracle.Scene.from_dict(sc)
    import paper_2604_05794_b300 as hf
    hyps = hf.fibonacci_hemisphere(H)
    hi = sc["N"] if hi is None else hi
    sel = np.linspace(lo, hi - 1, n_sample).astype(np.int64)
    orc = oracle.fuse(osc, hyps, T, idx=sel)
    a, b = gpu_dir[sel].astype(np.float64), orc["dir"]
    ang = np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1))))
    ok = orc["status"] == 0
    return {"median_deg": float(np.median(ang[ok])), "p95_deg": float(np.percentile(ang[ok], 95)),
            "within_0p1deg": float(np.mean(ang[ok] <= 0.1)), "sample": int(n_sample)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    if args.workload == "fpmvo":
        return run_reference_fpmvo(args, world)
    if args.workload == "phg":
        return run_reference_phg(args, world)
    if args.workload == "gabor":
        return run_reference_gabor(args, world)
    if args.workload == "serving16":
        scenes = serving_scenes(200)
    elif args.workload == "learned":
        import scenegen
        scenes = [scenegen.make_scene("full", seed=104)]
    else:
        scenes = [make_workload(args.workload)]
    osc = [oracle.Scene.from_dict(sc) for sc in scenes]
    hyps = {sc["cfg"]["H"]: oracle.fibonacci_hemisphere(sc["cfg"]["H"]) for sc in scenes}
    Ntot = sum(sc["N"] for sc in scenes)

    def fuse_sample(n_total):
        """The oracle's plain fusion of about n_total points spread over the scenes in proportion
        to their point counts (evenly spaced in each); returns the number fused."""
        n = 0
        for o, sc in zip(osc, scenes):
            m = max(1, int(n_total * sc["N"] / Ntot))
            oracle.fuse(o, hyps[sc["cfg"]["H"]], sc["cfg"]["T"], idx=np.linspace(0, sc["N"] - 1, m).astype(np.int64))
            n += m
        return n

    fuse_sample(64)                                      # thread start-up
    t0 = time.perf_counter()
    n_probe = fuse_sample(512)
    per_pt = (time.perf_counter() - t0) / n_probe
    # bounded sample per step so that warmup + steps finish within a few minutes
    budget = 90.0 / max(1, args.steps + args.warmup)
    n = int(min(Ntot, max(64, budget / max(per_pt, 1e-9))))
    for _ in range(args.warmup):
        fuse_sample(max(1, n // 8))
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += fuse_sample(n)
    dt = time.perf_counter() - t0
    value = done / dt
    sample = (f"{done // max(1, args.steps)} of {Ntot} points per step, spread over {len(scenes)} scene(s) in "
              "proportion to their point counts, evenly spaced; FP64 C + OpenMP, plain fusion")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "points_per_step": n},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_fpmvo(args, world):
    """The FP64 oracle's FPMVO on the host cores, a bounded evenly spaced sample of the scene per step."""
    import oracle
    import scenegen
    cfg = dict(FPMVO_CFG, eps_vis=float(np.float32(FPMVO_CFG["eps_vis"])))
    sc = scenegen.make_scene("full", seed=scenegen.PRESET_SEEDS["full"], depth=True)
    osc = oracle.Scene.from_dict(sc)
    N = sc["N"]
    run = lambda n: oracle.fpmvo(osc, sc["depth"], idx=np.linspace(0, N - 1, n).astype(np.int64), **cfg)
    run(64)
    t0 = time.perf_counter()
    run(1024)
    per_pt = (time.perf_counter() - t0) / 1024
    n = int(min(N, max(64, 90.0 / max(1, args.steps + args.warmup) / max(per_pt, 1e-9))))
    for _ in range(args.warmup):
        run(max(1, n // 8))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(n)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = f"{n} of {N} points per step, evenly spaced; FP64 C + OpenMP FPMVO"
    line = {"impl": "reference", "metric": "FPMVO points/s (depth-sample candidates, medoid fusion, patch "
            "consistency)", "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["fpmvo"], "points_per_step": n, **cfg},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_phg(args, world):
    """The oracle of the PHG consumer on the host, one scene of 400 strands of the same preset per step
    (single-threaded: its batches are sequential by construction)."""
    phg_cpu(400)
    t0 = time.perf_counter()
    n = 0
    for _ in range(args.warmup):
        phg_cpu(400)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        n += phg_cpu(400)[1]
    dt = time.perf_counter() - t0
    value = n / dt
    line = {"impl": "reference", "metric": "PHG input points/s (volumes, guide strands, segments, linking)",
            "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (int64 fixed-point sums)", "data": "synthetic",
            "config": {"workload": WORKLOADS["phg"], "points_per_step": n // max(1, args.steps), **PHG_CFG},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": "a 400-strand scene of the same preset and parameters per step"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2604_05794_b300 as hf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    sc = make_workload(args.workload, seed_offset=0 if args.partition else 100 * rank)
    N, V, H, W, k = sc["N"], sc["V"], sc["H"], sc["W"], sc["k"]
    Hh, T = sc["cfg"]["H"], sc["cfg"]["T"]
    stream = torch.cuda.current_stream(dev)
    f = hf.HairFuse(Hh, k, T, 0, stream=stream.cuda_stream)
    cams = torch.from_numpy(sc["cams"]).to(dev)
    ang = torch.from_numpy(sc["angle"]).to(dev)
    conf = torch.from_numpy(sc["conf"]).to(dev)
    pts = torch.from_numpy(sc["points"]).to(dev)
    nbr = torch.from_numpy(sc["nbr"]).to(dev)
    f.upload_views(cams, ang, conf)
    f.upload_points(pts, nbr)
    lo, hi = rank_range(N, rank, world) if args.partition else (0, N)
    R = hi - lo   # points this rank fuses
    out_dir = torch.empty((R, 3), device=dev)
    out_cost = torch.empty(R, device=dev)
    out_idx = torch.empty(R, dtype=torch.int32, device=dev)
    out_st = torch.empty(R, dtype=torch.uint8, device=dev)

    def step():
        if args.partition:
            f.fuse_range(lo, R, out_dir, out_cost, out_idx, out_st)
        else:
            f.fuse(out_dir, out_cost, out_idx, out_st)

    for _ in range(max(3, args.warmup)):
        step()
    f.sync()
    point_views = f.work()
    # timed region: device-resident inputs, CUDA events on the library's stream
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = f.stats()["launches"]
    f.profile(True)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kt = f.profile_read()
    f.profile(False)
    launches = f.stats()["launches"] - launches0
    ms = reduce_over_ranks(ms, pg, dev)
    f.sync()
    # whole-job points: one shared scene when partitioned, every rank's own scene otherwise
    value = (N if args.partition else reduce_over_ranks(N, pg, dev, "sum")) * args.steps / (ms / 1e3)
    if args.partition:
        point_views = point_views * R // N   # the range's share of the projection's work count

    # rooflines: the cost kernel is FP32-issue bound, the projection/gather kernel HBM bound
    ap = alu_peak()
    ca, cr = s8d_ops(k)
    conf_b = sc["conf"].itemsize
    rooflines = {}
    for name, per_pv, ndir in (("k_argmin", Hh * ca, Hh), ("k_refine", 6 * T * cr, 6 * T + 1)):
        if name not in kt:
            continue
        n_, t_ = kt[name]
        sec = t_ / n_ / 1e3
        ach = per_pv * point_views / sec
        issued = ndir * issued_per_dir_view(k) * point_views / sec
        traffic, tsrc = kernel_traffic(name, point_views)
        rooflines[name] = {
            "bound": "alu", "achieved": ach / 1e12, "peak": ap["peak"] / 1e12, "unit": "TFLOP/s",
            "frac": ach / ap["peak"], "traffic": traffic, "traffic_source": tsrc, "kernel": name,
            "peak_source": ap["source"], "peak_rates_ops_per_s": ap["rates_ops_per_s"],
            "work": (f"{Hh} x {ca} FP32 ops per (point, view) in V_i" if name == "k_argmin" else
                     f"{6 * T} x {cr} FP32 ops per (point, view) in V_i") +
                    f" (reference op count) x {point_views} point-views per launch",
            "builder_count": {"instr_per_dir_view": issued_per_dir_view(k), "directions": ndir,
                              "achieved_instr_per_s": issued,
                              "frac_of_ffma_issue": issued / ap["rates_ops_per_s"]["ffma"]},
            "units": point_views, "ms": t_ / n_, "share": t_ / ms}
    if "k_project" in kt:
        n_, t_ = kt["k_project"]
        sec = t_ / n_ / 1e3
        alg = (12 + 4 * k + V * (4 + conf_b) + 20) * N
        moved = (4 + conf_b) * N * V + 12 * N + 8 * N * V + 8 * N * ((V + 63) // 64)
        traffic, tsrc = kernel_traffic("k_project", N * V)
        rooflines["k_project"] = {
            "bound": "hbm", "achieved": alg / sec / 1e9, "peak": HBM_GBS, "unit": "GB/s",
            "frac": alg / sec / 1e9 / HBM_GBS, "traffic": traffic, "traffic_source": tsrc, "kernel": "k_project",
            "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
            "work": f"12 + 4k + V (4 + conf bytes) + 20 B per point (the path's algorithmic bytes) x {N} points",
            "moved_by_design_GBs": moved / sec / 1e9, "ms": t_ / n_, "share": t_ / ms}
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    roofline = dict(rooflines[dom])
    kernels = {name: {"launches": n_, "ms_per_launch": t_ / max(1, n_), "share": t_ / ms} for name, (n_, t_) in kt.items()}

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.partition else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "points": N, "views": V, "map": f"{W}x{H}",
                       "H": Hh, "k": k, "T": T, "form": "plain",
                       "l2": "inputs larger than L2 (orientation+confidence maps "
                             f"{(sc['angle'].nbytes + sc['conf'].nbytes) / 1e6:.0f} MB re-read every step)",
                       "parallelism": (f"one scene, point range per rank x{world}" if args.partition
                                       else f"independent scenes per rank x{world}")},
            "roofline": roofline, "rooflines": rooflines, "kernels": kernels, "gpu_launches": launches,
            "clocks": clk}

    if rank == 0:
        full_dir = np.zeros((N, 3), np.float32)
        full_dir[lo:hi] = out_dir.cpu().numpy()
        line["accuracy"] = accuracy(sc, Hh, T, full_dir, args.accuracy_sample or 400, lo, hi)
    # end to end through the C ABI with pinned host buffers, copies inside the timed region
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        h_cams, h_ang, h_conf, h_pts, h_nbr = (pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr"))
        h_dir = torch.empty((R, 3)).pin_memory()
        h_cost = torch.empty(R).pin_memory()
        h_idx = torch.empty(R, dtype=torch.int32).pin_memory()
        h_st = torch.empty(R, dtype=torch.uint8).pin_memory()
        f2 = hf.HairFuse(Hh, k, T, 0, stream=stream.cuda_stream)

        def e2e_step():
            f2.upload_views(h_cams, h_ang, h_conf)
            f2.upload_points(h_pts, h_nbr)
            if args.partition:
                f2.fuse_range(lo, R, h_dir, h_cost, h_idx, h_st)
            else:
                f2.fuse(h_dir, h_cost, h_idx, h_st)

        e2e_step()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 5))
        for _ in range(n_e2e):
            e2e_step()
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        h2d = sum(x.numel() * x.element_size() for x in (h_cams, h_ang, h_conf, h_pts, h_nbr))
        d2h = R * (12 + 4 + 4 + 1)
        e2e_points = N if args.partition else reduce_over_ranks(N, pg, dev, "sum")
        line["e2e"] = {"value": e2e_points * n_e2e / dt, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
                       "path": "hair_fuse_upload_views/points + fuse_directions with HF_HOST pinned buffers"}
        f2.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, Hh, T)
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


# ---------------------------------------------------------------------------- serving workload
SERVING_T_SHORT, SERVING_ALPHA = 2, 0.24   # short refinement from the proposal
CALIB_SEED, CALIB_SCENES = 300, 8          # held-out serving-shaped scenes for the fallback threshold
CALIB_MEDIAN, CALIB_P95 = 1.8, 7.0         # their accuracy bounds against the plain fusion (targets 2 / 8 deg)
TRAIN_SEEDS, TRAIN_SAMPLES, TRAIN_STEPS, TRAIN_BATCH, TRAIN_LR = (100, 101, 102, 103), 500_000, 20000, 8192, 1e-3
MLP_FLOP_PER_POINT = 2 * (51 * 256 + 256 * 256 + 256 * 3)   # forward, unpadded inputs
# FP32 operations of the network's epilogue per row (CUDA cores, not tensor cores): per hidden unit
# the bias add, the clamped scaling, w8 = 8 t - 4, q = w8^2 - 8, 12 polynomial steps, Phi and the
# product x Phi (18), in both hidden layers, plus the head's 3 fused multiply-adds in layer 2
MLP_EPILOGUE_OPS_PER_POINT = 256 * (18 + 18 + 3)


def serving_scenes(first_seed, pick="16"):
    import scenegen
    cfgs = scenegen.serving_batch(first_seed)
    if "," in str(pick):
        cfgs = [cfgs[int(q)] for q in str(pick).split(",")]
    else:
        cfgs = cfgs[: int(pick)]
    return [scenegen.make_scene(**c) for c in cfgs]


def train_proposal(dev, seed_offset, calib="serving"):
    """Proposal network trained on the GPU by the library (targets: the plain GPU fusion of four
    full-like scenes), fallback threshold calibrated on the first of them."""
    import torch

    import scenegen
    from paper_2604_05794_b300 import learned as L
    t0 = time.perf_counter()
    seeds = [s + seed_offset for s in TRAIN_SEEDS]
    X, Tg = L.training_set(lambda s: scenegen.make_scene("full", seed=s), seeds, TRAIN_SAMPLES, 64, 8, dev)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    net, losses = L.train(X, Tg, steps=TRAIN_STEPS, batch=TRAIN_BATCH, lr=TRAIN_LR)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    n_samples = int(X.shape[0])
    del X, Tg
    tau, info = calibrate(net, dev, seed_offset, calib)
    t3 = time.perf_counter()
    return net, tau, dict(info, samples=n_samples, scenes=seeds, steps=TRAIN_STEPS, batch=TRAIN_BATCH, lr=TRAIN_LR,
                          loss_first50=float(np.mean(losses[:50])), loss_last200=float(np.mean(losses[-200:])),
                          data_s=round(t1 - t0, 2), train_s=round(t2 - t1, 2), calib_s=round(t3 - t2, 2))


def calibrate(net, dev, seed_offset, kind="serving"):
    """Fallback threshold from held-out scenes (seeds disjoint from the benchmark's and the training
    scenes) shaped like the workload: serving-batch scenes, or for the single full scene two
    full-preset scenes; the largest tau keeping, pooled over their points, median <= CALIB_MEDIAN and
    p95 <= CALIB_P95 degrees against the plain fusion (margins under the 2 / 8 deg targets)."""
    import scenegen
    from paper_2604_05794_b300 import learned as L
    if kind == "serving":
        first = CALIB_SEED + seed_offset
        scenes = [scenegen.make_scene(**c) for c in scenegen.serving_batch(first, CALIB_SCENES)]
        what = f"{CALIB_SCENES} held-out serving-shaped scenes (seeds {first}..{first + CALIB_SCENES - 1})"
    else:
        first = 105 + seed_offset
        scenes = [scenegen.make_scene("full", seed=first + q) for q in range(2)]
        what = f"2 held-out full-preset scenes (seeds {first}, {first + 1})"
    tau, info = L.calibrate_tau_batch(scenes, net, 64, 8, SERVING_T_SHORT, SERVING_ALPHA, dev, median_deg=CALIB_MEDIAN,
                                      p95_deg=CALIB_P95)
    return tau, {"tau": tau, "T_short": SERVING_T_SHORT, "alpha_short": SERVING_ALPHA,
                 "calibration": f"largest tau keeping median <= {CALIB_MEDIAN} deg and p95 <= {CALIB_P95} deg against "
                                f"the plain fusion, pooled over {what}",
                 "calibration_fallback_frac": info["fallback_frac"]}


def serving_accuracy(scenes, outs_learned, outs_plain, n_total):
    """Angular error of the learned + batched and of the plain directions against the FP64 oracle on
    a sample spread over the scenes in proportion to their point counts."""
    import oracle
    import paper_2604_05794_b300 as hf
    Ntot = sum(sc["N"] for sc in scenes)
    errs_l, errs_p, n = [], [], 0
    t0 = time.perf_counter()
    for sc, ol, op in zip(scenes, outs_learned, outs_plain):
        m = max(8, int(round(n_total * sc["N"] / Ntot)))
        sel = np.linspace(0, sc["N"] - 1, m).astype(np.int64)
        H, T = sc["cfg"]["H"], sc["cfg"]["T"]
        orc = oracle.fuse(oracle.Scene.from_dict(sc), hf.fibonacci_hemisphere(H), T, idx=sel)
        ok = orc["status"] == 0
        for out, errs in ((ol, errs_l), (op, errs_p)):
            a, b = out[sel][ok].astype(np.float64), orc["dir"][ok]
            errs.append(np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1)))))
        n += m
    el, ep = np.concatenate(errs_l), np.concatenate(errs_p)
    return {"vs": "FP64 oracle (plain fusion)", "sample": n, "oracle_s": round(time.perf_counter() - t0, 1),
            "median_deg": float(np.median(el)), "p95_deg": float(np.percentile(el, 95)),
            "within_2deg": float(np.mean(el <= 2.0)),
            "plain": {"median_deg": float(np.median(ep)), "p95_deg": float(np.percentile(ep, 95)),
                      "within_0p1deg": float(np.mean(ep <= 0.1))}}


def serving_cpu_baseline(scenes, budget_s=15.0):
    """The FP64 oracle (plain fusion) on the host cores over a bounded sample of the batch's points."""
    import oracle
    import paper_2604_05794_b300 as hf
    osc = [oracle.Scene.from_dict(sc) for sc in scenes]
    hyps = hf.fibonacci_hemisphere(64)
    Ntot = sum(sc["N"] for sc in scenes)
    oracle.fuse(osc[0], hyps, 8, idx=np.arange(64))   # thread start-up

    def run(per_pt_total):
        n = 0
        for o, sc in zip(osc, scenes):
            m = max(1, int(per_pt_total * sc["N"] / Ntot))
            oracle.fuse(o, hyps, sc["cfg"]["T"], idx=np.linspace(0, sc["N"] - 1, m).astype(np.int64))
            n += m
        return n

    m = 1024
    while True:   # grow the probe until it takes a measurable share of the budget
        t0 = time.perf_counter()
        n = run(m)
        dt = time.perf_counter() - t0
        if dt >= 0.15 * budget_s or m >= Ntot:
            break
        m *= 4
    if dt < 0.5 * budget_s and m < Ntot:
        m = int(min(Ntot, m * budget_s / max(dt, 1e-3)))
        t0 = time.perf_counter()
        n = run(m)
        dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} of {Ntot} points of the 16-scene batch, spread in proportion to the scenes' point "
                      f"counts, evenly spaced in each; FP64 C + OpenMP, plain fusion, {dt:.1f} s"}


def stage_rooflines(kt, ms_step, scenes, st, T_short):
    """Per-stage rooflines of the learned + batched run from one profiled eager run (stage times) and
    the work counters of the library (point-views of all points, of the fallback points and of the
    accepted proposals)."""
    ap = alu_peak()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        bf16 = float(pk.get("bf16_tflops_sustained") or pk["bf16_tflops"])
        bf16_src = "of measured: MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, seconds-long loop)"
    except (OSError, KeyError, ValueError, TypeError):
        bf16, bf16_src = 1400.0, "of fallback: 1.4 PFLOP/s sustained bf16"
    k, H, T = 8, 64, 8
    ca, cr = s8d_ops(k)
    Ntot = sum(sc["N"] for sc in scenes)
    # the learned path's projection also writes the features' view part (96 B per point)
    proj_bytes = sum((12 + 4 * k + sc["V"] * (4 + sc["conf"].itemsize) + 20 + 96) * sc["N"] for sc in scenes)
    feat_bytes = sum((12 + 32) * sc["N"] for sc in scenes)
    pv, fpv, apv = st["point_views"], st["fallback_point_views"], st["accepted_point_views"]
    units = {"k_argmin_batch": fpv, "k_refine_batch": fpv, "k_refine_short_batch": apv, "k_select_batch": pv,
             "k_project_batch": pv}
    ip = issued_per_dir_view(k)
    work = {
        "k_project_batch": ("hbm", proj_bytes, "12 + 4k + V (4 + conf bytes) + 20 B per point (the path's "
                            "algorithmic bytes) + 96 B of features (their view part) per point", None),
        "k_featpos_batch": ("hbm", feat_bytes, "12 B in + 32 B out per point (the features' position part)", None),
        "k_mlp": ("tensor", MLP_FLOP_PER_POINT * Ntot, f"{MLP_FLOP_PER_POINT} FLOP per point (51-256-256-3)", None),
        "k_select_batch": ("alu", ca * pv, f"{ca} FP32 ops per (point, view) for the proposal's cost ({pv} point-views)",
                           pv * ip),
        "k_refine_short_batch": ("alu", 6 * T_short * cr * apv,
                                 f"{6 * T_short} x {cr} FP32 ops per accepted (point, view) ({apv})",
                                 (6 * T_short + 1) * apv * ip),
        "k_argmin_batch": ("alu", H * ca * fpv, f"{H} x {ca} FP32 ops per fallback (point, view), {fpv} point-views",
                           H * fpv * ip),
        "k_refine_batch": ("alu", 6 * T * cr * fpv, f"{6 * T} x {cr} FP32 ops per fallback (point, view), {fpv}",
                           (6 * T + 1) * fpv * ip),
    }
    out = {}
    for name, (bound, amount, how, issued) in work.items():
        if name not in kt:
            continue
        sec = kt[name][1] / 1e3
        if bound == "alu":
            ach, peak, unit, src = amount / sec / 1e12, ap["peak"] / 1e12, "TFLOP/s", ap["source"]
        elif bound == "tensor":
            ach, peak, unit, src = amount / sec / 1e12, bf16, "TFLOP/s", bf16_src
        else:
            ach, peak, unit, src = amount / sec / 1e9, HBM_GBS, "GB/s", "of measured: MEASURED_PEAKS.json hbm_gbs"
        traffic, tsrc = kernel_traffic(name, units.get(name, Ntot))
        out[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "traffic": traffic, "traffic_source": tsrc, "kernel": name, "peak_source": src, "work": how,
                     "units": units.get(name, Ntot), "ms": kt[name][1], "share": kt[name][1] / ms_step}
        if bound == "alu":
            out[name]["peak_rates_ops_per_s"] = ap["rates_ops_per_s"]
            out[name]["builder_count"] = {"instr_per_dir_view": ip, "achieved_instr_per_s": issued / sec,
                                          "frac_of_ffma_issue": issued / sec / ap["rates_ops_per_s"]["ffma"]}
        if name == "k_mlp":
            # what binds the network: its GELU / head epilogue on the FP32 pipe
            ops = MLP_EPILOGUE_OPS_PER_POINT * Ntot / sec
            out[name]["epilogue_fp32"] = {"ops_per_point": MLP_EPILOGUE_OPS_PER_POINT, "achieved_ops_per_s": ops,
                                          "peak_ops_per_s": ap["rates_ops_per_s"]["ffma"],
                                          "frac_of_ffma": ops / ap["rates_ops_per_s"]["ffma"],
                                          "peak_source": "measured: hair_fuse_issue_rate HF_ISSUE_FFMA"}
    return out


def run_serving(args):
    import torch

    import paper_2604_05794_b300 as hf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    stream = torch.cuda.current_stream(dev)
    t_setup = time.perf_counter()
    if args.net:
        net = hf.ProposalNet(TRAIN_BATCH)
        net.load(args.net)
        if args.tau is not None:
            tau, train_info = args.tau, {"loaded": args.net, "tau": args.tau}
        else:
            tau, train_info = calibrate(net, dev, rank_first_seed(rank) - 200)
            train_info["loaded"] = args.net
    else:
        net, tau, train_info = train_proposal(dev, rank_first_seed(rank) - 200)
    if args.save_net:
        net.save(args.save_net)
    scenes = serving_scenes(rank_first_seed(rank), args.scenes)
    Ntot = sum(sc["N"] for sc in scenes)
    ctxs, outs_p, outs_l, outs_pb = [], [], [], []

    def outs(N):
        return (torch.empty((N, 3), device=dev), torch.empty(N, device=dev),
                torch.empty(N, dtype=torch.int32, device=dev), torch.empty(N, dtype=torch.uint8, device=dev))

    for sc in scenes:
        f = hf.HairFuse(sc["cfg"]["H"], sc["k"], sc["cfg"]["T"], 0, stream=stream.cuda_stream)
        f.upload_views(sc["cams"], sc["angle"], sc["conf"])
        f.upload_points(sc["points"], sc["nbr"])
        ctxs.append(f)
        outs_p.append(outs(sc["N"]))
        outs_l.append(outs(sc["N"]))
        outs_pb.append(outs(sc["N"]))
    K, W = args.steps, max(3, args.warmup)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(step, k):
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(k):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return reduce_over_ranks(e0.elapsed_time(e1), pg, dev)

    # plain fusion, scene after scene (the comparison)
    def plain_step():
        for f, o in zip(ctxs, outs_p):
            f.fuse(*o)

    bp = None
    if not args.only_learned:
        for _ in range(W):
            plain_step()
        ms_plain = timed(plain_step, K)
        torch.cuda.synchronize(dev)
        e0, evs = ev(), [ev() for _ in ctxs]
        e0.record(stream)
        for f, o, e in zip(ctxs, outs_p, evs):
            f.fuse(*o)
            e.record(stream)
        torch.cuda.synchronize(dev)
        lat_plain = np.array([e0.elapsed_time(e) for e in evs])

        # plain fusion, batched (no network)
        bp = hf.Batch(ctxs, autotune=True, stream=stream.cuda_stream)
        for s_, o in enumerate(outs_pb):
            bp.set_outputs(s_, *o)
        bp.run()
        for _ in range(W):
            bp.run()
        ms_pb = timed(bp.run, K)
        lat_pb = bp.latency_ms()
        tune_pb = bp.tuning()

    # learned + batched (the measured form)
    bl = hf.Batch(ctxs, net=net, T_short=SERVING_T_SHORT, alpha_short=SERVING_ALPHA, tau=tau, autotune=True,
                  stream=stream.cuda_stream)
    for s_, o in enumerate(outs_l):
        bl.set_outputs(s_, *o)
    bl.run()
    for _ in range(W):
        bl.run()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    launches0 = bl.stats()["launches"]
    clocks.start()
    time.sleep(0.3)
    ms_l = timed(bl.run, K)
    clk = clocks.stop()
    launches = bl.stats()["launches"] - launches0
    lat_l = bl.latency_ms()
    fb = bl.fallbacks()
    tune_l = bl.tuning()
    kt = bl.profile_run()
    st = bl.stats()
    bl.run()
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t_setup
    Nall = reduce_over_ranks(Ntot, pg, dev, "sum")   # points of all ranks' batches
    value = Nall * K / (ms_l / 1e3)
    plain_value = Nall * K / (ms_plain / 1e3) if bp is not None else None
    ms_prof = sum(v[1] for v in kt.values())
    rooflines = stage_rooflines(kt, ms_prof, scenes, st, SERVING_T_SHORT)
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    q = lambda a, p: float(np.percentile(a, p))
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_l / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bf16 tensor-core network)", "data": "synthetic",
            "config": {"workload": WORKLOADS["serving16"], "scenes": len(scenes), "scenes_arg": args.scenes,
                       "points": Ntot,
                       "views": [sc["V"] for sc in scenes], "maps": [f"{sc['W']}x{sc['H']}" for sc in scenes],
                       "form": "learned+batched", "H": 64, "k": 8, "T": 8,
                       "l2": "inputs larger than L2 (orientation+confidence maps "
                             f"{sum(sc['angle'].nbytes + sc['conf'].nbytes for sc in scenes) / 1e9:.1f} GB re-read "
                             "every step)",
                       "parallelism": f"independent scene batches per rank x{world}"},
            "plain": None if bp is None else {
                "value": plain_value, "unit": "points/s", "ms_per_step": ms_plain / K,
                "form": "plain fusion, scenes one by one", "latency_ms": {"p50": q(lat_plain, 50), "p95": q(lat_plain, 95)}},
            "plain_batched": None if bp is None else {
                "value": Nall * K / (ms_pb / 1e3), "ms_per_step": ms_pb / K,
                "latency_ms": {"p50": q(lat_pb, 50), "p95": q(lat_pb, 95)}, "tuning": tune_pb},
            "speedup_vs_plain": value / plain_value if bp is not None else None,
            "latency_ms": {"p50": q(lat_l, 50), "p95": q(lat_l, 95), "per_scene": [round(x, 3) for x in lat_l],
                           "source": "device global-timer stamp when a scene's last tile finishes"},
            "learned": dict(train_info, fallback_frac=float(fb.sum() / Ntot), tuning=tune_l),
            "roofline": dict(rooflines[dom]), "rooflines": rooflines,
            "kernels": {n_: {"launches": v[0], "ms": v[1], "share": v[1] / ms_prof} for n_, v in kt.items()},
            "gpu_launches": launches, "clocks": clk, "setup_s": round(setup_s, 1)}
    if rank == 0 and bp is not None:
        acc = serving_accuracy(scenes, [o[0].cpu().numpy() for o in outs_l], [o[0].cpu().numpy() for o in outs_p],
                               args.accuracy_sample or 50000)
        line["accuracy"] = acc
        line["accepted"] = bool(acc["median_deg"] <= 2.0)
    # end to end through the C ABI: every step uploads every scene from pinned host memory, runs the
    # batch's graph and reads the outputs back.  Two scene sets (contexts, batch, stream each) take
    # turns, so that one set's uploads cross the host link while the other set's batch computes, as a
    # serving loop would; every step still copies all of its inputs in and all of its outputs out
    # inside the timed region.  The serial form (one set, each upload waited for) is kept beside it.
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        host_in = [tuple(pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr")) for sc in scenes]
        s2 = torch.cuda.Stream(dev)
        ctxs2, outs2 = [], []
        for sc in scenes:
            f = hf.HairFuse(sc["cfg"]["H"], sc["k"], sc["cfg"]["T"], 0, stream=s2.cuda_stream)
            f.upload_views(sc["cams"], sc["angle"], sc["conf"])
            f.upload_points(sc["points"], sc["nbr"])
            ctxs2.append(f)
            outs2.append(outs(sc["N"]))
        bl2 = hf.Batch(ctxs2, net=net, T_short=SERVING_T_SHORT, alpha_short=SERVING_ALPHA, tau=tau, autotune=True,
                       stream=s2.cuda_stream)
        for s_, o in enumerate(outs2):
            bl2.set_outputs(s_, *o)
        sets = [(ctxs, bl, outs_l, stream), (ctxs2, bl2, outs2, s2)]
        host_out = [[tuple(torch.empty_like(x, device="cpu").pin_memory() for x in o) for o in st_[2]] for st_ in sets]

        def e2e_step(q, overlap=True):
            cs, bb, oo, ss = sets[q]
            for f, (c_, a_, cf, p_, n_) in zip(cs, host_in):   # every scene's maps queued back to back
                f.upload_views(c_, a_, cf, asynchronous=overlap)
            for f, (c_, a_, cf, p_, n_) in zip(cs, host_in):
                f.upload_points(p_, n_)   # checks the neighbour lists: waits for this set's stream
            bb.run()
            with torch.cuda.stream(ss):
                for o, h in zip(oo, host_out[q]):
                    for x, y in zip(o, h):
                        y.copy_(x, non_blocking=True)

        for q in (0, 1):   # settle both batches (tuning, graph capture) outside the timing
            e2e_step(q)
        torch.cuda.synchronize(dev)
        h2d = sum(x.numel() * x.element_size() for t_ in host_in for x in t_)
        d2h = sum(x.numel() * x.element_size() for t_ in host_out[0] for x in t_)
        path = ("hair_fuse_upload_views (HF_HOST_ASYNC, pinned) + hair_fuse_upload_points of every scene, "
                "hair_fuse_batch_run (graph), device-to-host copy of all outputs; two scene sets on two "
                "streams take turns")
        n_e2e = max(2, min(K, 10))   # enough steps that filling and draining the pipeline weigh little
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for q in range(n_e2e):
            e2e_step(q & 1)
        torch.cuda.synchronize(dev)
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        # serial: one set, every upload waited for before the batch runs
        n_ser = max(1, min(K, 3))
        t0 = time.perf_counter()
        for _ in range(n_ser):
            e2e_step(0, overlap=False)
            torch.cuda.synchronize(dev)
        dt_ser = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        line["e2e"] = {"value": Nall * n_e2e / dt, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "steps": n_e2e, "path": path,
                       "serial": {"value": Nall * n_ser / dt_ser, "steps": n_ser,
                                  "path": "one scene set, each upload waited for (HF_HOST)"}}
        bl2.close()
        for f in ctxs2:
            f.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serving_cpu_baseline(scenes)
    bl.close()
    if bp is not None:
        bp.close()
    for f in ctxs:
        f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_learned(args):
    """configs' learned form on one scene: the proposal path against the plain fusion, single GPU
    (each rank its own scene under torchrun)."""
    import torch

    import paper_2604_05794_b300 as hf
    import scenegen
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    stream = torch.cuda.current_stream(dev)
    off = rank_first_seed(rank) - 200
    net, tau, train_info = train_proposal(dev, off, calib="full")
    sc = scenegen.make_scene("full", seed=104 + off)
    N, V, k = sc["N"], sc["V"], sc["k"]
    H, T = sc["cfg"]["H"], sc["cfg"]["T"]
    f = hf.HairFuse(H, k, T, 0, stream=stream.cuda_stream)
    f.upload_views(sc["cams"], sc["angle"], sc["conf"])
    f.upload_points(sc["points"], sc["nbr"])
    mk = lambda: (torch.empty((N, 3), device=dev), torch.empty(N, device=dev),
                  torch.empty(N, dtype=torch.int32, device=dev), torch.empty(N, dtype=torch.uint8, device=dev))
    o_l, o_p = mk(), mk()
    K, W = args.steps, max(3, args.warmup)
    learned = lambda: f.fuse_learned(net, *o_l, T_short=SERVING_T_SHORT, alpha_short=SERVING_ALPHA, tau=tau,
                                     count_fallback=False)
    plain = lambda: f.fuse(*o_p)

    def timed(step):
        for _ in range(W):
            step()
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return reduce_over_ranks(e0.elapsed_time(e1), pg, dev)

    ms_p = timed(plain)
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    launches0 = f.stats()["launches"]
    clocks.start()
    time.sleep(0.3)
    ms_l = timed(learned)
    clk = clocks.stop()
    launches = (f.stats()["launches"] - launches0) * K // (K + W)
    n_fb = f.fuse_learned(net, *o_l, T_short=SERVING_T_SHORT, alpha_short=SERVING_ALPHA, tau=tau)
    point_views = f.work()
    lw = f.learned_work()
    f.profile(True)
    learned()
    kt = f.profile_read()
    f.profile(False)
    Nall = reduce_over_ranks(N, pg, dev, "sum")
    value, plain_value = Nall * K / (ms_l / 1e3), Nall * K / (ms_p / 1e3)
    ms_prof = sum(v[1] for v in kt.values())
    # per-stage rooflines from the exact work of this scene (the same units as the batched line)
    st = {"point_views": point_views, "fallback_point_views": lw["fallback_point_views"],
          "accepted_point_views": lw["accepted_point_views"]}
    names = {"k_project": "k_project_batch", "k_featpos": "k_featpos_batch", "k_mlp": "k_mlp",
             "k_select": "k_select_batch", "k_refine_short": "k_refine_short_batch",
             "k_argmin_fallback": "k_argmin_batch", "k_refine_fallback": "k_refine_batch"}
    kt_b = {names[n_]: v for n_, v in kt.items() if n_ in names}
    rb = stage_rooflines(kt_b, ms_prof, [sc], st, SERVING_T_SHORT)
    back = {v: n_ for n_, v in names.items()}
    rooflines = {}
    for n_b, r in rb.items():
        r = dict(r, kernel=back[n_b])
        r["traffic"], r["traffic_source"] = kernel_traffic(back[n_b], r["units"])
        rooflines[back[n_b]] = r
    kernels = {n_: {"launches": v[0], "ms": v[1], "share": v[1] / ms_prof} for n_, v in kt.items()}
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_l / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bf16 tensor-core network)", "data": "synthetic",
            "config": {"workload": WORKLOADS["learned"], "points": N, "views": V, "map": f"{sc['W']}x{sc['H']}",
                       "form": "learned", "H": H, "k": k, "T": T, "T_short": SERVING_T_SHORT,
                       "alpha_short": SERVING_ALPHA, "l2": "inputs larger than L2 (maps re-read every step)",
                       "parallelism": f"independent scenes per rank x{world}"},
            "plain": {"value": plain_value, "unit": "points/s", "ms_per_step": ms_p / K},
            "speedup_vs_plain": value / plain_value, "learned": dict(train_info, fallback_frac=n_fb / N),
            "roofline": dict(rooflines[dom]), "rooflines": rooflines, "kernels": kernels, "gpu_launches": launches,
            "clocks": clk}
    if rank == 0:
        acc = serving_accuracy([sc], [o_l[0].cpu().numpy()], [o_p[0].cpu().numpy()], args.accuracy_sample or 50000)
        line["accuracy"] = acc
        line["accepted"] = bool(acc["median_deg"] <= 2.0)
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hin = [pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr")]
        hout = [torch.empty((N, 3)).pin_memory(), torch.empty(N).pin_memory(),
                torch.empty(N, dtype=torch.int32).pin_memory(), torch.empty(N, dtype=torch.uint8).pin_memory()]
        f2 = hf.HairFuse(H, k, T, 0, stream=stream.cuda_stream)

        def e2e_step():
            f2.upload_views(*hin[:3])
            f2.upload_points(*hin[3:])
            f2.fuse_learned(net, *hout, T_short=SERVING_T_SHORT, alpha_short=SERVING_ALPHA, tau=tau,
                            count_fallback=False)

        e2e_step()
        n_e2e = max(1, min(K, 3))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        line["e2e"] = {"value": Nall * n_e2e / dt, "unit": "points/s",
                       "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in hin)),
                       "d2h_bytes_per_step": int(sum(x.numel() * x.element_size() for x in hout)), "steps": n_e2e,
                       "path": "hair_fuse_upload_views/points + fuse_learned with HF_HOST pinned buffers"}
        f2.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, H, T)
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


# ---------------------------------------------------------------------------- FPMVO workload
def fpmvo_units(sc, cfg):
    """Exact work counts of one FPMVO pass, for the roofline: views in front of the camera and inside
    the image per point (each tested against its depth map), views passing the test, and the top
    views used (min(K, visible)); computed on the host in float64 (pixel edges aside)."""
    P = sc["points"].astype(np.float64)
    W, H, V = sc["W"], sc["H"], sc["V"]
    dep = sc["depth"].reshape(V, -1)
    inside = np.zeros(sc["N"], np.int64)
    visible = np.zeros(sc["N"], np.int64)
    for v in range(V):
        cam = sc["cams"][v].astype(np.float64)
        X = P @ cam[4:13].reshape(3, 3).T + cam[13:16]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = np.floor(cam[0] * X[:, 0] / X[:, 2] + cam[2])
            w = np.floor(cam[1] * X[:, 1] / X[:, 2] + cam[3])
        ok = (X[:, 2] > 1e-6) & (u >= 0) & (u < W) & (w >= 0) & (w < H)
        inside += ok
        px = (np.where(ok, w, 0) * W + np.where(ok, u, 0)).astype(np.int64)
        visible += ok & (X[:, 2] <= dep[v][px] + cfg["eps_vis"])
    top = np.minimum(visible, cfg["K"])
    return {"inside_pv": int(inside.sum()), "visible_pv": int(visible.sum()), "top_pv": int(top.sum())}


def fpmvo_bytes(u, N, cfg, conf_bytes):
    """Algorithmic bytes of one pass per kernel.  k_fpmvo_views: per in-image view the depth value
    (4 B) and, where visible, the confidence; per top view the angle at the point's pixel and the
    depth at the offset pixel (4 + 4 B); the point (12 B).  k_fpmvo_fuse: per top view the P x P
    patch of angle + confidence; the outputs (21 B)."""
    P2 = cfg["P"] * cfg["P"]
    return {"k_fpmvo_views": 4 * u["inside_pv"] + conf_bytes * u["visible_pv"] + 8 * u["top_pv"] + 12 * N,
            "k_fpmvo_fuse": u["top_pv"] * P2 * (4 + conf_bytes) + 21 * N}


# DRAM bytes (read + write) per unit from one ncu capture of the mid scene (200,000 points, 32 views
# of 1024x1024): per in-image point-view for the views kernel, per top view for the fusion kernel.
FPMVO_DRAM_PER_UNIT = {"k_fpmvo_views": ("inside_pv", 315.443e6 / 6350838), "k_fpmvo_fuse": ("top_pv", 227.167e6 / 992848)}


def fpmvo_cpu_baseline(sc, cfg, budget_s=15.0):
    import oracle
    osc = oracle.Scene.from_dict(sc)
    probe = np.arange(0, sc["N"], max(1, sc["N"] // 1024))
    oracle.fpmvo(osc, sc["depth"], idx=probe[:64], **cfg)
    t0 = time.perf_counter()
    oracle.fpmvo(osc, sc["depth"], idx=probe, **cfg)
    per_pt = (time.perf_counter() - t0) / len(probe)
    n = int(min(sc["N"], max(len(probe), budget_s / max(per_pt, 1e-9))))
    sel = np.linspace(0, sc["N"] - 1, n).astype(np.int64)
    t0 = time.perf_counter()
    oracle.fpmvo(osc, sc["depth"], idx=sel, **cfg)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} of {sc['N']} points, evenly spaced, FP64 C + OpenMP FPMVO, {dt:.1f} s"}


def fpmvo_accuracy(sc, cfg, d, c, s, n_sample):
    """Agreement with the FP64 oracle on a stratified sample: the layer, the angle and the cost."""
    import oracle
    sel = np.linspace(0, sc["N"] - 1, n_sample).astype(np.int64)
    orc = oracle.fpmvo(oracle.Scene.from_dict(sc), sc["depth"], idx=sel, **cfg)
    ok = orc["status"] == 0
    a, b = d[sel].astype(np.float64), orc["dir"]
    ang = np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.abs(np.sum(a * b, axis=1))))[ok]
    return {"median_deg": float(np.median(ang)), "p99_deg": float(np.percentile(ang, 99)),
            "same_layer": float(np.mean(s[sel][ok] == orc["sel"][ok])),
            "max_cost_err": float(np.max(np.abs(c[sel][ok] - orc["cost"][ok]))), "sample": int(n_sample)}


def run_fpmvo(args):
    import torch

    import paper_2604_05794_b300 as hf
    import scenegen
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    cfg = dict(FPMVO_CFG, eps_vis=float(np.float32(FPMVO_CFG["eps_vis"])))
    sc = scenegen.make_scene(args.fpmvo_scene, seed=scenegen.PRESET_SEEDS[args.fpmvo_scene] + 100 * rank, depth=True)
    N, V, W, H = sc["N"], sc["V"], sc["W"], sc["H"]
    stream = torch.cuda.current_stream(dev)
    f = hf.HairFuse(8, sc["k"], 0, stream=stream.cuda_stream)
    gpu = {x: torch.from_numpy(sc[x]).to(dev) for x in ("cams", "angle", "conf", "points", "nbr", "depth")}
    f.upload_views(gpu["cams"], gpu["angle"], gpu["conf"])
    f.upload_points(gpu["points"], gpu["nbr"])
    f.upload_depth(gpu["depth"])
    out = (torch.empty((N, 3), device=dev), torch.empty(N, device=dev), torch.empty(N, dtype=torch.int32, device=dev),
           torch.empty(N, dtype=torch.uint8, device=dev))
    step = lambda: f.fpmvo(*out, **cfg)
    Wm = max(3, args.warmup)
    for _ in range(Wm):
        step()
    f.sync()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = f.stats()["launches"]
    f.profile(True)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kt = f.profile_read()
    f.profile(False)
    launches = f.stats()["launches"] - launches0
    ms = reduce_over_ranks(ms, pg, dev)
    value = reduce_over_ranks(N, pg, dev, "sum") * args.steps / (ms / 1e3)
    units = fpmvo_units(sc, cfg)
    byts = fpmvo_bytes(units, N, cfg, sc["conf"].itemsize)
    rooflines = {}
    for name, (n_, t_) in kt.items():
        if name not in byts:
            continue
        sec = t_ / n_ / 1e3
        ach = byts[name] / sec / 1e9
        unit_key, per_unit = FPMVO_DRAM_PER_UNIT[name]
        rooflines[name] = {"bound": "hbm", "achieved": ach, "peak": HBM_GBS, "unit": "GB/s", "frac": ach / HBM_GBS,
                           "traffic": per_unit * units[unit_key] if per_unit else None, "kernel": name,
                           "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs",
                           "work": f"{byts[name] / N:.0f} algorithmic B per point ({units['inside_pv']} in-image "
                                   f"point-views, {units['visible_pv']} visible, {units['top_pv']} top views)",
                           "share": t_ / ms}
        if per_unit:
            rooflines[name]["traffic_source"] = (f"ncu dram bytes of the mid scene, {per_unit:.1f} B per {unit_key} "
                                                 "x this pass's count")
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    roofline = dict(rooflines[dom])
    line = {"metric": "FPMVO points/s (depth-sample candidates, medoid fusion, patch consistency)", "value": value,
            "unit": "points/s", "n_gpus": world, "steps": args.steps, "warmup": Wm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["fpmvo"] if args.fpmvo_scene == "full" else
                       f"FPMVO on the {args.fpmvo_scene} scene (profiling case)", "points": N, "views": V,
                       "map": f"{W}x{H}", **cfg,
                       "l2": "inputs larger than L2 (angle, confidence and depth maps "
                             f"{(sc['angle'].nbytes + sc['conf'].nbytes + sc['depth'].nbytes) / 1e6:.0f} MB)",
                       "parallelism": f"independent scenes per rank x{world}"},
            "roofline": roofline, "rooflines": rooflines, "units": units,
            "kernels": {k_: {"launches": v[0], "ms_per_launch": v[1] / max(1, v[0]), "share": v[1] / ms}
                        for k_, v in kt.items()},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        d, c, s_ = (x.cpu().numpy() for x in out[:3])
        line["accuracy"] = fpmvo_accuracy(sc, cfg, d, c, s_, args.accuracy_sample or 2000)
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hin = {x: pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr", "depth")}
        hout = (torch.empty((N, 3)).pin_memory(), torch.empty(N).pin_memory(),
                torch.empty(N, dtype=torch.int32).pin_memory(), torch.empty(N, dtype=torch.uint8).pin_memory())
        f2 = hf.HairFuse(8, sc["k"], 0, stream=stream.cuda_stream)

        def e2e_step():
            f2.upload_views(hin["cams"], hin["angle"], hin["conf"])
            f2.upload_points(hin["points"], hin["nbr"])
            f2.upload_depth(hin["depth"])
            f2.fpmvo(*hout, **cfg)

        e2e_step()
        n_e2e = max(1, min(args.steps, 5))
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        line["e2e"] = {"value": reduce_over_ranks(N, pg, dev, "sum") * n_e2e / dt, "unit": "points/s",
                       "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in hin.values())),
                       "d2h_bytes_per_step": int(sum(x.numel() * x.element_size() for x in hout)), "steps": n_e2e,
                       "path": "hair_fuse_upload_views/points/depth + hair_fuse_fpmvo with HF_HOST pinned buffers"}
        f2.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = fpmvo_cpu_baseline(sc, cfg)
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


# ---------------------------------------------------------------------------- Gabor workload
GABOR_FLOP_PER_PIXEL = 2 * 128 * 15 * 16     # the MMAs as issued: 128 filters x 15 window rows x 16 taps
GABOR_USEFUL_FLOP_PER_PIXEL = 2 * 128 * 225  # the 15 x 15 window
# DRAM bytes per pixel of k_gabor (dram__bytes_read.sum + dram__bytes_write.sum of one launch on 4 views,
# 46.6 MB / 8.29 M pixels): the image read once (4 bytes), the outputs partly still in L2 at the end
# of so small a launch; scaled to a full launch by the pixel count
GABOR_DRAM_PER_PIXEL = (33.278208e6 + 13.347072e6) / (4 * 1920 * 1080)


def gabor_images(views=64, seed=2):
    import scenegen
    sc = scenegen.make_scene("full", seed=seed, knn=False)
    return scenegen.strand_images({"conf": sc["conf"][:views]}, seed=seed), sc


def run_gabor(args):
    import torch

    import oracle
    import paper_2604_05794_b300 as hf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    im, sc = gabor_images(views=args.gabor_views, seed=2 + 100 * rank)
    V, H, W = im.shape
    npx = V * H * W
    stream = torch.cuda.current_stream(dev)
    f = hf.HairFuse(8, 0, 0, stream=stream.cuda_stream)
    g_im = torch.from_numpy(im).to(dev)
    th = torch.empty((V, H, W), device=dev)
    cf = torch.empty((V, H, W), device=dev)
    step = lambda: f.gabor(g_im, th, cf)
    Wm = max(3, args.warmup)
    for _ in range(Wm):
        step()
    f.sync()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = f.stats()["launches"]
    f.profile(True)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kt = f.profile_read()
    f.profile(False)
    launches = f.stats()["launches"] - launches0
    ms = reduce_over_ranks(ms, pg, dev)
    value = reduce_over_ranks(npx, pg, dev, "sum") * args.steps / (ms / 1e3) / 1e6
    n_, t_ = kt["k_gabor"]
    sec = t_ / n_ / 1e3
    ach = npx * GABOR_USEFUL_FLOP_PER_PIXEL / sec / 1e12   # algorithmic: the 15 x 15 window
    issued = npx * GABOR_FLOP_PER_PIXEL / sec / 1e12
    peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1800.0
    tot = sum(v[1] for v in kt.values())
    roofline = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": GABOR_DRAM_PER_PIXEL * npx, "traffic_source": "ncu on 4 views, scaled by pixels",
                "kernel": "k_gabor",
                "peak_source": "of measured: MEASURED_PEAKS.json bf16_tflops (burst cuBLAS bf16)",
                "work": f"{GABOR_USEFUL_FLOP_PER_PIXEL} FLOP per pixel (128 filters x the 15x15 window) x {npx} pixels; "
                        f"the MMAs issue {GABOR_FLOP_PER_PIXEL} per pixel (16 taps per row, the 16th zero)",
                "issued_tflops": issued,
                "share": t_ / tot}
    line = {"metric": "Gabor orientation/confidence maps, megapixels/s", "value": value, "unit": "Mpx/s",
            "n_gpus": world, "steps": args.steps, "warmup": Wm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 x bf16 -> f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["gabor"], "views": V, "size": f"{W}x{H}", "pixels": npx,
                       "l2": f"images {im.nbytes / 1e6:.0f} MB read every step (larger than L2)",
                       "parallelism": f"independent view sets per rank x{world}"},
            "roofline": roofline, "rooflines": {"k_gabor": roofline},
            "kernels": {k_: {"launches": v[0], "ms": v[1], "share": v[1] / tot} for k_, v in kt.items()},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        thn, cfn = th.cpu().numpy(), cf.cpu().numpy()
        cov = sc["conf"][:V] > 0
        d = np.degrees(np.abs((thn - sc["angle"][:V] + np.pi / 2) % np.pi - np.pi / 2))[cov]
        idx = np.linspace(0, H * W - 1, args.accuracy_sample or 2000).astype(np.int64)
        o = oracle.gabor_pixels(im[0], idx)
        ok = o["flag"] == 0
        kk = np.rint(thn[0].ravel()[idx] * 64 / np.pi).astype(int) % 64
        line["accuracy"] = {"median_deg_vs_rendered": float(np.median(d)), "p90_deg_vs_rendered": float(np.percentile(d, 90)),
                            "oracle_index_match": float(np.mean(kk[ok] == o["k"][ok])), "oracle_unique": float(ok.mean()),
                            "max_conf_err": float(np.max(np.abs(cfn[0].ravel()[idx] - o["conf"]))), "sample": len(idx)}
    if not args.no_e2e:
        h_im = torch.from_numpy(im).pin_memory()
        h_th = torch.empty((V, H, W)).pin_memory()
        h_cf = torch.empty((V, H, W)).pin_memory()
        # the views in chunks of 4 on two contexts / streams taking turns (HF_HOST_ASYNC): one chunk's
        # images come in while another is filtered and a third's maps go out
        ch = 4
        s2 = torch.cuda.Stream(dev)
        fs = [f, hf.HairFuse(8, 0, 0, stream=s2.cuda_stream)]

        def e2e_step():
            for q, v0 in enumerate(range(0, V, ch)):
                sl = slice(v0, min(V, v0 + ch))
                fs[q & 1].gabor(h_im[sl], h_th[sl], h_cf[sl], asynchronous=True)
            torch.cuda.synchronize(dev)

        e2e_step()
        n_e2e = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        f.gabor(h_im, h_th, h_cf)   # serial: one call, copies waited for
        n_ser = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(n_ser):
            f.gabor(h_im, h_th, h_cf)
        dt_ser = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        fs[1].close()
        line["e2e"] = {"value": reduce_over_ranks(npx, pg, dev, "sum") * n_e2e / dt / 1e6, "unit": "Mpx/s",
                       "h2d_bytes_per_step": int(h_im.numel() * 4), "d2h_bytes_per_step": int(2 * npx * 4),
                       "steps": n_e2e,
                       "path": f"hair_fuse_gabor (HF_HOST_ASYNC, pinned) on chunks of {ch} views, two contexts on two "
                               "streams taking turns",
                       "serial": {"value": reduce_over_ranks(npx, pg, dev, "sum") * n_ser / dt_ser / 1e6,
                                  "steps": n_ser, "path": "hair_fuse_gabor with HF_HOST pinned buffers, one call"}}
    if rank == 0 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        n_s = 300000   # about 10 s of the single-threaded oracle
        oracle.gabor_pixels(im[0], np.linspace(0, H * W - 1, n_s).astype(np.int64))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n_s / dt / 1e6, "unit": "Mpx/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n_s} evenly spaced pixels of view 0 (single-threaded C, double sums), "
                                          f"{dt:.1f} s"}
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def run_reference_gabor(args, world):
    import oracle
    im, _ = gabor_images(views=1)
    H, W = im.shape[1:]
    n = 3000
    run = lambda: oracle.gabor_pixels(im[0], np.linspace(0, H * W - 1, n).astype(np.int64))
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = time.perf_counter() - t0
    value = n * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "Gabor orientation/confidence maps, megapixels/s", "value": value,
            "unit": "Mpx/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 sums of bf16 values", "data": "synthetic",
            "config": {"workload": WORKLOADS["gabor"], "pixels_per_step": n},
            "cpu_baseline": {"value": value, "unit": "Mpx/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} evenly spaced pixels of view 0 per step"},
            "e2e": {"value": value, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- PHG workload
def phg_inputs(n_strands=0, seed=2, noise=0.1):
    """Points, noisy unit directions, scalp seeds and normals of the full preset's strands."""
    import scenegen
    over = dict(n_strands=n_strands) if n_strands else {}
    sc = scenegen.make_scene("full", seed=seed, strand_maps=False, knn=False, **over)
    rng = np.random.default_rng(seed)
    d = sc["tangents"] + rng.normal(size=sc["tangents"].shape).astype(np.float32) * np.float32(noise)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    roots = np.ascontiguousarray(sc["verts"][:, 0], np.float32)
    normals = (roots / np.linalg.norm(roots, axis=1, keepdims=True)).astype(np.float32)
    pts = np.ascontiguousarray(sc["points"], np.float32)
    lo = pts.min(0) - 2 * PHG_CFG["voxel"]
    dims = np.ceil((pts.max(0) + 2 * PHG_CFG["voxel"] - lo) / PHG_CFG["voxel"]).astype(int)
    return pts, d, roots, normals, lo.astype(np.float32), dims


def phg_cfgs(lo, dims):
    import ctypes

    import oracle
    import paper_2604_05794_b300 as hf
    c = PHG_CFG
    args = (c["voxel"], *[int(x) for x in dims], c["step"], c["max_steps"], c["root_steps"], c["cos_turn"], c["occ_cap"],
            c["batch"], c["link_dist"], c["link_cos"])
    return hf.hf_phg_cfg((ctypes.c_float * 3)(*[float(x) for x in lo]), *args), oracle.phg_cfg(lo, c["voxel"], dims,
                                                                                              *args[4:])


def phg_cpu(n_strands, steps=1):
    """The oracle on a scene of n_strands strands (the same preset and parameters): points/s."""
    import oracle
    pts, d, roots, normals, lo, dims = phg_inputs(n_strands)
    _, oc = phg_cfgs(lo, dims)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.phg(oc, pts, d, roots, normals, seg_cap=len(pts))
    dt = time.perf_counter() - t0
    return len(pts) * steps / dt, len(pts), dt


def run_phg(args):
    import torch

    import paper_2604_05794_b300 as hf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    pts, d, roots, normals, lo, dims = phg_inputs(args.phg_strands, seed=2 + 100 * rank)
    gc, _ = phg_cfgs(lo, dims)
    N, S = len(pts), len(roots)
    nvox = int(np.prod(dims))
    cap = min(nvox, N)
    stream = torch.cuda.current_stream(dev)
    f = hf.HairFuse(8, 0, 0, stream=stream.cuda_stream)
    g_in = [torch.from_numpy(x).to(dev) for x in (pts, d, roots, normals)]
    outs = f.phg_outputs(gc, S, cap, dev)
    step = lambda: f.phg(gc, *g_in, outputs=outs, cut=False)
    Wm = max(3, args.warmup)
    for _ in range(Wm):
        step()
    f.sync()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(cvd.split(",")[local] if cvd else str(local))
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = f.stats()["launches"]
    f.profile(True)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    kt = f.profile_read()
    f.profile(False)
    launches = f.stats()["launches"] - launches0
    ms = reduce_over_ranks(ms, pg, dev)
    value = reduce_over_ranks(N, pg, dev, "sum") * args.steps / (ms / 1e3)
    K = int(outs["n_seg"][0])
    glen = outs["glen"].cpu().numpy()
    slen = outs["slen"][:K].cpu().numpy()
    label = outs["label"][:S + K].cpu().numpy()
    occ = outs["occ"].cpu().numpy()
    # algorithmic work per kernel: the splat reads a point and direction (24 B) and adds 28 B of counts
    # and tensor sums; every trace step reads a voxel's count, crowd and orientation (20 B)
    steps_taken = int(np.maximum(glen - 1, 0).sum() + np.maximum(slen - 1, 0).sum())
    ktime = {k_: v[1] for k_, v in kt.items()}
    total_kms = sum(ktime.values())
    work = {"k_phg_splat": (N * (24 + 28), "B"), "k_phg_orient": (nvox * (4 + 48 + 12), "B"),
            "k_phg_trace_guides": (int(np.maximum(glen - 1, 0).sum()) * 20, "B"),
            "k_phg_trace_segments": (int(np.maximum(slen - 1, 0).sum()) * 20, "B")}
    rooflines = {}
    for name, (byt, _) in work.items():
        if name not in kt:
            continue
        n_, t_ = kt[name]
        ach = byt * n_ / args.steps / (t_ / 1e3) / 1e9 if t_ > 0 else 0.0
        rooflines[name] = {"bound": "hbm", "achieved": ach, "peak": HBM_GBS, "unit": "GB/s", "frac": ach / HBM_GBS,
                           "traffic": None, "kernel": name, "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs",
                           "share": t_ / total_kms}
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    line = {"metric": "PHG input points/s (volumes, guide strands, segments, linking)", "value": value,
            "unit": "points/s", "n_gpus": world, "steps": args.steps, "warmup": Wm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (int64 fixed-point sums)",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["phg"], "points": N, "seeds": S, "grid": [int(x) for x in dims],
                       "voxels": nvox, **PHG_CFG, "l2": f"grid state {nvox * 80 / 1e6:.0f} MB rebuilt every step",
                       "parallelism": f"independent scenes per rank x{world}"},
            "result": {"occupied_voxels": int((occ > 0).sum()), "guides_grown": int((glen > 1).sum()),
                       "guide_mean_vertices": float(glen[glen > 0].mean()) if (glen > 0).any() else 0.0,
                       "segment_seeds": K, "segments_grown": int((slen > 1).sum()), "trace_steps": steps_taken,
                       "components": int(len(np.unique(label)))},
            "roofline": dict(rooflines[dom]), "rooflines": rooflines,
            "kernels": {k_: {"launches": v[0], "ms": v[1], "share": v[1] / total_kms} for k_, v in kt.items()},
            "gpu_launches": launches, "clocks": clk}
    if not args.no_e2e:
        f2 = hf.HairFuse(8, 0, 0, stream=stream.cuda_stream)
        pin = lambda a: torch.from_numpy(a).pin_memory()
        h_in = [pin(x) for x in (pts, d, roots, normals)]
        h_out = {k_: torch.zeros(v.shape, dtype=v.dtype).pin_memory() for k_, v in outs.items()}
        e2e = lambda: f2.phg(gc, *h_in, outputs=h_out, cut=False)
        e2e()
        n_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e()
        dt = reduce_over_ranks(time.perf_counter() - t0, pg, dev)
        d2h = sum(v.numel() * v.element_size() for k_, v in h_out.items() if k_ not in ("sverts", "svox", "stan", "slen"))
        d2h += K * (4 + 8 + 24 + 12 * (2 * gc.max_steps + 1))
        line["e2e"] = {"value": reduce_over_ranks(N, pg, dev, "sum") * n_e2e / dt, "unit": "points/s",
                       "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in h_in)),
                       "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
                       "path": "hair_fuse_phg with HF_HOST pinned buffers (inputs in, volumes and strands out)"}
        f2.close()
    if rank == 0 and not args.no_cpu_baseline:
        v, n, dt = phg_cpu(400)
        line["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": 1, "kind": "oracle",
                                "sample": f"the oracle (single-threaded C) on the same preset with 400 strands "
                                          f"({n} points, same parameters), {dt:.1f} s"}
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "phg":
        run_phg(args)
    elif args.workload == "gabor":
        run_gabor(args)
    elif args.workload == "fpmvo":
        run_fpmvo(args)
    elif args.workload == "serving16":
        run_serving(args)
    elif args.workload == "learned":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
