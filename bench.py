"""Benchmark of the multi-view hair direction fusion on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload full|mid|tiny]

One step = one pass of the whole fusion path (per-scene constants, projection + gather, cost of
every hypothesis, argmin, refinement) over every point of a resident synthetic scene shaped like the
paper's outer point clouds (default: 1,000,000 points, 64 views of 1920x1080, H = 64, k = 8, T = 8).
Rank 0 prints one JSON line.  Under torchrun each rank fuses its own scene (independent problems,
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
    "full": "plain fusion, full: 1,000,000 points (20,000 strands x 50 segments), 64 views 1920x1080, "
            "f32 angle + fp16 confidence, 0.5 deg pose noise, H=64, k=8, T=8",
    "mid": "plain fusion, mid: 200,000 points, 32 views 1024x1024 with 10% outlier pixels, H=64, k=8, T=8",
    "tiny": "plain fusion, tiny: 2,000 points, 8 views 256x256, H=32, k=5, T=4",
}
SM_COUNT, FP32_LANES_PER_SM = 148, 128


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
    ap.add_argument("--workload", default="full", choices=list(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--accuracy-sample", type=int, default=400)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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


def accuracy(sc, H, T, gpu_dir, n_sample):
    """Angular error of the GPU directions against the FP64 oracle on a stratified sample."""
    import oracle
    osc = oracle.Scene.from_dict(sc)
    import paper_2604_05794_b300 as hf
    hyps = hf.fibonacci_hemisphere(H)
    sel = np.linspace(0, sc["N"] - 1, n_sample).astype(np.int64)
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
    sc = make_workload(args.workload)
    H, T = sc["cfg"]["H"], sc["cfg"]["T"]
    osc = oracle.Scene.from_dict(sc)
    hyps = oracle.fibonacci_hemisphere(H)
    # bounded sample per step so that warmup + steps finish within a few minutes
    probe = np.arange(0, sc["N"], max(1, sc["N"] // 512))
    oracle.fuse(osc, hyps, T, idx=probe[:64])             # thread start-up
    t0 = time.perf_counter()
    oracle.fuse(osc, hyps, T, idx=probe)
    per_pt = (time.perf_counter() - t0) / len(probe)
    budget = 90.0 / max(1, args.steps + args.warmup)
    n = int(min(sc["N"], max(64, budget / max(per_pt, 1e-9))))
    sel = np.linspace(0, sc["N"] - 1, n).astype(np.int64)
    for _ in range(args.warmup):
        oracle.fuse(osc, hyps, T, idx=sel[: max(1, n // 8)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fuse(osc, hyps, T, idx=sel)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = f"{n} of {sc['N']} points per step, evenly spaced; FP64 C + OpenMP"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "points_per_step": n},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
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
    sc = make_workload(args.workload, seed_offset=100 * rank)
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
    out_dir = torch.empty((N, 3), device=dev)
    out_cost = torch.empty(N, device=dev)
    out_idx = torch.empty(N, dtype=torch.int32, device=dev)
    out_st = torch.empty(N, dtype=torch.uint8, device=dev)

    def step():
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
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    f.sync()
    value = N * world * args.steps / (ms / 1e3)

    # rooflines: the cost kernels are FP32-issue bound, the projection/gather kernel HBM bound
    peak_alu = SM_COUNT * FP32_LANES_PER_SM * 2032.0e6
    per_member = 3 * (k + 1) + 6     # FP32 ops per (direction, view): 3 per patch member + 6
    conf_b = sc["conf"].itemsize
    work = {"k_argmin": (Hh * per_member, "alu"), "k_refine": (6 * T * per_member, "alu"),
            "k_project": (4 + conf_b + 16, "hbm")}
    rooflines = {}
    for name, (per_pv, bound) in work.items():
        if name not in kt:
            continue
        n_, t_ = kt[name]
        sec = t_ / n_ / 1e3
        if bound == "alu":
            ach, pk_, unit = per_pv * point_views / sec / 1e12, peak_alu / 1e12, "TFLOP/s"
            src = "derived: 148 SMs x 128 FP32 lanes x 2032 MHz max SM clock (1 op per lane per clock)"
            wk = f"{per_pv} FP32 ops per (point, view) in V_i x {point_views} point-views per launch"
        else:
            byt = per_pv * N * V + 12 * N
            ach, pk_, unit = byt / sec / 1e9, HBM_GBS, "GB/s"
            src = "of measured: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"
            wk = f"{per_pv} B per (point, view) x {N * V} point-views + 12 B per point"
        rooflines[name] = {"bound": bound, "achieved": ach, "peak": pk_, "unit": unit, "frac": ach / pk_,
                           "traffic": None, "kernel": name, "peak_source": src, "work": wk, "share": t_ / ms}
    dom = max(rooflines, key=lambda x: rooflines[x]["share"])
    roofline = dict(rooflines[dom])
    kernels = {name: {"launches": n_, "ms_per_launch": t_ / max(1, n_), "share": t_ / ms} for name, (n_, t_) in kt.items()}

    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "points": N, "views": V, "map": f"{W}x{H}",
                       "H": Hh, "k": k, "T": T, "form": "plain",
                       "l2": "inputs larger than L2 (orientation+confidence maps "
                             f"{(sc['angle'].nbytes + sc['conf'].nbytes) / 1e6:.0f} MB re-read every step)",
                       "parallelism": f"independent scenes per rank x{world}"},
            "roofline": roofline, "rooflines": rooflines, "kernels": kernels, "gpu_launches": launches,
            "clocks": clk}

    if rank == 0:
        line["accuracy"] = accuracy(sc, Hh, T, out_dir.cpu().numpy(), args.accuracy_sample)
    # end to end through the C ABI with pinned host buffers, copies inside the timed region
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        h_cams, h_ang, h_conf, h_pts, h_nbr = (pin(sc[x]) for x in ("cams", "angle", "conf", "points", "nbr"))
        h_dir = torch.empty((N, 3)).pin_memory()
        h_cost = torch.empty(N).pin_memory()
        h_idx = torch.empty(N, dtype=torch.int32).pin_memory()
        h_st = torch.empty(N, dtype=torch.uint8).pin_memory()
        f2 = hf.HairFuse(Hh, k, T, 0, stream=stream.cuda_stream)

        def e2e_step():
            f2.upload_views(h_cams, h_ang, h_conf)
            f2.upload_points(h_pts, h_nbr)
            f2.fuse(h_dir, h_cost, h_idx, h_st)

        e2e_step()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 5))
        for _ in range(n_e2e):
            e2e_step()
        dt = time.perf_counter() - t0
        if pg:
            t = torch.tensor([dt], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            dt = float(t.item())
        h2d = sum(x.numel() * x.element_size() for x in (h_cams, h_ang, h_conf, h_pts, h_nbr))
        d2h = N * (12 + 4 + 4 + 1)
        line["e2e"] = {"value": N * world * n_e2e / dt, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
