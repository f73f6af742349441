"""Seeded synthetic hair scenes (inputs only; none of the fusion arithmetic lives here).

A scene is what the fusion step of Sec. 3.1 consumes: a raw outer point cloud, calibrated
pinhole cameras, per-view orientation maps (angle in [0, pi)) with confidence maps, and each
point's k nearest neighbours.  Generation runs in ``libscenegen.so`` (C, OpenMP) and is a pure
function of the configuration and the seed.

Presets (workloads shaped like the paper's outer-layer point clouds):

``tiny``  2,000 points on 200 helical strands (10 per strand, evenly spaced in arc length),
          8 cameras on a ring of radius 3, f = 300 px, 256x256 maps, k = 5.
``mid``   200,000 points, one per segment midpoint of 5,000 strands x 40 segments
          (thirds straight / wavy / curly), 32 cameras on a half orbit with +-15 deg elevation
          jitter, f = 1200 px, 1024x1024 maps, 10 % outlier pixels (uniform angle, conf < 0.3), k = 8.
``full``  1,000,000 points from 20,000 strands x 50 segments, 64 cameras on a full orbit with
          0.5 deg per-frame pose noise, 1920x1080 maps, fp16 confidence, k = 8.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libscenegen.so")


class SgConfig(ctypes.Structure):
    _fields_ = [
        ("n_strands", ctypes.c_int), ("n_segments", ctypes.c_int), ("points_mode", ctypes.c_int),
        ("pts_per_strand", ctypes.c_int), ("strand_mix", ctypes.c_int),
        ("helix_r_lo", ctypes.c_double), ("helix_r_hi", ctypes.c_double),
        ("pitch_lo", ctypes.c_double), ("pitch_hi", ctypes.c_double),
        ("wave_a_lo", ctypes.c_double), ("wave_a_hi", ctypes.c_double),
        ("wave_len_lo", ctypes.c_double), ("wave_len_hi", ctypes.c_double),
        ("len_lo", ctypes.c_double), ("len_hi", ctypes.c_double), ("cap_deg", ctypes.c_double),
        ("V", ctypes.c_int), ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("f", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("cam_mode", ctypes.c_int), ("cam_radius", ctypes.c_double), ("elev_jitter_deg", ctypes.c_double),
        ("pose_noise_deg", ctypes.c_double), ("angle_noise_deg", ctypes.c_double),
        ("conf_lo", ctypes.c_double), ("conf_hi", ctypes.c_double),
        ("outlier_frac", ctypes.c_double), ("outlier_conf_hi", ctypes.c_double),
        ("k", ctypes.c_int), ("seed", ctypes.c_uint64),
    ]


PRESETS = {
    "tiny": dict(n_strands=200, n_segments=32, points_mode=0, pts_per_strand=10, strand_mix=0,
                 helix_r_lo=0.02, helix_r_hi=0.1, pitch_lo=0.05, pitch_hi=0.3,
                 V=8, width=256, height=256, f=300.0, cam_mode=0, elev_jitter_deg=0.0,
                 pose_noise_deg=0.0, outlier_frac=0.0, k=5, conf_f16=False, H=32, T=4),
    "mid": dict(n_strands=5000, n_segments=40, points_mode=1, strand_mix=1,
                helix_r_lo=0.01, helix_r_hi=0.08, pitch_lo=0.05, pitch_hi=0.3,
                V=32, width=1024, height=1024, f=1200.0, cam_mode=1, elev_jitter_deg=15.0,
                pose_noise_deg=0.0, outlier_frac=0.10, k=8, conf_f16=False, H=64, T=8),
    "full": dict(n_strands=20000, n_segments=50, points_mode=1, strand_mix=1,
                 helix_r_lo=0.01, helix_r_hi=0.08, pitch_lo=0.05, pitch_hi=0.3,
                 V=64, width=1920, height=1080, f=1300.0, cam_mode=2, elev_jitter_deg=0.0,
                 pose_noise_deg=0.5, outlier_frac=0.0, k=8, conf_f16=True, H=64, T=8),
}
PRESET_SEEDS = {"tiny": 0, "mid": 1, "full": 2}

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            build()
        lib = ctypes.CDLL(_LIB_PATH)
        p = ctypes.POINTER
        lib.sg_num_points.argtypes = [p(SgConfig)]
        lib.sg_num_points.restype = ctypes.c_longlong
        lib.sg_make_points.argtypes = [p(SgConfig), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.sg_make_cameras.argtypes = [p(SgConfig), ctypes.c_void_p, ctypes.c_void_p]
        lib.sg_render_strand_maps.argtypes = [p(SgConfig), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        lib.sg_render_exact_maps.argtypes = [p(SgConfig), ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.sg_knn.argtypes = [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        for fn in ("sg_make_points", "sg_make_cameras", "sg_render_strand_maps", "sg_render_exact_maps", "sg_knn"):
            getattr(lib, fn).restype = ctypes.c_int
        _lib = lib
    return _lib


def build():
    """Compile libscenegen.so next to this file (gcc, OpenMP)."""
    import subprocess
    src = os.path.join(_HERE, "scenegen.c")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB_PATH, src, "-lm"])


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def config(preset="tiny", seed=None, **over):
    """Resolved configuration dict for a preset with overrides."""
    cfg = dict(n_strands=200, n_segments=32, points_mode=0, pts_per_strand=10, strand_mix=0,
               helix_r_lo=0.02, helix_r_hi=0.1, pitch_lo=0.05, pitch_hi=0.3,
               wave_a_lo=0.01, wave_a_hi=0.08, wave_len_lo=0.05, wave_len_hi=0.15,
               len_lo=0.15, len_hi=0.35, cap_deg=70.0,
               V=8, width=256, height=256, f=300.0, cx=None, cy=None, cam_mode=0, cam_radius=3.0,
               elev_jitter_deg=0.0, pose_noise_deg=0.0, angle_noise_deg=5.0, conf_lo=0.5, conf_hi=1.0,
               outlier_frac=0.0, outlier_conf_hi=0.3, k=5, conf_f16=False, H=32, T=4)
    cfg.update(PRESETS[preset])
    cfg.update(over)
    if cfg["cx"] is None:
        cfg["cx"] = cfg["width"] / 2.0
    if cfg["cy"] is None:
        cfg["cy"] = cfg["height"] / 2.0
    cfg["seed"] = PRESET_SEEDS[preset] if seed is None else seed
    return cfg


def _cstruct(cfg):
    c = SgConfig()
    for name, _ in SgConfig._fields_:
        setattr(c, name, cfg[name])
    return c


def serving_batch(first_seed=200, n=16):
    """Scene configurations of an uneven serving batch (keyword arguments of make_scene): scene s
    draws, from its own seed, N log-uniform in [50k, 1M] (strands of 50 segments, one point per
    segment), V uniform in {16, ..., 64} and maps from {512x512, 1024x1024, 1920x1080} (focal length
    scaled with the width so the field of view stays that of the full preset; fp16 confidence at
    1920x1080); otherwise the full preset (orbit, 0.5 deg pose noise, H = 64, k = 8, T = 8)."""
    import math
    sizes = [(512, 512), (1024, 1024), (1920, 1080)]
    out = []
    for s in range(first_seed, first_seed + n):
        rng = np.random.default_rng(s)
        N = math.exp(rng.uniform(math.log(5e4), math.log(1e6)))
        V = int(rng.integers(16, 65))
        W, H = sizes[int(rng.integers(0, 3))]
        out.append(dict(preset="full", seed=s, n_strands=max(1, int(round(N / 50))), V=V, width=W, height=H,
                        f=1300.0 * W / 1920.0, conf_f16=(W == 1920)))
    return out


def make_scene(preset="tiny", seed=None, exact_maps=False, strand_maps=True, knn=True, depth=False, **over):
    """Generate one scene.  Returns a dict of numpy arrays and sizes:

    points (N,3) f32, tangents (N,3) f32 unit, strand_id (N,) i32,
    cams (V,16) f32 - the cameras handed to the fusion (noisy when pose noise is set),
    cams_clean (V,16) f32 - the cameras the maps were rendered with,
    angle (V,H,W) f32 in [0, pi), conf (V,H,W) f32 or f16 in [0, 1],
    exact_angle/exact_conf/owner (if exact_maps): point-splatted maps of the true tangents,
    nbr (N,k) i32 - k nearest other points, nearest first, ties to the lower index,
    depth (V,H,W) f32 (if depth) - camera-space depth Z of the front-most rendered strand, +inf where
    no strand covers the pixel (the renderer's z-buffer, depth interpolated linearly along segments).
    Camera record: fx, fy, cx, cy, R (3x3 row-major world->camera), t (3); pixel axes +u right, +v down.
    """
    lib = _load()
    cfg = config(preset, seed, **over)
    c = _cstruct(cfg)
    N = int(lib.sg_num_points(ctypes.byref(c)))
    V, W, H, k = cfg["V"], cfg["width"], cfg["height"], cfg["k"]
    pts = np.empty((N, 3), np.float32)
    tan = np.empty((N, 3), np.float32)
    sid = np.empty((N,), np.int32)
    verts = np.empty((cfg["n_strands"], cfg["n_segments"] + 1, 3), np.float32)
    lib.sg_make_points(ctypes.byref(c), _ptr(pts), _ptr(tan), _ptr(sid), _ptr(verts))
    cams_clean = np.empty((V, 16), np.float32)
    cams = np.empty((V, 16), np.float32)
    lib.sg_make_cameras(ctypes.byref(c), _ptr(cams_clean), _ptr(cams))
    out = dict(cfg=cfg, N=N, V=V, W=W, H=H, k=k, points=pts, tangents=tan, strand_id=sid,
               verts=verts, cams=cams, cams_clean=cams_clean)
    if strand_maps:
        angle = np.empty((V, H, W), np.float32)
        conf = np.empty((V, H, W), np.float16 if cfg["conf_f16"] else np.float32)
        dep = np.empty((V, H, W), np.float32) if depth else None
        lib.sg_render_strand_maps(ctypes.byref(c), _ptr(verts), _ptr(cams_clean), _ptr(angle), _ptr(conf),
                                  1 if cfg["conf_f16"] else 0, _ptr(dep))
        out["angle"], out["conf"] = angle, conf
        if depth:
            out["depth"] = dep
    if exact_maps:
        ea = np.empty((V, H, W), np.float32)
        ec = np.empty((V, H, W), np.float32)
        owner = np.empty((V, N), np.int32)
        lib.sg_render_exact_maps(ctypes.byref(c), N, _ptr(pts), _ptr(tan), _ptr(cams), _ptr(ea), _ptr(ec),
                                 _ptr(owner))
        out["exact_angle"], out["exact_conf"], out["owner"] = ea, ec, owner
    if knn and k > 0:
        out["nbr"] = knn_of(pts, k)
    return out


def knn_of(points, k):
    """k nearest other points (N,k) int32, nearest first, ties to the lower index."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    nbr = np.empty((pts.shape[0], k), np.int32)
    rc = lib.sg_knn(pts.shape[0], _ptr(pts), k, _ptr(nbr))
    if rc != 0:
        raise ValueError("knn: k must be < N")
    return nbr


def subset_scene(scene, idx):
    """Restrict a scene to the points idx, re-indexing neighbours by a fresh kNN on the subset."""
    out = dict(scene)
    out["points"] = np.ascontiguousarray(scene["points"][idx])
    out["tangents"] = np.ascontiguousarray(scene["tangents"][idx])
    out["strand_id"] = np.ascontiguousarray(scene["strand_id"][idx])
    out["N"] = len(idx)
    k = min(scene.get("k", 0), len(idx) - 1)
    out["k"] = k
    out["nbr"] = knn_of(out["points"], k) if k > 0 else np.zeros((len(idx), 0), np.int32)
    out.pop("owner", None)
    return out


def strand_images(scene, blur=0.8, noise=0.02, seed=0):
    """Grayscale views of the rendered strands, (V, H, W) f32 in [0, 1]: the strand coverage of the
    rasterised maps (confidence > 0) blurred by a Gaussian of `blur` px, scaled to a unit maximum per
    view, plus N(0, noise) pixel noise from `seed`, clipped to [0, 1]."""
    from scipy.ndimage import gaussian_filter
    conf = np.asarray(scene["conf"], np.float32)
    rng = np.random.default_rng(seed)
    out = np.empty(conf.shape, np.float32)
    for v in range(conf.shape[0]):
        im = gaussian_filter((conf[v] > 0).astype(np.float32), blur)
        m = im.max()
        im = im / m if m > 0 else im
        out[v] = np.clip(im + rng.normal(size=im.shape).astype(np.float32) * np.float32(noise), 0.0, 1.0)
    return out
