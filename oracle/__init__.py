"""FP64 CPU oracle for the multi-view direction fusion (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import
this package.  It shares no code with the CUDA library and never calls it.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double, one point at a time, OpenMP over
points); this module only marshals numpy arrays.  ``mlp.py`` holds the FP64 reference of the
learned proposal network.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, NO_VIEWS, BAD_INPUT = 0, 1, 2
FLAG_IDX_TIE, FLAG_REFINE_TIE, FLAG_BOUNDARY = 1, 2, 4


class _Scene(ctypes.Structure):
    _fields_ = [("N", ctypes.c_longlong), ("V", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("k", ctypes.c_int), ("pts", ctypes.c_void_p), ("cams", ctypes.c_void_p),
                ("angle", ctypes.c_void_p), ("conf", ctypes.c_void_p), ("conf_f16", ctypes.c_int),
                ("nbr", ctypes.c_void_p)]


_lib = None


_SOURCES = ("oracle.c", "phg.c", "gabor.c")


def build():
    """Compile liboracle.so next to this file (gcc -O2, OpenMP, no floating-point contraction: the
    single-precision parts round once per written operation)."""
    import subprocess
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", _LIB_PATH,
                           *[os.path.join(_HERE, f) for f in _SOURCES], "-lm"])


def _load():
    global _lib
    if _lib is None:
        newest = max(os.path.getmtime(os.path.join(_HERE, f)) for f in _SOURCES)
        if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
            build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, ll, i32 = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int
        lib.or_fuse.argtypes = [vp, ll, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, vp, i32]
        lib.or_eval_costs.argtypes = [vp, ll, vp, i32, vp, i32, vp, i32]
        lib.or_fibonacci_hemisphere.argtypes = [i32, vp]
        lib.or_fibonacci_hemisphere.restype = None
        lib.or_project.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
        lib.or_reproject_dir.argtypes = [vp, vp, vp, vp]
        lib.or_reproject_dir.restype = ctypes.c_double
        lib.or_view_term.argtypes = [vp, ll, i32, vp]
        lib.or_view_term.restype = ctypes.c_double
        lib.or_view_set.argtypes = [vp, ll, i32, vp]
        lib.or_max_threads.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Scene:
    """Holds contiguous copies of the scene arrays and the C view of them."""

    def __init__(self, points, cams, angle, conf, nbr):
        # f32 inputs widen exactly; callers may also pass float64 geometry directly
        self.points = np.ascontiguousarray(points, np.float64)
        self.cams = np.ascontiguousarray(cams, np.float64)
        self.angle = np.ascontiguousarray(angle, np.float32)
        self.conf_f16 = conf.dtype == np.float16
        self.conf = np.ascontiguousarray(conf, np.float16 if self.conf_f16 else np.float32)
        self.k = 0 if nbr is None else int(nbr.shape[1])
        self.nbr = np.ascontiguousarray(nbr if nbr is not None else np.zeros((len(self.points), 0)), np.int32)
        V, H, W = self.angle.shape
        self.V, self.H, self.W, self.N = V, H, W, len(self.points)
        self.c = _Scene(self.N, V, W, H, self.k, self.points.ctypes.data, self.cams.ctypes.data,
                        self.angle.ctypes.data, self.conf.ctypes.data, int(self.conf_f16), self.nbr.ctypes.data)

    @classmethod
    def from_dict(cls, sc, exact=False):
        if exact:
            return cls(sc["points"], sc["cams"], sc["exact_angle"], sc["exact_conf"], sc.get("nbr"))
        return cls(sc["points"], sc["cams"], sc["angle"], sc["conf"], sc.get("nbr"))


def fibonacci_hemisphere(H):
    """(H, 3) float64 Fibonacci hemisphere directions (z_m = 1 - (m+1/2)/H)."""
    out = np.empty((H, 3), np.float64)
    _load().or_fibonacci_hemisphere(H, _p(out))
    return out


def fuse(scene, hyps, T, top_k=0, idx=None, threads=0):
    """Oracle fusion of the listed points (all when idx is None).

    hyps: (H,3) unit directions (f32 values widen exactly).  Returns dict of
    dir (n,3) f64, cost (n,) f64, idx (n,) i32, status (n,) u8, flags (n,) u8 (FLAG_*),
    tie_step (n,) i8: first refinement round whose two best costs are within 2e-6, else -1."""
    lib = _load()
    hyps = np.ascontiguousarray(hyps, np.float64)
    H = hyps.shape[0]
    if idx is None:
        n, ip = scene.N, None
    else:
        idx = np.ascontiguousarray(idx, np.int64)
        n, ip = len(idx), _p(idx)
    out = dict(dir=np.empty((n, 3)), cost=np.empty(n), idx=np.empty(n, np.int32),
               status=np.empty(n, np.uint8), flags=np.empty(n, np.uint8), tie_step=np.empty(n, np.int8))
    lib.or_fuse(ctypes.byref(scene.c), n, ip, _p(hyps), H, T, top_k, _p(out["dir"]), _p(out["cost"]),
                _p(out["idx"]), _p(out["status"]), _p(out["flags"]), _p(out["tie_step"]), threads)
    return out


def eval_costs(scene, dirs, idx=None, top_k=0, threads=0):
    """c_i(d) for each listed point i and each of its M directions; dirs (n, M, 3)."""
    lib = _load()
    dirs = np.ascontiguousarray(dirs, np.float64)
    n, M = dirs.shape[0], dirs.shape[1]
    idx = np.arange(scene.N, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    assert len(idx) == n
    out = np.empty((n, M))
    lib.or_eval_costs(ctypes.byref(scene.c), n, _p(idx), M, _p(dirs), top_k, _p(out), threads)
    return out


def project(cam, p, W, H):
    """(visible, u, v, a, b) of point p (3,) in camera cam (16,)."""
    lib = _load()
    cam = np.ascontiguousarray(cam, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    u, v, a, b = (ctypes.c_double() for _ in range(4))
    vis = lib.or_project(_p(cam), _p(p), W, H, ctypes.byref(u), ctypes.byref(v), ctypes.byref(a), ctypes.byref(b))
    return vis, u.value, v.value, a.value, b.value


def reproject_dir(cam, p, d):
    """Image-plane offset r (2,) = dPi/dp . d of direction d at point p."""
    lib = _load()
    cam = np.ascontiguousarray(cam, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    r = np.empty(2)
    lib.or_reproject_dir(_p(cam), _p(p), _p(d), _p(r))
    return r


def view_term(scene, i, v, d):
    """L_v(d) of point i in view v."""
    d = np.ascontiguousarray(d, np.float64)
    return _load().or_view_term(ctypes.byref(scene.c), i, v, _p(d))


def view_set(scene, i, top_k=0):
    mask = np.zeros(scene.V, np.uint8)
    n = _load().or_view_set(ctypes.byref(scene.c), i, top_k, _p(mask))
    return n, mask


def max_threads():
    return int(_load().or_max_threads())


def refine(scene, d0, T, alpha0, top_k=0, idx=None, threads=0):
    """Learned-path oracle step: from start directions d0 (n, 3), the cost and T refinement rounds with
    first step alpha0 (radians).  Returns dict dir, cost, status, flags, tie_step."""
    lib = _load()
    lib.or_refine.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                              ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    d0 = np.ascontiguousarray(d0, np.float64)
    if idx is None:
        n, ip = scene.N, None
    else:
        idx = np.ascontiguousarray(idx, np.int64)
        n, ip = len(idx), _p(idx)
    out = dict(dir=np.empty((n, 3)), cost=np.empty(n), status=np.empty(n, np.uint8), flags=np.empty(n, np.uint8),
               tie_step=np.empty(n, np.int8))
    lib.or_refine(ctypes.byref(scene.c), n, ip, _p(d0), T, alpha0, top_k, _p(out["dir"]), _p(out["cost"]),
                  _p(out["status"]), _p(out["flags"]), _p(out["tie_step"]), threads)
    return out


def features(scene):
    """Proposal-network features (N, 64) float64 of every point (before bf16 rounding)."""
    lib = _load()
    lib.or_features_all.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    pts = scene.points
    fin = np.all(np.isfinite(pts), axis=1)
    box = np.concatenate([pts[fin].min(axis=0), pts[fin].max(axis=0)]).astype(np.float64)
    out = np.empty((scene.N, 64))
    lib.or_features_all(ctypes.byref(scene.c), _p(box), _p(out))
    return out


FLAG_MEDOID_TIE, FLAG_SEL_TIE, FLAG_DEPTH_EDGE = 8, 16, 32


class _FpmvoCfg(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("S", ctypes.c_int), ("P", ctypes.c_int), ("lambda_px", ctypes.c_double),
                ("delta", ctypes.c_double), ("eps_vis", ctypes.c_double)]


def backproject(cam, u, v, z):
    """World point at camera depth z on the ray through pixel (u, v) (inverse projection, Eq. 3)."""
    lib = _load()
    lib.or_backproject.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_void_p]
    c = np.ascontiguousarray(cam, np.float64)
    out = np.empty(3)
    lib.or_backproject(_p(c), u, v, z, _p(out))
    return out


def medoid(dirs, w):
    """(index, best score, runner-up score) of the weighted medoid of unit directions (n, 3)."""
    lib = _load()
    lib.or_medoid.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.or_medoid.restype = ctypes.c_int
    d = np.ascontiguousarray(dirs, np.float64)
    ww = np.ascontiguousarray(w, np.float64)
    b, s = ctypes.c_double(), ctypes.c_double()
    i = lib.or_medoid(len(ww), _p(d), _p(ww), ctypes.byref(b), ctypes.byref(s))
    return i, b.value, s.value


def fpmvo(scene, depth, K=5, S=5, P=5, lambda_px=4.0, delta=0.005, eps_vis=0.02, idx=None, threads=0,
          layers=False):
    """The paper's FPMVO step (Sec. 3.1.1-3.1.3) for the points idx: candidates from depth samples
    around pixel-offset points, medoid fusion per depth layer over the top-K views, P x P patch
    consistency.  depth: (V, H, W) f32 camera-space depth maps (+inf where no hair).  Returns dict
    dir (n, 3), cost (n,), sel (n,) chosen depth layer, status (n,), flags (n,); with layers=True
    also layer_L (n, S), every layer's mean consistency (-1 without candidates), and layer_dir
    (n, S, 3), its fused direction."""
    lib = _load()
    lib.or_fpmvo.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    dep = np.ascontiguousarray(depth, np.float32)
    cfg = _FpmvoCfg(K, S, P, lambda_px, delta, eps_vis)
    if idx is None:
        n, ip = scene.N, None
    else:
        idx = np.ascontiguousarray(idx, np.int64)
        n, ip = len(idx), _p(idx)
    out = dict(dir=np.empty((n, 3)), cost=np.empty(n), sel=np.empty(n, np.int32), status=np.empty(n, np.uint8),
               flags=np.empty(n, np.uint8))
    lp = ld = None
    if layers:
        out["layer_L"], out["layer_dir"] = np.empty((n, S)), np.empty((n, S, 3))
        lp, ld = _p(out["layer_L"]), _p(out["layer_dir"])
    rc = lib.or_fpmvo(ctypes.byref(scene.c), _p(dep), ctypes.byref(cfg), n, ip, _p(out["dir"]), _p(out["cost"]),
                      _p(out["sel"]), _p(out["status"]), _p(out["flags"]), lp, ld, threads)
    if rc != 0:
        raise ValueError("fpmvo: K and S in [1, 16], P odd")
    return out


# ---------------------------------------------------------------------------- Parallel Hair Growing
class _PhgCfg(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("step", ctypes.c_float), ("max_steps", ctypes.c_int),
                ("root_steps", ctypes.c_int), ("cos_turn", ctypes.c_float), ("occ_cap", ctypes.c_int),
                ("batch", ctypes.c_int), ("link_dist", ctypes.c_float), ("link_cos", ctypes.c_float)]


PHG_MAXLEN, PHG_OUTSIDE, PHG_EMPTY, PHG_CROWDED, PHG_TURN, PHG_NO_ROOT = 1, 2, 3, 4, 5, 6


def phg_cfg(origin, voxel, dims, step, max_steps, root_steps, cos_turn, occ_cap, batch, link_dist, link_cos):
    c = _PhgCfg()
    c.origin[:] = [float(np.float32(x)) for x in origin]
    c.voxel, (c.nx, c.ny, c.nz), c.step = voxel, [int(x) for x in dims], step
    c.max_steps, c.root_steps, c.cos_turn, c.occ_cap, c.batch = max_steps, root_steps, cos_turn, occ_cap, batch
    c.link_dist, c.link_cos = link_dist, link_cos
    return c


def phg_voxel(cfg, p):
    """Voxel index of the f32 point p (-1 outside the grid)."""
    lib = _load()
    lib.or_phg_voxel.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.or_phg_voxel.restype = ctypes.c_longlong
    q = np.ascontiguousarray(p, np.float32)
    return lib.or_phg_voxel(ctypes.byref(cfg), _p(q))


def phg_orient_one(t6, count):
    """Orientation of one voxel from its six fixed-point tensor sums (int64) and point count."""
    lib = _load()
    lib.or_phg_orient_one.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.or_phg_orient_one.restype = None
    t = np.ascontiguousarray(t6, np.int64)
    out = np.empty(3, np.float32)
    lib.or_phg_orient_one(_p(t), count, _p(out))
    return out


def phg_splat(cfg, pts, dirs, valid=None):
    """Step A: occupancy counts (nvox,) and fixed-point tensor sums (nvox, 6)."""
    lib = _load()
    lib.or_phg_splat.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]
    lib.or_phg_splat.restype = None
    nvox = cfg.nx * cfg.ny * cfg.nz
    p = np.ascontiguousarray(pts, np.float32)
    d = np.ascontiguousarray(dirs, np.float32)
    v = None if valid is None else np.ascontiguousarray(valid, np.uint8)
    occ = np.empty(nvox, np.int32)
    T = np.empty((nvox, 6), np.int64)
    lib.or_phg_splat(ctypes.byref(cfg), len(p), _p(p), _p(d), None if v is None else _p(v), _p(occ), _p(T))
    return occ, T


def phg(cfg, pts, dirs, seeds, normals, valid=None, seg_cap=None):
    """Steps A to E of the Parallel Hair Growing consumer.  Returns a dict: occ (nvox,), ori (nvox, 3),
    crowd (nvox,) strands per voxel at the end; guide strands: gverts (S, L+1, 3), glen (S,), gstop (S,),
    gtan (S, 3); segments (K of them): sverts (K, 2L+1, 3), slen (K,), svox (K,) seed voxels,
    stan (K, 2, 3) outward tangents at (start, end); label (S + K,) component labels."""
    lib = _load()
    lib.or_phg_run.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    lib.or_phg_run.restype = ctypes.c_longlong
    nvox = cfg.nx * cfg.ny * cfg.nz
    L = cfg.max_steps
    p = np.ascontiguousarray(pts, np.float32)
    d = np.ascontiguousarray(dirs, np.float32)
    v = None if valid is None else np.ascontiguousarray(valid, np.uint8)
    sd = np.ascontiguousarray(seeds, np.float32)
    nm = np.ascontiguousarray(normals, np.float32)
    S = len(sd)
    cap = nvox if seg_cap is None else seg_cap
    o = dict(occ=np.empty(nvox, np.int32), ori=np.empty((nvox, 3), np.float32), crowd=np.empty(nvox, np.int32),
             gverts=np.zeros((S, L + 1, 3), np.float32), glen=np.empty(S, np.int32), gstop=np.empty(S, np.int32),
             gtan=np.empty((S, 3), np.float32), sverts=np.zeros((cap, 2 * L + 1, 3), np.float32),
             slen=np.empty(cap, np.int32), svox=np.empty(cap, np.int64), stan=np.zeros((cap, 2, 3), np.float32),
             label=np.empty(S + cap, np.int32))
    K = lib.or_phg_run(ctypes.byref(cfg), len(p), _p(p), _p(d), None if v is None else _p(v), S, _p(sd), _p(nm),
                       _p(o["occ"]), _p(o["ori"]), _p(o["crowd"]), _p(o["gverts"]), _p(o["glen"]), _p(o["gstop"]),
                       _p(o["gtan"]), cap, _p(o["sverts"]), _p(o["slen"]), _p(o["svox"]), _p(o["stan"]),
                       _p(o["label"]))
    if K < 0:
        raise ValueError("phg: more segment seeds than seg_cap")
    for key in ("sverts", "slen", "svox", "stan"):
        o[key] = o[key][:K]
    o["label"] = o["label"][:S + K]
    return o


# ---------------------------------------------------------------------------- Gabor orientation maps
GABOR = dict(n_theta=64, r=7, sa=2.5, sb=1.5, lam=4.0)


def bf16(x):
    """Round f32 values to bfloat16 (nearest even), returned as f32."""
    lib = _load()
    lib.or_bf16.argtypes = [ctypes.c_float]
    lib.or_bf16.restype = ctypes.c_float
    return np.array([lib.or_bf16(float(v)) for v in np.ravel(x)], np.float32).reshape(np.shape(x))


def gabor_bank(n_theta=64, r=7, sa=2.5, sb=1.5, lam=4.0):
    """(n_theta, 2, 2r+1, 2r+1) f32 bfloat16-valued kernels: even (zero-mean) and odd per orientation."""
    lib = _load()
    lib.or_gabor_bank.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_void_p]
    lib.or_gabor_bank.restype = None
    w = 2 * r + 1
    out = np.empty((n_theta, 2, w, w), np.float32)
    lib.or_gabor_bank(n_theta, r, sa, sb, lam, _p(out))
    return out


def gabor_pixels(img, idx=None, n_theta=64, r=7, sa=2.5, sb=1.5, lam=4.0):
    """Orientation index, angle, confidence and near-tie flag at the pixels idx (flat) of one (H, W) image."""
    lib = _load()
    lib.or_gabor_pixels.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.or_gabor_pixels.restype = None
    im = np.ascontiguousarray(img, np.float32)
    H, W = im.shape
    bank = gabor_bank(n_theta, r, sa, sb, lam)
    idx = np.arange(H * W, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    n = len(idx)
    out = dict(k=np.empty(n, np.int32), theta=np.empty(n, np.float32), conf=np.empty(n, np.float32),
               flag=np.empty(n, np.uint8))
    lib.or_gabor_pixels(_p(im), H, W, n_theta, r, _p(bank), n, _p(idx), _p(out["k"]), _p(out["theta"]),
                        _p(out["conf"]), _p(out["flag"]))
    return out
