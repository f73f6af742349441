"""Python binding of libhairfuse (multi-view hair direction fusion on B300, sm_103a).

Argument marshalling only: every step of the fusion runs in the library's CUDA kernels.  The
functions below carry the C names of ``include/hair_fuse.h``; ``HairFuse`` wraps a context.
Tensors may be CUDA tensors (passed as device pointers, work queued on the context's stream) or
host tensors / numpy arrays (the library copies in and out and returns when done).

There is no CPU fallback: importing this package raises if the compiled library is missing.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhairfuse.so")

HF_OK, HF_ERR_INVALID_ARG, HF_ERR_NOT_UPLOADED, HF_ERR_OOM, HF_ERR_CUDA, HF_ERR_TIMEOUT, HF_ERR_SHAPE = 0, -1, -2, -3, -4, -5, -6
HF_HOST, HF_DEVICE, HF_HOST_ASYNC = 0, 1, 2
HF_F32, HF_F16 = 0, 1
HF_STATUS_OK, HF_STATUS_NO_VIEWS, HF_STATUS_BAD_INPUT, HF_STATUS_FELL_BACK = 0, 1, 2, 3

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhairfuse.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                      "python paper_2604_05794_b300/build.py")
_lib = ctypes.CDLL(LIB_PATH)


class hf_config(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("k", ctypes.c_int), ("T", ctypes.c_int), ("top_k_views", ctypes.c_int),
                ("fallback_tau", ctypes.c_float), ("flags", ctypes.c_int)]


class hf_fpmvo_cfg(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("S", ctypes.c_int), ("P", ctypes.c_int), ("lambda_px", ctypes.c_float),
                ("delta", ctypes.c_float), ("eps_vis", ctypes.c_float)]


class hf_phg_cfg(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("step", ctypes.c_float), ("max_steps", ctypes.c_int),
                ("root_steps", ctypes.c_int), ("cos_turn", ctypes.c_float), ("occ_cap", ctypes.c_int),
                ("batch", ctypes.c_int), ("link_dist", ctypes.c_float), ("link_cos", ctypes.c_float)]


class hf_phg_out(ctypes.Structure):
    _fields_ = [("occ", ctypes.c_void_p), ("ori", ctypes.c_void_p), ("crowd", ctypes.c_void_p),
                ("gverts", ctypes.c_void_p), ("glen", ctypes.c_void_p), ("gstop", ctypes.c_void_p),
                ("gtan", ctypes.c_void_p), ("seg_cap", ctypes.c_longlong), ("sverts", ctypes.c_void_p),
                ("slen", ctypes.c_void_p), ("svox", ctypes.c_void_p), ("stan", ctypes.c_void_p),
                ("label", ctypes.c_void_p), ("n_seg", ctypes.c_void_p)]


PHG_MAXLEN, PHG_OUTSIDE, PHG_EMPTY, PHG_CROWDED, PHG_TURN, PHG_NO_ROOT = 1, 2, 3, 4, 5, 6


class hf_gabor_cfg(ctypes.Structure):
    _fields_ = [("n_theta", ctypes.c_int), ("radius", ctypes.c_int), ("sigma_along", ctypes.c_float),
                ("sigma_across", ctypes.c_float), ("lambda_", ctypes.c_float)]


GABOR_DEFAULT = dict(n_theta=64, radius=7, sigma_along=2.5, sigma_across=1.5, lambda_=4.0)


class hf_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


_vp, _i, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
_SIGS = {
    "hair_fuse_create": ([ctypes.POINTER(_vp), ctypes.POINTER(hf_config), _vp], _i),
    "hair_fuse_set_stream": ([_vp, _vp], _i),
    "hair_fuse_upload_views": ([_vp, _i, _i, _i, _vp, _vp, _vp, _i, _i], _i),
    "hair_fuse_upload_points": ([_vp, _i, _vp, _vp, _i], _i),
    "hair_fuse_fuse_directions": ([_vp, _vp, _vp, _vp, _vp, _vp, _i], _i),
    "hair_fuse_fuse_directions_noalloc": ([ctypes.POINTER(hf_config), _i, _i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp,
                                           _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "hair_fuse_fuse_range": ([_vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _i], _i),
    "hair_fuse_upload_depth": ([_vp, _vp, _i], _i),
    "hair_fuse_fpmvo": ([_vp, _vp, _vp, _vp, _vp, _vp, _i], _i),
    "hair_fuse_eval_costs": ([_vp, _i, _vp, _vp, _i], _i),
    "hair_fuse_gabor": ([_vp, ctypes.POINTER(hf_gabor_cfg), _i, _i, _i, _vp, _vp, _vp, _i], _i),
    "hair_fuse_gabor_bank": ([ctypes.POINTER(hf_gabor_cfg), _vp], _i),
    "hair_fuse_phg": ([_vp, ctypes.POINTER(hf_phg_cfg), _ll, _vp, _vp, _vp, _ll, _vp, _vp, ctypes.POINTER(hf_phg_out),
                       _i], _i),
    "hair_fuse_fibonacci_hemisphere": ([_i, _vp], _i),
    "hair_fuse_gemm_bf16": ([_vp, _vp, _vp, _i, _i, _i, _vp], _i),
    "hair_fuse_gemm_bf16_bounded": ([_vp, _vp, _vp, _i, _i, _i, ctypes.c_ulonglong, _vp], _i),
    "hair_fuse_gelu_eval": ([_vp, _vp, _ll, _vp], _i),
    "hair_fuse_mlp_set_wait_limit": ([_vp, ctypes.c_ulonglong], _i),
    "hair_fuse_fail_alloc_after": ([_i], _i),
    "hair_fuse_sync": ([_vp], _i),
    "hair_fuse_profile": ([_vp, _i], _i),
    "hair_fuse_profile_read": ([_vp, ctypes.POINTER(hf_kernel_time), _i], _i),
    "hair_fuse_stats": ([_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll)], _i),
    "hair_fuse_work": ([_vp, ctypes.POINTER(_ll)], _i),
    "hair_fuse_destroy": ([_vp], None),
    "hair_fuse_last_error": ([_vp], ctypes.c_char_p),
    "hair_fuse_mlp_param_count": ([], _ll),
    "hair_fuse_mlp_create": ([ctypes.POINTER(_vp), _i, _vp], _i),
    "hair_fuse_mlp_destroy": ([_vp], None),
    "hair_fuse_mlp_init": ([_vp, ctypes.c_uint64], _i),
    "hair_fuse_mlp_set_params": ([_vp, _vp, _i], _i),
    "hair_fuse_mlp_get_params": ([_vp, _vp, _i], _i),
    "hair_fuse_mlp_train": ([_vp, _vp, _vp, _ll, _i, _i, ctypes.c_float, ctypes.c_uint64, _i, _vp], _i),
    "hair_fuse_mlp_grads": ([_vp, _vp, _vp, _ll, _i, ctypes.c_uint64, _vp, _vp, _vp, _vp], _i),
    "hair_fuse_mlp_forward": ([_vp, _vp, _i, _vp, _i], _i),
    "hair_fuse_mlp_forward_raw": ([_vp, _vp, _i, _vp, _i], _i),
    "hair_fuse_mlp_save": ([_vp, ctypes.c_char_p], _i),
    "hair_fuse_mlp_load": ([_vp, ctypes.c_char_p], _i),
    "hair_fuse_mlp_last_error": ([_vp], ctypes.c_char_p),
    "hair_fuse_features": ([_vp, _vp, _i], _i),
    "hair_fuse_fuse_learned": ([_vp, _vp, _i, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp, _vp,
                                ctypes.POINTER(_i), _i], _i),
    "hair_fuse_learned_work": ([_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll)], _i),
    "hair_fuse_batch_create": ([ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _vp, _vp, _vp], _i),
    "hair_fuse_batch_set_outputs": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "hair_fuse_batch_run": ([_vp, _i], _i),
    "hair_fuse_batch_sync": ([_vp], _i),
    "hair_fuse_batch_latency": ([_vp, _vp], _i),
    "hair_fuse_batch_fallbacks": ([_vp, _vp], _i),
    "hair_fuse_batch_tuning": ([_vp, _vp], _i),
    "hair_fuse_batch_tuned_from_cache": ([_vp], _i),
    "hair_fuse_batch_profile_run": ([_vp, ctypes.POINTER(hf_kernel_time), _i], _i),
    "hair_fuse_batch_stats": ([_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll), ctypes.POINTER(_ll),
                               ctypes.POINTER(_ll)], _i),
    "hair_fuse_batch_destroy": ([_vp], None),
    "hair_fuse_batch_last_error": ([_vp], ctypes.c_char_p),
    "hair_fuse_issue_rate": ([_i, _i, _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_float)], _i),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

# the C entry points, under their C names
hair_fuse_create = _lib.hair_fuse_create
hair_fuse_set_stream = _lib.hair_fuse_set_stream
hair_fuse_upload_views = _lib.hair_fuse_upload_views
hair_fuse_upload_points = _lib.hair_fuse_upload_points
hair_fuse_fuse_directions = _lib.hair_fuse_fuse_directions
hair_fuse_fuse_directions_noalloc = _lib.hair_fuse_fuse_directions_noalloc
hair_fuse_fuse_range = _lib.hair_fuse_fuse_range
hair_fuse_upload_depth = _lib.hair_fuse_upload_depth
hair_fuse_fpmvo = _lib.hair_fuse_fpmvo
hair_fuse_eval_costs = _lib.hair_fuse_eval_costs
hair_fuse_phg = _lib.hair_fuse_phg
hair_fuse_gabor = _lib.hair_fuse_gabor
hair_fuse_gabor_bank = _lib.hair_fuse_gabor_bank


def gabor_cfg(**kw):
    return hf_gabor_cfg(**dict(GABOR_DEFAULT, **kw))


def gabor_bank(**kw):
    """The Gabor bank (64, 2, 15, 15) f32 (bfloat16 values), host only."""
    out = np.empty((64, 2, 15, 15), np.float32)
    _check(hair_fuse_gabor_bank(ctypes.byref(gabor_cfg(**kw)), out.ctypes.data))
    return out
hair_fuse_fibonacci_hemisphere = _lib.hair_fuse_fibonacci_hemisphere
hair_fuse_gemm_bf16 = _lib.hair_fuse_gemm_bf16
hair_fuse_gemm_bf16_bounded = _lib.hair_fuse_gemm_bf16_bounded
hair_fuse_gelu_eval = _lib.hair_fuse_gelu_eval
hair_fuse_mlp_set_wait_limit = _lib.hair_fuse_mlp_set_wait_limit
hair_fuse_fail_alloc_after = _lib.hair_fuse_fail_alloc_after
hair_fuse_sync = _lib.hair_fuse_sync
hair_fuse_profile = _lib.hair_fuse_profile
hair_fuse_profile_read = _lib.hair_fuse_profile_read
hair_fuse_stats = _lib.hair_fuse_stats
hair_fuse_work = _lib.hair_fuse_work
hair_fuse_destroy = _lib.hair_fuse_destroy
hair_fuse_last_error = _lib.hair_fuse_last_error
hair_fuse_mlp_param_count = _lib.hair_fuse_mlp_param_count
hair_fuse_mlp_create = _lib.hair_fuse_mlp_create
hair_fuse_mlp_destroy = _lib.hair_fuse_mlp_destroy
hair_fuse_mlp_init = _lib.hair_fuse_mlp_init
hair_fuse_mlp_set_params = _lib.hair_fuse_mlp_set_params
hair_fuse_mlp_get_params = _lib.hair_fuse_mlp_get_params
hair_fuse_mlp_train = _lib.hair_fuse_mlp_train
hair_fuse_mlp_grads = _lib.hair_fuse_mlp_grads
hair_fuse_mlp_forward = _lib.hair_fuse_mlp_forward
hair_fuse_mlp_forward_raw = _lib.hair_fuse_mlp_forward_raw
hair_fuse_mlp_save = _lib.hair_fuse_mlp_save
hair_fuse_mlp_load = _lib.hair_fuse_mlp_load
hair_fuse_mlp_last_error = _lib.hair_fuse_mlp_last_error
hair_fuse_features = _lib.hair_fuse_features
hair_fuse_fuse_learned = _lib.hair_fuse_fuse_learned
hair_fuse_learned_work = _lib.hair_fuse_learned_work
hair_fuse_batch_create = _lib.hair_fuse_batch_create
hair_fuse_batch_set_outputs = _lib.hair_fuse_batch_set_outputs
hair_fuse_batch_run = _lib.hair_fuse_batch_run
hair_fuse_batch_sync = _lib.hair_fuse_batch_sync
hair_fuse_batch_latency = _lib.hair_fuse_batch_latency
hair_fuse_batch_fallbacks = _lib.hair_fuse_batch_fallbacks
hair_fuse_batch_tuning = _lib.hair_fuse_batch_tuning
hair_fuse_batch_tuned_from_cache = _lib.hair_fuse_batch_tuned_from_cache
hair_fuse_batch_profile_run = _lib.hair_fuse_batch_profile_run
hair_fuse_batch_stats = _lib.hair_fuse_batch_stats
hair_fuse_batch_destroy = _lib.hair_fuse_batch_destroy
hair_fuse_batch_last_error = _lib.hair_fuse_batch_last_error
hair_fuse_issue_rate = _lib.hair_fuse_issue_rate

HF_ISSUE_FFMA, HF_ISSUE_FFMA2, HF_ISSUE_FMUL2, HF_ISSUE_FMAX_ABS, HF_ISSUE_FMAX3, HF_ISSUE_PATCH = 0, 1, 2, 3, 4, 5
HF_ISSUE_FMAX3_ABS, HF_ISSUE_PATCH3, HF_ISSUE_PATCH3S = 6, 7, 8
ISSUE_KINDS = {"ffma": HF_ISSUE_FFMA, "ffma2": HF_ISSUE_FFMA2, "fmul2": HF_ISSUE_FMUL2,
               "fmax_abs": HF_ISSUE_FMAX_ABS, "fmax3": HF_ISSUE_FMAX3, "patch": HF_ISSUE_PATCH,
               "fmax3_abs": HF_ISSUE_FMAX3_ABS, "patch3": HF_ISSUE_PATCH3, "patch3s": HF_ISSUE_PATCH3S}


class HairFuseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hair_fuse error {code}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != HF_OK:
        msg = hair_fuse_last_error(ctx)
        raise HairFuseError(rc, msg.decode() if msg else "")
    return rc


def _ptr_kind(x):
    """(pointer, mem_kind, keepalive) of a torch tensor or numpy array; None -> NULL."""
    if x is None:
        return None, None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous")
        return x.ctypes.data, HF_HOST, x
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), (HF_DEVICE if x.is_cuda else HF_HOST), x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _same_kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("all buffers of one call must be either host or device memory")
    return ks.pop() if ks else HF_HOST


def current_stream_handle():
    """torch's current CUDA stream (cudaStream_t as int), or 0 (default stream) without CUDA."""
    import torch
    if not torch.cuda.is_available():
        return 0
    return torch.cuda.current_stream().cuda_stream


def fibonacci_hemisphere(H):
    """The library's built-in hypotheses, (H, 3) float32 (computed on the GPU)."""
    out = np.empty((H, 3), np.float32)
    _check(hair_fuse_fibonacci_hemisphere(H, out.ctypes.data))
    return out


def issue_rate(kind, iters=4096, stream=None):
    """One timed launch of the FP32 issue-rate microbenchmark (``kind`` a key of ISSUE_KINDS):
    dict(instr, ops, ms, instr_per_s, ops_per_s).  Synchronous."""
    instr, ops, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_float()
    rc = hair_fuse_issue_rate(ISSUE_KINDS[kind], iters, current_stream_handle() if stream is None else stream,
                              ctypes.byref(instr), ctypes.byref(ops), ctypes.byref(ms))
    if rc != HF_OK:
        raise HairFuseError(rc, f"issue-rate probe {kind} failed")
    sec = ms.value * 1e-3
    return dict(instr=instr.value, ops=ops.value, ms=ms.value, instr_per_s=instr.value / sec,
                ops_per_s=ops.value / sec)


def gemm_bf16(a, b, out=None, stream=None):
    """C = a @ b.T on the tensor cores: a (M, K), b (N, K) CUDA bf16 tensors -> (M, N) float32."""
    import torch
    assert a.is_cuda and b.is_cuda and a.dtype == torch.bfloat16 and b.dtype == torch.bfloat16
    M, K = a.shape
    N = b.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=a.device)
    _check(hair_fuse_gemm_bf16(a.data_ptr(), b.data_ptr(), out.data_ptr(), M, N, K,
                               current_stream_handle() if stream is None else stream))
    return out


def gelu_eval(x, out=None, stream=None):
    """The network's inference GELU on a CUDA float32 tensor (asynchronous on the stream)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    if out is None:
        out = torch.empty_like(x)
    _check(hair_fuse_gelu_eval(x.data_ptr(), out.data_ptr(), x.numel(),
                               current_stream_handle() if stream is None else stream))
    return out


class HairFuse:
    """One fusion context: a scene (views + points) and the configuration (H, k, T, top-K)."""

    def __init__(self, H, k, T, top_k_views=0, fallback_tau=0.0, stream=None):
        self.cfg = hf_config(H, k, T, top_k_views, fallback_tau, 0)
        if stream is None:
            stream = current_stream_handle()
        h = _vp()
        _check(hair_fuse_create(ctypes.byref(h), ctypes.byref(self.cfg), stream))
        self.h = h
        self.N = self.V = 0
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            hair_fuse_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, rc):
        return _check(rc, self.h)

    def set_stream(self, stream):
        self._c(hair_fuse_set_stream(self.h, stream))

    def upload_views(self, cams, angle, conf, asynchronous=False):
        """cams (V,16) f32, angle (V,H,W) f32, conf (V,H,W) f32 or f16.  asynchronous=True (pinned
        torch CPU tensors only, HF_HOST_ASYNC): the copies are queued on the context's stream and
        the call returns at once; keep the tensors unchanged until the stream has consumed them."""
        V, Hh, W = angle.shape
        cdt = HF_F16 if str(conf.dtype).endswith("float16") else HF_F32
        pc, k1, a = _ptr_kind(cams)
        pa, k2, b = _ptr_kind(angle)
        pf, k3, c = _ptr_kind(conf)
        kind = _same_kind(k1, k2, k3)
        if asynchronous:
            if kind != HF_HOST or not all(getattr(x, "is_pinned", lambda: False)() for x in (cams, angle, conf)):
                raise ValueError("asynchronous uploads take pinned torch CPU tensors")
            kind = HF_HOST_ASYNC
        self._c(hair_fuse_upload_views(self.h, V, W, Hh, pc, pa, pf, cdt, kind))
        self.V = V
        self._keep = [a, b, c]

    def upload_points(self, xyz, nbr):
        """xyz (N,3) f32, nbr (N,k) int32."""
        px, k1, a = _ptr_kind(xyz)
        pn, k2, b = _ptr_kind(nbr)
        self._c(hair_fuse_upload_points(self.h, xyz.shape[0], px, pn, _same_kind(k1, k2)))
        self.N = xyz.shape[0]
        self._keep += [a, b]

    def fuse(self, dir_out, cost_out=None, idx_out=None, status_out=None, hyps=None):
        """Fuse all points into caller buffers (all host or all device)."""
        ptrs = [_ptr_kind(x) for x in (hyps, dir_out, cost_out, idx_out, status_out)]
        kind = _same_kind(*[p[1] for p in ptrs])
        self._c(hair_fuse_fuse_directions(self.h, *[p[0] for p in ptrs], kind))

    def fuse_range(self, first, count, dir_out, cost_out=None, idx_out=None, status_out=None, hyps=None):
        """Fuse points first .. first + count - 1 into caller buffers of count rows."""
        ptrs = [_ptr_kind(x) for x in (hyps, dir_out, cost_out, idx_out, status_out)]
        kind = _same_kind(*[p[1] for p in ptrs])
        self._c(hair_fuse_fuse_range(self.h, first, count, *[p[0] for p in ptrs], kind))

    def upload_depth(self, depth):
        """Depth maps (V, H, W) f32 of the uploaded views (host array or CUDA tensor)."""
        p, kind, _keep = _ptr_kind(depth)
        self._c(hair_fuse_upload_depth(self.h, p, kind))

    def fpmvo(self, dir_out, cost_out=None, sel_out=None, status_out=None, K=5, S=5, P=5, lambda_px=4.0,
              delta=0.005, eps_vis=0.02):
        """The paper's FPMVO step (depth-sample candidates, medoid fusion, P x P patch consistency)."""
        cfg = hf_fpmvo_cfg(K, S, P, lambda_px, delta, eps_vis)
        ptrs = [_ptr_kind(x) for x in (dir_out, cost_out, sel_out, status_out)]
        kind = _same_kind(*[q[1] for q in ptrs])
        self._c(hair_fuse_fpmvo(self.h, ctypes.byref(cfg), *[q[0] for q in ptrs], kind))

    def phg_outputs(self, cfg, S, seg_cap, device=None):
        """Zeroed output arrays for phg (numpy, or CUDA tensors on `device`)."""
        nvox = cfg.nx * cfg.ny * cfg.nz
        L = cfg.max_steps
        if device is not None:
            import torch
            mk = lambda shape, dt: torch.zeros(shape, dtype=dt, device=device)
            i32, f32, i64 = torch.int32, torch.float32, torch.int64
        else:
            mk = lambda shape, dt: np.zeros(shape, dtype=dt)
            i32, f32, i64 = np.int32, np.float32, np.int64
        return dict(occ=mk(nvox, i32), ori=mk((nvox, 3), f32), crowd=mk(nvox, i32), gverts=mk((S, L + 1, 3), f32),
                    glen=mk(S, i32), gstop=mk(S, i32), gtan=mk((S, 3), f32), sverts=mk((seg_cap, 2 * L + 1, 3), f32),
                    slen=mk(seg_cap, i32), svox=mk(seg_cap, i64), stan=mk((seg_cap, 2, 3), f32),
                    label=mk(S + seg_cap, i32), n_seg=mk(1, i64))

    def phg(self, cfg, pts, dirs, seeds, normals, valid=None, seg_cap=None, outputs=None, cut=True):
        """The Parallel Hair Growing consumer (hair_fuse_phg).  cfg: hf_phg_cfg; inputs numpy arrays
        or CUDA tensors (one kind).  Outputs (of the inputs' kind) are `outputs` (from phg_outputs) or
        allocated here: a dict like the oracle's (occ, ori, crowd, gverts, glen, gstop, gtan, sverts,
        slen, svox, stan, label, n_seg), the segment arrays cut to the K segments unless cut=False."""
        ins = [_ptr_kind(x) for x in (pts, dirs, valid, seeds, normals)]
        kind = _same_kind(*[q[1] for q in ins])
        N, S = int(pts.shape[0]), int(seeds.shape[0])
        if outputs is None:
            cap = cfg.nx * cfg.ny * cfg.nz if seg_cap is None else int(seg_cap)
            outputs = self.phg_outputs(cfg, S, cap, pts.device if kind == HF_DEVICE else None)
        o = dict(outputs)
        cap = int(o["slen"].shape[0])
        ptr = {k: _ptr_kind(v)[0] for k, v in o.items()}
        out = hf_phg_out(ptr["occ"], ptr["ori"], ptr["crowd"], ptr["gverts"], ptr["glen"], ptr["gstop"], ptr["gtan"],
                         cap, ptr["sverts"], ptr["slen"], ptr["svox"], ptr["stan"], ptr["label"], ptr["n_seg"])
        self._c(hair_fuse_phg(self.h, ctypes.byref(cfg), N, ins[0][0], ins[1][0], ins[2][0], S, ins[3][0], ins[4][0],
                              ctypes.byref(out), kind))
        if kind == HF_DEVICE:
            self.sync()
        if cut:
            K = int(o["n_seg"][0])
            for k in ("sverts", "slen", "svox", "stan"):
                o[k] = o[k][:K]
            o["label"] = o["label"][:S + K]
        return o

    def gabor(self, images, theta_out=None, conf_out=None, asynchronous=False, **kw):
        """Orientation and confidence maps (hair_fuse_gabor) of images (V, H, W) f32, numpy or CUDA tensor;
        outputs allocated like the input unless given.  asynchronous=True (pinned torch CPU tensors,
        HF_HOST_ASYNC): copies and kernel are queued on the context's stream and the call returns at
        once; keep the buffers until the stream has consumed them."""
        V, H, W = (int(x) for x in images.shape)
        if theta_out is None:
            if isinstance(images, np.ndarray):
                theta_out, conf_out = np.empty((V, H, W), np.float32), np.empty((V, H, W), np.float32)
            else:
                import torch
                theta_out = torch.empty((V, H, W), dtype=torch.float32, device=images.device)
                conf_out = torch.empty((V, H, W), dtype=torch.float32, device=images.device)
        ptrs = [_ptr_kind(x) for x in (images, theta_out, conf_out)]
        kind = _same_kind(*[q[1] for q in ptrs])
        if asynchronous:
            if kind != HF_HOST or not all(getattr(x, "is_pinned", lambda: False)() for x in (images, theta_out, conf_out)):
                raise ValueError("asynchronous Gabor maps take pinned torch CPU tensors")
            kind = HF_HOST_ASYNC
        self._c(hair_fuse_gabor(self.h, ctypes.byref(gabor_cfg(**kw)), V, H, W, *[q[0] for q in ptrs], kind))
        return theta_out, conf_out

    def eval_costs(self, dirs, cost_out):
        """Costs (N,M) of the directions dirs (N,M,3)."""
        pd, k1, _ = _ptr_kind(dirs)
        pc, k2, _ = _ptr_kind(cost_out)
        self._c(hair_fuse_eval_costs(self.h, dirs.shape[1], pd, pc, _same_kind(k1, k2)))

    def sync(self):
        self._c(hair_fuse_sync(self.h))

    def profile(self, enable=True):
        self._c(hair_fuse_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (launches, total_ms)} of the launches since profile(True)."""
        buf = (hf_kernel_time * 64)()
        n = hair_fuse_profile_read(self.h, buf, 64)
        if n < 0:
            self._c(n)
        return {buf[q].name.decode(): (buf[q].launches, buf[q].total_ms) for q in range(min(n, 64))}

    def work(self):
        """(point, view) pairs in the view sets at the last fuse / eval call."""
        w = _ll()
        self._c(hair_fuse_work(self.h, ctypes.byref(w)))
        return w.value

    def stats(self):
        b, l = _ll(), _ll()
        self._c(hair_fuse_stats(self.h, ctypes.byref(b), ctypes.byref(l)))
        return {"device_bytes": b.value, "launches": l.value}


def _mlp_check(rc, h):
    if rc != HF_OK:
        msg = hair_fuse_mlp_last_error(h)
        raise HairFuseError(rc, msg.decode() if msg else "")
    return rc


class ProposalNet:
    """The learned proposal network (64 -> 256 -> 256 -> 3 MLP on the tensor cores)."""

    def __init__(self, max_batch=8192, stream=None):
        h = _vp()
        _check(hair_fuse_mlp_create(ctypes.byref(h), max_batch, current_stream_handle() if stream is None else stream))
        self.h = h
        self.max_batch = max_batch

    @staticmethod
    def param_count():
        return int(hair_fuse_mlp_param_count())

    def close(self):
        if getattr(self, "h", None):
            hair_fuse_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _c(self, rc):
        return _mlp_check(rc, self.h)

    def init(self, seed):
        self._c(hair_fuse_mlp_init(self.h, seed))

    def get_params(self):
        out = np.empty(self.param_count(), np.float32)
        self._c(hair_fuse_mlp_get_params(self.h, out.ctypes.data, HF_HOST))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.param_count()
        self._c(hair_fuse_mlp_set_params(self.h, p.ctypes.data, HF_HOST))

    def train(self, X, T, batch, steps, lr, seed, use_graph=True):
        """X (n, 64) bf16 CUDA tensor, T (n, 3) float32 CUDA tensor; returns the per-step losses."""
        losses = np.zeros(max(steps, 1), np.float32)
        self._c(hair_fuse_mlp_train(self.h, X.data_ptr(), T.data_ptr(), X.shape[0], batch, steps, lr, seed,
                                    1 if use_graph else 0, losses.ctypes.data))
        return losses[:steps]

    def grads(self, X, T, batch, seed):
        """(gradients, loss, batch features uint16 (batch, 64), batch targets) of the next batch."""
        g = np.empty(self.param_count(), np.float32)
        loss = np.zeros(1, np.float32)
        xb = np.empty((batch, 64), np.uint16)
        tb = np.empty((batch, 3), np.float32)
        self._c(hair_fuse_mlp_grads(self.h, X.data_ptr(), T.data_ptr(), X.shape[0], batch, seed, g.ctypes.data,
                                    loss.ctypes.data, xb.ctypes.data, tb.ctypes.data))
        return g, float(loss[0]), xb, tb

    def forward(self, X, out=None, raw=False):
        """Proposals (n, 3) for features X (n, 64) bf16 (CUDA tensor or uint16 numpy array); with
        raw=True the head's outputs before the normalisation."""
        fn = hair_fuse_mlp_forward_raw if raw else hair_fuse_mlp_forward
        n = X.shape[0]
        if isinstance(X, np.ndarray):
            out = np.empty((n, 3), np.float32) if out is None else out
            self._c(fn(self.h, np.ascontiguousarray(X).ctypes.data, n, out.ctypes.data, HF_HOST))
            return out
        import torch
        out = torch.empty((n, 3), device=X.device) if out is None else out
        self._c(fn(self.h, X.data_ptr(), n, out.data_ptr(), HF_DEVICE))
        return out

    def save(self, path):
        self._c(hair_fuse_mlp_save(self.h, str(path).encode()))

    def load(self, path):
        self._c(hair_fuse_mlp_load(self.h, str(path).encode()))


def _features(self, out):
    """Proposal-network features (N, 64) bf16 of the uploaded points into out (CUDA bf16/uint16
    tensor or uint16 numpy array)."""
    p, kind, _ = _ptr_kind(out)
    self._c(hair_fuse_features(self.h, p, kind))
    return out


def _fuse_learned(self, net, dir_out, cost_out=None, idx_out=None, status_out=None, T_short=2, alpha_short=0.16,
                  tau=0.5, count_fallback=True):
    """Learned fusion into caller buffers; returns the number of fallback points (or None)."""
    ptrs = [_ptr_kind(x) for x in (dir_out, cost_out, idx_out, status_out)]
    kind = _same_kind(*[q[1] for q in ptrs])
    nf = _i(0)
    self._c(hair_fuse_fuse_learned(self.h, net.h, T_short, alpha_short, tau, *[q[0] for q in ptrs],
                                   ctypes.byref(nf) if count_fallback else None, kind))
    return nf.value if count_fallback else None


def _learned_work(self):
    """(point, view) pairs of the fallback points and of the accepted proposals, last learned fusion."""
    fb, ac = _ll(0), _ll(0)
    self._c(hair_fuse_learned_work(self.h, ctypes.byref(fb), ctypes.byref(ac)))
    return dict(fallback_point_views=fb.value, accepted_point_views=ac.value)


HairFuse.features = _features
HairFuse.fuse_learned = _fuse_learned
HairFuse.learned_work = _learned_work


class hf_batch_cfg(ctypes.Structure):
    _fields_ = [("T_short", ctypes.c_int), ("alpha_short", ctypes.c_float), ("tau", ctypes.c_float),
                ("autotune", ctypes.c_int), ("cta_threads", ctypes.c_int), ("order", ctypes.c_int)]


class Batch:
    """Batched fusion of several HairFuse contexts (plain, or learned with a ProposalNet): one
    persistent launch per stage over all scenes, replayed as one CUDA graph."""

    def __init__(self, scenes, net=None, T_short=2, alpha_short=0.16, tau=0.5, autotune=True, cta_threads=0,
                 order=0, stream=None):
        self.scenes = list(scenes)
        self.net = net
        cfg = hf_batch_cfg(T_short, alpha_short, tau, 1 if autotune else 0, cta_threads, order)
        arr = (_vp * len(self.scenes))(*[sc.h for sc in self.scenes])
        h = _vp()
        rc = hair_fuse_batch_create(ctypes.byref(h), arr, len(self.scenes), net.h if net is not None else None,
                                    ctypes.byref(cfg), current_stream_handle() if stream is None else stream)
        if rc != HF_OK:
            msg = hair_fuse_batch_last_error(None)
            raise HairFuseError(rc, msg.decode() if msg else "")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            hair_fuse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, rc):
        if rc != HF_OK:
            msg = hair_fuse_batch_last_error(self.h)
            raise HairFuseError(rc, msg.decode() if msg else "")
        return rc

    def set_outputs(self, scene, dir_out, cost_out=None, idx_out=None, status_out=None):
        """CUDA tensors of scene `scene`: dir (N, 3) f32, cost (N,) f32, idx (N,) i32, status (N,) u8."""
        ptr = [x.data_ptr() if x is not None else None for x in (dir_out, cost_out, idx_out, status_out)]
        self._c(hair_fuse_batch_set_outputs(self.h, scene, *ptr))

    def run(self, use_graph=True):
        self._c(hair_fuse_batch_run(self.h, 1 if use_graph else 0))

    def sync(self):
        self._c(hair_fuse_batch_sync(self.h))

    def latency_ms(self):
        out = np.zeros(len(self.scenes), np.float64)
        self._c(hair_fuse_batch_latency(self.h, out.ctypes.data))
        return out

    def fallbacks(self):
        out = np.zeros(len(self.scenes), np.int32)
        self._c(hair_fuse_batch_fallbacks(self.h, out.ctypes.data))
        return out

    def tuning(self):
        out = np.zeros(2, np.int32)
        self._c(hair_fuse_batch_tuning(self.h, out.ctypes.data))
        cached = hair_fuse_batch_tuned_from_cache(self.h)
        if cached < 0:
            self._c(cached)
        return dict(cta_threads=int(out[0]),
                    order={1: "heaviest first", 2: "as given", 3: "lightest first"}.get(int(out[1]), "?"),
                    cached=bool(cached))

    def profile_run(self):
        """One eager run with events between the stages: {stage: (launches, ms)}."""
        recs = (hf_kernel_time * 16)()
        n = hair_fuse_batch_profile_run(self.h, recs, 16)
        if n < 0:
            self._c(n)
        return {recs[q].name.decode(): (recs[q].launches, recs[q].total_ms) for q in range(min(n, 16))}

    def stats(self):
        """launches so far; (point, view) pairs of all points, of the fallback points and of the
        accepted proposals (last run)."""
        l, pv, fpv, apv = _ll(0), _ll(0), _ll(0), _ll(0)
        self._c(hair_fuse_batch_stats(self.h, ctypes.byref(l), ctypes.byref(pv), ctypes.byref(fpv), ctypes.byref(apv)))
        return dict(launches=l.value, point_views=pv.value, fallback_point_views=fpv.value,
                    accepted_point_views=apv.value)
