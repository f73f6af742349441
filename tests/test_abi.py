"""The C-ABI library loads and exports every entry point its header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(hair_fuse_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hair_fuse_create", "hair_fuse_upload_views", "hair_fuse_upload_points",
                     "hair_fuse_fuse_directions", "hair_fuse_destroy", "hair_fuse_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2604_05794_b300 as hf
    lib = ctypes.CDLL(hf.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_exposes_c_names():
    import paper_2604_05794_b300 as hf
    for n in declared_functions():
        assert hasattr(hf, n), n


def test_create_argument_errors_without_touching_cuda():
    import paper_2604_05794_b300 as hf
    h = ctypes.c_void_p()
    for cfg in (hf.hf_config(0, 5, 4, 0, 0.0, 0), hf.hf_config(32, 99, 4, 0, 0.0, 0),
                hf.hf_config(32, 5, 99, 0, 0.0, 0), hf.hf_config(32, 5, 4, 99, 0.0, 0)):
        assert hf.hair_fuse_create(ctypes.byref(h), ctypes.byref(cfg), None) == hf.HF_ERR_INVALID_ARG
        assert hf.hair_fuse_last_error(None)
    assert hf.hair_fuse_create(None, None, None) == hf.HF_ERR_INVALID_ARG


def test_no_gpu_reports_cuda_error_instead_of_crashing():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2604_05794_b300 as hf
    with pytest.raises(hf.HairFuseError):
        hf.HairFuse(32, 5, 4, stream=None)
