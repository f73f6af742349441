"""The inference GELU's coefficients (hf_gemm.cu) are the ones the committed generator
(csrc/gen_gelu_poly.py) fits, and the generator's FP32 emulation of the kernel's operation sequence
keeps the stated bound |gelu(x) - x Phi(x)| <= 4.1e-7 |x| against FP64 erf.  CPU only; the GPU test
(test_gpu_mlp.test_inference_gelu_error_bound) checks the kernel itself against the same bound."""
import os
import re
import sys

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_05794_b300", "csrc")


def _kernel_coefficients():
    with open(os.path.join(CSRC, "hf_gemm.cu")) as f:
        src = f.read()
    m = re.search(r"kGeluC\[(\d+)\]\s*=\s*\{([^}]*)\}", src)
    assert m, "kGeluC initialiser not found"
    vals = [float(t.strip().rstrip("f")) for t in m.group(2).split(",") if t.strip()]
    assert len(vals) == int(m.group(1))
    return np.array(vals, np.float32)


def test_kernel_coefficients_come_from_the_generator():
    sys.path.insert(0, CSRC)
    try:
        import gen_gelu_poly as g
    finally:
        sys.path.pop(0)
    fitted = g.fit()
    # the same fit up to the last FP32 bit (the least-squares solver's rounding may differ by host)
    kc = _kernel_coefficients()
    assert np.allclose(fitted, kc, rtol=3e-7, atol=0.0), (fitted, kc)
    assert g.bound(kc) <= 4.1e-7


def test_emulated_sequence_special_points():
    sys.path.insert(0, CSRC)
    try:
        import gen_gelu_poly as g
    finally:
        sys.path.pop(0)
    c = _kernel_coefficients()
    x = np.array([0.0, 1e-30, -1e-30, 1.0, -1.0, 5.0, -5.0, 30.0, -30.0], np.float32)
    y = g.gelu_fp32(x, c).astype(np.float64)
    from scipy.special import erf
    xd = x.astype(np.float64)
    ref = 0.5 * xd * (1.0 + erf(xd / np.sqrt(2.0)))
    assert y[0] == 0.0 and y[1] == np.float32(0.5e-30) and y[2] == np.float32(-0.5e-30)
    assert np.all(np.abs(y - ref) <= 4.1e-7 * np.abs(xd))
