"""The inference kernel's GELU (gelu2 in csrc/fcc_mlp.cu) is a fitted form of
the exact-erf GELU: its constants must be the ones csrc/fit_gelu.py fits, and
that form, evaluated in FP32 in the kernel's order, must stay within its stated
error of x Phi(x)."""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2204_13622_gb300", "csrc")


def _fit_module():
    pytest.importorskip("scipy")
    spec = importlib.util.spec_from_file_location("fit_gelu", os.path.join(CSRC, "fit_gelu.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _kernel_constants():
    src = open(os.path.join(CSRC, "fcc_mlp.cu")).read()
    body = src[src.index("__device__ __forceinline__ f2 gelu2"):]
    body = body[:body.index("kHalfLog2e")]
    vals = [float(v) for v in re.findall(r"pk\(([-0-9.e+]+)f, \1f\)", body)]
    # the first pk() pair is (0.3, 0.3), then (1, 1); then c7 .. c0 in Horner order
    assert vals[:2] == [0.3, 1.0]
    return np.array(vals[2:][::-1])


def test_kernel_constants_are_the_fit():
    m = _fit_module()
    c = m.fit()
    k = _kernel_constants()
    assert k.size == m.DEG + 1
    assert np.allclose(k, c, rtol=1e-8, atol=1e-12)


def test_fitted_gelu_error_bound():
    m = _fit_module()
    from scipy.special import erfc
    c = m.fit()
    x = np.linspace(-12.0, 12.0, 400_001)
    exact = 0.5 * x * erfc(-x / np.sqrt(2.0))
    err = np.abs(m.gelu_fp32(x, c).astype(np.float64) - exact)
    assert err.max() <= 5e-7
    assert (err / np.maximum(1.0, np.abs(x))).max() <= 1.5e-7
    # special values: GELU(0) = 0, and GELU(x) - x / 2 is even: GELU(x) - GELU(-x) = x
    assert m.gelu_fp32(np.array([0.0]), c)[0] == 0.0
    xs = np.array([0.5, 1.0, 2.0, 3.0])
    g_pos, g_neg = m.gelu_fp32(xs, c).astype(np.float64), m.gelu_fp32(-xs, c).astype(np.float64)
    assert np.allclose(g_pos - g_neg, xs, atol=1e-6)  # GELU(x) - GELU(-x) = x
