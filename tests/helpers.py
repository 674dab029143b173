"""Comparison rules shared by the GPU parity tests."""
import numpy as np

VALUE_RTOL = 1e-4   # |y_gpu - y_oracle| <= 1e-4 * max_tau |y_oracle| per pair-frame
TIE_GAP = 4e-6      # argmax must match wherever the oracle's top-2 gap exceeds this


def check_corr(y_gpu, y_or, rtol=VALUE_RTOL):
    scale = np.maximum(np.abs(y_or).max(axis=-1, keepdims=True), 1e-30)
    err = np.abs(y_gpu - y_or) / scale
    assert err.max() <= rtol, f"max relative correlation error {err.max():.3e} > {rtol}"
    return float(err.max())


def check_argmax(idx_gpu, y_or, tie_gap=TIE_GAP):
    """Bit-exact argmax where the oracle's maximum is clear; elsewhere the GPU
    index must be one of the oracle's near-tied maxima.  Returns #near-ties."""
    y_or = np.asarray(y_or)
    idx_or = np.argmax(y_or, axis=-1)
    srt = np.sort(y_or, axis=-1)
    top = srt[..., -1]
    scale = np.maximum(np.abs(y_or).max(axis=-1), 1e-30)
    gap = (top - srt[..., -2]) / scale
    clear = gap > tie_gap
    bad = clear & (idx_gpu != idx_or)
    assert not bad.any(), f"{bad.sum()} clear argmax mismatches"
    amb = ~clear
    if amb.any():
        yg = np.take_along_axis(y_or, idx_gpu[..., None].astype(np.int64), -1)[..., 0]
        assert np.all((top[amb] - yg[amb]) <= tie_gap * scale[amb] * 2)
    return int(amb.sum())
