"""BF16 / FP16 precision forms (tensor-core projection) of the FCC path.

Two kinds of checks:
* plumbing: a numpy emulation of exactly what the tensor-core path computes --
  unit phases rounded to FP16, cross spectra and folds in FP32, projection
  operands rounded to BF16 / FP16, products accumulated exactly -- must match
  the GPU correlation to 2e-5 of each pair-frame's peak, on spectra whose unit
  phases are +-1 / +-j so that every one of those roundings is exact (layout or
  descriptor mistakes give O(1) errors);
* accuracy against the FP64 oracle: the argmax agreement rate and the peak
  error, which are the reported figures of merit of the precision forms.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_13622_gb300 import workloads  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding


def _round(x, prec):
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    t = t.to(torch.bfloat16 if prec == "bf16" else torch.float16)
    return t.to(torch.float64).numpy()


def emulate(plan, X, prec):
    """Correlation the tensor-core path computes, in float64 after the roundings."""
    Pe, Po, Ue, Uo = plan.bases()
    N, Q = plan.N, plan.Q
    X = X.astype(np.complex64)
    mag = np.abs(X).astype(np.float32)
    u = np.where(mag > 0, X / np.where(mag > 0, mag, 1), 0).astype(np.complex64)
    u = (_round(u.real, "fp16") + 1j * _round(u.imag, "fp16"))
    T, M, Bn = X.shape
    pe = _round(Pe[:, :Q], prec)
    po = _round(Po, prec)
    peq = Pe[:, Q].astype(np.float32).astype(np.float64)
    phi = np.exp(1j * np.pi * plan.taus() / 2)
    y = np.empty((T, plan.P, plan.I))
    p = 0
    for i in range(M):
        for j in range(i + 1, M):
            a = (u[:, i, :Q] * np.conj(u[:, j, :Q])).astype(np.complex64)
            b = (u[:, i, N // 2:Q:-1] * np.conj(u[:, j, N // 2:Q:-1])).astype(np.complex64)
            xs, xd = a + b, a - b
            xs = _round(xs.real, prec) + 1j * _round(xs.imag, prec)
            xd = _round(xd.real, prec) + 1j * _round(xd.imag, prec)
            lone = (u[:, i, Q] * np.conj(u[:, j, Q]))
            ze = xs @ pe.T + lone[:, None] * peq[None, :]
            zo = xd @ po.T
            y[:, p] = 2 * np.real(phi * (ze @ Ue.T + 1j * (zo @ Uo.T)))
            p += 1
    return y


def _exact_phase_spectra(T, M, N, seed):
    """Spectra whose unit phases are exactly +-1 or +-j (magnitudes powers of two):
    every rounding of the tensor-core pipeline is then exact."""
    rng = np.random.default_rng(seed)
    ph = np.array([1, 1j, -1, -1j])[rng.integers(0, 4, (T, M, N // 2 + 1))]
    mag = 2.0 ** rng.integers(-3, 4, (T, M, N // 2 + 1))
    return (ph * mag).astype(np.complex64)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("wl,T", [("CIRCLE8", 37), ("GRID16", 5), ("SQUARE4", 61)])
def test_tensor_core_matches_emulation(B, prec, wl, T):
    w = getattr(workloads, wl)
    X = _exact_phase_spectra(T, w.M, w.N, seed=T)
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, prec=prec)
    out = plan.tdoa(torch.from_numpy(X).cuda(), corr=True, tau_hat=True, coeffs=True)
    plan.sync()
    y = emulate(plan, X, prec)
    g = out["corr"].cpu().numpy()
    err = np.abs(g - y) / np.abs(y).max(-1, keepdims=True)
    assert err.max() < 2e-5, f"max rel err {err.max():.3e}"
    gi = out["lag_idx"].cpu().numpy()
    assert np.array_equal(gi, np.argmax(g, -1))
    plan.close()


@pytest.mark.parametrize("prec,min_agree,max_peak_err", [("bf16", 0.97, 3e-2), ("fp16", 0.99, 5e-3)])
def test_precision_vs_oracle(B, prec, min_agree, max_peak_err):
    from oracle import oracle as O
    w = workloads.GRID16
    X = w.spectra(T=48, seed=3).numpy()
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, prec=prec)
    out = plan.tdoa(torch.from_numpy(X).cuda(), corr=True)
    plan.sync()
    ref = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
    idx, peak, _, y = O.tdoa(X, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"].cpu().numpy()
    agree = float((gi == idx).mean())
    scale = np.abs(y).max(-1)
    perr = float(np.median(np.abs(out["peak"].cpu().numpy() - peak) / scale))
    print(f"{prec}: argmax agreement {agree:.4f}, median peak error {perr:.2e}")
    assert agree >= min_agree
    assert perr <= max_peak_err
    plan.close()


def test_unsupported_sizes_are_rejected(B):
    # the tensor-core path needs N >= 128 and an even number of mics
    with pytest.raises(B.FccError) as e:
        B.Plan(4, 16000.0, 64, 4, tau_max=2, prec="bf16")
    assert e.value.status == 2
    with pytest.raises(B.FccError):
        B.Plan(5, 16000.0, 512, 4, tau_max=3, prec="fp16")


@pytest.mark.parametrize("prec,min_agree,max_peak_err", [("bf16", 0.995, 3e-4), ("fp16", 0.999, 5e-5)])
def test_grid16_full_size_sampled(B, prec, min_agree, max_peak_err):
    """The 16-mic grid at its full 2^18 frames in one call (the bench's launch):
    frames sampled across the run (first, last, random) against the FP64
    oracle, argmax agreement on clear peaks and the median peak error.  On this
    grid (97 lag steps) the reconstruction itself runs on the tensor cores."""
    from oracle import oracle as O
    w = workloads.GRID16
    X = w.spectra(device="cuda", seed=2)
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, prec=prec)
    out = plan.tdoa(X)
    plan.sync()
    rng = np.random.default_rng(1)
    frames = np.unique(np.concatenate([[0, 1, w.T - 1], rng.integers(0, w.T, 96)]))
    sel = torch.from_numpy(frames).cuda()
    Xs = X[sel].cpu().numpy()
    ref = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
    idx, peak, _, y = O.tdoa(Xs, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"][sel].cpu().numpy()
    srt = np.sort(y, axis=-1)
    scale = np.abs(y).max(-1)
    clear = (srt[..., -1] - srt[..., -2]) > 1e-3 * scale
    agree = float((gi == idx)[clear].mean())
    perr = float(np.median(np.abs(out["peak"][sel].cpu().numpy() - peak) / scale))
    print(f"{prec}: {int(clear.sum())} clear pair-frames, agreement {agree:.4f}, median peak error {perr:.2e}")
    assert agree >= min_agree
    assert perr <= max_peak_err
    plan.close()
    del X
    torch.cuda.empty_cache()
