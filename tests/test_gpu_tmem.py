"""GPU parity of the tensor-memory engine (FCC_ENGINE_TENSOR_TMEM): the Eq. 9
projection as tcgen05 MMAs whose A operand is written into tensor memory.

* FP32 plans (TF32 with a two-term split of both operands) are held to the
  FP32 path's tolerances against the FP64 oracle (tests/helpers.py):
  correlation values within 1e-4 of each pair-frame's max |y|, the argmax
  bit-exact wherever the oracle's top-2 gap is clear;
* BF16 / FP16 plans: a numpy emulation of exactly what the kernel computes
  (FP32 unit phases and cross spectra, the two bins of every record rounded
  to the operand type, the fold applied by the rounded B operand, exact
  accumulation) on spectra whose roundings are all exact, then the argmax
  agreement and peak error against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_argmax, check_corr  # noqa: E402

from paper_2204_13622_gb300 import synth, workloads  # noqa: E402

ENGINE = "tensor_tmem"


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _random_spectra(T, M, N, seed, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((T, M, N // 2 + 1)) + 1j * rng.standard_normal((T, M, N // 2 + 1)))
    if zero_frac:
        X[rng.random(X.shape) < zero_frac] = 0
    return X.astype(np.complex64)


def _run_and_compare(B, O, X, N, L, den, M, K=0, fs=16000.0):
    plan = B.Plan(M, fs, N, den, tau_max=L, K=K, engine=ENGINE)
    assert plan.engine == ENGINE
    out = plan.tdoa(torch.from_numpy(X).cuda(), tau_hat=True, coeffs=True, corr=True)
    plan.sync()
    ref = O.Basis(N, L, den, K=plan.K)
    idx, peak, tau, y = O.tdoa(X, ref.WK, ref.taus, ref.delta, want_y=True)
    corr = out["corr"].cpu().numpy()
    check_corr(corr, y)
    gi = out["lag_idx"].cpu().numpy()
    check_argmax(gi, y)
    gp = out["peak"].cpu().numpy()
    assert np.array_equal(gp, np.take_along_axis(corr, gi[..., None].astype(np.int64), -1)[..., 0])
    same = gi == idx
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(gp - peak)[same] <= 1e-4 * scale[same])
    gt = out["tau_hat"].cpu().numpy()
    assert np.all(np.abs(gt - tau)[same] <= 2e-3)
    # the coefficients reproduce the correlation through the plan's bases
    Pe, Po, Ue, Uo = plan.bases()
    KE, KO = plan.K_even, plan.K_odd
    c = out["coeffs"].cpu().numpy().astype(np.float64)
    ze = c[..., :KE] + 1j * c[..., KE:2 * KE]
    zo = c[..., 2 * KE:2 * KE + KO] + 1j * c[..., 2 * KE + KO:]
    phi = np.exp(1j * np.pi * plan.taus() / 2)
    check_corr(2 * np.real(phi * (ze @ Ue.T + 1j * (zo @ Uo.T))), y)
    plan.close()
    return out


def test_small_square_parity(B, O):
    rec = synth.config_small_square(1)
    out = _run_and_compare(B, O, rec.spectra, 512, 3, 4, 4)
    assert out["lag_idx"].shape == (61, 6)


@pytest.mark.parametrize("M,N,den,L,T", [
    (2, 128, 4, 2, 77),
    (4, 256, 4, 3, 50),
    (6, 256, 4, 3, 37),
    (8, 512, 4, 5, 130),
    (10, 512, 4, 5, 11),
    (12, 512, 2, 4, 20),
    (14, 1024, 4, 6, 3),
    (16, 1024, 8, 12, 9),
])
def test_random_spectra_parity(B, O, M, N, den, L, T):
    X = _random_spectra(T, M, N, seed=M * 1000 + N + T)
    _run_and_compare(B, O, X, N, L, den, M)


def test_fixed_rank_and_ragged_tiles(B, O):
    # K below the energy rule, T not a multiple of the 4-frame tile, several tiles per CTA
    X = workloads.CIRCLE8.spectra(T=1203, seed=9).numpy()
    _run_and_compare(B, O, X, 512, 5, 4, 8, K=5)


def test_zero_bins_and_zero_frames(B, O):
    X = _random_spectra(24, 8, 512, seed=4, zero_frac=0.2)
    X[3] = 0
    X[5, 2] = 0
    out = _run_and_compare(B, O, X, 512, 5, 4, 8)
    assert np.all(out["lag_idx"][3].cpu().numpy() == 0)
    assert np.all(out["peak"][3].cpu().numpy() == 0)


def test_pure_delays_on_grid(B):
    N, M = 512, 2
    plan = B.Plan(M, 16000.0, N, 4, tau_max=3, engine=ENGINE)
    f = np.arange(N // 2 + 1)
    rng = np.random.default_rng(1)
    S = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
    Ds = np.arange(-3, 3.25, 0.25)
    X = np.stack([np.stack([S, S * np.exp(-2j * np.pi * f * D / N)]) for D in Ds]).astype(np.complex64)
    out = plan.tdoa(torch.from_numpy(X).cuda())
    plan.sync()
    got = plan.taus()[out["lag_idx"][:, 0].cpu().numpy()]
    assert np.array_equal(got, -Ds)
    assert np.all(np.abs(out["tau_hat"][:, 0].cpu().numpy() + Ds) < 0.05)
    plan.close()


def test_nonfinite_input_is_reported(B):
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3, engine=ENGINE)
    X = torch.from_numpy(_random_spectra(8, 4, 512, seed=2)).cuda()
    X[3, 1, 7] = complex(float("nan"), 0.0)
    plan.tdoa(X)
    with pytest.raises(B.FccError) as ei:
        plan.sync()
    assert ei.value.status == 6
    plan.tdoa(torch.from_numpy(_random_spectra(8, 4, 512, seed=3)).cuda())
    plan.sync()
    plan.close()


def test_expired_wait_reports_timeout_and_context_survives(B):
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5, engine=ENGINE)
    X = torch.from_numpy(_random_spectra(4000, 8, 512, seed=1)).cuda()
    ref = plan.tdoa(X)
    plan.sync()
    ref = {k: v.clone() for k, v in ref.items()}
    try:
        B.debug_set("wait_cycles", 200000)  # about 0.1 ms
        B.debug_set("withhold_copy", 1)
        plan.tdoa(X)
        with pytest.raises(B.FccError) as e:
            plan.sync()
        assert e.value.status == 5
    finally:
        B.debug_set("wait_cycles", 0)
        B.debug_set("withhold_copy", 0)
    out = plan.tdoa(X)
    plan.sync()
    for k in ref:
        assert torch.equal(out[k], ref[k])
    plan.close()


def test_engine_selection(B):
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5)
    plan.set_engine(ENGINE)
    assert plan.engine == ENGINE
    plan.set_engine("cuda_cores")
    assert plan.engine == "cuda_cores"
    with pytest.raises(B.FccError) as e:
        plan.set_engine("tensor_smem")  # 16-bit forms only
    assert e.value.status == 2
    plan.close()
    odd = B.Plan(5, 16000.0, 512, 4, tau_max=3)  # odd M: no tensor-memory kernel
    with pytest.raises(B.FccError) as e:
        odd.set_engine(ENGINE)
    assert e.value.status == 2
    odd.close()


def test_same_results_as_cuda_cores_within_fp32_rounding(B):
    w = workloads.CIRCLE8
    X = w.spectra(T=4096, seed=5).cuda()
    a = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, engine="cuda_cores")
    b = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, engine=ENGINE)
    oa = a.tdoa(X, corr=True)
    ob = b.tdoa(X, corr=True)
    a.sync()
    b.sync()
    ya, yb = oa["corr"].cpu().numpy(), ob["corr"].cpu().numpy()
    err = np.abs(ya - yb) / np.abs(ya).max(-1, keepdims=True)
    assert err.max() < 1e-5, err.max()
    a.close()
    b.close()


# --------------------------------------------------------------------------
# 16-bit operands
# --------------------------------------------------------------------------
def _round(x, prec):
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    t = t.to(torch.bfloat16 if prec == "bf16" else torch.float16)
    return t.to(torch.float64).numpy()


def emulate(plan, X, prec):
    """The correlation the 16-bit tensor-memory kernel computes, in float64:
    unit phases and cross spectra in FP32, a = R(f) and b = R(N/2 - f) rounded
    to the operand type, the fold and the projection by the rounded bases."""
    Pe, Po, Ue, Uo = plan.bases()
    N, Q = plan.N, plan.Q
    X = X.astype(np.complex64)
    mag = np.abs(X).astype(np.float32)
    u = np.where(mag > 0, X / np.where(mag > 0, mag, 1), 0).astype(np.complex64)
    T, M, _ = X.shape
    pe = _round(Pe, prec)        # [KE, Q + 1], bin N/4 included
    po = _round(Po, prec)        # [KO, Q]
    phi = np.exp(1j * np.pi * plan.taus() / 2)
    y = np.empty((T, plan.P, plan.I))
    p = 0
    for i in range(M):
        for j in range(i + 1, M):
            a = (u[:, i, :Q + 1] * np.conj(u[:, j, :Q + 1])).astype(np.complex64)
            b = (u[:, i, N // 2:Q:-1] * np.conj(u[:, j, N // 2:Q:-1])).astype(np.complex64)
            a = _round(a.real, prec) + 1j * _round(a.imag, prec)
            b = _round(b.real, prec) + 1j * _round(b.imag, prec)
            ze = a @ pe.T + b @ pe[:, :Q].T
            zo = a[:, :Q] @ po.T - b @ po.T
            y[:, p] = 2 * np.real(phi * (ze @ Ue.T + 1j * (zo @ Uo.T)))
            p += 1
    return y


def _exact_phase_spectra(T, M, N, seed):
    rng = np.random.default_rng(seed)
    ph = np.array([1, 1j, -1, -1j])[rng.integers(0, 4, (T, M, N // 2 + 1))]
    mag = 2.0 ** rng.integers(-3, 4, (T, M, N // 2 + 1))
    return (ph * mag).astype(np.complex64)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("wl,T", [("CIRCLE8", 37), ("GRID16", 5), ("SQUARE4", 61)])
def test_16bit_matches_emulation(B, prec, wl, T):
    w = getattr(workloads, wl)
    X = _exact_phase_spectra(T, w.M, w.N, seed=T)
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, prec=prec, engine=ENGINE)
    out = plan.tdoa(torch.from_numpy(X).cuda(), corr=True, tau_hat=True, coeffs=True)
    plan.sync()
    y = emulate(plan, X, prec)
    g = out["corr"].cpu().numpy()
    err = np.abs(g - y) / np.abs(y).max(-1, keepdims=True)
    assert err.max() < 2e-5, f"max rel err {err.max():.3e}"
    assert np.array_equal(out["lag_idx"].cpu().numpy(), np.argmax(g, -1))
    plan.close()


@pytest.mark.parametrize("prec,min_agree,max_peak_err", [("bf16", 0.97, 3e-2), ("fp16", 0.99, 5e-3)])
def test_16bit_vs_oracle(B, O, prec, min_agree, max_peak_err):
    w = workloads.GRID16
    X = w.spectra(T=48, seed=3).numpy()
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, prec=prec, engine=ENGINE)
    out = plan.tdoa(torch.from_numpy(X).cuda(), corr=True)
    plan.sync()
    ref = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
    idx, peak, _, y = O.tdoa(X, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"].cpu().numpy()
    agree = float((gi == idx).mean())
    perr = float(np.median(np.abs(out["peak"].cpu().numpy() - peak) / np.abs(y).max(-1)))
    print(f"{prec}: argmax agreement {agree:.4f}, median peak error {perr:.2e}")
    assert agree >= min_agree
    assert perr <= max_peak_err
    plan.close()
