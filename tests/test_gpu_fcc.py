"""GPU parity of the FCC C-ABI path against the FP64 oracle.

Every call goes through libfcc_gb300.so (ctypes); the oracle is the plain
FP64 C code in oracle/.  Tolerances (see tests/helpers.py): correlation values
within 1e-4 of the pair-frame's max |y|; argmax bit-exact wherever the
oracle's top-2 gap exceeds 4e-6 of max |y|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_argmax, check_corr  # noqa: E402

from paper_2204_13622_gb300 import synth, workloads  # noqa: E402


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


def _plan_WK(plan):
    """Rebuild the complex rank-K operator the plan's folded bases implement:
    W_K = diag(exp(j pi tau / 2)) (Ue Pe F_s + j Uo Po F_d), F_s / F_d the Eq. 8 folds."""
    Pe, Po, Ue, Uo = plan.bases()
    N, Q, B = plan.N, plan.Q, plan.B
    Fs = np.zeros((Q + 1, B))
    Fd = np.zeros((Q, B))
    for f in range(Q):
        Fs[f, f] = Fs[f, N // 2 - f] = 1
        Fd[f, f], Fd[f, N // 2 - f] = 1, -1
    Fs[Q, Q] = 1
    phi = np.exp(1j * np.pi * plan.taus() / 2)
    return phi[:, None] * (Ue @ Pe @ Fs + 1j * (Uo @ Po @ Fd))


# --------------------------------------------------------------------------
# plan construction (FP64 Jacobi on the GPU) against the oracle's SVD
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,L,den", [(64, 2, 4), (512, 3, 4), (512, 5, 4), (512, 8, 2), (1024, 12, 8)])
def test_plan_matches_oracle(B, O, N, L, den):
    plan = B.Plan(2, 16000.0, N, den, tau_max=L)
    ref = O.Basis(N, L, den)
    se, so = plan.singular_values()
    s = np.sort(np.concatenate([se, so]))[::-1][: len(ref.s)]
    assert np.max(np.abs(s - ref.s)) <= 1e-11 * ref.s[0]
    assert plan.K == ref.K
    assert plan.I == ref.I and np.array_equal(plan.taus(), ref.taus)
    WK = _plan_WK(plan)
    assert np.linalg.norm(WK - ref.WK) <= 1e-9 * np.linalg.norm(ref.WK)
    # the dictionary halves are even / odd in tau (used by the kernel's symmetric pass)
    _, _, Ue, Uo = plan.bases()
    assert np.allclose(Ue, Ue[::-1], atol=1e-10)
    assert np.allclose(Uo, -Uo[::-1], atol=1e-10)
    plan.close()


# --------------------------------------------------------------------------
# the hot path
# --------------------------------------------------------------------------
def _run_and_compare(B, O, X, N, L, den, M, K=0):
    plan = B.Plan(M, 16000.0, N, den, tau_max=L, K=K)
    Xd = torch.from_numpy(X).cuda()
    out = plan.tdoa(Xd, tau_hat=True, coeffs=True, corr=True)
    plan.sync()
    ref = O.Basis(N, L, den, K=plan.K)
    idx, peak, tau, y = O.tdoa(X, ref.WK, ref.taus, ref.delta, want_y=True)
    corr = out["corr"].cpu().numpy()
    check_corr(corr, y)
    gi = out["lag_idx"].cpu().numpy()
    check_argmax(gi, y)
    # the reported peak is the kernel's own y at its argmax
    gp = out["peak"].cpu().numpy()
    assert np.array_equal(gp, np.take_along_axis(corr, gi[..., None].astype(np.int64), -1)[..., 0])
    same = gi == idx
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(gp - peak)[same] <= 1e-4 * scale[same])
    # quadratic refinement: same FP64 formula on FP32 correlation values
    gt = out["tau_hat"].cpu().numpy()
    assert np.all(np.abs(gt - tau)[same] <= 2e-3)
    # projection coefficients reproduce the correlation through the plan's bases
    Pe, Po, Ue, Uo = plan.bases()
    KE, KO = plan.K_even, plan.K_odd
    c = out["coeffs"].cpu().numpy().astype(np.float64)
    ze = c[..., :KE] + 1j * c[..., KE:2 * KE]
    zo = c[..., 2 * KE:2 * KE + KO] + 1j * c[..., 2 * KE + KO:]
    phi = np.exp(1j * np.pi * plan.taus() / 2)
    yc = 2 * np.real(phi * (ze @ Ue.T + 1j * (zo @ Uo.T)))
    check_corr(yc, y)
    plan.close()
    return out


def test_small_square_parity(B, O):
    rec = synth.config_small_square(1)
    out = _run_and_compare(B, O, rec.spectra, 512, 3, 4, 4)
    assert out["lag_idx"].shape == (61, 6)


@pytest.mark.parametrize("M,N,den,L,T", [
    (2, 16, 1, 2, 5),
    (3, 64, 2, 3, 33),
    (4, 256, 4, 3, 1),
    (5, 128, 4, 2, 17),
    (6, 256, 4, 3, 50),
    (7, 32, 4, 1, 3),
    (8, 512, 4, 5, 130),
    (12, 512, 2, 4, 20),
    (16, 1024, 8, 12, 9),
])
def test_random_spectra_parity(B, O, M, N, den, L, T):
    X = _random_spectra(T, M, N, seed=M * 1000 + N + T)
    _run_and_compare(B, O, X, N, L, den, M)


def test_fixed_rank_and_ragged_tiles(B, O):
    # K below the energy rule, and T not a multiple of any tile size
    X = workloads.CIRCLE8.spectra(T=203, seed=9).numpy()
    _run_and_compare(B, O, X, 512, 5, 4, 8, K=5)


def test_zero_bins_and_zero_frames(B, O):
    X = _random_spectra(24, 8, 512, seed=4, zero_frac=0.2)
    X[3] = 0          # a silent frame: y == 0 everywhere, argmax -> index 0
    X[5, 2] = 0       # one silent microphone
    out = _run_and_compare(B, O, X, 512, 5, 4, 8)
    assert np.all(out["lag_idx"][3].cpu().numpy() == 0)
    assert np.all(out["peak"][3].cpu().numpy() == 0)


def test_pure_delays_on_grid(B):
    # X_j = X_i exp(-j 2 pi f D / N): the pair (0, 1) peaks at tau = -D
    N, M = 512, 2
    plan = B.Plan(M, 16000.0, N, 4, tau_max=3)
    f = np.arange(N // 2 + 1)
    rng = np.random.default_rng(1)
    S = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
    Ds = np.arange(-3, 3.25, 0.25)
    X = np.stack([np.stack([S, S * np.exp(-2j * np.pi * f * D / N)]) for D in Ds]).astype(np.complex64)
    out = plan.tdoa(torch.from_numpy(X).cuda())
    plan.sync()
    taus = plan.taus()
    got = taus[out["lag_idx"][:, 0].cpu().numpy()]
    assert np.array_equal(got, -Ds)
    assert np.all(np.abs(out["tau_hat"][:, 0].cpu().numpy() + Ds) < 0.05)
    plan.close()


def test_empty_input_is_noop(B):
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)
    X = torch.empty((0, 4, 257), dtype=torch.complex64, device="cuda")
    out = plan.tdoa(X)
    plan.sync()
    assert out["lag_idx"].numel() == 0
    plan.close()


def test_nonfinite_input_is_reported(B):
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)
    X = torch.from_numpy(_random_spectra(8, 4, 512, seed=2)).cuda()
    X[3, 1, 7] = complex(float("nan"), 0.0)
    plan.tdoa(X)
    with pytest.raises(B.FccError) as ei:
        plan.sync()
    assert ei.value.status == 6
    plan.tdoa(torch.from_numpy(_random_spectra(8, 4, 512, seed=3)).cuda())
    plan.sync()  # the error word was cleared
    plan.close()


def test_invalid_arguments(B):
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)
    X = torch.from_numpy(_random_spectra(4, 4, 512, seed=2)).cuda()
    lib = B.lib()
    import ctypes
    o = torch.empty((4, 6), dtype=torch.int32, device="cuda")
    pk = torch.empty((4, 6), dtype=torch.float32, device="cuda")
    # misaligned spectra pointer
    st = lib.fcc_tdoa(plan._h, ctypes.c_void_p(X.data_ptr() + 8), 3, ctypes.c_void_p(o.data_ptr()),
                      ctypes.c_void_p(pk.data_ptr()), None, None, None, None)
    assert st == 1
    st = lib.fcc_tdoa(plan._h, ctypes.c_void_p(X.data_ptr()), -1, ctypes.c_void_p(o.data_ptr()),
                      ctypes.c_void_p(pk.data_ptr()), None, None, None, None)
    assert st == 1
    plan.close()


def test_host_entry_point_matches_device(B):
    X = workloads.CIRCLE8.spectra(T=1500, seed=5)
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5)
    dev = plan.tdoa(X.cuda())
    plan.sync()
    host = plan.tdoa_host(X.pin_memory())
    for k in ("lag_idx", "peak", "tau_hat"):
        assert torch.equal(dev[k].cpu(), host[k]), k
    plan.close()


def test_host_entry_point_odd_mics_and_chunking(B):
    # 3 microphones: a frame (6168 B) is not a multiple of 16 bytes, so the
    # kernel stages with plain loads; 40001 frames leave a ragged last tile
    rng = np.random.default_rng(8)
    T = 40001
    X = (rng.standard_normal((T, 3, 257)) + 1j * rng.standard_normal((T, 3, 257))).astype(np.complex64)
    plan = B.Plan(3, 16000.0, 512, 4, tau_max=3)
    dev = plan.tdoa(torch.from_numpy(X).cuda())
    plan.sync()
    host = plan.tdoa_host(torch.from_numpy(X).pin_memory())
    for k in ("lag_idx", "peak", "tau_hat"):
        assert torch.equal(dev[k].cpu(), host[k]), k
    plan.close()


# --------------------------------------------------------------------------
# GCC-PHAT baseline (full rank, cuFFT) against eq. 2 in the oracle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("M,N,den,L,T", [(4, 512, 4, 3, 61), (3, 64, 1, 4, 20), (5, 128, 2, 3, 11)])
def test_gcc_baseline_parity(B, O, M, N, den, L, T):
    if (M, N) == (4, 512):
        X = synth.config_small_square(1).spectra
    else:
        X = _random_spectra(T, M, N, seed=N + M)
    plan = B.Plan(M, 16000.0, N, den, tau_max=L)
    out = plan.gcc_tdoa(torch.from_numpy(X).cuda(), corr=True)
    plan.sync()
    taus = O.grid(L, den)
    W = O.build_W(N, taus)
    idx, peak, tau, y = O.tdoa(X, W, taus, 1.0 / den, want_y=True)
    check_corr(out["corr"].cpu().numpy(), y)
    check_argmax(out["lag_idx"].cpu().numpy(), y)
    plan.close()


# --------------------------------------------------------------------------
# full-size 8-mic circle workload (2^20 frames, the benchmark's launch) on samples
# --------------------------------------------------------------------------
def test_circle8_full_size_sampled(B, O):
    w = workloads.CIRCLE8
    X = w.spectra(device="cuda", seed=2)
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L)
    out = plan.tdoa(X, tau_hat=True)
    plan.sync()
    rng = np.random.default_rng(0)
    frames = np.unique(np.concatenate([[0, 1, w.T - 1], rng.integers(0, w.T, 400)]))
    Xs = X[torch.from_numpy(frames).cuda()].cpu().numpy()
    ref = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
    idx, peak, tau, y = O.tdoa(Xs, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"][torch.from_numpy(frames).cuda()].cpu().numpy()
    check_argmax(gi, y)
    gp = out["peak"][torch.from_numpy(frames).cuda()].cpu().numpy()
    same = gi == idx
    assert np.all(np.abs(gp - peak)[same] <= 1e-4 * np.abs(y).max(-1)[same])
    plan.close()
    del X
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------
# lag grid on the tensor cores (long grids, 6-8 bases per parity) against the
# CUDA-core scan: the same argmax wherever the FP32 values' top two differ by
# more than the FP32 tolerance, and there the same peak and refinement bit for
# bit (both evaluate the chosen lag and its neighbours in FP32)
# --------------------------------------------------------------------------
def _with_ties(X, N, den, seed):
    """Frames that stress the selection: a silent frame (every lag ties), a frame
    whose microphones all carry one signal (zero lag wins, y symmetric), and
    microphone m delayed by m h with h half-way between grid steps (pairs an odd
    number of microphones apart sit between two lags: near-ties)."""
    X = X.copy()
    T, M = X.shape[:2]
    rng = np.random.default_rng(seed)
    f = np.arange(N // 2 + 1)
    X[0] = 0
    X[1] = X[1, :1]
    for t in range(2, min(T, 40)):
        S = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
        h = (rng.integers(0, 6) + 0.5) / den
        X[t] = np.stack([S * np.exp(-2j * np.pi * f * h * m / N) for m in range(M)])
    return X.astype(np.complex64)


@pytest.mark.parametrize("M,N,den,L,T", [
    (16, 1024, 8, 12, 1500),
    (16, 512, 4, 12, 700),
    (13, 1024, 8, 12, 300),
    (12, 1024, 8, 12, 300),
])
def test_tensor_core_lag_grid_against_cuda_core_scan(B, monkeypatch, M, N, den, L, T):
    if (M, N) == (16, 1024):
        X = workloads.GRID16.spectra(T=T, seed=5).numpy()
    else:
        X = _random_spectra(T, M, N, seed=M + T)
    X = _with_ties(X, N, den, seed=M + T)
    Xd = torch.from_numpy(X).cuda()
    plan = B.Plan(M, 16000.0, N, den, tau_max=L)
    monkeypatch.setenv("FCC_FP32_MMA_RECON", "0")
    ref = B.Plan(M, 16000.0, N, den, tau_max=L)
    monkeypatch.delenv("FCC_FP32_MMA_RECON")
    b = ref.tdoa(Xd, corr=True)
    ref.sync()
    yb = b["corr"].cpu().numpy().astype(np.float64)
    for corr in (False, True):
        a = plan.tdoa(Xd, corr=corr)
        plan.sync()
        ia = a["lag_idx"].cpu().numpy()
        check_argmax(ia, yb)
        same = ia == b["lag_idx"].cpu().numpy()
        assert same.mean() > 0.999
        for key in ("peak", "tau_hat"):
            assert np.array_equal(a[key].cpu().numpy()[same], b[key].cpu().numpy()[same]), key
        if corr:
            ca = a["corr"].cpu().numpy()
            check_corr(ca, yb, rtol=1e-5)
            # the kernel's peak is its own y at its argmax
            own = np.take_along_axis(ca, ia[..., None].astype(np.int64), -1)[..., 0]
            assert np.array_equal(a["peak"].cpu().numpy(), own)
            if (M, N) == (16, 1024):
                # the tensor-core values differ from the CUDA-core scan's in the last bits
                assert not np.array_equal(ca, yb.astype(np.float32))
    plan.close()
    ref.close()
