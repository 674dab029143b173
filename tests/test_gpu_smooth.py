"""GPU parity of the smoothed path (Sec. 2, Eq. 1 with alpha < 1; include/
fcc_smooth.h) against the FP64 oracle's recursion.  Tolerances as the FP32
path (tests/helpers.py): peaks within 1e-4 of the pair-frame's max |y|, argmax
bit-exact wherever the oracle's top-2 gap is clear; the carried state within
1e-4 of its magnitude (an FP32 recursion whose memory is about 1 / alpha frames)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_argmax  # noqa: E402


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


def _spectra(T, M, N, seed, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    B = N // 2 + 1
    X = rng.standard_normal((T, M, B)) + 1j * rng.standard_normal((T, M, B))
    if zero_frac:
        X[rng.random(X.shape) < zero_frac] = 0
    return X.astype(np.complex64)


def _state(P, B, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return (scale * (rng.standard_normal((P, B)) + 1j * rng.standard_normal((P, B)))).astype(np.complex64)


def _check(out, ref, R_gpu=None, R_ref=None):
    idx, peak, tau, y, R_end = ref
    check_argmax(out["lag_idx"].cpu().numpy(), y)
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(out["peak"].cpu().numpy() - peak) <= 1e-4 * scale)
    if R_gpu is not None:
        err = np.abs(R_gpu - R_end) / np.maximum(np.abs(R_end), 1e-30)
        assert np.quantile(err, 0.999) <= 1e-4 and np.abs(R_gpu - R_end).max() <= 1e-4 * np.abs(R_end).max()


@pytest.mark.parametrize("M,N,den,L,T,alpha,K", [(8, 512, 4, 5, 300, 0.1, 0), (8, 512, 4, 5, 97, 0.5, 0),
                                               (4, 256, 4, 3, 261, 0.1, 0), (2, 128, 2, 2, 150, 0.05, 0),
                                               (6, 512, 4, 3, 130, 0.3, 0), (4, 512, 2, 8, 120, 0.2, 0),
                                               (4, 256, 4, 6, 77, 0.1, 16)])
def test_smoothed_matches_oracle(B, O, M, N, den, L, T, alpha, K):
    # the last two cases take 6 and 8 bases of each parity (K = 11 by the energy
    # rule, and K = 16 given)
    X = _spectra(T, M, N, seed=M * 100 + T)
    plan = B.Plan(M, 16000.0, N, den, tau_max=L, K=K)
    P, Bn = plan.P, plan.B
    R0 = _state(P, Bn, seed=T, scale=2.0)
    state = torch.from_numpy(R0).cuda()
    out = plan.tdoa_smoothed(torch.from_numpy(X).cuda(), alpha, state=state)
    plan.sync()
    basis = O.Basis(N, L, den, K=plan.K)
    ref = O.tdoa_smoothed(X, basis.WK, basis.taus, basis.delta, alpha, R0=R0, want_y=True)
    _check(out, ref, state.cpu().numpy(), ref[4])
    plan.close()


def test_alpha_one_matches_the_unsmoothed_path(B, O):
    X = _spectra(120, 8, 512, seed=3)
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5)
    a = plan.tdoa_smoothed(torch.from_numpy(X).cuda(), 1.0)
    b = plan.tdoa(torch.from_numpy(X).cuda())
    plan.sync()
    basis = O.Basis(512, 5, 4, K=plan.K)
    _, _, _, y = O.tdoa(X, basis.WK, basis.taus, basis.delta, want_y=True)
    check_argmax(a["lag_idx"].cpu().numpy(), y)
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(a["peak"].cpu().numpy() - b["peak"].cpu().numpy()) <= 2e-4 * scale)
    plan.close()


def test_stream_continues_across_calls(B, O):
    X = _spectra(400, 8, 512, seed=7)
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5)
    state = torch.zeros((plan.P, plan.B), dtype=torch.complex64, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    o1 = plan.tdoa_smoothed(Xd[:150].contiguous(), 0.1, state=state)
    o2 = plan.tdoa_smoothed(Xd[150:].contiguous(), 0.1, state=state)
    plan.sync()
    basis = O.Basis(512, 5, 4, K=plan.K)
    ref = O.tdoa_smoothed(X, basis.WK, basis.taus, basis.delta, 0.1, want_y=True)
    out = {k: torch.cat([o1[k], o2[k]]) for k in ("lag_idx", "peak")}
    _check(out, ref, state.cpu().numpy(), ref[4])
    plan.close()


@pytest.mark.parametrize("scale", [1e-17, 1e17])
def test_extreme_magnitudes(B, O, scale):
    # |R|^2 underflows (1e-17) or overflows (1e17) FP32 although R itself is a
    # normal number: the phase transform must rescale rather than lose R_hat
    X = (_spectra(90, 4, 256, seed=21).astype(np.complex128) * scale).astype(np.complex64)
    plan = B.Plan(4, 16000.0, 256, 4, tau_max=3)
    out = plan.tdoa_smoothed(torch.from_numpy(X).cuda(), 0.1)
    plan.sync()
    basis = O.Basis(256, 3, 4, K=plan.K)
    ref = O.tdoa_smoothed(X, basis.WK, basis.taus, basis.delta, 0.1, want_y=True)
    _check(out, ref)
    plan.close()


def test_zero_bins_nan_and_arguments(B):
    plan = B.Plan(4, 16000.0, 256, 4, tau_max=3)
    X = _spectra(80, 4, 256, seed=9, zero_frac=0.3)  # zero cross-spectra where a mic bin is 0
    out = plan.tdoa_smoothed(torch.from_numpy(X).cuda(), 0.2)
    plan.sync()
    assert np.isfinite(out["peak"].cpu().numpy()).all()
    X[40, 1, 7] = np.nan
    plan.tdoa_smoothed(torch.from_numpy(X).cuda(), 0.2)
    with pytest.raises(B.FccError) as e:
        plan.sync()
    assert e.value.status == 6
    for bad_alpha in (0.0, 1.5, -0.1):
        with pytest.raises(B.FccError):
            plan.tdoa_smoothed(torch.from_numpy(X).cuda(), bad_alpha)
    plan.close()
    for args in ((16, 16000.0, 512, 4), (5, 16000.0, 512, 4), (4, 16000.0, 1024, 4)):
        p2 = B.Plan(*args, tau_max=3)
        with pytest.raises(B.FccError) as e:
            p2.smooth_workspace(10)
        assert e.value.status == 2
        p2.close()
