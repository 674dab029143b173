"""GPU parity of the DoA search over candidate directions (include/fcc_doa.h)
against the FP64 oracle (oracle.doa_srp), on the same float32 correlations.

Tolerance: a score is a sum of P interpolated FP32 values, each within a few
ulps of max |y|, so |score_gpu - score_oracle| <= 1e-5 * P * max|y|.  The
chosen candidate equals the oracle's wherever the oracle's best score leads the
runner-up by more than twice that; elsewhere the GPU's candidate must score
within twice that of the oracle's best."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_13622_gb300 import synth  # noqa: E402

FS, C = 16000.0, 343.0


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


def _check(idx, score, y, L, den, xyz, dirs, O, fs=FS):
    ref_idx, ref_best, scores = O.doa_srp(y.astype(np.float64), L, den, xyz, fs, C, dirs, want_scores=True)
    tol = 1e-5 * y.shape[1] * np.abs(y).max()
    T = y.shape[0]
    got = scores[np.arange(T), idx]
    assert np.all(np.abs(score - got) <= tol), np.abs(score - got).max()
    srt = np.sort(scores, axis=1)
    gap = srt[:, -1] - (srt[:, -2] if scores.shape[1] > 1 else -np.inf)
    clear = gap > 2 * tol
    assert np.array_equal(idx[clear], ref_idx[clear])
    assert np.all(ref_best[~clear] - got[~clear] <= 2 * tol)


def _source_spectra(xyz, N, T, seed, dirs_true):
    # one far-field white source per frame from the given directions, white noise at 10 dB
    rng = np.random.default_rng(seed)
    f = np.arange(N // 2 + 1)
    M = xyz.shape[0]
    X = np.empty((T, M, N // 2 + 1), np.complex128)
    for t in range(T):
        s = rng.standard_normal(N // 2 + 1) + 1j * rng.standard_normal(N // 2 + 1)
        delta = synth.far_field_delays(xyz, dirs_true[t], FS)
        X[t] = s[None] * np.exp(-2j * np.pi * np.outer(delta, f) / N)
        X[t] += 0.3 * (rng.standard_normal((M, N // 2 + 1)) + 1j * rng.standard_normal((M, N // 2 + 1)))
    return X.astype(np.complex64)


@pytest.mark.parametrize("M,N,den,D,T", [(8, 512, 4, 300, 37), (4, 512, 4, 1, 20), (2, 256, 4, 700, 9),
                                         (6, 512, 4, 257, 64), (16, 1024, 8, 64, 5)])
def test_search_matches_oracle(B, O, M, N, den, D, T):
    xyz = synth.circular_array(M, 0.05) if M != 16 else synth.grid_array(4, 4, 0.02)
    fs = FS if M != 16 else 48000.0
    L = synth.lag_extent(xyz, fs)
    plan = B.Plan(M, fs, N, den, mic_xyz=xyz)
    dirs = synth.fibonacci_directions(D)
    rng = np.random.default_rng(M * 10 + T)
    truth = synth.fibonacci_directions(97)[rng.integers(0, 97, T)]
    X = _source_spectra(xyz, N, T, seed=T, dirs_true=truth)
    o = plan.tdoa(torch.from_numpy(X).cuda(), corr=True)
    plan.sync()
    y = o["corr"].cpu().numpy()
    doa = B.Doa(plan, xyz, dirs)
    out = doa.search(o["corr"])
    plan.sync()
    _check(out["dir_idx"].cpu().numpy(), out["score"].cpu().numpy().astype(np.float64), y, L, den, xyz, dirs, O,
           fs=fs)
    doa.close()
    plan.close()


def test_spectra_to_doa_in_chunks(B, O):
    # more frames than one chunk of the fused call: the per-frame result must equal
    # fcc_tdoa's correlations searched in one call, bit for bit
    xyz = synth.circular_array(8, 0.05)
    N, den = 512, 4
    L = synth.lag_extent(xyz, FS)
    plan = B.Plan(8, FS, N, den, mic_xyz=xyz)
    dirs = synth.fibonacci_directions(512)
    doa = B.Doa(plan, xyz, dirs)
    T = 6000
    Xd = synth.stft_domain_spectra(T, xyz, FS, N, 128, seed=3, device="cuda")
    out = doa.tdoa_doa(Xd, pairs=True)
    ref = plan.tdoa(Xd, corr=True)
    s = doa.search(ref["corr"])
    plan.sync()
    assert torch.equal(out["dir_idx"], s["dir_idx"]) and torch.equal(out["score"], s["score"])
    assert torch.equal(out["lag_idx"], ref["lag_idx"]) and torch.equal(out["peak"], ref["peak"])
    # a sample against the oracle's correlations of the same spectra
    basis = O.Basis(N, L, den, K=plan.K)
    sel = np.arange(0, T, 250)
    Xh = Xd[sel].cpu().numpy()
    _, _, _, y = O.tdoa(Xh, basis.WK, basis.taus, basis.delta, want_y=True)
    ref_idx, _, scores = O.doa_srp(y, L, den, xyz, FS, C, dirs, want_scores=True)
    got = out["dir_idx"][sel].cpu().numpy()
    tol = 1e-4 * 28 * np.abs(y).max()  # FP32 FCC + FP32 search against FP64 throughout
    srt = np.sort(scores, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * tol
    assert np.array_equal(got[clear], ref_idx[clear])
    assert np.all(scores[np.arange(len(sel)), ref_idx] - scores[np.arange(len(sel)), got] <= 2 * tol)
    doa.close()
    plan.close()


def test_source_directions_are_found(B):
    # noiseless far-field sources from candidate directions: the search returns them
    xyz = synth.circular_array(8, 0.05)
    plan = B.Plan(8, FS, 512, 4, mic_xyz=xyz)
    dirs = synth.fibonacci_directions(128)
    ks = np.array([3, 40, 77, 100, 127])
    f = np.arange(257)
    X = np.stack([np.exp(-2j * np.pi * np.outer(synth.far_field_delays(xyz, dirs[k], FS), f) / 512) for k in ks])
    doa = B.Doa(plan, xyz, dirs)
    out = doa.tdoa_doa(torch.from_numpy(X.astype(np.complex64)).cuda())
    plan.sync()
    assert np.array_equal(out["dir_idx"].cpu().numpy(), ks)
    doa.close()
    plan.close()


def test_errors_and_edges(B):
    xyz = synth.circular_array(4, 0.05)
    plan = B.Plan(4, FS, 512, 4, mic_xyz=xyz)
    with pytest.raises(B.FccError):
        B.Doa(plan, xyz, np.zeros((0, 3)))
    with pytest.raises(B.FccError):
        B.Doa(plan, xyz, np.array([[np.nan, 0, 1.0]]))
    doa = B.Doa(plan, xyz, synth.fibonacci_directions(33))
    corr = torch.zeros((0, plan.P, plan.I), device="cuda")
    out = doa.search(corr)  # T = 0: no launch
    assert out["dir_idx"].numel() == 0
    y = torch.randn((12, plan.P, plan.I), device="cuda")
    y[7, 2, :] = float("nan")  # every candidate reads pair 2 somewhere on its grid
    doa.search(y)
    with pytest.raises(B.FccError) as e:
        plan.sync()
    assert e.value.status == 6
    with pytest.raises(ValueError):
        doa.search(torch.zeros((4, plan.P, plan.I + 1), device="cuda"))
    X = torch.zeros((3, 4, 257), dtype=torch.complex64, device="cuda")
    with pytest.raises(B.FccError):
        doa.tdoa_doa(X, work=torch.empty(8, dtype=torch.uint8, device="cuda"))  # workspace too small
    doa.close()
    plan.close()
