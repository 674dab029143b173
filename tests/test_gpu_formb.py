"""GPU parity of the split form (FCC_FORM_REIM_SPLIT: cosine bases on Re x,
sine bases on Im x, each truncated by its own SVD) against the oracle's form B
(oracle.BasisB: y = 2 Re{(C_K + j S_K) x}), for alpha = 1 (fcc_tdoa, the FP32
tile kernel: any M, N <= 1024) and alpha < 1 (fcc_tdoa_smoothed, the per-pair
kernel).  Tolerances as the FP32 path (tests/helpers.py): peaks and
correlations within 1e-4 of the pair-frame's max |y|, argmax exact where the
oracle's top-2 gap is clear."""
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


def _spectra(T, M, N, seed):
    rng = np.random.default_rng(seed)
    Bn = N // 2 + 1
    return (rng.standard_normal((T, M, Bn)) + 1j * rng.standard_normal((T, M, Bn))).astype(np.complex64)


def _check(out, ref):
    idx, peak, tau, y = ref[:4]
    check_argmax(out["lag_idx"].cpu().numpy(), y)
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(out["peak"].cpu().numpy() - peak) <= 1e-4 * scale)


@pytest.mark.parametrize("M,N,den,L,T", [(8, 512, 4, 5, 211), (4, 256, 4, 3, 150), (2, 128, 2, 2, 97),
                                         (6, 512, 8, 2, 64), (5, 1024, 4, 3, 40), (3, 64, 2, 2, 53),
                                         (16, 256, 4, 2, 30), (7, 512, 4, 12, 19)])
def test_split_form_matches_oracle(B, O, M, N, den, L, T):
    plan = B.Plan(M, 16000.0, N, den, tau_max=L, form="reim")
    ob = O.BasisB(N, L, den)
    assert (plan.K_even, plan.K_odd) == (ob.Kc, ob.Ks)
    X = _spectra(T, M, N, seed=M + T)
    out = plan.tdoa(torch.from_numpy(X).cuda(), corr=True)
    plan.sync()
    ref = O.tdoa(X, ob.WK, ob.taus, ob.delta, want_y=True)
    _check(out, ref)
    y = ref[3]
    scale = np.abs(y).max(-1, keepdims=True)
    assert np.all(np.abs(out["corr"].cpu().numpy() - y) <= 1e-4 * scale)
    # the plan's FP64 bases give the same truncated C and S as the oracle's
    Pe, Po, Ue, Uo = plan.bases()
    assert np.abs(Ue @ Pe - ob.CK).max() < 1e-9 and np.abs(Uo @ Po - ob.SK).max() < 1e-9
    plan.close()


def test_split_form_smoothed(B, O):
    M, N, den, L, T, alpha = 8, 512, 4, 5, 240, 0.2
    plan = B.Plan(M, 16000.0, N, den, tau_max=L, form="reim")
    ob = O.BasisB(N, L, den)
    X = _spectra(T, M, N, seed=5)
    state = torch.zeros((plan.P, plan.B), dtype=torch.complex64, device="cuda")
    out = plan.tdoa_smoothed(torch.from_numpy(X).cuda(), alpha, state=state)
    plan.sync()
    ref = O.tdoa_smoothed(X, ob.WK, ob.taus, ob.delta, alpha, want_y=True)
    _check(out, ref)
    plan.close()


def test_split_form_options(B):
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3, form="reim")
    X = torch.from_numpy(_spectra(20, 4, 512, seed=1)).cuda()
    with pytest.raises(B.FccError) as e:
        plan.tdoa(X, coeffs=True)
    assert e.value.status == 2
    with pytest.raises(B.FccError):
        plan.tdoa_smoothed(X, 0.5, coeffs=True)
    with pytest.raises(B.FccError):
        plan.autotune(max_candidates=1)
    # alpha = 1 through the per-pair kernel (fcc_tdoa_smoothed) and through the
    # FP32 tile kernel (fcc_tdoa): two kernels, one argmax where the top-2 gap is clear
    a = plan.tdoa_smoothed(X, 1.0)
    b = plan.tdoa(X, corr=True)
    plan.sync()
    check_argmax(a["lag_idx"].cpu().numpy(), b["corr"].cpu().numpy().astype(np.float64))
    # the PCM front-end runs on split-form plans too
    rng = np.random.default_rng(3)
    pcm = torch.from_numpy((rng.standard_normal((128 * 30 + 512, 4)) * 3000).astype(np.int16)).cuda()
    a = plan.tdoa_pcm(pcm, 128)
    b = plan.tdoa(plan.stft(pcm, 128))
    plan.sync()
    assert torch.equal(a["lag_idx"], b["lag_idx"]) and torch.equal(a["peak"], b["peak"])
    plan.close()
    with pytest.raises(B.FccError) as e:
        B.Plan(4, 16000.0, 512, 4, tau_max=3, form="reim", prec="bf16")
    assert e.value.status == 2


def test_split_form_doa(B, O):
    # the fused spectra -> DoA call on a split-form plan: the same bytes as the
    # correlations of fcc_tdoa searched separately, and the oracle's form B
    # correlations searched by the oracle on a sample of frames
    from paper_2204_13622_gb300 import synth
    xyz = synth.circular_array(8, 0.05)
    N, den, fs, c = 512, 4, 16000.0, 343.0
    L = synth.lag_extent(xyz, fs)
    plan = B.Plan(8, fs, N, den, mic_xyz=xyz, form="reim")
    dirs = synth.fibonacci_directions(256)
    doa = B.Doa(plan, xyz, dirs)
    T = 3000
    Xd = synth.stft_domain_spectra(T, xyz, fs, N, 128, seed=4, device="cuda")
    out = doa.tdoa_doa(Xd, pairs=True)
    ref = plan.tdoa(Xd, corr=True)
    s = doa.search(ref["corr"])
    plan.sync()
    assert torch.equal(out["dir_idx"], s["dir_idx"]) and torch.equal(out["score"], s["score"])
    assert torch.equal(out["lag_idx"], ref["lag_idx"]) and torch.equal(out["peak"], ref["peak"])
    ob = O.BasisB(N, L, den)
    sel = np.arange(0, T, 150)
    _, _, _, y = O.tdoa(Xd[sel].cpu().numpy(), ob.WK, ob.taus, ob.delta, want_y=True)
    ref_idx, _, scores = O.doa_srp(y, L, den, xyz, fs, c, dirs, want_scores=True)
    got = out["dir_idx"][sel].cpu().numpy()
    tol = 1e-4 * plan.P * np.abs(y).max()  # FP32 FCC + FP32 search against FP64 throughout
    srt = np.sort(scores, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 2 * tol
    assert np.array_equal(got[clear], ref_idx[clear])
    rows = np.arange(len(sel))
    assert np.all(scores[rows, ref_idx] - scores[rows, got] <= 2 * tol)
    doa.close()
    plan.close()
