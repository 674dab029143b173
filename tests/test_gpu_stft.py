"""GPU parity of the STFT front-end (include/fcc_stft.h) against the FP64
oracle (oracle.stft, numpy's rfft as the DFT).

Spectra: an FP32 FFT of N points has a 2-norm error of a few times
log2(N) * 2^-24 of the frame's spectrum norm, so every bin must be within
1e-5 * ||X_oracle(t, m)||_2.  TDoA from PCM: the FP32 path (FP32 STFT, FP32
FCC) against the FP64 chain (oracle STFT, oracle FCC on W_K) with the FP32
path's tolerances (tests/helpers.py): peaks within 1e-4 of the pair-frame's
max |y|, argmax exact where the oracle's top-2 gap is clear."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_argmax  # noqa: E402

from paper_2204_13622_gb300 import synth  # noqa: E402


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


def _pcm(n, M, seed, kind="f32", delays=None):
    """Seeded multichannel PCM: a white source seen by every mic with an
    integer delay (samples) plus independent noise at about 10 dB SNR."""
    rng = np.random.default_rng(seed)
    d = np.zeros(M, int) if delays is None else np.asarray(delays)
    pad = int(np.abs(d).max()) + 1
    s = rng.standard_normal(n + 2 * pad)
    x = np.stack([s[pad - d[m]:pad - d[m] + n] for m in range(M)], axis=1)
    x = 0.3 * x + 0.1 * rng.standard_normal((n, M))
    if kind == "s16":
        return np.clip(np.round(x * 8000), -32768, 32767).astype(np.int16)
    return x.astype(np.float32)


@pytest.mark.parametrize("M,N,hop,extra,kind", [(8, 512, 128, 77, "f32"), (4, 256, 100, 3, "s16"),
                                                (2, 64, 64, 0, "f32"), (6, 1024, 333, 300, "s16"),
                                                (3, 2048, 512, 1, "f32"), (8, 128, 32, 31, "s16")])
def test_stft_matches_oracle(B, O, M, N, hop, extra, kind):
    T = 37
    n = (T - 1) * hop + N + extra
    x = _pcm(n, M, seed=N + M, kind=kind)
    plan = B.Plan(M, 16000.0, N, 4, tau_max=2)
    assert plan.stft_frames(n, hop) == T
    X = plan.stft(torch.from_numpy(x).cuda(), hop)
    plan.sync()
    ref = O.stft(x, N, hop)
    got = X.cpu().numpy().astype(np.complex128)
    norm = np.linalg.norm(ref, axis=2, keepdims=True)
    assert np.all(np.abs(got - ref) <= 1e-5 * norm), (np.abs(got - ref) / norm).max()
    plan.close()


def test_pcm_to_tdoa_matches_oracle_chain(B, O):
    xyz = synth.circular_array(8, 0.05)
    N, hop, den = 512, 128, 4
    L = synth.lag_extent(xyz, 16000.0)
    plan = B.Plan(8, 16000.0, N, den, mic_xyz=xyz)
    T = 300
    n = (T - 1) * hop + N + 5
    x = _pcm(n, 8, seed=5, kind="s16", delays=[0, 1, 3, 4, 4, 3, 1, 0])
    pcm = torch.from_numpy(x).cuda()
    out = plan.tdoa_pcm(pcm, hop)
    # the same kernels in two calls give the same bytes
    X = plan.stft(pcm, hop)
    ref = plan.tdoa(X)
    plan.sync()
    for k in ("lag_idx", "peak", "tau_hat"):
        assert torch.equal(out[k], ref[k]), k
    basis = O.Basis(N, L, den, K=plan.K)
    Xo = O.stft(x, N, hop).astype(np.complex64)
    idx, peak, _, y = O.tdoa(Xo, basis.WK, basis.taus, basis.delta, want_y=True)
    check_argmax(out["lag_idx"].cpu().numpy(), y)
    scale = np.abs(y).max(-1)
    assert np.all(np.abs(out["peak"].cpu().numpy() - peak) <= 1e-4 * scale)
    plan.close()


def test_delayed_channel_sign(B):
    # mic 1 hears the source 3 samples after mic 0: tau_01 = t_0 - t_1 = -3
    plan = B.Plan(2, 16000.0, 512, 4, tau_max=5)
    x = _pcm(128 * 40 + 512, 2, seed=9, delays=[0, 3])
    out = plan.tdoa_pcm(torch.from_numpy(x).cuda(), 128)
    plan.sync()
    taus = plan.taus()
    assert np.all(taus[out["lag_idx"].cpu().numpy()[:, 0]] == -3.0)
    plan.close()


def test_host_path_equals_device_path(B):
    # more frames than one host chunk (65536 frames)
    plan = B.Plan(4, 16000.0, 256, 4, tau_max=3)
    hop, T = 64, 70000
    n = (T - 1) * hop + 256
    x = _pcm(n, 4, seed=11, kind="s16", delays=[0, 1, 2, 1])
    host = torch.from_numpy(x).pin_memory()
    a = plan.tdoa_pcm_host(host, hop)
    b = plan.tdoa_pcm(host.cuda(), hop)
    plan.sync()
    for k in ("lag_idx", "peak", "tau_hat"):
        assert torch.equal(a[k], b[k].cpu()), k
    plan.close()


def test_errors_and_edges(B):
    plan = B.Plan(4, 16000.0, 256, 4, tau_max=3)
    x = torch.from_numpy(_pcm(1000, 4, seed=1)).cuda()
    with pytest.raises(B.FccError):
        plan.stft(x, 0)  # hop < 1
    assert plan.stft_frames(255, 64) == 0 and plan.stft(x[:255].contiguous(), 64).shape[0] == 0
    out = plan.tdoa_pcm(x[:100].contiguous(), 64)  # no frame: no launch
    assert out["lag_idx"].shape[0] == 0
    with pytest.raises(ValueError):
        plan.stft(x[:, :3].contiguous(), 64)  # wrong mic count
    y = x.clone()
    y[500, 2] = float("nan")
    plan.tdoa_pcm(y, 64)
    with pytest.raises(B.FccError) as e:
        plan.sync()
    assert e.value.status == 6
    # full-scale int16 stays finite
    s = torch.full((600, 4), -32768, dtype=torch.int16, device="cuda")
    s[::2] = 32767
    o = plan.tdoa_pcm(s, 64)
    plan.sync()
    assert torch.isfinite(o["peak"]).all()
    plan.close()
    big = B.Plan(4, 16000.0, 4096, 4, tau_max=3)
    with pytest.raises(B.FccError) as e:
        big.stft(torch.zeros((5000, 4), device="cuda"), 1024)
    assert e.value.status == 2
    big.close()
