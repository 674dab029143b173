"""Pins of the oracle's STFT front-end (Sec. 2: the method starts from the
microphones' STFT; window and framing as read in the design notes: periodic
Hann, frames of N every hop samples, no padding).  Pinned by the direct O(N^2)
DFT sum, a cosine on a bin (closed form for the periodic Hann window),
Parseval, the framing, int16 scaling, and the TDoA sign of a delayed channel
through the FCC oracle."""
import numpy as np


def test_direct_dft_sum(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(1)
    N, hop, M = 16, 4, 3
    x = rng.standard_normal((N + 3 * hop + 2, M))
    X = O.stft(x, N, hop)
    assert X.shape == (4, M, N // 2 + 1)
    n = np.arange(N)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * n / N)
    for t in range(4):
        for m in range(M):
            for k in range(N // 2 + 1):
                ref = sum(w[i] * x[t * hop + i, m] * np.exp(-2j * np.pi * k * i / N) for i in range(N))
                assert abs(X[t, m, k] - ref) < 1e-12


def test_cosine_on_a_bin():
    # periodic Hann = 1/2 - (e^{j2pi n/N} + e^{-j2pi n/N}) / 4: a unit cosine on bin k0
    # gives N/4 at k0, -N/8 at k0 +- 1 and zero elsewhere
    from oracle import oracle as O
    N, k0 = 64, 9
    n = np.arange(N)
    x = np.cos(2 * np.pi * k0 * n / N)[:, None]
    X = O.stft(x, N, N)[0, 0]
    expect = np.zeros(N // 2 + 1, complex)
    expect[k0], expect[k0 - 1], expect[k0 + 1] = N / 4, -N / 8, -N / 8
    assert np.abs(X - expect).max() < 1e-12


def test_parseval_framing_and_int16(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(2)
    N, hop = 32, 8
    x = rng.standard_normal((N + 5 * hop + 3, 2))
    X = O.stft(x, N, hop)
    assert X.shape[0] == 6 and O.stft(x[:N - 1], N, hop).shape[0] == 0
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(N) / N)
    for t in range(6):
        e_time = np.sum((w * x[t * hop:t * hop + N, 0]) ** 2)
        a = np.abs(X[t, 0]) ** 2
        e_freq = (a[0] + a[-1] + 2 * a[1:-1].sum()) / N
        assert abs(e_time - e_freq) < 1e-12 * e_time
        # frame t of x is frame 0 of x shifted by t hops
        assert np.abs(X[t] - O.stft(x[t * hop:], N, hop)[0]).max() < 1e-12
    s = rng.integers(-32768, 32767, (N + hop, 3), dtype=np.int16)
    assert np.abs(O.stft(s, N, hop) - O.stft(s.astype(np.float64) / 32768.0, N, hop)).max() == 0.0


def test_delayed_channel_sign(oracle_mod):
    # mic 1 hears the same noise D samples later: tau_01 = t_0 - t_1 = -D
    O = oracle_mod
    rng = np.random.default_rng(3)
    N, hop, D = 512, 128, 3
    src = rng.standard_normal(N + 8 * hop + D)
    x = np.stack([src[D:], src[:-D]], axis=1)  # x1[n] = x0[n - D]
    X = O.stft(x, N, hop).astype(np.complex64)
    basis = O.Basis(N, 4, 4)
    idx, _, _, _ = O.tdoa(X, basis.W, basis.taus, basis.delta)
    assert np.all(basis.taus[idx[:, 0]] == -D)
