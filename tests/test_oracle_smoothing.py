"""Pins of the oracle's recursive cross-spectrum (Sec. 2, Eq. 1 with alpha < 1):
R(t,f) = (1 - alpha) R(t-1,f) + alpha X_i(t,f) X_j(t,f)^*, then R_hat = R / |R|.
The recursion is checked against its closed form written independently, alpha = 1
against the unsmoothed path, a stream split in two calls against one call, and
constant frames against the unsmoothed path."""
import numpy as np
import pytest


def _W(N, taus):
    f = np.arange(N // 2 + 1)
    return np.exp(2j * np.pi * np.outer(taus, f) / N)


def _rand(T, M, B, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((T, M, B)) + 1j * rng.standard_normal((T, M, B))).astype(np.complex64)


def test_recursion_matches_closed_form(oracle_mod):
    O = oracle_mod
    T, M, N, alpha = 7, 3, 16, 0.3
    B = N // 2 + 1
    X = _rand(T, M, B, 1)
    rng = np.random.default_rng(2)
    P = M * (M - 1) // 2
    R0 = rng.standard_normal((P, B)) + 1j * rng.standard_normal((P, B))
    taus = np.arange(-2, 2.25, 0.25)
    W = _W(N, taus)
    idx, peak, tau, y, R_end = O.tdoa_smoothed(X, W, taus, 0.25, alpha, R0=R0, want_y=True)
    Xd = X.astype(np.complex128)
    pairs = [(i, j) for i in range(M) for j in range(i + 1, M)]
    for p, (i, j) in enumerate(pairs):
        C = Xd[:, i, :] * np.conj(Xd[:, j, :])  # [T, B]
        for t in range(T):
            # R(t) = (1-a)^(t+1) R0 + sum_{s<=t} a (1-a)^(t-s) C_s (frames counted from 0)
            R = (1 - alpha) ** (t + 1) * R0[p] + sum(alpha * (1 - alpha) ** (t - s) * C[s] for s in range(t + 1))
            Rh = R / np.abs(R)
            yt = 2 * np.real(W @ Rh)
            assert np.allclose(y[t, p], yt, rtol=0, atol=1e-10 * np.abs(yt).max())
            assert idx[t, p] == np.argmax(yt)
        assert np.allclose(R_end[p], R, rtol=1e-12, atol=0)


def test_alpha_one_is_the_unsmoothed_path(oracle_mod):
    O = oracle_mod
    X = _rand(9, 4, 33, 3)
    taus = np.arange(-3, 3.25, 0.25)
    W = _W(64, taus)
    a = O.tdoa(X, W, taus, 0.25, want_y=True)
    rng = np.random.default_rng(4)
    R0 = rng.standard_normal((6, 33)) + 1j * rng.standard_normal((6, 33))
    b = O.tdoa_smoothed(X, W, taus, 0.25, 1.0, R0=R0, want_y=True)
    for u, v in zip(a, b[:4]):
        assert np.array_equal(u, v)


def test_stream_split_equals_one_call(oracle_mod):
    O = oracle_mod
    X = _rand(20, 4, 33, 5)
    taus = np.arange(-3, 3.25, 0.25)
    W = _W(64, taus)
    full = O.tdoa_smoothed(X, W, taus, 0.25, 0.1, want_y=True)
    first = O.tdoa_smoothed(X[:8], W, taus, 0.25, 0.1, want_y=True)
    second = O.tdoa_smoothed(X[8:], W, taus, 0.25, 0.1, R0=first[4], want_y=True)
    for k in range(4):
        assert np.array_equal(np.concatenate([first[k], second[k]]), full[k])
    assert np.array_equal(second[4], full[4])


def test_constant_frames_keep_the_unsmoothed_phase(oracle_mod):
    O = oracle_mod
    one = _rand(1, 4, 33, 6)
    X = np.repeat(one, 12, axis=0)
    taus = np.arange(-3, 3.25, 0.25)
    W = _W(64, taus)
    a = O.tdoa(X, W, taus, 0.25, want_y=True)
    b = O.tdoa_smoothed(X, W, taus, 0.25, 0.2, want_y=True)  # R(t) = (1 - 0.8^(t+1)) X_i X_j^*
    assert np.allclose(a[3], b[3], rtol=0, atol=1e-12 * np.abs(a[3]).max())
    assert np.array_equal(a[0], b[0])
