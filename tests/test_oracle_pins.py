"""Pins for the FP64 oracle: each check ties it to something other than itself.

Kinds of pins used here:
* numbers the paper prints (flop counts of Sec. 3/4 and Table 1, I = 33);
* library routines that compute the same quantity another way (LAPACK SVD,
  numpy's zero-padded inverse real FFT for eq. 2);
* closed forms (a pure delay peaks at exactly N + 2; ||W||_F^2 = I (N/2+1));
* brute force on tiny inputs (direct O(N^2) circular cross-correlation);
* invariants the paper states or implies (even/odd bases, Eq. 6; the folded
  product of Eqs. 8-9 equals P x; r_ij(tau) = r_ji(-tau)).
"""
import json
import os

import numpy as np
import pytest

from paper_2204_13622_gb300 import flops, synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.json")


# --------------------------------------------------------------------------
# paper's printed numbers
# --------------------------------------------------------------------------
def test_paper_flop_counts():
    g = json.load(open(GOLD))
    N, I = g["N"], g["I_r2"]
    assert flops.n_candidates(g["tau_max"], 2) == I == 33
    for r, v in g["gcc_flops"].items():
        assert flops.gcc_flops(N, int(r)) == v
    assert flops.direct_flops(N, I) == g["direct_flops"]
    assert flops.lowrank_flops(N, I, 8) == g["lowrank_flops_K8"]
    for K, v in g["fcc_flops"].items():
        assert flops.fcc_flops(N, I, int(K)) == v
    ratio = flops.gcc_flops(N, 2) / flops.fcc_flops(N, I, 8)
    assert round(ratio, 1) == g["fcc_vs_gcc_r2_reduction"]


def test_grid_matches_paper_example(oracle_mod):
    taus = oracle_mod.grid(8, 2)
    assert len(taus) == 33
    assert taus[0] == -8 and taus[-1] == 8 and taus[16] == 0
    assert np.allclose(np.diff(taus), 0.5)


# --------------------------------------------------------------------------
# W (eq. 3) and its SVD (Sec. 4)
# --------------------------------------------------------------------------
def test_W_integer_rows_are_dft_rows(oracle_mod):
    # for an integer lag m, w(m) is the conjugate DFT of a unit impulse at m
    N = 64
    taus = np.array([-3.0, 0.0, 2.0, 5.0])
    W = oracle_mod.build_W(N, taus)
    for row, m in zip(W, taus.astype(int)):
        e = np.zeros(N)
        e[m % N] = 1.0
        ref = np.conj(np.fft.rfft(e))
        assert np.allclose(row, ref, atol=1e-13)


@pytest.mark.parametrize("N,L,den", [(512, 3, 4), (512, 5, 4), (512, 8, 2), (256, 2, 8)])
def test_svd_matches_lapack(oracle_mod, N, L, den):
    b = oracle_mod.Basis(N, L, den)
    s_ref = np.linalg.svd(b.W, compute_uv=False)
    assert np.max(np.abs(b.s - s_ref[: len(b.s)])) <= 1e-12 * s_ref[0]
    U, s, Vh = np.linalg.svd(b.W, full_matrices=False)
    WK = (U[:, : b.K] * s[: b.K]) @ Vh[: b.K]
    assert np.linalg.norm(WK - b.WK) <= 1e-10 * np.linalg.norm(WK)
    # Frobenius norm: every entry of W has modulus one
    assert abs(np.sum(b.s ** 2) - b.I * b.B) <= 1e-9 * b.I * b.B
    # Eckart-Young: the rank-K residual carries exactly the dropped energy
    res = np.linalg.norm(b.W - b.WK) ** 2
    assert abs(res - np.sum(b.s[b.K:] ** 2)) <= 1e-8 * b.I * b.B


def test_svd_random_complex_matrix(oracle_mod):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((17, 40)) + 1j * rng.standard_normal((17, 40))
    U, s, V = oracle_mod.svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
    assert np.allclose((U * s) @ V.conj().T, A, atol=1e-12)
    assert np.allclose(U.conj().T @ U, np.eye(17), atol=1e-12)
    assert np.allclose(V.conj().T @ V, np.eye(17), atol=1e-12)


def test_rank_energy_rule(oracle_mod):
    s = np.sqrt(np.array([50.0, 30.0, 15.0, 4.0, 0.9, 0.1]))
    assert oracle_mod.rank_energy(s, 0.95) == 3       # 95 of 100
    assert oracle_mod.rank_energy(s, 0.99) == 4       # 99 of 100
    assert oracle_mod.rank_energy(s, 0.998) == 5      # 99.9 of 100 >= 99.8
    assert oracle_mod.rank_energy(s, 0.9995) == 6     # needs the last value
    # a tie at the cut pulls in the whole tied group
    t = np.array([3.0, 2.0, 2.0, 2.0, 0.1])
    assert oracle_mod.rank_energy(t, 0.5) == 4
    t = np.array([3.0, 2.0, 1.999, 1.5, 0.1])
    assert oracle_mod.rank_energy(t, 0.5, tie_rel=1e-3) == 3
    assert oracle_mod.rank_energy(t, 0.5, tie_rel=1e-12) == 2


def test_basis_parity_structure(oracle_mod):
    """Eq. 6: the bases are even or odd about f = N/4 (after a phase choice)."""
    b = oracle_mod.Basis(512, 5, 4)
    WhW = b.W.conj().T @ b.W
    assert np.max(np.abs(WhW.imag)) <= 1e-9 * np.max(np.abs(WhW.real))
    n_even = n_odd = 0
    for k in range(b.K):
        gap = min(abs(b.s[k] - b.s[k - 1]) if k else np.inf, abs(b.s[k] - b.s[k + 1]))
        if gap < 1e-8 * b.s[0]:
            continue
        v = b.V[:, k]
        v = v * np.exp(-1j * np.angle(v[np.argmax(np.abs(v))]))
        assert np.max(np.abs(v.imag)) < 1e-9
        refl = v.real[::-1]  # f -> N/2 - f
        if np.allclose(refl, v.real, atol=1e-9):
            n_even += 1
        else:
            assert np.allclose(refl, -v.real, atol=1e-9)
            n_odd += 1
    assert n_even >= 3 and n_odd >= 3


def test_folded_projection_equals_Px(oracle_mod):
    """Eqs. 6-9: the cropped bases applied to x_s / x_d give exactly z = P x."""
    b = oracle_mod.Basis(512, 5, 4)
    N, Q = b.N, b.N // 4
    P = (b.s[: b.K, None] * b.V[:, : b.K].conj().T)  # K x B
    rng = np.random.default_rng(7)
    x = np.exp(1j * rng.uniform(0, 2 * np.pi, b.B))
    z_ref = P @ x
    xs = np.concatenate([x[:Q] + x[N // 2: Q: -1], [x[Q]]])
    xd = np.concatenate([x[:Q] - x[N // 2: Q: -1], [x[Q]]])
    z = np.empty(b.K, complex)
    for k in range(b.K):
        p = P[k]
        even = np.allclose(p, p[::-1], atol=1e-8)
        assert even or np.allclose(p, -p[::-1], atol=1e-8)
        z[k] = p[: Q + 1] @ (xs if even else xd)
    assert np.allclose(z, z_ref, atol=1e-9)
    # and y = 2 Re{D z} with D = U_K reproduces 2 Re{W_K x}
    y = 2 * np.real(b.U[:, : b.K] @ z)
    assert np.allclose(y, oracle_mod.correlate(b.WK, x), atol=1e-9)


# --------------------------------------------------------------------------
# correlation (eq. 2 / eq. 4), PHAT and the pipeline
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,L,den", [(64, 4, 1), (64, 4, 2), (128, 3, 4), (512, 5, 4)])
def test_full_rank_equals_zero_padded_irfft(oracle_mod, N, L, den):
    """Eq. 2 on the 1/r grid = rN * irfft of the r-times zero-padded spectrum,
    with the DC bin doubled (and, for r = 1, the Nyquist bin doubled)."""
    r = den
    taus = oracle_mod.grid(L, den)
    W = oracle_mod.build_W(N, taus)
    rng = np.random.default_rng(N + L + den)
    B = N // 2 + 1
    x = np.exp(1j * rng.uniform(0, 2 * np.pi, B))
    x[0] = np.sign(rng.standard_normal())  # real DC / Nyquist as for real signals
    x[-1] = np.sign(rng.standard_normal())
    y = oracle_mod.correlate(W, x)
    spec = np.zeros(r * N // 2 + 1, complex)
    spec[:B] = x
    spec[0] *= 2
    if r == 1:
        spec[-1] *= 2
    g = r * N * np.fft.irfft(spec, r * N)
    m = np.round(taus * r).astype(int) % (r * N)
    assert np.allclose(y, g[m], atol=1e-10 * N)


def test_phat_definition(oracle_mod):
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((3, 33)) + 1j * rng.standard_normal((3, 33))).astype(np.complex64)
    X[1, 5] = 0
    x = oracle_mod.phat(X, 0, 1)
    assert x[5] == 0
    mask = np.arange(33) != 5
    assert np.allclose(np.abs(x[mask]), 1.0, atol=1e-12)
    ref = X[0].astype(complex) * np.conj(X[1].astype(complex))
    assert np.allclose(x[mask], ref[mask] / np.abs(ref[mask]), atol=1e-12)


@pytest.mark.parametrize("N", [8, 16])
def test_brute_force_time_domain(oracle_mod, N):
    """Tiny N, integer lags, real signals: the direct O(N^2) circular
    cross-correlation of the whitened signals gives eq. 2 up to the DC/Nyquist
    terms that eq. 2 counts twice."""
    rng = np.random.default_rng(N)
    M = 3
    xt = rng.standard_normal((M, N))
    X = np.fft.rfft(xt, axis=-1).astype(np.complex64)[None]  # [1, M, B]
    L = N // 2 - 1
    taus = oracle_mod.grid(L, 1)
    W = oracle_mod.build_W(N, taus)
    _, _, _, y = oracle_mod.tdoa(X, W, taus, 1.0, want_y=True)
    p = 0
    for i in range(M):
        for j in range(i + 1, M):
            X64 = X[0].astype(complex)
            u = X64 / np.abs(X64)
            wi, wj = np.fft.irfft(u[i], N), np.fft.irfft(u[j], N)
            R0 = (u[i, 0] * np.conj(u[j, 0])).real
            RN = (u[i, -1] * np.conj(u[j, -1])).real
            for k, tau in enumerate(taus.astype(int)):
                direct = N * sum(wi[n] * wj[(n - tau) % N] for n in range(N))
                assert abs(direct - (y[0, p, k] - R0 - RN * (1 - 2 * (tau % 2)))) < 1e-9
            p += 1


def test_pure_delay_peak(oracle_mod):
    """X_j delayed by D relative to X_i: y peaks at tau = -D... in the
    tau_ij = t_i - t_j convention, i.e. at delta_i - delta_j, with value N + 2."""
    N = 512
    b = oracle_mod.Basis(N, 3, 4)
    B = N // 2 + 1
    f = np.arange(B)
    rng = np.random.default_rng(5)
    S = rng.standard_normal(B) + 1j * rng.standard_normal(B)
    for D in [-2.75, -1.0, 0.0, 0.5, 1.25, 3.0]:
        X = np.stack([S, S * np.exp(-2j * np.pi * f * D / N)])[None].astype(np.complex64)
        idx, peak, tau, _ = oracle_mod.tdoa(X, b.W, b.taus, b.delta)
        assert b.taus[idx[0, 0]] == -D
        assert abs(peak[0, 0] - (N + 2)) < 1e-3
        assert abs(tau[0, 0] + D) < 1e-9
        idx_k, _, _, _ = oracle_mod.tdoa(X, b.WK, b.taus, b.delta)
        assert idx_k[0, 0] == idx[0, 0]


def test_pair_reversal_symmetry(oracle_mod):
    """r_ij(tau) = r_ji(-tau) at rank K (the grid is symmetric)."""
    b = oracle_mod.Basis(512, 5, 4)
    rec = synth.time_domain_spectra(synth.circular_array(8, 0.05), 16000, 512, 256, 4000, 3)
    X = rec.spectra[4]
    for (i, j) in [(0, 3), (2, 7), (5, 6)]:
        yij = oracle_mod.correlate(b.WK, oracle_mod.phat(X, i, j))
        yji = oracle_mod.correlate(b.WK, oracle_mod.phat(X, j, i))
        assert np.allclose(yij, yji[::-1], atol=1e-9 * np.abs(yij).max())


def test_pipeline_pair_order(oracle_mod):
    """Pairs come out lexicographically (i < j) and match the step functions."""
    b = oracle_mod.Basis(512, 3, 4)
    rec = synth.config_small_square(1)
    X = rec.spectra[:5]
    idx, peak, tau, y = oracle_mod.tdoa(X, b.WK, b.taus, b.delta, want_y=True)
    p = 0
    for i in range(4):
        for j in range(i + 1, 4):
            for t in range(5):
                yy = oracle_mod.correlate(b.WK, oracle_mod.phat(X[t], i, j))
                assert np.allclose(y[t, p], yy, atol=1e-12)
                k = oracle_mod.argmax(yy)
                assert idx[t, p] == k and peak[t, p] == yy[k]
            p += 1


def test_argmax_lowest_index_on_ties(oracle_mod):
    assert oracle_mod.argmax(np.array([1.0, 3.0, 2.0, 3.0])) == 1
    assert oracle_mod.argmax(np.array([5.0, 5.0])) == 0


def test_parabola(oracle_mod):
    taus = np.arange(-3, 3.25, 0.25)
    for t0 in [-0.6, 0.1, 1.37, 2.5]:
        y = -(taus - t0) ** 2 + 7.0
        k = int(np.argmax(y))
        assert abs(oracle_mod.parabola(y, k, taus[k], 0.25) - t0) < 1e-12
    y = -(taus + 3.1) ** 2
    assert oracle_mod.parabola(y, 0, taus[0], 0.25) == taus[0]  # grid edge
    flat = np.ones_like(taus)
    assert oracle_mod.parabola(flat, 5, taus[5], 0.25) == taus[5]  # not concave


def test_config_small_square_recovers_direction(oracle_mod):
    """The 20 dB single-source recording: FCC TDoAs match the true delays."""
    rec = synth.config_small_square(1)
    assert rec.spectra.shape == (61, 4, 257)
    L = synth.lag_extent(rec.xyz, rec.fs)
    assert L == 3
    b = oracle_mod.Basis(512, L, 4)
    assert b.K == 6
    idx, peak, tau, _ = oracle_mod.tdoa(rec.spectra, b.WK, b.taus, b.delta)
    p = 0
    for i in range(4):
        for j in range(i + 1, 4):
            true = rec.delays[i] - rec.delays[j]
            assert np.median(np.abs(tau[:, p] - true)) < 0.2
            p += 1
