"""Pins of the oracle's second basis split ("form B": C = Re W on cosine bases,
S = Im W on sine bases, each truncated by its own SVD; y_B = 2 Re{(C_K + j S_K) x}).
Pinned by: full rank reproduces W itself (hence Eq. 2), the singular values
and Eckart-Young residuals against LAPACK, the energy rule recomputed from
LAPACK's values, and the parity of the kept U vectors in tau (C even, S odd),
which the GPU's symmetric reconstruction relies on."""
import numpy as np
import pytest


@pytest.mark.parametrize("N,L,den", [(64, 3, 4), (512, 5, 4), (256, 3, 2)])
def test_form_b_against_lapack(oracle_mod, N, L, den):
    O = oracle_mod
    b = O.BasisB(N, L, den)
    W = O.build_W(N, b.taus)
    for A, s, K in ((W.real, b.sc, b.Kc), (W.imag, b.ss, b.Ks)):
        ref = np.linalg.svd(A, compute_uv=False)
        r = min(len(ref), len(s))
        assert np.allclose(s[:r], ref[:r], rtol=0, atol=1e-12 * ref[0])
        # the energy rule from LAPACK's values
        e = np.cumsum(ref ** 2) / np.sum(ref ** 2)
        assert K == int(np.argmax(e >= 0.999 - 1e-15)) + 1
    # Eckart-Young: ||C - C_K||_F^2 = sum_{k > K} s_k^2, likewise S
    for A, AK, K in ((W.real, b.CK, b.Kc), (W.imag, b.SK, b.Ks)):
        ref = np.linalg.svd(A, compute_uv=False)
        assert abs(np.sum((A - AK) ** 2) - np.sum(ref[K:] ** 2)) <= 1e-10 * np.sum(ref ** 2)


def test_full_rank_is_w(oracle_mod):
    # I = 25 lags: C and S have rank <= 25, so K = 25 keeps all of each and gives W back
    O = oracle_mod
    full = O.BasisB(128, 3, 4, Kc=25, Ks=25)
    W = O.build_W(128, full.taus)
    assert np.abs(full.WK - W).max() < 1e-10


def test_u_parity(oracle_mod):
    # C(-tau) = C(tau) and S(-tau) = -S(tau): kept left vectors are even / odd in tau
    O = oracle_mod
    b = O.BasisB(512, 5, 4)
    I = b.I
    for k in range(b.Kc):
        u = b.Uc[:, k]
        assert np.abs(u[::-1] - u).max() < 1e-9 * np.abs(u).max()
    for k in range(b.Ks):
        u = b.Us[:, k]
        assert np.abs(u[::-1] + u).max() < 1e-9 * np.abs(u).max()
    assert I == 41
