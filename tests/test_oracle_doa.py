"""Pins of the oracle's DoA search over direction candidates (the next step
named in the paper's conclusion: use every pair's correlation to find the best
DoA candidate).  The paper prints no formula; the oracle reads each pair's
correlation at the candidate's TDoA by linear interpolation on the lag grid and
sums over pairs.  Pinned by: a linear correlation whose interpolation is exact
(closed form in the candidate's direction cosine), on-grid lookups, clamping at
the grid's ends, linearity in y, the tie rule, and a far-field source found by
the FCC oracle's own full-rank correlations."""
import math

import numpy as np

from paper_2204_13622_gb300 import synth

FS, C = 16000.0, 343.0


def _two_mics(d):
    return np.array([[-d / 2, 0.0, 0.0], [d / 2, 0.0, 0.0]])


def test_linear_correlation_gives_the_direction_cosine(oracle_mod):
    # y(tau) = tau is reproduced exactly by linear interpolation, and for mics at
    # -d/2 and +d/2 on x a plane wave from u reaches mic 0 later by (fs d / c) u_x
    O = oracle_mod
    L, den = 4, 4
    taus = -L + np.arange(2 * L * den + 1) / den
    d = 0.08  # fs d / c = 3.73 < L: never clamped
    dirs = synth.fibonacci_directions(200, hemisphere=False)
    y = np.broadcast_to(taus, (3, 1, len(taus))).copy()
    idx, best, scores = O.doa_srp(y, L, den, _two_mics(d), FS, C, dirs, want_scores=True)
    expect = FS * d / C * dirs[:, 0]
    assert np.allclose(scores, expect[None, :], rtol=0, atol=1e-12)
    assert np.all(idx == np.argmax(dirs[:, 0]))
    assert np.allclose(best, expect.max(), rtol=0, atol=1e-12)


def test_on_grid_lookups_and_clamping(oracle_mod):
    O = oracle_mod
    L, den = 3, 4
    I = 2 * L * den + 1
    center = L * den
    rng = np.random.default_rng(5)
    y = rng.standard_normal((4, 1, I))
    d = 2.0 * C / FS  # fs d / c = 2 samples exactly
    dirs = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 0, 1.0], [0, 1.0, 0]])
    _, _, s = O.doa_srp(y, L, den, _two_mics(d), FS, C, dirs, want_scores=True)
    # u = +x: mic 0 (at -d/2) hears 2 samples later: tau_01 = +2
    assert np.allclose(s[:, 0], y[:, 0, center + 2 * den], rtol=0, atol=1e-13)
    assert np.allclose(s[:, 1], y[:, 0, center - 2 * den], rtol=0, atol=1e-13)
    assert np.allclose(s[:, 2], y[:, 0, center], rtol=0, atol=1e-13)
    assert np.allclose(s[:, 3], y[:, 0, center], rtol=0, atol=1e-13)
    # a 5-sample baseline exceeds L = 3: the lookups clamp to the grid's ends
    _, _, s2 = O.doa_srp(y, L, den, _two_mics(5.0 * C / FS), FS, C, dirs[:2], want_scores=True)
    assert np.allclose(s2[:, 0], y[:, 0, I - 1], rtol=0, atol=1e-13)
    assert np.allclose(s2[:, 1], y[:, 0, 0], rtol=0, atol=1e-13)


def test_linearity_and_ties(oracle_mod):
    O = oracle_mod
    L, den = 5, 4
    xyz = synth.circular_array(6, 0.05)
    P, I = 15, 2 * L * den + 1
    rng = np.random.default_rng(8)
    y1, y2 = rng.standard_normal((3, P, I)), rng.standard_normal((3, P, I))
    dirs = synth.fibonacci_directions(50)
    _, _, s1 = O.doa_srp(y1, L, den, xyz, FS, C, dirs, want_scores=True)
    _, _, s2 = O.doa_srp(y2, L, den, xyz, FS, C, dirs, want_scores=True)
    _, _, s12 = O.doa_srp(y1 + 2.5 * y2, L, den, xyz, FS, C, dirs, want_scores=True)
    assert np.allclose(s12, s1 + 2.5 * s2, rtol=0, atol=1e-12)
    # a repeated candidate never displaces the first copy
    best = np.argmax(s1, axis=1)
    for t in range(3):
        d3 = np.concatenate([dirs[best[t]][None], dirs, dirs[best[t]][None]])
        i, sc, _ = O.doa_srp(y1[t:t + 1], L, den, xyz, FS, C, d3)
        assert i[0] == 0 and math.isclose(sc[0], s1[t, best[t]], rel_tol=0, abs_tol=1e-12)


def test_far_field_source_is_found(oracle_mod):
    # pure far-field delays built in the frequency domain, full-rank correlations
    # from the FCC oracle (Eq. 2), then the search over 64 hemisphere candidates
    O = oracle_mod
    N, den = 512, 4
    xyz = synth.circular_array(8, 0.05)
    L = synth.lag_extent(xyz, FS)
    basis = O.Basis(N, L, den)
    dirs = synth.fibonacci_directions(64)
    f = np.arange(N // 2 + 1)
    for k in (5, 17, 40, 63):
        delta = synth.far_field_delays(xyz, dirs[k], FS)
        X = np.exp(-2j * np.pi * np.outer(delta, f) / N)[None].astype(np.complex64)
        _, _, _, y = O.tdoa(X, basis.W, basis.taus, basis.delta, want_y=True)
        idx, score, _ = O.doa_srp(y, L, den, xyz, FS, C, dirs)
        assert idx[0] == k
        # every pair's correlation peaks at N + 2 exactly at its own TDoA, and the
        # interpolated reads sit a little below it
        assert 0.9 * 28 * (N + 2) < score[0] <= 28 * (N + 2) + 1e-9
