"""Pins of the seeded input generators (paper_2204_13622_gb300/synth.py) to the
recipes they state: far-field phase ramps from a direction in the upper
hemisphere, a pink (1/f power) source spectrum, the SNR as the scale of the
added noise, on/off gating with pauses, the learned head's known TDoA, and
the batched workload's draws and totals.  CPU only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_13622_gb300 import synth  # noqa: E402

FS, C = 16000.0, 343.0


def _delay_differences(X):
    """Per microphone m, d_m - d_0 (samples) from the per-bin phase step of
    X_m / X_0 = exp(-j 2 pi f (d_m - d_0) / N), averaged over frames and bins."""
    N = 2 * (X.shape[-1] - 1)
    r = X / X[:, :1, :]
    step = (r[:, :, 1:] * np.conj(r[:, :, :-1])).mean(axis=(0, 2))
    return -np.angle(step) * N / (2 * np.pi), r


def _three_d_array():
    # six mics on a 5 cm circle plus two off the plane, so that the direction's
    # z component is observable
    xyz = synth.circular_array(6, 0.05)
    return np.vstack([xyz, [[0.0, 0.0, 0.03], [0.01, -0.01, -0.03]]])


def test_stft_domain_far_field_geometry():
    xyz = _three_d_array()
    # one source, no noise to speak of; 100 frames at hop 128 stay inside one
    # 1-s segment, so one direction
    X = synth.stft_domain_spectra(100, xyz, FS, 512, 128, seed=5, max_sources=1,
                                  snr_db=(200.0, 200.0)).numpy().astype(np.complex128)
    dd, r = _delay_differences(X)
    # a pure phase transfer: equal magnitudes at every microphone
    assert np.abs(np.abs(r) - 1.0).max() < 1e-5
    # d_m = -(fs / c) r_m . u for one unit vector u with u_z >= 0 (elevation in [0, pi/2])
    A = xyz[1:] - xyz[:1]
    u, *_ = np.linalg.lstsq(A, -(C / FS) * dd[1:], rcond=None)
    assert np.abs(A @ u + (C / FS) * dd[1:]).max() < 1e-5 * C / FS
    assert abs(np.linalg.norm(u) - 1.0) < 1e-4
    assert u[2] >= -1e-4


def test_stft_domain_pink_spectrum():
    xyz = synth.circular_array(4, 0.05)
    X = synth.stft_domain_spectra(3000, xyz, FS, 512, 128, seed=6, max_sources=1,
                                  snr_db=(200.0, 200.0)).numpy()
    P = (np.abs(X[:, 0, :]) ** 2).mean(axis=0)
    f = np.arange(2, 257)
    slope = np.polyfit(np.log(f), np.log(P[f]), 1)[0]
    assert abs(slope + 1.0) < 0.05, slope
    # unit mean power over the bins
    assert abs(P.mean() - 1.0) < 0.05


@pytest.mark.parametrize("snr", [0.0, 10.0])
def test_stft_domain_snr_is_the_noise_scale(snr):
    # the same seed draws the same sources and noise; only the noise scale differs
    xyz = synth.circular_array(4, 0.05)
    clean = synth.stft_domain_spectra(500, xyz, FS, 512, 128, seed=7, max_sources=1,
                                      snr_db=(200.0, 200.0)).numpy().astype(np.complex128)
    noisy = synth.stft_domain_spectra(500, xyz, FS, 512, 128, seed=7, max_sources=1,
                                      snr_db=(snr, snr)).numpy().astype(np.complex128)
    p_sig = (np.abs(clean) ** 2).mean()
    p_noise = (np.abs(noisy - clean) ** 2).mean()
    assert abs(10 * np.log10(p_sig / p_noise) - snr) < 0.1


def test_stft_domain_gating_and_seeding():
    xyz = synth.circular_array(8, 0.05)
    X = synth.stft_domain_spectra(2000, xyz, FS, 512, 128, seed=8, snr_db=(200.0, 200.0)).numpy()
    p = (np.abs(X) ** 2).mean(axis=(1, 2))
    # frames whose segment's sources are all in an off run carry noise alone (a
    # pause); most frames carry at least one source, some several
    quiet = p < 1e-6
    assert 0.05 < quiet.mean() < 0.30, quiet.mean()
    assert p[~quiet].min() > 0.05
    assert p.max() > 1.5 * np.median(p[~quiet])
    again = synth.stft_domain_spectra(2000, xyz, FS, 512, 128, seed=8, snr_db=(200.0, 200.0)).numpy()
    assert np.array_equal(X, again)
    other = synth.stft_domain_spectra(50, xyz, FS, 512, 128, seed=9, snr_db=(200.0, 200.0)).numpy()
    assert not np.array_equal(X[:50], other)


def test_pair_delay_spectra_known_tdoa_and_chunking():
    N, tau_max = 512, 4.66
    X, t, snr = synth.pair_delay_spectra(300, N, tau_max, seed=11, snr_db=(200.0, 200.0))
    X = X.numpy().astype(np.complex128)
    assert np.all(np.abs(t) <= tau_max)
    # mic 1 = mic 0 times exp(+j 2 pi f t / N): the phase step per bin gives t back
    r = X[:, 1, :] / X[:, 0, :]
    step = (r[:, 1:] * np.conj(r[:, :-1])).mean(axis=1)
    assert np.abs(np.angle(step) * N / (2 * np.pi) - t).max() < 1e-4
    # blocks of 2^16 make chunked generation equal to one call
    a, ta, _ = synth.pair_delay_spectra(100, N, tau_max, seed=12)
    b1, tb1, _ = synth.pair_delay_spectra(60, N, tau_max, seed=12)
    b2, tb2, _ = synth.pair_delay_spectra(40, N, tau_max, seed=12, start=60)
    assert np.array_equal(ta, np.concatenate([tb1, tb2]))
    assert (a - torch.cat([b1, b2])).abs().max() <= 2.4e-7  # float32 rounding of the ramp


def test_batched_arrays_recipe_and_totals():
    arrs = synth.batched_arrays(4096, 4)
    assert {a["n_mics"] for a in arrs} == {2, 4, 6, 8, 12, 16}
    assert {a["N"] for a in arrs} == {256, 512, 1024}
    assert {a["fs"] for a in arrs} == {16000.0, 48000.0}
    assert all(64 <= a["T"] <= 4096 and a["lag_den"] == 4 for a in arrs)
    # aperture = the circle's diameter, uniform in 2..8 cm (the largest pair
    # distance equals the diameter for an even microphone count)
    d = np.array([synth.max_distance(a["mic_xyz"]) for a in arrs])
    assert d.min() >= 0.02 - 1e-12 and d.max() <= 0.08 + 1e-12
    # the totals the benchmark's batched workload is quoted with
    T = sum(a["T"] for a in arrs)
    pf = sum(a["T"] * a["n_mics"] * (a["n_mics"] - 1) // 2 for a in arrs)
    nbytes = sum(a["T"] * a["n_mics"] * (a["N"] // 2 + 1) * 8 for a in arrs)
    assert (T, pf) == (8670813, 354008202) and abs(nbytes / 1e9 - 169.798) < 1e-3


def test_array_spectra_far_field():
    arr = dict(synth.batched_arrays(3, 21)[1])
    arr["T"] = 40
    X = synth.array_spectra(arr, snr_db=(200.0, 200.0)).numpy().astype(np.complex128)
    dd, r = _delay_differences(X)
    assert np.abs(np.abs(r) - 1.0).max() < 1e-5
    xyz = arr["mic_xyz"]
    A = (xyz[1:] - xyz[:1])[:, :2]  # a planar array: the in-plane part of u
    u, *_ = np.linalg.lstsq(A, -(C / arr["fs"]) * dd[1:], rcond=None)
    assert np.abs(A @ u + (C / arr["fs"]) * dd[1:]).max() < 1e-5 * C / arr["fs"]
    assert np.linalg.norm(u) <= 1.0 + 1e-4


def test_pcm_far_field_integer_delays_and_int16_scale():
    xyz = synth.circular_array(4, 0.05)
    n = 4000
    x = synth.pcm_far_field(n, xyz, FS, seed=3, segment=n, snr_db=200.0, kind="f32").numpy()
    L = synth.lag_extent(xyz, FS) + 1
    lags = []
    for m in range(1, 4):
        # channel m is channel 0 shifted by a whole number of samples, |shift| <= L
        hit = [k for k in range(-L, L + 1)
               if np.allclose(x[L + k:n - L + k, m], x[L:n - L, 0], rtol=0, atol=1e-6)]
        assert len(hit) == 1
        lags.append(hit[0])
    assert any(k != 0 for k in lags)
    # int16 PCM is the same draw scaled by 6000, rounded and clipped
    s16 = synth.pcm_far_field(n, xyz, FS, seed=3, segment=n, snr_db=200.0, kind="s16").numpy()
    assert s16.dtype == np.int16
    ref = np.clip(np.round(x * np.float32(6000.0)), -32768, 32767).astype(np.int16)  # FP32, as generated
    assert np.array_equal(s16, ref)
