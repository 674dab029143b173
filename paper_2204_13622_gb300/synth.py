"""Seeded synthetic microphone-array spectra.

This module only makes inputs: array geometries, far-field sources with
fractional delays, additive noise and an STFT front-end.  It contains none of
the FCC method's arithmetic (no phase transform, no correlation, no bases), so
that both the CUDA path and the FP64 oracle can be fed the same bytes.

Two generators:

* :func:`time_domain_spectra` -- the front-end of Sec. 2 done literally: a time
  signal per microphone (white Gaussian source, fractional delays applied as a
  phase ramp on a zero-padded FFT of the whole signal, white noise at a given
  SNR), then a periodic-Hann STFT with frame N and hop N/2 (50 % overlap).
* :func:`stft_domain_spectra` -- for large frame counts: sources drawn directly
  in the STFT domain (complex Gaussian shaped to a pink 1/f power spectrum,
  random on/off envelopes of 20-200 ms), each delayed per microphone by the
  exact phase ramp exp(-j 2 pi f delay / N), plus white noise at a per-segment
  SNR.  Runs on any torch device, chunked, so 17 GB tensors can be made on
  the GPU.

Delay convention: a microphone at position r hears a far-field source in unit
direction u at time offset delay = -fs (r . u) / c samples (closer = earlier).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SPEED_OF_SOUND = 343.0


# ----------------------------------------------------------------------------
# geometries
# ----------------------------------------------------------------------------
def square_array(side: float) -> np.ndarray:
    """Four mics on the corners of a square of the given side (metres)."""
    a = side / 2.0
    return np.array([[a, a, 0.0], [-a, a, 0.0], [-a, -a, 0.0], [a, -a, 0.0]])


def circular_array(n_mics: int, radius: float) -> np.ndarray:
    """Uniform circular array, mic m at angle 2 pi m / n_mics."""
    ang = 2.0 * np.pi * np.arange(n_mics) / n_mics
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n_mics)], axis=1)


def grid_array(nx: int, ny: int, pitch: float) -> np.ndarray:
    """nx x ny planar grid with the given pitch, centred on the origin."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    return np.array([[x, y, 0.0] for y in ys for x in xs])


def max_distance(xyz: np.ndarray) -> float:
    d = xyz[:, None, :] - xyz[None, :, :]
    return float(np.sqrt((d ** 2).sum(-1)).max())


def lag_extent(xyz: np.ndarray, fs: float, c: float = SPEED_OF_SOUND) -> int:
    """L = ceil(d_max fs / c): the integer lag half-range that holds every pair."""
    return int(math.ceil(max_distance(xyz) * fs / c - 1e-9))


def unit_vector(azimuth: float, elevation: float = 0.0) -> np.ndarray:
    return np.array([math.cos(elevation) * math.cos(azimuth),
                     math.cos(elevation) * math.sin(azimuth), math.sin(elevation)])


def fibonacci_directions(n: int, hemisphere: bool = True) -> np.ndarray:
    """n quasi-uniform unit vectors on the sphere (Fibonacci lattice), [n, 3];
    z in (0, 1) for the upper hemisphere (enough for a planar array, whose
    delays cannot tell z from -z), else in (-1, 1)."""
    k = np.arange(n) + 0.5
    z = 1.0 - k / n if hemisphere else 1.0 - 2.0 * k / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * k
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def pcm_far_field(n_samples: int, xyz: np.ndarray, fs: float, seed: int, device="cpu", segment: int = 16000,
                  snr_db: float = 10.0, kind: str = "s16", c: float = SPEED_OF_SOUND):
    """Interleaved multichannel PCM [n_samples, M] (int16 or float32): per
    segment of `segment` samples one far-field white source from a seeded
    random direction (azimuth U[0, 2 pi), elevation U[0, pi/2]), seen by each
    mic with its delay rounded to whole samples, plus white noise at `snr_db`.
    Generated with torch on `device`."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    M = xyz.shape[0]
    n_seg = (n_samples + segment - 1) // segment
    az = torch.rand(n_seg, generator=g, dtype=torch.float64) * 2 * math.pi
    el = torch.rand(n_seg, generator=g, dtype=torch.float64) * math.pi / 2
    u = torch.stack([torch.cos(el) * torch.cos(az), torch.cos(el) * torch.sin(az), torch.sin(el)], 1)
    d = torch.round(-fs * (u @ torch.from_numpy(np.asarray(xyz, np.float64)).T) / c).to(torch.int64)  # [n_seg, M]
    pad = int(d.abs().max()) + 1
    gd = torch.Generator(device=device).manual_seed(int(seed) + 1)
    src = torch.randn(n_samples + 2 * pad, generator=gd, device=device)
    seg = torch.arange(n_samples, device=device) // segment
    out = torch.empty((n_samples, M), dtype=torch.int16 if kind == "s16" else torch.float32, device=device)
    amp_n = 10.0 ** (-snr_db / 20.0)
    dd = d.to(device)
    for m in range(M):
        x = src[torch.arange(n_samples, device=device) + pad - dd[seg, m]]
        x = x + amp_n * torch.randn(n_samples, generator=gd, device=device)
        if kind == "s16":
            out[:, m] = torch.clamp(torch.round(x * 6000.0), -32768, 32767).to(torch.int16)
        else:
            out[:, m] = x
    return out


def image_source_rir(room, src, mics, beta: float, fs: float, c: float, t_max: float, taps: int = 32,
                     device="cpu"):
    """Room impulse responses of a shoebox room by the image-source method
    (Allen and Berkley, 1979): every image of the source in the six walls whose
    delay is below t_max, with amplitude beta^(number of wall reflections) /
    (4 pi r) (one reflection coefficient for all walls), placed at its
    fractional delay r fs / c by a Hann-windowed sinc of 2 taps + 1 samples.
    room [3] (m, corner at the origin), src [3], mics [M, 3].  Returns [M, n]
    float32 (torch, on `device`), n = ceil(t_max fs) + taps + 1."""
    import torch
    room = np.asarray(room, np.float64)
    src = np.asarray(src, np.float64)
    mics = np.asarray(mics, np.float64).reshape(-1, 3)
    n_out = int(math.ceil(t_max * fs)) + taps + 1
    reach = c * t_max
    axes = []
    for a in range(3):
        nmax = int(math.ceil(reach / (2 * room[a]))) + 1
        n = np.arange(-nmax, nmax + 1)
        pos = np.concatenate([src[a] + 2 * n * room[a], -src[a] + 2 * n * room[a]])
        refl = np.concatenate([np.abs(n) + np.abs(n), np.abs(n - 1) + np.abs(n)])
        axes.append((torch.tensor(pos, device=device), torch.tensor(refl, device=device)))
    (px, rx), (py, ry), (pz, rz) = axes
    order = (rx[:, None, None] + ry[None, :, None] + rz[None, None, :]).reshape(-1).double()
    out = torch.zeros((mics.shape[0], n_out), dtype=torch.float64, device=device)
    k = torch.arange(-taps, taps + 1, device=device, dtype=torch.float64)
    for m in range(mics.shape[0]):
        d2 = ((px - mics[m, 0]) ** 2)[:, None, None] + ((py - mics[m, 1]) ** 2)[None, :, None] \
            + ((pz - mics[m, 2]) ** 2)[None, None, :]
        dist = torch.sqrt(d2.reshape(-1))
        keep = dist < reach
        dist, o = dist[keep], order[keep]
        amp = torch.pow(torch.tensor(beta, dtype=torch.float64, device=device), o) / (4 * math.pi * dist)
        delay = dist * fs / c
        base = torch.floor(delay)
        idx = base[:, None] + k[None, :]
        x = idx - delay[:, None]  # distance of each tap to the image's delay; the window is centred there
        w = torch.sinc(x) * (0.5 + 0.5 * torch.cos(math.pi * x / (taps + 1))) * amp[:, None]
        valid = (idx >= 0) & (idx < n_out)
        out[m].index_add_(0, idx[valid].long(), w[valid])
    return out.float()


def far_field_delays(xyz: np.ndarray, direction: np.ndarray, fs: float,
                     c: float = SPEED_OF_SOUND) -> np.ndarray:
    """Per-mic delay (samples) of a far-field source from `direction`."""
    return -fs * (xyz @ direction) / c


# ----------------------------------------------------------------------------
# time-domain path (small inputs)
# ----------------------------------------------------------------------------
def stft(x: np.ndarray, N: int, hop: int) -> np.ndarray:
    """Periodic-Hann STFT without centre padding: [n_ch, L] -> [T, n_ch, N/2+1]."""
    n_ch, L = x.shape
    T = 1 + (L - N) // hop
    win = 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(N) / N)
    idx = np.arange(T)[:, None] * hop + np.arange(N)[None, :]
    frames = x[:, idx] * win  # [n_ch, T, N]
    return np.ascontiguousarray(np.fft.rfft(frames, axis=-1).transpose(1, 0, 2))


@dataclass
class Recording:
    spectra: np.ndarray  # complex64 [T, M, N/2+1]
    xyz: np.ndarray
    fs: float
    N: int
    hop: int
    delays: np.ndarray  # per-mic delays of the (first) source, samples
    meta: dict = field(default_factory=dict)


def time_domain_spectra(xyz: np.ndarray, fs: float, N: int, hop: int, n_samples: int,
                        seed: int, snr_db: float = 20.0, azimuth: float | None = None,
                        elevation: float = 0.0, c: float = SPEED_OF_SOUND) -> Recording:
    """One far-field white-Gaussian source plus white noise, then the STFT."""
    rng = np.random.default_rng(seed)
    if azimuth is None:
        azimuth = float(rng.uniform(0.0, 2.0 * np.pi))
    delays = far_field_delays(xyz, unit_vector(azimuth, elevation), fs, c)
    src = rng.standard_normal(n_samples)
    nfft = 1 << int(math.ceil(math.log2(2 * n_samples)))
    S = np.fft.rfft(src, nfft)
    k = np.arange(nfft // 2 + 1)
    sig = np.stack([np.fft.irfft(S * np.exp(-2j * np.pi * k * d / nfft), nfft)[:n_samples]
                    for d in delays])
    noise = rng.standard_normal(sig.shape) * (sig.std() * 10.0 ** (-snr_db / 20.0))
    X = stft(sig + noise, N, hop).astype(np.complex64)
    return Recording(X, xyz, fs, N, hop, delays, dict(azimuth=azimuth, snr_db=snr_db))


def config_small_square(seed: int = 1) -> Recording:
    """4-mic square (4.5 cm side), fs 16 kHz, N 512 / hop 256, 1 s, 20 dB SNR."""
    return time_domain_spectra(square_array(0.045), 16000.0, 512, 256, 16000, seed, 20.0)


# ----------------------------------------------------------------------------
# STFT-domain path (large inputs, any torch device)
# ----------------------------------------------------------------------------
def stft_domain_spectra(T: int, xyz: np.ndarray, fs: float, N: int, hop: int, seed: int,
                        device="cpu", out=None, max_sources: int = 3,
                        snr_db: tuple = (0.0, 30.0), segment_s: float = 1.0,
                        onoff_ms: tuple = (20.0, 200.0), chunk: int | None = None,
                        c: float = SPEED_OF_SOUND):
    """Spectra [T, M, N/2+1] complex64 made directly in the STFT domain.

    Per 1-s segment: 1..max_sources sources with uniform azimuth in [0, 2 pi)
    and elevation in [0, pi/2], and an SNR uniform in `snr_db`.  Each source is
    complex Gaussian with a pink (1/f power) spectral shape, gated by on/off
    runs whose lengths are uniform in `onoff_ms`.  Microphone m sees source s
    through exp(-j 2 pi f delay_{m,s} / N).  Deterministic for a given seed and
    device.
    """
    import torch

    M = xyz.shape[0]
    B = N // 2 + 1
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    frames_per_seg = max(1, int(round(segment_s * fs / hop)))
    n_seg = (T + frames_per_seg - 1) // frames_per_seg
    # per-segment scene, drawn on the host (small)
    n_src = rng.integers(1, max_sources + 1, size=n_seg)
    az = rng.uniform(0.0, 2.0 * np.pi, size=(n_seg, max_sources))
    el = rng.uniform(0.0, np.pi / 2.0, size=(n_seg, max_sources))
    snr = rng.uniform(snr_db[0], snr_db[1], size=n_seg)
    u = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], axis=-1)
    delays = -fs * np.einsum("mk,gsk->gsm", xyz, u) / c  # [n_seg, S, M]
    active = (np.arange(max_sources)[None, :] < n_src[:, None]).astype(np.float32)
    # on/off envelope per source, in frames
    frame_ms = 1000.0 * hop / fs
    env = np.zeros((max_sources, T), np.float32)
    for s in range(max_sources):
        pos, on = 0, bool(rng.integers(0, 2))
        while pos < T:
            run = max(1, int(round(rng.uniform(*onoff_ms) / frame_ms)))
            if on:
                env[s, pos:pos + run] = 1.0
            pos += run
            on = not on
    # where every envelope is off, source 0's is turned on; a frame in which every
    # source active in its segment is in an off run still carries noise alone
    # (about 16 % of frames with three envelopes), like a pause in speech
    env[0, env.sum(0) == 0] = 1.0

    delays_t = torch.tensor(delays, dtype=torch.float64, device=dev)
    active_t = torch.tensor(active, device=dev)
    noise_amp_t = torch.tensor(10.0 ** (-snr / 20.0), dtype=torch.float32, device=dev)
    env_t = torch.tensor(env, device=dev)
    f = torch.arange(B, device=dev, dtype=torch.float64)
    pink = (1.0 / torch.sqrt(torch.clamp(f, min=1.0))).to(torch.float32)
    pink = pink / torch.sqrt((pink ** 2).mean())
    if out is None:
        out = torch.empty((T, M, B), dtype=torch.complex64, device=dev)
    if chunk is None:  # keep each float64 temporary near 2^27 elements
        chunk = max(1, (1 << 27) // (max_sources * M * B))
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 7919 + 17)
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        n = t1 - t0
        seg = torch.arange(t0, t1, device=dev) // frames_per_seg  # [n]
        src = torch.randn((max_sources, n, B), dtype=torch.complex64, device=dev, generator=gen)
        src = src * pink  # [S, n, B]
        gate = env_t[:, t0:t1] * active_t[seg].T  # [S, n]
        src = src * gate[:, :, None]
        # exact phase ramp per (segment, source, mic): exp(-j 2 pi f d / N)
        d = delays_t[seg]  # [n, S, M]
        ph = (-2.0 * math.pi / N) * d[..., None] * f  # [n, S, M, B] float64
        ramp = torch.polar(torch.ones_like(ph, dtype=torch.float32), ph.to(torch.float32))
        X = torch.einsum("snb,nsmb->nmb", src, ramp)
        noise = torch.randn((n, M, B), dtype=torch.complex64, device=dev, generator=gen)
        X = X + noise * noise_amp_t[seg][:, None, None]
        out[t0:t1] = X
        del src, ramp, X, noise, ph
    return out


# ----------------------------------------------------------------------------
# learned head: two-microphone pair spectra with a known TDoA, initial weights
# ----------------------------------------------------------------------------
def pair_delay_spectra(n: int, N: int, tau_max: float, seed: int, device="cpu",
                       snr_db: tuple = (-5.0, 30.0), start: int = 0):
    """Two-microphone spectra [n, 2, N/2+1] complex64 with a known TDoA each.

    Pair-frame s draws a true TDoA t_s uniform in [-tau_max, tau_max] (samples,
    tau = t_0 - t_1 as for pair (0, 1)), an SNR uniform in `snr_db`, and a
    source that is white or pink (1/f power) with equal odds, complex Gaussian
    per bin with unit mean power.  Microphone 0 hears S(f); microphone 1 hears
    S(f) exp(+j 2 pi f t_s / N), i.e. mic 1 lags mic 0 by -t_s samples, so the
    pair's correlation peaks at tau = t_s.  Each microphone adds independent
    complex white noise of power 10^(-SNR/10).  Returns (X, t [n] float64
    numpy, snr [n] float64 numpy).  Sample s depends only on (seed, start + s)
    blocks of 2^16, so chunked generation draws the same set (equal values up
    to the last bit of float32 rounding in the phase ramp).
    """
    import torch

    B = N // 2 + 1
    dev = torch.device(device)
    X = torch.empty((n, 2, B), dtype=torch.complex64, device=dev)
    t_all = np.empty(n)
    snr_all = np.empty(n)
    f = torch.arange(B, device=dev, dtype=torch.float64)
    pink = 1.0 / torch.sqrt(torch.clamp(f, min=1.0))
    pink = (pink / torch.sqrt((pink ** 2).mean())).to(torch.float32)
    blk = 1 << 16
    s = 0
    while s < n:
        g0 = (start + s) // blk
        off = (start + s) - g0 * blk
        m = min(n - s, blk - off)
        rng = np.random.default_rng([int(seed), int(g0)])
        t = rng.uniform(-tau_max, tau_max, size=blk)[off:off + m]
        snr = rng.uniform(snr_db[0], snr_db[1], size=blk)[off:off + m]
        is_pink = rng.integers(0, 2, size=blk)[off:off + m].astype(bool)
        gen = torch.Generator(device=dev)
        gen.manual_seed(int(seed) * 1000003 + int(g0))
        src = torch.randn((blk, B), dtype=torch.complex64, device=dev, generator=gen)[off:off + m]
        noise = torch.randn((blk, 2, B), dtype=torch.complex64, device=dev, generator=gen)[off:off + m]
        shape = torch.where(torch.tensor(is_pink, device=dev)[:, None], pink[None, :],
                            torch.ones_like(pink)[None, :])
        src = src * shape
        ph = (2.0 * math.pi / N) * torch.tensor(t, dtype=torch.float64, device=dev)[:, None] * f
        ramp = torch.polar(torch.ones_like(ph, dtype=torch.float32), ph.to(torch.float32))
        amp = torch.tensor(10.0 ** (-snr / 20.0), dtype=torch.float32, device=dev)[:, None]
        X[s:s + m, 0] = src + noise[:, 0] * amp
        X[s:s + m, 1] = src * ramp + noise[:, 1] * amp
        t_all[s:s + m] = t
        snr_all[s:s + m] = snr
        s += m
    return X, t_all, snr_all


def mlp_init_params(n_in: int, hidden: int, seed: int) -> np.ndarray:
    """Initial parameters of the learned head, packed W1[H][n_in], b1[H],
    W2[H][H], b2[H], W3[2][H], b3[2]: weights uniform in +-1/sqrt(fan_in),
    biases zero.  float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((hidden, n_in), (hidden, hidden), (2, hidden)):
        a = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-a, a, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


# ----------------------------------------------------------------------------
# batched form: many independent arrays
# ----------------------------------------------------------------------------
def batched_arrays(n: int, seed: int, mics=(2, 4, 6, 8, 12, 16), aperture=(0.02, 0.08),
                   Ns=(256, 512, 1024), rates=(16000.0, 48000.0), frames=(64, 4096), lag_den: int = 4):
    """Seeded descriptions of n independent arrays: per array a microphone count
    drawn from `mics`, a uniform circular array whose diameter (the aperture) is
    uniform in `aperture` metres, N from `Ns`, fs from `rates`, T uniform in
    [frames[0], frames[1]] and the lag grid step 1/lag_den.  Returns a list of
    dicts (n_mics, fs, N, lag_den, mic_xyz, T, seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for a in range(n):
        M = int(rng.choice(mics))
        ap = float(rng.uniform(*aperture))
        out.append(dict(n_mics=M, fs=float(rng.choice(rates)), N=int(rng.choice(Ns)), lag_den=int(lag_den),
                        mic_xyz=circular_array(M, ap / 2.0), T=int(rng.integers(frames[0], frames[1] + 1)),
                        seed=int(rng.integers(0, 2 ** 31))))
    return out


def array_spectra(arr: dict, device="cpu", snr_db=(0.0, 30.0), c: float = SPEED_OF_SOUND):
    """Spectra [T, M, N/2+1] complex64 of one array from `batched_arrays`: one
    far-field complex white source from a seeded direction, delayed per
    microphone by exp(-j 2 pi f delay / N), plus white noise at a seeded SNR."""
    import torch

    rng = np.random.default_rng(arr["seed"])
    xyz, fs, N, T = arr["mic_xyz"], arr["fs"], arr["N"], arr["T"]
    M, B = xyz.shape[0], N // 2 + 1
    direction = unit_vector(rng.uniform(0, 2 * np.pi), rng.uniform(0, np.pi / 2))
    d = far_field_delays(xyz, direction, fs, c)
    snr = rng.uniform(*snr_db)
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(arr["seed"]))
    f = np.arange(B)
    ramp = torch.from_numpy(np.exp(-2j * np.pi * np.outer(d, f) / N).astype(np.complex64)).to(dev)
    src = torch.randn((T, 1, B), dtype=torch.complex64, device=dev, generator=gen)
    X = torch.randn((T, M, B), dtype=torch.complex64, device=dev, generator=gen)
    X.mul_(10.0 ** (-snr / 20.0)).add_(src * ramp)
    return X
