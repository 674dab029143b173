"""Named synthetic workloads shaped like the paper's setting (inputs only).

Each names an array geometry, sample rate, frame size N, hop, lag-grid step
1/lag_den and frame count, and makes seeded spectra [T, M, N/2+1] through
:mod:`synth`.  The paper's own evaluation uses the BIRD room simulations,
which are not available here; these seeded far-field scenes stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth


@dataclass(frozen=True)
class Workload:
    name: str
    xyz: np.ndarray
    fs: float
    N: int
    hop: int
    lag_den: int
    T: int

    @property
    def M(self) -> int:
        return self.xyz.shape[0]

    @property
    def P(self) -> int:
        return self.M * (self.M - 1) // 2

    @property
    def B(self) -> int:
        return self.N // 2 + 1

    @property
    def L(self) -> int:
        return synth.lag_extent(self.xyz, self.fs)

    def spectra(self, T: int | None = None, seed: int = 2, device="cpu", out=None):
        """STFT-domain scene (pink sources with on/off gating, 0-30 dB SNR)."""
        return synth.stft_domain_spectra(self.T if T is None else T, self.xyz, self.fs, self.N,
                                         self.hop, seed, device=device, out=out)


# 4-mic square (4.5 cm side), 16 kHz, N = 512, hop 256, 1 s (61 frames), grid [-3, 3] at 1/4
SQUARE4 = Workload("square4-4.5cm-16kHz-N512-61frames", synth.square_array(0.045), 16000.0, 512,
                   256, 4, 61)
# 8-mic circle (5 cm radius), 16 kHz, N = 512, hop 128, 2^20 frames, grid [-5, 5] at 1/4
CIRCLE8 = Workload("circle8-5cm-16kHz-N512-2^20frames", synth.circular_array(8, 0.05), 16000.0, 512,
                   128, 4, 1 << 20)
# 16-mic 4x4 grid (2 cm pitch), 48 kHz, N = 1024, hop 512, 2^18 frames, grid [-12, 12] at 1/8
GRID16 = Workload("grid16-2cm-48kHz-N1024-2^18frames", synth.grid_array(4, 4, 0.02), 48000.0, 1024,
                  512, 8, 1 << 18)
