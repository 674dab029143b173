"""Operation and byte accounting for GCC and FCC, as the paper counts them.

* Sec. 3: GCC with an r-times zero-padded real IFFT costs about 5 (rN/2)
  log2(rN) flops (radix-2, real data of rN samples); with N = 512 this gives
  11520 / 25600 / 56320 for r = 1 / 2 / 4 (Table 1).
* Sec. 3: the grid of an r-times interpolated GCC has I = 2 r ceil(tau_max) + 1
  candidates (I = 33 for tau_max = 8, r = 2).
* Sec. 4, Eq. 4: the direct product y = 2 Re{W x} costs I (4N + 6) flops.
* Sec. 4: the unfolded low-rank form costs K (4N + 6) + I (4K - 1) flops.
* Sec. 4, Eq. 9: the folded FCC form costs K (N + 2) + N + I (4K - 1) flops.

The byte model is this library's: the only mandatory HBM traffic of the fused
path is reading every microphone spectrum once and writing the per-pair result.
"""
from __future__ import annotations

import math


def gcc_flops(N: int, r: int) -> int:
    return int(round(5 * (r * N / 2) * math.log2(r * N)))


def n_candidates(tau_max: float, r: int) -> int:
    return 2 * r * int(math.ceil(tau_max)) + 1


def direct_flops(N: int, I: int) -> int:
    return I * (4 * N + 6)


def lowrank_flops(N: int, I: int, K: int) -> int:
    return K * (4 * N + 6) + I * (4 * K - 1)


def fcc_flops(N: int, I: int, K: int) -> int:
    return K * (N + 2) + N + I * (4 * K - 1)


def fcc_bytes_per_pair_frame(M: int, N: int, out_bytes_per_pair: int = 8) -> float:
    """(M (N/2+1) 8 + P out) / P: spectra read once per frame, results written."""
    B = N // 2 + 1
    P = M * (M - 1) // 2
    return (M * B * 8 + P * out_bytes_per_pair) / P
