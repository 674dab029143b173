"""FP64 CPU oracle for FCC TDoA estimation -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this module.  The product package never imports it and
shares no code with it.

This is a thin numpy/ctypes shell over ``fcc_oracle.c`` (compiled on first use
with the system C compiler).  Every numeric step lives in the C file, except
the STFT, where numpy's rfft serves as the DFT of each windowed frame (a
library primitive used as one step); the C file follows the paper's
definitions literally in FP64:

* Sec. 3 -- candidate grid tau_i = -L + i/r  (I = 2rL + 1).
* Eq. 3 -- W(i, f) = exp(j 2 pi f tau_i / N), f = 0..N/2.
* Sec. 4 -- W = U S V^H by the C file's own complex Jacobi SVD, truncated to
  rank K (W_K); K from the energy rule when not given.
* Sec. 2 (eq. 1, alpha = 1) -- R_hat = X_i X_j^* / |X_i X_j^*|.
* Eq. 2 / Eq. 4 -- y = 2 Re{W_K x}; argmax; three-point quadratic refinement.
* Sec. 2 -- the STFT X(t, f) of the microphone signals (``stft``): periodic
  Hann window, frames of N samples every hop samples, no padding.
* Conclusion (next step: a DoA search over candidates using every pair's
  TDoA) -- steered-response power over unit-vector candidates from the
  pairs' correlations on the lag grid (``doa_srp``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_fcc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile fcc_oracle.c into liboracle_fcc.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.or_grid.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
            lib.or_grid.restype = ctypes.c_int
            lib.or_build_W.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            lib.or_build_W.restype = None
            lib.or_svd.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                   ctypes.c_int]
            lib.or_svd.restype = ctypes.c_int
            lib.or_rank_energy.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.or_rank_energy.restype = ctypes.c_int
            lib.or_lowrank.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                       _dp, _dp, _dp, _dp, _dp, _dp]
            lib.or_lowrank.restype = None
            lib.or_phat.argtypes = [_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.or_phat.restype = None
            lib.or_correlate.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.or_correlate.restype = None
            lib.or_argmax.argtypes = [_dp, ctypes.c_int]
            lib.or_argmax.restype = ctypes.c_int
            lib.or_parabola.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double]
            lib.or_parabola.restype = ctypes.c_double
            lib.or_tdoa.argtypes = [_fp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _ip, _dp, _dp,
                                    _dp, ctypes.c_int]
            lib.or_tdoa.restype = None
            lib.or_tdoa_smoothed.argtypes = [_fp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                             _ip, _dp, _dp, _dp, ctypes.c_int]
            lib.or_tdoa_smoothed.restype = None
            lib.or_mlp_nparams.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.or_mlp_nparams.restype = ctypes.c_longlong
            lib.or_mlp_forward.argtypes = [_dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.or_mlp_forward.restype = None
            lib.or_mlp_loss_grad.argtypes = [_dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                             ctypes.c_double, _dp]
            lib.or_mlp_loss_grad.restype = ctypes.c_double
            lib.or_adam.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.or_adam.restype = None
            lib.or_doa_srp.argtypes = [_dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _dp, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int, _ip, _dp, _dp,
                                       ctypes.c_int]
            lib.or_doa_srp.restype = None
            lib.or_max_threads.argtypes = []
            lib.or_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def max_threads() -> int:
    return int(_load().or_max_threads())


def grid(L: int, den: int) -> np.ndarray:
    """Sec. 3: the candidate grid tau_i = -L + i/den (I = 2*L*den + 1)."""
    lib = _load()
    I = lib.or_grid(L, den, None)
    taus = np.empty(I, np.float64)
    lib.or_grid(L, den, _d(taus))
    return taus


def build_W(N: int, taus: np.ndarray) -> np.ndarray:
    """Eq. 3: W(i, f) = exp(j 2 pi f tau_i / N), shape [I, N/2+1], complex128."""
    taus = np.ascontiguousarray(taus, np.float64)
    I, B = len(taus), N // 2 + 1
    wr = np.empty((I, B), np.float64)
    wi = np.empty((I, B), np.float64)
    _load().or_build_W(N, I, _d(taus), _d(wr), _d(wi))
    return wr + 1j * wi


def svd(A: np.ndarray, max_sweeps: int = 80):
    """Sec. 4: A = U diag(s) V^H by the oracle's own complex Jacobi SVD.

    Returns (U [m, r], s [r] descending, V [n, r]) with r = min(m, n).
    """
    A = np.asarray(A, np.complex128)
    m, n = A.shape
    r = min(m, n)
    ar = np.ascontiguousarray(A.real)
    ai = np.ascontiguousarray(A.imag)
    s = np.empty(r)
    ur, ui = np.empty((m, r)), np.empty((m, r))
    vr, vi = np.empty((n, r)), np.empty((n, r))
    sweeps = _load().or_svd(m, n, _d(ar), _d(ai), _d(s), _d(ur), _d(ui), _d(vr), _d(vi),
                            max_sweeps)
    if sweeps < 0:
        raise RuntimeError("oracle Jacobi SVD did not converge")
    return ur + 1j * ui, s, vr + 1j * vi


def rank_energy(s: np.ndarray, energy: float = 0.999, tie_rel: float = 1e-12) -> int:
    """Sec. 4 ("K set experimentally"): smallest K holding `energy` of sum(s^2)."""
    s = np.ascontiguousarray(s, np.float64)
    return int(_load().or_rank_energy(_d(s), len(s), energy, tie_rel))


def lowrank(U, s, V, K: int) -> np.ndarray:
    """Sec. 4: W_K = U_K diag(s_K) V_K^H."""
    m, r = U.shape
    n = V.shape[0]
    ur, ui = np.ascontiguousarray(U.real), np.ascontiguousarray(U.imag)
    vr, vi = np.ascontiguousarray(V.real), np.ascontiguousarray(V.imag)
    s = np.ascontiguousarray(s, np.float64)
    wr, wi = np.empty((m, n)), np.empty((m, n))
    _load().or_lowrank(m, n, r, K, _d(s), _d(ur), _d(ui), _d(vr), _d(vi), _d(wr), _d(wi))
    return wr + 1j * wi


def phat(X_frame: np.ndarray, i: int, j: int) -> np.ndarray:
    """Sec. 2: R_hat = X_i X_j^* / |X_i X_j^*| for one frame X[m, f] (complex64)."""
    X = np.ascontiguousarray(X_frame, np.complex64)
    B = X.shape[1]
    xr, xi = np.empty(B), np.empty(B)
    _load().or_phat(X.ctypes.data_as(_fp), B, i, j, _d(xr), _d(xi))
    return xr + 1j * xi


def correlate(W: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 4: y = 2 Re{W x}."""
    I, B = W.shape
    wr, wi = np.ascontiguousarray(W.real), np.ascontiguousarray(W.imag)
    xr, xi = np.ascontiguousarray(np.real(x), np.float64), np.ascontiguousarray(np.imag(x), np.float64)
    y = np.empty(I)
    _load().or_correlate(I, B, _d(wr), _d(wi), _d(xr), _d(xi), _d(y))
    return y


def argmax(y: np.ndarray) -> int:
    y = np.ascontiguousarray(y, np.float64)
    return int(_load().or_argmax(_d(y), len(y)))


def parabola(y: np.ndarray, idx: int, tau_idx: float, delta: float) -> float:
    y = np.ascontiguousarray(y, np.float64)
    return float(_load().or_parabola(_d(y), len(y), idx, tau_idx, delta))


class Basis:
    """The oracle's rank-K operator for one (N, lag grid) key.

    W (Eq. 3) -> complex Jacobi SVD (Sec. 4) -> K by the energy rule unless
    given -> W_K.  `full` keeps W itself (the eq. 2 / GCC-PHAT operator).
    """

    def __init__(self, N: int, L: int, den: int, K: int | None = None, energy: float = 0.999):
        self.N, self.L, self.den = N, L, den
        self.B = N // 2 + 1
        self.taus = grid(L, den)
        self.I = len(self.taus)
        self.delta = 1.0 / den
        self.W = build_W(N, self.taus)
        self.U, self.s, self.V = svd(self.W)
        self.K = rank_energy(self.s, energy) if K is None else int(K)
        self.WK = lowrank(self.U, self.s, self.V, self.K)


class BasisB:
    """The second basis split of the problem statement (real part of the
    cross-spectrum on cosine bases, imaginary part on sine bases; the paper
    itself folds, Eqs. 6-9): with C = Re W and S = Im W (Eq. 3),
        y_B = 2 (C_Kc Re x - S_Ks Im x) = 2 Re{(C_Kc + j S_Ks) x},
    where C_Kc and S_Ks are each truncated from the oracle's own Jacobi SVD of
    that matrix, K by the energy rule applied to its own singular values (Sec. 4
    rule), or given.  `WK` is the complex operator C_Kc + j S_Ks, so `tdoa` and
    `tdoa_smoothed` compute form B unchanged."""

    def __init__(self, N: int, L: int, den: int, Kc: int | None = None, Ks: int | None = None,
                 energy: float = 0.999):
        self.N, self.L, self.den = N, L, den
        self.B = N // 2 + 1
        self.taus = grid(L, den)
        self.I = len(self.taus)
        self.delta = 1.0 / den
        W = build_W(N, self.taus)
        self.C, self.S = np.ascontiguousarray(W.real), np.ascontiguousarray(W.imag)
        self.Uc, self.sc, self.Vc = svd(self.C)
        self.Us, self.ss, self.Vs = svd(self.S)
        self.Kc = rank_energy(self.sc, energy) if Kc is None else int(Kc)
        self.Ks = rank_energy(self.ss, energy) if Ks is None else int(Ks)
        self.CK = lowrank(self.Uc, self.sc, self.Vc, self.Kc).real
        self.SK = lowrank(self.Us, self.ss, self.Vs, self.Ks).real
        self.WK = self.CK + 1j * self.SK


def tdoa(X: np.ndarray, W: np.ndarray, taus: np.ndarray, delta: float, want_y: bool = False,
         threads: int | None = None):
    """The per-pair-frame pipeline over spectra X[T, M, N/2+1] (complex64).

    For every frame and every pair i < j (lexicographic): R_hat (Sec. 2),
    y = 2 Re{W x} (Eq. 4), argmax (lowest index on ties), quadratic refinement.
    Returns (idx [T, P] int32, peak [T, P] f64, tau_hat [T, P] f64, y [T, P, I] or None).
    """
    X = np.ascontiguousarray(X, np.complex64)
    T, M, B = X.shape
    N = 2 * (B - 1)
    I = W.shape[0]
    assert W.shape[1] == B and len(taus) == I
    P = M * (M - 1) // 2
    wr, wi = np.ascontiguousarray(W.real), np.ascontiguousarray(W.imag)
    taus = np.ascontiguousarray(taus, np.float64)
    idx = np.empty((T, P), np.int32)
    peak = np.empty((T, P))
    tau = np.empty((T, P))
    y = np.empty((T, P, I)) if want_y else None
    nt = max_threads() if threads is None else int(threads)
    _load().or_tdoa(X.ctypes.data_as(_fp), T, M, N, I, _d(wr), _d(wi), _d(taus), float(delta),
                    idx.ctypes.data_as(_ip), _d(peak), _d(tau),
                    _d(y) if want_y else None, nt)
    return idx, peak, tau, y


def stft(pcm: np.ndarray, N: int, hop: int) -> np.ndarray:
    """The STFT the method starts from (Sec. 2: X_m(t, f) of each microphone
    signal; the window and framing are not printed, so: periodic Hann window
    w[n] = 0.5 - 0.5 cos(2 pi n / N), frame t = samples t hop .. t hop + N - 1,
    no padding, T = 1 + (n_samples - N) // hop frames, 0 if n_samples < N).
    pcm: interleaved [n_samples, M], float (used as is) or int16 (divided by
    32768).  Returns X [T, M, N/2 + 1] complex128 with X[t, m, k] =
    sum_n w[n] x[t hop + n, m] exp(-j 2 pi k n / N) (numpy's rfft is the DFT)."""
    x = np.asarray(pcm)
    x = x.astype(np.float64) / 32768.0 if x.dtype == np.int16 else x.astype(np.float64)
    n_samples, M = x.shape
    T = 0 if n_samples < N else 1 + (n_samples - N) // hop
    n = np.arange(N)
    w = 0.5 - 0.5 * np.cos(2.0 * np.pi * n / N)
    X = np.empty((T, M, N // 2 + 1), np.complex128)
    for t in range(T):
        frame = x[t * hop:t * hop + N, :] * w[:, None]  # [N, M]
        X[t] = np.fft.rfft(frame, axis=0).T
    return X


def doa_srp(y: np.ndarray, L: int, den: int, mic_xyz: np.ndarray, fs: float, c: float, dirs: np.ndarray,
            want_scores: bool = False, threads: int | None = None):
    """DoA search over candidate directions (the next step named in the paper's
    conclusion; it prints no formula): score(u) = sum over pairs i < j of the
    pair's correlation y_ij read at tau_ij(u) = -(fs/c)(r_i - r_j).u samples by
    linear interpolation on the lag grid tau_k = -L + k/den (clamped to the
    grid's ends).  y: [T, P, I]; mic_xyz: [M, 3] metres; dirs: [D, 3] unit
    vectors.  Returns (best index [T] int32, best score [T], scores [T, D] or
    None); the lowest index wins an exact tie."""
    y = np.ascontiguousarray(y, np.float64)
    T, P, I = y.shape
    xyz = np.ascontiguousarray(mic_xyz, np.float64)
    M = xyz.shape[0]
    assert P == M * (M - 1) // 2 and I == 2 * L * den + 1
    dirs = np.ascontiguousarray(dirs, np.float64)
    D = dirs.shape[0]
    idx = np.empty(T, np.int32)
    score = np.empty(T)
    scores = np.empty((T, D)) if want_scores else None
    nt = max_threads() if threads is None else int(threads)
    _load().or_doa_srp(_d(y), T, M, I, L, den, _d(xyz), float(fs), float(c), _d(dirs), D, idx.ctypes.data_as(_ip),
                       _d(score), _d(scores) if want_scores else None, nt)
    return idx, score, scores


# ----------------------------------------------------------------------------
# learned TDoA head (not in the paper): FP64 reference of the MLP
# ----------------------------------------------------------------------------
def tdoa_smoothed(X: np.ndarray, W: np.ndarray, taus: np.ndarray, delta: float, alpha: float, R0=None,
                  want_y: bool = False, threads: int | None = None):
    """The pipeline with Eq. 1's recursive cross-spectrum for a smoothing factor
    alpha in (0, 1]: R(t) = (1 - alpha) R(t-1) + alpha X_i X_j^*, from R0 ([P, B]
    complex, None = zero), then R_hat = R / |R| and the rest as `tdoa`.
    Returns (idx, peak, tau_hat, y or None, R_end [P, B] complex128)."""
    X = np.ascontiguousarray(X, np.complex64)
    T, M, B = X.shape
    N = 2 * (B - 1)
    I = W.shape[0]
    assert W.shape[1] == B and len(taus) == I
    P = M * (M - 1) // 2
    wr, wi = np.ascontiguousarray(W.real), np.ascontiguousarray(W.imag)
    taus = np.ascontiguousarray(taus, np.float64)
    r0 = None if R0 is None else np.ascontiguousarray(np.asarray(R0, np.complex128).reshape(P, B))
    r_end = np.empty((P, B), np.complex128)
    idx = np.empty((T, P), np.int32)
    peak = np.empty((T, P))
    tau = np.empty((T, P))
    y = np.empty((T, P, I)) if want_y else None
    nt = max_threads() if threads is None else int(threads)
    _load().or_tdoa_smoothed(X.ctypes.data_as(_fp), T, M, N, I, _d(wr), _d(wi), _d(taus), float(delta),
                             float(alpha), None if r0 is None else r0.ctypes.data_as(_dp),
                             r_end.ctypes.data_as(_dp), idx.ctypes.data_as(_ip), _d(peak), _d(tau),
                             _d(y) if want_y else None, nt)
    return idx, peak, tau, y, r_end


def mlp_nparams(nin: int, H: int) -> int:
    return int(_load().or_mlp_nparams(nin, H))


def mlp_forward(x, params, nin: int, H: int) -> np.ndarray:
    """y [n, 2] = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3 (exact erf GELU)."""
    x = np.ascontiguousarray(x, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    y = np.empty((x.shape[0], 2))
    _load().or_mlp_forward(_d(x), x.shape[0], nin, H, _d(params), _d(y))
    return y


def mlp_loss_grad(x, params, t, tfcc, nin: int, H: int, lam: float):
    """Mean of (y0 - t)^2 + lam * BCE(sigmoid(y1), [|y0 - t| <= |tfcc - t|]) and its gradient."""
    x = np.ascontiguousarray(x, np.float64)
    params = np.ascontiguousarray(params, np.float64)
    t = np.ascontiguousarray(t, np.float64)
    tfcc = np.ascontiguousarray(tfcc, np.float64)
    g = np.empty_like(params)
    loss = _load().or_mlp_loss_grad(_d(x), x.shape[0], nin, H, _d(params), _d(t), _d(tfcc), lam, _d(g))
    return float(loss), g


def adam(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of params, m, v (float64 arrays)."""
    _load().or_adam(_d(params), _d(np.ascontiguousarray(grad, np.float64)), _d(m), _d(v), len(params), step, lr,
                    beta1, beta2, eps)


def round_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)
