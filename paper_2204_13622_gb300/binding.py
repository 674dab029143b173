"""Thin ctypes binding of libfcc_gb300.so (the C ABI in include/fcc.h).

Argument marshalling only: every step of the FCC path runs in the library's
CUDA kernels.  PyTorch is used to allocate device / pinned-host buffers and to
supply the current CUDA stream.  There is no CPU fallback: if the library is
missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfcc_gb300.so")

FCC_OK = 0
STATUS = {0: "FCC_OK", 1: "FCC_ERR_INVALID_ARG", 2: "FCC_ERR_UNSUPPORTED", 3: "FCC_ERR_OOM",
          4: "FCC_ERR_CUDA", 5: "FCC_ERR_TIMEOUT", 6: "FCC_ERR_NONFINITE", 7: "FCC_ERR_NOT_CONVERGED"}
PREC = {"fp32": 0, "bf16": 1, "fp16": 2}
FORM = {"folded": 0, "reim": 1}
ENGINE = {"auto": 0, "cuda_cores": 1, "tensor_tmem": 2, "tensor_smem": 3}

# every symbol include/fcc.h declares
EXPORTS = ["fcc_plan_create", "fcc_plan_destroy", "fcc_plan_info", "fcc_plan_taus",
           "fcc_plan_singular_values", "fcc_plan_bases", "fcc_tdoa", "fcc_tdoa_host", "fcc_gcc_tdoa",
           "fcc_plan_sync", "fcc_status_string", "fcc_last_error", "fcc_plan_bases_noalloc",
           "fcc_plan_set_engine", "fcc_plan_get_engine",
           # include/fcc_mlp.h
           "fcc_mlp_num_params", "fcc_mlp_create", "fcc_mlp_destroy", "fcc_mlp_get_state",
           "fcc_mlp_set_state", "fcc_mlp_gradient", "fcc_mlp_train_step", "fcc_mlp_infer", "fcc_mlp_sync", "fcc_tdoa_learned",
           # include/fcc_tune.h
           "fcc_plan_geometry", "fcc_plan_autotune",
           # include/fcc_batch.h
           "fcc_batch_create", "fcc_batch_destroy", "fcc_batch_info", "fcc_batch_array_info", "fcc_batch_bind",
           "fcc_batch_run", "fcc_batch_sync",
           # include/fcc_debug.h
           "fcc_debug_set",
           # include/fcc_smooth.h
           "fcc_smooth_workspace", "fcc_tdoa_smoothed",
           # include/fcc_doa.h
           "fcc_doa_create", "fcc_doa_destroy", "fcc_doa_search", "fcc_doa_workspace", "fcc_tdoa_doa",
           # include/fcc_stft.h
           "fcc_stft_frames", "fcc_stft", "fcc_pcm_workspace", "fcc_tdoa_pcm", "fcc_tdoa_pcm_host"]
PCM = {"f32": 0, "s16": 1}


class PlanDesc(ctypes.Structure):
    _fields_ = [("n_mics", ctypes.c_int), ("mic_xyz", ctypes.POINTER(ctypes.c_double)),
                ("fs", ctypes.c_double), ("N", ctypes.c_int), ("c", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("lag_den", ctypes.c_int), ("K", ctypes.c_int),
                ("energy", ctypes.c_double), ("prec", ctypes.c_int), ("device", ctypes.c_int),
                ("form", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("P", ctypes.c_int), ("N", ctypes.c_int), ("B", ctypes.c_int),
                ("Q", ctypes.c_int), ("L", ctypes.c_int), ("den", ctypes.c_int), ("I", ctypes.c_int),
                ("center", ctypes.c_int), ("K", ctypes.c_int), ("K_even", ctypes.c_int),
                ("K_odd", ctypes.c_int), ("prec", ctypes.c_int), ("delta", ctypes.c_double),
                ("fs", ctypes.c_double), ("c", ctypes.c_double), ("form", ctypes.c_int)]


class Geometry(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int), ("warps_per_group", ctypes.c_int), ("groups", ctypes.c_int),
                ("frames_per_stage", ctypes.c_int), ("stages", ctypes.c_int), ("threads", ctypes.c_int),
                ("smem_bytes", ctypes.c_longlong)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_arrays", ctypes.c_int), ("n_classes", ctypes.c_int), ("n_jobs", ctypes.c_int),
                ("n_bases", ctypes.c_int), ("frames", ctypes.c_longlong), ("pair_frames", ctypes.c_longlong),
                ("spectra_bytes", ctypes.c_double), ("result_bytes", ctypes.c_double), ("n_launches", ctypes.c_int)]


FCC_BATCH_AUTOTUNE = 1
FCC_BATCH_SINGLE_LAUNCH = 2
DEBUG_HOOKS = {"wait_cycles": 0, "withhold_copy": 1, "fail_alloc": 2}


def debug_set(hook: str, value: int):
    """Test hooks of include/fcc_debug.h (wait bound, withheld copies, failing allocations)."""
    check(lib().fcc_debug_set(DEBUG_HOOKS[hook], int(value)), "fcc_debug_set")


class FccError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.fcc_plan_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(_vp)]
        L.fcc_plan_destroy.argtypes = [_vp]
        L.fcc_plan_destroy.restype = None
        L.fcc_plan_info.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
        L.fcc_plan_taus.argtypes = [_vp, _dp]
        L.fcc_plan_singular_values.argtypes = [_vp, _dp, _ip, _dp, _ip]
        L.fcc_plan_bases.argtypes = [_vp, _dp, _dp, _dp, _dp]
        L.fcc_tdoa.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, _vp]
        L.fcc_tdoa_host.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp]
        L.fcc_gcc_tdoa.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp]
        L.fcc_plan_sync.argtypes = [_vp, _vp]
        L.fcc_plan_set_engine.argtypes = [_vp, ctypes.c_int]
        L.fcc_plan_get_engine.argtypes = [_vp, _ip]
        L.fcc_plan_bases_noalloc.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(PlanInfo), _dp, _dp,
                                             _dp, _dp, _dp, _dp, _vp]
        L.fcc_status_string.argtypes = [ctypes.c_int]
        L.fcc_status_string.restype = ctypes.c_char_p
        L.fcc_last_error.argtypes = []
        L.fcc_last_error.restype = ctypes.c_char_p
        _fp = ctypes.POINTER(ctypes.c_float)
        L.fcc_mlp_num_params.argtypes = [ctypes.c_int, ctypes.c_int]
        L.fcc_mlp_num_params.restype = ctypes.c_longlong
        L.fcc_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, _fp, ctypes.c_double, _fp,
                                     ctypes.c_int, ctypes.POINTER(_vp)]
        L.fcc_mlp_destroy.argtypes = [_vp]
        L.fcc_mlp_destroy.restype = None
        L.fcc_mlp_get_state.argtypes = [_vp, _fp, _fp, _fp, ctypes.POINTER(ctypes.c_longlong)]
        L.fcc_mlp_set_state.argtypes = [_vp, _fp, _fp, _fp, ctypes.c_longlong]
        L.fcc_mlp_gradient.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp]
        L.fcc_mlp_train_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_longlong, ctypes.c_float, _vp, _vp]
        L.fcc_mlp_infer.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_float, _vp, _vp, _vp, _vp]
        L.fcc_mlp_sync.argtypes = [_vp, _vp]
        L.fcc_tdoa_learned.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_float, _vp, _vp, _vp, _vp, _vp,
                                       _vp, _vp]
        L.fcc_tdoa_learned.restype = ctypes.c_int
        L.fcc_plan_geometry.argtypes = [_vp, ctypes.POINTER(Geometry)]
        L.fcc_plan_autotune.argtypes = [_vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, _dp]
        L.fcc_batch_create.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(_vp)]
        L.fcc_batch_destroy.argtypes = [_vp]
        L.fcc_batch_destroy.restype = None
        L.fcc_batch_info.argtypes = [_vp, ctypes.POINTER(BatchInfo)]
        L.fcc_batch_array_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(PlanInfo)]
        L.fcc_batch_bind.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     ctypes.POINTER(_vp)]
        L.fcc_batch_run.argtypes = [_vp, _vp]
        L.fcc_debug_set.argtypes = [ctypes.c_int, ctypes.c_longlong]
        L.fcc_debug_set.restype = ctypes.c_int
        L.fcc_smooth_workspace.argtypes = [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.fcc_smooth_workspace.restype = ctypes.c_int
        L.fcc_tdoa_smoothed.argtypes = [_vp, _vp, ctypes.c_longlong, ctypes.c_double, _vp, _vp, ctypes.c_longlong,
                                        _vp, _vp, _vp, _vp, _vp, _vp]
        L.fcc_tdoa_smoothed.restype = ctypes.c_int
        L.fcc_batch_sync.argtypes = [_vp, _vp]
        L.fcc_doa_create.argtypes = [_vp, _dp, _dp, ctypes.c_int, ctypes.POINTER(_vp)]
        L.fcc_doa_destroy.argtypes = [_vp]
        L.fcc_doa_destroy.restype = None
        L.fcc_doa_search.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp, _vp]
        L.fcc_doa_workspace.argtypes = [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
        L.fcc_tdoa_doa.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, ctypes.c_longlong, _vp]
        for name in ("fcc_doa_create", "fcc_doa_search", "fcc_doa_workspace", "fcc_tdoa_doa"):
            getattr(L, name).restype = ctypes.c_int
        _ll, _i = ctypes.c_longlong, ctypes.c_int
        L.fcc_stft_frames.argtypes = [_vp, _ll, _i, ctypes.POINTER(_ll)]
        L.fcc_stft.argtypes = [_vp, _vp, _i, _ll, _i, _vp, _vp]
        L.fcc_pcm_workspace.argtypes = [_vp, _ll, _i, ctypes.POINTER(_ll)]
        L.fcc_tdoa_pcm.argtypes = [_vp, _vp, _i, _ll, _i, _vp, _vp, _vp, _vp, _ll, _vp]
        L.fcc_tdoa_pcm_host.argtypes = [_vp, _vp, _i, _ll, _i, _vp, _vp, _vp, _vp]
        for name in ("fcc_stft_frames", "fcc_stft", "fcc_pcm_workspace", "fcc_tdoa_pcm", "fcc_tdoa_pcm_host"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("fcc_plan_geometry", "fcc_plan_autotune", "fcc_batch_create", "fcc_batch_info",
                     "fcc_batch_array_info", "fcc_batch_bind", "fcc_batch_run", "fcc_batch_sync"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("fcc_mlp_create", "fcc_mlp_get_state", "fcc_mlp_set_state", "fcc_mlp_gradient",
                     "fcc_mlp_train_step", "fcc_mlp_infer", "fcc_mlp_sync"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("fcc_plan_create", "fcc_plan_info", "fcc_plan_taus", "fcc_plan_singular_values",
                     "fcc_plan_bases", "fcc_tdoa", "fcc_tdoa_host", "fcc_gcc_tdoa", "fcc_plan_sync",
                     "fcc_plan_bases_noalloc"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def check(status: int, where: str):
    if status != FCC_OK:
        raise FccError(status, where, lib().fcc_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def frame_range(T_total: int, rank: int, world: int):
    """Frames [t0, t1) of rank `rank` when T_total frames are split across `world`
    GPUs: contiguous, balanced (the first T_total % world ranks take one frame
    more), together covering [0, T_total) once.  Frames are independent at
    alpha = 1, so each rank runs fcc_tdoa on its own slice with no exchange."""
    if world < 1 or not 0 <= rank < world or T_total < 0:
        raise ValueError("need 0 <= rank < world and T_total >= 0")
    base, extra = divmod(int(T_total), int(world))
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


class Plan:
    """An FCC plan: lag grid, rank-K even/odd bases and kernel tables on one GPU."""

    def __init__(self, n_mics: int, fs: float, N: int, lag_den: int, tau_max: float = 0.0,
                 mic_xyz=None, c: float = 343.0, K: int = 0, energy: float = 0.999,
                 prec: str = "fp32", device: int | None = None, form: str = "folded", engine: str = "auto"):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        xyz = None
        if mic_xyz is not None:
            xyz = np.ascontiguousarray(mic_xyz, np.float64).reshape(n_mics, 3)
        desc = PlanDesc(n_mics, xyz.ctypes.data_as(_dp) if xyz is not None else None, float(fs), int(N),
                        float(c), float(tau_max), int(lag_den), int(K), float(energy), PREC[prec],
                        self.device, FORM[form])
        h = _vp()
        check(lib().fcc_plan_create(ctypes.byref(desc), ctypes.byref(h)), "fcc_plan_create")
        self._h = h
        info = PlanInfo()
        check(lib().fcc_plan_info(h, ctypes.byref(info)), "fcc_plan_info")
        self.info = {k: getattr(info, k) for k, _ in PlanInfo._fields_}
        if engine != "auto":
            self.set_engine(engine)

    def set_engine(self, engine: str):
        """fcc_plan_set_engine: the kernel fcc_tdoa runs (see ENGINE)."""
        check(lib().fcc_plan_set_engine(self._h, ENGINE[engine]), "fcc_plan_set_engine")

    @property
    def engine(self) -> str:
        e = ctypes.c_int()
        check(lib().fcc_plan_get_engine(self._h, ctypes.byref(e)), "fcc_plan_get_engine")
        return {v: k for k, v in ENGINE.items()}[e.value]

    def __getattr__(self, name):
        info = self.__dict__.get("info")
        if info is not None and name in info:
            return info[name]
        raise AttributeError(name)

    def close(self):
        if getattr(self, "_h", None):
            lib().fcc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host-side queries
    def taus(self) -> np.ndarray:
        out = np.empty(self.I)
        check(lib().fcc_plan_taus(self._h, out.ctypes.data_as(_dp)), "fcc_plan_taus")
        return out

    def singular_values(self):
        ne, no = ctypes.c_int(), ctypes.c_int()
        check(lib().fcc_plan_singular_values(self._h, None, ctypes.byref(ne), None, ctypes.byref(no)),
              "fcc_plan_singular_values")
        se, so = np.empty(ne.value), np.empty(no.value)
        check(lib().fcc_plan_singular_values(self._h, se.ctypes.data_as(_dp), None,
                                             so.ctypes.data_as(_dp), None), "fcc_plan_singular_values")
        return se, so

    def bases(self):
        KE, KO, Q, I = self.K_even, self.K_odd, self.Q, self.I
        if self.form == FORM["reim"]:  # cosine / sine bases over all N/2 + 1 bins
            Pe, Po = np.empty((KE, self.B)), np.empty((KO, self.B))
        else:
            Pe, Po = np.empty((KE, Q + 1)), np.empty((KO, Q))
        Ue, Uo = np.empty((I, KE)), np.empty((I, KO))
        check(lib().fcc_plan_bases(self._h, Pe.ctypes.data_as(_dp), Po.ctypes.data_as(_dp),
                                   Ue.ctypes.data_as(_dp), Uo.ctypes.data_as(_dp)), "fcc_plan_bases")
        return Pe, Po, Ue, Uo

    # ---- device entry points
    def _check_spectra(self, X):
        import torch
        if X.dtype != torch.complex64 or X.dim() != 3 or X.shape[1] != self.M or X.shape[2] != self.B:
            raise ValueError(f"spectra must be complex64 [T, {self.M}, {self.B}]")
        if not X.is_contiguous():
            raise ValueError("spectra must be contiguous")

    def tdoa(self, X, tau_hat: bool = True, coeffs: bool = False, corr: bool = False, stream=None,
             out=None):
        """FCC on device spectra X [T, M, B] (complex64): dict of device tensors."""
        import torch
        self._check_spectra(X)
        T = X.shape[0]
        dev = X.device
        if out is None:
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, device=dev),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, device=dev)}
            if tau_hat:
                out["tau_hat"] = torch.empty((T, self.P), dtype=torch.float32, device=dev)
            if coeffs:
                out["coeffs"] = torch.empty((T, self.P, 2 * self.K), dtype=torch.float32, device=dev)
            if corr:
                out["corr"] = torch.empty((T, self.P, self.I), dtype=torch.float32, device=dev)
        check(lib().fcc_tdoa(self._h, _ptr(X), T, _ptr(out["lag_idx"]), _ptr(out["peak"]),
                             _ptr(out.get("tau_hat")), _ptr(out.get("coeffs")), _ptr(out.get("corr")),
                             _stream(stream, dev)), "fcc_tdoa")
        return out

    def tdoa_host(self, X_host, tau_hat: bool = True, out=None, stream=None):
        """FCC from host spectra to host results (pinned host memory recommended)."""
        import torch
        self._check_spectra(X_host)
        T = X_host.shape[0]
        if out is None:
            pin = X_host.is_pinned()
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, pin_memory=pin),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, pin_memory=pin)}
            if tau_hat:
                out["tau_hat"] = torch.empty((T, self.P), dtype=torch.float32, pin_memory=pin)
        check(lib().fcc_tdoa_host(self._h, _ptr(X_host), T, _ptr(out["lag_idx"]), _ptr(out["peak"]),
                                  _ptr(out.get("tau_hat")), _stream(stream, self.device)), "fcc_tdoa_host")
        return out

    def gcc_tdoa(self, X, corr: bool = False, stream=None, out=None):
        """Same-GPU GCC-PHAT baseline (full rank, r = den) on device spectra."""
        import torch
        self._check_spectra(X)
        T = X.shape[0]
        dev = X.device
        if out is None:
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, device=dev),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, device=dev)}
            if corr:
                out["corr"] = torch.empty((T, self.P, self.I), dtype=torch.float32, device=dev)
        check(lib().fcc_gcc_tdoa(self._h, _ptr(X), T, _ptr(out["lag_idx"]), _ptr(out["peak"]),
                                 _ptr(out.get("corr")), _stream(stream, dev)), "fcc_gcc_tdoa")
        return out

    def sync(self, stream=None):
        """Synchronise and raise if a kernel latched an error (NaN/Inf input, timeout)."""
        check(lib().fcc_plan_sync(self._h, _stream(stream, self.device)), "fcc_plan_sync")

    def tdoa_learned(self, X, mlp, threshold: float, stream=None, out=None):
        """fcc_tdoa_learned: FCC then the learned head's gated TDoA per pair-frame."""
        import torch
        self._check_spectra(X)
        T, dev = X.shape[0], X.device
        if out is None:
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, device=dev),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, device=dev),
                   "tau_fcc": torch.empty((T, self.P), dtype=torch.float32, device=dev),
                   "coeffs": torch.empty((T, self.P, 2 * self.K), dtype=torch.float32, device=dev),
                   "tau": torch.empty((T, self.P), dtype=torch.float32, device=dev),
                   "conf": torch.empty((T, self.P), dtype=torch.float32, device=dev)}
        check(lib().fcc_tdoa_learned(self._h, mlp._h, _ptr(X), T, float(threshold), _ptr(out["lag_idx"]),
                                     _ptr(out["peak"]), _ptr(out["tau_fcc"]), _ptr(out["coeffs"]), _ptr(out["tau"]),
                                     _ptr(out.get("conf")), _stream(stream, dev)), "fcc_tdoa_learned")
        return out

    def smooth_workspace(self, T: int) -> int:
        b = ctypes.c_longlong()
        check(lib().fcc_smooth_workspace(self._h, int(T), ctypes.byref(b)), "fcc_smooth_workspace")
        return b.value

    def tdoa_smoothed(self, X, alpha: float, state=None, tau_hat: bool = True, coeffs: bool = False,
                      corr: bool = False, work=None, stream=None, out=None):
        """fcc_tdoa_smoothed: Eq. 1's recursive cross-spectrum with factor alpha,
        then FCC.  `state`: complex64 [P, B] device tensor holding R(0) on entry
        and R(T) on return (None: a fresh stream, final state dropped)."""
        import torch
        self._check_spectra(X)
        T, dev = X.shape[0], X.device
        if state is not None and (state.dtype != torch.complex64 or tuple(state.shape) != (self.P, self.B)
                                  or not state.is_contiguous()):
            raise ValueError(f"state must be contiguous complex64 [{self.P}, {self.B}]")
        if work is None:
            nbytes = self.smooth_workspace(T)
            work = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=dev)
        if out is None:
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, device=dev),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, device=dev)}
            if tau_hat:
                out["tau_hat"] = torch.empty((T, self.P), dtype=torch.float32, device=dev)
            if coeffs:
                out["coeffs"] = torch.empty((T, self.P, 2 * self.K), dtype=torch.float32, device=dev)
            if corr:
                out["corr"] = torch.empty((T, self.P, self.I), dtype=torch.float32, device=dev)
        check(lib().fcc_tdoa_smoothed(self._h, _ptr(X), T, float(alpha), _ptr(state), _ptr(work), work.numel(),
                                      _ptr(out["lag_idx"]), _ptr(out["peak"]), _ptr(out.get("tau_hat")),
                                      _ptr(out.get("coeffs")), _ptr(out.get("corr")), _stream(stream, dev)),
              "fcc_tdoa_smoothed")
        return out

    # ---- STFT front-end (include/fcc_stft.h)
    def _pcm_type(self, pcm):
        import torch
        kinds = {torch.float32: PCM["f32"], torch.int16: PCM["s16"]}
        if pcm.dtype not in kinds or pcm.dim() != 2 or pcm.shape[1] != self.M or not pcm.is_contiguous():
            raise ValueError(f"PCM must be contiguous float32 or int16 [n_samples, {self.M}]")
        return kinds[pcm.dtype]

    def stft_frames(self, n_samples: int, hop: int) -> int:
        T = ctypes.c_longlong()
        check(lib().fcc_stft_frames(self._h, int(n_samples), int(hop), ctypes.byref(T)), "fcc_stft_frames")
        return T.value

    def stft(self, pcm, hop: int, stream=None, out=None):
        """fcc_stft: device PCM [n_samples, M] -> spectra complex64 [T, M, N/2+1]."""
        import torch
        kind = self._pcm_type(pcm)
        T, dev = self.stft_frames(pcm.shape[0], hop), pcm.device
        if out is None:
            out = torch.empty((T, self.M, self.B), dtype=torch.complex64, device=dev)
        check(lib().fcc_stft(self._h, _ptr(pcm), kind, pcm.shape[0], int(hop), _ptr(out), _stream(stream, dev)),
              "fcc_stft")
        return out

    def pcm_workspace(self, n_samples: int, hop: int) -> int:
        b = ctypes.c_longlong()
        check(lib().fcc_pcm_workspace(self._h, int(n_samples), int(hop), ctypes.byref(b)), "fcc_pcm_workspace")
        return b.value

    def tdoa_pcm(self, pcm, hop: int, tau_hat: bool = True, work=None, stream=None, out=None):
        """fcc_tdoa_pcm: device PCM in, per-pair TDoA out (the spectra stay on chip in chunks)."""
        import torch
        kind = self._pcm_type(pcm)
        T, dev = self.stft_frames(pcm.shape[0], hop), pcm.device
        if work is None:
            work = torch.empty(max(self.pcm_workspace(pcm.shape[0], hop), 16), dtype=torch.uint8, device=dev)
        if out is None:
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, device=dev),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, device=dev)}
            if tau_hat:
                out["tau_hat"] = torch.empty((T, self.P), dtype=torch.float32, device=dev)
        check(lib().fcc_tdoa_pcm(self._h, _ptr(pcm), kind, pcm.shape[0], int(hop), _ptr(out["lag_idx"]),
                                 _ptr(out["peak"]), _ptr(out.get("tau_hat")), _ptr(work), work.numel(),
                                 _stream(stream, dev)), "fcc_tdoa_pcm")
        return out

    def tdoa_pcm_host(self, pcm, hop: int, tau_hat: bool = True, stream=None, out=None):
        """fcc_tdoa_pcm_host: host PCM (a CPU tensor; pinned for full link speed)
        in, host results out; synchronous."""
        import torch
        kind = self._pcm_type(pcm)
        if pcm.device.type != "cpu":
            raise ValueError("tdoa_pcm_host takes host PCM")
        T = self.stft_frames(pcm.shape[0], hop)
        if out is None:
            pin = pcm.is_pinned()
            out = {"lag_idx": torch.empty((T, self.P), dtype=torch.int32, pin_memory=pin),
                   "peak": torch.empty((T, self.P), dtype=torch.float32, pin_memory=pin)}
            if tau_hat:
                out["tau_hat"] = torch.empty((T, self.P), dtype=torch.float32, pin_memory=pin)
        check(lib().fcc_tdoa_pcm_host(self._h, _ptr(pcm), kind, pcm.shape[0], int(hop), _ptr(out["lag_idx"]),
                                      _ptr(out["peak"]), _ptr(out.get("tau_hat")), _stream(stream, self.device)),
              "fcc_tdoa_pcm_host")
        return out

    def geometry(self) -> dict:
        g = Geometry()
        check(lib().fcc_plan_geometry(self._h, ctypes.byref(g)), "fcc_plan_geometry")
        return {k: getattr(g, k) for k, _ in Geometry._fields_}

    def autotune(self, cache_path: str | None = None, force: bool = False, max_candidates: int = 0) -> float:
        """Time the FP32 kernel's candidate tile shapes and keep the fastest
        (fcc_plan_autotune); returns microseconds per frame."""
        us = ctypes.c_double()
        check(lib().fcc_plan_autotune(self._h, cache_path.encode() if cache_path else None, int(force),
                                      int(max_candidates), ctypes.byref(us)), "fcc_plan_autotune")
        return us.value


class Doa:
    """include/fcc_doa.h: the search over candidate directions (unit vectors
    `dirs` [D, 3]) from the pairs' correlations on `plan`'s lag grid; `mic_xyz`
    [M, 3] metres.  The plan must stay open while this object is used."""

    def __init__(self, plan: Plan, mic_xyz, dirs):
        xyz = np.ascontiguousarray(mic_xyz, np.float64)
        d = np.ascontiguousarray(dirs, np.float64)
        if xyz.shape != (plan.M, 3) or d.ndim != 2 or d.shape[1] != 3:
            raise ValueError(f"mic_xyz must be [{plan.M}, 3] and dirs [D, 3]")
        h = _vp()
        check(lib().fcc_doa_create(plan._h, xyz.ctypes.data_as(_dp), d.ctypes.data_as(_dp), d.shape[0],
                                   ctypes.byref(h)), "fcc_doa_create")
        self._h, self.plan, self.D = h, plan, d.shape[0]

    def close(self):
        if getattr(self, "_h", None):
            lib().fcc_doa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, T: int) -> int:
        b = ctypes.c_longlong()
        check(lib().fcc_doa_workspace(self._h, int(T), ctypes.byref(b)), "fcc_doa_workspace")
        return b.value

    def _out(self, T, dev, out):
        import torch
        if out is None:
            out = {"dir_idx": torch.empty(T, dtype=torch.int32, device=dev),
                   "score": torch.empty(T, dtype=torch.float32, device=dev)}
        return out

    def search(self, corr, stream=None, out=None):
        """fcc_doa_search over correlations corr float32 [T, P, I] on the device."""
        import torch
        p = self.plan
        if corr.dtype != torch.float32 or corr.dim() != 3 or tuple(corr.shape[1:]) != (p.P, p.I) \
                or not corr.is_contiguous():
            raise ValueError(f"corr must be contiguous float32 [T, {p.P}, {p.I}]")
        T, dev = corr.shape[0], corr.device
        out = self._out(T, dev, out)
        check(lib().fcc_doa_search(self._h, _ptr(corr), T, _ptr(out["dir_idx"]), _ptr(out["score"]),
                                   _stream(stream, dev)), "fcc_doa_search")
        return out

    def tdoa_doa(self, X, pairs: bool = False, work=None, stream=None, out=None):
        """fcc_tdoa_doa: spectra X complex64 [T, M, B] in, per-frame candidate
        index and score out (and, with pairs=True, the per-pair lag_idx / peak)."""
        import torch
        p = self.plan
        p._check_spectra(X)
        T, dev = X.shape[0], X.device
        if work is None:
            work = torch.empty(max(self.workspace(T), 16), dtype=torch.uint8, device=dev)
        out = self._out(T, dev, out)
        if pairs and "lag_idx" not in out:
            out["lag_idx"] = torch.empty((T, p.P), dtype=torch.int32, device=dev)
            out["peak"] = torch.empty((T, p.P), dtype=torch.float32, device=dev)
        check(lib().fcc_tdoa_doa(self._h, _ptr(X), T, _ptr(out["dir_idx"]), _ptr(out["score"]),
                                 _ptr(out.get("lag_idx")), _ptr(out.get("peak")), _ptr(work), work.numel(),
                                 _stream(stream, dev)), "fcc_tdoa_doa")
        return out


def plan_bases_noalloc(n_mics: int, fs: float, N: int, lag_den: int, tau_max: float = 0.0, mic_xyz=None,
                       c: float = 343.0, K: int = 0, energy: float = 0.999, device: int = 0, stream=None):
    """fcc_plan_bases_noalloc: the plan's bases built in the library's static
    device scratch (no device allocation).  Returns (info dict, s_even, s_odd,
    Pe, Po, Ue, Uo) as numpy arrays."""
    xyz = None
    if mic_xyz is not None:
        xyz = np.ascontiguousarray(mic_xyz, np.float64).reshape(n_mics, 3)
    desc = PlanDesc(n_mics, xyz.ctypes.data_as(_dp) if xyz is not None else None, float(fs), int(N),
                    float(c), float(tau_max), int(lag_den), int(K), float(energy), 0, int(device))
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    info = PlanInfo()
    check(lib().fcc_plan_bases_noalloc(ctypes.byref(desc), ctypes.byref(info), None, None, None, None, None,
                                       None, st), "fcc_plan_bases_noalloc")
    I, Q, KE, KO = info.I, info.Q, info.K_even, info.K_odd
    se, so = np.empty(min(I, Q + 1)), np.empty(min(I, Q))
    Pe, Po, Ue, Uo = np.empty((KE, Q + 1)), np.empty((KO, Q)), np.empty((I, KE)), np.empty((I, KO))
    check(lib().fcc_plan_bases_noalloc(ctypes.byref(desc), ctypes.byref(info), se.ctypes.data_as(_dp),
                                       so.ctypes.data_as(_dp), Pe.ctypes.data_as(_dp), Po.ctypes.data_as(_dp),
                                       Ue.ctypes.data_as(_dp), Uo.ctypes.data_as(_dp), st),
          "fcc_plan_bases_noalloc")
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}, se, so, Pe, Po, Ue, Uo


_fptr = ctypes.POINTER(ctypes.c_float)


class MLP:
    """The learned TDoA head (include/fcc_mlp.h): 2K -> 128 -> 128 -> 2 with BF16
    weights and FP32 masters, trained by the library's own kernels."""

    HIDDEN = 128

    def __init__(self, n_in: int, params: np.ndarray, in_scale=None, conf_weight: float = 0.1,
                 device: int | None = None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device, self.n_in = int(device), int(n_in)
        self.n_params = int(lib().fcc_mlp_num_params(self.n_in, self.HIDDEN))
        p = np.ascontiguousarray(params, np.float32).ravel()
        if p.size != self.n_params:
            raise ValueError(f"params must hold {self.n_params} floats")
        sc = None
        if in_scale is not None:
            sc = np.ascontiguousarray(np.broadcast_to(np.asarray(in_scale, np.float32), (self.n_in,)))
        h = _vp()
        check(lib().fcc_mlp_create(self.n_in, self.HIDDEN, None if sc is None else sc.ctypes.data_as(_fptr),
                                   float(conf_weight), p.ctypes.data_as(_fptr), self.device, ctypes.byref(h)),
              "fcc_mlp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().fcc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_state(self):
        p, m, v = (np.empty(self.n_params, np.float32) for _ in range(3))
        step = ctypes.c_longlong()
        check(lib().fcc_mlp_get_state(self._h, p.ctypes.data_as(_fptr), m.ctypes.data_as(_fptr),
                                      v.ctypes.data_as(_fptr), ctypes.byref(step)), "fcc_mlp_get_state")
        return p, m, v, step.value

    def set_state(self, params, m=None, v=None, step: int = 0):
        arrs = [None if a is None else np.ascontiguousarray(a, np.float32).ravel() for a in (params, m, v)]
        ptrs = [None if a is None else a.ctypes.data_as(_fptr) for a in arrs]
        check(lib().fcc_mlp_set_state(self._h, *ptrs, int(step)), "fcc_mlp_set_state")

    def _check(self, feat, *vecs):
        import torch
        if feat.dtype != torch.float32 or feat.dim() != 2 or feat.shape[1] != self.n_in or not feat.is_contiguous():
            raise ValueError(f"features must be contiguous float32 [n, {self.n_in}]")
        for v in vecs:
            if v is not None and (v.dtype != torch.float32 or v.numel() != feat.shape[0] or not v.is_contiguous()):
                raise ValueError("per-sample vectors must be contiguous float32 [n]")

    def gradient(self, feat, tau_true, tau_fcc, stream=None):
        """(grad [n_params], mean loss) as device tensors."""
        import torch
        self._check(feat, tau_true, tau_fcc)
        g = torch.empty(self.n_params, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        check(lib().fcc_mlp_gradient(self._h, _ptr(feat), _ptr(tau_true), _ptr(tau_fcc), feat.shape[0], _ptr(g),
                                     _ptr(loss), _stream(stream, feat.device)), "fcc_mlp_gradient")
        return g, loss

    def train_step(self, feat, tau_true, tau_fcc, lr: float, loss=None, stream=None):
        """One Adam step; the batch loss (before the update) goes to `loss` if given."""
        self._check(feat, tau_true, tau_fcc)
        check(lib().fcc_mlp_train_step(self._h, _ptr(feat), _ptr(tau_true), _ptr(tau_fcc), feat.shape[0],
                                       float(lr), _ptr(loss), _stream(stream, feat.device)), "fcc_mlp_train_step")

    def sync(self, stream=None):
        """Synchronise and raise if the inference kernel latched a timeout."""
        import torch
        check(lib().fcc_mlp_sync(self._h, _stream(stream, torch.device("cuda", self.device))), "fcc_mlp_sync")

    def infer(self, feat, tau_fcc=None, threshold: float = 0.5, stream=None, out=None):
        """dict(tau, conf, raw) of device tensors [n]."""
        import torch
        self._check(feat, tau_fcc)
        n = feat.shape[0]
        if out is None:
            out = {k: torch.empty(n, dtype=torch.float32, device=feat.device) for k in ("tau", "conf", "raw")}
        check(lib().fcc_mlp_infer(self._h, _ptr(feat), _ptr(tau_fcc), n, float(threshold), _ptr(out["tau"]),
                                  _ptr(out.get("conf")), _ptr(out.get("raw")), _stream(stream, feat.device)),
              "fcc_mlp_infer")
        return out


def _desc(n_mics, fs, N, lag_den, tau_max=0.0, mic_xyz=None, c=343.0, K=0, energy=0.999, keep=None):
    xyz = None
    if mic_xyz is not None:
        xyz = np.ascontiguousarray(mic_xyz, np.float64).reshape(n_mics, 3)
        if keep is not None:
            keep.append(xyz)
    return PlanDesc(int(n_mics), xyz.ctypes.data_as(_dp) if xyz is not None else None, float(fs), int(N), float(c),
                    float(tau_max), int(lag_den), int(K), float(energy), 0, 0)


_DESC_KEYS = ("n_mics", "fs", "N", "lag_den", "tau_max", "mic_xyz", "c", "K", "energy")


class Batch:
    """Many arrays in persistent launches under one CUDA graph (include/fcc_batch.h):
    one per kernel class, or one for the whole batch with single_launch=True.

    `arrays`: list of dicts with the Plan keywords (n_mics, fs, N, lag_den and
    optionally tau_max, mic_xyz, c, K, energy) plus T (frames); other keys are
    ignored."""

    def __init__(self, arrays, device: int | None = None, autotune: bool = False, tune_cache: str | None = None,
                 single_launch: bool = False):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        keep = []
        n = len(arrays)
        descs = (PlanDesc * n)()
        T = (ctypes.c_longlong * n)()
        for a, d in enumerate(arrays):
            kw = {k: v for k, v in d.items() if k in _DESC_KEYS}
            descs[a] = _desc(keep=keep, **kw)
            T[a] = int(d["T"])
        h = _vp()
        flags = (FCC_BATCH_AUTOTUNE if autotune else 0) | (FCC_BATCH_SINGLE_LAUNCH if single_launch else 0)
        check(lib().fcc_batch_create(descs, T, n, self.device, flags,
                                     tune_cache.encode() if tune_cache else None, ctypes.byref(h)),
              "fcc_batch_create")
        self._h = h
        self.T = [int(d["T"]) for d in arrays]
        self.arrays = []
        for a in range(n):
            info = PlanInfo()
            check(lib().fcc_batch_array_info(h, a, ctypes.byref(info)), "fcc_batch_array_info")
            self.arrays.append({k: getattr(info, k) for k, _ in PlanInfo._fields_})
        self._bound = None

    def info(self) -> dict:
        i = BatchInfo()
        check(lib().fcc_batch_info(self._h, ctypes.byref(i)), "fcc_batch_info")
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def outputs(self, tau_hat: bool = True):
        """Device output tensors for every array: list of dicts."""
        import torch
        dev = torch.device("cuda", self.device)
        out = []
        for a, info in enumerate(self.arrays):
            o = {"lag_idx": torch.empty((self.T[a], info["P"]), dtype=torch.int32, device=dev),
                 "peak": torch.empty((self.T[a], info["P"]), dtype=torch.float32, device=dev)}
            if tau_hat:
                o["tau_hat"] = torch.empty((self.T[a], info["P"]), dtype=torch.float32, device=dev)
            out.append(o)
        return out

    def bind(self, spectra, outputs):
        """Bind device spectra (list of complex64 [T, M, B] tensors) and outputs."""
        n = len(self.arrays)
        if len(spectra) != n or len(outputs) != n:
            raise ValueError("one spectra tensor and one output dict per array")
        for a, X in enumerate(spectra):
            info = self.arrays[a]
            if tuple(X.shape) != (self.T[a], info["M"], info["B"]) or not X.is_contiguous():
                raise ValueError(f"array {a}: spectra must be contiguous [{self.T[a]}, {info['M']}, {info['B']}]")
        P = (_vp * n)
        sp, ix, pk = P(), P(), P()
        has_tau = any("tau_hat" in o for o in outputs)
        tu = P() if has_tau else None
        for a in range(n):
            sp[a] = spectra[a].data_ptr()
            ix[a] = outputs[a]["lag_idx"].data_ptr()
            pk[a] = outputs[a]["peak"].data_ptr()
            if has_tau:
                tu[a] = outputs[a]["tau_hat"].data_ptr() if "tau_hat" in outputs[a] else None
        check(lib().fcc_batch_bind(self._h, sp, ix, pk, tu), "fcc_batch_bind")
        self._bound = (spectra, outputs)  # keep the tensors alive while bound

    def run(self, stream=None):
        check(lib().fcc_batch_run(self._h, _stream(stream, self.device)), "fcc_batch_run")

    def sync(self, stream=None):
        check(lib().fcc_batch_sync(self._h, _stream(stream, self.device)), "fcc_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            lib().fcc_batch_destroy(self._h)
            self._h = None
            self._bound = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
