"""FCC TDoA benchmark on the 8-mic circle workload (2^20 frames, 28 pairs).

One step = one pass of the whole FCC path (PHAT -> fold -> projection ->
reconstruction on the lag grid -> argmax -> quadratic refinement) over every
frame and pair of the workload, with the spectra already resident in HBM.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fcc|reference]
                  [--workload circle8|grid16|square4|batched|learned]

The default line is the 8-mic circle.  --workload batched times 4096
independent arrays under one CUDA graph; --workload learned trains and
evaluates the learned head (RMSE in samples).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.  Under torchrun every rank runs its own 2^20 frames
(weak scaling, no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDoA pair-frames/s, FCC vs GCC-PHAT on 1 GB300 at stated accuracy; % HBM roofline"
UNIT = "pair-frames/s"


# ----------------------------------------------------------------------------
# distributed plumbing (host logic; exercised on CPU with gloo in the tests)
# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29512")
        dist.init_process_group(backend)
    return dist.is_initialized()


def barrier(enabled):
    if enabled:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, enabled: bool, device="cpu") -> float:
    if not enabled:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Weak scaling: every rank processes `units_per_rank`; the job's rate is all
    ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def rank_seed(rank: int) -> int:
    """Seed of the scene segment a rank's frames come from (disjoint segments of
    one scene, same statistics)."""
    return 2 + 7919 * rank


def rank_frames(T: int, rank: int, world: int):
    """Weak scaling: the job's scene has world * T frames and rank r takes the
    contiguous slice binding.frame_range(world * T, r, world) of it."""
    from paper_2204_13622_gb300 import binding
    return binding.frame_range(world * T, rank, world)


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling (every 100 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)  # first sample before the timed work starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            cols = [c.strip() for c in line.split(",")]
            if len(cols) == 9:
                self.rows.append(cols)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in self.rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in self.rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in self.rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ----------------------------------------------------------------------------
def oracle_rate(w, budget_s: float, X_sample_fn, threads=None):
    """Time the FP64 oracle (as it stands) on a sample sized to ~budget_s."""
    from oracle import oracle as O
    basis = O.Basis(w.N, w.L, w.lag_den)
    nt = len(os.sched_getaffinity(0)) if threads is None else threads
    X = X_sample_fn(64)
    t0 = time.perf_counter()
    O.tdoa(X, basis.WK, basis.taus, basis.delta, threads=nt)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(w.T, max(64, 64 * budget_s / dt)))
    X = X_sample_fn(n)
    t0 = time.perf_counter()
    O.tdoa(X, basis.WK, basis.taus, basis.delta, threads=nt)
    dt = time.perf_counter() - t0
    return {"value": n * w.P / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"first {n} frames of the {w.name} workload ({n * w.P} pair-frames), "
                      f"FP64 C oracle, {dt:.1f} s on {nt} host threads"}, n, dt


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample."""
    from paper_2204_13622_gb300 import workloads
    w = workloads.CIRCLE8
    if rank != 0:
        return None
    # each step is a bounded sample sized so the whole run stays near 1.5 minutes
    budget = float(os.environ.get("FCC_REF_STEP_SECONDS", str(max(0.5, min(8.0, 90.0 / max(1, args.steps))))))
    sample = {}

    def gen(n):
        if n not in sample:
            sample[n] = w.spectra(T=n, seed=rank_seed(0)).numpy()
        return sample[n]
    # every host core this process may use (a launcher's OMP_NUM_THREADS = 1 would
    # otherwise leave the oracle on one thread)
    nt = len(os.sched_getaffinity(0))
    info, n, _ = oracle_rate(w, budget / 2, gen, threads=nt)
    from oracle import oracle as O
    basis = O.Basis(w.N, w.L, w.lag_den)
    X = gen(n)
    for _ in range(args.warmup):
        O.tdoa(X[: max(1, n // 8)], basis.WK, basis.taus, basis.delta, threads=nt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.tdoa(X, basis.WK, basis.taus, basis.delta, threads=nt)
        times.append(time.perf_counter() - t0)
    v = n * w.P * args.steps / sum(times)
    info["value"] = v
    return {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "frames_per_step": n, "pairs": w.P,
                                            "sample": "bounded CPU sample of the workload"},
            "cpu_baseline": info,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def accuracy_vs_oracle(w, plan, X, out, n=1 << 14):
    """Argmax agreement and peak error against the FP64 oracle on n frames spread
    evenly over the seeded workload (2^14 frames: 458 752 pair-frames on the
    8-mic circle, 1.97 M on the 16-mic grid)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    T = X.shape[0]
    n = min(n, T)
    frames = torch.from_numpy(np.linspace(0, T - 1, n).astype(np.int64)).to(X.device)
    Xs = X[frames].cpu().numpy()
    ref = O.Basis(w.N, w.L, w.lag_den)  # K from the oracle's own energy rule
    if ref.K != plan.K:
        raise RuntimeError(f"plan K {plan.K} differs from the oracle's K {ref.K}")
    idx, peak, _, y = O.tdoa(Xs, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"][frames].cpu().numpy()
    gp = out["peak"][frames].cpu().numpy()
    scale = np.abs(y).max(-1)
    srt = np.sort(y, -1)
    clear = (srt[..., -1] - srt[..., -2]) / scale > 4e-6
    return {"frames_sampled": n, "pair_frames": int(gi.size),
            "argmax_agreement": float((gi == idx).mean()),
            "argmax_agreement_clear": float((gi == idx)[clear].mean()),
            "peak_rel_err_median": float(np.median(np.abs(gp - peak) / scale)),
            "peak_rel_err_max": float(np.max(np.abs(gp - peak) / scale))}


def accuracy_time_domain(w, plan, n_frames=1 << 14, seed=7):
    """Accuracy on a subset made by the time-domain path (one far-field white
    source per recording, fractional delays on the full-signal FFT, white noise
    at 20 dB, STFT): FCC on the GPU against the FP64 oracle on every pair-frame,
    and the refined TDoA against the true delays t_i - t_j."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2204_13622_gb300 import synth
    n_samples = (n_frames - 1) * w.hop + w.N
    rec = synth.time_domain_spectra(w.xyz, w.fs, w.N, w.hop, n_samples, seed=seed, elevation=0.3)
    X = torch.from_numpy(np.ascontiguousarray(rec.spectra)).to(torch.device("cuda", plan.device))
    out = plan.tdoa(X)
    plan.sync()
    ref = O.Basis(w.N, w.L, w.lag_den)
    if ref.K != plan.K:
        raise RuntimeError(f"plan K {plan.K} differs from the oracle's K {ref.K}")
    idx, _, _, y = O.tdoa(rec.spectra, ref.WK, ref.taus, ref.delta, want_y=True)
    gi = out["lag_idx"].cpu().numpy()
    srt = np.sort(y, -1)
    clear = (srt[..., -1] - srt[..., -2]) / np.abs(y).max(-1) > 4e-6
    pairs = [(i, j) for i in range(w.M) for j in range(i + 1, w.M)]
    true = np.array([rec.delays[i] - rec.delays[j] for i, j in pairs])
    err = out["tau_hat"].cpu().numpy() - true[None, :]
    return {"frames": int(rec.spectra.shape[0]), "pair_frames": int(gi.size),
            "argmax_agreement": float((gi == idx).mean()),
            "argmax_agreement_clear": float((gi == idx)[clear].mean()),
            "tau_rmse_samples": float(np.sqrt(np.mean(err ** 2))),
            "source": "time-domain path: one far-field white source, 20 dB white noise"}


def run_fcc(args, rank, world, local):
    import torch

    from paper_2204_13622_gb300 import binding, flops, workloads
    w = {"circle8": workloads.CIRCLE8, "grid16": workloads.GRID16, "square4": workloads.SQUARE4}[args.workload]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    T, P = (args.frames or w.T), w.P
    t0, t1 = rank_frames(T, rank, world)  # this rank's slice of the job's frames
    X = w.spectra(T=t1 - t0, device=dev, seed=rank_seed(rank))
    plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, device=local, prec=args.prec, engine=args.engine)
    out = plan.tdoa(X, tau_hat=True)  # allocates the outputs once
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.tdoa(X, out=out)
    plan.sync()

    # ---- device-resident timing: one fcc_tdoa launch per step
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            plan.tdoa(X, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    plan.sync()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    value = whole_job_rate(T * P, world, ms_max / 1000.0)

    # ---- roofline of the dominant (only) kernel: algorithmic bytes per launch
    bytes_per_launch = T * (w.M * w.B * 8) + T * P * 12  # spectra read + idx/peak/tau_hat written
    # and its CUDA-core arithmetic: FP32 operations per pair-frame (FMA = 1)
    ops_pf = fp32_ops_per_pair_frame(w.M, w.N, plan.K_even, plan.K_odd, plan.I)
    acc = accuracy_vs_oracle(w, plan, X, out) if rank == 0 else None
    achieved = bytes_per_launch / (ms / 1000.0) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))

    if args.only == "fcc":
        res = None
        if rank == 0:
            res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                   "warmup": args.warmup, "ms_per_step": ms_max, "config": {"workload": w.name, "frames": T},
                   "note": "FCC kernel only (profiling run)", "roofline_achieved_gbs": achieved,
                   "engine": plan.engine,
                   "dtype": args.prec, "roofline_frac": achieved / float(json.load(open(os.path.join(
                       ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) if os.path.exists(os.path.join(
                           ROOT, "MEASURED_PEAKS.json")) else None, "accuracy_vs_oracle": acc,
                   "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
        plan.close()
        return res

    # ---- same-GPU GCC-PHAT baseline on the same frames
    gout = plan.gcc_tdoa(X)
    plan.gcc_tdoa(X, out=gout)
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gsteps = max(1, min(args.steps, 2))
    g0.record(stream)
    for _ in range(gsteps):
        plan.gcc_tdoa(X, out=gout)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    plan.sync()
    gms = g0.elapsed_time(g1) / gsteps
    agree = float((gout["lag_idx"] == out["lag_idx"]).float().mean().item())
    # the paper's GCC setting, r = 2 (a grid of step 1/2 over the same lag range), for context
    gcc2 = None
    if w.lag_den != 2:
        p2 = binding.Plan(w.M, w.fs, w.N, 2, tau_max=w.L, device=local)
        g2 = p2.gcc_tdoa(X)
        torch.cuda.synchronize(dev)
        g0.record(stream)
        for _ in range(gsteps):
            p2.gcc_tdoa(X, out=g2)
        g1.record(stream)
        torch.cuda.synchronize(dev)
        p2.sync()
        g2ms = g0.elapsed_time(g1) / gsteps
        gcc2 = {"value": world * T * P / (g2ms / 1000.0), "unit": UNIT, "ms_per_step": g2ms, "r": 2}
        del g2
        p2.close()

    # ---- end to end through the host entry point (pinned host in, host out)
    Xh = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    Xh.copy_(X)
    del X
    torch.cuda.empty_cache()
    hout = {"lag_idx": torch.empty((T, P), dtype=torch.int32, pin_memory=True),
            "peak": torch.empty((T, P), dtype=torch.float32, pin_memory=True),
            "tau_hat": torch.empty((T, P), dtype=torch.float32, pin_memory=True)}
    plan.tdoa_host(Xh, out=hout)  # warm (allocates the staging ring)
    e2e_steps = max(1, min(args.steps, 3))
    barrier(distributed)
    e2e_per = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        plan.tdoa_host(Xh, out=hout)
        e2e_per.append(time.perf_counter() - t0)
    e2e_s = sum(e2e_per) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, distributed, dev)
    # the host link runs at about 211 GB/s with intermittent slow periods, so the
    # per-step times are kept beside the mean
    e2e = {"value": world * T * P / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(Xh.numel() * 8),
           "d2h_bytes_per_step": int(T * P * 12), "ms_per_step": 1000 * e2e_s,
           "step_ms": [round(1000 * x, 1) for x in e2e_per]}

    res = None
    if rank == 0:
        cpu, _, _ = oracle_rate(w, float(os.environ.get("FCC_CPU_BASELINE_SECONDS", "12")),
                                lambda n: Xh[:n].numpy())
        # the same oracle on one host thread, on a smaller sample
        cpu1, _, _ = oracle_rate(w, 2.0, lambda n: Xh[:n].numpy(), threads=1)
        cpu["single_thread"] = {"value": cpu1["value"], "sample": cpu1["sample"]}
        cpu["host"] = {"machine": platform.machine(), "nproc": os.cpu_count()}
        # DRAM bytes per launch from the committed ncu capture, valid only while
        # the kernel source is the one that was captured
        traffic = None
        tfile = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tfile) and args.workload == "circle8" and args.prec == "fp32":
            import hashlib
            rec = json.load(open(tfile))
            h = hashlib.sha256()
            for f in rec.get("source_files", []):
                h.update(open(os.path.join(ROOT, f), "rb").read())
            if rec.get("source_files") and h.hexdigest()[:16] == rec.get("fcc_fp32_kernel_source_sha256_16"):
                traffic = rec.get("fcc_fp32_kernel_circle8_bytes_per_launch")
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp16": "f16"}[args.prec],
            "data": "synthetic", "accuracy_vs_oracle": acc,
            "config": {"workload": w.name if T == w.T else f"{w.name} truncated to {T} frames",
                       "frames": T, "mics": w.M, "pairs": P, "N": w.N,
                       "lag_grid": f"[-{w.L}, {w.L}] step 1/{w.lag_den} (I={plan.I})",
                       "K": plan.K, "K_even": plan.K_even, "K_odd": plan.K_odd,
                       "outputs": "lag_idx, peak, tau_hat",
                       "l2": "inputs (17.25 GB) larger than L2; no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "fcc_fp32_kernel" if args.prec == "fp32" else "fcc_tc_kernel",
                         "bytes_per_launch": bytes_per_launch,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"},
            "roofline_alu": alu_roofline(ops_pf * T * P, ms, "fcc_fp32_kernel") if args.prec == "fp32" else None,
            "gcc_phat": {"value": world * T * P / (gms / 1000.0), "unit": UNIT, "ms_per_step": gms,
                         "r": w.lag_den, "argmax_agreement_with_fcc": agree},
            "gcc_phat_r2": gcc2,
            "accuracy_time_domain": (accuracy_time_domain(w, plan) if args.workload == "circle8"
                                     and args.prec == "fp32" else None),
            "fcc_vs_gcc": (gms / ms),
            "flops_per_pair_frame": {"fcc_paper": flops.fcc_flops(w.N, plan.I, plan.K),
                                     "gcc_paper_r": flops.gcc_flops(w.N, w.lag_den)},
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
    plan.close()
    return res


# FP32 pipe of one GB300: 152 SMs x 128 FP32 lanes x 2070 MHz (maximum SM clock),
# one FMA (or add, or multiply) per lane per clock
FP32_PEAK_OPS = 152 * 128 * 2.070e9


def fp32_ops_per_pair_frame(M: int, N: int, KE: int, KO: int, I: int) -> float:
    """FP32 operations per pair-frame of the FP32 kernel's arithmetic (FMA = 1):
    the cross spectrum (4 per bin), the Eq. 8 fold (4 per bin pair), the even and
    odd projections (2 per basis and bin), the reconstruction over tau >= 0 (per
    lag step m, S = sum of K weights times Re z and D = sum of K weights times
    Im z, then y(-m) = S + D and y(+m) = S - D: 2K + 2) and this pair's share of
    the per-microphone PHAT (5 per microphone bin)."""
    B, Q = N // 2 + 1, N // 4
    P = M * (M - 1) // 2
    center = (I - 1) // 2
    return (4 * B + 4 * Q + 2 * (KE * (Q + 1) + KO * Q) + (center + 1) * (2 * (KE + KO) + 2)
            + 5.0 * M * B / P)


def reim_ops_per_pair_frame(M: int, N: int, Kc: int, Ks: int, I: int) -> float:
    """FP32 operations per pair-frame of the split form at alpha = 1 (FMA = 1):
    the cross spectrum (4 per bin), the cosine and sine projections (one per
    basis and bin: c = C_K-rows . Re x, s = S_K-rows . Im x, no fold), the
    reconstruction over tau >= 0 (K_c + K_s + 2 per lag step, both signs at
    once) and this pair's share of the per-microphone PHAT (5 per microphone
    bin)."""
    B = N // 2 + 1
    P = M * (M - 1) // 2
    center = (I - 1) // 2
    return 4 * B + (Kc + Ks) * B + (center + 1) * (Kc + Ks + 2) + 5.0 * M * B / P


def smooth_ops_per_pair_frame(M: int, N: int, KE: int, KO: int, I: int) -> float:
    """FP32 operations per pair-frame of one smoothed step (Eq. 1; FMA = 1): the
    chunk-sum pass (cross spectrum 4 + update 2 per bin) and the main pass
    (cross spectrum 4, update 2 and phase transform 6 per bin: power-of-two
    scaling 2, |R|^2 2, final scaling 2), then the fold, the projections and the
    reconstruction as the unsmoothed kernel.  Rsqrt and the carry scan are not
    counted."""
    B, Q = N // 2 + 1, N // 4
    center = (I - 1) // 2
    return (6 * B + 12 * B + 4 * Q + 2 * (KE * (Q + 1) + KO * Q) + (center + 1) * (2 * (KE + KO) + 2))


SMEM_PEAK_BPS = 152 * 128 * 2.070e9  # shared memory: 128 bytes per clock per SM


def smem_roofline(nbytes: float, ms: float, kernel: str, alu=None) -> dict:
    """A kernel bound by shared-memory bandwidth: `nbytes` the algorithmic bytes
    read from shared memory per launch (8 per candidate, pair and frame for the
    DoA search: the interpolation pair (y_k, y_{k+1} - y_k))."""
    achieved = nbytes / (ms / 1000.0)
    r = {"bound": "smem", "achieved": achieved / 1e9, "peak": SMEM_PEAK_BPS / 1e9, "unit": "GB/s",
         "frac": achieved / SMEM_PEAK_BPS, "kernel": kernel, "bytes_per_launch": nbytes, "traffic": None,
         "peak_source": "152 SMs x 128 B/clock x 2070 MHz"}
    if alu is not None:
        r["alu"] = {k: alu[k] for k in ("achieved", "peak", "unit", "frac")}
    return r


def alu_roofline(ops: float, ms: float, kernel: str) -> dict:
    achieved = ops / (ms / 1000.0)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": FP32_PEAK_OPS / 1e12, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_OPS, "kernel": kernel, "ops_per_launch": ops,
            "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (FMA counted once)"}


def _peak_hbm():
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(f):
        return float(json.load(open(f)).get("hbm_gbs", 6800.0)), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback"


def run_precision(args, local, steps):
    """The 16-microphone grid (2^18 frames, N = 1024, I = 193, K = 15) in the three
    precisions: FP32 (CUDA-core projection), BF16 and FP16 (tcgen05 projection,
    FP32 accumulation).  Per precision: device time per pass, pair-frames/s, the
    HBM roofline of its kernel, and agreement with the FP64 oracle on 2^14
    frames spread over the workload (the oracle runs once; every precision is
    compared with the same values)."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2204_13622_gb300 import binding, workloads
    w = workloads.GRID16
    dev = torch.device("cuda", local)
    T, P = w.T, w.P
    X = w.spectra(T=T, device=dev, seed=rank_seed(0) + 1)
    n = min(1 << 14, T)
    frames = torch.from_numpy(np.linspace(0, T - 1, n).astype(np.int64)).to(dev)
    Xs = X[frames].cpu().numpy()
    ref = O.Basis(w.N, w.L, w.lag_den)
    t0 = time.perf_counter()
    idx, peak, _, y = O.tdoa(Xs, ref.WK, ref.taus, ref.delta, want_y=True)
    t_or = time.perf_counter() - t0
    scale = np.abs(y).max(-1)
    srt = np.sort(y, -1)
    clear = (srt[..., -1] - srt[..., -2]) / scale > 4e-6
    del y, srt
    peak_hbm, psrc = _peak_hbm()
    bytes_per_launch = T * (w.M * w.B * 8) + T * P * 12
    stream = torch.cuda.current_stream(dev)
    res = {"workload": w.name, "frames": T, "mics": w.M, "pairs": P, "N": w.N,
           "lag_grid": f"[-{w.L}, {w.L}] step 1/{w.lag_den}", "K": ref.K, "steps": steps,
           "oracle_sample": f"{n} frames spread over the workload ({n * P} pair-frames), FP64 C oracle "
                            f"({t_or:.1f} s on {O.max_threads()} host threads)",
           "l2": f"inputs ({X.numel() * 8 / 1e9:.1f} GB) larger than L2; no flush"}
    for prec in ("fp32", "bf16", "fp16"):
        plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, device=local, prec=prec)
        if plan.K != ref.K:
            raise RuntimeError(f"{prec} plan K {plan.K} differs from the oracle's K {ref.K}")
        out = plan.tdoa(X, tau_hat=True)
        for _ in range(3):
            plan.tdoa(X, out=out)
        plan.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clk:
            ev[0].record(stream)
            for k in range(steps):
                plan.tdoa(X, out=out)
                ev[k + 1].record(stream)
            torch.cuda.synchronize(dev)
        plan.sync()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        ms = sum(per) / steps
        gi = out["lag_idx"][frames].cpu().numpy()
        gp = out["peak"][frames].cpu().numpy()
        achieved = bytes_per_launch / (ms / 1000.0) / 1e9
        res[prec] = {"ms_per_step": ms, "value": T * P / (ms / 1000.0), "unit": UNIT,
                     "step_ms": [round(x, 3) for x in per], "gpu_launches": steps,
                     "kernel": "fcc_fp32_kernel" if prec == "fp32" else "fcc_tc_kernel",
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                                  "frac": achieved / peak_hbm, "bytes_per_launch": bytes_per_launch,
                                  "peak_source": psrc},
                     "accuracy_vs_oracle": {
                         "pair_frames": int(gi.size), "argmax_agreement": float((gi == idx).mean()),
                         "argmax_agreement_clear": float((gi == idx)[clear].mean()),
                         "peak_rel_err_median": float(np.median(np.abs(gp - peak) / scale)),
                         "peak_rel_err_max": float(np.max(np.abs(gp - peak) / scale))},
                     "clocks": clk.summary()}
        if prec == "fp32":
            res[prec]["roofline_alu"] = alu_roofline(
                fp32_ops_per_pair_frame(w.M, w.N, plan.K_even, plan.K_odd, plan.I) * T * P, ms, "fcc_fp32_kernel")
        del out
        plan.close()
    del X
    torch.cuda.empty_cache()
    return res


def run_batched(args, rank, world, local):
    """Batched form: 4096 independent arrays (mixed M, aperture, N, fs, T) in one
    persistent launch per kernel class (or one for the batch) captured in a CUDA
    graph; one step = one graph launch over every frame and pair of every array."""
    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    arrs = synth.batched_arrays(args.arrays, seed=4 + 7919 * rank)
    t0 = time.perf_counter()
    cache = os.environ.get("FCC_TUNE_CACHE") or os.path.join("/tmp", f"fcc_tune_{os.getpid()}.json")
    batch = binding.Batch(arrs, device=local, autotune=args.autotune, tune_cache=cache,
                          single_launch=args.batch_single_launch)
    t_create = time.perf_counter() - t0
    info = batch.info()
    need = info["spectra_bytes"] + 1.5 * info["pair_frames"] * 12
    free, _ = torch.cuda.mem_get_info(dev)
    if need > 0.97 * free:
        raise RuntimeError(f"batched workload needs {need / 1e9:.1f} GB, {free / 1e9:.1f} GB free")
    X = [synth.array_spectra(a, device=dev) for a in arrs]
    out = batch.outputs(tau_hat=True)
    batch.bind(X, out)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        batch.run(stream)
    batch.sync(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            batch.run(stream)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    batch.sync(stream)
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    value = whole_job_rate(info["pair_frames"], world, ms_max / 1000.0)
    bytes_per_step = info["spectra_bytes"] + info["result_bytes"]
    achieved = bytes_per_step / (ms / 1000.0) / 1e9
    ops = sum(fp32_ops_per_pair_frame(a["M"], a["N"], a["K_even"], a["K_odd"], a["I"]) * t * a["P"]
              for a, t in zip(batch.arrays, batch.T))
    peak, psrc = _peak_hbm()
    res = None
    if rank == 0:
        # accuracy: 8 arrays x 16 frames against the FP64 oracle; CPU baseline:
        # the oracle on the same sample
        from oracle import oracle as O
        agree, n_pf, t_or = [], 0, 0.0
        for a in np.linspace(0, len(arrs) - 1, 8).astype(int):
            inf = batch.arrays[a]
            basis = O.Basis(inf["N"], inf["L"], inf["den"], K=inf["K"])
            Xs = X[a][:16].cpu().numpy()
            t1 = time.perf_counter()
            idx, _, _, y = O.tdoa(Xs, basis.WK, basis.taus, basis.delta, want_y=True)
            t_or += time.perf_counter() - t1
            n_pf += idx.size
            agree.append((out[a]["lag_idx"][:16].cpu().numpy() == idx).astype(np.float64).ravel())
        agree = np.concatenate(agree)
        res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": f"batched: {args.arrays} arrays, M in {{2,4,6,8,12,16}}, aperture 2-8 cm, "
                                      "N in {256,512,1024}, fs in {16,48} kHz, 64-4096 frames each",
                          "arrays": info["n_arrays"], "frames": info["frames"], "pair_frames": info["pair_frames"],
                          "classes": info["n_classes"], "launches": info["n_launches"], "jobs": info["n_jobs"],
                          "bases": info["n_bases"],
                          "autotune": bool(args.autotune), "create_s": round(t_create, 2),
                          "l2": f"inputs ({info['spectra_bytes'] / 1e9:.1f} GB) larger than L2; no flush"},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None, "kernel": "fcc_fp32_batch_kernel",
                            "bytes_per_launch": bytes_per_step, "peak_source": psrc},
               "roofline_alu": alu_roofline(ops, ms, "fcc_fp32_batch_kernel"),
               "accuracy_vs_oracle": {"pair_frames": int(n_pf), "argmax_agreement": float(agree.mean())},
               "cpu_baseline": {"value": n_pf / t_or, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                                "sample": f"16 frames of 8 arrays ({n_pf} pair-frames), FP64 C oracle"},
               "e2e": None, "gpu_launches": args.steps * info["n_launches"],
               "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
    batch.close()
    return res


def run_pcm(args, rank, world, local):
    """STFT front-end: interleaved int16 PCM of the 8-mic circle in, per-pair
    TDoA out (fcc_tdoa_pcm: STFT and FCC chunk by chunk, the spectra kept in
    L2-sized chunks); e2e through fcc_tdoa_pcm_host from pinned host PCM."""
    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, synth, workloads
    w = workloads.CIRCLE8
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    T, P, hop = (args.frames or w.T), w.P, w.hop
    n = (T - 1) * hop + w.N
    pcm = synth.pcm_far_field(n, w.xyz, w.fs, seed=rank_seed(rank), device=dev)
    plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, mic_xyz=w.xyz, device=local)
    work = torch.empty(plan.pcm_workspace(n, hop), dtype=torch.uint8, device=dev)
    out = plan.tdoa_pcm(pcm, hop, work=work)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.tdoa_pcm(pcm, hop, work=work, out=out)
    plan.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            plan.tdoa_pcm(pcm, hop, work=work, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    plan.sync()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    res = None
    if rank == 0:
        # the stages alone over 2^18 frames: STFT to HBM, FCC from HBM
        nf = min(T, 1 << 18)
        sub = pcm[:(nf - 1) * hop + w.N]
        X = plan.stft(sub, hop)
        o = plan.tdoa(X)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for _ in range(2):
            e[0].record(stream)
            plan.stft(sub, hop, out=X)
            e[1].record(stream)
            plan.tdoa(X, out=o)
            e[2].record(stream)
        torch.cuda.synchronize(dev)
        stft_ms, fcc_ms = e[0].elapsed_time(e[1]) * T / nf, e[1].elapsed_time(e[2]) * T / nf
        del X, o
        # e2e: pinned host PCM in, host results out
        host = pcm.cpu().pin_memory()
        hout = plan.tdoa_pcm_host(host, hop)
        t1 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            plan.tdoa_pcm_host(host, hop, out=hout)
        e2e_s = (time.perf_counter() - t1) / reps
        h2d = host.numel() * host.element_size()
        d2h = T * P * 12
        # accuracy: 64 sampled frames through the FP64 chain (oracle STFT + FCC)
        from oracle import oracle as O
        sel = np.linspace(0, T - 1, 64).astype(np.int64)
        seg = torch.cat([pcm[t * hop:t * hop + w.N] for t in sel]).cpu().numpy()
        basis = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
        t2 = time.perf_counter()
        Xo = O.stft(seg, w.N, w.N).astype(np.complex64)
        idx, _, _, y = O.tdoa(Xo, basis.WK, basis.taus, basis.delta, want_y=True)
        t_or = time.perf_counter() - t2
        got = out["lag_idx"][torch.from_numpy(sel).to(dev)].cpu().numpy()
        srt = np.sort(y, axis=-1)
        clear = (srt[..., -1] - srt[..., -2]) > 4e-6 * np.abs(y).max(-1)
        H = w.N // 2
        import math as _m
        p4 = int(round(_m.log(H, 4) - 0.5))  # radix-4 passes
        r2 = 1 if 4 ** p4 < H else 0
        stft_ops = w.M * T * (p4 * (H // 4) * 28 + r2 * (H // 2) * 8 + (H + 1) * 14 + 2 * w.N)
        res = {"metric": METRIC, "value": whole_job_rate(T * P, world, ms_max / 1000.0), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"{w.name}, int16 PCM in (hop {hop}) through the STFT front-end",
                          "frames": T, "pairs": P, "pcm_bytes": h2d, "l2": "inputs larger than L2; no flush"},
               "stages_ms": {"stft_to_hbm": stft_ms, "fcc_from_hbm": fcc_ms},
               "e2e": {"value": T * P / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": e2e_s * 1000.0, "path": "fcc_tdoa_pcm_host, pinned host PCM"},
               "roofline": dict(alu_roofline(stft_ops, stft_ms, "stft_kernel (alone, spectra to HBM)"),
                                traffic=None, hbm_write_gb=T * w.M * w.B * 8 / 1e9),
               "accuracy_vs_oracle": {"pair_frames": int(got.size),
                                      "argmax_agreement_clear": float((got == idx)[clear].mean()),
                                      "argmax_agreement": float((got == idx).mean())},
               "cpu_baseline": {"value": len(sel) * P / t_or, "unit": UNIT, "cores": O.max_threads(),
                                "kind": "oracle", "sample": "64 frames: FP64 STFT + FP64 FCC"},
               "gpu_launches": 2 * args.steps * ((T + plan.pcm_workspace(n, hop) // (w.M * w.B * 8) - 1)
                                                 // (plan.pcm_workspace(n, hop) // (w.M * w.B * 8))),
               "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
    plan.close()
    return res


def run_doa(args, rank, world, local):
    """DoA search (the step after per-pair TDoA named in the paper's conclusion):
    spectra in, per frame the best of D candidate directions out, through
    fcc_tdoa_doa (FCC with the lag-grid correlations, chunk by chunk, then the
    search); also times FCC with the correlation output and the search alone."""
    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, synth, workloads
    w = workloads.CIRCLE8
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    T, P = (args.frames or w.T), w.P
    t0, t1 = rank_frames(T, rank, world)  # this rank's slice of the job's frames
    X = w.spectra(T=t1 - t0, device=dev, seed=rank_seed(rank))
    plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, mic_xyz=w.xyz, device=local)
    dirs = synth.fibonacci_directions(args.dirs)
    doa = binding.Doa(plan, w.xyz, dirs)
    work = torch.empty(doa.workspace(T), dtype=torch.uint8, device=dev)
    out = doa.tdoa_doa(X, work=work)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        doa.tdoa_doa(X, work=work, out=out)
    plan.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            doa.tdoa_doa(X, work=work, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    plan.sync()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    res = None
    if rank == 0:
        # the two stages alone: FCC with the correlation output, the search over it
        n = min(T, 1 << 18)
        o = plan.tdoa(X[:n], tau_hat=False, corr=True)
        s_out = doa.search(o["corr"])
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for _ in range(2):
            e[0].record(stream)
            plan.tdoa(X[:n], tau_hat=False, corr=True, out=o)
            e[1].record(stream)
            doa.search(o["corr"], out=s_out)
            e[2].record(stream)
        torch.cuda.synchronize(dev)
        fcc_ms, srp_ms = e[0].elapsed_time(e[1]) * T / n, e[1].elapsed_time(e[2]) * T / n
        # accuracy: 64 sampled frames against the oracle's FP64 correlations and search
        from oracle import oracle as O
        sel = np.linspace(0, T - 1, 64).astype(np.int64)
        basis = O.Basis(w.N, w.L, w.lag_den, K=plan.K)
        t1 = time.perf_counter()
        _, _, _, y = O.tdoa(X[sel].cpu().numpy(), basis.WK, basis.taus, basis.delta, want_y=True)
        ref_idx, _, scores = O.doa_srp(y, w.L, w.lag_den, w.xyz, w.fs, 343.0, dirs, want_scores=True)
        t_or = time.perf_counter() - t1
        got = out["dir_idx"][torch.from_numpy(sel).to(dev)].cpu().numpy()
        srp_ops = 2.0 * args.dirs * P * T  # one FMA and one add per (candidate, pair, frame)
        res = {"metric": METRIC, "value": whole_job_rate(T * P, world, ms_max / 1000.0), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"{w.name}, DoA search over {args.dirs} hemisphere candidates",
                          "frames": T, "pairs": P, "candidates": args.dirs,
                          "l2": "inputs larger than L2; no flush"},
               "frames_per_s": T / (ms_max / 1000.0),
               "stages_ms": {"fcc_with_corr": fcc_ms, "search": srp_ms},
               "roofline": smem_roofline(8.0 * args.dirs * P * T, srp_ms, "srp_kernel (the search alone)",
                                         alu=alu_roofline(srp_ops, srp_ms, "srp_kernel")),
               "accuracy_vs_oracle": {"frames": int(len(sel)),
                                      "dir_agreement": float((got == ref_idx).mean()),
                                      "score_loss_max": float((scores[np.arange(len(sel)), ref_idx]
                                                               - scores[np.arange(len(sel)), got]).max())},
               "cpu_baseline": {"value": len(sel) * P / t_or, "unit": UNIT, "cores": O.max_threads(),
                                "kind": "oracle", "sample": "64 frames: FP64 FCC correlations + FP64 search"},
               "gpu_launches": 2 * args.steps * ((T + doa_chunk(doa, T) - 1) // doa_chunk(doa, T)),
               "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
    doa.close()
    plan.close()
    return res


def doa_chunk(doa, T):
    """Frames per chunk of fcc_tdoa_doa (its workspace holds one chunk's
    correlations, lag indices and peaks: P (I + 2) 4 bytes per frame)."""
    p = doa.plan
    return max(1, min(T, doa.workspace(T) // (p.P * (p.I + 2) * 4)))


def run_split_form(args, rank, world, local):
    """The split form (cosine bases on Re x, sine bases on Im x) on the 8-mic
    circle: fcc_tdoa on a FCC_FORM_REIM_SPLIT plan (the FP32 tile kernel's
    split-form instance), alpha = 1."""
    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, workloads
    w = {"circle8": workloads.CIRCLE8, "square4": workloads.SQUARE4}[args.workload]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    T, P = (args.frames or w.T), w.P
    t0, t1 = rank_frames(T, rank, world)  # this rank's slice of the job's frames
    X = w.spectra(T=t1 - t0, device=dev, seed=rank_seed(rank))
    plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, device=local, form="reim")
    out = plan.tdoa(X)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.tdoa(X, out=out)
    plan.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            plan.tdoa(X, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    plan.sync()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    res = None
    if rank == 0:
        from oracle import oracle as O
        n = min(256, T)
        ob = O.BasisB(w.N, w.L, w.lag_den)
        t1 = time.perf_counter()
        idx, _, _, _ = O.tdoa(X[:n].cpu().numpy(), ob.WK, ob.taus, ob.delta)
        t_or = time.perf_counter() - t1
        got = out["lag_idx"][:n].cpu().numpy()
        ops = T * P * reim_ops_per_pair_frame(w.M, w.N, plan.K_even, plan.K_odd, plan.I)
        bytes_alg = T * (w.M * w.B * 8) + T * P * 12
        peak, psrc = _peak_hbm()
        res = {"metric": METRIC, "value": whole_job_rate(T * P, world, ms_max / 1000.0), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"{w.name}, split form (cosine / sine bases)", "frames": T, "pairs": P,
                          "K_c": plan.K_even, "K_s": plan.K_odd, "l2": "inputs larger than L2; no flush"},
               "roofline": dict(alu_roofline(ops, ms, "fcc_fp32_reim_kernel"), traffic=None,
                                hbm={"achieved": bytes_alg / (ms / 1000.0) / 1e9, "peak": peak,
                                     "frac": bytes_alg / (ms / 1000.0) / 1e9 / peak, "peak_source": psrc}),
               "accuracy_vs_oracle": {"pair_frames": int(got.size), "argmax_agreement": float((got == idx).mean())},
               "cpu_baseline": {"value": n * P / t_or, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                                "sample": f"first {n} frames, FP64 form B"},
               "gpu_launches": args.steps, "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
    plan.close()
    return res


def run_table1(args, rank, world, local):
    """Synthetic reproduction of the Table 1 accuracy sweep: two microphones
    d apart (d = 0.05 .. 0.15 m) in shoebox rooms made like the paper's (5-15 m
    by 5-15 m by 3-4 m, absorption 0.2-0.8, source 1-5 m away, c 335-350 m/s,
    white noise through image-source RIRs), STFT (N 512, hop 256) by the
    library's front-end, then FCC with K = 1..8 on the grid step 1/2 (Eq. 1
    smoothing alpha = 0.1, parabolic refinement) and GCC-PHAT with r = 1, 2, 4
    on the same smoothed cross-spectrum; MAE of theta = arccos(tau c / (d fs))
    in degrees against the geometric TDoA."""
    import math

    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    FS, N, HOP, L, ALPHA, SIG, TRIR = 16000.0, 512, 256, 8, 0.1, 16000, 0.5
    rng = np.random.default_rng(2022 + rank)
    gen = torch.Generator(device=dev).manual_seed(2022 + rank)
    ds = [round(0.05 + 0.01 * i, 2) for i in range(11)]
    fcc = {k: binding.Plan(2, FS, N, 2, tau_max=L, K=k, device=local) for k in range(1, 9)}
    gcc = {r: binding.Plan(2, FS, N, r, tau_max=L, device=local) for r in (1, 2, 4)}
    names = [f"GCC r={r}" for r in (1, 2, 4)] + [f"FCC K={k}" for k in range(1, 9)]
    err = {nm: [[] for _ in ds] for nm in names}

    def unit(v):
        return v / np.linalg.norm(v)

    def parabola(y, i):
        """Three-point refinement of the peak at index i (none at the ends or
        when the points are not concave; offset clamped to +-1/2)."""
        if i <= 0 or i >= len(y) - 1:
            return 0.0
        den = y[i - 1] - 2 * y[i] + y[i + 1]
        return float(np.clip(0.5 * (y[i - 1] - y[i + 1]) / den, -0.5, 0.5)) if den < 0 else 0.0

    t0 = time.perf_counter()
    launches = 0
    for di, d in enumerate(ds):
        for _ in range(args.rooms):
            room = np.array([rng.uniform(5, 15), rng.uniform(5, 15), rng.uniform(3, 4)])
            beta = math.sqrt(1.0 - rng.uniform(0.2, 0.8))
            c = rng.uniform(335.0, 350.0)
            while True:
                center = rng.uniform(0.5, room - 0.5)
                axis = unit(rng.standard_normal(3))
                dd = d + rng.uniform(-0.001, 0.001)
                mics = np.stack([center + 0.5 * dd * axis, center - 0.5 * dd * axis])
                src = center + rng.uniform(1.0, 5.0) * unit(rng.standard_normal(3))
                if np.all(src > 0.3) and np.all(src < room - 0.3):
                    break
            h = synth.image_source_rir(room, src, mics, beta, FS, c, TRIR, device=dev)  # [2, n]
            nr = h.shape[1]
            noise = torch.randn(nr + SIG, generator=gen, device=dev)
            nf = 1 << int(math.ceil(math.log2(2 * nr + SIG)))
            x = torch.fft.irfft(torch.fft.rfft(noise, nf)[None] * torch.fft.rfft(h, nf), nf)[:, nr:nr + SIG]
            pcm = (x / x.abs().max()).T.contiguous()
            X = fcc[1].stft(pcm, HOP)
            tau_true = (np.linalg.norm(src - mics[0]) - np.linalg.norm(src - mics[1])) * FS / c
            th_true = math.degrees(math.acos(max(-1.0, min(1.0, tau_true * c / (dd * FS)))))
            for k, plan in fcc.items():
                o = plan.tdoa_smoothed(X, ALPHA)
                tau = o["tau_hat"][:, 0].double().cpu().numpy()
                th = np.degrees(np.arccos(np.clip(tau * c / (dd * FS), -1.0, 1.0)))
                err[f"FCC K={k}"][di].append(np.abs(th - th_true))
            # GCC on the smoothed cross-spectrum R: spectra (R, 1) give R_hat through the
            # baseline's own phase transform
            R = torch.zeros(X.shape[2], dtype=torch.complex64, device=dev)
            Y = torch.ones((X.shape[0], 2, X.shape[2]), dtype=torch.complex64, device=dev)
            for t in range(X.shape[0]):
                R = (1 - ALPHA) * R + ALPHA * X[t, 0] * X[t, 1].conj()
                Y[t, 0] = R
            for r, plan in gcc.items():
                g = plan.gcc_tdoa(Y, corr=True)
                yc = g["corr"][:, 0].double().cpu().numpy()
                idx = g["lag_idx"][:, 0].cpu().numpy()
                tau = np.array([(i - L * r + parabola(yc[t], i)) / r for t, i in enumerate(idx)])
                th = np.degrees(np.arccos(np.clip(tau * c / (dd * FS), -1.0, 1.0)))
                err[f"GCC r={r}"][di].append(np.abs(th - th_true))
            launches += 1 + 3 * len(fcc) + 3 * len(gcc)
    for p in list(fcc.values()) + list(gcc.values()):
        p.sync()
        p.close()
    mae = {nm: [float(np.concatenate(e).mean()) for e in err[nm]] for nm in names}
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_table1.json")))
    res = None
    if rank == 0:
        res = {"metric": "TDoA mean absolute error (degrees), synthetic Table 1 sweep", "value":
               float(np.mean(mae["FCC K=8"])), "unit": "degrees (FCC K=8, mean over d)", "n_gpus": world,
               "steps": 1, "warmup": 0, "ms_per_step": 1000 * (time.perf_counter() - t0),
               "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (image-source rooms standing in for BIRD)",
               "config": {"workload": "Table 1 sweep: 2 mics, d = 0.05..0.15 m, N 512, hop 256, alpha 0.1, "
                                      "tau_max 8, FCC grid step 1/2, GCC r = 1, 2, 4",
                          "rooms_per_d": args.rooms, "frames_per_room": int(X.shape[0]), "rir_s": TRIR},
               "d_m": ds, "mae_deg": mae, "paper_mae_deg": gold["mae_deg"],
               "gpu_launches": launches}
    return res


def run_smoothed(args, rank, world, local):
    """Eq. 1 with alpha < 1 on a single-array workload: chunk sums, carry scan and
    the FCC pass per step, the stream state carried from step to step."""
    import numpy as np
    import torch

    from paper_2204_13622_gb300 import binding, workloads
    w = {"circle8": workloads.CIRCLE8, "grid16": workloads.GRID16, "square4": workloads.SQUARE4}[args.workload]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    distributed = dist_init(world, "nccl")
    T, P = (args.frames or w.T), w.P
    t0, t1 = rank_frames(T, rank, world)  # this rank's slice of the job's frames
    X = w.spectra(T=t1 - t0, device=dev, seed=rank_seed(rank))
    plan = binding.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, device=local, form=args.form)
    state = torch.zeros((P, w.B), dtype=torch.complex64, device=dev)
    work = torch.empty(max(plan.smooth_workspace(T), 8), dtype=torch.uint8, device=dev)
    out = plan.tdoa_smoothed(X, args.alpha, state=state, work=work)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.tdoa_smoothed(X, args.alpha, state=state, work=work, out=out)
    plan.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(distributed)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            plan.tdoa_smoothed(X, args.alpha, state=state, work=work, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier(distributed)
    plan.sync()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = sum(per) / args.steps
    ms_max = max_over_ranks(ms, distributed, dev)
    bytes_alg = 2 * T * (w.M * w.B * 8) + T * P * 12
    peak, psrc = _peak_hbm()
    res = None
    if rank == 0:
        # accuracy: the first 256 frames from a zero state against the FP64 recursion
        from oracle import oracle as O
        n = min(256, T)
        st0 = torch.zeros_like(state)
        o2 = plan.tdoa_smoothed(X[:n].contiguous(), args.alpha, state=st0)
        plan.sync()
        basis = O.Basis(w.N, w.L, w.lag_den, K=plan.K) if args.form == "folded" else O.BasisB(w.N, w.L, w.lag_den)
        t1 = time.perf_counter()
        idx, pk_, _, y, _ = O.tdoa_smoothed(X[:n].cpu().numpy(), basis.WK, basis.taus, basis.delta, args.alpha,
                                           want_y=True)
        t_or = time.perf_counter() - t1
        gi = o2["lag_idx"].cpu().numpy()
        res = {"metric": METRIC, "value": whole_job_rate(T * P, world, ms_max / 1000.0), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": f"{w.name}, Eq. 1 smoothing alpha={args.alpha}"
                                      + (", split form" if args.form == "reim" else ""), "frames": T, "pairs": P,
                          "state": "carried from step to step",
                          "l2": "inputs larger than L2; no flush"},
               "roofline": dict(alu_roofline(T * P * smooth_ops_per_pair_frame(w.M, w.N, plan.K_even, plan.K_odd, plan.I),
                                             ms, "chunk_sums_kernel + carry_kernel + fcc_smooth_kernel (one step)"),
                                traffic=None,
                                hbm={"achieved": bytes_alg / (ms / 1000.0) / 1e9, "peak": peak, "unit": "GB/s",
                                     "frac": bytes_alg / (ms / 1000.0) / 1e9 / peak, "bytes_per_step": bytes_alg,
                                     "peak_source": psrc,
                                     "note": "the spectra read twice (chunk sums, main pass) plus the outputs"}),
               "accuracy_vs_oracle": {"pair_frames": int(gi.size), "argmax_agreement": float((gi == idx).mean())},
               "cpu_baseline": {"value": n * P / t_or, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                                "sample": f"first {n} frames, FP64 recursion (pairs in parallel)"},
               "gpu_launches": 3 * args.steps, "step_ms": [round(x, 3) for x in per], "clocks": clk.summary()}
    plan.close()
    return res


def run_learned(args, rank, world, local):
    """Learned head: train on FCC coefficients of synthetic pair-frames with the
    library's kernels, report held-out TDoA RMSE against FCC + parabola and the
    head's training / inference throughput."""
    import torch

    from paper_2204_13622_gb300 import learned
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    plan = learned.pair_plan(device=local)
    t0 = time.perf_counter()
    tr = learned.make_dataset(plan, args.train, seed=101, tau_max=4.66, device=dev)
    va = learned.make_dataset(plan, 1 << 18, seed=303, tau_max=4.66, device=dev)
    te = learned.make_dataset(plan, args.heldout, seed=202, tau_max=4.66, device=dev)
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    mlp = learned.new_head(2 * plan.K, learned.feature_scale(tr["features"]), seed=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hist = learned.train(mlp, tr, epochs=args.epochs, batch=4096)
    e1.record()
    torch.cuda.synchronize(dev)
    train_s = e0.elapsed_time(e1) / 1000.0
    th = learned.pick_threshold(mlp, va)
    r = learned.evaluate(mlp, te, th)
    # inference throughput (gated forward over the held-out set)
    outb = {k: torch.empty(te["t"].numel(), device=dev) for k in ("tau", "conf", "raw")}
    for _ in range(3):
        mlp.infer(te["features"], te["tau_fcc"], th, out=outb)
    e0.record()
    for _ in range(args.steps):
        mlp.infer(te["features"], te["tau_fcc"], th, out=outb)
    e1.record()
    torch.cuda.synchronize(dev)
    inf_ms = e0.elapsed_time(e1) / args.steps
    # FCC then the head on the 8-mic circle workload (its grid is the pair grid
    # the head was trained on): pair-frames/s through fcc_tdoa_learned
    from paper_2204_13622_gb300 import binding, workloads
    w = workloads.CIRCLE8
    frames = args.frames or w.T
    Xc = w.spectra(T=frames, device=dev, seed=2)
    plan8 = binding.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L, device=local)
    if plan8.K != plan.K:
        raise RuntimeError("the circle's grid gives a different K than the pair grid")
    lo = plan8.tdoa_learned(Xc, mlp, th)
    for _ in range(3):
        plan8.tdoa_learned(Xc, mlp, th, out=lo)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(args.steps):
        plan8.tdoa_learned(Xc, mlp, th, out=lo)
    e1.record()
    torch.cuda.synchronize(dev)
    plan8.sync()
    mlp.sync()
    c8_ms = e0.elapsed_time(e1) / args.steps

    # the chain's parts timed alone: FCC without and with the coefficient output,
    # then the head on those coefficients.  The difference between the first two
    # plus the head's reading of the coefficients is what the coefficients' trip
    # through HBM costs.
    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    fo = plan8.tdoa(Xc)
    fcc_ms = timed(lambda: plan8.tdoa(Xc, out=fo))
    fo["coeffs"] = lo["coeffs"]
    fcc_coef_ms = timed(lambda: plan8.tdoa(Xc, out=fo))
    feat, tfcc = lo["coeffs"].view(-1, 2 * plan8.K), lo["tau_fcc"].view(-1)
    ho = {k: torch.empty(tfcc.numel(), device=dev) for k in ("tau", "conf", "raw")}
    head_ms = timed(lambda: mlp.infer(feat, tfcc, th, out=ho))
    plan8.sync()
    mlp.sync()
    coef_bytes = lo["coeffs"].numel() * 4
    c8 = {"workload": w.name if frames == w.T else f"{w.name} truncated to {frames} frames",
          "ms_per_step": c8_ms, "pair_frames_per_s": frames * w.P / (c8_ms / 1000.0),
          "head_share_of_pair_frames": float((lo["conf"] >= th).float().mean()),
          "kernels": "fcc_fp32_kernel (with coefficients) + mlp_infer_tc_kernel",
          "parts_ms": {"fcc_tdoa": fcc_ms, "fcc_tdoa_with_coefficients": fcc_coef_ms, "head_alone": head_ms},
          "coefficient_bytes": coef_bytes,
          "coefficient_round_trip_ms_at_measured_hbm": 2 * coef_bytes / (_peak_hbm()[0] * 1e6),
          "ratio_to_fcc_tdoa": c8_ms / fcc_ms}
    del Xc, lo, fo, ho
    plan8.close()
    res = {"metric": "learned-head TDoA RMSE (samples) vs FCC + parabolic refinement", "unit": "samples",
           "value": r["rmse_mlp_gated"], "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
           "warmup": 3, "dtype": "bf16 weights, f32 accumulate", "data": "synthetic", "vs_baseline": None,
           "config": {"workload": "learned: 2 mics, N=512, grid [-5, 5] step 1/4 (I=41), K=%d, tau_max 4.66, "
                                  "SNR U[-5, 30] dB" % plan.K, "train_pair_frames": args.train,
                      "heldout_pair_frames": args.heldout, "epochs": args.epochs, "batch": 4096},
           "rmse": r, "threshold": th, "loss_per_epoch": [round(x, 5) for x in hist],
           "train_samples_per_s": args.epochs * (args.train // 4096) * 4096 / train_s,
           "infer_pair_frames_per_s": te["t"].numel() / (inf_ms / 1000.0), "data_s": round(t_data, 1),
           "fcc_then_head": c8}
    mlp.close()
    plan.close()
    return res


def run_extras(args, local):
    """The default line's other workloads, each at its full size: the 16-mic
    grid in FP32 / BF16 / FP16 ("precision"), 4096 mixed arrays in one step
    ("batched"), the learned head ("learned") and the headline workload from
    int16 PCM through the STFT front-end, whose e2e leg moves 8x fewer bytes
    over the host link than spectra ("pcm").  Each leg frees its device memory
    before the next one starts."""
    import copy

    import torch
    steps = max(3, min(args.steps, 5))
    extras = {}
    t0 = time.perf_counter()
    extras["precision"] = run_precision(args, local, steps)
    extras["precision"]["wall_s"] = round(time.perf_counter() - t0, 1)
    torch.cuda.empty_cache()
    a = copy.copy(args)
    a.steps, a.warmup = steps, 3
    t0 = time.perf_counter()
    extras["batched"] = run_batched(a, 0, 1, local)
    extras["batched"]["wall_s"] = round(time.perf_counter() - t0, 1)
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    extras["learned"] = run_learned(a, 0, 1, local)
    extras["learned"]["wall_s"] = round(time.perf_counter() - t0, 1)
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    extras["pcm"] = run_pcm(a, 0, 1, local)
    extras["pcm"]["wall_s"] = round(time.perf_counter() - t0, 1)
    torch.cuda.empty_cache()
    return extras


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fcc", choices=["fcc", "reference"])
    ap.add_argument("--frames", type=int, default=0, help="override the frame count (profiling)")
    ap.add_argument("--only", default="all", choices=["all", "fcc"], help="fcc: skip GCC, e2e, CPU legs")
    ap.add_argument("--workload", default="circle8",
                    choices=["circle8", "grid16", "square4", "batched", "learned", "doa", "pcm", "table1"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--engine", default="auto", choices=["auto", "cuda_cores", "tensor_tmem", "tensor_smem"],
                    help="the kernel fcc_tdoa runs (fcc_plan_set_engine)")
    ap.add_argument("--alpha", type=float, default=1.0,
                    help="Eq. 1 smoothing factor; < 1 times the smoothed path (FCC leg only)")
    ap.add_argument("--arrays", type=int, default=4096, help="batched: number of arrays")
    ap.add_argument("--dirs", type=int, default=1024, help="doa: candidate directions (hemisphere)")
    ap.add_argument("--rooms", type=int, default=24, help="table1: simulated rooms per microphone spacing")
    ap.add_argument("--form", default="folded", choices=["folded", "reim"],
                    help="basis split: the paper's folded form, or cosine/sine bases on Re/Im")
    ap.add_argument("--batch-single-launch", action="store_true",
                    help="batched: one persistent launch for the whole batch instead of one per kernel class")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="batched: keep the heuristic tile shapes (default: autotuned)")
    ap.add_argument("--train", type=int, default=10_000_000, help="learned: training pair-frames")
    ap.add_argument("--heldout", type=int, default=1_000_000, help="learned: held-out pair-frames")
    ap.add_argument("--epochs", type=int, default=20, help="learned: training epochs")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="default line: skip the 16-mic precision, batched and learned-head legs")
    args = ap.parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        import __graft_entry__ as g
        g.build() if rank == 0 and world == 1 else None
        if args.alpha < 1.0:
            res = run_smoothed(args, rank, world, local)
        elif args.form == "reim":
            res = run_split_form(args, rank, world, local)
        elif args.workload == "batched":
            res = run_batched(args, rank, world, local)
        elif args.workload == "learned":
            res = run_learned(args, rank, world, local) if rank == 0 else None
        elif args.workload == "doa":
            res = run_doa(args, rank, world, local)
        elif args.workload == "pcm":
            res = run_pcm(args, rank, world, local)
        elif args.workload == "table1":
            res = run_table1(args, rank, world, local) if rank == 0 else None
        else:
            res = run_fcc(args, rank, world, local)
            if res is not None and args.extras and world == 1 and args.workload == "circle8" \
                    and args.prec == "fp32" and args.only == "all" and not args.frames:
                res.update(run_extras(args, local))
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
