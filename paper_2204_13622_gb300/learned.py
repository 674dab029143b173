"""Data set, training loop and evaluation of the learned TDoA head.

Host orchestration only: spectra come from :mod:`synth`, coefficients and the
plain FCC estimate from the library's ``fcc_tdoa`` (coefficient output on),
gradients, Adam steps and gated inference from the library's MLP kernels
(include/fcc_mlp.h).  The loop itself (batch order, learning-rate schedule,
held-out evaluation) is plain Python/torch bookkeeping.

The head is an extension of the paper's method (it stops at the argmax and a
sub-sample refinement, Sec. 3): it maps the 2K projection coefficients of a
pair-frame to a sub-sample TDoA and a confidence, trained on (coefficients,
true delay) pairs that FCC produces from synthetic fractional-delay sources.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding, synth

HIDDEN = 128


def pair_plan(N: int = 512, fs: float = 16000.0, tau_max: float = 4.66, lag_den: int = 4,
              energy: float = 0.999, device: int | None = None):
    """Two-microphone FCC plan whose lag grid covers [-tau_max, tau_max]."""
    return binding.Plan(2, fs, N, lag_den, tau_max=tau_max, energy=energy, device=device)


def make_dataset(plan, n: int, seed: int, tau_max: float, snr_db=(-5.0, 30.0), chunk: int = 1 << 20,
                 device="cuda"):
    """n pair-frames: dict of device tensors features [n, 2K] (FCC coefficients),
    t [n] (true TDoA), tau_fcc [n] (FCC argmax + parabola) and snr [n]."""
    import torch

    K2 = 2 * plan.K
    feat = torch.empty((n, K2), dtype=torch.float32, device=device)
    t = torch.empty(n, dtype=torch.float32, device=device)
    tau_fcc = torch.empty(n, dtype=torch.float32, device=device)
    snr = torch.empty(n, dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        X, tt, sn = synth.pair_delay_spectra(m, plan.N, tau_max, seed, device=device, snr_db=snr_db, start=s)
        out = plan.tdoa(X, tau_hat=True, coeffs=True)
        feat[s:s + m] = out["coeffs"].view(m, K2)
        tau_fcc[s:s + m] = out["tau_hat"].view(m)
        t[s:s + m] = torch.from_numpy(tt).to(device=device, dtype=torch.float32)
        snr[s:s + m] = torch.from_numpy(sn).to(device=device, dtype=torch.float32)
        del X, out
    plan.sync()
    return {"features": feat, "t": t, "tau_fcc": tau_fcc, "snr": snr}


def feature_scale(features) -> np.ndarray:
    """Per-coefficient input scale 1 / RMS over the training set."""
    rms = features.double().pow(2).mean(0).sqrt().cpu().numpy()
    return (1.0 / np.maximum(rms, 1e-12)).astype(np.float32)


def new_head(n_in: int, scale, seed: int = 0, conf_weight: float = 0.1, device: int | None = None):
    return binding.MLP(n_in, synth.mlp_init_params(n_in, HIDDEN, seed), in_scale=scale,
                       conf_weight=conf_weight, device=device)


def train(mlp, data, epochs: int, batch: int = 4096, lr_max: float = 1e-3, lr_min: float = 1e-5,
          seed: int = 0, log_every: int = 0):
    """Adam with a cosine learning-rate schedule over `epochs` passes; batches are
    contiguous slices taken in a seeded random order.  Returns the mean loss of
    each epoch."""
    import torch

    n = data["t"].numel()
    nb = n // batch
    if nb < 1:
        raise ValueError("fewer samples than one batch")
    total = epochs * nb
    rng = np.random.default_rng(seed)
    loss = torch.zeros(nb, dtype=torch.float32, device=data["t"].device)
    hist = []
    step = 0
    for ep in range(epochs):
        order = rng.permutation(nb)
        for k, b in enumerate(order):
            lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * step / total))
            sl = slice(int(b) * batch, (int(b) + 1) * batch)
            mlp.train_step(data["features"][sl], data["t"][sl], data["tau_fcc"][sl], lr, loss=loss[k:k + 1])
            step += 1
        hist.append(float(loss.mean()))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.5f}", flush=True)
    return hist


def rmse(a, b) -> float:
    return float((a.double() - b.double()).pow(2).mean().sqrt())


def evaluate(mlp, data, threshold: float = 0.5):
    """TDoA RMSE (samples) on a data set: plain FCC + parabola, the head's raw
    output, and the gated head (FCC where the confidence is below threshold)."""
    out = mlp.infer(data["features"], data["tau_fcc"], threshold)
    t = data["t"]
    return {"rmse_fcc": rmse(data["tau_fcc"], t), "rmse_mlp_raw": rmse(out["raw"], t),
            "rmse_mlp_gated": rmse(out["tau"], t), "frac_mlp": float((out["conf"] >= threshold).float().mean()),
            "n": int(t.numel())}


THRESHOLDS = (0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4, 0.45, 0.5, 0.6, 0.7)


def pick_threshold(mlp, data, grid=THRESHOLDS) -> float:
    """Confidence threshold of the gate with the lowest RMSE on `data` (a
    validation set, not the held-out one)."""
    import torch

    out = mlp.infer(data["features"], data["tau_fcc"], 0.5)
    t, raw, fcc, conf = data["t"], out["raw"], data["tau_fcc"], out["conf"]
    best = min(grid, key=lambda th: rmse(torch.where(conf >= th, raw, fcc), t))
    return float(best)


# ---------------------------------------------------------------------------
# checkpoint / resume: a flat little-endian file
#   magic "FCCMLP01", header length (u32), JSON header (n_in, hidden, step,
#   threshold, conf_weight, basis_sha256 of the plan the head was trained on),
#   then float32 in_scale[n_in], params[n], adam_m[n], adam_v[n]
# ---------------------------------------------------------------------------
MAGIC = b"FCCMLP01"


def basis_hash(plan) -> str:
    """SHA-256 of the plan's FP64 bases and lag grid: a head is only valid for the
    coefficients of the bases it was trained on."""
    import hashlib
    h = hashlib.sha256()
    for a in plan.bases() + (plan.taus(),):
        h.update(np.ascontiguousarray(a, np.float64).tobytes())
    return h.hexdigest()


def save(path: str, mlp, plan, scale, threshold: float, conf_weight: float = 0.1) -> None:
    import json
    import struct
    p, m, v, step = mlp.get_state()
    scale = np.ascontiguousarray(scale, np.float32).reshape(mlp.n_in)
    hdr = json.dumps({"n_in": mlp.n_in, "hidden": HIDDEN, "n_params": int(p.size), "step": int(step),
                      "threshold": float(threshold), "conf_weight": float(conf_weight),
                      "basis_sha256": basis_hash(plan)}).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(hdr)))
        f.write(hdr)
        for a in (scale, p, m, v):
            f.write(np.ascontiguousarray(a, "<f4").tobytes())


def load(path: str, plan, device: int | None = None):
    """Returns (mlp, threshold).  Raises if the file is not a head checkpoint or
    was trained on other bases than `plan`'s."""
    import json
    import struct
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a learned-head checkpoint")
        (n,) = struct.unpack("<I", f.read(4))
        hdr = json.loads(f.read(n).decode())
        if hdr["basis_sha256"] != basis_hash(plan):
            raise ValueError(f"{path}: trained on other bases than this plan's")
        if hdr["n_in"] != 2 * plan.K or hdr["hidden"] != HIDDEN:
            raise ValueError(f"{path}: shape does not match the plan")
        k, npar = hdr["n_in"], hdr["n_params"]
        body = np.frombuffer(f.read(4 * (k + 3 * npar)), "<f4")
    if body.size != k + 3 * npar:
        raise ValueError(f"{path}: truncated")
    scale, p, m, v = body[:k], body[k:k + npar], body[k + npar:k + 2 * npar], body[k + 2 * npar:]
    mlp = binding.MLP(k, p, in_scale=scale, conf_weight=hdr["conf_weight"], device=device)
    mlp.set_state(p, m, v, step=hdr["step"])
    return mlp, hdr["threshold"]
