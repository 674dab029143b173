"""The synthetic Table 1 sweep (bench.py --workload table1) end to end on a
few rooms: every method and spacing gets an MAE, and the ordering the paper
reports at its extremes holds (FCC with K = 8 far below K = 1; GCC with r = 2
no worse than r = 1 by more than sampling noise)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_table1_sweep_runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "table1", "--rooms", "3"],
                       capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(d["d_m"]) == 11
    for name, v in d["mae_deg"].items():
        assert len(v) == 11 and all(0.0 <= x <= 180.0 for x in v), name
    k1 = sum(d["mae_deg"]["FCC K=1"]) / 11
    k8 = sum(d["mae_deg"]["FCC K=8"]) / 11
    assert k8 < 0.5 * k1
    assert set(d["paper_mae_deg"]) == set(d["mae_deg"])


def _room_spectra(seed=5):
    """One room of the Table 1 sweep's kind: two mics 0.1 m apart in a shoebox
    room, white noise through image-source RIRs (the seeded generator in synth),
    then the oracle's own STFT (N 512, hop 256)."""
    import math

    import numpy as np

    from oracle import oracle as O
    from paper_2204_13622_gb300 import synth
    FS, N, HOP, SIG = 16000.0, 512, 256, 16000
    rng = np.random.default_rng(seed)
    room = np.array([8.0, 6.5, 3.2])
    center = np.array([3.1, 2.4, 1.3])
    axis = np.array([0.6, 0.8, 0.0])
    mics = np.stack([center + 0.05 * axis, center - 0.05 * axis])
    src = center + 2.5 * np.array([0.0, 0.6, 0.8])
    h = synth.image_source_rir(room, src, mics, math.sqrt(1.0 - 0.5), FS, 343.0, 0.5).double().numpy()
    nr = h.shape[1]
    noise = rng.standard_normal(nr + SIG)
    nf = 1 << int(math.ceil(math.log2(2 * nr + SIG)))
    x = np.fft.irfft(np.fft.rfft(noise, nf)[None] * np.fft.rfft(h, nf), nf)[:, nr:nr + SIG]
    pcm = (x / np.abs(x).max()).T.astype(np.float32)
    return O.stft(pcm, N, HOP).astype(np.complex64)


def test_table1_room_matches_oracle():
    """The sweep's two legs on one room, element by element against the oracle's
    Eq. 1 recursion: FCC with K = 8 on the grid step 1/2 (alpha = 0.1), and
    GCC-PHAT (full-rank W, Eq. 2) with r = 1, 2, 4 on the same smoothed
    cross-spectrum; FP32 tolerances (tests/helpers.py)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np

    import __graft_entry__ as g
    g.build()
    from helpers import check_argmax, check_corr
    from oracle import oracle as O
    from paper_2204_13622_gb300 import binding as B
    FS, N, L, ALPHA = 16000.0, 512, 8, 0.1
    X = _room_spectra()
    Xd = torch.from_numpy(X).cuda()
    # FCC, K = 8, grid step 1/2, smoothed
    plan = B.Plan(2, FS, N, 2, tau_max=L, K=8)
    out = plan.tdoa_smoothed(Xd, ALPHA, corr=True)
    plan.sync()
    basis = O.Basis(N, L, 2, K=8)
    _, _, tau, y, _ = O.tdoa_smoothed(X, basis.WK, basis.taus, basis.delta, ALPHA, want_y=True)
    check_corr(out["corr"].cpu().numpy(), y)
    gi = out["lag_idx"].cpu().numpy()
    check_argmax(gi, y)
    same = gi == np.argmax(y, -1)
    assert np.all(np.abs(out["tau_hat"].cpu().numpy() - tau)[same] <= 2e-3)
    plan.close()
    # GCC-PHAT on the smoothed cross-spectrum R (spectra (R, 1) give R_hat through the
    # baseline's own phase transform), R by the recursion in FP64
    R = np.zeros(X.shape[2], np.complex128)
    Y = np.ones((X.shape[0], 2, X.shape[2]), np.complex64)
    for t in range(X.shape[0]):
        R = (1 - ALPHA) * R + ALPHA * X[t, 0].astype(np.complex128) * np.conj(X[t, 1].astype(np.complex128))
        Y[t, 0] = R
    for r in (1, 2, 4):
        gp = B.Plan(2, FS, N, r, tau_max=L)
        go = gp.gcc_tdoa(torch.from_numpy(Y).cuda(), corr=True)
        gp.sync()
        full = O.Basis(N, L, r)
        _, _, _, yg, _ = O.tdoa_smoothed(X, full.W, full.taus, full.delta, ALPHA, want_y=True)
        check_corr(go["corr"].cpu().numpy(), yg)
        check_argmax(go["lag_idx"].cpu().numpy(), yg)
        gp.close()
