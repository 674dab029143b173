"""GPU tests of the batched form (include/fcc_batch.h) and the tile autotuner
(include/fcc_tune.h).

The batched kernel runs the same per-tile pipeline as fcc_tdoa, so every
array's results must equal, bit for bit, fcc_tdoa on a plan with the same
geometry; a sample of arrays is also checked against the FP64 oracle with the
tolerances of tests/helpers.py.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_argmax, check_corr  # noqa: E402,F401

from paper_2204_13622_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def _small_arrays(n, seed):
    # mixed mic counts (odd ones take the plain-load staging path), N, fs,
    # apertures; few frames, including 1 and ragged tile tails
    arrs = synth.batched_arrays(n, seed, mics=(2, 3, 4, 5, 6, 8, 12, 16), frames=(1, 300))
    arrs[0]["T"] = 1
    return arrs


def _plan_kw(a):
    return {k: a[k] for k in ("n_mics", "fs", "N", "lag_den", "mic_xyz")}


def test_batch_equals_single_plans(B):
    arrs = _small_arrays(40, seed=4)
    batch = B.Batch(arrs)
    info = batch.info()
    assert info["n_arrays"] == 40 and info["n_classes"] >= 2
    assert info["n_launches"] == info["n_classes"]  # one persistent launch per class
    assert info["frames"] == sum(a["T"] for a in arrs)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    out = batch.outputs()
    batch.bind(X, out)
    batch.run()
    batch.sync()
    for a, arr in enumerate(arrs):
        plan = B.Plan(**_plan_kw(arr))
        assert plan.geometry() is not None
        ref = plan.tdoa(X[a])
        plan.sync()
        for k in ("lag_idx", "peak", "tau_hat"):
            assert torch.equal(ref[k], out[a][k]), (a, k, arr["n_mics"], arr["N"], arr["T"])
        plan.close()
    # a second run of the same graph gives the same bytes
    first = [{k: v.clone() for k, v in o.items()} for o in out]
    for o in out:
        for v in o.values():
            v.fill_(-7)
    batch.run()
    batch.sync()
    for o, f in zip(out, first):
        for k in o:
            assert torch.equal(o[k], f[k])
    batch.close()


def test_batch_sampled_arrays_match_oracle(B, O):
    arrs = _small_arrays(12, seed=9)
    batch = B.Batch(arrs)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    out = batch.outputs()
    batch.bind(X, out)
    batch.run()
    batch.sync()
    for a in range(0, 12, 3):
        info = batch.arrays[a]
        basis = O.Basis(info["N"], info["L"], info["den"], K=info["K"])
        Xh = X[a][:16].cpu().numpy()
        idx, peak, tau, y = O.tdoa(Xh, basis.WK, basis.taus, basis.delta, want_y=True)
        check_argmax(out[a]["lag_idx"][:16].cpu().numpy(), y)
        got_peak = out[a]["peak"][:16].cpu().numpy().astype(np.float64)
        scale = np.abs(y).max(axis=-1)
        assert np.all(np.abs(got_peak - peak) <= 1e-4 * scale + 1e-30)
    batch.close()


def test_batch_nonfinite_and_errors(B):
    arrs = _small_arrays(6, seed=5)
    batch = B.Batch(arrs)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    out = batch.outputs(tau_hat=False)
    with pytest.raises(B.FccError):
        batch.run()  # not bound yet
    X[3][-1, 0, 5] = float("nan")
    batch.bind(X, out)
    batch.run()
    with pytest.raises(B.FccError) as e:
        batch.sync()
    assert e.value.status == 6  # FCC_ERR_NONFINITE
    X[3][-1, 0, 5] = 1.0
    batch.run()
    batch.sync()
    batch.close()
    bad = dict(arrs[0], T=0)
    with pytest.raises(B.FccError):
        B.Batch([bad])


def test_autotune_cache_and_parity(B, O, tmp_path):
    cache = str(tmp_path / "tune.json")
    from paper_2204_13622_gb300 import workloads
    w = workloads.SQUARE4
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, mic_xyz=w.xyz)
    us = plan.autotune(cache, max_candidates=4)
    assert us > 0
    data = json.load(open(cache))
    assert len(data["entries"]) == 1
    entry = next(iter(data["entries"].values()))
    g = plan.geometry()
    assert (entry["C"], entry["G"], entry["S"]) == (g["C"], g["groups"], g["stages"])
    # a second plan with the same key takes the cached shape without timing
    plan2 = B.Plan(w.M, w.fs, w.N, w.lag_den, mic_xyz=w.xyz)
    us2 = plan2.autotune(cache)
    assert us2 == pytest.approx(us, rel=1e-6)
    assert plan2.geometry() == g
    # the tuned plan still matches the oracle
    X = w.spectra(T=40, seed=3)
    out = plan.tdoa(X.cuda(), corr=True)
    plan.sync()
    info = plan.info
    basis = O.Basis(w.N, info["L"], w.lag_den, K=info["K"])
    idx, peak, tau, y = O.tdoa(X.numpy(), basis.WK, basis.taus, basis.delta, want_y=True)
    check_corr(out["corr"].cpu().numpy(), y)
    check_argmax(out["lag_idx"].cpu().numpy(), y)
    plan.close()
    plan2.close()


def test_batch_autotune_flag(B, tmp_path):
    cache = str(tmp_path / "tune.json")
    arrs = _small_arrays(8, seed=6)
    batch = B.Batch(arrs, autotune=True, tune_cache=cache)
    assert os.path.exists(cache)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    out = batch.outputs()
    batch.bind(X, out)
    batch.run()
    batch.sync()
    batch.close()


def test_batch_rebind_to_new_buffers(B):
    arrs = _small_arrays(10, seed=11)
    batch = B.Batch(arrs)
    X1 = [synth.array_spectra(a, device="cuda") for a in arrs]
    X2 = [synth.array_spectra(dict(a, seed=a["seed"] + 1), device="cuda") for a in arrs]
    o1, o2 = batch.outputs(), batch.outputs()
    batch.bind(X1, o1)
    batch.run()
    batch.sync()
    batch.bind(X2, o2)  # the same graph reads the new parameter table
    batch.run()
    batch.sync()
    for a, arr in enumerate(arrs):
        plan = B.Plan(**_plan_kw(arr))
        r1, r2 = plan.tdoa(X1[a]), plan.tdoa(X2[a])
        plan.sync()
        for k in ("lag_idx", "peak", "tau_hat"):
            assert torch.equal(r1[k], o1[a][k]) and torch.equal(r2[k], o2[a][k]), (a, k)
        plan.close()
    batch.close()


def test_autotune_ignores_a_corrupt_cache(B, tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{ this is not json")
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)
    us = plan.autotune(str(cache), max_candidates=2)
    assert us > 0
    data = json.load(open(cache))  # rewritten as a valid cache
    assert len(data["entries"]) == 1
    plan.close()


def test_single_launch_equals_per_class_launches(B):
    # FCC_BATCH_SINGLE_LAUNCH: every class in one persistent launch (geometries
    # limited to its eight warps, same chunk counts); every array's results equal
    # the per-class launches' bit for bit
    arrs = _small_arrays(24, seed=11)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    one = B.Batch(arrs, single_launch=True)
    many = B.Batch(arrs)
    assert one.info()["n_launches"] == 1
    assert many.info()["n_launches"] == many.info()["n_classes"] >= 2
    o1, o2 = one.outputs(), many.outputs()
    one.bind(X, o1)
    many.bind(X, o2)
    one.run()
    many.run()
    one.sync()
    many.sync()
    for a in range(len(arrs)):
        for k in ("lag_idx", "peak", "tau_hat"):
            assert torch.equal(o1[a][k], o2[a][k]), (a, k)
    one.close()
    many.close()
