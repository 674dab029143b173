"""GPU parity of the learned head's kernels (include/fcc_mlp.h) against the FP64
oracle (forward, loss gradient, Adam), and the trained head's gain over plain
FCC + parabolic refinement.

Both sides see the same BF16-rounded weights, FP32 biases and FP32 inputs (the
per-feature scale is applied in FP32 on both sides); the oracle then runs in
FP64, the GPU in FP32 with FP32 accumulation.  Tolerances: a forward output is
a chain of three dot products (depths n_in, 128, 128) and two erf evaluations;
its FP32 rounding error is below ~(n_in + 256) * 2^-24 * (sum of |terms|), about
2e-5 of the largest output here, so outputs must agree within 1e-4 of
max |y|.  A gradient entry is a sum over the batch of such products; the same
bound per term summed over n terms gives the 2e-4 of the largest entry of its
parameter block used below.  The confidence target g of each sample is a
comparison that FP32 and FP64 could decide differently only within that error,
so the inputs give every sample a margin of at least 25 % of |y0 - t|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_13622_gb300 import synth  # noqa: E402

H = 128


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


def _blocks(nin):
    """(name, slice) of each parameter block in the packed vector."""
    o, out = 0, []
    for name, size in (("W1", H * nin), ("b1", H), ("W2", H * H), ("b2", H), ("W3", 2 * H), ("b3", 2)):
        out.append((name, slice(o, o + size)))
        o += size
    return out


def _bf16_params(O, p, nin):
    """Oracle view of the kernels' parameters: BF16-rounded weights, FP32 biases."""
    q = p.astype(np.float64)
    for name, sl in _blocks(nin):
        if name.startswith("W"):
            q[sl] = O.round_bf16(p[sl])
    return q


def _inputs(O, n, nin, seed, params):
    """Features, scale, true delays and FCC estimates with a clear margin on the
    confidence target of every sample."""
    rng = np.random.default_rng(seed)
    feat = rng.standard_normal((n, nin)).astype(np.float32) * 3.0
    scale = rng.uniform(0.2, 0.6, nin).astype(np.float32)
    x = (feat * scale).astype(np.float32)  # the FP32 product both sides use
    y0 = O.mlp_forward(x, _bf16_params(O, params, nin), nin, H)[:, 0]
    t = rng.uniform(-4.0, 4.0, n).astype(np.float32)
    err = np.abs(y0 - t.astype(np.float64))
    factor = np.where(rng.random(n) < 0.5, 0.75, 1.25)  # g = 0 or 1, 25 % margin
    tfcc = (t + np.where(rng.random(n) < 0.5, -1.0, 1.0) * err * factor).astype(np.float32)
    return feat, scale, x, t, tfcc


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


@pytest.mark.parametrize("n,nin", [(1000, 16), (10017, 16), (77, 5), (4896, 32)])
def test_gradient_matches_oracle(B, O, n, nin):
    p = synth.mlp_init_params(nin, H, seed=n + nin)
    p[H * nin:H * nin + H] = np.random.default_rng(3).normal(0, 0.1, H)  # nonzero b1
    feat, scale, x, t, tfcc = _inputs(O, n, nin, 11 + n, p)
    mlp = B.MLP(nin, p, in_scale=scale, conf_weight=0.1)
    f_d, t_d, c_d = _dev(feat, t, tfcc)
    g, loss = mlp.gradient(f_d, t_d, c_d)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    loss_o, g_o = O.mlp_loss_grad(x, _bf16_params(O, p, nin), t, tfcc, nin, H, 0.1)
    assert abs(float(loss.item()) - loss_o) <= 1e-5 * abs(loss_o)
    for name, sl in _blocks(nin):
        scale_g = np.max(np.abs(g_o[sl]))
        assert scale_g > 0, name
        err = np.max(np.abs(g[sl] - g_o[sl]))
        assert err <= 2e-4 * scale_g, (name, err, scale_g)
    # fixed-order reduction: bitwise reproducible
    g2, _ = mlp.gradient(f_d, t_d, c_d)
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)
    mlp.close()


@pytest.mark.parametrize("n,nin", [(3001, 16), (100000, 16), (777, 5), (2048, 32)])
def test_forward_and_gate_match_oracle(B, O, n, nin):
    # inference runs on the tensor cores: BF16 weights, activations split into
    # two BF16 terms (about 2^-17 relative), FP32 accumulation
    p = synth.mlp_init_params(nin, H, seed=5 + nin)
    feat, scale, x, t, tfcc = _inputs(O, n, nin, 7, p)
    mlp = B.MLP(nin, p, in_scale=scale)
    f_d, c_d = _dev(feat, tfcc)
    out = mlp.infer(f_d, c_d, threshold=0.5)
    torch.cuda.synchronize()
    y = O.mlp_forward(x, _bf16_params(O, p, nin), nin, H)
    raw, conf, tau = (out[k].cpu().numpy().astype(np.float64) for k in ("raw", "conf", "tau"))
    assert np.max(np.abs(raw - y[:, 0])) <= 1e-4 * np.max(np.abs(y[:, 0]))
    conf_o = 1.0 / (1.0 + np.exp(-y[:, 1]))
    assert np.max(np.abs(conf - conf_o)) <= 2.5e-5 * max(1.0, np.max(np.abs(y[:, 1])))
    # the gate: the head's output where its own confidence clears the threshold
    use = conf >= 0.5
    assert np.array_equal(tau[use], raw[use])
    assert np.array_equal(tau[~use], tfcc[~use].astype(np.float64))
    # no fallback estimate: always the head's output
    out2 = mlp.infer(f_d, None, threshold=0.5)
    assert np.array_equal(out2["tau"].cpu().numpy(), out["raw"].cpu().numpy())
    # threshold 0 / above 1: all head / all fallback
    assert np.array_equal(mlp.infer(f_d, c_d, 0.0)["tau"].cpu().numpy(), out["raw"].cpu().numpy())
    assert np.array_equal(mlp.infer(f_d, c_d, 1.5)["tau"].cpu().numpy(), tfcc)
    mlp.sync()
    mlp.close()


def test_adam_steps_match_oracle_and_refresh_bf16(B, O):
    n, nin, lr = 2048, 16, 1e-3
    p = synth.mlp_init_params(nin, H, seed=9)
    feat, scale, x, t, tfcc = _inputs(O, n, nin, 13, p)
    mlp = B.MLP(nin, p, in_scale=scale)
    f_d, t_d, c_d = _dev(feat, t, tfcc)
    p_o = p.astype(np.float64)
    m_o, v_o = np.zeros_like(p_o), np.zeros_like(p_o)
    for step in (1, 2, 3):
        g, _ = mlp.gradient(f_d, t_d, c_d)
        mlp.train_step(f_d, t_d, c_d, lr)
        torch.cuda.synchronize()
        O.adam(p_o, g.cpu().numpy(), m_o, v_o, step, lr)
        pg, mg, vg, st = mlp.get_state()
        assert st == step
        assert np.max(np.abs(pg - p_o)) <= 1e-6 * lr + 2e-7 * np.max(np.abs(p_o))
        assert np.max(np.abs(mg - m_o)) <= 1e-6 * np.max(np.abs(m_o))
        assert np.max(np.abs(vg - v_o)) <= 1e-5 * np.max(np.abs(v_o))
    # the BF16 copies used by the forward follow the updated masters
    pg = mlp.get_state()[0]
    y = O.mlp_forward(x, _bf16_params(O, pg, nin), nin, H)
    raw = mlp.infer(f_d, None)["raw"].cpu().numpy()
    assert np.max(np.abs(raw - y[:, 0])) <= 1e-4 * np.max(np.abs(y[:, 0]))
    mlp.close()


def test_checkpoint_resume_is_bitwise(B, O):
    n, nin = 4096, 16
    p = synth.mlp_init_params(nin, H, seed=21)
    feat, scale, x, t, tfcc = _inputs(O, n, nin, 23, p)
    f_d, t_d, c_d = _dev(feat, t, tfcc)
    a = B.MLP(nin, p, in_scale=scale)
    for _ in range(3):
        a.train_step(f_d, t_d, c_d, 1e-3)
    state = a.get_state()
    b = B.MLP(nin, synth.mlp_init_params(nin, H, seed=99), in_scale=scale)
    b.set_state(*state[:3], step=state[3])
    a.train_step(f_d, t_d, c_d, 1e-3)
    b.train_step(f_d, t_d, c_d, 1e-3)
    sa, sb = a.get_state(), b.get_state()
    for u, v in zip(sa[:3], sb[:3]):
        assert np.array_equal(u, v)
    assert sa[3] == sb[3] == 4
    a.close()
    b.close()


def test_invalid_arguments(B):
    p = synth.mlp_init_params(16, H, seed=1)
    lib = B.lib()
    import ctypes
    h = ctypes.c_void_p()
    fp = ctypes.POINTER(ctypes.c_float)
    assert lib.fcc_mlp_create(16, 64, None, 0.1, p.ctypes.data_as(fp), 0, ctypes.byref(h)) == 2
    assert lib.fcc_mlp_create(33, 128, None, 0.1, p.ctypes.data_as(fp), 0, ctypes.byref(h)) == 2
    assert lib.fcc_mlp_create(16, 128, None, -1.0, p.ctypes.data_as(fp), 0, ctypes.byref(h)) == 1
    assert lib.fcc_mlp_create(16, 128, None, 0.1, None, 0, ctypes.byref(h)) == 1
    mlp = B.MLP(16, p)
    f = torch.zeros((4, 16), device="cuda")
    v = torch.zeros(4, device="cuda")
    with pytest.raises(B.FccError):
        mlp.train_step(f, v, v, 0.0)
    assert lib.fcc_mlp_gradient(mlp._h, f.data_ptr(), v.data_ptr(), v.data_ptr(), 0, v.data_ptr(), None,
                                None) == 1
    out = mlp.infer(f[:0], None)  # n = 0: no-op
    assert out["tau"].numel() == 0
    mlp.close()


def test_trained_head_beats_plain_fcc(B):
    """Statistical: a head trained on 2^21 synthetic pair-frames (the 8-mic
    circle's lag grid, tau_max 4.66, SNR U[-5, 30] dB), with its gate threshold
    picked on a validation set, has a held-out TDoA RMSE at least 15 % below
    FCC + parabolic refinement."""
    from paper_2204_13622_gb300 import learned
    plan = learned.pair_plan()
    train = learned.make_dataset(plan, 1 << 21, seed=101, tau_max=4.66)
    val = learned.make_dataset(plan, 1 << 17, seed=303, tau_max=4.66)
    held = learned.make_dataset(plan, 1 << 17, seed=202, tau_max=4.66)
    mlp = learned.new_head(2 * plan.K, learned.feature_scale(train["features"]), seed=0)
    hist = learned.train(mlp, train, epochs=10, batch=4096)
    torch.cuda.synchronize()
    assert hist[-1] < hist[0]
    th = learned.pick_threshold(mlp, val)
    r = learned.evaluate(mlp, held, th)
    print(th, r)
    assert r["rmse_mlp_raw"] < r["rmse_fcc"], r
    assert r["rmse_mlp_gated"] < 0.85 * r["rmse_fcc"], r
    mlp.close()
    plan.close()


def test_tdoa_learned_chains_fcc_and_head(B):
    """fcc_tdoa_learned = fcc_tdoa (tau_hat, coefficients) then the gated head on
    every pair-frame's coefficients, bit for bit."""
    from paper_2204_13622_gb300 import workloads
    w = workloads.CIRCLE8
    X = w.spectra(T=300, seed=5).cuda()
    plan = B.Plan(w.M, w.fs, w.N, w.lag_den, tau_max=w.L)
    K2 = 2 * plan.K
    mlp = B.MLP(K2, synth.mlp_init_params(K2, H, seed=3), in_scale=0.5)
    out = plan.tdoa_learned(X, mlp, threshold=0.4)
    ref = plan.tdoa(X, tau_hat=True, coeffs=True)
    plan.sync()
    assert torch.equal(out["lag_idx"], ref["lag_idx"]) and torch.equal(out["peak"], ref["peak"])
    assert torch.equal(out["tau_fcc"], ref["tau_hat"]) and torch.equal(out["coeffs"], ref["coeffs"])
    head = mlp.infer(ref["coeffs"].view(-1, K2), ref["tau_hat"].view(-1), threshold=0.4)
    mlp.sync()
    assert torch.equal(out["tau"].view(-1), head["tau"]) and torch.equal(out["conf"].view(-1), head["conf"])
    bad = B.MLP(K2 + 2, synth.mlp_init_params(K2 + 2, H, seed=3))
    with pytest.raises(B.FccError):
        plan.tdoa_learned(X, bad, threshold=0.4)
    for m in (mlp, bad):
        m.close()
    plan.close()


def test_checkpoint_file_roundtrip_and_basis_binding(B, tmp_path):
    from paper_2204_13622_gb300 import learned
    plan = learned.pair_plan()
    K2 = 2 * plan.K
    scale = np.linspace(0.5, 2.0, K2).astype(np.float32)
    mlp = learned.new_head(K2, scale, seed=4)
    rng = np.random.default_rng(0)
    f_d = torch.from_numpy(rng.standard_normal((4096, K2)).astype(np.float32)).cuda()
    t_d = torch.from_numpy(rng.uniform(-4, 4, 4096).astype(np.float32)).cuda()
    mlp.train_step(f_d, t_d, t_d + 0.1, 1e-3)
    path = str(tmp_path / "head.bin")
    learned.save(path, mlp, plan, scale, threshold=0.35)
    back, th = learned.load(path, plan)
    assert th == 0.35
    for u, v in zip(mlp.get_state(), back.get_state()):
        assert np.array_equal(u, v)
    a = mlp.infer(f_d, t_d, 0.35)
    b = back.infer(f_d, t_d, 0.35)
    assert torch.equal(a["tau"], b["tau"]) and torch.equal(a["conf"], b["conf"])  # same scale, same weights
    other = B.Plan(2, 16000.0, 512, 8, tau_max=4.66)  # another lag grid: other bases
    with pytest.raises(ValueError):
        learned.load(path, other)
    for o in (mlp, back, other, plan):
        o.close()
