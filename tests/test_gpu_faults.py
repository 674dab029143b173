"""Failure paths on the GPU without faulting it: a bounded device wait that runs
out (a bulk copy the test hook withholds, with a short wait bound) must come back
as FCC_ERR_TIMEOUT with the context still usable, and a failing allocation
during plan creation as FCC_ERR_OOM."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2204_13622_gb300 import synth  # noqa: E402

TIMEOUT, OOM = 5, 3


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding


@pytest.fixture
def hooks(B):
    yield B
    B.debug_set("wait_cycles", 0)
    B.debug_set("withhold_copy", 0)
    B.debug_set("fail_alloc", 0)


def _spectra(T, M, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((T, M, 257)) + 1j * rng.standard_normal((T, M, 257))
    return torch.from_numpy(X.astype(np.complex64)).cuda()


def test_expired_wait_reports_timeout_and_context_survives(hooks):
    B = hooks
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)
    X = _spectra(5000, 4, 1)
    ref = plan.tdoa(X)
    plan.sync()
    ref = {k: v.clone() for k, v in ref.items()}
    B.debug_set("wait_cycles", 200000)  # about 0.1 ms
    B.debug_set("withhold_copy", 1)
    plan.tdoa(X)
    with pytest.raises(B.FccError) as e:
        plan.sync()
    assert e.value.status == TIMEOUT
    B.debug_set("wait_cycles", 0)
    out = plan.tdoa(X)  # the next launch runs normally on the same context
    plan.sync()
    for k in ref:
        assert torch.equal(out[k], ref[k])
    plan.close()


def test_expired_wait_in_the_batched_form(hooks):
    B = hooks
    arrs = synth.batched_arrays(6, 3, mics=(4, 8), frames=(200, 400))
    batch = B.Batch(arrs)
    X = [synth.array_spectra(a, device="cuda") for a in arrs]
    out = batch.outputs()
    B.debug_set("wait_cycles", 200000)
    B.debug_set("withhold_copy", 1)  # applies to the parameters written at bind
    batch.bind(X, out)
    batch.run()
    with pytest.raises(B.FccError) as e:
        batch.sync()
    assert e.value.status == TIMEOUT
    B.debug_set("wait_cycles", 0)
    batch.bind(X, out)  # fresh parameters without the hook
    batch.run()
    batch.sync()
    batch.close()


def test_allocation_failure_during_plan_creation(hooks):
    B = hooks
    B.debug_set("fail_alloc", 1)
    with pytest.raises(B.FccError) as e:
        B.Plan(4, 16000.0, 512, 4, tau_max=3)
    assert e.value.status == OOM
    plan = B.Plan(4, 16000.0, 512, 4, tau_max=3)  # the hook is spent
    plan.close()


@pytest.mark.parametrize("form,alpha", [("folded", 0.1), ("reim", 0.5), ("reim", 1.0)])
def test_per_pair_kernel_timeout_path(hooks, form, alpha):
    # the per-pair kernel (smoothed path, both forms) and the split-form FP32
    # kernel (alpha = 1) take the same exit: the first copy withheld in CTA 0, a
    # short wait bound, FCC_ERR_TIMEOUT, and the next launch on the same context
    # equal to the reference
    B = hooks
    plan = B.Plan(8, 16000.0, 512, 4, tau_max=5, form=form)
    X = _spectra(3000, 8, 2)
    run = (lambda: plan.tdoa_smoothed(X, alpha)) if alpha < 1.0 else (lambda: plan.tdoa(X))
    ref = run()
    plan.sync()
    ref = {k: v.clone() for k, v in ref.items()}
    B.debug_set("wait_cycles", 200000)  # about 0.1 ms
    B.debug_set("withhold_copy", 1)
    run()
    with pytest.raises(B.FccError) as e:
        plan.sync()
    assert e.value.status == TIMEOUT
    B.debug_set("wait_cycles", 0)
    out = run()
    plan.sync()
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    plan.close()
