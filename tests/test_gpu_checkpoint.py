"""Checkpoint / restart (lb_save, lb_load): a run interrupted by a save and
continued in a fresh context from the loaded state gives fields and FP64
diagnostics bitwise equal to the uninterrupted run, for every storage, at odd
and even times (the AA parity and the moment-only buffer follow t) and at
t = 0 (the moment-only first step evaluates the stored equilibrium
coefficients), with the linear forcing controller's state carried over."""
import numpy as np
import pytest

from paper_2505_01126_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbgb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


def make(lbgb, w, storage):
    n = w.phi.shape[0]
    return lbgb.Box(n, n, n, w.tau, w.M, w.W, w.sigma, force=lbgb.Force(kind=3, T_relax=w.T_relax),
                    storage=storage)


@pytest.mark.parametrize("storage", ["f32", "f16", "moments", "f16g"])
@pytest.mark.parametrize("split", [0, 25, 26])
def test_interrupted_run_equals_uninterrupted(lbgb, storage, split):
    w = inputs.bubbly_hit(32, 1, 8.0, seed=5)
    a = make(lbgb, w, storage)
    a.init(w.phi, w.u)
    a.step(50)
    want = a.moments_numpy(), a.diagnostics()
    a.close()
    b = make(lbgb, w, storage)
    b.init(w.phi, w.u)
    b.step(split)
    ck = b.save()
    b.close()
    c = make(lbgb, w, storage)  # never initialised: lb_load makes it so
    c.load(ck)
    assert c.time == split
    c.step(50 - split)
    for x, y in zip(want[0], c.moments_numpy()):
        assert np.array_equal(x, y)
    assert np.array_equal(want[1], c.diagnostics())
    c.close()


def test_rollback_in_the_same_context(lbgb):
    w = inputs.bubbly_hit(32, 1, 8.0, seed=6)
    b = make(lbgb, w, "f32")
    b.init(w.phi, w.u)
    b.step(7)
    ck = b.save()
    b.step(5)
    first = b.moments_numpy()
    b.load(ck)
    b.step(5)
    for x, y in zip(first, b.moments_numpy()):
        assert np.array_equal(x, y)
    b.close()


def test_checkpoint_errors(lbgb):
    w = inputs.bubbly_hit(32, 1, 8.0, seed=7)
    b = make(lbgb, w, "f32")
    with pytest.raises(lbgb.LBError) as e:
        b.save()
    assert e.value.code == lbgb.LB_ESTATE
    b.init(w.phi, w.u)
    ck = b.save()
    other = lbgb.Box(32, 32, 16, w.tau, w.M, w.W, w.sigma)
    with pytest.raises(lbgb.LBError) as e:
        other.load(ck)
    assert e.value.code == lbgb.LB_EINVAL
    f16 = make(lbgb, w, "f16")
    with pytest.raises(lbgb.LBError) as e:
        f16.load(ck)
    assert e.value.code == lbgb.LB_EINVAL
    with pytest.raises(lbgb.LBError) as e:
        b.load(ck[: ck.size // 2])
    assert e.value.code == lbgb.LB_EINVAL
    bad = ck.copy()
    bad[:8] = 0
    with pytest.raises(lbgb.LBError) as e:
        b.load(bad)
    assert e.value.code == lbgb.LB_EINVAL
    for x in (b, other, f16):
        x.close()
