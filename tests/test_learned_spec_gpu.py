"""The learned corrector's parameter image (BF16 load / save) and the
specification-driven training entry point (pairs generated on the device
from fine plain runs, then trained on), through the C ABI."""
import numpy as np
import pytest

from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

NX, NY, NZ = 128, 32, 32
H_C = 1.0 / 128


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def ctx():
    return ls.LevelSet(NX, NY, NZ, H_C, ls.LS_FP32)


def test_bf16_save_rounds_to_nearest_even_and_load_widens():
    a = ctx()
    a.learned_init(seed=3)
    p = a.learned_params()
    b = a.learned_save()
    u = p.view(np.uint32).astype(np.uint64)
    assert np.array_equal(b, ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16))
    c = ctx()
    c.learned_load(b)
    assert np.array_equal(c.learned_params().view(np.uint32), b.astype(np.uint32) << 16)
    assert np.array_equal(c.learned_save(), b)        # a BF16 image survives the round trip
    with pytest.raises(ls.LSError) as e:
        c.learned_load(b[:-1])
    assert e.value.status == ls.LS_EINVAL


@pytest.mark.parametrize("spec", ["colour=red", "dt=abc", "dt=-1", "source=elsewhere", "problems=0",
                                  "halfwidth", "", None])
def test_spec_errors(spec):
    a = ctx()
    a.learned_init(seed=1)
    with pytest.raises(ls.LSError) as e:
        a.learned_train_spec(spec, 1, 1e-3)              # stored pairs need dt; none stored either
    assert e.value.status == ls.LS_EINVAL


def test_training_needs_parameters_first():
    a = ctx()
    with pytest.raises(ls.LSError) as e:
        a.learned_train_spec("source=fine,problems=1,pairs=1", 1, 1e-3)
    assert e.value.status in (ls.LS_ESTATE, ls.LS_EINVAL)


def test_generated_pairs_are_chained_deterministic_and_train():
    spec = "source=fine, problems=2; pairs=6, gen_seed=5, seed=1"
    a = ctx()
    a.learned_init(seed=1)
    loss = a.learned_train_spec(spec, 400, 1e-3)
    assert np.isfinite(loss)
    assert a.learned_num_pairs() == 12
    b = ctx()
    b.learned_init(seed=1)
    b.learned_train_spec(spec, 0, 1e-3)                  # generation only
    assert b.learned_num_pairs() == 12
    for i in (0, 5, 6, 11):
        for x, y in zip(a.learned_get_pair(i), b.learned_get_pair(i)):
            assert np.array_equal(x.view(np.int32), y.view(np.int32))
    for prob in (0, 1):
        pairs = [a.learned_get_pair(6 * prob + j) for j in range(6)]
        for j in range(5):
            assert np.array_equal(pairs[j][1], pairs[j + 1][0])   # phi_ref(j) = phi_n(j + 1)
            assert np.array_equal(pairs[j][2], pairs[j + 1][2])   # one speed per problem
        phi0, _, F = pairs[0]
        assert phi0.min() < 0.0 < phi0.max()
        assert np.max(np.abs(F)) <= 1.0 + 1e-6
    # the trained network fits the stored pairs better than a fresh one
    dt = 0.5 * H_C
    trained = np.mean([a.learned_train_spec("dt=%r,seed=%d" % (dt, s), 1, 1e-12) for s in range(8)])
    fresh = np.mean([b.learned_train_spec("dt=%r,seed=%d" % (dt, s), 1, 1e-12) for s in range(8)])
    assert trained < 0.7 * fresh, (trained, fresh)
