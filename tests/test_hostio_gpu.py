"""Stream-ordered host input/output: a sequence of problems run with the next
inputs staged and the previous result read back while the current problem
computes gives, for every problem, the same bits as the synchronous calls
(ls_set_phi / ls_set_speed / ls_get_phi) on a fresh context; the calls
report misuse and non-finite inputs."""
import numpy as np
import pytest
import torch

from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

SHAPE, H = (48, 40, 56), 1.0 / 48


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def problem(k):
    w = inputs.SphereUnion(n=48, count=3 + k, seed=900 + k)
    phi = inputs.sphere_union_sdf(SHAPE, H, w.centres, w.radii).float()
    F = (inputs.speed_sinusoid(SHAPE, H) * (1.0 + 0.25 * k)).float()
    return phi.contiguous().pin_memory(), F.contiguous().pin_memory()


def run_sync(phi, F, steps):
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32)
    g.set_phi(phi)
    g.set_speed(F)
    g.band_rebuild(5.0)
    g.step(steps, 0.5, ls.LS_DT_CFL, 5)
    return g.get_phi()


def test_pipelined_sequence_equals_synchronous_calls():
    probs = [problem(k) for k in range(4)]
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32, stream=torch.cuda.current_stream().cuda_stream)
    outs = [torch.empty(SHAPE, dtype=torch.float32).pin_memory() for _ in probs]
    steps = 13
    g.stage_inputs(*probs[0])
    for k in range(len(probs)):
        g.load_staged()
        if k + 1 < len(probs):
            g.stage_inputs(*probs[k + 1])
        g.band_rebuild(5.0)
        g.step(steps, 0.5, ls.LS_DT_CFL, 5)
        g.get_phi_async(outs[k])
    g.wait_host()
    for k, (phi, F) in enumerate(probs):
        ref = run_sync(phi, F, steps)
        assert np.array_equal(outs[k].numpy().view(np.int32), ref.view(np.int32)), k
    assert g.status() == ls.LS_OK


def test_stage_phi_only_keeps_the_speed_field():
    (phi0, F0), (phi1, _) = problem(0), problem(1)
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32)
    g.stage_inputs(phi0, F0)
    g.load_staged()
    g.stage_inputs(phi1)
    g.load_staged()
    g.band_rebuild(5.0)
    g.step(6, 0.5, ls.LS_DT_CFL, 5)
    out = torch.empty(SHAPE, dtype=torch.float32).pin_memory()
    g.get_phi_async(out)
    g.wait_host()
    assert np.array_equal(out.numpy().view(np.int32), run_sync(phi1, F0, 6).view(np.int32))


def test_misuse_and_non_finite_inputs():
    phi, F = problem(0)
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32)
    out = torch.empty(SHAPE, dtype=torch.float32).pin_memory()
    with pytest.raises(ls.LSError) as e:
        g.get_phi_async(out)  # phi not set
    assert e.value.status == ls.LS_ESTATE
    with pytest.raises(ls.LSError) as e:
        g.load_staged()  # nothing staged
    assert e.value.status == ls.LS_ESTATE
    g.stage_inputs(phi, F)
    with pytest.raises(ls.LSError) as e:
        g.stage_inputs(phi, F)  # staged twice without a load
    assert e.value.status == ls.LS_ESTATE
    g.load_staged()
    bad = phi.clone().pin_memory()
    bad[3, 4, 5] = float("nan")
    g.stage_inputs(bad)
    with pytest.raises(ls.LSError) as e:
        g.load_staged()
    assert e.value.status == ls.LS_ENONFINITE
    with pytest.raises(ValueError):
        g.stage_inputs(phi.cuda())  # a device array is not a host buffer
    g.wait_host()
