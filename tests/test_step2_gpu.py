"""Two upwind steps per pass (temporal blocking): the same bits as one step
per pass, on trajectories that mix two-step and one-step passes (odd
rebuild periods, chunked calls), with speed fields and constant speeds of
both signs, bands touching the domain faces, both face rules, the full
domain, the tube test before each rebuild and graph replay."""
import numpy as np
import pytest

from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def pair(shape, h, phi, F=None, Fc=None, bc=None):
    nz, ny, nx = shape
    out = []
    for spp in (1, 2):
        g = ls.LevelSet(nx, ny, nz, h, ls.LS_FP32)
        g.set_phi(phi.astype(np.float32))
        if F is not None:
            g.set_speed(F.astype(np.float32))
        else:
            g.set_speed_const(Fc)
        if bc is not None:
            g.set_bc(bc)
        g.set_steps_per_pass(spp)
        out.append(g)
    return out


def same(a, b):
    return np.array_equal(a.get_phi().view(np.int32), b.get_phi().view(np.int32))


@pytest.mark.parametrize("rebuild_every", [5, 4, 2, 0])
def test_union_with_field(rebuild_every):
    shape, h = (56, 64, 72), 1.0 / 64
    w = inputs.SphereUnion(n=64, count=6)
    phi = inputs.sphere_union_sdf(shape, h, w.centres, w.radii).numpy()
    F = inputs.speed_sinusoid(shape, h).numpy()
    a, b = pair(shape, h, phi, F=F)
    for g in (a, b):
        g.band_rebuild(6.0)
    for n in (3, 7, 4, 11):
        a.step(n, 0.5, ls.LS_DT_CFL, rebuild_every)
        b.step(n, 0.5, ls.LS_DT_CFL, rebuild_every)
        assert same(a, b)
        assert np.array_equal(a.active_tiles(), b.active_tiles())
    if rebuild_every in (4, 2, 0):
        assert b.profile()["two_step_points"] > 0


@pytest.mark.parametrize("Fc,bc", [(-0.7, None), (0.9, ls.LS_BC_NEUMANN), (0.6, None)])
def test_band_on_the_domain_faces(Fc, bc):
    """A sphere cut by three domain faces (the corner at the origin) and a
    sign-changing-free constant speed: face layers at the domain faces take
    the face rule, neighbours off the grid do not exist."""
    shape, h = (40, 48, 32), 1.0 / 32
    phi = inputs.sphere_union_sdf(shape, h, [(0.05, 0.1, 0.0)], [0.5]).numpy()
    a, b = pair(shape, h, phi, Fc=Fc, bc=bc)
    for g in (a, b):
        g.band_rebuild(5.0)
    for n in (6, 9):
        a.step(n, 0.45, ls.LS_DT_CFL, 4)
        b.step(n, 0.45, ls.LS_DT_CFL, 4)
        assert same(a, b)


def test_sign_changing_field_full_domain_and_graphs():
    shape, h = (48, 48, 48), 1.0 / 48
    w = inputs.PerturbedSphere(n=48)
    phi = w.phi().numpy()
    F = inputs.speed_cos_cos(shape, h).numpy()
    a, b = pair(shape, h, phi, F=F)
    for g in (a, b):
        g.set_full_domain(True)
    a.step(6, 0.4, ls.LS_DT_CFL, 0)
    b.step(6, 0.4, ls.LS_DT_CFL, 0)
    assert same(a, b)
    a2, b2 = pair(shape, h, phi, F=F)
    b2.set_graphs(True)
    for g in (a2, b2):
        g.band_rebuild(6.0)
    for _ in range(3):
        a2.step(8, 0.4, ls.LS_DT_CFL, 4)
        b2.step(8, 0.4, ls.LS_DT_CFL, 4)
    assert same(a2, b2)


def test_autotuner_considers_two_steps_and_errors():
    shape, h = (64, 64, 64), 1.0 / 64
    w = inputs.SphereUnion(n=64, count=5)
    phi = w.phi().numpy()
    a, _ = pair(shape, h, phi, F=w.speed().numpy())
    a.band_rebuild(6.0)
    a.step(2, 0.5, ls.LS_DT_CFL, 5)
    a.autotune(reps=2)
    assert a.steps_per_pass() in (1, 2)
    with pytest.raises(ls.LSError) as e:
        a.set_steps_per_pass(3)
    assert e.value.status == ls.LS_EINVAL
