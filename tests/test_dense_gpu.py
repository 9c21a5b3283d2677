"""Full-domain mode's column-streaming kernel (tile columns walked along z,
z halos from the neighbouring stages): the same bits as the active-list
kernel over all tiles, and within the FP32 bar of the oracle."""
import numpy as np
import pytest

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def run(shape, h, phi, F=None, Fc=None, dense=True, steps=(3, 4), bc=None, ppt=4):
    nz, ny, nx = shape
    g = ls.LevelSet(nx, ny, nz, h, ls.LS_FP32)
    g.set_phi(phi.astype(np.float32))
    if F is not None:
        g.set_speed(F.astype(np.float32))
    else:
        g.set_speed_const(Fc)
    if bc is not None:
        g.set_bc(bc)
    g.set_full_domain(True)
    g.set_dense_kernel(dense)
    g.set_step_config(3, 100, ppt)
    outs = []
    for n in steps:
        g.step(n, 0.45, ls.LS_DT_CFL, 0)
        outs.append(g.get_phi())
    return outs


@pytest.mark.parametrize("ppt", [4, 8])
@pytest.mark.parametrize("shape", [(40, 24, 56), (8, 16, 8), (64, 64, 64), (24, 8, 16)])
def test_same_bits_as_the_list_kernel(shape, ppt):
    h = 1.0 / 64
    w = inputs.SphereUnion(n=64, count=5)
    phi = inputs.sphere_union_sdf(shape, h, w.centres, w.radii).numpy()
    F = inputs.speed_cos_cos(shape, h).numpy()
    a = run(shape, h, phi, F=F, dense=True, ppt=ppt)
    b = run(shape, h, phi, F=F, dense=False, ppt=ppt)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.int32), y.view(np.int32))


@pytest.mark.parametrize("Fc,bc", [(0.8, None), (-0.6, ls.LS_BC_NEUMANN)])
def test_constant_speed_against_the_oracle(Fc, bc):
    shape, h = (32, 40, 48), 1.0 / 48
    phi = inputs.sphere_union_sdf(shape, h, [(0.5, 0.4, 0.3)], [0.25]).numpy()
    got = run(shape, h, phi, Fc=Fc, steps=(5,), bc=bc)[0]
    o = oracle.Oracle(shape, h, bc="neumann" if bc is not None else "extrapolate")
    o.set_phi(phi.astype(np.float32).astype(np.float64))
    o.set_speed_const(Fc)
    o.set_full_domain(True)
    o.step(5, 0.45, oracle.DT_CFL, 0)
    near = np.abs(o.phi) < 10 * h   # band points: far out one FP32 ulp of |phi| ~ 1 exceeds the bar
    assert np.max(np.abs(got.astype(np.float64) - o.phi)[near]) <= 1e-5 * h * 5
