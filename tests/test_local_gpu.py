"""GPU parity of the local level-set scheme (section 1.1, Steps 1-3: the
cut-off advance of Eq. 7-8 on T, the reinitialisation of Eq. 12-13 on N of
Eq. 11, the clamp of Eq. 10) through the C ABI, against the FP64 CPU
oracle on the same seeded inputs.

Bars:
* FP64: bit for bit along whole trajectories (the kernels follow the
  oracle's operation order with round-to-nearest intrinsics), dt bitwise,
  active tiles identical at every rebuild;
* FP32: one step from a given state within (1 + K) * 1e-5 * h (1e-5 h per
  pass: the advance and K reinitialisation passes), and along a trajectory
  within (1 + K) * 1e-5 * h * nsteps; every set decision (T, N, the cut-off
  branches) is taken with thresholds that decide as the FP64 comparisons do;
* no N point outside the active tiles (ls_band_breaches == 0 and the
  oracle's own count == 0) on the standard cases, and a positive count on
  both sides when the band is left stale on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

SHAPE = (72, 56, 64)          # (nz, ny, nx): three different edges, 9 x 7 x 8 tiles
H = 1.0 / 64
HW, BETA, K, DTAU = 5.0, 2.5, 4, 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def case(seed=11):
    g = np.random.default_rng(seed)
    nz, ny, nx = SHAPE
    box = (nx * H, ny * H, nz * H)
    k = 5
    centres = [tuple(float(g.uniform(0.3 * b, 0.7 * b)) for b in box) for _ in range(k)]
    radii = [float(g.uniform(0.08, 0.2)) for _ in range(k)]
    phi = inputs.sphere_union_sdf(SHAPE, H, centres, radii).numpy()
    F = inputs.speed_fourier(SHAPE, H, inputs.fourier_modes(g, count=6, kmax=2)).numpy()
    return phi, F


def make(prec, phi, F, Fc=None, full=False, iters=K):
    nz, ny, nx = SHAPE
    dt = np.float32 if prec == ls.LS_FP32 else np.float64
    g = ls.LevelSet(nx, ny, nz, H, prec)
    o = oracle.Oracle(SHAPE, H)
    p = np.ascontiguousarray(phi, dtype=dt)
    g.set_phi(p)
    o.set_phi(p.astype(np.float64))
    if F is not None:
        f = np.ascontiguousarray(F, dtype=dt)
        g.set_speed(f)
        o.set_speed(f.astype(np.float64))
    else:
        g.set_speed_const(Fc)
        o.set_speed_const(Fc)
    g.band_rebuild(HW)
    o.band_rebuild(HW)
    if full:
        g.set_full_domain(True)
        o.set_full_domain(True)
    g.set_scheme(ls.LS_SCHEME_LOCAL, BETA, iters, DTAU)
    o.set_scheme(oracle.SCHEME_LOCAL, BETA, iters if iters >= 0 else int(np.ceil(HW / DTAU)), DTAU)
    return g, o


@pytest.mark.parametrize("iters,mode", [(K, ls.LS_REBUILD_FULL), (0, ls.LS_REBUILD_FULL),
                                        (-1, ls.LS_REBUILD_FULL), (K, ls.LS_REBUILD_INCREMENTAL)])
def test_fp64_trajectory_bitwise(iters, mode):
    phi, F = case()
    g, o = make(ls.LS_FP64, phi, F, iters=iters)
    g.set_rebuild_mode(mode)
    for n in (1, 2, 4, 5):
        dg = g.step(n, 0.45, ls.LS_DT_CFL, 3, want_dt=True)
        do = o.step(n, 0.45, oracle.DT_CFL, 3)
        assert dg == do
        assert np.array_equal(g.active_tiles(), o.active_tiles())
        assert np.array_equal(bits(g.get_phi()), bits(o.phi))
    assert g.band_breaches() == 0 and o.breaches == 0


def test_fp64_full_domain_constant_speed_bitwise():
    phi, _ = case(12)
    g, o = make(ls.LS_FP64, phi, None, Fc=-0.8, full=True)
    for n in (3, 4):
        g.step(n, H / 3, ls.LS_DT_FIXED, 0)
        o.step(n, H / 3, oracle.DT_FIXED, 0)
        assert np.array_equal(bits(g.get_phi()), bits(o.phi))


def test_fp32_one_step_from_a_state():
    """Each of several steps, recomputed by the oracle from the library's own
    FP32 state, within (1 + K) 1e-5 h."""
    phi, F = case(13)
    g, _ = make(ls.LS_FP32, phi, F)
    F64 = F.astype(np.float32).astype(np.float64)
    gamma = HW * H
    for _ in range(4):
        g.step(2, 0.45, ls.LS_DT_CFL, 3)
        before = g.get_phi().astype(np.float64)
        tiles = g.active_tiles()
        dt = g.step(1, 0.45, ls.LS_DT_CFL, 3, want_dt=True)
        after = g.get_phi().astype(np.float64)
        ref, nmask = oracle.local_step(before, H, dt, BETA * H, gamma, K, DTAU * H, F=F64)
        act = np.zeros(9 * 7 * 8, dtype=bool)
        act[tiles] = True
        pts = np.repeat(np.repeat(np.repeat(act.reshape(9, 7, 8), 8, 0), 8, 1), 8, 2)
        assert not np.any(nmask.astype(bool) & ~pts)
        assert np.max(np.abs(after - ref)) <= (1 + K) * 1e-5 * H
        assert np.array_equal(after[~pts], before[~pts])
        # clamped values stay outside T, as in FP64
        assert np.all(np.abs(after[nmask.astype(bool)]) <= np.float32(gamma) * (1 + 2.5e-7))
    assert g.band_breaches() == 0


def test_fp32_trajectory():
    phi, F = case(14)
    g, o = make(ls.LS_FP32, phi, F)
    done = 0
    for n in (2, 3, 5):
        g.step(n, 0.45, ls.LS_DT_CFL, 3)
        o.step(n, 0.45, oracle.DT_CFL, 3)
        done += n
        assert np.array_equal(g.active_tiles(), o.active_tiles())
        assert np.max(np.abs(g.get_phi().astype(np.float64) - o.phi)) <= (1 + K) * 1e-5 * H * done
    assert g.band_breaches() == 0 and o.breaches == 0


@pytest.mark.parametrize("iters,full,Fc", [(K, False, None), (0, False, None), (-1, False, None),
                                           (K, True, -0.8), (3, False, 0.6)])
def test_one_warp_per_tile_passes_bitwise(iters, full, Fc):
    """With 16 points per thread the cut-off advance runs one warp per tile
    and computes the bits of the 4-point advance (the N bits and tile flags
    that the reinitialisation passes then use, the clamp when there are no
    reinitialisation iterations, the tube test, the breach count); speed
    field and constant speeds, the full domain."""
    phi, F = case(16)
    outs = []
    for ppt in (4, 16):
        g, _ = make(ls.LS_FP32, phi, None if Fc is not None else F, Fc=Fc, full=full, iters=iters)
        g.set_step_config(2, 100, ppt)
        for n in (2, 3, 4):
            g.step(n, 0.45, ls.LS_DT_CFL, 0 if full else 3)
        outs.append((g.get_phi(), None if full else g.active_tiles(), g.band_breaches(),
                     g.profile()["reinit_updates"]))
    a, b = outs
    assert np.array_equal(a[0].view(np.int32), b[0].view(np.int32))
    if a[1] is not None:
        assert np.array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]


def test_graph_replay_matches_eager_bitwise():
    phi, F = case(15)
    a, _ = make(ls.LS_FP32, phi, F)
    b, _ = make(ls.LS_FP32, phi, F)
    b.set_graphs(True)
    for _ in range(3):
        a.step(6, 0.45, ls.LS_DT_CFL, 3)
        b.step(6, 0.45, ls.LS_DT_CFL, 3)
    assert np.array_equal(a.get_phi().view(np.int32), b.get_phi().view(np.int32))


def test_stale_band_is_reported():
    """A band never rebuilt while the front runs off it: the library and the
    oracle both see N points in inactive tiles."""
    phi, _ = case(16)
    g, o = make(ls.LS_FP64, phi, None, Fc=1.0)
    g.step(40, 0.5, ls.LS_DT_CFL, 0)
    o.step(40, 0.5, oracle.DT_CFL, 0)
    assert g.band_breaches() > 0 and o.breaches > 0


def test_profile_counts_reinit_passes():
    phi, F = case(17)
    g, _ = make(ls.LS_FP32, phi, F)
    g.reset_profile()
    g.profile_enable(True)
    g.step(5, 0.45, ls.LS_DT_CFL, 3)
    p = g.profile()
    g.profile_enable(False)
    assert p["stencil_timed"] == 5 * (1 + K)
    assert p["reinit_timed"] == 5 * K
    assert 0.0 < p["reinit_ms"] < p["stencil_ms"]
    # the reinitialisation passes visit only the tiles holding points of N
    assert 0 < p["reinit_updates"] < K * g.updates()


def test_argument_and_state_errors():
    phi, F = case(18)
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32)
    for args in [(2, 1.0, 1, 0.5), (1, 0.0, 1, 0.5), (1, float("nan"), 1, 0.5), (1, 1.0, -2, 0.5),
                 (1, 1.0, 1, 0.0)]:
        with pytest.raises(ls.LSError) as e:
            g.set_scheme(*args)
        assert e.value.status == ls.LS_EINVAL
    g.set_phi(phi.astype(np.float32))
    g.set_speed(F.astype(np.float32))
    g.band_rebuild(3.0)
    g.set_scheme(ls.LS_SCHEME_LOCAL, 3.0, 2, 0.5)      # beta = halfwidth: not a cut-off
    with pytest.raises(ls.LSError) as e:
        g.step(1, 0.4, ls.LS_DT_CFL, 2)
    assert e.value.status == ls.LS_ESTATE
    g.set_scheme(ls.LS_SCHEME_PLAIN)
    g.step(1, 0.4, ls.LS_DT_CFL, 2)
    b = ls.Batch([16, 24], [1 / 16, 1 / 24])
    with pytest.raises(ls.LSError) as e:
        b.set_scheme(ls.LS_SCHEME_LOCAL, 1.0, 1, 0.5)
    assert e.value.status == ls.LS_EINVAL
