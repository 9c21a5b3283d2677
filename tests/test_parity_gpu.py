"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Bars (stated once, used below):
* active-tile sets: identical ids, in ascending order, at every rebuild;
* FP64 mode: bit for bit (1e-12 max-abs is the stated bar; the kernel follows
  the definition's operation order with round-to-nearest intrinsics, so it
  lands on the same bits);
* FP32 mode: max |phi_gpu - phi_oracle| <= 1e-5 * h * nsteps on the points of
  the tiles active at the last rebuild.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def tile_mask(active, shape):
    return np.repeat(np.repeat(np.repeat(active.astype(bool), 8, 0), 8, 1), 8, 2)[
        :shape[0], :shape[1], :shape[2]]


def make_pair(shape, h, prec, phi0, F=None, Fc=None, device_inputs=False, bc="extrapolate"):
    nz, ny, nx = shape
    g = ls.LevelSet(nx, ny, nz, h, prec)
    dt = np.float32 if prec == ls.LS_FP32 else np.float64
    p = np.ascontiguousarray(phi0, dtype=dt)
    g.set_phi(torch.from_numpy(p).cuda() if device_inputs else p)
    o = oracle.Oracle(shape, h, bc=bc)
    o.set_phi(p.astype(np.float64))
    if F is not None:
        f = np.ascontiguousarray(F, dtype=dt)
        g.set_speed(torch.from_numpy(f).cuda() if device_inputs else f)
        o.set_speed(f.astype(np.float64))
    else:
        g.set_speed_const(Fc)
        o.set_speed_const(Fc)
    if bc == "neumann":
        g.set_bc(ls.LS_BC_NEUMANN)
    return g, o


def run_chunks(g, o, chunks, value, mode, rebuild_every, check_tiles=True):
    for n in chunks:
        dg = g.step(n, value, mode, rebuild_every, want_dt=True)
        do = o.step(n, value, mode, rebuild_every)
        assert dg == do, (dg, do)  # dt is bitwise (max is order-independent)
        if check_tiles and not o.full_domain:
            assert np.array_equal(g.active_tiles(), o.active_tiles())


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


# ------------------------------------------------------------------ FP64 ----

def test_fp64_single_sphere_full_domain_bitwise():
    """64^3 sphere, F = 1, dt = h/2, 100 full-domain steps: bit for bit."""
    w = inputs.SingleSphere()
    shape = (w.n,) * 3
    g, o = make_pair(shape, w.h, ls.LS_FP64, w.phi().numpy(), Fc=w.speed)
    g.set_full_domain(True)
    o.set_full_domain(True)
    for n in (1, 9, 40, 50):
        g.step(n, w.h / 2, ls.LS_DT_FIXED)
        o.step(n, w.h / 2, oracle.DT_FIXED)
        out = g.get_phi()
        assert np.array_equal(bits(out), bits(o.phi))
    assert g.updates() == 100 * w.n ** 3


@pytest.mark.parametrize("device_inputs", [False, True])
@pytest.mark.parametrize("mode", [ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL])
def test_fp64_narrow_band_field_bitwise(device_inputs, mode):
    """Union of spheres, sinusoidal F field, band 6h, rebuild every 5 steps,
    CFL 0.5, on a non-cubic grid: phi bit for bit and the active-tile set
    identical at every rebuild, with the periodic rebuilds walking every
    tile or marked from the previous list's core entries."""
    shape = (64, 48, 80)
    h = 1.0 / 64
    w = inputs.SphereUnion(n=64, count=6)
    phi0 = inputs.sphere_union_sdf(shape, h, w.centres, w.radii).numpy()
    F = inputs.speed_sinusoid(shape, h).numpy()
    g, o = make_pair(shape, h, ls.LS_FP64, phi0, F=F, device_inputs=device_inputs)
    g.set_rebuild_mode(mode)
    ng = g.band_rebuild(6.0)
    no = o.band_rebuild(6.0)
    assert ng == no
    run_chunks(g, o, [5, 5, 3, 7, 10], 0.5, ls.LS_DT_CFL, 5)
    assert np.array_equal(bits(g.get_phi()), bits(o.phi))


def test_fp64_six_neighbour_dilation_bitwise():
    """The band dilated over the 6 face neighbours only (ls_set_dilation):
    the same trajectory and tile sets as the oracle's 6-neighbour dilation,
    and a smaller band than the 26-neighbour one."""
    shape = (64, 48, 80)
    h = 1.0 / 64
    w = inputs.SphereUnion(n=64, count=6)
    phi0 = inputs.sphere_union_sdf(shape, h, w.centres, w.radii).numpy()
    F = inputs.speed_sinusoid(shape, h).numpy()
    g, _ = make_pair(shape, h, ls.LS_FP64, phi0, F=F)
    o = oracle.Oracle(shape, h, conn=6)
    o.set_phi(phi0)
    o.set_speed(F)
    g.set_dilation(6)
    g.set_rebuild_mode(ls.LS_REBUILD_INCREMENTAL)   # the 6-neighbour marks
    n6 = g.band_rebuild(6.0)
    assert n6 == o.band_rebuild(6.0)
    g26, _ = make_pair(shape, h, ls.LS_FP64, phi0, F=F)
    assert n6 < g26.band_rebuild(6.0)
    run_chunks(g, o, [5, 5, 3, 7], 0.5, ls.LS_DT_CFL, 5)
    assert np.array_equal(bits(g.get_phi()), bits(o.phi))
    with pytest.raises(ls.LSError):
        g.set_dilation(8)


def test_fp64_non_power_of_two_h_bitwise():
    """h = 1/48 (not a power of two: the kernel divides by h like the
    definition) with a sign-changing F."""
    shape = (48, 48, 48)
    h = 1.0 / 48
    phi0 = inputs.torus_sdf(shape, h, (0.5, 0.5, 0.5), (0.0, 0.6, 0.8), 0.25, 0.08).numpy()
    F = inputs.speed_cos_cos(shape, h).numpy()
    g, o = make_pair(shape, h, ls.LS_FP64, phi0, F=F)
    g.band_rebuild(4.0)
    o.band_rebuild(4.0)
    run_chunks(g, o, [4, 4, 4], 0.5, ls.LS_DT_CFL, 4)
    assert np.array_equal(bits(g.get_phi()), bits(o.phi))


def test_fp64_extreme_magnitudes_bitwise():
    """For a power-of-two h the kernel works on unscaled differences while
    every intermediate stays a normal number, and falls back to the scaled
    sequence otherwise. Blocks of phi scaled so that the squares of the
    differences are subnormal (1e-155), underflow (1e-300) or are huge
    (1e149), and speeds that are tiny (1e-130), +0 or -0, mix both paths
    inside warps; every point must still match the oracle bit for bit."""
    shape = (32, 32, 32)
    h = 1.0 / 32
    phi0 = inputs.sphere_union_sdf(shape, h, [(0.5, 0.5, 0.5)], [0.3]).numpy()
    phi0[0:8, 0:8, 0:16] *= 1e-155
    phi0[8:16, 0:8, 0:16] *= 1e-300
    phi0[16:24, 8:16, 4:28] *= 1e149
    phi0[24:32, 24:32, 3:29] *= 1e-155
    F = inputs.speed_cos_cos(shape, h).numpy()
    F[:, :, 5] = 1e-130
    F[:, 3, :] = 0.0
    F[7, :, :] = -0.0
    F[:, 20:24, 9] = -3e-140
    g, o = make_pair(shape, h, ls.LS_FP64, phi0, F=F)
    g.set_full_domain(True)
    o.set_full_domain(True)
    for n in (1, 2):
        g.step(n, h / 4, ls.LS_DT_FIXED)
        o.step(n, h / 4, oracle.DT_FIXED)
        out = g.get_phi()
        assert np.isfinite(out).all()
        assert np.array_equal(bits(out), bits(o.phi))


def test_fp64_neumann_faces_bitwise():
    """The neumann face rule, with a front that reaches the domain faces."""
    shape = (32, 32, 32)
    h = 1.0 / 32
    phi0 = inputs.sphere_union_sdf(shape, h, [(0.2, 0.5, 0.85)], [0.3]).numpy()
    g, o = make_pair(shape, h, ls.LS_FP64, phi0, Fc=-0.7, bc="neumann")
    g.set_full_domain(True)
    o.set_full_domain(True)
    run_chunks(g, o, [7, 8], 0.45, ls.LS_DT_CFL, 0)
    assert np.array_equal(bits(g.get_phi()), bits(o.phi))


# ------------------------------------------------------------------ FP32 ----

@pytest.mark.parametrize("config", [None, (2, 100, 8), (2, 100, 16)])
def test_fp32_sphere_union_reduced_size(config):
    """The 512^3 sphere-union recipe at 128^3 (same seeds, centres, radii and
    F), 60 steps: band sets identical at every rebuild, phi within
    1e-5 h nsteps on the final band.  Each stencil decomposition (4, 8, 16
    points per thread), all of which read the x-faces of frozen neighbours
    from the copy the rebuild makes."""
    w = inputs.SphereUnion(n=128)
    shape = (w.n,) * 3
    g, o = make_pair(shape, w.h, ls.LS_FP32, w.phi().numpy(), F=w.speed().numpy())
    if config:
        g.set_step_config(*config)
    assert g.band_rebuild(w.halfwidth) == o.band_rebuild(w.halfwidth)
    nsteps = 0
    for n in (5,) * 12:
        dg = g.step(n, w.cfl, ls.LS_DT_CFL, w.rebuild_every, want_dt=True)
        do = o.step(n, w.cfl, oracle.DT_CFL, w.rebuild_every)
        nsteps += n
        assert dg == do
        assert np.array_equal(g.active_tiles(), o.active_tiles())
    out = g.get_phi().astype(np.float64)
    m = tile_mask(o.active, shape)
    err = np.max(np.abs(out[m] - o.phi[m]))
    assert err <= 1e-5 * w.h * nsteps, err


@pytest.mark.parametrize("ppt,mode", [(4, ls.LS_REBUILD_FULL), (8, ls.LS_REBUILD_FULL),
                                      (16, ls.LS_REBUILD_FULL), (16, ls.LS_REBUILD_INCREMENTAL)])
def test_fp32_frozen_face_copies_follow_the_band(ppt, mode):
    """The steps read the x-faces of frozen neighbours from copies made after
    each rebuild; the copies stay right through rebuilds with no step
    between them, graph replay in uneven chunks, the autotuner's probe
    launches and a new phi in the middle of a run (oracle parity on the
    band, identical band sets)."""
    w = inputs.SphereUnion(n=64, count=6)
    shape = (w.n,) * 3
    F = w.speed().numpy()
    g, o = make_pair(shape, w.h, ls.LS_FP32, w.phi().numpy(), F=F)
    g.set_step_config(2, 100, ppt)
    g.set_rebuild_mode(mode)
    for _ in range(2):  # two rebuilds, no step between them
        assert g.band_rebuild(w.halfwidth) == o.band_rebuild(w.halfwidth)
    g.set_graphs(True)
    run_chunks(g, o, [3, 4, 3, 5, 5, 2], w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    g.autotune(reps=1)
    g.set_step_config(2, 100, ppt)
    run_chunks(g, o, [6, 4], w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    # a new level set (the spheres moved by 3h): a full rebuild, new copies
    w2 = inputs.SphereUnion(n=64, count=6)
    w2.centres = [(x + 3 * w.h, y, z) for (x, y, z) in w2.centres]
    p2 = w2.phi().numpy().astype(np.float32)
    g.set_phi(p2)
    o.set_phi(p2.astype(np.float64))
    run_chunks(g, o, [5, 5, 1, 4], w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    out = g.get_phi().astype(np.float64)
    m = tile_mask(o.active, shape)
    assert np.max(np.abs(out[m] - o.phi[m])) <= 1e-5 * w.h * 15


@pytest.mark.parametrize("ppt", [4, 8, 16])
def test_fp32_non_cubic_band_each_decomposition(ppt):
    """A non-cubic grid (7 x 5 x 9 tiles, every tile count odd, h fixed by
    the z edge) with two spheres whose band reaches domain faces: the band sets
    agree with the oracle at every rebuild and phi stays within the FP32 bar
    on the band, for each stencil decomposition (the one-warp kernel with
    its frozen x-face copies included)."""
    nz, ny, nx = 72, 40, 56
    h = 1.0 / 72
    shape = (nz, ny, nx)
    phi0 = inputs.sphere_union_sdf(shape, h, [(0.30, 0.28, 0.35), (0.55, 0.30, 0.70)],
                                   [0.22, 0.18]).numpy()
    F = inputs.speed_sinusoid(shape, h).numpy()
    g, o = make_pair(shape, h, ls.LS_FP32, phi0, F=F)
    g.set_step_config(2, 100, ppt)
    assert g.band_rebuild(5.0) == o.band_rebuild(5.0)
    run_chunks(g, o, [5, 5, 3, 7], 0.5, ls.LS_DT_CFL, 5)
    out = g.get_phi().astype(np.float64)
    m = tile_mask(o.active, shape)
    assert m.any()
    assert np.max(np.abs(out[m] - o.phi[m])) <= 1e-5 * h * 20


def test_profile_sampling_counts():
    """Event timing of every run of stencil launches, and of one run in N:
    the timed launches and their point updates are counted exactly."""
    w = inputs.SphereUnion(n=64, count=5)
    g, _ = make_pair((64,) * 3, w.h, ls.LS_FP32, w.phi().numpy(), F=w.speed().numpy())
    g.band_rebuild(w.halfwidth)
    g.step(1, w.cfl, ls.LS_DT_CFL, 5)  # the next call starts at a rebuild
    g.step(4, w.cfl, ls.LS_DT_CFL, 5)
    for every, runs_timed in ((1, 6), (4, 2)):
        g.reset_profile()
        g.profile_enable(every)
        u0 = g.updates()
        g.step(30, w.cfl, ls.LS_DT_CFL, 5)  # 6 runs of 5 launches, a rebuild before each
        p = g.profile()
        g.profile_enable(False)
        assert p["stencil_launches"] == 30
        assert p["stencil_timed"] == 5 * runs_timed
        assert p["stencil_ms"] > 0.0
        if every == 1:
            assert p["stencil_updates"] == g.updates() - u0
        else:
            assert 0 < p["stencil_updates"] < g.updates() - u0
    with pytest.raises(ls.LSError):
        g.profile_enable(-1)


def test_fp32_tube_test_matches_oracle_on_gpu_snapshot():
    """The GPU's band decision on its own FP32 state equals the oracle's FP64
    tube test + dilation applied to that same state (exact)."""
    w = inputs.SphereUnion(n=96, count=8)
    shape = (w.n,) * 3
    g, _ = make_pair(shape, w.h, ls.LS_FP32, w.phi().numpy(), F=w.speed().numpy())
    g.band_rebuild(w.halfwidth)
    for k in range(6):
        g.step(5 if k == 0 else 4, 0.5, ls.LS_DT_CFL, 5)
        snap = g.get_phi().astype(np.float64)
        g.step(1, 0.5, ls.LS_DT_CFL, 5)  # rebuilds first, from the fused tube flags
        core = oracle.classify(snap, w.halfwidth * w.h)
        assert np.array_equal(g.active_tiles(), oracle.compact(oracle.dilate(core, 26)))


def test_fp32_constant_speed_shrinking():
    """Constant negative F (a shrinking torus and a shrinking sphere) with the
    4h band."""
    e = 64
    h = 1.0 / e
    shape = (e, e, e)
    cases = [
        (inputs.torus_sdf(shape, h, (0.5, 0.45, 0.55), (0.36, 0.48, 0.8), 0.25, 0.12).numpy(), 10),
        (inputs.sphere_union_sdf(shape, h, [(0.52, 0.47, 0.5)], [0.35]).numpy(), 40),
    ]
    for phi0, nsteps in cases:
        g, o = make_pair(shape, h, ls.LS_FP32, phi0, Fc=-0.8)
        g.band_rebuild(4.0)
        o.band_rebuild(4.0)
        run_chunks(g, o, [5] * (nsteps // 5), 0.5, ls.LS_DT_CFL, 5)
        out = g.get_phi().astype(np.float64)
        m = tile_mask(o.active, shape)
        assert m.any()
        assert np.max(np.abs(out[m] - o.phi[m])) <= 1e-5 * h * nsteps


# ------------------------------------------------------------ edge cases ----

def test_single_tile_grid():
    """8^3 grid: one tile, every neighbour outside the domain."""
    h = 1.0 / 8
    phi0 = inputs.sphere_union_sdf((8, 8, 8), h, [(0.5, 0.5, 0.5)], [0.3]).numpy()
    for prec in (ls.LS_FP32, ls.LS_FP64):
        g, o = make_pair((8, 8, 8), h, prec, phi0, Fc=1.0)
        g.band_rebuild(3.0)
        o.band_rebuild(3.0)
        run_chunks(g, o, [3, 3], 0.5, ls.LS_DT_CFL, 2)
        if prec == ls.LS_FP64:
            assert np.array_equal(bits(g.get_phi()), bits(o.phi))
        else:
            assert np.max(np.abs(g.get_phi() - o.phi)) <= 1e-5 * h * 6


def test_ragged_tile_grid_fp64():
    """Tile grid 1 x 3 x 5 (nx = 8): x faces on both sides of every tile."""
    shape = (40, 24, 8)
    h = 1.0 / 32
    g_ = np.random.default_rng(4)
    phi0 = inputs.sphere_union_sdf(shape, h, [(0.1, 0.4, 0.6)], [0.25]).numpy()
    F = g_.uniform(-1, 1, size=shape)
    g, o = make_pair(shape, h, ls.LS_FP64, phi0, F=F)
    g.band_rebuild(5.0)
    o.band_rebuild(5.0)
    run_chunks(g, o, [2, 2, 2, 2], 0.4, ls.LS_DT_CFL, 2)
    assert np.array_equal(bits(g.get_phi()), bits(o.phi))


def test_empty_band():
    """No point within gamma: no active tile, phi unchanged, dt = CFL h."""
    h = 1.0 / 32
    phi0 = np.full((32, 32, 32), 0.5)
    g, o = make_pair((32, 32, 32), h, ls.LS_FP64, phi0, Fc=1.0)
    assert g.band_rebuild(2.0) == 0 == o.band_rebuild(2.0)
    dt = g.step(5, 0.5, ls.LS_DT_CFL, 5, want_dt=True)
    assert dt == 0.5 * h
    assert np.array_equal(g.get_phi(), phi0)
    assert g.updates() == 0


def test_zero_speed_identity_gpu():
    """F = 0: phi unchanged bit for bit on the GPU too (FP32 and FP64)."""
    w = inputs.SphereUnion(n=32, count=3)
    phi0 = w.phi().numpy()
    for prec, dt in ((ls.LS_FP32, np.float32), (ls.LS_FP64, np.float64)):
        g, _ = make_pair((32,) * 3, w.h, prec, phi0, F=np.zeros((32,) * 3))
        g.band_rebuild(4.0)
        g.step(7, 0.5, ls.LS_DT_CFL, 3)
        assert np.array_equal(g.get_phi(), phi0.astype(dt))


def test_split_run_equals_unsplit_run_gpu():
    """Resume == continue: 12 steps in one call equal 5 + 7 (FP32, bitwise)."""
    w = inputs.SphereUnion(n=64, count=5)
    phi0, F = w.phi().numpy(), w.speed().numpy()
    outs = []
    for parts in ((12,), (5, 7)):
        g, _ = make_pair((64,) * 3, w.h, ls.LS_FP32, phi0, F=F)
        g.band_rebuild(6.0)
        for p in parts:
            g.step(p, 0.5, ls.LS_DT_CFL, 5)
        outs.append(g.get_phi())
    assert np.array_equal(outs[0], outs[1])


def test_state_errors():
    g = ls.LevelSet(16, 16, 16, 1 / 16, ls.LS_FP32)
    with pytest.raises(ls.LSError) as e:
        g.step(1, 0.5, ls.LS_DT_CFL, 5)
    assert e.value.status == ls.LS_ESTATE
    phi = np.zeros((16, 16, 16), np.float32)
    phi[3, 4, 5] = np.nan
    with pytest.raises(ls.LSError) as e:
        g.set_phi(phi)
    assert e.value.status == ls.LS_ENONFINITE
    g.set_phi(np.ones((16, 16, 16), np.float32))
    g.set_speed_const(1.0)
    with pytest.raises(ls.LSError) as e:
        g.step(1, 0.5, ls.LS_DT_CFL, 5)  # no halfwidth yet
    assert e.value.status == ls.LS_ESTATE
    with pytest.raises(ls.LSError) as e:
        g.band_rebuild(-1.0)
    assert e.value.status == ls.LS_EINVAL
    for mode in (ls.LS_REBUILD_AUTO, ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL):
        g.set_rebuild_mode(mode)
    with pytest.raises(ls.LSError) as e:
        g.set_rebuild_mode(3)
    assert e.value.status == ls.LS_EINVAL
    assert g.status() == ls.LS_OK
