"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test names the passage it follows.  They are chosen so that a plausible
slip in the oracle fails at least one of them:

* a dropped or mis-signed term of Eq. 4/5, max and min swapped, or F's sign
  routed to the wrong gradient  -> the V / Lambda kink tests;
* a wrong stride or axis (x/y/z mixed up) -> the per-axis plane and kink tests
  on a non-cubic grid;
* a wrong domain-face rule -> the exact plane translation (faces included)
  and the neumann face test;
* a scheme that is not first order, or moves the front the wrong way -> the
  sphere radius r0 + F t convergence test;
* an operation order that breaks the mirror symmetry -> the bitwise octant
  reflection test;
* band, dilation, compaction or CFL slips -> brute-force enumerations on tiny
  grids and the huge-band == full-domain identity.
"""
import itertools

import numpy as np
import pytest

import oracle
from _geom import radius_error
from paper_1612_04040_b300 import inputs


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def axis_coord(shape, h, axis):
    """Cell-centred coordinate along array axis (0 = z, 1 = y, 2 = x)."""
    n = shape[axis]
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    sh = [1, 1, 1]
    sh[axis] = n
    return np.broadcast_to(c.reshape(sh), shape).copy()


SHAPE = (16, 24, 40)  # (nz, ny, nx): every axis a different length


# ---------------------------------------------------------------- Eq. 3 ----

def test_zero_speed_leaves_phi_unchanged():
    """Eq. 3 with F = 0: phi^{n+1} = phi^n, bit for bit (field and constant)."""
    g = np.random.default_rng(7)
    phi = g.normal(size=SHAPE)
    out = oracle.step(phi, h=1 / 16, dt=0.013, F=np.zeros(SHAPE))
    assert np.array_equal(bits(out), bits(phi))
    out = oracle.step(phi, h=1 / 16, dt=0.013, F=None, Fc=0.0)
    assert np.array_equal(bits(out), bits(phi))
    out = oracle.step(phi, h=1 / 16, dt=0.013, F=None, Fc=-0.0)
    assert np.array_equal(out, phi)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("F", [1.0, -0.5, 0.75])
def test_plane_translates_exactly(axis, sign, F):
    """Eq. 2-5: a plane phi = +-(x - x0) has |grad phi| = 1, so every step
    lowers phi by F dt.  With dyadic h, x0 and dt every operation is exact, so
    phi^n = phi^0 - n F dt holds bit for bit, at the domain faces too (the
    extrapolating face rule keeps the one-sided difference equal to 1)."""
    h = 2.0 ** -6
    phi0 = sign * (axis_coord(SHAPE, h, axis) - 5.0 / 16.0)
    o = oracle.Oracle(SHAPE, h)
    o.set_phi(phi0)
    o.set_speed_const(F)
    o.set_full_domain(True)
    dt = h / 2
    for n in range(1, 11):
        o.step(1, dt, oracle.DT_FIXED)
        assert np.array_equal(bits(o.phi), bits(phi0 - n * F * dt)), n


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_neumann_faces(axis):
    """The neumann face rule (ghost = edge value) makes the missing one-sided
    difference 0: for phi = x - x0 and F > 0 (Eq. 4 picks max(D-,0)) the low
    face point does not move, every other point drops by F dt; for F < 0
    (Eq. 5 picks max(D+,0)) the high face point does not move."""
    h = 2.0 ** -6
    dt = h / 2
    phi0 = axis_coord(SHAPE, h, axis) - 5.0 / 16.0
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis], hi[axis] = 0, -1
    out = oracle.step(phi0, h, dt, Fc=1.0, bc="neumann")
    exp = phi0 - dt
    exp[tuple(lo)] = phi0[tuple(lo)]
    assert np.array_equal(bits(out), bits(exp))
    out = oracle.step(phi0, h, dt, Fc=-1.0, bc="neumann")
    exp = phi0 + dt
    exp[tuple(hi)] = phi0[tuple(hi)]
    assert np.array_equal(bits(out), bits(exp))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_upwind_kinks(axis):
    """Eq. 4/5 at a kink.  For the V phi = |x - x_k| the apex has D- = -1,
    D+ = +1: G+ = sqrt(max(-1,0)^2 + min(1,0)^2) = 0 and G- = sqrt(2).  So F > 0
    leaves the apex in place and F < 0 raises it by |F| dt sqrt(2).  The
    Lambda phi = -|x - x_k| is the mirror case.  Every other point has
    |grad phi| = 1 and moves by F dt."""
    h = 2.0 ** -6
    dt = h / 2
    n = SHAPE[axis]
    k = n // 2
    i = np.arange(n, dtype=np.float64)
    sh = [1, 1, 1]
    sh[axis] = n
    v = np.broadcast_to((np.abs(i - k) * h).reshape(sh), SHAPE).copy()
    apex = [slice(None)] * 3
    apex[axis] = k
    apex = tuple(apex)
    r2 = np.sqrt(2.0)
    for phi0, F, apex_val in [
        (v, 1.0, lambda a: a),
        (v, -1.0, lambda a: a - dt * (-1.0 * r2)),
        (-v, 1.0, lambda a: a - dt * (1.0 * r2)),
        (-v, -1.0, lambda a: a),
    ]:
        out = oracle.step(phi0, h, dt, Fc=F)
        exp = phi0 - F * dt
        exp[apex] = apex_val(phi0[apex])
        assert np.array_equal(bits(out), bits(exp)), (F, apex_val)


def test_sphere_radius_first_order():
    """Eq. 1-3: a sphere of radius r0 under constant F = 1 has radius r0 + t.
    The first-order scheme's radius error must fall by ~2x each time h is
    halved (first order in h) and stay within one cell."""
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        phi = inputs.sphere_union_sdf((n,) * 3, h, [(0.5, 0.5, 0.5)], [0.25]).numpy()
        o = oracle.Oracle(phi.shape, h)
        o.set_phi(phi)
        o.set_speed_const(1.0)
        o.set_full_domain(True)
        steps = int(round(0.125 / (h / 2)))
        o.step(steps, h / 2, oracle.DT_FIXED)
        mean_h, max_h = radius_error(o.phi, h, (0.5, 0.5, 0.5), 0.25 + 0.125)
        assert abs(mean_h) <= 1.0 and max_h <= 1.0, (n, mean_h, max_h)
        errs.append(mean_h * h)
    for a, b in zip(errs, errs[1:]):
        assert 1.6 <= a / b <= 2.4, errs
    # the front must have moved outward (a sign slip moves it inward by 2t)
    assert all(abs(e) < 0.01 for e in errs)


def test_sphere_radius_standard_case():
    """The 64^3 single-sphere workload (h = 1/64, F = 1, dt = h/2): radius
    error within 1 h at every step n <= 24 (before the front nears the
    domain faces)."""
    w = inputs.SingleSphere()
    o = oracle.Oracle((w.n,) * 3, w.h)
    o.set_phi(w.phi().numpy())
    o.set_speed_const(w.speed)
    o.set_full_domain(True)
    for n in range(1, 25):
        o.step(1, w.h / 2, oracle.DT_FIXED)
        mean_h, max_h = radius_error(o.phi, w.h, w.centre, w.r0 + n * w.h / 2)
        assert max_h <= 1.0, (n, mean_h, max_h)


def test_octant_reflection_is_bitwise():
    """Eq. 4/5 are symmetric under x -> -x (the two addends of an axis swap;
    FP addition commutes), so the centred sphere stays mirror-symmetric bit
    for bit in every axis; axis permutations hold to rounding only."""
    w = inputs.SingleSphere()
    o = oracle.Oracle((w.n,) * 3, w.h)
    phi0 = w.phi().numpy()
    for ax in range(3):
        assert np.array_equal(bits(phi0), bits(np.flip(phi0, ax)))
    o.set_phi(phi0)
    o.set_speed_const(w.speed)
    o.set_full_domain(True)
    o.step(20, w.h / 2, oracle.DT_FIXED)
    for ax in range(3):
        assert np.array_equal(bits(o.phi), bits(np.ascontiguousarray(np.flip(o.phi, ax))))
    for perm in itertools.permutations(range(3)):
        assert np.max(np.abs(o.phi - np.transpose(o.phi, perm))) < 1e-14


# ------------------------------------------------------- band (Eq. 6, 11) --

def _naive_T(phi, gamma):
    nz, ny, nx = phi.shape
    T = np.zeros(phi.shape, dtype=bool)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                T[z, y, x] = abs(phi[z, y, x]) < gamma
    return T


def _naive_N(T):
    """Eq. 11 with the figure's reading (N contains T): x is in N when x or one
    of its +-dx neighbours along an axis is in T."""
    nz, ny, nx = T.shape
    N = np.zeros_like(T)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                on = T[z, y, x]
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    Z, Y, X = z + dz, y + dy, x + dx
                    if 0 <= Z < nz and 0 <= Y < ny and 0 <= X < nx and T[Z, Y, X]:
                        on = True
                N[z, y, x] = on
    return N


def test_pointwise_T_and_N_brute_force():
    """Eq. 6 and Eq. 11: with tile = 1 and the 6-neighbour dilation the band
    machinery gives exactly the pointwise tube T and region N."""
    g = np.random.default_rng(3)
    phi = g.uniform(-1, 1, size=(7, 9, 11))
    gamma = 0.3
    T = _naive_T(phi, gamma)
    core = oracle.classify(phi, gamma, tile=1)
    assert np.array_equal(core.astype(bool), T)
    N = oracle.dilate(core, conn=6)
    assert np.array_equal(N.astype(bool), _naive_N(T))


@pytest.mark.parametrize("tile", [2, 4, 8])
def test_tile_sets_brute_force(tile):
    """Per-tile Eq. 6, 26-neighbour one-tile dilation and ascending compaction
    against naive enumeration (partial edge tiles included for tile 8)."""
    g = np.random.default_rng(11 + tile)
    shape = (12, 20, 28)
    phi = g.uniform(-1, 1, size=shape) * 4
    gamma = 0.5
    core = oracle.classify(phi, gamma, tile)
    tnz, tny, tnx = core.shape
    T = _naive_T(phi, gamma)
    for tz in range(tnz):
        for ty in range(tny):
            for tx in range(tnx):
                blk = T[tz * tile:(tz + 1) * tile, ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile]
                assert core[tz, ty, tx] == int(blk.any())
    act = oracle.dilate(core, 26)
    for tz in range(tnz):
        for ty in range(tny):
            for tx in range(tnx):
                nb = core[max(tz - 1, 0):tz + 2, max(ty - 1, 0):ty + 2, max(tx - 1, 0):tx + 2]
                assert act[tz, ty, tx] == int(nb.any())
    ids = oracle.compact(act)
    flat = act.reshape(-1)
    assert ids.tolist() == [t for t in range(flat.size) if flat[t]]


def test_max_abs_speed_brute_force():
    """CFL bound: max |F| over the points of active tiles only (a huge value in
    an inactive tile must not count); 0 for an empty active set."""
    g = np.random.default_rng(5)
    shape = (16, 16, 24)
    F = g.uniform(-2, 2, size=shape)
    F[0:8, 0:8, 0:8] = 1e6
    act = np.zeros((2, 2, 3), dtype=np.uint8)
    act[1, 1, 2] = 1
    act[0, 1, 0] = 1
    mask = np.repeat(np.repeat(np.repeat(act, 8, 0), 8, 1), 8, 2).astype(bool)
    assert oracle.max_abs_speed(shape, F, 0.0, act) == np.abs(F[mask]).max()
    assert oracle.max_abs_speed(shape, F, 0.0, np.zeros_like(act)) == 0.0
    assert oracle.max_abs_speed(shape, None, -0.7, act) == 0.7
    assert oracle.max_abs_speed(shape, F) == 1e6


def test_cfl_dt_rule():
    """dt = CFL h / M with M the max |F| over the active set, and CFL h when
    M = 0 (F = 0 leaves phi unchanged anyway)."""
    w = inputs.SphereUnion(n=64, count=4)
    o = oracle.Oracle((64,) * 3, w.h)
    o.set_phi(w.phi().numpy())
    F = w.speed().numpy()
    o.set_speed(F)
    o.band_rebuild(6.0)
    dt = o.step(1, 0.5, oracle.DT_CFL, 5)
    M = oracle.max_abs_speed(F.shape, F, 0.0, o.active)
    assert dt == 0.5 * w.h / M
    o.set_speed_const(0.0)
    o.band_rebuild(6.0)
    assert o.step(1, 0.5, oracle.DT_CFL, 5) == 0.5 * w.h


def test_huge_band_equals_full_domain():
    """A band half-width larger than the domain makes every tile active, and
    the narrow-band run must equal the full-domain run bit for bit."""
    w = inputs.SphereUnion(n=32, count=3)
    phi0 = w.phi().numpy()
    F = w.speed().numpy()
    a = oracle.Oracle(phi0.shape, w.h)
    a.set_phi(phi0)
    a.set_speed(F)
    a.band_rebuild(1e6)
    a.step(12, 0.5, oracle.DT_CFL, 5)
    b = oracle.Oracle(phi0.shape, w.h)
    b.set_phi(phi0)
    b.set_speed(F)
    b.set_full_domain(True)
    b.step(12, 0.5, oracle.DT_CFL)
    assert np.array_equal(bits(a.phi), bits(b.phi))


def test_frozen_points_do_not_move():
    """Points outside the active tiles keep their value bit for bit."""
    w = inputs.SphereUnion(n=64, count=3)
    phi0 = w.phi().numpy()
    o = oracle.Oracle(phi0.shape, w.h)
    o.set_phi(phi0)
    o.set_speed(w.speed().numpy())
    o.band_rebuild(6.0)
    act = o.active.copy()
    o.step(5, 0.5, oracle.DT_CFL, 5)
    mask = np.repeat(np.repeat(np.repeat(act, 8, 0), 8, 1), 8, 2).astype(bool)
    assert np.array_equal(bits(o.phi[~mask]), bits(phi0[~mask]))
    assert not np.array_equal(o.phi[mask], phi0[mask])


def test_narrow_band_front_matches_full_domain():
    """Freezing points outside the band must not disturb the front: with
    rebuild_every <= gamma/(CFL h) - 2 the zero set of the narrow-band run
    stays within 0.1 h of the full-domain run."""
    w = inputs.SphereUnion(n=64, count=4)
    phi0 = w.phi().numpy()
    F = w.speed().numpy()
    a = oracle.Oracle(phi0.shape, w.h)
    a.set_phi(phi0)
    a.set_speed(F)
    a.band_rebuild(6.0)
    a.step(40, 0.5, oracle.DT_CFL, 5)
    b = oracle.Oracle(phi0.shape, w.h)
    b.set_phi(phi0)
    b.set_speed(F)
    b.set_full_domain(True)
    # same dt sequence: full domain uses max over the whole grid, so drive it
    # with the narrow-band run's dt values step by step
    c = oracle.Oracle(phi0.shape, w.h)
    c.set_phi(phi0)
    c.set_speed(F)
    c.band_rebuild(6.0)
    for _ in range(40):
        dt = c.step(1, 0.5, oracle.DT_CFL, 5)
        b.step(1, dt, oracle.DT_FIXED)
    assert np.array_equal(bits(c.phi), bits(a.phi))
    near = np.abs(b.phi) < w.h
    assert near.sum() > 1000
    assert np.max(np.abs(a.phi[near] - b.phi[near])) < 0.1 * w.h


def test_split_run_equals_unsplit_run():
    """The schedule depends only on the step count since the last rebuild, so
    5 + 7 steps in two calls equal 12 steps in one, bit for bit."""
    w = inputs.SphereUnion(n=32, count=3)
    phi0 = w.phi().numpy()
    F = w.speed().numpy()
    runs = []
    for parts in ((12,), (5, 7), (3, 3, 6)):
        o = oracle.Oracle(phi0.shape, w.h)
        o.set_phi(phi0)
        o.set_speed(F)
        o.band_rebuild(4.0)
        for p in parts:
            o.step(p, 0.5, oracle.DT_CFL, 5)
        runs.append((o.phi, o.rebuild_log))
    for phi, log in runs[1:]:
        assert np.array_equal(bits(phi), bits(runs[0][0]))
        assert len(log) == len(runs[0][1])
        for x, y in zip(log, runs[0][1]):
            assert np.array_equal(x, y)


def test_tube_test_is_strict():
    """Eq. 6 uses a strict inequality: a tile whose smallest |phi| equals gamma
    exactly is outside T; one ulp below gamma is inside (for either sign)."""
    gamma = 6.0 / 512.0
    for s in (1.0, -1.0):
        phi = np.full((8, 8, 16), 1.0)
        phi[3, 4, 5] = s * gamma
        phi[2, 2, 12] = s * np.nextafter(gamma, 0.0)
        core = oracle.classify(phi, gamma, tile=8)
        assert core.tolist() == [[[0, 1]]]
