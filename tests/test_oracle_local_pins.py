"""Pins of the oracle's local level-set scheme (section 1.1, Steps 1-3: the
cut-off PDE of Eq. 7-8, the region N of Eq. 11, the reinitialisation of
Eq. 12-13 and the clamp of Eq. 10) against closed forms, fixed points,
brute force, symmetry and convergence -- never against the oracle's own
formulas retyped."""
import numpy as np
import pytest

import oracle

H = 2.0 ** -5   # dyadic spacing: plane values and differences are exact


def grid_x(shape, h, axis):
    n = shape[2 - axis]
    c = (np.arange(n) + 0.5) * h
    sh = [1, 1, 1]
    sh[2 - axis] = n
    return np.broadcast_to(c.reshape(sh), shape)


def smoothstep_cut(a, beta, gamma):
    """Eq. 7 rewritten in s = (a - beta)/(gamma - beta): 1 - 3 s^2 + 2 s^3 on
    [beta, gamma] (expand (s-1)^2 (2s+1)), 1 below, 0 above."""
    s = (a - beta) / (gamma - beta)
    return np.where(a <= beta, 1.0, np.where(a >= gamma, 0.0, 1.0 - 3.0 * s * s + 2.0 * s ** 3))


# -- Eq. 7 -----------------------------------------------------------------

def test_cutoff_endpoints_midpoint_and_smoothness():
    beta, gamma = 1.0, 3.0
    assert oracle.cutoff(beta, beta, gamma) == 1.0
    assert oracle.cutoff(gamma, beta, gamma) == 0.0
    assert oracle.cutoff(2.0, beta, gamma) == 0.5          # midpoint, exact
    assert oracle.cutoff(0.0, beta, gamma) == 1.0
    assert oracle.cutoff(7.0, beta, gamma) == 0.0
    a = np.linspace(0.0, 4.0, 4001)
    got = np.array([oracle.cutoff(v, beta, gamma) for v in a])
    assert np.max(np.abs(got - smoothstep_cut(a, beta, gamma))) < 1e-14
    # C1 at both ends: the one-sided slopes vanish (second-order contact)
    for eps in (1e-2, 1e-3):
        assert abs(oracle.cutoff(beta + eps, beta, gamma) - 1.0) < 3.0 * (eps / 2.0) ** 2 * 1.01
        assert abs(oracle.cutoff(gamma - eps, beta, gamma)) < 3.0 * (eps / 2.0) ** 2 * 1.01
    assert np.all(np.diff(got) <= 0.0)                       # monotone


# -- Eq. 8 -----------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sgn", [1.0, -1.0])
def test_cut_step_on_a_plane_moves_by_c_times_dt(axis, sgn):
    """phi = x - x0 has one-sided differences exactly 1 (face rule
    included), so one step moves each point by -F dt c(|phi|)."""
    shape = (16, 16, 16)
    beta, gamma = 3 * H, 6 * H
    phi = grid_x(shape, H, axis) - 0.5 + H / 2          # dyadic values k*H
    dt = H / 4
    out = oracle.cut_step(phi, H, dt, beta, gamma, Fc=sgn)
    exp = phi - sgn * dt * smoothstep_cut(np.abs(phi), beta, gamma)
    assert np.max(np.abs(out - exp)) < 1e-15
    far = np.abs(phi) >= gamma
    assert np.array_equal(out[far], phi[far])                 # outside T: frozen
    inner = np.abs(phi) <= beta
    assert np.array_equal(out[inner], phi[inner] - sgn * dt)


def test_cut_step_without_cutoff_is_the_plain_step():
    g = np.random.default_rng(4)
    phi = g.uniform(-0.3, 0.3, (12, 10, 14))
    F = g.uniform(-1.0, 1.0, phi.shape)
    out = oracle.cut_step(phi, H, 0.2 * H, 1.0, 2.0, F=F)   # |phi| < beta: c = 1
    assert np.array_equal(out, oracle.step(phi, H, 0.2 * H, F=F))


# -- Eq. 11 ----------------------------------------------------------------

def test_region_n_brute_force():
    g = np.random.default_rng(5)
    gamma = 0.25
    phi = g.uniform(-1.0, 1.0, (9, 10, 12))
    got = oracle.region_n(phi, gamma)
    nz, ny, nx = phi.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cand = [(z, y, x), (z, y, x - 1), (z, y, x + 1), (z, y - 1, x), (z, y + 1, x),
                        (z - 1, y, x), (z + 1, y, x)]
                want = any(0 <= c[0] < nz and 0 <= c[1] < ny and 0 <= c[2] < nx
                           and abs(phi[c]) < gamma for c in cand)
                assert got[z, y, x] == int(want), (z, y, x)
    # T is inside N, and N is T grown by exactly one face-connected cell
    T = np.abs(phi) < gamma
    assert np.all(got[T] == 1)


# -- Eq. 12-13 -------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("orient", [1.0, -1.0])
def test_reinit_leaves_a_signed_distance_plane_unchanged(axis, orient):
    shape = (12, 12, 12)
    d = orient * (grid_x(shape, H, axis) - 0.5)
    out = oracle.reinit_iter(d, H, 0.5 * H)
    assert np.array_equal(out, d)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_reinit_straightens_a_steep_plane_to_the_distance(axis, shift):
    """d = 2 (x - x0) relaxes to x - x0 (the steady state |grad d| = 1 with
    the zero set fixed), with x0 on a grid point or half-way between."""
    shape = (8, 8, 24) if axis == 0 else ((8, 24, 8) if axis == 1 else (24, 8, 8))
    x = grid_x(shape, H, axis)
    x0 = (11 + 0.5 + shift) * H
    d = 2.0 * (x - x0)
    for _ in range(400):
        d = oracle.reinit_iter(d, H, 0.5 * H)
    assert np.max(np.abs(d - (x - x0))) < 1e-9 * H


def test_reinit_far_from_the_front_moves_at_unit_speed():
    """Eq. 13 makes S a sign function smoothed over about one cell: where
    |d| >> |Dd| dx, S = sign(d) and one iteration on the steep plane
    d = 2(x - x0) moves d by -sign(d) dtau (|grad d| - 1) = -sign(d) dtau."""
    shape = (8, 8, 96)
    x = grid_x(shape, H, 0)
    x0 = 48 * H
    d = 2.0 * (x - x0)
    dtau = 0.5 * H
    out = oracle.reinit_iter(d, H, dtau)
    far = (np.abs(d) >= 32 * H) & (x > H) & (x < 95 * H)
    step = out[far] - d[far]
    assert np.max(np.abs(step + np.sign(d[far]) * dtau)) < 0.01 * dtau
    # and the closer to the front, the slower (S grows with |d|)
    row = out[0, 0] - d[0, 0]
    right = np.abs(row[49:90])
    assert np.all(np.diff(right) >= -1e-18)


def test_reinit_of_a_sphere_converges_at_first_order():
    """d0 = 3(|x-c|^2 - r^2) (the sphere as zero set, not a distance):
    iterated to steady state, d approaches |x-c| - r near the front with an
    error that falls by about 2 per halving of h."""
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        rr = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
        d = 3.0 * (rr ** 2 - 0.09)
        for _ in range(4 * n):
            d = oracle.reinit_iter(d, h, 0.5 * h)
        near = np.abs(rr - 0.3) < 3 * h
        e = np.max(np.abs(d - (rr - 0.3))[near])
        assert e < 0.7 * h
        errs.append(e)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 <= r1 <= 3.0 and 1.6 <= r2 <= 3.0, errs


def test_reinit_only_touches_the_mask():
    g = np.random.default_rng(6)
    d = g.uniform(-1, 1, (8, 9, 10))
    m = (g.uniform(size=d.shape) < 0.5).astype(np.uint8)
    out = oracle.reinit_iter(d, H, 0.5 * H, m)
    assert np.array_equal(out[m == 0], d[m == 0])
    full = oracle.reinit_iter(d, H, 0.5 * H)
    assert np.array_equal(out[m == 1], full[m == 1])


# -- Eq. 10 ----------------------------------------------------------------

def test_clamp():
    d = np.array([-3.0, -2.0, -1.5, 0.0, 1.5, 2.0, 2.5]).reshape(1, 1, 7)
    assert np.array_equal(oracle.clamp(d, 2.0).ravel(), [-2.0, -2.0, -1.5, 0.0, 1.5, 2.0, 2.0])
    m = np.array([1, 0, 1, 1, 1, 1, 0], dtype=np.uint8).reshape(d.shape)
    assert np.array_equal(oracle.clamp(d, 1.0, m).ravel(), [-1.0, -2.0, -1.0, 0.0, 1.0, 1.0, 2.5])


# -- Steps 1-3 together ----------------------------------------------------

def sphere_phi(n, r0):
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - r0, h


def crossing_radii(phi, h):
    """Distances from the centre of the linearly interpolated zero crossings
    along every grid edge whose ends differ in sign."""
    n = phi.shape[0]
    x = (np.arange(n) + 0.5) * h
    out = []
    for ax in range(3):
        a = np.moveaxis(phi, ax, 2)
        s0, s1 = a[..., :-1], a[..., 1:]
        i0, i1, i2 = np.nonzero((s0 < 0) != (s1 < 0))
        t = s0[i0, i1, i2] / (s0[i0, i1, i2] - s1[i0, i1, i2])
        p = [x[i0], x[i1], x[i2] + t * h]
        out.append(np.sqrt(sum((q - 0.5) ** 2 for q in p)))
    return np.concatenate(out)


def test_local_scheme_sphere_radius_first_order():
    """Constant F = 1 from r0 = 1/4: the front of Steps 1-3 sits at r0 + t
    with an error proportional to h (first-order scheme), below one cell."""
    errs = []
    for n in (32, 64, 128):
        phi, h = sphere_phi(n, 0.25)
        o = oracle.Oracle(phi.shape, h)
        o.set_phi(phi)
        o.set_speed_const(1.0)
        o.band_rebuild(6.0)
        o.set_scheme(oracle.SCHEME_LOCAL, 3.0, 5, 0.5)
        steps = 12 * n // 32
        o.step(steps, 0.5 * h, oracle.DT_FIXED, 5)
        e = crossing_radii(o.phi, h) - (0.25 + steps * 0.5 * h)
        assert np.max(np.abs(e)) < 1.0 * h
        assert o.breaches == 0
        errs.append(abs(float(np.mean(e))))
    assert 1.6 <= errs[0] / errs[1] <= 2.4 and 1.6 <= errs[1] / errs[2] <= 2.4, errs


def test_local_scheme_octant_symmetry_bitwise():
    phi, h = sphere_phi(32, 0.2)
    o = oracle.Oracle(phi.shape, h)
    o.set_phi(phi)
    o.set_speed_const(-0.75)
    o.band_rebuild(5.0)
    o.set_scheme(oracle.SCHEME_LOCAL, 2.5, 4, 0.5)
    o.step(9, 0.5, oracle.DT_CFL, 4)
    p = o.phi
    for ax in range(3):
        assert np.array_equal(p, np.flip(p, axis=ax))


def test_local_scheme_without_cutoff_reinit_or_clamp_is_the_plain_step():
    g = np.random.default_rng(8)
    phi = g.uniform(-0.2, 0.2, (10, 12, 8))
    F = g.uniform(-1, 1, phi.shape)
    out, m = oracle.local_step(phi, H, 0.3 * H, 1.0, 2.0, 0, 0.5 * H, F=F)
    assert np.all(m == 1)
    assert np.array_equal(out, oracle.step(phi, H, 0.3 * H, F=F))


def test_local_scheme_clamps_n_and_freezes_the_rest():
    phi, h = sphere_phi(24, 0.2)
    gamma = 4 * h
    out, m = oracle.local_step(phi, h, 0.5 * h, 2 * h, gamma, 3, 0.5 * h, Fc=1.0)
    assert np.all(np.abs(out[m == 1]) <= gamma)
    assert np.array_equal(out[m == 0], phi[m == 0])
