"""Pins of the oracle's corrected step and training step (the learned
corrector is not in the paper; its readings are this project's): features,
the output scaling, the band-residual check, the plain fallback, the masked
mean-squared-error gradient, Adam and one whole training iteration.  Each
pin is a fact fixed independently of the oracle's code: exact values of a
plane front, the boundary of the check to one ulp, closed forms of the loss
and of Adam's first steps, finite differences of the whole training loss."""
import numpy as np
import pytest

import oracle

H = 1.0 / 64            # dyadic: phi / h and the plane step are exact


def plane(shape, h, x0, slope=1.0):
    nz, ny, nx = shape
    x = (np.arange(nx) + 0.5) * h - x0
    return np.broadcast_to(slope * x[None, None, :], shape).copy()


# ---------------------------------------------------------------- features

def test_features_of_a_moving_plane_are_exact():
    """phi = x - x0 (unit gradient), F = 1/2, dt = h/2: the plain step moves
    the plane by exactly F dt (Eq. 3 with D = 1), so the third channel is
    -F dt / h = -1/4 at every point; the first is phi / h clamped to +-8."""
    shape = (8, 8, 64)
    phi = plane(shape, H, 0.5)
    phit = oracle.step(phi, H, H / 2, Fc=0.5)
    X = oracle.features(phi, phit, H, Fc=0.5)
    assert X.shape == shape + (3,)
    cells = (np.arange(64) + 0.5) - 32.0                       # phi / h along x
    assert np.array_equal(X[0, 0, :, 0], np.clip(cells, -8.0, 8.0))
    assert np.all(X[..., 1] == 0.5)
    assert np.all(X[..., 2] == -0.25)


def test_feature_clamp_is_inclusive_at_eight_cells():
    phi = np.array([-9.0, -8.0, -7.5, 0.0, 7.5, 8.0, 1e9]).reshape(1, 1, 7) * H
    X = oracle.features(phi, phi, H, F=np.zeros_like(phi))
    assert np.array_equal(X[0, 0, :, 0], [-8.0, -8.0, -7.5, 0.0, 7.5, 8.0, 8.0])
    assert np.all(X[..., 2] == 0.0)


def test_features_take_the_speed_field_pointwise():
    g = np.random.default_rng(1)
    phi = g.normal(size=(4, 5, 6)) * H
    F = g.normal(size=(4, 5, 6))
    X = oracle.features(phi, phi + 2 * H, H, F=F)
    assert np.array_equal(X[..., 1], F)
    assert np.allclose(X[..., 2], 2.0, rtol=0, atol=1e-12)


# ------------------------------------------------- correction and the check

def test_correction_is_h_z_on_active_tiles_only():
    active = np.zeros((2, 2, 2), dtype=np.uint8)
    active[0, 1, 0] = active[1, 1, 1] = 1
    z = np.full((16, 16, 16), 3.0)
    c = oracle.correction(z, H, active)
    assert np.count_nonzero(c) == 2 * 512
    assert np.all(c[0:8, 8:16, 0:8] == 3.0 * H) and np.all(c[8:16, 8:16, 8:16] == 3.0 * H)
    assert np.all(c[0:8, 0:8, 0:8] == 0.0)


def test_residual_check_boundary_is_exact():
    """Accept at exactly dt*M, reject one ulp above, either sign."""
    active = np.ones((1, 1, 1), dtype=np.uint8)
    dt, M = H / 2, 1.5
    bound = dt * M
    c = np.zeros((8, 8, 8))
    c[3, 4, 5] = bound
    assert not oracle.residual_check(c, active, dt, M)
    c[3, 4, 5] = -bound
    assert not oracle.residual_check(c, active, dt, M)
    c[3, 4, 5] = np.nextafter(bound, np.inf)
    assert oracle.residual_check(c, active, dt, M)
    c[3, 4, 5] = -np.nextafter(bound, np.inf)
    assert oracle.residual_check(c, active, dt, M)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_residual_check_rejects_non_finite_values(bad):
    active = np.ones((1, 1, 1), dtype=np.uint8)
    c = np.zeros((8, 8, 8))
    c[0, 0, 0] = bad
    assert oracle.residual_check(c, active, 1.0, 1.0)


def test_residual_check_ignores_points_outside_the_band():
    active = np.zeros((1, 1, 2), dtype=np.uint8)
    active[0, 0, 0] = 1
    c = np.zeros((8, 8, 16))
    c[:, :, 8:] = np.nan                      # the inactive tile
    c[:, :, :8] = 0.25
    assert not oracle.residual_check(c, active, 0.5, 0.5)
    assert not oracle.residual_check(c, np.zeros_like(active), 0.0, 0.0)   # empty band


# ------------------------------------------------------- the corrected step

def zero_net(last_bias=0.0):
    chans = [3, 16, 16, 16, 1]
    ps = [(np.zeros((27, chans[k], chans[k + 1])), np.zeros(chans[k + 1])) for k in range(4)]
    ps[-1][1][0] = last_bias
    return ps


def sphere(n):
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.25


def test_zero_network_gives_the_plain_step_exactly():
    phi = sphere(32)
    active = oracle.dilate(oracle.classify(phi, 4.0 / 32))
    out, phit, z, rej = oracle.learned_step(phi, 1.0 / 32, 0.5 / 32, active, zero_net(), Fc=1.0)
    assert not rej and np.all(z == 0.0)
    assert np.array_equal(out, oracle.step(phi, 1.0 / 32, 0.5 / 32, Fc=1.0, tile_active=active))
    assert np.array_equal(out, phit)


@pytest.mark.parametrize("b,rejected", [(0.25, False), (0.5, False), (0.75, True), (-0.75, True)])
def test_constant_correction_and_plain_fallback(b, rejected):
    """A network whose last layer has zero weights and bias b outputs z = b
    everywhere: the correction is h b on the band, accepted up to one plain
    step's motion dt * M = h/2 (F = 1, dt = h/2), else the step is plain."""
    h = 1.0 / 32
    phi = sphere(32)
    active = oracle.dilate(oracle.classify(phi, 4 * h))
    out, phit, z, rej = oracle.learned_step(phi, h, h / 2, active, zero_net(b), Fc=1.0)
    assert rej == rejected and np.all(z == b)
    pts = oracle.tile_points(active)
    if rejected:
        assert np.array_equal(out, phit)
    else:
        assert np.array_equal(out[pts], phit[pts] + b * h)
        assert np.array_equal(out[~pts], phi[~pts])


# ---------------------------------------------------------------- the loss

def test_mse_loss_closed_form_and_mask():
    """z - t = r on every point of the tube gives loss r^2 and gradient
    2 r / |T| there; points outside the tube get no gradient."""
    g = np.random.default_rng(2)
    phi = g.uniform(-1, 1, size=(6, 7, 8))
    phit = g.normal(size=phi.shape)
    ref = g.normal(size=phi.shape)
    h, gamma, r = 0.125, 0.5, 0.375
    phi[0, 0, :2] = (gamma, -gamma)           # on the tube's edge: outside (Eq. 6 is strict)
    t = (ref - phit) / h
    loss, dz, n = oracle.mse_loss_grad(t + r, phi, phit, ref, h, gamma)
    mask = np.abs(phi) < gamma
    assert n == np.count_nonzero(mask) > 0
    assert abs(loss - r * r) <= 1e-14
    assert np.allclose(dz[mask], 2 * r / n, rtol=1e-13, atol=0)
    assert np.all(dz[~mask] == 0.0)
    loss0, dz0, n0 = oracle.mse_loss_grad(t + r, phi + 10.0, phit, ref, h, gamma)   # empty tube
    assert (loss0, n0) == (0.0, 0) and np.all(dz0 == 0.0)


def test_mse_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    phi = g.uniform(-1, 1, size=(4, 5, 6))
    phit, ref, z = (g.normal(size=phi.shape) for _ in range(3))
    _, dz, _ = oracle.mse_loss_grad(z, phi, phit, ref, 0.25, 0.6)
    eps = 1e-6
    for _ in range(10):
        i = tuple(int(g.integers(s)) for s in phi.shape)
        zp, zm = z.copy(), z.copy()
        zp[i] += eps
        zm[i] -= eps
        fd = (oracle.mse_loss_grad(zp, phi, phit, ref, 0.25, 0.6)[0] -
              oracle.mse_loss_grad(zm, phi, phit, ref, 0.25, 0.6)[0]) / (2 * eps)
        assert abs(fd - dz[i]) <= 1e-7 * max(1.0, abs(fd))


# ------------------------------------------------------------------- Adam

def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias corrections undo the moment decay
    exactly (m^ = g, v^ = g^2), so every step moves w by -lr g / (|g| + eps)."""
    g = np.array([2.0, -0.5, 1e-3, 0.0])
    w = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr = 1e-2
    for t in range(1, 6):
        w, m, v = oracle.adam_step(w, g, m, v, t, lr)
    step = g / (np.abs(g) + oracle.ADAM_EPS)
    assert np.allclose(w, 1.0 - 5 * lr * step, rtol=0, atol=1e-13)
    assert w[3] == 1.0


def test_adam_second_step_closed_form():
    """g1 = 1, g2 = -1: m2 = 0.9*0.1 - 0.1 = -0.01, v2 = 0.999*0.001 + 0.001,
    m^ = -0.01 / (1 - 0.81) = -1/19, v^ = v2 / (1 - 0.998001) = 1."""
    lr = 0.1
    w, m, v = oracle.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, lr)
    assert abs(w[0] + lr / (1 + oracle.ADAM_EPS)) <= 1e-15
    w2, m2, v2 = oracle.adam_step(w, -np.ones(1), m, v, 2, lr)
    assert abs(m2[0] + 0.01) <= 1e-17 and abs(v2[0] - 0.001999) <= 1e-17
    assert abs(w2[0] - (w[0] + lr * (1.0 / 19.0) / (1.0 + oracle.ADAM_EPS))) <= 1e-14


# ---------------------------------------------------- one training iteration

def test_training_iteration_gradient_matches_finite_differences():
    """The flat gradient of one training iteration (plain step, features,
    network, masked MSE, backward) against central differences of the whole
    loss in the parameters, and the returned parameters are Adam's step on it."""
    g = np.random.default_rng(4)
    shape, h = (6, 6, 8), 1.0 / 8
    c = (np.arange(8) + 0.5) * h
    phi = (np.sqrt((c[None, None, :] - 0.5) ** 2 + ((np.arange(6)[None, :, None] + 0.5) * h - 0.4) ** 2 +
                   ((np.arange(6)[:, None, None] + 0.5) * h - 0.35) ** 2) - 0.25)
    F = 0.5 + 0.25 * g.uniform(-1, 1, size=shape)
    ref = phi - 0.4 * h + 0.05 * h * g.normal(size=shape)
    chans = [3, 16, 16, 16, 1]
    flat = oracle.pack_params([(g.normal(size=(27, chans[k], chans[k + 1])) * 0.2,
                                g.normal(size=chans[k + 1]) * 0.05) for k in range(4)])
    dt, gamma = 0.5 * h, 3 * h
    zeros = np.zeros_like(flat)
    w1, m1, v1, loss, gflat = oracle.train_iteration(phi, ref, F, h, dt, gamma, flat, zeros, zeros, 1, 1e-3)

    def loss_of(p):
        return oracle.train_iteration(phi, ref, F, h, dt, gamma, p, zeros, zeros, 1, 1e-3)[3]

    assert abs(loss_of(flat) - loss) == 0.0
    eps = 1e-6
    sizes = [27 * chans[k] * chans[k + 1] + chans[k + 1] for k in range(4)]
    starts = np.cumsum([0] + sizes)
    for k in range(4):
        for i in g.choice(sizes[k], 4, replace=False):
            j = int(starts[k] + i)
            pp, pm = flat.copy(), flat.copy()
            pp[j] += eps
            pm[j] -= eps
            fd = (loss_of(pp) - loss_of(pm)) / (2 * eps)
            assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, gflat[j])
    w_ref, _, _ = oracle.adam_step(flat, gflat, zeros, zeros, 1, 1e-3)
    assert np.array_equal(w1, w_ref)
