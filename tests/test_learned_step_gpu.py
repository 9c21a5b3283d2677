"""The corrected coarse step and the training step on the GPU against the
oracle's definitions (the learned corrector is not in the paper): features,
masked MSE gradient and Adam element by element; one whole corrected step
(plain step, features, network with the BF16 weights loaded through
ls_learned_load, residual check, apply) against the oracle's composition; a
correction forced over the bound, which must leave exactly the plain step;
and one training iteration's parameter update.

Bars: BF16 values within one BF16 rounding (2^-8 relative) of the oracle's
value rounded the same way; FP32 reductions within 1e-5 relative; the
network's correction within 5e-2 of its largest magnitude (four BF16
layers); the plain part of a step within the FP32 bar 1e-5 h."""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

CHANS = [3, 16, 16, 16, 1]


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def bf16_bits(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).view(torch.int16).numpy()


def cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def problem(shape, h, seed, count=6):
    """Seeded sphere union and 8-mode Fourier speed (|F| <= 1), FP32."""
    g = inputs.rng(seed)
    nz, ny, nx = shape
    box = np.array([nx, ny, nz]) * h
    k = count
    centres = [tuple(float(v) for v in g.uniform(0.25 * box, 0.75 * box)) for _ in range(k)]
    radii = [float(g.uniform(0.08, 0.2) * box.min()) for _ in range(k)]
    phi = inputs.sphere_union_sdf(shape, h, centres, radii).numpy().astype(np.float32)
    F = inputs.speed_fourier(shape, h, inputs.fourier_modes(g, 8, 2)).numpy().astype(np.float32)
    return phi, F


def random_params(seed, last_scale=0.05, last_bias=0.0):
    r = np.random.default_rng(seed)
    ps = []
    for k in range(4):
        ci, co = CHANS[k], CHANS[k + 1]
        W = r.normal(size=(27, ci, co)) * np.sqrt(2.0 / (27 * ci))
        b = r.normal(size=co) * 0.05
        if k == 3:
            W *= last_scale
            b = np.full(co, last_bias)
        ps.append((bf16_round(W).astype(np.float64), bf16_round(b).astype(np.float64)))
    return ps


# ------------------------------------------------------- element-wise steps

def test_features_match_oracle():
    shape, h = (8, 16, 128), 1.0 / 128
    phi, F = problem(shape, h, 11)
    g = np.random.default_rng(12)
    phit = (phi + h * g.uniform(-0.6, 0.6, size=shape)).astype(np.float32)
    phi[0, 0, :4] = np.array([9.0, -9.0, 8.0, -8.0], dtype=np.float32) * h      # the clamp
    for Fa, Fc in ((F, 0.0), (None, -0.375)):
        X = ls.learned_features(cuda32(phi), cuda32(phit), h, None if Fa is None else cuda32(Fa), Fc)
        torch.cuda.synchronize()
        got = X.float().cpu().numpy()
        ref = bf16_round(oracle.features(phi, phit, h, Fa, Fc))
        assert np.all(got[..., 3:] == 0.0)
        assert np.array_equal(got[..., :2], ref[..., :2])            # phi / h and F: one rounding
        # (phit - phi) / h: FP32 difference, then BF16: within one BF16 step
        assert np.all(np.abs(got[..., 2] - ref[..., 2]) <= np.abs(ref[..., 2]) * 2.0 ** -8 + 1e-30)


def test_loss_gradient_matches_oracle():
    shape, h = (16, 16, 64), 1.0 / 64
    g = np.random.default_rng(13)
    phi = g.uniform(-12 * h, 12 * h, size=shape).astype(np.float32)
    gamma = 6 * h
    phi[0, 0, :2] = (np.float32(gamma), -np.float32(gamma))      # on the edge of the tube: outside
    phit = (phi - 0.4 * h).astype(np.float32)
    ref = (phit + h * g.normal(scale=0.2, size=shape)).astype(np.float32)
    z = g.normal(scale=0.3, size=shape).astype(np.float32)
    dz, count, loss = ls.learned_loss_grad(cuda32(z), cuda32(phi), cuda32(phit), cuda32(ref), h, gamma)
    torch.cuda.synchronize()
    rl, rdz, rn = oracle.mse_loss_grad(z, phi, phit, ref, h, gamma)
    assert int(count.item()) == rn > 0
    assert abs(float(loss.item()) - rl) <= 1e-5 * rl
    got = dz.float().cpu().numpy()
    assert np.all(got[..., 1:] == 0.0)
    assert np.all(np.abs(got[..., 0] - bf16_round(rdz)) <= np.abs(rdz) * 2.0 ** -8 + 1e-30)
    assert np.all(got[..., 0][np.abs(phi) >= gamma] == 0.0)


def test_adam_matches_oracle():
    g = np.random.default_rng(14)
    n = 10000
    w = g.normal(size=n).astype(np.float32)
    dw, dm, dv = cuda32(w), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    rw, rm, rv = w.astype(np.float64), np.zeros(n), np.zeros(n)
    gsum = np.zeros(n)
    for t in range(1, 6):
        grad = (g.normal(size=n) * 10.0 ** g.uniform(-4, 1, size=n)).astype(np.float32)
        ls.adam_step(dw, cuda32(grad), dm, dv, t, 1e-3)
        rw, rm, rv = oracle.adam_step(rw, grad, rm, rv, t, 1e-3)
        gsum += np.abs(grad)
    torch.cuda.synchronize()
    assert np.max(np.abs(dw.cpu().numpy() - rw)) <= 1e-5 * 5e-3 + 1e-6 * np.max(np.abs(rw))
    # m sums gradients of either sign: FP32 rounding is bounded by the terms'
    # magnitudes, not by the (possibly cancelled) result; v sums squares
    assert np.all(np.abs(dm.cpu().numpy() - rm) <= 1e-5 * np.abs(rm) + 2e-6 * gsum)
    assert np.allclose(dv.cpu().numpy(), rv, rtol=1e-5, atol=1e-20)


# ------------------------------------------------- the whole corrected step

SHAPE_STEP = (64, 64, 128)      # 1024 convolution blocks: every CTA runs several
H_STEP = 1.0 / 128


def learned_ctx(phi, F, params_bf16):
    nz, ny, nx = phi.shape
    c = ls.LevelSet(nx, ny, nz, H_STEP, ls.LS_FP32)
    c.learned_load(params_bf16)
    c.set_phi(phi)
    c.set_speed(F)
    return c


def weights_image(params):
    return bf16_bits(oracle.pack_params(params)).view(np.uint16)


def run_steps(c, mode, nsteps, dt, halfwidth):
    c.set_step_mode(mode)
    c.band_rebuild(halfwidth)
    c.step(nsteps, dt, ls.LS_DT_FIXED, 1)
    out = c.get_phi()
    return out


def test_corrected_step_matches_oracle_composition():
    """The network's last layer is scaled by a power of two (exact in BF16)
    so that the largest correction is 1/8 .. 1/4 of the bound dt M: large
    enough to compare, clear of the check's edge on both sides."""
    phi, F = problem(SHAPE_STEP, H_STEP, 21)
    dt, hw = 0.5 * H_STEP, 6.0
    active = oracle.dilate(oracle.classify(phi, hw * H_STEP))
    pts = oracle.tile_points(active)
    M = oracle.max_abs_speed(phi.shape, F, 0.0, active)
    params = random_params(22, last_scale=1.0)
    _, _, z1, _ = oracle.learned_step(phi, H_STEP, dt, active, params, F=F, round_features=bf16_round)
    s = 2.0 ** np.floor(np.log2(0.25 * dt * M / (H_STEP * np.max(np.abs(z1[pts])))))
    params[3] = (params[3][0] * s, params[3][1])
    ref, phit, z, rejected = oracle.learned_step(phi, H_STEP, dt, active, params, F=F,
                                                 round_features=bf16_round)
    assert not rejected
    c = learned_ctx(phi, F, weights_image(params))
    got = run_steps(c, ls.LS_LEARNED, 1, dt, hw)
    assert np.array_equal(oracle.compact(active), c.active_tiles())
    assert c.learned_fallbacks() == 0
    c.set_phi(phi)
    plain = run_steps(c, ls.LS_PLAIN, 1, dt, hw)
    c.close()
    # the plain part and the frozen points
    assert np.max(np.abs(plain[pts] - phit[pts])) <= 1e-5 * H_STEP
    assert np.array_equal(got[~pts], phi[~pts])
    # the correction the GPU applied against the oracle's h z
    corr_gpu = got.astype(np.float64) - plain.astype(np.float64)
    corr_ref = H_STEP * z
    scale = np.max(np.abs(corr_ref[pts]))
    assert 0.1 * dt * M <= scale <= 0.25 * dt * M
    assert np.max(np.abs(corr_gpu[pts] - corr_ref[pts])) <= 5e-2 * scale + 2e-7
    assert np.max(np.abs(got[pts] - ref[pts])) <= 5e-2 * scale + 1e-5 * H_STEP


def test_correction_over_the_bound_falls_back_to_the_plain_step_bitwise():
    """A last-layer bias of 4 cells puts |h z| far above one plain step's
    motion (dt M <= h/2): every step must keep exactly the plain result and
    count one fallback."""
    phi, F = problem(SHAPE_STEP, H_STEP, 23)
    params = random_params(24, last_scale=0.0, last_bias=4.0)
    dt, hw = 0.5 * H_STEP, 6.0
    c = learned_ctx(phi, F, weights_image(params))
    got = run_steps(c, ls.LS_LEARNED, 3, dt, hw)
    assert c.learned_fallbacks() == 3
    c.set_phi(phi)
    plain = run_steps(c, ls.LS_PLAIN, 3, dt, hw)
    c.close()
    assert np.array_equal(got.view(np.int32), plain.view(np.int32))
    # and the oracle agrees that the check rejects it
    active = oracle.dilate(oracle.classify(phi, hw * H_STEP))
    assert oracle.learned_step(phi, H_STEP, dt, active, params, F=F, round_features=bf16_round)[3]


# ------------------------------------------------ one training iteration

def test_training_iteration_update_matches_oracle():
    """One Adam step from zero moments moves each parameter by lr g / (|g| +
    eps), i.e. by about lr against the sign of its gradient: the update's
    sign must equal the oracle's for every parameter whose gradient is not
    small, and the loss must agree."""
    shape, h = (32, 32, 128), 1.0 / 128
    phi, F = problem(shape, h, 31)
    ref = (phi - 0.45 * h + 0.05 * h * np.sin(np.arange(phi.size).reshape(shape) * 0.01)).astype(np.float32)
    params = random_params(32, last_scale=1.0)
    flat = oracle.pack_params(params)
    nz, ny, nx = shape
    c = ls.LevelSet(nx, ny, nz, h, ls.LS_FP32)
    c.learned_load(weights_image(params))
    c.learned_add_pair(cuda32(phi), cuda32(ref), cuda32(F))
    before = c.learned_params().astype(np.float64)
    assert np.array_equal(before, flat)
    lr, dt, hw = 1e-3, 0.5 * h, 6.0
    loss = c.learned_train(1, lr, dt, hw, seed=0)
    after = c.learned_params().astype(np.float64)
    c.close()
    zeros = np.zeros_like(flat)
    w1, _, _, rloss, g = oracle.train_iteration(phi, ref, F, h, dt, hw * h, flat, zeros, zeros, 1, lr,
                                                round_features=bf16_round)
    assert abs(loss - rloss) <= 2e-2 * rloss
    step = after - before
    o = 0
    for k in range(4):
        n = 27 * CHANS[k] * CHANS[k + 1] + CHANS[k + 1]
        gk, sk = g[o:o + n], step[o:o + n]
        big = np.abs(gk) > 0.05 * np.max(np.abs(gk))
        assert np.count_nonzero(big) > 0
        assert np.all(np.sign(sk[big]) == -np.sign(gk[big])), k
        assert np.allclose(np.abs(sk[big]), lr, rtol=1e-3), k
        o += n
    assert np.allclose(w1[np.abs(g) > 0.05 * np.max(np.abs(g))],
                       after[np.abs(g) > 0.05 * np.max(np.abs(g))], rtol=0, atol=1e-5)


def test_corrected_step_with_an_empty_band_leaves_phi_unchanged():
    """No point within the band: no active tile, no convolution block, no
    correction, no fallback, phi unchanged bit for bit."""
    shape = (32, 32, 128)
    nz, ny, nx = shape
    phi = np.full(shape, 0.5, dtype=np.float32)          # |phi| = 64 cells everywhere
    F = np.full(shape, 0.5, dtype=np.float32)
    params = random_params(41, last_scale=1.0, last_bias=2.0)
    c = ls.LevelSet(nx, ny, nz, H_STEP, ls.LS_FP32)
    c.learned_load(weights_image(params))
    c.set_phi(phi)
    c.set_speed(F)
    got = run_steps(c, ls.LS_LEARNED, 3, 0.5 * H_STEP, 6.0)
    assert c.active_tiles().size == 0
    assert c.learned_fallbacks() == 0
    c.close()
    assert np.array_equal(got.view(np.int32), phi.view(np.int32))
