"""The corrector end to end on a reduced grid: pairs from fine plain runs,
training on the GPU with the library's own forward / backward kernels, and
what the trained network gains over the plain coarse method against the
restricted fine run (the reference for its error)."""
import numpy as np
import pytest
import torch

from paper_1612_04040_b300 import corrector
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu

CS = (32, 32, 128)   # coarse (nz, ny, nx); the fine grid is 4x finer
H_C = 1.0 / 128


@pytest.fixture(scope="module")
def trained(cuda_ok):
    ls.load()
    gen = corrector.PairGenerator(CS, H_C)
    ctx = ls.LevelSet(CS[2], CS[1], CS[0], H_C, ls.LS_FP32)
    ctx.learned_init(seed=1)
    rng = np.random.default_rng(123)
    for _ in range(8):
        c, r, m = corrector.random_problem(rng, gen.box())
        for a, b, F in gen.run(c, r, m, 24):
            ctx.learned_add_pair(a, b, F)
    losses = [ctx.learned_train(1, 1e-3, gen.dt_c, 6.0, seed=s) for s in range(8)]
    final = ctx.learned_train(800, 1e-3, gen.dt_c, 6.0, seed=11)
    after = [ctx.learned_train(1, 1e-12, gen.dt_c, 6.0, seed=s) for s in range(8)]
    return gen, ctx, float(np.mean(losses)), float(np.mean(after)), final


def test_training_lowers_the_loss(trained):
    _, _, before, after, final = trained
    assert np.isfinite(final)
    assert after < 0.7 * before, (before, after)


def test_learned_corrector_gains_over_plain(trained):
    gen, ctx, _, _, _ = trained
    c, r, m = corrector.random_problem(np.random.default_rng(999), gen.box())
    pairs = gen.run(c, r, m, 16)
    phi0, F_c, ref = pairs[0][0], pairs[0][2], pairs[-1][1]
    plain = corrector.coarse_run(ctx, phi0, F_c, 16, gen.dt_c, 6.0, learned=False)
    learned = corrector.coarse_run(ctx, phi0, F_c, 16, gen.dt_c, 6.0, learned=True)
    ep = corrector.front_error(plain, ref, H_C)
    el = corrector.front_error(learned, ref, H_C)
    print("front error (max, mean) in h_c: plain", ep, "learned", el,
          "fallbacks", ctx.learned_fallbacks())
    assert el[1] < ep[1], (ep, el)
    assert ctx.learned_fallbacks() <= 2


def test_untrained_corrector_is_close_to_plain(cuda_ok):
    """A freshly initialised corrector (last layer scaled near zero) changes
    the plain step by far less than a cell, and never trips the check."""
    ls.load()
    gen = corrector.PairGenerator(CS, H_C)
    ctx = ls.LevelSet(CS[2], CS[1], CS[0], H_C, ls.LS_FP32)
    ctx.learned_init(seed=5)
    c, r, m = corrector.random_problem(np.random.default_rng(7), gen.box())
    pairs = gen.run(c, r, m, 2)
    phi0, F_c = pairs[0][0], pairs[0][2]
    plain = corrector.coarse_run(ctx, phi0, F_c, 4, gen.dt_c, 6.0, learned=False)
    learned = corrector.coarse_run(ctx, phi0, F_c, 4, gen.dt_c, 6.0, learned=True)
    assert float((plain - learned).abs().max()) < 0.5 * H_C
    assert ctx.learned_fallbacks() == 0
