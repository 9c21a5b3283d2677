"""Batched contexts (many independent grids, one stencil launch per step),
CUDA-graph replay and the autotuner, against the FP64 CPU oracle run on each
instance separately."""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


def tile_mask(active, shape):
    return np.repeat(np.repeat(np.repeat(active.astype(bool), 8, 0), 8, 1), 8, 2)[
        :shape[0], :shape[1], :shape[2]]


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def small_batch(count=7, seed=5):
    """Seeded instances of the batch recipe, with small grid edges."""
    return inputs.batch_instances(count=count, seed=seed, edges=(32, 40, 48, 56, 64))


def make_batch(insts, graphs=False):
    b = ls.Batch([i.edge for i in insts], [i.h for i in insts])
    phis = []
    for k, it in enumerate(insts):
        p = it.phi().numpy().astype(np.float32)
        phis.append(p)
        b.set_phi_i(k, torch.from_numpy(p).cuda() if k % 2 else p)
        b.set_speed_const_i(k, it.speed)
    b.set_graphs(graphs)
    return b, phis


@pytest.mark.parametrize("mode", [ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL])
def test_batch_matches_per_instance_oracle(mode):
    insts = small_batch()
    b, phis = make_batch(insts)
    b.set_rebuild_mode(mode)
    b.band_rebuild(4.0)
    oracles = []
    for it, p in zip(insts, phis):
        o = oracle.Oracle(p.shape, it.h)
        o.set_phi(p.astype(np.float64))
        o.set_speed_const(float(np.float64(it.speed)))
        o.band_rebuild(4.0)
        oracles.append(o)
    nsteps = 0
    for chunk in (5, 5, 5, 5):
        b.step(chunk, 0.5, ls.LS_DT_CFL, 5)
        nsteps += chunk
        for k, (it, o) in enumerate(zip(insts, oracles)):
            do = o.step(chunk, 0.5, oracle.DT_CFL, 5)
            assert b.last_dt_i(k) == do
            assert np.array_equal(b.active_tiles_i(k), o.active_tiles()), k
    for k, (it, o) in enumerate(zip(insts, oracles)):
        out = b.get_phi_i(k).astype(np.float64)
        m = tile_mask(o.active, o.shape)
        if m.any():
            assert np.max(np.abs(out[m] - o.phi[m])) <= 1e-5 * it.h * nsteps, k


@pytest.mark.parametrize("ppt", [4, 16])
def test_batch_step_configs_agree(ppt):
    """The batched stencil with 4 or 16 points per thread computes the bits
    of the 8-point one (constant speeds of both signs, instances whose bands
    touch the domain faces, the tube test before each rebuild)."""
    insts = small_batch(count=6, seed=11)
    outs = []
    for p in (8, ppt):
        b, _ = make_batch(insts)
        b.set_step_config(3, 100, p)
        b.band_rebuild(4.0)
        b.step(12, 0.5, ls.LS_DT_CFL, 5)
        outs.append([b.get_phi_i(k) for k in range(len(insts))])
        outs[-1].append([b.active_tiles_i(k) for k in range(len(insts))])
        b.close()
    for a, c in zip(outs[0][:-1], outs[1][:-1]):
        assert np.array_equal(a, c)
    for a, c in zip(outs[0][-1], outs[1][-1]):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("stages,pct", [(2, 100), (4, 50), (6, 100)])
def test_batch_one_warp_rings_agree(stages, pct):
    """The one-warp batched stencil (bulk-staged tile blocks and z faces, the
    entries' instance data loaded a tile after them) computes the 8-point
    kernel's bits for every ring depth and a partial grid, across rebuilds."""
    insts = small_batch(count=7, seed=13)
    outs = []
    for cfg in ((3, 100, 8), (stages, pct, 16)):
        b, _ = make_batch(insts)
        b.set_step_config(*cfg)
        b.band_rebuild(4.0)
        b.step(11, 0.5, ls.LS_DT_CFL, 5)
        outs.append([b.get_phi_i(k) for k in range(len(insts))])
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_batch_incremental_rebuild_equals_full_scan():
    """The periodic rebuilds of the full-size batch (256 grids of
    32^3..192^3, 1.12 M tiles) marked from the previous list's core entries
    give, over 40 steps (seven such rebuilds), the lists, dt and bits of
    rebuilds that walk every tile (the leaving tiles' copies into the other
    buffer included)."""
    dev = torch.device("cuda")
    insts = inputs.batch_instances()
    runs = []
    for mode in (ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL):
        b = ls.Batch([i.edge for i in insts], [i.h for i in insts])
        b.set_rebuild_mode(mode)
        for k, it in enumerate(insts):
            b.set_phi_i(k, it.phi(device=dev).to(torch.float32).contiguous())
            b.set_speed_const_i(k, it.speed)
        b.band_rebuild(4.0)
        b.step(40, 0.5, ls.LS_DT_CFL, 5)
        b.step(1, 0.5, ls.LS_DT_CFL, 5)    # one more rebuild, then a step
        runs.append(([b.active_tiles_i(k) for k in range(len(insts))],
                     [b.last_dt_i(k) for k in range(len(insts))],
                     [torch.from_numpy(b.get_phi_i(k)) for k in range(len(insts))]))
        b.close()
    (la, da, pa), (lb, db, pb) = runs
    assert sum(len(x) for x in la) > 100000
    for k in range(len(insts)):
        assert np.array_equal(la[k], lb[k]), k
        assert da[k] == db[k], k
        assert torch.equal(pa[k], pb[k]), k


@pytest.mark.parametrize("F", [0.7, -0.9])
def test_single_grid_constant_speed_one_warp_agrees(F):
    """Single grid, constant speed (the one-warp kernel's variant without
    speed loads): every ring depth gives the 8-point kernel's bits, the
    frozen x-face copies included."""
    w = inputs.SphereUnion(n=48, count=4)
    p = w.phi().numpy().astype(np.float32)
    ref = None
    for cfg in ((3, 100, 8), (2, 100, 16), (4, 75, 16), (6, 50, 16)):
        g = ls.LevelSet(48, 48, 48, w.h, ls.LS_FP32)
        g.set_phi(p)
        g.set_speed_const(F)
        g.set_step_config(*cfg)
        g.band_rebuild(4.0)
        g.step(12, 0.5, ls.LS_DT_CFL, 5)
        out = g.get_phi()
        g.close()
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out, ref), cfg


@pytest.mark.parametrize("mode", [ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL])
def test_batch_graph_replay_equals_eager(mode):
    insts = small_batch(count=5, seed=9)
    outs = []
    for graphs in (False, True):
        b, _ = make_batch(insts, graphs=graphs)
        b.set_rebuild_mode(mode)
        b.band_rebuild(4.0)
        for _ in range(3):
            b.step(7, 0.5, ls.LS_DT_CFL, 5)   # the same call three times: replayed
        outs.append([b.get_phi_i(k) for k in range(len(insts))])
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_single_grid_graph_and_autotune_bitwise():
    """Graph replay (with either rebuild) and every autotuner configuration
    compute the same bits."""
    w = inputs.SphereUnion(n=64, count=5)
    p = w.phi().numpy().astype(np.float32)
    F = w.speed().numpy().astype(np.float32)
    outs = []
    for mode in ("eager", "graph", "tuned", "graph-incremental"):
        g = ls.LevelSet(64, 64, 64, w.h, ls.LS_FP32)
        g.set_phi(p)
        g.set_speed(F)
        if mode == "graph-incremental":
            g.set_rebuild_mode(ls.LS_REBUILD_INCREMENTAL)
        g.band_rebuild(6.0)
        if mode.startswith("graph"):
            g.set_graphs(True)
        if mode == "tuned":
            g.step(1, 0.5, ls.LS_DT_CFL, 5)
            st, pct, ppt = g.autotune(reps=2)
            assert st in (2, 3, 4, 6) and pct in (50, 75, 100) and ppt in (4, 8, 16)
            g.step(11, 0.5, ls.LS_DT_CFL, 5)
        else:
            g.step(1, 0.5, ls.LS_DT_CFL, 5)
            for _ in range(2):
                g.step(3, 0.5, ls.LS_DT_CFL, 5)
            g.step(5, 0.5, ls.LS_DT_CFL, 5)
        outs.append(g.get_phi())
        g.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[0], outs[3])


@pytest.mark.parametrize("stages,pct,ppt", [(2, 50, 4), (4, 100, 8), (3, 75, 4), (2, 100, 8), (6, 100, 4), (6, 75, 8),
                                             (2, 100, 16), (3, 50, 16), (4, 75, 16), (6, 100, 16)])
def test_step_configs_agree(stages, pct, ppt):
    """Every launch configuration computes the same bits (both stencil
    decompositions, constant and field speeds)."""
    w = inputs.SphereUnion(n=48, count=4)
    p = w.phi().numpy().astype(np.float32)
    ref = None
    for cfg in ((3, 100, 8), (stages, pct, ppt)):
        g = ls.LevelSet(48, 48, 48, w.h, ls.LS_FP32)
        g.set_phi(p)
        g.set_speed(w.speed().numpy().astype(np.float32) - 1.0)  # sign-changing field
        g.set_step_config(*cfg)
        g.band_rebuild(4.0)
        g.step(10, 0.5, ls.LS_DT_CFL, 5)
        out = g.get_phi()
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out, ref)


def test_batch_full_domain_matches_oracle():
    insts = small_batch(count=3, seed=21)
    b, phis = make_batch(insts)
    b.set_full_domain(True)
    b.step(6, 0.45, ls.LS_DT_CFL, 0)
    for k, (it, p) in enumerate(zip(insts, phis)):
        o = oracle.Oracle(p.shape, it.h)
        o.set_phi(p.astype(np.float64))
        o.set_speed_const(it.speed)
        o.set_full_domain(True)
        o.step(6, 0.45, oracle.DT_CFL)
        assert np.max(np.abs(b.get_phi_i(k) - o.phi)) <= 1e-5 * it.h * 6


def test_batch_rejects_mixed_speeds_and_fp64():
    with pytest.raises(ls.LSError):
        ls.Batch([16, 16], [1 / 16, 1 / 16], precision=ls.LS_FP64)
    b = ls.Batch([16, 24], [1 / 16, 1 / 24])
    b.set_phi_i(0, np.ones((16, 16, 16), np.float32))
    b.set_phi_i(1, np.ones((24, 24, 24), np.float32))
    b.set_speed_const_i(0, 1.0)
    b.set_speed_i(1, np.ones((24, 24, 24), np.float32))
    b.band_rebuild(2.0)
    with pytest.raises(ls.LSError) as e:
        b.step(1, 0.5, ls.LS_DT_CFL, 5)
    assert e.value.status == ls.LS_ESTATE


def test_snapshot_restore_resumes_exactly():
    """Checkpoint / resume: restore + rerun equals the first run bit for bit."""
    insts = small_batch(count=4, seed=33)
    b, _ = make_batch(insts)
    b.snapshot()
    runs = []
    for _ in range(2):
        b.restore()
        b.band_rebuild(4.0)
        b.step(12, 0.5, ls.LS_DT_CFL, 5)
        runs.append([b.get_phi_i(k) for k in range(len(insts))])
    for a, c in zip(*runs):
        assert np.array_equal(a, c)
