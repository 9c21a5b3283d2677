"""The slab split on one GPU: several slab contexts of the library on the
same device, exchanging their boundary planes and ghost rows through the
same code path that moves them between GPUs (here device copies), the
common dt from the all-reduced M, and Eq. 14 re-partitions that migrate
rows between slabs.  Bars: bitwise equal to one unsplit context in FP32 and
FP64 (same per-point arithmetic, same band, same dt), and FP64 bitwise equal
to the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls
from paper_1612_04040_b300 import slab

pytestmark = pytest.mark.gpu

SHAPE = (96, 48, 48)
H = 1.0 / 48
HW = 4.0
NSTEPS = 30


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def fields(dtype):
    Z = SHAPE[0] * H
    phi = inputs.sphere_union_sdf(SHAPE, H, [(0.5, 0.5, 0.25 * Z), (0.35, 0.6, 0.8 * Z), (0.7, 0.3, 0.7 * Z)],
                                  [0.18, 0.1, 0.08]).numpy().astype(dtype)
    z = (np.arange(SHAPE[0]) + 0.5) * H
    F = np.broadcast_to((1.0 - 1.6 * z / Z)[:, None, None], SHAPE).astype(dtype)
    return phi, np.ascontiguousarray(F)


def unsplit(phi, F, prec, mode=ls.LS_REBUILD_AUTO):
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, prec)
    g.set_rebuild_mode(mode)
    g.set_phi(phi)
    g.set_speed(F)
    g.band_rebuild(HW)
    dt = g.step(NSTEPS, 0.5, ls.LS_DT_CFL, 5, want_dt=True)
    out = g.get_phi()
    g.close()
    return out, dt


def split(phi, F, prec, nparts, mode=ls.LS_REBUILD_AUTO):
    dphi, dF = torch.from_numpy(phi).cuda(), torch.from_numpy(F).cuda()

    def make(nx, ny, rows, h, lo, hi):
        part = slab.GpuSlab(nx, ny, rows, h, lo, hi, prec)
        part.ctx.set_rebuild_mode(mode)
        return part

    run = slab.SlabRun(slab.LocalComm(nparts), make, SHAPE, H, HW, lambda z0, z1: (dphi[z0:z1], dF[z0:z1]))
    first = run.migrations
    run.step(NSTEPS, 0.5, 5)
    got = np.full_like(phi, np.nan)
    for p, (z0, planes) in run.gather_phi().items():
        got[z0:z0 + planes.shape[0]] = planes.cpu().numpy()
    out = (got, run.dt, run.migrations - first, list(run.bounds))
    run.close()
    return out


@pytest.mark.parametrize("nparts", [2, 3, 6])
@pytest.mark.parametrize("prec", [ls.LS_FP32, ls.LS_FP64])
def test_split_equals_unsplit_bitwise(prec, nparts):
    dt_np = np.float32 if prec == ls.LS_FP32 else np.float64
    phi, F = fields(dt_np)
    ref, ref_dt = unsplit(phi, F, prec)
    got, dt, moved, bounds = split(phi, F, prec, nparts)
    assert dt == ref_dt
    assert np.array_equal(got.view(np.int32 if prec == ls.LS_FP32 else np.int64),
                          ref.view(np.int32 if prec == ls.LS_FP32 else np.int64))
    if nparts >= 3:
        assert moved >= 1, bounds


def test_split_with_incremental_rebuild_mode_equals_unsplit_bitwise():
    """Slab contexts hold ghost rows, so their rebuilds walk every tile even
    with the incremental rebuild asked for; the split run still equals one
    grid whose periodic rebuilds are incremental."""
    phi, F = fields(np.float32)
    ref, ref_dt = unsplit(phi, F, ls.LS_FP32, ls.LS_REBUILD_INCREMENTAL)
    got, dt, _, _ = split(phi, F, ls.LS_FP32, 2, ls.LS_REBUILD_INCREMENTAL)
    assert dt == ref_dt
    assert np.array_equal(got.view(np.int32), ref.view(np.int32))


def split_device(phi, F, prec, nparts, graphs):
    dphi, dF = torch.from_numpy(phi).cuda(), torch.from_numpy(F).cuda()
    stream = torch.cuda.Stream()

    def make(nx, ny, rows, h, lo, hi):
        return slab.GpuSlab(nx, ny, rows, h, lo, hi, prec, stream.cuda_stream)

    run = slab.DeviceSlabRun(slab.LocalComm(nparts), make, SHAPE, H, HW,
                             lambda z0, z1: (dphi[z0:z1], dF[z0:z1]), rebalance=True,
                             rebalance_gain=0.0, rebalance_every=2, graphs=graphs, stream=stream)
    first = run.migrations
    run.step(NSTEPS, 0.5, 5)
    torch.cuda.synchronize()
    got = np.full_like(phi, np.nan)
    for p, (z0, planes) in run.gather_phi().items():
        got[z0:z0 + planes.shape[0]] = planes.cpu().numpy()
    moved = run.migrations - first
    updates = run.updates_done
    run.close()
    return got, moved, updates


@pytest.mark.parametrize("graphs", [False, True], ids=["eager", "graphs"])
@pytest.mark.parametrize("nparts", [1, 3])
@pytest.mark.parametrize("prec", [ls.LS_FP32, ls.LS_FP64])
def test_device_dt_split_equals_unsplit_bitwise(prec, nparts, graphs):
    """The dt made on the device from the max-reduced bounds, the steps in
    LS_DT_KEEP mode, two periods at a time replayed from a CUDA graph:
    still the unsplit run bit for bit (rows migrating between slabs every
    second period at most)."""
    dt_np = np.float32 if prec == ls.LS_FP32 else np.float64
    phi, F = fields(dt_np)
    ref, _ = unsplit(phi, F, prec)
    got, moved, updates = split_device(phi, F, prec, nparts, graphs)
    view = np.int32 if prec == ls.LS_FP32 else np.int64
    assert np.array_equal(got.view(view), ref.view(view))
    assert updates > 0


def test_split_fp64_equals_oracle_bitwise():
    phi, F = fields(np.float64)
    got, dt, _, _ = split(phi, F, ls.LS_FP64, 3)
    o = oracle.Oracle(SHAPE, H)
    o.set_phi(phi)
    o.set_speed(F)
    o.band_rebuild(HW)
    o.step(NSTEPS, 0.5, oracle.DT_CFL, 5)
    assert dt == o.last_dt
    assert np.array_equal(got, o.phi)


def test_ghost_row_calls_refuse_owned_rows():
    g = ls.LevelSet(16, 16, 32, 1.0 / 16, ls.LS_FP32)
    g.set_phi(np.zeros((32, 16, 16), dtype=np.float32) + 1.0)
    buf = torch.zeros(4 * 64, device="cuda")
    with pytest.raises(ls.LSError):
        g.set_tile_rows(0, 1, 0, buf)                  # no ghost rows declared
    g.set_ghost_rows(1, 0)
    g.set_tile_rows(0, 1, 0, buf)                      # the bottom ghost row takes it
    with pytest.raises(ls.LSError):
        g.set_tile_rows(3, 1, 0, buf)                  # the top row is owned
    with pytest.raises(ls.LSError):
        g.set_ghost_rows(2, 0)
    g.close()


def test_keep_mode_and_slab_calls_refuse_misuse():
    """LS_DT_KEEP needs a band and leaves every rebuild to the caller; the
    ghost-row copy needs matching contexts and a ghost row to write."""
    phi, F = fields(np.float32)
    nz, ny, nx = SHAPE
    g = ls.LevelSet(nx, ny, nz, H, ls.LS_FP32)
    g.set_phi(phi)
    g.set_speed(F)
    with pytest.raises(ls.LSError) as e:                 # no band yet
        g.step(1, 1.0, ls.LS_DT_KEEP, 5)
    assert e.value.status == ls.LS_ESTATE
    g.band_rebuild(HW)
    g.step(5, 1.0, ls.LS_DT_KEEP, 5)                     # one whole period: fine
    with pytest.raises(ls.LSError) as e:                 # the next step would need a rebuild
        g.step(1, 1.0, ls.LS_DT_KEEP, 5)
    assert e.value.status == ls.LS_ESTATE
    M = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.band_refresh_async()
    g.band_speed_bound(M)
    Mh = np.zeros(1)
    g.band_speed_bound(Mh)
    assert float(M.item()) == Mh[0] > 0.0
    h2 = ls.LevelSet(nx, ny, 2 * 8, H, ls.LS_FP32)
    h2.set_phi(np.ones((16, ny, nx), dtype=np.float32))
    with pytest.raises(ls.LSError):                      # no ghost rows declared
        h2.copy_ghost_row(g, 3, 0, 0)
    h2.set_ghost_rows(1, 0)
    h2.copy_ghost_row(g, 3, 0, 7)                        # the bottom ghost row takes it
    with pytest.raises(ls.LSError):                      # the top row is owned
        h2.copy_ghost_row(g, 3, 1, 7)
    h3 = ls.LevelSet(nx, 2 * ny, 16, H, ls.LS_FP32)
    h3.set_phi(np.ones((16, 2 * ny, nx), dtype=np.float32))
    h3.set_ghost_rows(1, 0)
    with pytest.raises(ls.LSError):                      # other tile rows
        h3.copy_ghost_row(g, 3, 0, 7)
    for c in (g, h2, h3):
        c.close()
