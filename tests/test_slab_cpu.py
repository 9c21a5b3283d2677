"""The slab split's host logic on the CPU: the Eq. 14 partition against the
paper's inequality evaluated exactly, its readings for the degenerate cases,
and whole split runs (exchanges, common dt, re-partition after every
rebuild with rows migrating between parts) whose engines are the FP64
oracle: bitwise equal to one unsplit oracle run, with every part in one
process and with two gloo ranks."""
import os
import socket
import sys
from fractions import Fraction

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import slab

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, HERE)
from _slab_oracle import OracleSlab  # noqa: E402


# ------------------------------------------------------------------ Eq. 14

def brute_partition(counts, n):
    """The paper's rule as written: the next row of c > 0 active tiles joins
    the current part iff |S - M/n| > |S + c - M/n| (exact rationals).  For
    an empty row (c = 0) the two sides are equal, and the paper's own
    consequence S < M/n - c/2 = M/n is taken (an empty row stays with a
    part that is still below M/n).  The same readings for the degenerate
    cases (at least one row per part, enough rows left)."""
    M = Fraction(sum(counts))
    t = M / n
    bounds, S = [0], Fraction(0)
    for r, c in enumerate(counts):
        part = len(bounds) - 1
        if part < n - 1 and r > bounds[-1]:
            joins = abs(S - t) > abs(S + c - t) if c > 0 else S < t
            if len(counts) - r == n - 1 - part or not joins:
                bounds.append(r)
                S = Fraction(0)
        S += c
    return bounds + [len(counts)]


def test_partition_equals_the_inequality_of_eq14():
    g = np.random.default_rng(1)
    for trial in range(3000):
        nrows = int(g.integers(1, 40))
        n = int(g.integers(1, nrows + 1))
        kind = trial % 3
        if kind == 0:
            counts = g.integers(0, 50, nrows)
        elif kind == 1:
            counts = g.integers(0, 3, nrows) * g.integers(0, 400, nrows)   # sparse, spiky
        else:
            counts = np.zeros(nrows, dtype=int)
            counts[g.integers(0, nrows)] = int(g.integers(1, 1000))
        b = slab.partition_rows(counts, n)
        assert b == brute_partition([int(c) for c in counts], n)
        assert len(b) == n + 1 and b[0] == 0 and b[-1] == nrows
        assert all(b[i] < b[i + 1] for i in range(n))            # every part holds a row


def test_partition_balances_a_uniform_band():
    assert slab.partition_rows([10] * 12, 4) == [0, 3, 6, 9, 12]
    assert slab.partition_rows([10] * 12, 3) == [0, 4, 8, 12]
    # the rule's tie: S = M/n - c/2 closes the part (strict inequality)
    assert slab.partition_rows([2, 2, 2, 2], 2) == [0, 2, 4]
    assert slab.partition_rows([1, 0, 0, 5, 5, 1], 2) == [0, 4, 6]
    with pytest.raises(ValueError):
        slab.partition_rows([1, 2], 3)


# ------------------------------------------------------------ split runs

SHAPE = (96, 48, 48)          # (nz, ny, nx): 12 tile rows of 36 tiles
H = 1.0 / 48
HW = 4.0
NSTEPS = 30


def fields():
    """Three spheres at different heights; F = 1 - 1.6 z / Z grows the lower
    ones and shrinks the upper ones, so the band's weight moves between tile
    rows and Eq. 14 moves rows between parts during the run."""
    Z = SHAPE[0] * H
    phi = inputs.sphere_union_sdf(SHAPE, H, [(0.5, 0.5, 0.25 * Z), (0.35, 0.6, 0.8 * Z), (0.7, 0.3, 0.7 * Z)],
                                  [0.18, 0.1, 0.08]).numpy()
    z = (np.arange(SHAPE[0]) + 0.5) * H
    F = np.broadcast_to((1.0 - 1.6 * z / Z)[:, None, None], SHAPE).copy()
    return phi, F


def unsplit(phi, F, nsteps, rebuild_every):
    o = oracle.Oracle(SHAPE, H)
    o.set_phi(phi)
    o.set_speed(F)
    o.band_rebuild(HW)
    o.step(nsteps, 0.5, oracle.DT_CFL, rebuild_every)
    return o


def source_of(phi, F):
    return lambda z0, z1: (torch.from_numpy(phi[z0:z1].copy()), torch.from_numpy(F[z0:z1].copy()))


@pytest.mark.parametrize("nparts", [3, 6])
def test_local_split_equals_unsplit_oracle_bitwise(nparts):
    phi, F = fields()
    run = slab.SlabRun(slab.LocalComm(nparts), OracleSlab, SHAPE, H, HW, source_of(phi, F))
    first = run.migrations
    run.step(NSTEPS, 0.5, 5)
    ref = unsplit(phi, F, NSTEPS, 5)
    got = np.empty_like(phi)
    for p, (z0, planes) in run.gather_phi().items():
        got[z0:z0 + planes.shape[0]] = planes.numpy()
    assert np.array_equal(got, ref.phi)
    assert run.dt == ref.last_dt
    assert run.migrations > first                # Eq. 14 moved rows during the run
    counts = run.active_rows()
    best = slab.partition_rows(counts, nparts)
    assert slab.SlabRun._largest(counts, run.bounds) <= slab.SlabRun._largest(counts, best)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import torch.distributed as dist
    from paper_1612_04040_b300 import slab as slab_mod
    from _slab_oracle import OracleSlab as Eng
    dist.init_process_group("gloo", rank=rank, world_size=world)
    phi, F = fields()
    run = slab_mod.SlabRun(slab_mod.DistComm(dist, "cpu"), Eng, SHAPE, H, HW, source_of(phi, F))
    run.step(NSTEPS, 0.5, 5)
    (p, (z0, planes)), = run.gather_phi().items()
    q.put((rank, z0, planes.numpy().copy(), run.dt, run.migrations, list(run.bounds)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_unsplit_oracle_bitwise():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    phi, F = fields()
    ref = unsplit(phi, F, NSTEPS, 5)
    got = np.full_like(phi, np.nan)
    for rank, z0, planes, dt, mig, bounds in res:
        got[z0:z0 + planes.shape[0]] = planes
        assert dt == ref.last_dt and mig >= 1
        assert bounds == res[0][5]
    assert np.array_equal(got, ref.phi)


def test_parts_with_an_empty_band_and_a_single_row():
    """A front only in the top rows: the lower parts hold no active tile (M = 0
    there, the all-reduced M comes from the top), one part is a single tile
    row, and the split is still the unsplit run bit for bit."""
    shape, h = (96, 32, 32), 1.0 / 32
    Z = shape[0] * h
    phi = inputs.sphere_union_sdf(shape, h, [(0.5, 0.5, 0.85 * Z)], [0.12]).numpy()
    F = np.full(shape, 0.75)
    src = lambda z0, z1: (torch.from_numpy(phi[z0:z1].copy()), torch.from_numpy(F[z0:z1].copy()))
    run = slab.SlabRun(slab.LocalComm(5), OracleSlab, shape, h, 3.0, src)
    counts = run.active_rows()
    assert counts[:6].sum() == 0 and counts.sum() > 0
    assert min(run.bounds[i + 1] - run.bounds[i] for i in range(5)) == 1
    run.step(20, 0.5, 5)
    o = oracle.Oracle(shape, h)
    o.set_phi(phi)
    o.set_speed(F)
    o.band_rebuild(3.0)
    o.step(20, 0.5, oracle.DT_CFL, 5)
    got = np.empty_like(phi)
    for p, (z0, planes) in run.gather_phi().items():
        got[z0:z0 + planes.shape[0]] = planes.numpy()
    assert np.array_equal(got, o.phi)
