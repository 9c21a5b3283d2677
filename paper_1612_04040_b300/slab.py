"""Slab split of the narrow-band step along z (section 2 of the paper).

The paper decomposes the grid by one axis, each core holding its rows plus
a ghost row from each neighbour, and shares the tube out row by row with a
greedy rule (Eq. 14): a core takes the next row while that brings its count
S of active points closer to M/n, i.e. while S < M/n - c/2 for a next row of
c points.  Here a "row" is a tile row (the 8 z-planes of one layer of 8^3
tiles), its weight the active tiles in it, and a part is a slab of whole
tile rows held by one engine (one GPU, one process, or one of several slabs
on the same GPU).

Per step the parts exchange one z-plane across every boundary (the plane
next to the neighbour's first or last owned row) into the neighbour's ghost
row; before every band rebuild they exchange whole rows, so that each part
can make the tube test of its ghost rows and dilate the band across the
boundary, and all-reduce M = max |F| over the active points for the common
dt.  After a rebuild the rows are shared out again by Eq. 14 and rows that
change owner move between parts.

This module holds the host logic only: the partition, the exchange plan and
the schedule.  The arithmetic runs in the engines (the library's kernels
for ``GpuSlab``); the data moves through a ``comm`` object: ``LocalComm``
(every part in this process) or ``DistComm`` (one part per rank of a
torch.distributed group: NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np
import torch

from . import native as ls

TILE = 8


# --------------------------------------------------------------------------
# Eq. 14
# --------------------------------------------------------------------------

def partition_rows(counts, nparts):
    """Bounds [b_0 = 0, b_1, ..., b_n = len(counts)] of n consecutive row
    ranges.  Rows are taken in order; the current part takes the next row of
    c active tiles while S < M/n - c/2 (Eq. 14, evaluated exactly as
    n (2 S + c) < 2 M), where S is what it holds and M the total.  Readings
    for the cases the rule does not settle: every part takes at least one
    row (a part has a slab to hold), a part stops when the rows left are
    just enough for one each of the parts after it, and the last part takes
    what remains.  For a row with c > 0 the rule is the paper's
    |S - M/n| > |S + c - M/n|; for an empty row (c = 0) both sides are
    equal and the paper's consequence S < M/n is what decides."""
    counts = [int(c) for c in counts]
    nrows = len(counts)
    if nparts < 1 or nrows < nparts:
        raise ValueError("need 1 <= parts <= rows (%d parts, %d rows)" % (nparts, nrows))
    if any(c < 0 for c in counts):
        raise ValueError("row counts must be non-negative")
    M = sum(counts)
    bounds = [0]
    S = 0
    for r, c in enumerate(counts):
        part = len(bounds) - 1
        held = r - bounds[-1]
        if part < nparts - 1 and held > 0:
            rows_left = nrows - r
            must_close = rows_left == nparts - 1 - part
            if must_close or not (nparts * (2 * S + c) < 2 * M):
                bounds.append(r)
                S = 0
        S += c
    bounds.append(nrows)
    return bounds


def even_rows(nrows, nparts):
    """The global decomposition (equal numbers of rows), used before any
    band exists."""
    if nparts < 1 or nrows < nparts:
        raise ValueError("need 1 <= parts <= rows")
    return [(nrows * p) // nparts for p in range(nparts + 1)]


# --------------------------------------------------------------------------
# transports
# --------------------------------------------------------------------------

class LocalComm:
    """Every part lives in this process; moving data is a copy."""

    def __init__(self, nparts):
        self.nparts = int(nparts)
        self.parts = list(range(self.nparts))

    def max(self, values):
        return max(float(v) for v in values.values())

    def sum_arrays(self, arrays):
        return np.sum([np.asarray(a, dtype=np.int64) for a in arrays.values()], axis=0)

    def max_device(self, tensors):
        """Max of the parts' device scalars, as a device scalar (no host
        synchronisation)."""
        ts = list(tensors.values())
        return ts[0] if len(ts) == 1 else torch.amax(torch.cat(ts), dim=0, keepdim=True)

    def transfer(self, moves):
        """moves: (src_part, dst_part, src_buffer, dst_buffer); src_buffer
        is read, dst_buffer written."""
        for _, _, src, dst in moves:
            dst.copy_(src)


class DistComm:
    """Part p lives on rank p of a torch.distributed group (NCCL with CUDA
    buffers, gloo with CPU buffers)."""

    def __init__(self, dist, device):
        self.dist = dist
        self.device = torch.device(device)
        self.nparts = dist.get_world_size()
        self.parts = [dist.get_rank()]

    def max(self, values):
        t = torch.tensor([max(float(v) for v in values.values())], dtype=torch.float64,
                         device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def max_device(self, tensors):
        (t,) = tensors.values()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t

    def sum_arrays(self, arrays):
        a = np.sum([np.asarray(v, dtype=np.int64) for v in arrays.values()], axis=0)
        t = torch.from_numpy(a).to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.cpu().numpy()

    def transfer(self, moves):
        me = self.parts[0]
        ops = []
        for src_part, dst_part, src, dst in moves:
            if src_part == me and dst_part == me:
                dst.copy_(src)
            elif src_part == me:
                ops.append(self.dist.P2POp(self.dist.isend, src, dst_part))
            elif dst_part == me:
                ops.append(self.dist.P2POp(self.dist.irecv, dst, src_part))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()


# --------------------------------------------------------------------------
# the library engine of one slab
# --------------------------------------------------------------------------

class GpuSlab:
    """One slab of tile rows (plus ghost rows) in a library context on the
    current CUDA device, fed from row-major device tensors."""

    def __init__(self, nx, ny, rows, h, lo, hi, precision=ls.LS_FP32, stream=None, step_config=None):
        """step_config: (stages, grid_pct, points_per_thread) of the stencil
        launches, e.g. what ls_autotune picked on the unsplit grid."""
        self.nx, self.ny, self.rows, self.lo, self.hi = nx, ny, rows, int(lo), int(hi)
        self.h = float(h)
        self.dtype = torch.float32 if precision == ls.LS_FP32 else torch.float64
        self.ctx = ls.LevelSet(nx, ny, TILE * rows, h, precision, stream)
        if step_config is not None:
            self.ctx.set_step_config(*step_config)
        self.tiles_per_row = (nx // TILE) * (ny // TILE)

    def close(self):
        self.ctx.close()

    def setup(self, phi, F, halfwidth):
        """phi, F: row-major (8 rows, ny, nx) tensors of the whole slab,
        ghost rows included (their F is not used)."""
        self.ctx.set_phi(phi.contiguous())
        self.ctx.set_speed(F.contiguous())
        self.ctx.set_ghost_rows(self.lo, self.hi)
        self.ctx.band_rebuild(halfwidth, want_count=False)

    def refresh(self):
        return self.ctx.band_refresh()

    def row_counts(self):
        return self.ctx.band_row_counts()

    def step(self, dt, rebuild_every, n=1):
        self.ctx.step(n, dt, ls.LS_DT_FIXED, rebuild_every)

    def buffer(self, plane):
        n = self.tiles_per_row * (512 if plane < 0 else 64)
        return torch.empty(n, dtype=self.dtype, device="cuda")

    def export_row(self, row, plane, out):
        self.ctx.get_tile_rows(row, 1, plane, out)

    def import_row(self, row, plane, src):
        self.ctx.set_tile_rows(row, 1, plane, src)

    def phi(self):
        out = torch.empty((TILE * self.rows, self.ny, self.nx), dtype=self.dtype, device="cuda")
        self.ctx.get_phi(out)
        return out

    def speed(self):
        out = torch.empty((TILE * self.rows, self.ny, self.nx), dtype=self.dtype, device="cuda")
        self.ctx.get_speed(out)
        return out

    def zeros(self, nplanes):
        return torch.zeros((nplanes, self.ny, self.nx), dtype=self.dtype, device="cuda")


# --------------------------------------------------------------------------
# the schedule
# --------------------------------------------------------------------------

class SlabRun:
    """A narrow-band run split into z-slabs.

    make_engine(nx, ny, rows, h, lo, hi) builds the engine of one slab (rows =
    tile rows including the ghost rows lo / hi); source(z0, z1) returns the
    row-major (z1 - z0, ny, nx) planes [z0, z1) of phi and of F (both as
    engine tensors) for the initial state.  The parts start from the even
    row split, rebuild, and are then shared out by Eq. 14; with
    ``rebalance`` they are shared out again after every rebuild, when the
    Eq. 14 partition lowers the largest part's active tiles by more than
    the fraction ``rebalance_gain`` (0: whenever it lowers it).  Moving rows
    gives the moved parts new contexts, so a run on GPUs asks for a gain of
    some per cent before it pays (``bench.py`` uses 10 %)."""

    def __init__(self, comm, make_engine, shape, h, halfwidth, source, rebalance=True,
                 rebalance_gain=0.0):
        self.comm = comm
        self.make_engine = make_engine
        self.nz, self.ny, self.nx = (int(v) for v in shape)
        if self.nz % TILE or self.ny % TILE or self.nx % TILE:
            raise ValueError("grid edges must be multiples of 8")
        self.nrows = self.nz // TILE
        self.h = float(h)
        self.halfwidth = float(halfwidth)
        self.rebalance = bool(rebalance)
        self.rebalance_gain = float(rebalance_gain)
        self.engines = {}
        self.n_active = 0
        self.bounds = even_rows(self.nrows, comm.nparts)
        self.since_rebuild = 0
        self.updates = 0
        self.migrations = 0
        self.dt = None
        self._build({p: self._initial_rows(source, p) for p in comm.parts})
        self._rebuild(first=True)

    # -- layout -------------------------------------------------------------
    def _span(self, p, bounds=None):
        """(owned rows r0..r1, ghost flags lo / hi, first tile row held)"""
        b = self.bounds if bounds is None else bounds
        r0, r1 = b[p], b[p + 1]
        lo = 1 if p > 0 else 0
        hi = 1 if p < self.comm.nparts - 1 else 0
        return r0, r1, lo, hi, r0 - lo

    def _initial_rows(self, source, p):
        r0, r1, lo, hi, first = self._span(p)
        return source(TILE * first, TILE * (r1 + hi))

    def _build(self, fields):
        """New engines for the parts in `fields` (the others keep theirs)."""
        for p in fields:
            if p in self.engines:
                self.engines.pop(p).close()
        for p, (phi, F) in fields.items():
            r0, r1, lo, hi, _ = self._span(p)
            e = self.make_engine(self.nx, self.ny, r1 - r0 + lo + hi, self.h, lo, hi)
            e.setup(phi, F, self.halfwidth)
            self.engines[p] = e

    # -- exchanges ----------------------------------------------------------
    def _exchange(self, plane_up, plane_down):
        """Across every boundary p | p+1: p's last owned row -> p+1's bottom
        ghost row (plane_up of it), p+1's first owned row -> p's top ghost
        row (plane_down); -1 means whole rows."""
        moves, keep = [], []
        for p in range(self.comm.nparts - 1):
            q = p + 1
            for src, dst, plane in ((p, q, plane_up), (q, p, plane_down)):
                s_in = src in self.engines
                d_in = dst in self.engines
                if not (s_in or d_in):
                    continue
                sbuf = dbuf = None
                if s_in:
                    e = self.engines[src]
                    r0, r1, lo, hi, _ = self._span(src)
                    row = lo + (r1 - r0 - 1) if dst > src else lo
                    sbuf = e.buffer(plane)
                    e.export_row(row, plane, sbuf)
                if d_in:
                    e = self.engines[dst]
                    r0, r1, lo, hi, _ = self._span(dst)
                    row = 0 if src < dst else lo + (r1 - r0)
                    # both parts here: the neighbour reads the exported buffer itself
                    dbuf = sbuf if s_in else e.buffer(plane)
                    keep.append((e, row, plane, dbuf))
                if not (s_in and d_in):
                    moves.append((src, dst, sbuf, dbuf))
        self.comm.transfer(moves)
        for e, row, plane, dbuf in keep:
            e.import_row(row, plane, dbuf)

    # -- rebuild, balance and dt ----------------------------------------------
    def _refresh_all(self):
        res = {p: e.refresh() for p, e in self.engines.items()}
        self.n_active = sum(n for _, n in res.values())   # active tiles of this process's parts
        return {p: M for p, (M, _) in res.items()}

    @staticmethod
    def _largest(counts, bounds):
        return max(int(np.sum(counts[bounds[i]:bounds[i + 1]])) for i in range(len(bounds) - 1))

    def _rebuild(self, first=False):
        self._exchange(-1, -1)
        Ms = self._refresh_all()
        if self.rebalance and self.comm.nparts > 1:
            counts = self.row_counts()
            new = partition_rows(counts, self.comm.nparts)
            now, then = self._largest(counts, self.bounds), self._largest(counts, new)
            if new != self.bounds and (first or then < (1.0 - self.rebalance_gain) * now):
                self._migrate(new)
                self._exchange(-1, -1)
                Ms = self._refresh_all()
        M = self.comm.max(Ms)
        self.M = M
        self.since_rebuild = 0

    def row_counts(self):
        """Active tiles per tile row of the whole grid (gathered)."""
        arrays = {}
        for p, e in self.engines.items():
            r0, r1, lo, hi, _ = self._span(p)
            full = np.zeros(self.nrows, dtype=np.int64)
            full[r0:r1] = e.row_counts()[lo:lo + (r1 - r0)]
            arrays[p] = full
        return self.comm.sum_arrays(arrays)

    def _migrate(self, new):
        """Move owned rows to their new parts (Eq. 14 after a rebuild):
        every overlap of an old and a new range goes from its old to its new
        owner; ghost rows are filled by the next exchange."""
        old = self.bounds
        # a part whose rows do not change keeps its engine (and its rows)
        same = {q for q in range(self.comm.nparts) if old[q] == new[q] and old[q + 1] == new[q + 1]}
        held = {}
        for p, e in self.engines.items():
            if p in same:
                continue
            r0, r1, lo, hi, _ = self._span(p)
            held[p] = (e.phi()[TILE * lo:TILE * (lo + r1 - r0)], e.speed()[TILE * lo:TILE * (lo + r1 - r0)])
        # receive buffers of the new slabs (owned planes; ghosts zero for now)
        fresh = {}
        for q in self.comm.parts:
            if q in same:
                continue
            r0, r1, lo, hi, _ = self._span(q, new)
            proto = next(iter(self.engines.values()))
            fresh[q] = (proto.zeros(TILE * (r1 - r0 + lo + hi)), proto.zeros(TILE * (r1 - r0 + lo + hi)))
        moves = []
        for p in range(self.comm.nparts):
            for q in range(self.comm.nparts):
                a = max(old[p], new[q])
                b = min(old[p + 1], new[q + 1])
                if a >= b or p in same or q in same:
                    continue
                if p not in held and q not in fresh:
                    continue
                for k in (0, 1):
                    src = dst = None
                    if p in held:
                        src = held[p][k][TILE * (a - old[p]):TILE * (b - old[p])].contiguous()
                    if q in fresh:
                        lo_q = 1 if q > 0 else 0
                        dst = fresh[q][k][TILE * (lo_q + a - new[q]):TILE * (lo_q + b - new[q])]
                    moves.append((p, q, src, dst))
        # views of the receive buffers may be non-contiguous for P2P: receive
        # into contiguous staging and copy back
        staged = []
        for i, (p, q, src, dst) in enumerate(moves):
            if dst is not None and not dst.is_contiguous():
                tmp = torch.empty_like(dst, memory_format=torch.contiguous_format)
                staged.append((tmp, dst))
                moves[i] = (p, q, src, tmp)
        self.comm.transfer(moves)
        for tmp, dst in staged:
            dst.copy_(tmp)
        self.bounds = list(new)
        self.migrations += 1
        self._build(fresh)

    # -- stepping -------------------------------------------------------------
    def step(self, nsteps, cfl, rebuild_every):
        """nsteps steps at dt = cfl h / M (cfl h when M = 0), M taken over
        the whole band at each rebuild, a rebuild every rebuild_every steps
        (the same schedule and dt as one unsplit context)."""
        k = 0
        while k < nsteps:
            if self.since_rebuild >= rebuild_every:
                self._rebuild()
            ch = cfl * self.h
            self.dt = ch / self.M if self.M > 0.0 else ch
            if self.comm.nparts == 1:
                # nothing to exchange: the rest of the rebuild period in one call
                n = min(nsteps - k, rebuild_every - self.since_rebuild)
                for e in self.engines.values():
                    e.step(self.dt, rebuild_every, n)
            else:
                n = 1
                self._exchange(TILE - 1, 0)
                for e in self.engines.values():
                    e.step(self.dt, rebuild_every)
            self.updates += n * self.n_active * TILE ** 3
            self.since_rebuild += n
            k += n

    def gather_phi(self):
        """Owned planes of the parts in this process: {part: (z0, planes)}."""
        out = {}
        for p, e in self.engines.items():
            r0, r1, lo, hi, _ = self._span(p)
            out[p] = (TILE * r0, e.phi()[TILE * lo:TILE * (lo + r1 - r0)])
        return out

    def active_rows(self):
        return self.row_counts()

    def close(self):
        for e in self.engines.values():
            e.close()
        self.engines = {}


class DeviceSlabRun(SlabRun):
    """The same schedule with the common dt made on the device: after each
    rebuild the slabs' bounds M are max-reduced into a device scalar
    (``comm.max_device``: a device max, or an NCCL all-reduce) and every
    slab sets dt = CFL h / M from it (``ls_set_dt_from_bound``), and the
    steps run with that dt (``LS_DT_KEEP``).  A rebuild period then waits
    for nothing on the host, and with ``graphs`` (every part in this
    process) two periods at a time (an even number of steps, so each
    context's ping-pong and traversal state comes back to where it was) are
    captured in one CUDA graph on ``stream`` and replayed.  The Eq. 14
    re-partition needs the row counts on the host: it is checked every
    ``rebalance_every`` periods.  Library slab engines (``GpuSlab``) only."""

    def __init__(self, comm, make_engine, shape, h, halfwidth, source, rebalance=True,
                 rebalance_gain=0.05, rebalance_every=4, graphs=False, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.graphs = bool(graphs) and isinstance(comm, LocalComm)
        self.rebalance_every = max(int(rebalance_every), 1)
        self._bufs = {}
        self._graph = None
        self._graph_period = None
        self._counted = 0
        self.cfl = None
        with torch.cuda.stream(self.stream):
            super().__init__(comm, make_engine, shape, h, halfwidth, source, rebalance, rebalance_gain)
            self.Mdev = {p: torch.zeros(1, dtype=torch.float64, device="cuda") for p in comm.parts}

    # engines change on migration: keep their update counts, drop buffers
    # and the captured graph
    def _build(self, fields):
        for p in fields:
            if p in getattr(self, "engines", {}):
                self._counted += self.engines[p].ctx.updates()
        self._graph = None
        super()._build(fields)

    def _buffer(self, key, e, plane):
        b = self._bufs.get(key)
        if b is None:
            b = e.buffer(plane)
            self._bufs[key] = b
        return b

    def _exchange(self, plane_up, plane_down):
        moves, keep = [], []
        for p in range(self.comm.nparts - 1):
            q = p + 1
            for src, dst, plane in ((p, q, plane_up), (q, p, plane_down)):
                s_in, d_in = src in self.engines, dst in self.engines
                if not (s_in or d_in):
                    continue
                kind = "row" if plane < 0 else "plane"
                sbuf = dbuf = None
                if s_in and not d_in:
                    e = self.engines[src]
                    r0, r1, lo, hi, _ = self._span(src)
                    row = lo + (r1 - r0 - 1) if dst > src else lo
                    sbuf = self._buffer(("s", src, dst, kind), e, plane)
                    e.export_row(row, plane, sbuf)
                if d_in:
                    e = self.engines[dst]
                    r0, r1, lo, hi, _ = self._span(dst)
                    row = 0 if src < dst else lo + (r1 - r0)
                    if s_in:
                        # both slabs here: straight from the neighbour's rows
                        sr0, sr1, slo, _, _ = self._span(src)
                        srow = slo + (sr1 - sr0 - 1) if dst > src else slo
                        e.ctx.copy_ghost_row(self.engines[src].ctx, srow, row, plane)
                        continue
                    dbuf = self._buffer(("r", src, dst, kind), e, plane)
                    keep.append((e, row, plane, dbuf))
                moves.append((src, dst, sbuf, dbuf))
        self.comm.transfer(moves)
        for e, row, plane, dbuf in keep:
            e.import_row(row, plane, dbuf)

    def _rebuild_device(self):
        self._exchange(-1, -1)
        for p, e in self.engines.items():
            e.ctx.band_refresh_async()
            e.ctx.band_speed_bound(self.Mdev[p])
        M = self.comm.max_device(self.Mdev)
        for e in self.engines.values():
            e.ctx.set_dt_from_bound(M, self.cfl)

    def _period(self, rebuild_every):
        self._rebuild_device()
        for _ in range(rebuild_every):
            self._exchange(TILE - 1, 0)
            for e in self.engines.values():
                e.ctx.step(1, 1.0, ls.LS_DT_KEEP, rebuild_every)

    def _check_balance(self):
        """Eq. 14 on the current band (host: row counts); rows move when
        that lowers the largest part by more than rebalance_gain."""
        if not self.rebalance or self.comm.nparts == 1:
            return
        counts = self.row_counts()
        new = partition_rows(counts, self.comm.nparts)
        now, then = self._largest(counts, self.bounds), self._largest(counts, new)
        if new != self.bounds and then < (1.0 - self.rebalance_gain) * now:
            self._migrate(new)

    def _capture(self, rebuild_every):
        # recording does not run the work, and the contexts' host state
        # moves on by the two periods recorded: the next replay brings the
        # device to the same point
        self._graph = torch.cuda.CUDAGraph()
        self._graph_period = rebuild_every
        with torch.cuda.graph(self._graph, stream=self.stream):
            self._period(rebuild_every)
            self._period(rebuild_every)

    def prepare(self, cfl, rebuild_every):
        """Record the graph of the next two periods now (set-up), so that
        step() starts by replaying it."""
        self.cfl = float(cfl)
        if self.graphs and self._graph is None:
            with torch.cuda.stream(self.stream):
                self._capture(rebuild_every)

    def step(self, nsteps, cfl, rebuild_every):
        """nsteps (a multiple of rebuild_every) steps in whole rebuild periods."""
        if nsteps % rebuild_every:
            raise ValueError("nsteps must be a multiple of rebuild_every here")
        if self._graph is not None and (self._graph_period != rebuild_every or self.cfl != float(cfl)):
            raise ValueError("a graph is recorded for another period or CFL number")
        self.cfl = float(cfl)
        periods = nsteps // rebuild_every
        done = 0
        with torch.cuda.stream(self.stream):
            while done < periods:
                if done and done % self.rebalance_every == 0:
                    self._check_balance()
                if self.graphs and periods - done >= 2:
                    if self._graph is None:
                        self._capture(rebuild_every)
                    self._graph.replay()
                    done += 2
                else:
                    self._period(rebuild_every)
                    done += 1
        self.since_rebuild = rebuild_every

    @property
    def updates_done(self):
        return self._counted + sum(e.ctx.updates() for e in self.engines.values())
