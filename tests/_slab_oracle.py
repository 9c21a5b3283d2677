"""A slab engine made of the FP64 oracle (test infrastructure): the same
interface as the library's ``slab.GpuSlab``, so that the slab split's host
logic (Eq. 14 partition, exchange plan, schedule, migration) can be checked
on the CPU against one unsplit oracle run."""
import numpy as np
import torch

import oracle


class OracleSlab:
    def __init__(self, nx, ny, rows, h, lo, hi):
        self.nx, self.ny, self.rows, self.lo, self.hi = nx, ny, rows, lo, hi
        self.h = float(h)

    def close(self):
        pass

    def setup(self, phi, F, halfwidth):
        self.p = np.array(torch.as_tensor(phi).cpu().numpy(), dtype=np.float64)
        self.F = np.array(torch.as_tensor(F).cpu().numpy(), dtype=np.float64)
        assert self.p.shape == (8 * self.rows, self.ny, self.nx)
        self.gamma = float(halfwidth) * self.h
        self.active = None

    def refresh(self):
        act = oracle.dilate(oracle.classify(self.p, self.gamma))
        if self.lo:
            act[0] = 0          # a ghost row is never active
        if self.hi:
            act[-1] = 0
        self.active = act
        M = oracle.max_abs_speed(self.p.shape, self.F, 0.0, act)
        return M, int(act.sum())

    def row_counts(self):
        return self.active.reshape(self.rows, -1).sum(axis=1).astype(np.int64)

    def step(self, dt, rebuild_every, n=1):
        for _ in range(n):
            self.p = oracle.step(self.p, self.h, dt, self.F, 0.0, self.active)

    def buffer(self, plane):
        return torch.empty((8 if plane < 0 else 1) * self.ny * self.nx, dtype=torch.float64)

    def _planes(self, row, plane):
        return slice(8 * row, 8 * row + 8) if plane < 0 else slice(8 * row + plane, 8 * row + plane + 1)

    def export_row(self, row, plane, out):
        out.copy_(torch.from_numpy(np.ascontiguousarray(self.p[self._planes(row, plane)]).reshape(-1)))

    def import_row(self, row, plane, src):
        sl = self._planes(row, plane)
        self.p[sl] = src.numpy().reshape(self.p[sl].shape)

    def phi(self):
        return torch.from_numpy(self.p)

    def speed(self):
        return torch.from_numpy(self.F)

    def zeros(self, nplanes):
        return torch.zeros((nplanes, self.ny, self.nx), dtype=torch.float64)
