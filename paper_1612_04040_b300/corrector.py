"""Learned coarse-grid corrector: training pairs, training and evaluation.

Orchestration only; every numerical step runs in the library's kernels
through the C ABI (fine plain runs, restriction, training, corrected
steps).  This part is not in the paper.

* Pairs: a fine grid (4x finer) runs the plain narrow-band method with a
  fixed dt_f; every 4 fine steps give one pair (R(phi_f^n), R(phi_f^{n+4}),
  R(F_f)) on the coarse grid, R = restriction by 4 (mean of the 2^3 fine
  points around each coarse cell centre).  The fine band is 4x as wide (in
  fine cells) as the coarse band, so the reference is a solution of the
  plain scheme everywhere the coarse band and its loss look.
* Coarse step: dt_c = 4 dt_f, so one coarse step spans one pair.
* Error: over coarse points within 1.5 h_c of the reference's zero set,
  max |phi - phi_ref| / h_c (|grad phi| ~ 1 near the front, so this is the
  zero-level-set displacement in coarse cells).
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs
from . import native as ls


def random_problem(g: np.random.Generator, box):
    """Seeded sphere union inside `box` (extent per axis, x y z) and an
    8-mode low-frequency Fourier speed with |F| <= 1."""
    lo = np.array([0.2 * b for b in box])
    hi = np.array([0.8 * b for b in box])
    rmax = 0.35 * min(box)
    k = int(g.integers(2, 6))
    centres = [tuple(float(v) for v in g.uniform(lo, hi)) for _ in range(k)]
    radii = [float(g.uniform(0.3 * rmax, rmax)) for _ in range(k)]
    modes = inputs.fourier_modes(g, count=8, kmax=2)
    return centres, radii, modes


class PairGenerator:
    """Fine plain runs restricted to the coarse grid of `coarse_shape`
    (nz, ny, nx) with coarse spacing h_c."""

    def __init__(self, coarse_shape, h_c, halfwidth_c=6.0, cfl=0.5, device="cuda"):
        self.cs = tuple(coarse_shape)
        self.fs = tuple(4 * n for n in coarse_shape)
        self.h_c = float(h_c)
        self.h_f = self.h_c / 4
        self.hw_f = 4.0 * halfwidth_c
        self.dt_f = cfl * self.h_f
        self.dt_c = 4 * self.dt_f
        self.device = device
        nz, ny, nx = self.fs
        self.fine = ls.LevelSet(nx, ny, nz, self.h_f, ls.LS_FP32)
        self.buf = torch.empty(self.fs, dtype=torch.float32, device=device)

    def box(self):
        nz, ny, nx = self.fs
        return (nx * self.h_f, ny * self.h_f, nz * self.h_f)

    def fields(self, centres, radii, modes):
        """Step 0 on the fine grid by the library's device generators
        (ls_init_phi / ls_init_speed); returns (phi, F) as device tensors."""
        self.fine.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(centres, radii))
        self.fine.init_speed(ls.LS_SPEED_FOURIER, inputs.fourier_params(modes))
        phi = torch.empty(self.fs, dtype=torch.float32, device=self.device)
        F = torch.empty(self.fs, dtype=torch.float32, device=self.device)
        self.fine.get_phi(phi)
        self.fine.get_speed(F)
        return phi, F

    def restrict(self, a):
        return ls.restrict4(a)

    def run(self, centres, radii, modes, npairs):
        """Yields (phi_c^n, phi_c^{n+4}, F_c) for n = 0, 4, ... (coarse device
        tensors), plus the coarse initial state first."""
        phi, F = self.fields(centres, radii, modes)   # also the fine context's phi and F
        self.fine.band_rebuild(self.hw_f)
        F_c = self.restrict(F)
        prev = self.restrict(phi)
        out = []
        for _ in range(npairs):
            self.fine.step(4, self.dt_f, ls.LS_DT_FIXED, 4)
            self.fine.get_phi(self.buf)
            cur = self.restrict(self.buf)
            out.append((prev, cur, F_c))
            prev = cur
        return out


def front_error(phi, ref, h):
    """(max, mean) of |phi - ref| / h over the points with |ref| < 1.5 h."""
    near = ref.abs() < 1.5 * h
    if int(near.sum()) == 0:
        return float("nan"), float("nan")
    d = (phi - ref).abs()[near] / h
    return float(d.max()), float(d.mean())


def coarse_run(ctx: ls.LevelSet, phi0, F_c, nsteps, dt, halfwidth, learned):
    ctx.set_phi(phi0)
    ctx.set_speed(F_c)
    ctx.set_step_mode(ls.LS_LEARNED if learned else ls.LS_PLAIN)
    ctx.band_rebuild(halfwidth)
    ctx.step(nsteps, dt, ls.LS_DT_FIXED, 1)
    out = torch.empty_like(phi0)
    ctx.get_phi(out)
    ctx.set_step_mode(ls.LS_PLAIN)
    return out
