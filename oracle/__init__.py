"""Plain FP64 CPU oracle of the narrow-band first-order upwind level-set method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` are the only callers.  The
product path (the CUDA library and its binding) never imports this package,
and this package imports nothing from the product.

What it computes, and where the paper defines it (arXiv 1612.04040):

* ``step``            -- Eq. 3-5 (section 1), one explicit upwind step on the
                         points of active tiles; every other point is frozen.
* ``classify``        -- Eq. 6 (section 1.1), tube T tested per tile.
* ``dilate``          -- Eq. 11 (section 1.1), region N as a one-tile dilation.
* ``compact``         -- the array of active points (section 2), as tile ids.
* ``max_abs_speed``   -- CFL bound (the paper gives no rule for dt in Eq. 3).
* ``cutoff``, ``cut_step`` -- Eq. 7 and Eq. 8 (section 1.1): the advance of the
                         local scheme with the cut-off factor c(|phi|).
* ``region_n``        -- Eq. 11 pointwise: T plus its one-cell face ring.
* ``reinit_iter``, ``clamp`` -- Eq. 12-13 (one pseudo-time iteration of the
                         reinitialisation) and Eq. 10 (section 1.1).
* ``local_step``      -- Steps 1-3 of the narrow-band algorithm (section 1.1)
                         as one step: N, cut-off advance, reinitialisation on
                         N, clamp.
* ``Oracle``          -- the rebuild / step schedule of Steps 0-2 of the
                         narrow-band algorithm (section 1.1), with the same
                         call semantics as the C ABI of the library.

Learned coarse-grid corrector (not in the paper; the readings are this
project's): ``conv3_*``, ``cnn_forward`` / ``cnn_backward`` (network),
``restrict4`` (fine -> coarse), ``features``, ``correction``,
``residual_check``, ``learned_step`` (one corrected step with the plain
fallback), ``mse_loss_grad``, ``adam_step``, ``train_iteration``.

The arithmetic of the scheme and of the convolutions lives in
``levelset_oracle.c`` (plain C, no FMA contraction); this module marshals
arrays and runs the schedule, and writes the corrector's element-wise
definitions (features, correction, check, loss, Adam) as numpy
expressions.  Parity pins are in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "levelset_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"extrapolate": 0, "neumann": 1}


def build(force: bool = False) -> str:
    """Compile the C oracle in place (gcc, -O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            ci, cd, c64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            lib.orc_point_update.restype = cd
            lib.orc_point_update.argtypes = [ci, ci, ci, cd, ci, dp, cd, cd, ci, ci, ci]
            lib.orc_step.restype = None
            lib.orc_step.argtypes = [ci, ci, ci, cd, ci, dp, dp, cd, u8p, ci, cd, dp]
            lib.orc_step_points.restype = None
            lib.orc_step_points.argtypes = [ci, ci, ci, cd, ci, dp, dp, cd, i64p, c64, dp]
            lib.orc_classify.restype = None
            lib.orc_classify.argtypes = [ci, ci, ci, ci, dp, cd, u8p]
            lib.orc_dilate.restype = None
            lib.orc_dilate.argtypes = [ci, ci, ci, u8p, ci, u8p]
            lib.orc_compact.restype = c64
            lib.orc_compact.argtypes = [u8p, c64, i32p]
            lib.orc_max_abs_speed.restype = cd
            lib.orc_max_abs_speed.argtypes = [ci, ci, ci, ci, dp, cd, u8p]
            lib.orc_conv3_fwd.restype = None
            lib.orc_conv3_fwd.argtypes = [ci, ci, ci, ci, ci, dp, dp, dp, dp]
            lib.orc_conv3_bwd_data.restype = None
            lib.orc_conv3_bwd_data.argtypes = [ci, ci, ci, ci, ci, dp, dp, dp]
            lib.orc_conv3_bwd_weight.restype = None
            lib.orc_conv3_bwd_weight.argtypes = [ci, ci, ci, ci, ci, dp, dp, dp, dp]
            lib.orc_restrict4.restype = None
            lib.orc_restrict4.argtypes = [ci, ci, ci, dp, dp]
            lib.orc_cutoff.restype = cd
            lib.orc_cutoff.argtypes = [cd, cd, cd]
            lib.orc_cut_step.restype = None
            lib.orc_cut_step.argtypes = [ci, ci, ci, cd, ci, dp, dp, cd, cd, cd, cd, dp]
            lib.orc_region_n.restype = None
            lib.orc_region_n.argtypes = [ci, ci, ci, dp, cd, u8p]
            lib.orc_reinit_iter.restype = None
            lib.orc_reinit_iter.argtypes = [ci, ci, ci, cd, ci, dp, u8p, cd, dp]
            lib.orc_clamp.restype = None
            lib.orc_clamp.argtypes = [c64, dp, u8p, cd]
            lib.orc_local_step.restype = None
            lib.orc_local_step.argtypes = [ci, ci, ci, cd, ci, dp, dp, cd, cd, cd, cd, ci, cd, dp, dp,
                                           u8p]
            _lib = lib
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def tiles_shape(shape, tile):
    nz, ny, nx = shape
    return (-(-nz // tile), -(-ny // tile), -(-nx // tile))


def step(phi, h, dt, F=None, Fc=0.0, tile_active=None, tile=8, bc="extrapolate"):
    """Eq. 3-5: one upwind step.  phi: (nz, ny, nx) array.  F: field or None
    (then the constant Fc).  tile_active: (tnz, tny, tnx) flags or None for the
    whole domain."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    Fa = None if F is None else _f64(F)
    if Fa is not None and Fa.shape != phi.shape:
        raise ValueError("F shape")
    ta = None
    if tile_active is not None:
        ta = np.ascontiguousarray(tile_active, dtype=np.uint8)
        if ta.shape != tiles_shape(phi.shape, tile):
            raise ValueError("tile_active shape")
    out = np.empty_like(phi)
    lib.orc_step(nx, ny, nz, float(h), BC[bc], _ptr(phi, ctypes.c_double),
                 _ptr(Fa, ctypes.c_double), float(Fc), _ptr(ta, ctypes.c_uint8), int(tile),
                 float(dt), _ptr(out, ctypes.c_double))
    return out


def step_points(phi, h, dt, flat_idx, F_at_pts, bc="extrapolate"):
    """Eq. 3-5 evaluated at selected flat indices of phi (no other point is
    touched).  F_at_pts: the speed at each selected point."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    fp = _f64(np.broadcast_to(np.asarray(F_at_pts, dtype=np.float64), idx.shape))
    out = np.empty(idx.shape, dtype=np.float64)
    lib.orc_step_points(nx, ny, nz, float(h), BC[bc], _ptr(phi, ctypes.c_double),
                        _ptr(fp, ctypes.c_double), float(dt), _ptr(idx, ctypes.c_int64),
                        int(idx.size), _ptr(out, ctypes.c_double))
    return out


def classify(phi, gamma, tile=8):
    """Eq. 6 per tile: 1 where some point of the tile has |phi| < gamma."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    core = np.zeros(tiles_shape(phi.shape, tile), dtype=np.uint8)
    lib.orc_classify(nx, ny, nz, int(tile), _ptr(phi, ctypes.c_double), float(gamma),
                     _ptr(core, ctypes.c_uint8))
    return core


def dilate(core, conn=26):
    """Eq. 11 as a one-tile dilation of the core set (6 or 26 neighbours)."""
    lib = _load()
    core = np.ascontiguousarray(core, dtype=np.uint8)
    tnz, tny, tnx = core.shape
    active = np.zeros_like(core)
    lib.orc_dilate(tnx, tny, tnz, _ptr(core, ctypes.c_uint8), int(conn),
                   _ptr(active, ctypes.c_uint8))
    return active


def compact(flags):
    """Ascending ids of the set flags (the active array of section 2)."""
    lib = _load()
    f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
    ids = np.empty(f.size, dtype=np.int32)
    n = lib.orc_compact(_ptr(f, ctypes.c_uint8), f.size, _ptr(ids, ctypes.c_int32))
    return ids[:n].copy()


def max_abs_speed(shape, F=None, Fc=0.0, tile_active=None, tile=8):
    """max |F| over the points of active tiles (every point if tile_active is
    None); 0 if there is none."""
    lib = _load()
    nz, ny, nx = shape
    Fa = None if F is None else _f64(F)
    ta = None if tile_active is None else np.ascontiguousarray(tile_active, dtype=np.uint8)
    return float(lib.orc_max_abs_speed(nx, ny, nz, int(tile), _ptr(Fa, ctypes.c_double),
                                       float(Fc), _ptr(ta, ctypes.c_uint8)))


def cutoff(a, beta, gamma):
    """Eq. 7: c at a = |phi| (scalar)."""
    return float(_load().orc_cutoff(float(a), float(beta), float(gamma)))


def cut_step(phi, h, dt, beta, gamma, F=None, Fc=0.0, bc="extrapolate"):
    """Eq. 8 as Eq. 3 with the speed c(|phi|) F, at every point."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    Fa = None if F is None else _f64(F)
    out = np.empty_like(phi)
    lib.orc_cut_step(nx, ny, nz, float(h), BC[bc], _ptr(phi, ctypes.c_double),
                     _ptr(Fa, ctypes.c_double), float(Fc), float(beta), float(gamma), float(dt),
                     _ptr(out, ctypes.c_double))
    return out


def region_n(phi, gamma):
    """Eq. 11 pointwise: 1 where the point or a face neighbour has |phi| < gamma."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    m = np.empty(phi.shape, dtype=np.uint8)
    lib.orc_region_n(nx, ny, nz, _ptr(phi, ctypes.c_double), float(gamma), _ptr(m, ctypes.c_uint8))
    return m


def reinit_iter(d, h, dtau, nmask=None, bc="extrapolate"):
    """One pseudo-time iteration of Eq. 12 on the points of nmask (all if None)."""
    lib = _load()
    d = _f64(d)
    nz, ny, nx = d.shape
    m = None if nmask is None else np.ascontiguousarray(nmask, dtype=np.uint8)
    out = np.empty_like(d)
    lib.orc_reinit_iter(nx, ny, nz, float(h), BC[bc], _ptr(d, ctypes.c_double),
                        _ptr(m, ctypes.c_uint8), float(dtau), _ptr(out, ctypes.c_double))
    return out


def clamp(d, gamma, nmask=None):
    """Eq. 10 on the points of nmask (all if None); returns a new array."""
    lib = _load()
    out = _f64(d).copy()
    m = None if nmask is None else np.ascontiguousarray(nmask, dtype=np.uint8)
    lib.orc_clamp(out.size, _ptr(out, ctypes.c_double), _ptr(m, ctypes.c_uint8), float(gamma))
    return out


def local_step(phi, h, dt, beta, gamma, iters, dtau, F=None, Fc=0.0, bc="extrapolate"):
    """Steps 1-3 of section 1.1 as one step; returns (phi^{n+1}, N mask)."""
    lib = _load()
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    Fa = None if F is None else _f64(F)
    out = np.empty_like(phi)
    work = np.empty(2 * phi.size)
    m = np.empty(phi.shape, dtype=np.uint8)
    lib.orc_local_step(nx, ny, nz, float(h), BC[bc], _ptr(phi, ctypes.c_double),
                       _ptr(Fa, ctypes.c_double), float(Fc), float(beta), float(gamma), float(dt),
                       int(iters), float(dtau), _ptr(out, ctypes.c_double),
                       _ptr(work, ctypes.c_double), _ptr(m, ctypes.c_uint8))
    return out, m


DT_FIXED, DT_CFL = 0, 1
SCHEME_PLAIN, SCHEME_LOCAL = 0, 1


class Oracle:
    """The narrow-band schedule (section 1.1, Steps 1-2) with the library's
    call semantics:

    * ``band_rebuild(halfwidth)``: gamma = halfwidth*h (FP64); core tiles by
      Eq. 6 on the whole grid, active = dilation of core; M = max|F| over the
      active points (CFL bound).
    * ``step(nsteps, dt_or_cfl, mode, rebuild_every)``: before each step, the
      band is rebuilt if it is stale (after ``set_phi`` / ``set_speed``) or if
      ``rebuild_every`` steps have run since the last rebuild.  dt = CFL*h/M
      (CFL*h when M = 0) in DT_CFL mode, else dt_or_cfl.
    * full-domain mode: every tile active, no rebuilds, M over the whole grid.
    * ``set_scheme(SCHEME_LOCAL, beta_in_h, iters, dtau_in_h)``: each step is
      ``local_step`` (section 1.1, Steps 1-3) over the whole grid; the tiles
      serve only the CFL bound.  ``breaches`` counts N points that lay in
      inactive tiles (where a tiled engine would not update them).
    """

    def __init__(self, shape, h, tile=8, conn=26, bc="extrapolate"):
        self.shape = tuple(int(s) for s in shape)
        self.h = float(h)
        self.tile = int(tile)
        self.conn = int(conn)
        self.bc = bc
        self.tshape = tiles_shape(self.shape, self.tile)
        self.phi = None
        self.F = None
        self.Fc = None
        self.full_domain = False
        self.halfwidth = None
        self.active = None
        self.band_valid = False
        self.since_rebuild = 0
        self.M = None
        self.last_dt = None
        self.rebuild_log = []  # active-tile id arrays, one per rebuild
        self.scheme = SCHEME_PLAIN
        self.local = None      # (beta_in_h, iters, dtau_in_h)
        self.breaches = 0

    # -- state -----------------------------------------------------------
    def set_phi(self, phi):
        phi = _f64(phi).reshape(self.shape)
        if not np.all(np.isfinite(phi)):
            raise ValueError("non-finite phi")
        self.phi = phi.copy()
        self.band_valid = False

    def set_speed(self, F):
        F = _f64(F).reshape(self.shape)
        if not np.all(np.isfinite(F)):
            raise ValueError("non-finite F")
        self.F, self.Fc = F.copy(), None
        self.band_valid = False

    def set_speed_const(self, Fc):
        self.F, self.Fc = None, float(Fc)
        self.band_valid = False

    def set_full_domain(self, on):
        self.full_domain = bool(on)
        self.band_valid = False

    def set_scheme(self, scheme, beta_in_h=None, iters=None, dtau_in_h=None):
        self.scheme = int(scheme)
        if self.scheme == SCHEME_LOCAL:
            self.local = (float(beta_in_h), int(iters), float(dtau_in_h))

    # -- band ------------------------------------------------------------
    def _speed_bound(self, active):
        if self.F is None and self.Fc is None:
            return None
        return max_abs_speed(self.shape, self.F, self.Fc or 0.0, active, self.tile)

    def _rebuild(self):
        gamma = self.halfwidth * self.h
        # Eq. 6 over the whole grid every time (the plain definition; the
        # library scans only the previous active set, and the tests check the
        # two agree).
        core = classify(self.phi, gamma, self.tile)
        self.active = dilate(core, self.conn)
        self.M = self._speed_bound(self.active)
        self.band_valid = True
        self.since_rebuild = 0
        self.rebuild_log.append(compact(self.active))

    def band_rebuild(self, halfwidth):
        self.halfwidth = float(halfwidth)
        self._rebuild()
        return int(self.active.sum())

    def active_tiles(self):
        return compact(self.active)

    # -- stepping ----------------------------------------------------------
    def step(self, nsteps, dt_or_cfl, mode=DT_CFL, rebuild_every=0):
        if self.phi is None:
            raise RuntimeError("phi not set")
        if mode == DT_CFL and self.F is None and self.Fc is None:
            raise RuntimeError("speed not set")
        if self.F is None and self.Fc is None:
            raise RuntimeError("speed not set")
        for _ in range(int(nsteps)):
            if self.full_domain:
                if not self.band_valid:
                    self.M = self._speed_bound(None)
                    self.band_valid = True
                active = None
            else:
                if self.halfwidth is None:
                    raise RuntimeError("no band")
                if not self.band_valid:
                    self._rebuild()
                elif rebuild_every > 0 and self.since_rebuild >= rebuild_every:
                    self._rebuild()
                active = self.active
            if mode == DT_CFL:
                dt = float(dt_or_cfl) * self.h / self.M if self.M > 0 else float(dt_or_cfl) * self.h
            else:
                dt = float(dt_or_cfl)
            if self.scheme == SCHEME_LOCAL:
                b_h, iters, dtau_h = self.local
                gamma = self.halfwidth * self.h
                self.phi, nmask = local_step(self.phi, self.h, dt, b_h * self.h, gamma, iters,
                                             dtau_h * self.h, self.F, self.Fc or 0.0, self.bc)
                if active is not None:
                    t = self.tile
                    act_pts = np.repeat(np.repeat(np.repeat(active, t, 0), t, 1), t, 2)
                    act_pts = act_pts[:self.shape[0], :self.shape[1], :self.shape[2]]
                    self.breaches += int(np.count_nonzero(nmask.astype(bool) & ~act_pts.astype(bool)))
            else:
                self.phi = step(self.phi, self.h, dt, self.F, self.Fc or 0.0, active, self.tile,
                                self.bc)
            self.since_rebuild += 1
            self.last_dt = dt
        return self.last_dt


# --------------------------------------------------------------------------
# learned coarse-grid corrector (not in the paper): FP64 definitions
# --------------------------------------------------------------------------

def conv3_fwd(x, W, b=None):
    """3x3x3 convolution, zero padding.  x: (nz, ny, nx, ci), W: (27, ci, co)
    with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), b: (co,) or None."""
    lib = _load()
    x = _f64(x)
    W = _f64(W)
    nz, ny, nx, ci = x.shape
    co = W.shape[2]
    y = np.empty((nz, ny, nx, co))
    bb = None if b is None else _f64(b)
    lib.orc_conv3_fwd(nx, ny, nz, ci, co, _ptr(x, ctypes.c_double), _ptr(W, ctypes.c_double),
                      _ptr(bb, ctypes.c_double), _ptr(y, ctypes.c_double))
    return y


def conv3_bwd_data(dy, W):
    """Gradient of conv3_fwd with respect to its input."""
    lib = _load()
    dy = _f64(dy)
    W = _f64(W)
    nz, ny, nx, co = dy.shape
    ci = W.shape[1]
    dx = np.empty((nz, ny, nx, ci))
    lib.orc_conv3_bwd_data(nx, ny, nz, ci, co, _ptr(dy, ctypes.c_double), _ptr(W, ctypes.c_double),
                           _ptr(dx, ctypes.c_double))
    return dx


def conv3_bwd_weight(x, dy):
    """Gradients of conv3_fwd with respect to W (27, ci, co) and b (co,)."""
    lib = _load()
    x = _f64(x)
    dy = _f64(dy)
    nz, ny, nx, ci = x.shape
    co = dy.shape[3]
    dW = np.empty((27, ci, co))
    db = np.empty((co,))
    lib.orc_conv3_bwd_weight(nx, ny, nz, ci, co, _ptr(x, ctypes.c_double), _ptr(dy, ctypes.c_double),
                             _ptr(dW, ctypes.c_double), _ptr(db, ctypes.c_double))
    return dW, db


def restrict4(fine):
    """Fine -> coarse (factor 4): the trilinear value at each coarse cell
    centre, i.e. the mean of the 2^3 fine points around it."""
    lib = _load()
    f = _f64(fine)
    nfz, nfy, nfx = f.shape
    c = np.empty((nfz // 4, nfy // 4, nfx // 4))
    lib.orc_restrict4(nfx, nfy, nfz, _ptr(f, ctypes.c_double), _ptr(c, ctypes.c_double))
    return c


def relu(a):
    return np.maximum(a, 0.0)


def cnn_forward(x, params):
    """The corrector network: conv-ReLU-conv-ReLU-conv-ReLU-conv.
    params: list of (W, b).  Returns the list of layer outputs [a1, a2, a3, z4]
    (post-ReLU for the hidden layers)."""
    acts = []
    a = x
    for k, (W, b) in enumerate(params):
        z = conv3_fwd(a, W, b)
        a = relu(z) if k < len(params) - 1 else z
        acts.append(a)
    return acts


def cnn_backward(x, params, acts, dz_out):
    """Gradients of sum(dz_out * z4) with respect to every (W, b)."""
    grads = [None] * len(params)
    g = dz_out
    for k in range(len(params) - 1, -1, -1):
        inp = x if k == 0 else acts[k - 1]
        dW, db = conv3_bwd_weight(inp, g)
        grads[k] = (dW, db)
        if k > 0:
            g = conv3_bwd_data(g, params[k][0]) * (acts[k - 1] > 0)
    return grads


# --------------------------------------------------------------------------
# the corrected coarse step and its training step (not in the paper): FP64
# numpy definitions, written out one expression per reading
# --------------------------------------------------------------------------

FEATURE_CLAMP = 8.0


def features(phi, phit, h, F=None, Fc=0.0):
    """Corrector inputs, channels-last (nz, ny, nx, 3):
    [clamp(phi^n / h, -8, 8), F, (phi~ - phi^n) / h], where phi~ is the plain
    step (Eq. 3) of phi^n.  phi is scaled by the grid spacing so the network
    sees cell units; F keeps its own units."""
    phi = _f64(phi)
    phit = _f64(phit)
    Fa = np.full(phi.shape, float(Fc)) if F is None else _f64(F)
    return np.stack([np.clip(phi / h, -FEATURE_CLAMP, FEATURE_CLAMP), Fa, (phit - phi) / h], axis=-1)


def tile_points(active, tile=8):
    """Point mask (nz, ny, nx) of the points of the flagged tiles."""
    a = np.asarray(active, dtype=bool)
    return np.repeat(np.repeat(np.repeat(a, tile, 0), tile, 1), tile, 2)


def correction(z, h, active, tile=8):
    """The corrector's output in phi units: h * z on the points of active
    tiles, 0 elsewhere (points outside the band stay frozen)."""
    return np.where(tile_points(active, tile), float(h) * _f64(z), 0.0)


def residual_check(corr, active, dt, M, tile=8):
    """True when the correction must be rejected: some value on the points of
    active tiles is not finite, or its magnitude exceeds dt * M, the motion of
    one plain step (M = max |F| over the band)."""
    c = _f64(corr)[tile_points(active, tile)]
    if c.size == 0:
        return False
    if not np.all(np.isfinite(c)):
        return True
    return bool(np.max(np.abs(c)) > float(dt) * float(M))


def learned_step(phi, h, dt, active, params, F=None, Fc=0.0, M=None, bc="extrapolate", tile=8,
                 round_features=None):
    """One corrected coarse step: phi~ = Eq. 3 on the active tiles;
    z = network(features); the correction h z on the active tiles is applied
    unless residual_check rejects it, in which case the result is phi~ (the
    plain fallback).  M defaults to max |F| over the active points.
    round_features, if given, is applied to the features before the network
    (a test uses it to feed the network the same rounded inputs as the
    device).  Returns (phi^{n+1}, phi~, z, rejected)."""
    phit = step(phi, h, dt, F, Fc, active, tile, bc)
    X = features(phi, phit, h, F, Fc)
    if round_features is not None:
        X = round_features(X)
    z = cnn_forward(X, params)[-1][..., 0]
    corr = correction(z, h, active, tile)
    if M is None:
        M = max_abs_speed(np.shape(phi), F, Fc, active, tile)
    rejected = residual_check(corr, active, dt, M, tile)
    return (phit if rejected else phit + corr), phit, z, rejected


def mse_loss_grad(z, phi, phit, phiref, h, gamma):
    """Training loss and its gradient with respect to z.  Target
    t = (phi_ref - phi~) / h, the correction (in cells) that would turn the
    plain step into the reference; loss = mean over the tube T of Eq. 6
    (|phi^n| < gamma) of (z - t)^2; dloss/dz = 2 (z - t) / |T| on T, 0 off T.
    An empty tube gives loss 0 and a zero gradient."""
    z = _f64(z)
    t = (_f64(phiref) - _f64(phit)) / h
    mask = np.abs(_f64(phi)) < gamma
    n = int(np.count_nonzero(mask))
    r = np.where(mask, z - t, 0.0)
    cnt = max(n, 1)
    return float(np.sum(r * r) / cnt), 2.0 * r / cnt, n


ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(w, g, m, v, t, lr, beta1=ADAM_BETA1, beta2=ADAM_BETA2, eps=ADAM_EPS):
    """Adam (Kingma and Ba): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    m^ = m / (1 - b1^t), v^ = v / (1 - b2^t), w <- w - lr m^ / (sqrt(v^) + eps),
    for step number t >= 1.  Returns (w, m, v)."""
    g = _f64(g)
    m = beta1 * _f64(m) + (1.0 - beta1) * g
    v = beta2 * _f64(v) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return _f64(w) - lr * mh / (np.sqrt(vh) + eps), m, v


def unpack_params(flat, chans=(3, 16, 16, 16, 1)):
    """Split the library's flat parameter vector (per layer W [27][ci][co]
    then b [co]) into [(W, b), ...]."""
    flat = _f64(flat)
    out, o = [], 0
    for k in range(len(chans) - 1):
        ci, co = chans[k], chans[k + 1]
        W = flat[o:o + 27 * ci * co].reshape(27, ci, co)
        o += 27 * ci * co
        b = flat[o:o + co]
        o += co
        out.append((W, b))
    if o != flat.size:
        raise ValueError("parameter vector has %d values, the network %d" % (flat.size, o))
    return out


def pack_params(params):
    return np.concatenate([np.concatenate([_f64(W).reshape(-1), _f64(b).reshape(-1)]) for W, b in params])


def train_iteration(phi, phiref, F, h, dt, gamma, flat, m, v, t, lr, bc="extrapolate",
                    round_features=None):
    """One training iteration on one pair (phi^n, phi_ref, F) over the whole
    grid: phi~ = Eq. 3 everywhere, features, network forward, masked MSE
    gradient, backward through the network, Adam step t.  Returns
    (flat', m', v', loss, flat gradient)."""
    phit = step(phi, h, dt, F, 0.0, None, 8, bc)
    X = features(phi, phit, h, F)
    if round_features is not None:
        X = round_features(X)
    params = unpack_params(flat)
    acts = cnn_forward(X, params)
    loss, dz, _ = mse_loss_grad(acts[-1][..., 0], phi, phit, phiref, h, gamma)
    grads = cnn_backward(X, params, acts, dz[..., None])
    gflat = pack_params(grads)
    w2, m2, v2 = adam_step(flat, gflat, m, v, t, lr)
    return w2, m2, v2, loss, gflat
