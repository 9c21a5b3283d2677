"""ctypes binding of libls.so (the C ABI in include/ls.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Functions keep the C names (``ls_create``, ``ls_step`` ...) and
raise ``LSError`` on a non-zero status.  Arrays may be torch tensors (CUDA or
CPU) or numpy arrays; they must be C-contiguous, of the context's precision
(float32 for LS_FP32, float64 for LS_FP64) and hold nx*ny*nz values in
[z][y][x] order.  There is no fallback: if libls.so is missing or cannot be
loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the image
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libls.so")

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ECUDA, LS_ETIMEOUT, LS_ENONFINITE, LS_ESTATE, LS_EIO = 0, -1, -2, -3, -4, -5, -6, -7
LS_FP32, LS_FP64 = 0, 1
LS_DT_FIXED, LS_DT_CFL, LS_DT_KEEP = 0, 1, 2
LS_PLAIN, LS_LEARNED = 0, 1
LS_SCHEME_PLAIN, LS_SCHEME_LOCAL = 0, 1
LS_OUTPUT_VTS, LS_OUTPUT_VTI = 0, 1
LS_BC_EXTRAPOLATE, LS_BC_NEUMANN = 0, 1
LS_REBUILD_AUTO, LS_REBUILD_FULL, LS_REBUILD_INCREMENTAL = 0, 1, 2
LS_REBUILD_AUTO_TILES = 1 << 19
LS_SHAPE_SPHERES, LS_SHAPE_TORUS, LS_SHAPE_SH = 0, 1, 2
LS_SPEED_SINUSOID, LS_SPEED_COSCOS, LS_SPEED_FOURIER = 0, 1, 2

_lib = None

# name -> (restype, argtypes); every entry point declared in include/ls.h
_c = ctypes
_vp, _i, _d, _ll = _c.c_void_p, _c.c_int, _c.c_double, _c.c_longlong
_pp = _c.POINTER(_c.c_void_p)
SIGNATURES = {
    "ls_create": (_i, [_i, _i, _i, _d, _i, _pp]),
    "ls_destroy": (_i, [_vp]),
    "ls_set_stream": (_i, [_vp, _vp]),
    "ls_set_phi": (_i, [_vp, _vp, _i]),
    "ls_set_speed": (_i, [_vp, _vp, _i]),
    "ls_set_speed_const": (_i, [_vp, _d]),
    "ls_set_bc": (_i, [_vp, _i]),
    "ls_init_phi": (_i, [_vp, _i, _vp, _i]),
    "ls_init_speed": (_i, [_vp, _i, _vp, _i]),
    "ls_inst_init_phi": (_i, [_vp, _i, _i, _vp, _i]),
    "ls_inst_init_speed": (_i, [_vp, _i, _i, _vp, _i]),
    "ls_selftest_bounded_wait": (_i, [_vp, _ll, _vp]),
    "ls_band_rebuild": (_i, [_vp, _d, _c.POINTER(_ll)]),
    "ls_step": (_i, [_vp, _i, _d, _i, _i, _c.POINTER(_d)]),
    "ls_set_full_domain": (_i, [_vp, _i]),
    "ls_get_phi": (_i, [_vp, _vp, _i]),
    "ls_get_speed": (_i, [_vp, _vp, _i]),
    "ls_set_ghost_rows": (_i, [_vp, _i, _i]),
    "ls_band_refresh": (_i, [_vp, _vp, _vp]),
    "ls_band_speed_bound": (_i, [_vp, _vp, _i]),
    "ls_set_dt_from_bound": (_i, [_vp, _vp, _d]),
    "ls_band_row_counts": (_i, [_vp, _vp, _i]),
    "ls_get_tile_rows": (_i, [_vp, _i, _i, _i, _vp, _i]),
    "ls_set_tile_rows": (_i, [_vp, _i, _i, _i, _vp, _i]),
    "ls_copy_ghost_row": (_i, [_vp, _i, _vp, _i, _i]),
    "ls_stage_inputs": (_i, [_vp, _vp, _vp]),
    "ls_load_staged": (_i, [_vp]),
    "ls_get_phi_async": (_i, [_vp, _vp]),
    "ls_wait_host": (_i, [_vp]),
    "ls_snapshot": (_i, [_vp]),
    "ls_restore": (_i, [_vp]),
    "ls_get_active_tiles": (_i, [_vp, _c.POINTER(_c.c_int), _ll, _c.POINTER(_ll)]),
    "ls_get_updates": (_i, [_vp, _c.POINTER(_c.c_ulonglong)]),
    "ls_set_graphs": (_i, [_vp, _i]),
    "ls_autotune": (_i, [_vp, _i, _c.POINTER(_i), _c.POINTER(_i), _c.POINTER(_i)]),
    "ls_set_step_config": (_i, [_vp, _i, _i, _i]),
    "ls_batch_create": (_i, [_i, _c.POINTER(_i), _c.POINTER(_i), _c.POINTER(_i), _c.POINTER(_d), _i, _pp]),
    "ls_batch_size": (_i, [_vp, _c.POINTER(_i)]),
    "ls_inst_set_phi": (_i, [_vp, _i, _vp, _i]),
    "ls_inst_set_speed": (_i, [_vp, _i, _vp, _i]),
    "ls_inst_set_speed_const": (_i, [_vp, _i, _d]),
    "ls_inst_get_phi": (_i, [_vp, _i, _vp, _i]),
    "ls_inst_get_active_tiles": (_i, [_vp, _i, _c.POINTER(_c.c_int), _ll, _c.POINTER(_ll)]),
    "ls_inst_last_dt": (_i, [_vp, _i, _c.POINTER(_d)]),
    "ls_learned_num_params": (_i, [_c.POINTER(_ll)]),
    "ls_learned_init": (_i, [_vp, _c.c_ulonglong]),
    "ls_learned_set_params": (_i, [_vp, _vp, _ll]),
    "ls_learned_get_params": (_i, [_vp, _vp, _ll]),
    "ls_learned_add_pair": (_i, [_vp, _vp, _vp, _vp, _i]),
    "ls_learned_num_pairs": (_i, [_vp, _c.POINTER(_ll)]),
    "ls_learned_train_stored": (_i, [_vp, _i, _d, _d, _d, _c.c_ulonglong, _c.POINTER(_d)]),
    "ls_learned_train": (_i, [_vp, _c.c_char_p, _i, _d, _c.POINTER(_d)]),
    "ls_learned_load": (_i, [_vp, _vp, _c.c_size_t]),
    "ls_learned_save": (_i, [_vp, _vp, _c.c_size_t]),
    "ls_learned_get_pair": (_i, [_vp, _c.c_longlong, _vp, _vp, _vp, _i]),
    "ls_set_step_mode": (_i, [_vp, _i]),
    "ls_set_scheme": (_i, [_vp, _i, _c.c_double, _i, _c.c_double]),
    "ls_set_dilation": (_i, [_vp, _i]),
    "ls_set_rebuild_mode": (_i, [_vp, _i]),
    "ls_set_dense_kernel": (_i, [_vp, _i]),
    "ls_set_steps_per_pass": (_i, [_vp, _i]),
    "ls_get_steps_per_pass": (_i, [_vp, _c.POINTER(_i)]),
    "ls_output_open": (_i, [_vp, _c.c_char_p, _i, _i, _i]),
    "ls_output_stats": (_i, [_vp, _vp]),
    "ls_output_close": (_i, [_vp, _vp]),
    "ls_write_vtk": (_i, [_c.c_char_p, _vp, _i, _i, _i, _c.c_double, _i, _i]),
    "ls_probe_dfma": (_i, [_ll, _c.POINTER(_d), _vp]),
    "ls_band_breaches": (_i, [_vp, _c.POINTER(_c.c_ulonglong)]),
    "ls_learned_fallbacks": (_i, [_vp, _c.POINTER(_c.c_ulonglong)]),
    "ls_conv3_bf16": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "ls_conv3_wgrad": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "ls_restrict4": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "ls_learned_features": (_i, [_vp, _vp, _vp, _d, _d, _ll, _vp, _vp]),
    "ls_learned_loss_grad": (_i, [_vp, _vp, _vp, _vp, _ll, _d, _d, _vp, _vp, _vp, _vp]),
    "ls_adam_step": (_i, [_vp, _vp, _vp, _vp, _i, _d, _i, _vp]),
    "ls_profile_enable": (_i, [_vp, _i]),
    "ls_get_profile": (_i, [_vp, _vp]),
    "ls_reset_profile": (_i, [_vp]),
    "ls_get_status": (_i, [_vp]),
    "ls_band_tiles_noalloc": (_i, [_vp, _i, _i, _i, _d, _i, _d, _vp, _ll, _vp, _vp]),
    "ls_strerror": (_c.c_char_p, [_i]),
    "ls_last_cuda_error": (_i, []),
}


class Profile(ctypes.Structure):
    """ls_profile of include/ls.h."""
    _fields_ = [("kernel_launches", ctypes.c_ulonglong), ("stencil_launches", ctypes.c_ulonglong),
                ("stencil_ms", ctypes.c_double), ("stencil_timed", ctypes.c_ulonglong),
                ("reinit_ms", ctypes.c_double), ("reinit_timed", ctypes.c_ulonglong),
                ("reinit_updates", ctypes.c_ulonglong), ("two_step_points", ctypes.c_ulonglong),
                ("stencil_updates", ctypes.c_ulonglong)]


class OutputReport(ctypes.Structure):
    """ls_output_report of include/ls.h."""
    _fields_ = [("files", ctypes.c_ulonglong), ("bytes", ctypes.c_ulonglong),
                ("write_seconds", ctypes.c_double), ("wait_seconds", ctypes.c_double),
                ("status", ctypes.c_int)]


class LSError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = "%s: %s (%d)" % (what, strerror(status), status)
        if status == LS_ECUDA and _lib is not None:
            msg += " [cuda error %d]" % _lib.ls_last_cuda_error()
        super().__init__(msg)


def load():
    """Load libls.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libls.so not found at %s; build it with "
                               "`python -m paper_1612_04040_b300.build`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def strerror(status):
    if _lib is None:
        return "status %d" % status
    return _lib.ls_strerror(status).decode()


def check(status, what=""):
    if status != LS_OK:
        raise LSError(status, what)
    return status


def array_ptr(a, dtype, count):
    """(pointer, on_device) of a contiguous array of `count` values of dtype
    (np.float32 / np.float64)."""
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float32 if dtype == np.float32 else torch.float64
        if a.dtype != want:
            raise TypeError("expected %s, got %s" % (want, a.dtype))
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if a.numel() != count:
            raise ValueError("expected %d values, got %d" % (count, a.numel()))
        return ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError("expected %s, got %s" % (dtype, a.dtype))
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.size != count:
            raise ValueError("expected %d values, got %d" % (count, a.size))
        return ctypes.c_void_p(a.ctypes.data), 0
    raise TypeError("expected a torch tensor or numpy array")


LS_NOALLOC_MAX_TILES = 1 << 21


def band_tiles_noalloc(phi, h, halfwidth, tiles_out, count_out, stream=None):
    """ls_band_tiles_noalloc: active-tile ids of a row-major device phi
    (torch CUDA tensor of shape (nz, ny, nx)) into the caller's device
    buffers tiles_out (int32, >= number of tiles) and count_out (int32, 1),
    without any allocation by the library.  Asynchronous on `stream`."""
    lib = load()
    if phi.dtype == torch.float32:
        prec = LS_FP32
    elif phi.dtype == torch.float64:
        prec = LS_FP64
    else:
        raise TypeError("phi must be float32 or float64, got %s" % phi.dtype)
    if tiles_out.dtype != torch.int32 or count_out.dtype != torch.int32:
        raise TypeError("tiles_out and count_out must be int32")
    if phi.dim() != 3 or not phi.is_cuda or not phi.is_contiguous():
        raise ValueError("phi must be a contiguous 3-D CUDA tensor")
    for name, t in (("tiles_out", tiles_out), ("count_out", count_out)):
        if not t.is_cuda or not t.is_contiguous() or t.device != phi.device:
            raise ValueError("%s must be a contiguous CUDA tensor on %s" % (name, phi.device))
    if count_out.numel() < 1:
        raise ValueError("count_out must hold at least one int32")
    nz, ny, nx = phi.shape
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_band_tiles_noalloc(ctypes.c_void_p(phi.data_ptr()), nx, ny, nz, float(h), prec,
                                    float(halfwidth), ctypes.c_void_p(tiles_out.data_ptr()),
                                    tiles_out.numel(), ctypes.c_void_p(count_out.data_ptr()),
                                    ctypes.c_void_p(stream)), "ls_band_tiles_noalloc")


LS_CONV3_WORK_BYTES = 13824


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def conv3_bf16(x, W, bias, mode, mask=None, out=None, stream=None):
    """ls_conv3_bf16 on torch CUDA tensors: x bf16 (nz, ny, nx, 16), W float32
    (27, ci, co), bias float32 (co,).  Returns (out, status word)."""
    lib = load()
    nz, ny, nx, _ = x.shape
    ci, co = W.shape[1], W.shape[2]
    if out is None:
        out = (torch.empty((nz, ny, nx), dtype=torch.float32, device=x.device) if mode == 1
               else torch.empty((nz, ny, nx, 16), dtype=torch.bfloat16, device=x.device))
    work = torch.empty(LS_CONV3_WORK_BYTES, dtype=torch.uint8, device=x.device)
    status = torch.zeros(1, dtype=torch.int32, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_conv3_bf16(_dptr(x), nx, ny, nz, _dptr(W), ci, co, _dptr(bias), int(mode), _dptr(mask),
                            _dptr(out), _dptr(work), _dptr(status), ctypes.c_void_p(stream)), "ls_conv3_bf16")
    return out, status


def selftest_bounded_wait(polls, stream=None):
    """ls_selftest_bounded_wait: returns the status word after the wait gave up."""
    lib = load()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_selftest_bounded_wait(_dptr(status), int(polls), ctypes.c_void_p(stream)),
          "ls_selftest_bounded_wait")
    torch.cuda.synchronize()
    return int(status.item())


def conv3_wgrad(x, dy, ci, co, stream=None, with_status=False):
    """ls_conv3_wgrad: returns (dW (27, ci, co), db (co,)) as float32 tensors
    (and the status word when with_status)."""
    lib = load()
    nz, ny, nx, _ = x.shape
    dW = torch.zeros((27, ci, co), dtype=torch.float32, device=x.device)
    db = torch.zeros((co,), dtype=torch.float32, device=x.device)
    status = torch.zeros(1, dtype=torch.int32, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_conv3_wgrad(_dptr(x), _dptr(dy), nx, ny, nz, ci, co, _dptr(dW), _dptr(db), _dptr(status),
                             ctypes.c_void_p(stream)), "ls_conv3_wgrad")
    return (dW, db, status) if with_status else (dW, db)


def restrict4(fine, stream=None):
    """ls_restrict4 on a float32 CUDA tensor (nz, ny, nx)."""
    lib = load()
    nz, ny, nx = fine.shape
    out = torch.empty((nz // 4, ny // 4, nx // 4), dtype=torch.float32, device=fine.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_restrict4(_dptr(fine), nx, ny, nz, _dptr(out), ctypes.c_void_p(stream)), "ls_restrict4")
    return out


def _f32_cuda(name, t, n=None):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must hold %d values" % (name, n))
    return _dptr(t)


def learned_features(phi, phit, h, F=None, Fc=0.0, stream=None):
    """ls_learned_features: BF16 (..., 16) features of float32 CUDA tensors."""
    lib = load()
    n = phi.numel()
    X = torch.empty(tuple(phi.shape) + (16,), dtype=torch.bfloat16, device=phi.device)
    Fp = None if F is None else _f32_cuda("F", F, n)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_learned_features(_f32_cuda("phi", phi), _f32_cuda("phit", phit, n), Fp, float(Fc),
                                  float(h), n, _dptr(X), ctypes.c_void_p(stream)), "ls_learned_features")
    return X


def learned_loss_grad(z, phi, phit, phiref, h, gamma, stream=None):
    """ls_learned_loss_grad: returns (dz BF16 (..., 16), count int32 (1,),
    loss float64 (1,)) as CUDA tensors."""
    lib = load()
    n = phi.numel()
    dz = torch.empty(tuple(phi.shape) + (16,), dtype=torch.bfloat16, device=phi.device)
    count = torch.empty(1, dtype=torch.int32, device=phi.device)
    loss = torch.empty(1, dtype=torch.float64, device=phi.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_learned_loss_grad(_f32_cuda("z", z, n), _f32_cuda("phi", phi), _f32_cuda("phit", phit, n),
                                   _f32_cuda("phiref", phiref, n), n, float(h), float(gamma), _dptr(dz),
                                   _dptr(count), _dptr(loss), ctypes.c_void_p(stream)),
          "ls_learned_loss_grad")
    return dz, count, loss


def adam_step(w, g, m, v, t, lr, stream=None):
    """ls_adam_step on float32 CUDA tensors (w, m, v updated in place)."""
    lib = load()
    n = w.numel()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib.ls_adam_step(_f32_cuda("w", w), _f32_cuda("g", g, n), _f32_cuda("m", m, n),
                           _f32_cuda("v", v, n), n, float(lr), int(t), ctypes.c_void_p(stream)),
          "ls_adam_step")


def probe_dfma(iters=1 << 16, stream=None):
    """Measured FP64 peak of the current device (TFLOP/s, FMA = 2)."""
    lib = load()
    t = ctypes.c_double(0.0)
    check(lib.ls_probe_dfma(int(iters), ctypes.byref(t), None if stream is None else ctypes.c_void_p(stream)),
          "ls_probe_dfma")
    return t.value


def write_vtk(path, phi, h, fmt=LS_OUTPUT_VTS):
    """ls_write_vtk of a row-major host array (nz, ny, nx), float32 or float64."""
    lib = load()
    a = np.ascontiguousarray(phi)
    if a.dtype not in (np.float32, np.float64) or a.ndim != 3:
        raise ValueError("phi: 3-D float32 / float64 array")
    nz, ny, nx = a.shape
    prec = LS_FP32 if a.dtype == np.float32 else LS_FP64
    check(lib.ls_write_vtk(str(path).encode(), a.ctypes.data, nx, ny, nz, float(h), prec, int(fmt)),
          "ls_write_vtk")


class LevelSet:
    """One grid behind an ls_ctx.  Thin wrapper: each method is one ABI call."""

    def __init__(self, nx, ny, nz, h, precision=LS_FP32, stream=None):
        self.lib = load()
        self.shape = (int(nz), int(ny), int(nx))
        self.count = int(nx) * int(ny) * int(nz)
        self.precision = precision
        self.dtype = np.float32 if precision == LS_FP32 else np.float64
        self.h = float(h)
        h_ = ctypes.c_void_p()
        check(self.lib.ls_create(int(nx), int(ny), int(nz), float(h), int(precision), ctypes.byref(h_)),
              "ls_create")
        self.ctx = h_
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        if stream is not None:
            check(self.lib.ls_set_stream(self.ctx, ctypes.c_void_p(stream)), "ls_set_stream")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ls_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        check(self.lib.ls_set_stream(self.ctx, ctypes.c_void_p(stream)), "ls_set_stream")

    def set_phi(self, a):
        p, dev = array_ptr(a, self.dtype, self.count)
        check(self.lib.ls_set_phi(self.ctx, p, dev), "ls_set_phi")

    def set_speed(self, a):
        p, dev = array_ptr(a, self.dtype, self.count)
        check(self.lib.ls_set_speed(self.ctx, p, dev), "ls_set_speed")

    def init_phi(self, shape, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        check(self.lib.ls_init_phi(self.ctx, int(shape), ctypes.c_void_p(p.ctypes.data), p.size), "ls_init_phi")

    def init_speed(self, kind, params=None):
        p = np.ascontiguousarray(params if params is not None else [0.0], dtype=np.float64)
        check(self.lib.ls_init_speed(self.ctx, int(kind), ctypes.c_void_p(p.ctypes.data), p.size),
              "ls_init_speed")

    def set_speed_const(self, F):
        check(self.lib.ls_set_speed_const(self.ctx, float(F)), "ls_set_speed_const")

    def set_bc(self, bc):
        check(self.lib.ls_set_bc(self.ctx, int(bc)), "ls_set_bc")

    def set_full_domain(self, on):
        check(self.lib.ls_set_full_domain(self.ctx, int(bool(on))), "ls_set_full_domain")

    def band_rebuild(self, halfwidth, want_count=True):
        n = ctypes.c_longlong(-1)
        check(self.lib.ls_band_rebuild(self.ctx, float(halfwidth), ctypes.byref(n) if want_count else None),
              "ls_band_rebuild")
        return n.value if want_count else None

    def step(self, nsteps, dt_or_cfl, dt_mode=LS_DT_CFL, rebuild_every=0, want_dt=False):
        d = ctypes.c_double(0.0)
        check(self.lib.ls_step(self.ctx, int(nsteps), float(dt_or_cfl), int(dt_mode), int(rebuild_every),
                               ctypes.byref(d) if want_dt else None), "ls_step")
        return d.value if want_dt else None

    def snapshot(self):
        check(self.lib.ls_snapshot(self.ctx), "ls_snapshot")

    def restore(self):
        check(self.lib.ls_restore(self.ctx), "ls_restore")

    def get_phi(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev = array_ptr(out, self.dtype, self.count)
        check(self.lib.ls_get_phi(self.ctx, p, dev), "ls_get_phi")
        return out

    def get_speed(self, out=None):
        """The speed field F (row-major, context precision)."""
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev = array_ptr(out, self.dtype, self.count)
        check(self.lib.ls_get_speed(self.ctx, p, dev), "ls_get_speed")
        return out

    # -- slab split (section 2) ---------------------------------------------
    def set_ghost_rows(self, lo, hi):
        check(self.lib.ls_set_ghost_rows(self.ctx, int(lo), int(hi)), "ls_set_ghost_rows")

    def band_refresh(self):
        """The rebuild the next step would make; returns (M, active tiles)."""
        M = ctypes.c_double(0.0)
        n = ctypes.c_longlong(0)
        check(self.lib.ls_band_refresh(self.ctx, ctypes.byref(M), ctypes.byref(n)), "ls_band_refresh")
        return M.value, n.value

    def band_refresh_async(self):
        """The rebuild the next step would make, without synchronising."""
        check(self.lib.ls_band_refresh(self.ctx, None, None), "ls_band_refresh")

    def band_speed_bound(self, out):
        """Copy M of the current band into `out` (float64 tensor / array, 1 value)."""
        p, dev = array_ptr(out, np.float64, 1)
        check(self.lib.ls_band_speed_bound(self.ctx, p, dev), "ls_band_speed_bound")
        return out

    def set_dt_from_bound(self, M_device, cfl):
        """dt = cfl h / M with M read from a float64 CUDA tensor of 1 value."""
        if not (M_device.is_cuda and M_device.dtype == torch.float64 and M_device.numel() >= 1):
            raise ValueError("M_device must be a float64 CUDA tensor")
        check(self.lib.ls_set_dt_from_bound(self.ctx, ctypes.c_void_p(M_device.data_ptr()), float(cfl)),
              "ls_set_dt_from_bound")

    def band_row_counts(self):
        nz = self.shape[0] // 8
        out = np.zeros(nz, dtype=np.int64)
        check(self.lib.ls_band_row_counts(self.ctx, out.ctypes.data_as(ctypes.c_void_p), nz),
              "ls_band_row_counts")
        return out

    def _rows_ptr(self, a, nrows, plane):
        n = nrows * (self.shape[1] // 8) * (self.shape[2] // 8) * (512 if plane < 0 else 64)
        return array_ptr(a, self.dtype, n)

    def get_tile_rows(self, row0, nrows, plane, out):
        p, dev = self._rows_ptr(out, nrows, plane)
        check(self.lib.ls_get_tile_rows(self.ctx, int(row0), int(nrows), int(plane), p, dev),
              "ls_get_tile_rows")
        return out

    def set_tile_rows(self, row0, nrows, plane, src):
        p, dev = self._rows_ptr(src, nrows, plane)
        check(self.lib.ls_set_tile_rows(self.ctx, int(row0), int(nrows), int(plane), p, dev),
              "ls_set_tile_rows")

    def copy_ghost_row(self, src, src_row, row, plane):
        """Tile row src_row of the LevelSet `src` into this context's ghost row."""
        check(self.lib.ls_copy_ghost_row(src.ctx, int(src_row), self.ctx, int(row), int(plane)),
              "ls_copy_ghost_row")

    # stream-ordered host input/output (ls_stage_inputs ... ls_wait_host);
    # the arrays must be host (CPU) arrays, page-locked for the copies to
    # overlap the computation, and stay alive until the copies are done
    def _host_ptr(self, a):
        p, dev = array_ptr(a, self.dtype, self.count)
        if dev:
            raise ValueError("expected a host array")
        return p

    def stage_inputs(self, phi, speed=None):
        """Start copying the next problem's phi (and speed field) to the device."""
        self._staged = (phi, speed)  # keep the host arrays alive
        check(self.lib.ls_stage_inputs(self.ctx, self._host_ptr(phi),
                                       None if speed is None else self._host_ptr(speed)),
              "ls_stage_inputs")

    def load_staged(self):
        """Make the staged arrays the context's phi (and speed field)."""
        check(self.lib.ls_load_staged(self.ctx), "ls_load_staged")
        self._staged = None

    def get_phi_async(self, out):
        """Start copying the current phi into the host array `out`."""
        self._pending = getattr(self, "_pending", []) + [out]
        check(self.lib.ls_get_phi_async(self.ctx, self._host_ptr(out)), "ls_get_phi_async")

    def wait_host(self):
        """Wait for every staged copy and read-back."""
        check(self.lib.ls_wait_host(self.ctx), "ls_wait_host")
        self._pending = []

    def active_tiles(self):
        n = ctypes.c_longlong(0)
        check(self.lib.ls_get_active_tiles(self.ctx, None, 0, ctypes.byref(n)), "ls_get_active_tiles")
        buf = np.empty(max(n.value, 1), dtype=np.int32)
        check(self.lib.ls_get_active_tiles(self.ctx, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                           n.value, ctypes.byref(n)), "ls_get_active_tiles")
        return buf[:n.value].copy()

    def updates(self):
        n = ctypes.c_ulonglong(0)
        check(self.lib.ls_get_updates(self.ctx, ctypes.byref(n)), "ls_get_updates")
        return n.value

    def status(self):
        return self.lib.ls_get_status(self.ctx)

    def set_graphs(self, on=True):
        check(self.lib.ls_set_graphs(self.ctx, int(bool(on))), "ls_set_graphs")

    def autotune(self, reps=5):
        st, pct, ppt = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        check(self.lib.ls_autotune(self.ctx, int(reps), ctypes.byref(st), ctypes.byref(pct), ctypes.byref(ppt)),
              "ls_autotune")
        return st.value, pct.value, ppt.value

    def set_step_config(self, stages, grid_pct, ppt=8):
        check(self.lib.ls_set_step_config(self.ctx, int(stages), int(grid_pct), int(ppt)), "ls_set_step_config")

    # -- learned corrector --------------------------------------------------
    def learned_init(self, seed=0):
        check(self.lib.ls_learned_init(self.ctx, ctypes.c_ulonglong(seed)), "ls_learned_init")

    def learned_params(self):
        n = ctypes.c_longlong(0)
        check(self.lib.ls_learned_num_params(ctypes.byref(n)), "ls_learned_num_params")
        out = np.empty(n.value, dtype=np.float32)
        check(self.lib.ls_learned_get_params(self.ctx, ctypes.c_void_p(out.ctypes.data), n.value),
              "ls_learned_get_params")
        return out

    def learned_set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(self.lib.ls_learned_set_params(self.ctx, ctypes.c_void_p(p.ctypes.data), p.size),
              "ls_learned_set_params")

    def learned_add_pair(self, phi_n, phi_ref, F):
        ptrs, devs = zip(*(array_ptr(a, np.float32, self.count) for a in (phi_n, phi_ref, F)))
        if len(set(devs)) != 1:
            raise ValueError("pair arrays must all be on the device or all on the host")
        check(self.lib.ls_learned_add_pair(self.ctx, ptrs[0], ptrs[1], ptrs[2], devs[0]),
              "ls_learned_add_pair")

    def learned_train(self, iters, lr, dt, halfwidth, seed=0):
        """Adam on the stored pairs (ls_learned_train_stored); returns the last loss."""
        loss = ctypes.c_double(0.0)
        check(self.lib.ls_learned_train_stored(self.ctx, int(iters), float(lr), float(dt), float(halfwidth),
                                               ctypes.c_ulonglong(seed), ctypes.byref(loss)),
              "ls_learned_train_stored")
        return loss.value

    def learned_num_pairs(self):
        n = ctypes.c_longlong(0)
        check(self.lib.ls_learned_num_pairs(self.ctx, ctypes.byref(n)), "ls_learned_num_pairs")
        return n.value

    def learned_train_spec(self, spec, iters, lr):
        """ls_learned_train with a pair specification string; returns the last loss."""
        loss = ctypes.c_double(0.0)
        check(self.lib.ls_learned_train(self.ctx, None if spec is None else spec.encode(), int(iters),
                                        float(lr), ctypes.byref(loss)), "ls_learned_train")
        return loss.value

    def learned_load(self, bf16):
        """Parameters from a BF16 image (numpy uint16 / bytes of 2 * num_params bytes)."""
        buf = np.ascontiguousarray(np.frombuffer(bytes(bf16), dtype=np.uint16))
        check(self.lib.ls_learned_load(self.ctx, buf.ctypes.data, buf.nbytes), "ls_learned_load")

    def learned_save(self):
        n = ctypes.c_longlong(0)
        check(self.lib.ls_learned_num_params(ctypes.byref(n)), "ls_learned_num_params")
        out = np.empty(n.value, dtype=np.uint16)
        check(self.lib.ls_learned_save(self.ctx, out.ctypes.data, out.nbytes), "ls_learned_save")
        return out

    def learned_get_pair(self, i):
        shape = self.shape
        a, b, f = (np.empty(shape, dtype=np.float32) for _ in range(3))
        check(self.lib.ls_learned_get_pair(self.ctx, int(i), a.ctypes.data, b.ctypes.data, f.ctypes.data, 0),
              "ls_learned_get_pair")
        return a, b, f

    def set_step_mode(self, mode):
        check(self.lib.ls_set_step_mode(self.ctx, int(mode)), "ls_set_step_mode")

    def output_open(self, prefix, every, fmt=LS_OUTPUT_VTS, slots=2):
        check(self.lib.ls_output_open(self.ctx, str(prefix).encode(), int(every), int(fmt), int(slots)),
              "ls_output_open")

    def output_stats(self):
        r = OutputReport()
        check(self.lib.ls_output_stats(self.ctx, ctypes.byref(r)), "ls_output_stats")
        return {k: getattr(r, k) for k, _ in OutputReport._fields_}

    def output_close(self):
        r = OutputReport()
        check(self.lib.ls_output_close(self.ctx, ctypes.byref(r)), "ls_output_close")
        return {k: getattr(r, k) for k, _ in OutputReport._fields_}

    def set_scheme(self, scheme, beta_in_h=0.0, reinit_iters=-1, dtau_in_h=0.5):
        check(self.lib.ls_set_scheme(self.ctx, int(scheme), float(beta_in_h), int(reinit_iters),
                                     float(dtau_in_h)), "ls_set_scheme")

    def set_steps_per_pass(self, steps):
        check(self.lib.ls_set_steps_per_pass(self.ctx, int(steps)), "ls_set_steps_per_pass")

    def steps_per_pass(self):
        k = ctypes.c_int(0)
        check(self.lib.ls_get_steps_per_pass(self.ctx, ctypes.byref(k)), "ls_get_steps_per_pass")
        return k.value

    def set_dense_kernel(self, on=True):
        check(self.lib.ls_set_dense_kernel(self.ctx, int(bool(on))), "ls_set_dense_kernel")

    def set_dilation(self, neighbours):
        check(self.lib.ls_set_dilation(self.ctx, int(neighbours)), "ls_set_dilation")

    def set_rebuild_mode(self, mode):
        check(self.lib.ls_set_rebuild_mode(self.ctx, int(mode)), "ls_set_rebuild_mode")

    def band_breaches(self):
        n = ctypes.c_ulonglong(0)
        check(self.lib.ls_band_breaches(self.ctx, ctypes.byref(n)), "ls_band_breaches")
        return n.value

    def learned_fallbacks(self):
        n = ctypes.c_ulonglong(0)
        check(self.lib.ls_learned_fallbacks(self.ctx, ctypes.byref(n)), "ls_learned_fallbacks")
        return n.value

    def profile_enable(self, on=True):
        """True / False, or an int N >= 1: time one run of stencil launches in N."""
        check(self.lib.ls_profile_enable(self.ctx, int(on)), "ls_profile_enable")

    def profile(self):
        p = Profile()
        check(self.lib.ls_get_profile(self.ctx, ctypes.byref(p)), "ls_get_profile")
        return {k: getattr(p, k) for k, _ in Profile._fields_}

    def reset_profile(self):
        check(self.lib.ls_reset_profile(self.ctx), "ls_reset_profile")


class Batch(LevelSet):
    """A batched context: n independent grids advanced by one stencil launch
    per step (ls_batch_create).  Per-instance calls take the instance index."""

    def __init__(self, edges, hs, precision=LS_FP32, stream=None):
        self.lib = load()
        self.n = len(edges)
        nx = [int(e[0]) if hasattr(e, "__len__") else int(e) for e in edges]
        ny = [int(e[1]) if hasattr(e, "__len__") else int(e) for e in edges]
        nz = [int(e[2]) if hasattr(e, "__len__") else int(e) for e in edges]
        self.shapes = [(z, y, x) for x, y, z in zip(nx, ny, nz)]
        self.precision = precision
        self.dtype = np.float32 if precision == LS_FP32 else np.float64
        arr_i = ctypes.c_int * self.n
        arr_d = ctypes.c_double * self.n
        h_ = ctypes.c_void_p()
        check(self.lib.ls_batch_create(self.n, arr_i(*nx), arr_i(*ny), arr_i(*nz),
                                       arr_d(*[float(h) for h in hs]), int(precision), ctypes.byref(h_)),
              "ls_batch_create")
        self.ctx = h_
        self.shape = None
        self.count = None
        if stream is None and torch is not None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        if stream is not None:
            check(self.lib.ls_set_stream(self.ctx, ctypes.c_void_p(stream)), "ls_set_stream")

    def _count(self, i):
        z, y, x = self.shapes[i]
        return x * y * z

    def set_phi_i(self, i, a):
        p, dev = array_ptr(a, self.dtype, self._count(i))
        check(self.lib.ls_inst_set_phi(self.ctx, int(i), p, dev), "ls_inst_set_phi")

    def set_speed_i(self, i, a):
        p, dev = array_ptr(a, self.dtype, self._count(i))
        check(self.lib.ls_inst_set_speed(self.ctx, int(i), p, dev), "ls_inst_set_speed")

    def init_phi_i(self, i, shape, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        check(self.lib.ls_inst_init_phi(self.ctx, int(i), int(shape), ctypes.c_void_p(p.ctypes.data), p.size),
              "ls_inst_init_phi")

    def set_speed_const_i(self, i, F):
        check(self.lib.ls_inst_set_speed_const(self.ctx, int(i), float(F)), "ls_inst_set_speed_const")

    def get_phi_i(self, i, out=None):
        if out is None:
            out = np.empty(self.shapes[i], dtype=self.dtype)
        p, dev = array_ptr(out, self.dtype, self._count(i))
        check(self.lib.ls_inst_get_phi(self.ctx, int(i), p, dev), "ls_inst_get_phi")
        return out

    def active_tiles_i(self, i):
        n = ctypes.c_longlong(0)
        check(self.lib.ls_inst_get_active_tiles(self.ctx, int(i), None, 0, ctypes.byref(n)),
              "ls_inst_get_active_tiles")
        buf = np.empty(max(n.value, 1), dtype=np.int32)
        check(self.lib.ls_inst_get_active_tiles(self.ctx, int(i), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                n.value, ctypes.byref(n)), "ls_inst_get_active_tiles")
        return buf[:n.value].copy()

    def last_dt_i(self, i):
        d = ctypes.c_double(0.0)
        check(self.lib.ls_inst_last_dt(self.ctx, int(i), ctypes.byref(d)), "ls_inst_last_dt")
        return d.value
