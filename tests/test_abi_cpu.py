"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/*.h declares; argument errors that are
decided on the host come back as status codes."""
import ctypes
import glob
import os
import re

import pytest

from paper_1612_04040_b300 import build as lsbuild
from paper_1612_04040_b300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ls_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    lsbuild.build()
    return native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ls_create", "ls_destroy", "ls_set_stream", "ls_set_phi", "ls_set_speed",
                     "ls_set_speed_const", "ls_band_rebuild", "ls_step", "ls_set_full_domain",
                     "ls_get_phi", "ls_get_active_tiles", "ls_get_status", "ls_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert declared_functions() <= set(native.SIGNATURES)


def test_build_targets_sm103a_only():
    assert lsbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_argument_errors(lib):
    out = ctypes.c_void_p()
    assert lib.ls_create(12, 16, 16, 0.1, 0, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_create(16, 16, 0, 0.1, 0, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_create(16, 16, 16, -1.0, 0, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_create(16, 16, 16, float("nan"), 0, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_create(16, 16, 16, 0.1, 7, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_create(16, 16, 16, 0.1, 0, None) == native.LS_EINVAL
    assert lib.ls_create(2048, 2048, 1024, 0.1, 0, ctypes.byref(out)) == native.LS_EINVAL
    assert lib.ls_destroy(None) == native.LS_OK
    assert lib.ls_step(None, 1, 0.5, 1, 5, None) == native.LS_EINVAL
    assert lib.ls_get_status(None) == native.LS_EINVAL
    assert lib.ls_strerror(native.LS_ENONFINITE).decode() == "non-finite value in input"


_NEWER_CALLS_CHILD = r"""
import ctypes, sys
sys.path.insert(0, %(root)r)
from paper_1612_04040_b300 import native
lib = native.load()
P = ctypes.c_void_p(256)      # placeholder, never dereferenced when a check holds
d = ctypes.c_double(0.0)
n = ctypes.c_longlong(0)
codes = [
    lib.ls_set_ghost_rows(None, 1, 0),
    lib.ls_band_refresh(None, ctypes.byref(d), ctypes.byref(n)),
    lib.ls_band_row_counts(None, P, 1),
    lib.ls_get_tile_rows(None, 0, 1, -1, P, 1),
    lib.ls_set_tile_rows(None, 0, 1, -1, P, 1),
    lib.ls_copy_ghost_row(None, 0, None, 0, -1),
    lib.ls_band_speed_bound(None, P, 1),
    lib.ls_set_dt_from_bound(None, P, 0.5),
    lib.ls_get_speed(None, P, 1),
    lib.ls_learned_features(None, P, None, 0.0, 1.0, 1, P, None),
    lib.ls_learned_features(P, P, None, 0.0, float("nan"), 1, P, None),
    lib.ls_learned_features(P, P, None, 0.0, 1.0, 0, P, None),
    lib.ls_learned_loss_grad(P, P, P, P, 8, 1.0, -1.0, P, P, P, None),
    lib.ls_adam_step(P, P, P, P, 8, 1e-3, 0, None),               # step t >= 1
    lib.ls_adam_step(P, P, P, P, 8, float("inf"), 1, None),
    lib.ls_conv3_wgrad(P, P, 48, 16, 16, 16, 16, P, P, P, None),  # nx not a multiple of 64
    lib.ls_conv3_wgrad(P, P, 64, 16, 16, 16, 16, P, P, None, None),  # no status word
    lib.ls_step(None, 1, 1.0, native.LS_DT_KEEP, 5, None),
    lib.ls_set_rebuild_mode(None, native.LS_REBUILD_FULL),
]
print(",".join(str(c) for c in codes))
"""


def test_newer_calls_refuse_bad_arguments_on_the_host():
    """The slab-split, learned-primitive and dt calls refuse NULL contexts
    and bad arguments before any CUDA call.  Run in a child process that sees
    no CUDA device, so even a broken check could only end in a CUDA error
    status, never in a kernel reading the placeholder pointers."""
    import subprocess
    import sys
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", _NEWER_CALLS_CHILD % {"root": ROOT}], env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    codes = [int(v) for v in out.stdout.strip().splitlines()[-1].split(",")]
    assert codes == [native.LS_EINVAL] * len(codes), codes


def _struct_fields(header, name):
    """Field names of `typedef struct { ... } name;` in the header, in order."""
    body = re.search(r"typedef struct \{([^{}]*)\} %s;" % name, header).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return [m.group(1) for m in re.finditer(r"(\w+)\s*;", body)]


def test_binding_structs_match_the_header():
    """The ctypes mirrors of ls_profile and ls_output_report list the
    header's fields in the header's order (a field added on one side only
    would shift every later one)."""
    header = open(os.path.join(ROOT, "include", "ls.h")).read()
    assert [f for f, _ in native.Profile._fields_] == _struct_fields(header, "ls_profile")
    assert [f for f, _ in native.OutputReport._fields_] == _struct_fields(header, "ls_output_report")
