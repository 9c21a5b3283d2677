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
