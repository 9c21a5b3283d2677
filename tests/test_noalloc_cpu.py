"""Host-side checks of the allocation-free band tile list: the binding
refuses unsupported dtypes and buffers before it reaches the library, and
the library refuses bad sizes and scalars before its first CUDA call.  The
library part runs in a child process that sees no CUDA device, so even a
broken check could only end in a CUDA error status, never in a kernel
reading the placeholder pointers."""
import os
import subprocess
import sys

import pytest
import torch

from paper_1612_04040_b300 import build as lsbuild
from paper_1612_04040_b300 import native as ls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lsbuild.build()
    ls.load()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16, torch.int32, torch.int64])
def test_binding_rejects_phi_dtypes(dtype):
    phi = torch.zeros((8, 8, 8), dtype=dtype)
    tiles = torch.zeros(1, dtype=torch.int32)
    count = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(TypeError):
        ls.band_tiles_noalloc(phi, 1.0, 2.0, tiles, count)


def test_binding_rejects_output_dtypes_and_host_buffers():
    phi = torch.zeros((8, 8, 8), dtype=torch.float32)
    with pytest.raises(TypeError):
        ls.band_tiles_noalloc(phi, 1.0, 2.0, torch.zeros(1, dtype=torch.int64),
                              torch.zeros(1, dtype=torch.int32))
    with pytest.raises(TypeError):
        ls.band_tiles_noalloc(phi, 1.0, 2.0, torch.zeros(1, dtype=torch.int32),
                              torch.zeros(1, dtype=torch.float32))
    with pytest.raises(ValueError):   # host tensors are not device buffers
        ls.band_tiles_noalloc(phi, 1.0, 2.0, torch.zeros(1, dtype=torch.int32),
                              torch.zeros(1, dtype=torch.int32))


_CHILD = r"""
import ctypes, sys
sys.path.insert(0, %(root)r)
from paper_1612_04040_b300 import native as ls
lib = ls.load()
P = ctypes.c_void_p(256)      # placeholder, never dereferenced when a check holds
M = 1 << 21
inf, nan = float("inf"), float("nan")
cases = [
    (P, 8, 8, 8 * (M + 1), 1.0, 0, 2.0, P, M + 1, P),   # more tiles than the scratch holds
    (P, 8, 8, 8, inf, 0, 2.0, P, 1, P),
    (P, 8, 8, 8, nan, 0, 2.0, P, 1, P),
    (P, 8, 8, 8, 1.0, 0, inf, P, 1, P),
    (P, 8, 8, 8, 1.0, 0, -2.0, P, 1, P),
    (P, 8, 8, 8, 1e300, 0, 1e300, P, 1, P),             # gamma overflows to inf
    (P, 8, 8, 8, 1.0, 2, 2.0, P, 1, P),                 # no such precision
    (P, 12, 8, 8, 1.0, 0, 2.0, P, 1, P),                # not a multiple of 8
    (P, 16, 8, 8, 1.0, 0, 2.0, P, 1, P),                # tiles_cap 1 < 2 tiles
    (None, 8, 8, 8, 1.0, 0, 2.0, P, 1, P),
    (P, 8, 8, 8, 1.0, 0, 2.0, P, 1, None),
]
print(",".join(str(lib.ls_band_tiles_noalloc(*(c + (None,)))) for c in cases))
"""


def test_library_rejects_on_the_host_before_any_cuda_call():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", _CHILD % {"root": ROOT}], env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    codes = [int(v) for v in out.stdout.strip().splitlines()[-1].split(",")]
    assert codes == [ls.LS_EINVAL] * len(codes), codes
