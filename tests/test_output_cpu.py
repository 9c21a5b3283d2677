"""The VTK XML writer of the overlapped output (section 2's output files),
called on host arrays: layout, point coordinates, image geometry, errors.
Needs the library but no GPU."""
import os

import numpy as np
import pytest

from paper_1612_04040_b300 import native as ls

import _vtk


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("fmt", [ls.LS_OUTPUT_VTS, ls.LS_OUTPUT_VTI])
def test_written_file_holds_the_array(tmp_path, dtype, fmt):
    g = np.random.default_rng(2)
    phi = g.standard_normal((5, 6, 7)).astype(dtype)
    h = 0.125
    path = tmp_path / ("a.vts" if fmt == ls.LS_OUTPUT_VTS else "a.vti")
    ls.write_vtk(path, phi, h, fmt)
    kind, ext, attrs, arrays = _vtk.read(str(path))
    assert ext == (7, 6, 5)
    got = arrays["phi"]
    assert got.dtype == dtype and np.array_equal(got, phi)
    c = lambda n: (np.arange(n) + 0.5) * h
    if fmt == ls.LS_OUTPUT_VTS:
        assert kind == "StructuredGrid"
        P = arrays["Points"].astype(np.float64)
        Z, Y, X = np.meshgrid(c(5), c(6), c(7), indexing="ij")
        assert np.array_equal(P[..., 0], X.astype(dtype)) and np.array_equal(P[..., 1], Y.astype(dtype))
        assert np.array_equal(P[..., 2], Z.astype(dtype))
    else:
        assert kind == "ImageData"
        assert [float(v) for v in attrs["Origin"].split()] == [h / 2] * 3
        assert [float(v) for v in attrs["Spacing"].split()] == [h] * 3


def test_errors(tmp_path):
    phi = np.zeros((2, 2, 2), np.float32)
    with pytest.raises(ls.LSError) as e:
        ls.write_vtk(tmp_path / "missing_dir" / "x.vts", phi, 1.0)
    assert e.value.status == ls.LS_EIO
    with pytest.raises(ls.LSError) as e:
        ls.write_vtk(tmp_path / "x.vts", phi, 0.0)
    assert e.value.status == ls.LS_EINVAL
    with pytest.raises(ls.LSError) as e:
        ls.write_vtk(tmp_path / "x.vts", phi, 1.0, fmt=7)
    assert e.value.status == ls.LS_EINVAL
    assert not os.path.exists(tmp_path / "x.vts")
