"""Overlapped output (section 2's output strategy) on the GPU: the files
written by the host writer thread while ls_step keeps running hold exactly
the states after the snapshot steps."""
import numpy as np
import pytest

from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

import _vtk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def pair(local=False):
    w = inputs.SphereUnion(n=64, count=5)
    p = w.phi().numpy().astype(np.float32)
    F = w.speed().numpy().astype(np.float32)
    out = []
    for _ in range(2):
        g = ls.LevelSet(64, 64, 64, w.h, ls.LS_FP32)
        g.set_phi(p)
        g.set_speed(F)
        g.band_rebuild(6.0)
        if local:
            g.set_scheme(ls.LS_SCHEME_LOCAL, 3.0, 4, 0.5)
        out.append(g)
    return out


@pytest.mark.parametrize("fmt,graphs,local", [(ls.LS_OUTPUT_VTS, False, False),
                                              (ls.LS_OUTPUT_VTI, True, False),
                                              (ls.LS_OUTPUT_VTI, False, True)])
def test_snapshots_hold_the_states(tmp_path, fmt, graphs, local):
    a, b = pair(local)
    a.set_graphs(graphs)
    a.output_open(str(tmp_path / "run_"), every=3, fmt=fmt, slots=2)
    a.step(10, 0.5, ls.LS_DT_CFL, 5)      # snapshots after steps 3, 6, 9
    a.step(2, 0.5, ls.LS_DT_CFL, 5)       # and 12
    rep = a.output_close()
    assert rep["files"] == 4 and rep["status"] == ls.LS_OK and rep["bytes"] > 4 * 64 ** 3 * 4
    ext = ".vts" if fmt == ls.LS_OUTPUT_VTS else ".vti"
    for k in (3, 6, 9, 12):
        b.step(3, 0.5, ls.LS_DT_CFL, 5)
        _, _, _, arrays = _vtk.read(str(tmp_path / ("run_%08d%s" % (k, ext))))
        assert np.array_equal(arrays["phi"].view(np.int32), b.get_phi().view(np.int32)), k


def test_state_errors(tmp_path):
    a, _ = pair()
    a.output_open(str(tmp_path / "x_"), every=1)
    with pytest.raises(ls.LSError) as e:
        a.output_open(str(tmp_path / "y_"), every=1)
    assert e.value.status == ls.LS_ESTATE
    a.output_close()
    assert a.output_close()["files"] == 0          # nothing attached: a no-op
    for args in [("z_", 0), ("z_", 1, 5), ("z_", 1, ls.LS_OUTPUT_VTS, 0)]:
        with pytest.raises(ls.LSError) as e:
            a.output_open(str(tmp_path / args[0]), *args[1:])
        assert e.value.status == ls.LS_EINVAL
    bt = ls.Batch([16, 24], [1 / 16, 1 / 24])
    with pytest.raises(ls.LSError) as e:
        bt.output_open(str(tmp_path / "b_"), 1)
    assert e.value.status == ls.LS_EINVAL


def test_unwritable_prefix_reports_io_error(tmp_path):
    a, _ = pair()
    a.output_open(str(tmp_path / "no_such_dir" / "x_"), every=2)
    a.step(4, 0.5, ls.LS_DT_CFL, 5)
    with pytest.raises(ls.LSError) as e:
        a.output_close()
    assert e.value.status == ls.LS_EIO
