"""The oracle against the hand-derived closed-form values of
tests/golden/closed_forms.txt (Eq. 7 cut-off, Eq. 3-5 plane-front step):
exact FP64 equality."""
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _records(kind):
    out = []
    with open(os.path.join(HERE, "golden", "closed_forms.txt")) as f:
        for line in f:
            parts = line.split("#", 1)[0].split()
            if parts and parts[0] == kind:
                out.append([float(v) for v in parts[1:]])
    return out


def test_cutoff_closed_forms():
    recs = _records("cutoff")
    assert len(recs) == 7
    for beta, gamma, a, c in recs:
        assert oracle.cutoff(a, beta, gamma) == c, (beta, gamma, a)


def test_plane_front_step_closed_forms():
    recs = _records("plane")
    assert len(recs) == 5
    for n, F, i, expected in recs:
        n, i = int(n), int(i)
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h - 0.25
        phi = np.broadcast_to(x[None, None, :], (n, n, n)).copy()
        out = oracle.step(phi, h, h / 2, Fc=F)
        assert np.all(out[:, :, i] == expected), (n, F, i, out[0, 0, i])
