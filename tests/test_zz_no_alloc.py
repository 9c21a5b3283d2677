"""ls_band_tiles_noalloc: the allocation-free band tile list.

Callers that cannot allocate device memory (code running during someone
else's graph capture, allocation-free real-time sections, hosts whose memory
pool owns the device) use this entry point; it must give exactly the
active-tile list of the context path (ls_band_rebuild + ls_get_active_tiles),
here on two calls in a row with different inputs, since every call reuses the
same fixed scratch array.  The file name sorts last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


def context_tiles(phi, h, halfwidth, prec):
    nz, ny, nx = phi.shape
    g = ls.LevelSet(nx, ny, nz, h, prec)
    g.set_phi(phi)
    g.band_rebuild(halfwidth)
    ids = g.active_tiles()
    g.close()
    return ids


def test_noalloc_matches_context_path_twice(cuda_ok):
    ls.load()
    w = inputs.SphereUnion(n=128, count=12)
    cases = [
        (w.phi().numpy().astype(np.float32), w.h, 6.0, ls.LS_FP32),
        (inputs.torus_sdf((64, 96, 80), 1.0 / 64, (0.6, 0.7, 0.5), (0.0, 0.6, 0.8), 0.3, 0.1)
         .numpy(), 1.0 / 64, 4.0, ls.LS_FP64),
    ]
    ntiles_max = max(p.size // 512 for p, _, _, _ in cases)
    tiles = torch.full((ntiles_max,), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    for phi, h, hw, prec in cases:
        expect = context_tiles(phi, h, hw, prec)
        assert expect.size > 0
        d_phi = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        ls.band_tiles_noalloc(d_phi, h, hw, tiles, count)
        torch.cuda.synchronize()
        n = int(count.item())
        assert n == expect.size
        assert np.array_equal(tiles[:n].cpu().numpy(), expect)


def test_noalloc_rejects_bad_scalars_with_real_buffers(cuda_ok):
    """Arguments the host rejects (non-finite or non-positive h or halfwidth,
    too small an output) come back as LS_EINVAL with nothing queued; the
    buffers are real device memory, so a broken check could not reach a
    wild address either."""
    ls.load()
    phi = torch.ones((16, 16, 16), dtype=torch.float32, device="cuda")
    tiles = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    inf, nan = float("inf"), float("nan")
    for h, hw in ((inf, 2.0), (-inf, 2.0), (nan, 2.0), (0.0, 2.0), (1.0 / 16, inf), (1.0 / 16, nan),
                  (1.0 / 16, -1.0), (1e300, 1e300)):
        with pytest.raises(ls.LSError) as e:
            ls.band_tiles_noalloc(phi, h, hw, tiles, count)
        assert e.value.status == ls.LS_EINVAL, (h, hw)
    with pytest.raises(ls.LSError) as e:
        ls.band_tiles_noalloc(phi, 1.0 / 16, 2.0, tiles[:7], count)   # 8 tiles need tiles_cap >= 8
    assert e.value.status == ls.LS_EINVAL
    torch.cuda.synchronize()
    assert int(count.item()) == -7 and int(tiles.min().item()) == -7
