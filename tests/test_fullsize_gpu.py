"""Parity at the standard workloads' full sizes, in the launch configuration
the benchmark times.  The oracle cannot run these grids end to end, so the
checks are (a) one step of Eq. 3-5 recomputed by the oracle on sampled tiles
of the GPU's own state (each sampled tile with its one-cell halo, clipped at
the domain faces so the face rule applies there), within 1e-5 h for FP32
and bit for bit for FP64; (b) frozen points unchanged; (c) the band
rebuilt from that state equals the oracle's tube test + dilation of it."""
import numpy as np
import pytest
import torch

import oracle
from paper_1612_04040_b300 import inputs
from paper_1612_04040_b300 import native as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ok):
    ls.load()


def tile_block(a, tz, ty, tx):
    """Tile (tz, ty, tx) of a (nz, ny, nx) tensor with a one-cell halo,
    clipped to the domain; returns (block, offsets of the tile inside it)."""
    nz, ny, nx = a.shape
    lo = [max(0, 8 * t - 1) for t in (tz, ty, tx)]
    hi = [min(n, 8 * t + 9) for t, n in zip((tz, ty, tx), (nz, ny, nx))]
    blk = a[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    return blk, [8 * t - l for t, l in zip((tz, ty, tx), lo)]


def check_sampled_step(before, after, F, Fc, h, dt, tiles, tshape, ntiles_sample, seed, exact,
                       band=None):
    """before/after: device tensors (nz, ny, nx); F: device tensor or None.
    band: compare only points with |phi| < band (full-domain FP32 runs, where
    far from the front |phi| ~ 1 and one FP32 ulp exceeds the band bar)."""
    tnz, tny, tnx = tshape
    g = np.random.default_rng(seed)
    pick = g.choice(tiles, size=min(ntiles_sample, len(tiles)), replace=False)
    # always include tiles touching the domain faces if there are any
    edge = [t for t in tiles if (t % tnx in (0, tnx - 1)) or ((t // tnx) % tny in (0, tny - 1))
            or (t // (tnx * tny) in (0, tnz - 1))]
    pick = np.unique(np.concatenate([pick, np.asarray(edge[:16], dtype=pick.dtype)]))
    worst = 0.0
    for t in pick:
        tz, ty, tx = int(t) // (tnx * tny), (int(t) // tnx) % tny, int(t) % tnx
        blk, o = tile_block(before, tz, ty, tx)
        b = blk.double().cpu().numpy()
        Fb = None if F is None else tile_block(F, tz, ty, tx)[0].double().cpu().numpy()
        ref = oracle.step(b, h, dt, F=Fb, Fc=Fc)[o[0]:o[0] + 8, o[1]:o[1] + 8, o[2]:o[2] + 8]
        got = after[8 * tz:8 * tz + 8, 8 * ty:8 * ty + 8, 8 * tx:8 * tx + 8].double().cpu().numpy()
        if exact:
            assert np.array_equal(got.view(np.int64), ref.view(np.int64)), int(t)
        else:
            d = np.abs(got - ref)
            if band is not None:
                near = np.abs(b[o[0]:o[0] + 8, o[1]:o[1] + 8, o[2]:o[2] + 8]) < band
                d = d[near] if near.any() else np.zeros(1)
            worst = max(worst, float(np.max(d)))
    return worst


def band_from(state, gamma):
    core = oracle.classify(state.double().cpu().numpy(), gamma)
    return oracle.compact(oracle.dilate(core, 26))


@pytest.mark.parametrize("config", [(3, 100, 4), (2, 100, 16)])
def test_sphere_union_512(config):
    """512^3 FP32, 20 spheres, sinusoidal F, band 6h, rebuild every 5, CFL 0.5,
    with 4 points per thread and with the one-warp-per-tile decomposition the
    autotuner picks for this workload."""
    w = inputs.SphereUnion()
    dev = torch.device("cuda")
    phi0 = w.phi(device=dev).to(torch.float32).contiguous()
    F = w.speed(device=dev).to(torch.float32).contiguous()
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32)
    g.set_step_config(*config)
    g.set_speed(F)
    g.set_phi(phi0)
    g.band_rebuild(w.halfwidth)
    g.step(23, w.cfl, ls.LS_DT_CFL, w.rebuild_every)   # since the last rebuild: 3 steps
    before = torch.empty_like(phi0)
    g.get_phi(before)
    tiles = g.active_tiles()
    dt = g.step(1, w.cfl, ls.LS_DT_CFL, w.rebuild_every, want_dt=True)
    after = torch.empty_like(phi0)
    g.get_phi(after)
    worst = check_sampled_step(before, after, F, 0.0, w.h, dt, tiles, (64, 64, 64), 300, 1, False)
    assert worst <= 1e-5 * w.h, worst
    # frozen points: everything outside the active tiles is unchanged
    act = np.zeros(64 ** 3, dtype=bool)
    act[tiles] = True
    mask = torch.from_numpy(np.repeat(np.repeat(np.repeat(act.reshape(64, 64, 64), 8, 0), 8, 1), 8, 2)).cuda()
    assert torch.equal(before[~mask], after[~mask])
    # the next rebuild (after one more step) equals the oracle's band of the
    # state it is built from
    g.step(1, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    state = torch.empty_like(phi0)
    g.get_phi(state)
    g.step(1, w.cfl, ls.LS_DT_CFL, w.rebuild_every)   # rebuilds from `state`, then steps
    assert np.array_equal(g.active_tiles(), band_from(state, w.halfwidth * w.h))


@pytest.mark.parametrize("scheme", ["plain", "local"])
def test_sphere_union_512_incremental_rebuild_equals_full_scan(scheme):
    """The periodic rebuilds marked from the core entries of the previous
    list (the tube test fused into the last step, or, in the local scheme,
    into its last reinitialisation pass) give, on the 512^3 workload in the
    benchmark's launch configuration over 40 steps, the list, the dt and the
    bits (the frozen x-face copies and the leaving tiles' values included)
    of rebuilds that walk every tile."""
    w = inputs.SphereUnion()
    runs = []
    for mode in (ls.LS_REBUILD_FULL, ls.LS_REBUILD_INCREMENTAL):
        g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32)
        g.set_step_config(2, 100, 16)
        g.set_rebuild_mode(mode)
        g.init_speed(ls.LS_SPEED_SINUSOID)
        g.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(w.centres, w.radii))
        if scheme == "local":
            g.set_scheme(ls.LS_SCHEME_LOCAL, 3.0, 12, 0.5)
        g.band_rebuild(w.halfwidth)
        g.step(40, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
        dt = g.step(1, w.cfl, ls.LS_DT_CFL, w.rebuild_every, want_dt=True)
        out = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
        g.get_phi(out)
        runs.append((g.active_tiles(), dt, out))
        g.close()
    (la, da, pa), (lb, db, pb) = runs
    assert len(la) > 10000
    assert np.array_equal(la, lb)
    assert da == db
    assert torch.equal(pa, pb)


def test_maximum_grid_fp32():
    """The largest grid the ABI accepts: 2^31 points (nx = ny = 1024,
    nz = 2048; 2^22 tiles, element offsets up to 2^31 - 1), FP32, three
    spheres, one of them cut by the top z face so that the highest tile ids
    are active; sampled one-step parity, frozen points unchanged."""
    nz, ny, nx = 2048, 1024, 1024
    h = 1.0 / 1024
    shape = (nz, ny, nx)
    dev = torch.device("cuda")
    centres = [(0.5, 0.5, 0.5), (0.3, 0.6, 1.2), (0.55, 0.45, 1.9)]
    radii = [0.2, 0.15, 0.2]
    phi0 = inputs.sphere_union_sdf(shape, h, centres, radii, device=dev, out_dtype=torch.float32)
    F = inputs.speed_sinusoid(shape, h, device=dev, out_dtype=torch.float32)
    g = ls.LevelSet(nx, ny, nz, h, ls.LS_FP32)
    g.set_step_config(2, 100, 16)  # the largest element offsets in the one-warp kernel
    g.set_speed(F)
    g.set_phi(phi0)
    del phi0
    g.band_rebuild(6.0)
    g.step(3, 0.5, ls.LS_DT_CFL, 5)
    before = torch.empty(shape, dtype=torch.float32, device=dev)
    g.get_phi(before)
    tiles = g.active_tiles()
    tshape = (nz // 8, ny // 8, nx // 8)
    assert tiles.max() >= tshape[0] * tshape[1] * tshape[2] - tshape[1] * tshape[2]  # top layer
    dt = g.step(1, 0.5, ls.LS_DT_CFL, 5, want_dt=True)
    after = torch.empty_like(before)
    g.get_phi(after)
    worst = check_sampled_step(before, after, F, 0.0, h, dt, tiles, tshape, 200, 3, False)
    assert worst <= 1e-5 * h, worst
    act = torch.zeros(tshape[0] * tshape[1] * tshape[2], dtype=torch.bool, device=dev)
    act[torch.from_numpy(tiles.astype(np.int64)).to(dev)] = True
    mask = act.view(tshape).repeat_interleave(8, 0).repeat_interleave(8, 1).repeat_interleave(8, 2)
    assert torch.equal(before[~mask], after[~mask])
    assert g.status() == ls.LS_OK


@pytest.fixture(scope="module")
def perturbed_1024():
    w = inputs.PerturbedSphere()
    dev = torch.device("cuda")
    return w, w.phi(device=dev).contiguous(), w.speed(device=dev).contiguous()


@pytest.mark.parametrize("prec", [ls.LS_FP32, ls.LS_FP64])
@pytest.mark.parametrize("full_domain", [False, True])
def test_perturbed_sphere_1024(perturbed_1024, prec, full_domain):
    """1024^3, spherical-harmonic sphere, F = cos 4 pi x cos 4 pi y
    (sign-changing), band 6h; FP32 and FP64, narrow band and full domain."""
    w, phi64, F64 = perturbed_1024
    dev = torch.device("cuda")
    dt_t = torch.float32 if prec == ls.LS_FP32 else torch.float64
    F = F64.to(dt_t).contiguous()
    g = ls.LevelSet(w.n, w.n, w.n, w.h, prec)
    if prec == ls.LS_FP32:
        g.set_step_config(2, 100 if not full_domain else 50, 16)  # the benchmark's picks
    g.set_speed(F)
    g.set_phi(phi64.to(dt_t).contiguous())
    if full_domain:
        g.set_full_domain(True)
    else:
        g.band_rebuild(w.halfwidth)
    g.step(8, 0.5, ls.LS_DT_CFL, 5)
    before = torch.empty((w.n,) * 3, dtype=dt_t, device=dev)
    g.get_phi(before)
    tiles = g.active_tiles()
    dt = g.step(1, 0.5, ls.LS_DT_CFL, 5, want_dt=True)
    after = torch.empty_like(before)
    g.get_phi(after)
    exact = prec == ls.LS_FP64
    # band points: within the band (6h) plus the one-tile dilation (<= 16h more)
    band = 22 * w.h if full_domain else None
    worst = check_sampled_step(before, after, F, 0.0, w.h, dt, tiles, (128, 128, 128), 120, 2, exact,
                               band)
    if not exact:
        assert worst <= 1e-5 * w.h, worst
    g.close()


def test_batch_256_in_bench_configuration():
    """The 256-instance batch with the autotuned stencil and graph replay:
    sampled instances against the oracle on their whole grid, one step from
    the GPU's own state, plus their band sets."""
    insts = inputs.batch_instances()
    dev = torch.device("cuda")
    b = ls.Batch([i.edge for i in insts], [i.h for i in insts])
    for k, it in enumerate(insts):
        b.set_phi_i(k, it.phi(device=dev).to(torch.float32).contiguous())
        b.set_speed_const_i(k, it.speed)
    b.band_rebuild(4.0)
    b.step(5, 0.5, ls.LS_DT_CFL, 5)
    b.autotune(reps=3)
    b.set_graphs(True)
    for _ in range(3):
        b.step(6, 0.5, ls.LS_DT_CFL, 5)   # since the last rebuild: 3 steps
    sample = np.random.default_rng(3).choice(len(insts), size=10, replace=False)
    before = {int(k): b.get_phi_i(int(k)) for k in sample}
    tiles = {int(k): b.active_tiles_i(int(k)) for k in sample}
    b.set_graphs(False)
    b.step(1, 0.5, ls.LS_DT_CFL, 5)
    for k in sample:
        k = int(k)
        it = insts[k]
        out = b.get_phi_i(k).astype(np.float64)
        e = it.edge
        act = np.zeros((e // 8) ** 3, dtype=np.uint8)
        act[tiles[k]] = 1
        ref = oracle.step(before[k].astype(np.float64), it.h, b.last_dt_i(k), Fc=it.speed,
                          tile_active=act.reshape((e // 8,) * 3))
        assert np.max(np.abs(out - ref)) <= 1e-5 * it.h, k


def test_local_scheme_sphere_union_512():
    """The 512^3 sphere-union run with the local scheme (beta 3h, gamma 6h,
    12 reinitialisation iterations of dtau = h/2, clamp) in the benchmark's
    configuration: one step recomputed by the oracle on sampled tiles, each
    with a halo of 1 + 12 cells (one cell per pass), within (1 + 12) 1e-5 h;
    frozen points unchanged; no N point outside the active tiles."""
    w = inputs.SphereUnion()
    dev = torch.device("cuda")
    K = 12
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32)
    g.init_speed(ls.LS_SPEED_SINUSOID)
    g.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(w.centres, w.radii))
    g.set_scheme(ls.LS_SCHEME_LOCAL, 3.0, K, 0.5)
    g.band_rebuild(w.halfwidth)
    g.step(23, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    F = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    before = torch.empty_like(F)
    g.get_phi(before)
    tiles = g.active_tiles()
    dt = g.step(1, w.cfl, ls.LS_DT_CFL, w.rebuild_every, want_dt=True)
    after = torch.empty_like(before)
    g.get_phi(after)
    Fh = w.speed(out_dtype=torch.float32).numpy().astype(np.float64)
    pick = np.random.default_rng(4).choice(tiles, size=60, replace=False)
    halo = 1 + K
    worst = 0.0
    for t in pick:
        tz, ty, tx = int(t) // 4096, (int(t) // 64) % 64, int(t) % 64
        lo = [max(0, 8 * v - halo) for v in (tz, ty, tx)]
        hi = [min(w.n, 8 * v + 8 + halo) for v in (tz, ty, tx)]
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        blk = before[sl].double().cpu().numpy()
        ref, _ = oracle.local_step(blk, w.h, dt, 3.0 * w.h, w.halfwidth * w.h, K, 0.5 * w.h, F=Fh[sl])
        o = [8 * v - a for v, a in zip((tz, ty, tx), lo)]
        ref = ref[o[0]:o[0] + 8, o[1]:o[1] + 8, o[2]:o[2] + 8]
        got = after[8 * tz:8 * tz + 8, 8 * ty:8 * ty + 8, 8 * tx:8 * tx + 8].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - ref))))
    assert worst <= (1 + K) * 1e-5 * w.h, worst
    act = np.zeros(64 ** 3, dtype=bool)
    act[tiles] = True
    mask = torch.from_numpy(np.repeat(np.repeat(np.repeat(act.reshape(64, 64, 64), 8, 0), 8, 1), 8, 2)).cuda()
    assert torch.equal(before[~mask], after[~mask])
    assert g.band_breaches() == 0
    g.close()


def test_slab_split_512_equals_one_grid_bitwise():
    """The 512^3 sphere-union run split into two z-slabs on this GPU (the
    path bench.py --parallelism slab times: device-side dt, two rebuild
    periods per CUDA-graph replay, rows moved by Eq. 14 when that pays, the
    autotuner's stencil configuration) against one context, 100 steps: the
    same bits everywhere."""
    from paper_1612_04040_b300 import slab
    w = inputs.SphereUnion(n=512)
    g = ls.LevelSet(w.n, w.n, w.n, w.h, ls.LS_FP32)
    g.init_speed(ls.LS_SPEED_SINUSOID)
    g.init_phi(ls.LS_SHAPE_SPHERES, inputs.spheres_params(w.centres, w.radii))
    phi0 = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
    F0 = torch.empty_like(phi0)
    g.get_phi(phi0)
    g.get_speed(F0)
    g.set_step_config(2, 100, 16)
    g.band_rebuild(w.halfwidth, want_count=False)
    g.step(100, w.cfl, ls.LS_DT_CFL, w.rebuild_every)
    ref = torch.empty_like(phi0)
    g.get_phi(ref)
    g.close()
    stream = torch.cuda.Stream()

    def make(nx, ny, rows, h, lo, hi):
        return slab.GpuSlab(nx, ny, rows, h, lo, hi, ls.LS_FP32, stream.cuda_stream, (2, 100, 16))

    run = slab.DeviceSlabRun(slab.LocalComm(2), make, (w.n,) * 3, w.h, w.halfwidth,
                             lambda z0, z1: (phi0[z0:z1], F0[z0:z1]), rebalance=True,
                             rebalance_gain=0.0, rebalance_every=4, graphs=True, stream=stream)
    run.prepare(w.cfl, w.rebuild_every)
    run.step(100, w.cfl, w.rebuild_every)
    torch.cuda.synchronize()
    got = torch.full_like(ref, float("nan"))
    for p, (z0, planes) in run.gather_phi().items():
        got[z0:z0 + planes.shape[0]] = planes
    run.close()
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
