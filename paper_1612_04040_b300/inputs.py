"""Seeded synthetic inputs: initial level-set functions (Eq. 1, Step 0 of the
narrow-band algorithm, section 1.1) and speed fields F.

This module holds none of the method's arithmetic (no upwind step, no band
test, no time-step rule).  It only draws the seeded shape parameters and
evaluates closed-form signed distances and speed fields, in FP64, so that the
CUDA path and the CPU oracle can be fed the very same arrays.  Both sides
import it; neither imports the other.

Grid convention (cell-centred): point (i, j, k) sits at ((i+1/2)h, (j+1/2)h,
(k+1/2)h) and arrays are indexed [z][y][x] (x fastest), the index order of
the paper's GPU listing in section 3.

Random numbers come from numpy's PCG64 with a fixed seed per workload
(``seed_for``); evaluation uses torch in FP64 on the requested device, slab
by slab along z so that 1024^3 grids fit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

F64 = torch.float64


def seed_for(workload_index: int) -> int:
    """Fixed seed of each standard workload (0..4)."""
    return 1000 + int(workload_index)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def coords(n: int, h: float, device="cpu") -> torch.Tensor:
    """Cell-centred coordinates (i + 1/2) h, i = 0..n-1, FP64."""
    return (torch.arange(n, dtype=F64, device=device) + 0.5) * h


def _by_slab(shape, h, fn, device="cpu", slab_points=1 << 22, out_dtype=F64):
    """Evaluate fn(X, Y, Z) -> tensor over the grid, a few z planes at a time."""
    nz, ny, nx = shape
    out = torch.empty((nz, ny, nx), dtype=out_dtype, device=device)
    xs, ys, zs = coords(nx, h, device), coords(ny, h, device), coords(nz, h, device)
    step = max(1, slab_points // (nx * ny))
    for z0 in range(0, nz, step):
        z1 = min(nz, z0 + step)
        Z = zs[z0:z1].view(-1, 1, 1)
        Y = ys.view(1, -1, 1)
        X = xs.view(1, 1, -1)
        out[z0:z1] = fn(X, Y, Z).to(out_dtype)
    return out


# --------------------------------------------------------------------------
# closed-form signed distances (Eq. 1: phi(x, 0) = +-d, negative inside)
# --------------------------------------------------------------------------

def sphere_union_sdf(shape, h, centres, radii, device="cpu", out_dtype=F64):
    """phi = min_i(|x - c_i| - r_i): exact distance outside the union, a valid
    level-set function (negative) inside."""
    centres = [tuple(float(v) for v in c) for c in centres]
    radii = [float(r) for r in radii]

    def fn(X, Y, Z):
        best = None
        for (cx, cy, cz), r in zip(centres, radii):
            d = torch.sqrt((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) - r
            best = d if best is None else torch.minimum(best, d)
        return best

    return _by_slab(shape, h, fn, device, out_dtype=out_dtype)


def torus_sdf(shape, h, centre, axis, R, r, device="cpu", out_dtype=F64):
    """Signed distance to a torus with centre c, unit axis a, major radius R,
    minor radius r: sqrt((rho - R)^2 + s^2) - r, with s = (x-c).a and rho the
    distance from the axis line."""
    cx, cy, cz = (float(v) for v in centre)
    ax, ay, az = (float(v) for v in axis)

    def fn(X, Y, Z):
        px, py, pz = X - cx, Y - cy, Z - cz
        s = px * ax + py * ay + pz * az
        qx, qy, qz = px - s * ax, py - s * ay, pz - s * az
        rho = torch.sqrt(qx * qx + qy * qy + qz * qz)
        return torch.sqrt((rho - R) ** 2 + s * s) - r

    return _by_slab(shape, h, fn, device, out_dtype=out_dtype)


def _real_sh_basis(lmax, ux, uy, uz):
    """Real orthonormal spherical harmonics Y_lm, 1 <= l <= lmax, evaluated at
    unit vectors; returns a list of tensors in (l, m) order m = -l..l."""
    ct = uz.clamp(-1.0, 1.0)
    st = torch.sqrt(torch.clamp(1.0 - ct * ct, min=0.0))
    ph = torch.atan2(uy, ux)
    # associated Legendre functions P_l^m(ct), no Condon-Shortley phase
    P = {}
    for m in range(lmax + 1):
        pmm = torch.ones_like(ct)
        fact = 1.0
        for _ in range(m):
            pmm = pmm * fact * st
            fact += 2.0
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = ct * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * ct * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    out = []
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(norm * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2.0) * norm * P[(l, am)] * torch.cos(am * ph))
            else:
                out.append(math.sqrt(2.0) * norm * P[(l, am)] * torch.sin(am * ph))
    return out


def sh_radius_fn(coeffs, lmax, scale, base, amp):
    """r(u) = base + amp * scale * sum a_lm Y_lm(u) for unit vectors u."""
    coeffs = [float(c) for c in coeffs]

    def r_of(ux, uy, uz):
        basis = _real_sh_basis(lmax, ux, uy, uz)
        s = torch.zeros_like(ux)
        for a, y in zip(coeffs, basis):
            s = s + a * y
        return base + amp * scale * s

    return r_of


def sh_sphere_phi(shape, h, centre, radius_fn, device="cpu", out_dtype=F64):
    """Radial level-set function |x - c| - r(direction): negative inside the
    perturbed sphere (a level-set function with the right zero set; not an
    exact distance)."""
    cx, cy, cz = (float(v) for v in centre)

    def fn(X, Y, Z):
        px, py, pz = torch.broadcast_tensors(X - cx, Y - cy, Z - cz)
        rr = torch.sqrt(px * px + py * py + pz * pz)
        return rr - radius_fn(px / rr, py / rr, pz / rr)

    return _by_slab(shape, h, fn, device, slab_points=1 << 20, out_dtype=out_dtype)


# --------------------------------------------------------------------------
# speed fields
# --------------------------------------------------------------------------

def speed_sinusoid(shape, h, device="cpu", out_dtype=F64):
    """F = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z), in [0.5, 1.5]."""
    tp = 2.0 * math.pi
    return _by_slab(shape, h, lambda X, Y, Z: 1.0 + 0.5 * torch.sin(tp * X) * torch.sin(tp * Y)
                    * torch.sin(tp * Z), device, out_dtype=out_dtype)


def speed_cos_cos(shape, h, device="cpu", out_dtype=F64):
    """Sign-changing F = cos(4 pi x) cos(4 pi y) (independent of z)."""
    fp = 4.0 * math.pi
    return _by_slab(shape, h, lambda X, Y, Z: (torch.cos(fp * X) * torch.cos(fp * Y)).expand(
        Z.shape[0], Y.shape[1], X.shape[2]), device, out_dtype=out_dtype)


def speed_fourier(shape, h, modes, device="cpu", out_dtype=F64):
    """F = sum_m a_m cos(2 pi k_m . x + theta_m) / sum_m |a_m|  (|F| <= 1)."""
    norm = sum(abs(a) for a, _, _ in modes) or 1.0

    def fn(X, Y, Z):
        s = None
        for a, k, th in modes:
            t = a * torch.cos(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + th)
            s = t if s is None else s + t
        return (s / norm).expand(Z.shape[0], Y.shape[1], X.shape[2])

    return _by_slab(shape, h, fn, device, out_dtype=out_dtype)


# --------------------------------------------------------------------------
# the five standard workloads
# --------------------------------------------------------------------------

@dataclass
class SingleSphere:
    """64^3, h = 1/64, sphere r0 = 0.25 at the domain centre, F = 1,
    dt = h/2, 100 full-domain steps, FP64."""
    n: int = 64
    r0: float = 0.25
    centre: tuple = (0.5, 0.5, 0.5)
    speed: float = 1.0
    steps: int = 100

    @property
    def h(self):
        return 1.0 / self.n

    def phi(self, device="cpu", out_dtype=F64):
        return sphere_union_sdf((self.n,) * 3, self.h, [self.centre], [self.r0], device, out_dtype)


@dataclass
class SphereUnion:
    """n^3 (512 in the standard workload), union of 20 seeded spheres
    (centres U[0.15, 0.85]^3, radii U[0.05, 0.15]), F = 1 + 0.5 sin sin sin,
    band half-width 6h, rebuild every 5 steps, 500 steps at CFL 0.5, FP32."""
    n: int = 512
    count: int = 20
    seed: int = seed_for(1)
    halfwidth: float = 6.0
    rebuild_every: int = 5
    steps: int = 500
    cfl: float = 0.5
    centres: list = field(default_factory=list)
    radii: list = field(default_factory=list)

    def __post_init__(self):
        g = rng(self.seed)
        self.centres = [tuple(g.uniform(0.15, 0.85, 3)) for _ in range(self.count)]
        self.radii = [float(g.uniform(0.05, 0.15)) for _ in range(self.count)]

    @property
    def h(self):
        return 1.0 / self.n

    def phi(self, device="cpu", out_dtype=F64):
        return sphere_union_sdf((self.n,) * 3, self.h, self.centres, self.radii, device, out_dtype)

    def speed(self, device="cpu", out_dtype=F64):
        return speed_sinusoid((self.n,) * 3, self.h, device, out_dtype)


@dataclass
class BatchInstance:
    edge: int
    kind: str            # "sphere" or "torus"
    centre: tuple
    params: dict
    speed: float

    @property
    def h(self):
        return 1.0 / self.edge

    def phi(self, device="cpu", out_dtype=F64):
        shape = (self.edge,) * 3
        if self.kind == "sphere":
            return sphere_union_sdf(shape, self.h, [self.centre], [self.params["r"]], device, out_dtype)
        return torus_sdf(shape, self.h, self.centre, self.params["axis"], self.params["R"],
                         self.params["r"], device, out_dtype)


def batch_instances(count=256, seed=seed_for(2), edges=tuple(range(32, 193, 16))):
    """Independent interfaces: cubic grid edge uniform in {32, 48, ..., 192}
    (box [0,1]^3, h = 1/edge), a sphere (centre U[0.35,0.65]^3, radius
    U[0.1,0.25]) or a torus (random axis, R U[0.2,0.3], r U[0.05,0.1]) with
    equal odds, constant F uniform in [-1, 1]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        e = int(g.choice(np.asarray(edges)))
        c = tuple(float(v) for v in g.uniform(0.35, 0.65, 3))
        if g.uniform() < 0.5:
            kind, params = "sphere", {"r": float(g.uniform(0.1, 0.25))}
        else:
            v = g.normal(size=3)
            v = v / np.linalg.norm(v)
            kind, params = "torus", {"axis": tuple(float(a) for a in v),
                                     "R": float(g.uniform(0.2, 0.3)), "r": float(g.uniform(0.05, 0.1))}
        F = float(g.uniform(-1.0, 1.0))
        out.append(BatchInstance(e, kind, c, params, F))
    return out


@dataclass
class PerturbedSphere:
    """n^3 (1024 in the standard workload), r(theta, phi) = 0.3 + 0.03 S with S
    a seeded random combination of real spherical harmonics 1 <= l <= 8,
    normalised so max|S| = 1 on a 512 x 1024 (theta, phi) sampling;
    F = cos(4 pi x) cos(4 pi y); band half-width 6h; 1000 steps."""
    n: int = 1024
    seed: int = seed_for(3)
    lmax: int = 8
    base: float = 0.3
    amp: float = 0.03
    halfwidth: float = 6.0
    steps: int = 1000
    coeffs: list = field(default_factory=list)
    scale: float = 1.0

    def __post_init__(self):
        g = rng(self.seed)
        nmodes = (self.lmax + 1) ** 2 - 1
        self.coeffs = [float(v) for v in g.normal(size=nmodes)]
        th = (torch.arange(512, dtype=F64) + 0.5) * (math.pi / 512)
        ph = (torch.arange(1024, dtype=F64) + 0.5) * (2 * math.pi / 1024)
        T, P = torch.meshgrid(th, ph, indexing="ij")
        ux, uy, uz = torch.sin(T) * torch.cos(P), torch.sin(T) * torch.sin(P), torch.cos(T)
        s = sh_radius_fn(self.coeffs, self.lmax, 1.0, 0.0, 1.0)(ux, uy, uz)
        self.scale = 1.0 / float(s.abs().max())

    @property
    def h(self):
        return 1.0 / self.n

    def radius_fn(self):
        return sh_radius_fn(self.coeffs, self.lmax, self.scale, self.base, self.amp)

    def phi(self, device="cpu", out_dtype=F64):
        return sh_sphere_phi((self.n,) * 3, self.h, (0.5, 0.5, 0.5), self.radius_fn(), device, out_dtype)

    def speed(self, device="cpu", out_dtype=F64):
        return speed_cos_cos((self.n,) * 3, self.h, device, out_dtype)


def fourier_modes(g: np.random.Generator, count=8, kmax=2):
    """count modes (a, k, theta): k uniform on {-kmax..kmax}^3 without 0,
    theta U[0, 2 pi), a U[-1, 1]."""
    modes = []
    while len(modes) < count:
        k = tuple(int(v) for v in g.integers(-kmax, kmax + 1, 3))
        if k == (0, 0, 0):
            continue
        modes.append((float(g.uniform(-1.0, 1.0)), k, float(g.uniform(0.0, 2.0 * math.pi))))
    return modes


def random_sphere_union(g: np.random.Generator, count_range=(3, 12)):
    """Seeded sphere union for learned-corrector training pairs."""
    k = int(g.integers(count_range[0], count_range[1] + 1))
    centres = [tuple(float(v) for v in g.uniform(0.2, 0.8, 3)) for _ in range(k)]
    radii = [float(g.uniform(0.06, 0.16)) for _ in range(k)]
    return centres, radii


# --------------------------------------------------------------------------
# parameter vectors of the library's device-side Step 0 generators
# (ls_init_phi / ls_init_speed); same formulas as the functions above
# --------------------------------------------------------------------------

def spheres_params(centres, radii):
    out = [float(len(radii))]
    for c, r in zip(centres, radii):
        out += [float(c[0]), float(c[1]), float(c[2]), float(r)]
    return np.asarray(out, dtype=np.float64)


def torus_params(centre, axis, R, r):
    return np.asarray(list(centre) + list(axis) + [R, r], dtype=np.float64)


def sh_params(w: "PerturbedSphere", centre=(0.5, 0.5, 0.5)):
    """[cx, cy, cz, base, amp, lmax, a_lm...]: the device generator computes
    the normalisations of the real spherical harmonics itself."""
    return np.asarray(list(centre) + [w.base, w.amp * w.scale, float(w.lmax)] + list(w.coeffs),
                      dtype=np.float64)


def fourier_params(modes):
    out = [float(len(modes))]
    for a, k, th in modes:
        out += [float(a), float(k[0]), float(k[1]), float(k[2]), float(th)]
    return np.asarray(out, dtype=np.float64)
