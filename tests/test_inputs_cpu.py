"""Pins of the Step 0 inputs that the device generators are checked against:
the real spherical-harmonic basis of the perturbed-sphere workload is
orthonormal on the sphere (exact product quadrature) and equals the
textbook closed forms for l = 1, 2; the sphere-union and Fourier-speed
generators equal their definitions at hand-picked points."""
import math

import numpy as np
import torch

from paper_1612_04040_b300 import inputs


def quadrature(n_theta=24, n_phi=48):
    """Gauss-Legendre in cos(theta) x uniform in phi: exact for the products
    of two harmonics of degree <= 8 (polynomials of degree <= 16 in cos
    theta, trigonometric degree <= 16 in phi)."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    ph = (np.arange(n_phi) + 0.5) * (2 * math.pi / n_phi)
    CT, PH = np.meshgrid(ct, ph, indexing="ij")
    W = np.outer(wt, np.full(n_phi, 2 * math.pi / n_phi))
    st = np.sqrt(1 - CT * CT)
    u = [torch.from_numpy(v) for v in (st * np.cos(PH), st * np.sin(PH), CT)]
    return u, W


def test_real_harmonics_are_orthonormal():
    (ux, uy, uz), W = quadrature()
    Y = np.stack([y.numpy() for y in inputs._real_sh_basis(8, ux, uy, uz)])
    assert Y.shape[0] == 80                                   # l = 1..8, m = -l..l
    G = np.einsum("iab,jab,ab->ij", Y, Y, W)
    assert np.max(np.abs(G - np.eye(80))) <= 1e-12


def test_real_harmonics_closed_forms():
    g = np.random.default_rng(1)
    v = g.normal(size=(3, 50))
    v /= np.linalg.norm(v, axis=0)
    x, y, z = v
    Y = [t.numpy() for t in inputs._real_sh_basis(2, *(torch.from_numpy(a) for a in v))]
    c1 = math.sqrt(3 / (4 * math.pi))
    expect = [c1 * y, c1 * z, c1 * x,                          # l = 1: m = -1, 0, 1
              math.sqrt(15 / (4 * math.pi)) * x * y,           # l = 2: m = -2
              math.sqrt(15 / (4 * math.pi)) * y * z,           # m = -1
              math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1),  # m = 0
              math.sqrt(15 / (4 * math.pi)) * x * z,           # m = 1
              math.sqrt(15 / (16 * math.pi)) * (x * x - y * y)]  # m = 2
    for k, (a, b) in enumerate(zip(Y, expect)):
        assert np.max(np.abs(a - b)) <= 1e-13, k


def test_perturbed_sphere_radius_scale():
    """max |S| = 1 on the (theta, phi) sampling, so r stays in base +- amp."""
    w = inputs.PerturbedSphere(n=32)
    th = (np.arange(512) + 0.5) * (math.pi / 512)
    ph = (np.arange(1024) + 0.5) * (2 * math.pi / 1024)
    T, P = np.meshgrid(th, ph, indexing="ij")
    u = [torch.from_numpy(a) for a in (np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T))]
    r = w.radius_fn()(*u).numpy()
    assert abs(np.max(np.abs(r - w.base)) - w.amp) <= 1e-12


def test_sphere_union_and_fourier_speed_at_points():
    h = 1.0 / 8
    phi = inputs.sphere_union_sdf((8, 8, 8), h, [(0.5, 0.5, 0.5), (0.0625, 0.0625, 0.0625)], [0.25, 0.1]).numpy()
    assert phi[0, 0, 0] == -0.1                                # the small sphere's centre
    assert abs(phi[4, 4, 4] - (math.sqrt(3) / 16 - 0.25)) <= 1e-15   # (0.5625,)*3 from (0.5,)*3
    modes = [(0.5, (1, 0, 0), 0.0), (-1.5, (0, 1, -1), 0.25)]
    F = inputs.speed_fourier((8, 8, 8), h, modes).numpy()
    x = y = z = 0.0625
    exp = (0.5 * math.cos(2 * math.pi * x) - 1.5 * math.cos(2 * math.pi * (y - z) + 0.25)) / 2.0
    assert abs(F[0, 0, 0] - exp) <= 1e-15
