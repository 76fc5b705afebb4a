"""Pins for the oracle's tensor-product derivatives and Q-criterion (CPU only).

Closed forms: exact gradients of polynomials of degree <= N per direction (on affine
and on curved trilinear elements), the analytic Taylor-Green Q, solid-body rotation
(Q = w^2) and pure strain (Q = -a^2).
"""
import math

import numpy as np
import pytest
import torch

import sem_inputs as si


def _poly(X, Y, Z):
    # degree <= 3 in each direction, with cross terms
    f = X ** 3 * Y ** 2 * Z + 2.0 * X * Y * Z ** 3 - 0.5 * Y ** 3 + Z ** 2 * X + 1.0
    fx = 3 * X ** 2 * Y ** 2 * Z + 2.0 * Y * Z ** 3 + Z ** 2
    fy = 2 * X ** 3 * Y * Z + 2.0 * X * Z ** 3 - 1.5 * Y ** 2
    fz = X ** 3 * Y ** 2 + 6.0 * X * Y * Z ** 2 + 2 * Z * X
    return f, fx, fy, fz


@pytest.mark.parametrize("N", [3, 5, 7])
def test_gradient_exact_polynomial_affine(orc, N):
    m = si.BoxMesh(N, np.array([-1.0, -0.2, 0.7, 1.5]), np.array([0.0, 0.4, 1.1]), np.array([-0.5, 0.3]))
    xyz = m.xyz().numpy()
    f, fx, fy, fz = _poly(*xyz)
    g = orc.gradient(N, xyz, f)[0]
    scale = max(np.abs(fx).max(), np.abs(fy).max(), np.abs(fz).max())
    for a, ref in enumerate((fx, fy, fz)):
        assert np.abs(g[a] - ref).max() < 1e-12 * scale


def _trilinear_mesh(N, E=3, seed=0):
    """Curved (non-affine) elements: each is a random trilinear map of the reference cube."""
    rng = np.random.default_rng(seed)
    xi = si.gll_points(N)
    NP = N + 1
    r = np.broadcast_to(xi[None, None, :], (NP, NP, NP)).reshape(-1)
    s = np.broadcast_to(xi[None, :, None], (NP, NP, NP)).reshape(-1)
    t = np.broadcast_to(xi[:, None, None], (NP, NP, NP)).reshape(-1)
    xyz = np.zeros((3, E, NP ** 3))
    for e in range(E):
        corners = np.array([[(v & 1), (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], float) * 2 - 1
        corners = corners + 0.25 * rng.uniform(-1, 1, size=(8, 3)) + 3.0 * e
        for v in range(8):
            a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
            wgt = ((1 + r) / 2 if a else (1 - r) / 2) * ((1 + s) / 2 if b else (1 - s) / 2) * \
                  ((1 + t) / 2 if c else (1 - t) / 2)
            xyz[:, e] += corners[v][:, None] * wgt[None, :]
    return xyz


@pytest.mark.parametrize("N", [2, 4, 7])
def test_gradient_exact_curved_elements(orc, N):
    # On a trilinear map, a field of total degree <= 2 in x is degree <= 2 per reference
    # direction, so the isoparametric chain rule is exact for N >= 2.
    xyz = _trilinear_mesh(N)
    X, Y, Z = xyz
    f = 1.0 + 2 * X - Y + 0.5 * Z + X * Y - 0.3 * Z * Z + 0.7 * X * Z
    fx = 2 + Y + 0.7 * Z
    fy = -1 + X
    fz = 0.5 - 0.6 * Z + 0.7 * X
    g = orc.gradient(N, xyz, f)[0]
    for a, ref in enumerate((fx, fy, fz)):
        assert np.abs(g[a] - ref).max() < 1e-11


def test_q_solid_rotation_and_strain(orc):
    m = si.uniform_box((2, 2, 2), (0, 0, 0), (1, 1, 1), 3)
    xyz = m.xyz().numpy()
    X, Y, Z = xyz
    w = 1.7
    rot = np.stack([-w * Y, w * X, np.zeros_like(X)])
    np.testing.assert_allclose(orc.qcriterion(3, xyz, rot), w * w, rtol=1e-12)
    a = 0.9
    strain = np.stack([a * X, -a * Y, np.zeros_like(X)])
    np.testing.assert_allclose(orc.qcriterion(3, xyz, strain), -a * a, rtol=1e-12)
    # a rotation about x combined with strain along z: Q = w^2 - (a^2 + a^2 + 4a^2)/2
    mix = np.stack([np.zeros_like(X), -w * Z - a * Y, w * Y - a * Z]) + np.stack([2 * a * X, 0 * X, 0 * X])
    np.testing.assert_allclose(orc.qcriterion(3, xyz, mix), w * w - 3 * a * a, rtol=1e-12)


def test_q_taylor_green_analytic(orc):
    # u = sin x cos y cos z, v = -cos x sin y cos z, w = 0:
    # Q = cos^2 z (sin^2 x sin^2 y - cos^2 x cos^2 y) = -(1 + cos 2z)(cos 2x + cos 2y)/4
    w = si.tgv_box(noise=0.0)
    xyz = w.mesh.xyz().numpy()
    Q = orc.qcriterion(7, xyz, w.fields.numpy())
    X, Y, Z = xyz
    Qa = -(1 + np.cos(2 * Z)) * (np.cos(2 * X) + np.cos(2 * Y)) / 4
    assert np.abs(Q - Qa).max() < 1e-7
    assert abs(Q.max() - 1.0) < 1e-7


def test_q_taylor_green_converges(orc):
    errs = []
    for N in (3, 5, 7):
        w = si.tgv_box(nel=4, N=N, noise=0.0)
        xyz = w.mesh.xyz().numpy()
        X, Y, Z = xyz
        Qa = -(1 + np.cos(2 * Z)) * (np.cos(2 * X) + np.cos(2 * Y)) / 4
        errs.append(np.abs(orc.qcriterion(N, xyz, w.fields.numpy()) - Qa).max())
    # spectral convergence: each step of 2 in N gains well over an order of magnitude
    assert errs[1] < errs[0] / 20 and errs[2] < errs[1] / 20


def test_q_noise_is_element_local(orc):
    # elements are independent: Q of a slab equals the slab of Q
    w = si.tgv_box(nel=4, N=5)
    xyz = w.mesh.xyz().numpy()
    Q = orc.qcriterion(5, xyz, w.fields.numpy())
    Qs = orc.qcriterion(5, xyz[:, 10:20], w.fields.numpy()[:, 10:20])
    np.testing.assert_array_equal(Qs, Q[10:20])
