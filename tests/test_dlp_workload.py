"""The double-layer-potential workload (the paper's second experiment).

G = 1/2 I + G_dlp with the kernel (1 - i kappa r) exp(i kappa r) / (4 pi r^3)
<x - y, n(y)>, the normal derivative of the single-layer kernel in y
(Section 7, "DLP matrix"; collocation stands in for the Galerkin matrix and
the identity for the mass matrix).  The compression itself only reads
matrix entries, so these tests pin the input generator against its
definition and the oracle's error guarantee on a matrix that, unlike the
single-layer one, is not symmetric.
"""
import math

import numpy as np
import pytest

from oracle import dh2_oracle as O
from synth import dlp_matrix, ellipsoid_normals, fibonacci_sphere, random_ellipsoid, sphere_normals


def _slp(x, y, kappa):
    r = np.linalg.norm(x - y)
    return np.exp(1j * kappa * r) / (4.0 * math.pi * r)


def test_dlp_entries_are_normal_derivatives_of_the_single_layer_kernel():
    pts = random_ellipsoid(300)
    nrm = ellipsoid_normals(pts)
    kappa = 7.0
    G = dlp_matrix(pts, nrm, kappa)
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(40):
        i, j = rng.choice(len(pts), 2, replace=False)
        fd = (_slp(pts[i], pts[j] + h * nrm[j], kappa) - _slp(pts[i], pts[j] - h * nrm[j], kappa)) / (2 * h)
        assert abs(G[i, j] - fd) <= 1e-6 * abs(fd) + 1e-8
    np.testing.assert_array_equal(np.diag(G), 0.5)


def test_ellipsoid_normals_are_gradients_of_the_surface_equation():
    axes = (1.0, 0.5, 0.5)
    pts = random_ellipsoid(200, axes)
    np.testing.assert_allclose(((pts / np.asarray(axes)) ** 2).sum(1), 1.0, rtol=1e-12)
    nrm = ellipsoid_normals(pts, axes)
    np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, rtol=1e-12)
    # tangent directions along the surface are orthogonal to the normal
    t = np.cross(nrm, np.array([0.3, -0.7, 0.2]))
    eps = 1e-6
    q = pts + eps * t
    lvl = ((q / np.asarray(axes)) ** 2).sum(1)
    assert np.max(np.abs(lvl - 1.0)) <= 1e-10


def test_dlp_on_a_sphere_is_symmetric_and_on_an_ellipsoid_is_not():
    p = fibonacci_sphere(400)
    G = dlp_matrix(p, sphere_normals(p), 5.0)
    assert np.max(np.abs(G - G.T)) <= 1e-12 * np.max(np.abs(G))
    q = random_ellipsoid(400)
    H = dlp_matrix(q, ellipsoid_normals(q), 5.0)
    assert np.max(np.abs(H - H.T)) >= 1e-2 * np.max(np.abs(H))


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_oracle_error_bound_on_the_double_layer_matrix(eps):
    pts = random_ellipsoid(1024)
    G = dlp_matrix(pts, ellipsoid_normals(pts), 8.0)
    tp = O.TreeParams(leaf_size=32, kappa=8.0)
    cp = O.CompressParams(eps=eps)
    tr, V, W, S, Gp = O.run(pts, G, tp, cp)
    assert sum(1 for b in tr.blocks if b[2]) > 0  # admissible blocks exist
    err = O.error_fro(tr, Gp, V, W, S)
    assert err <= eps
    Gt = O.dense_approximation(tr, Gp, V, W, S)
    np.testing.assert_allclose(np.linalg.norm(Gp - Gt) / np.linalg.norm(Gp), err, rtol=1e-6)
