"""Seeded synthetic workloads for directional H^2 compression.

The paper's experiments (Section 7) use Galerkin boundary-element matrices of
the Helmholtz single-layer potential on a sphere.  Those matrices need a mesh
and singular quadrature; the stand-in used here is the point-collocation form
of the same kernel, Eq. (helmholtz):

    G_ij = exp(i*kappa*r_ij) / (4*pi*r_ij),   r_ij = |x_i - x_j|,

with the singular diagonal replaced by 1/(4*pi*h), h the mean nearest-neighbour
spacing of the point set.  Everything here is input generation: no part of the
compression is computed in this module.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 151007087


def fibonacci_sphere(n: int) -> np.ndarray:
    """Fibonacci lattice on the unit sphere, (n, 3) float64, row-major.

    z_i = 1 - (2i+1)/n, r_i = sqrt(1 - z_i^2), phi_i = i * pi * (3 - sqrt 5).
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    return np.ascontiguousarray(np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1))


def random_sphere(n: int, seed: int = SEED) -> np.ndarray:
    """Uniform random points on the unit sphere (normalised Gaussian vectors)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return np.ascontiguousarray(x)


def random_ellipsoid(n: int, axes=(1.0, 0.5, 0.5), seed: int = SEED) -> np.ndarray:
    """Uniform random points on an ellipsoid surface.

    Sphere points are mapped by the semi-axes and accepted with probability
    proportional to the surface area element of the map (rejection sampling).
    """
    rng = np.random.default_rng(seed)
    a = np.asarray(axes, dtype=np.float64)
    out = []
    have = 0
    # area element of x = a*u on the unit sphere: |a| * |u / a|
    gmax = np.prod(a) / np.min(a)
    while have < n:
        u = rng.standard_normal((2 * n, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        g = np.prod(a) * np.linalg.norm(u / a, axis=1)
        keep = rng.random(2 * n) * gmax <= g
        out.append(u[keep] * a)
        have += int(keep.sum())
    return np.ascontiguousarray(np.concatenate(out, axis=0)[:n])


def random_cube_surface(n: int, seed: int = SEED) -> np.ndarray:
    """Uniform random points on the surface of the unit cube [0,1]^3."""
    rng = np.random.default_rng(seed)
    face = rng.integers(0, 6, size=n)
    uv = rng.random((n, 2))
    x = np.empty((n, 3), dtype=np.float64)
    axis = face // 2
    side = (face % 2).astype(np.float64)
    for ax in range(3):
        sel = axis == ax
        others = [d for d in range(3) if d != ax]
        x[sel, ax] = side[sel]
        x[sel, others[0]] = uv[sel, 0]
        x[sel, others[1]] = uv[sel, 1]
    return np.ascontiguousarray(x)


def mean_nn_distance(points: np.ndarray) -> float:
    """Mean over i of min_{j != i} |x_i - x_j| (exact nearest neighbours)."""
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    if n < 2:
        return 1.0
    try:
        from scipy.spatial import cKDTree

        d, _ = cKDTree(pts).query(pts, k=2)
        return float(np.mean(d[:, 1]))
    except ImportError:  # pragma: no cover - scipy is present on both machines
        best = np.empty(n)
        for s in range(0, n, 1024):
            blk = pts[s:s + 1024]
            d2 = ((blk[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
            d2[np.arange(blk.shape[0]), np.arange(s, s + blk.shape[0])] = np.inf
            best[s:s + 1024] = np.sqrt(d2.min(1))
        return float(best.mean())


def helmholtz_matrix(points: np.ndarray, kappa: float, h: float | None = None,
                     dtype=np.complex128) -> np.ndarray:
    """Dense collocation matrix G (numpy, C order, G[i, j] = g(x_i, x_j)).

    The matrix is complex symmetric, so its C-order buffer is also its
    column-major buffer.
    """
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    if h is None:
        h = mean_nn_distance(pts)
    G = np.empty((n, n), dtype=dtype)
    for s in range(0, n, 512):
        blk = pts[s:s + 512]
        d = blk[:, None, :] - pts[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.exp(1j * kappa * r) / (4.0 * math.pi * r)
        rows = np.arange(blk.shape[0])
        g[rows, s + rows] = 1.0 / (4.0 * math.pi * h)
        G[s:s + 512] = g.astype(dtype)
    return G


def helmholtz_matrix_torch(points: np.ndarray, kappa: float, h: float, dtype, device):
    """Same matrix built with torch on a device, in column-major order.

    Returns a torch tensor M of shape (n, n) whose row-major memory is G in
    column-major order (M[j, i] = G[i, j]); since G is symmetric M equals G.
    """
    import torch

    pts = torch.as_tensor(np.asarray(points, dtype=np.float64), device=device)
    n = pts.shape[0]
    M = torch.empty((n, n), dtype=dtype, device=device)
    step = 2048
    for s in range(0, n, step):
        blk = pts[s:s + step]
        d = blk[:, None, :] - pts[None, :, :]
        r = torch.sqrt((d * d).sum(-1))
        ph = kappa * r
        g = torch.complex(torch.cos(ph), torch.sin(ph)) / (4.0 * math.pi * r)
        rows = torch.arange(blk.shape[0], device=device)
        g[rows, s + rows] = 1.0 / (4.0 * math.pi * h)
        M[s:s + step] = g.to(dtype)
    return M


def sphere_normals(points: np.ndarray) -> np.ndarray:
    """Outward unit normals of points on a sphere centred at the origin."""
    pts = np.asarray(points, dtype=np.float64)
    return pts / np.linalg.norm(pts, axis=1, keepdims=True)


def ellipsoid_normals(points: np.ndarray, axes=(1.0, 0.5, 0.5)) -> np.ndarray:
    """Outward unit normals of points on the ellipsoid sum_d (x_d / a_d)^2 = 1."""
    pts = np.asarray(points, dtype=np.float64)
    g = pts / np.asarray(axes, dtype=np.float64) ** 2
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def dlp_matrix(points: np.ndarray, normals: np.ndarray, kappa: float, dtype=np.complex128) -> np.ndarray:
    """Dense collocation matrix of 1/2 I + the Helmholtz double layer potential.

    G[i, j] = (1 - i kappa r) exp(i kappa r) / (4 pi r^3) <x_i - x_j, n(x_j)>
    with r = |x_i - x_j| for i != j, and G[i, i] = 1/2: the kernel's normal
    derivative in the second argument, and the identity standing in for the
    mass matrix of a Galerkin discretisation in a collocation setting.  On a
    sphere centred at the origin the matrix is symmetric; in general it is
    not.  It is returned in C order (G[i, j]).
    """
    pts = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    n = pts.shape[0]
    G = np.empty((n, n), dtype=dtype)
    for s in range(0, n, 512):
        blk = pts[s:s + 512]
        d = blk[:, None, :] - pts[None, :, :]
        r = np.sqrt((d * d).sum(-1))
        dn = (d * nrm[None, :, :]).sum(-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            g = (1.0 - 1j * kappa * r) * np.exp(1j * kappa * r) / (4.0 * math.pi * r ** 3) * dn
        rows = np.arange(blk.shape[0])
        g[rows, s + rows] = 0.5
        G[s:s + 512] = g.astype(dtype)
    return G


def dlp_matrix_torch(points: np.ndarray, normals: np.ndarray, kappa: float, dtype, device):
    """The double-layer matrix of `dlp_matrix`, built with torch on a device.

    Returns a torch tensor whose row-major memory is G in column-major order:
    a view M with M.t()[i, j] = G[i, j] (shape (n, n)).
    """
    import torch

    pts = torch.as_tensor(np.asarray(points, dtype=np.float64), device=device)
    nrm = torch.as_tensor(np.asarray(normals, dtype=np.float64), device=device)
    n = pts.shape[0]
    M = torch.empty((n, n), dtype=dtype, device=device)  # M[j, i] = G[i, j]
    step = 2048
    for s in range(0, n, step):
        src = pts[s:s + step]        # columns j of G
        d = pts[None, :, :] - src[:, None, :]   # d[jj, i] = x_i - x_j
        r = torch.sqrt((d * d).sum(-1))
        dn = (d * nrm[s:s + step][:, None, :]).sum(-1)
        ph = kappa * r
        e = torch.complex(torch.cos(ph), torch.sin(ph))
        g = torch.complex(torch.ones_like(r), -ph) * e * (dn / (4.0 * math.pi * r ** 3))
        rows = torch.arange(src.shape[0], device=device)
        g[rows, s + rows] = 0.5
        M[s:s + step] = g.to(dtype)
    return M.t()


def planted_separable_matrix(points: np.ndarray, rank: int = 3, seed: int = SEED) -> np.ndarray:
    """G_ij = sum_p a_p(x_i) * b_p(x_j) with smooth random a_p, b_p (exact rank <= `rank`)."""
    rng = np.random.default_rng(seed)
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    G = np.zeros((n, n), dtype=np.complex128)
    for _ in range(rank):
        w = rng.standard_normal(3)
        v = rng.standard_normal(3)
        a = np.exp(1j * (pts @ w)) * (1.0 + 0.5 * np.cos(pts @ v))
        b = np.cos(pts @ v) + 1j * np.sin(2.0 * (pts @ w))
        G += np.outer(a, b)
    return G


def random_complex_vectors(n: int, count: int = 1, seed: int = SEED) -> np.ndarray:
    """(n, count) complex128 with independent standard normal real/imag parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, count)) + 1j * rng.standard_normal((n, count))
