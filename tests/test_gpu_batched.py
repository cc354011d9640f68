"""Batched compression of independent problems of uneven size: every problem's
result must equal its single compression (same kernels, one schedule), and the
FP32 batch must meet the error bound against complex128."""
import math

import numpy as np
import pytest

from synth import (fibonacci_sphere, helmholtz_matrix, mean_nn_distance, random_complex_vectors,
                   random_cube_surface, random_ellipsoid, random_sphere, SEED)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_07087_gb300 as D
    return D


def _problems():
    """Spheres, 2:1:1 ellipsoids and unit cubes, uniform random points, n in
    [1024, 3072], kappa with kappa * diameter in [8, 40]."""
    rng = np.random.default_rng(SEED)
    out = []
    gens = [(random_sphere, 2.0), (random_ellipsoid, 2.0), (random_cube_surface, math.sqrt(3.0))]
    for i in range(6):
        g, diam = gens[i % 3]
        n = int(rng.integers(1024, 3073))
        kappa = float(rng.uniform(8.0, 40.0)) / diam
        pts = g(n, seed=SEED + i)
        out.append((pts, kappa))
    return out


def _setup(D, dt, leaf=32, eta1=2 * math.sqrt(2), eta2=1.0):
    trees, Gs, Gh = [], [], []
    for pts, kappa in _problems():
        T = D.dh2_tree_build(pts, leaf, kappa, eta1, eta2)
        perm = T.perm()
        G = helmholtz_matrix(pts, kappa)[np.ix_(perm, perm)]
        trees.append(T)
        Gh.append(G)
        Gs.append(torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", dt).t())
    return trees, Gs, Gh


@pytest.mark.parametrize("params", [dict(), dict(eta1=20.0, eta2=5.0, leaf=16)])
def test_batched_equals_single_fp64(params):
    D = _dev()
    trees, Gs, _ = _setup(D, torch.complex128, **params)
    Mb = D.dh2_compress_batched(trees, Gs, eps=1e-4)
    for T, G, M in zip(trees, Gs, Mb):
        Ms = D.dh2_compress(T, G, eps=1e-4)
        for side in (0, 1):
            assert np.array_equal(M.ranks(side), Ms.ranks(side))
        n = G.shape[0]
        x = torch.from_numpy(np.ascontiguousarray(random_complex_vectors(n, 2, seed=7).T)).to("cuda").t()
        yb = torch.empty_like(x.t().contiguous()).t()
        ys = torch.empty_like(yb.t().contiguous()).t()
        D.dh2_matvec(M, x, yb)
        D.dh2_matvec(Ms, x, ys)
        torch.cuda.synchronize()
        assert torch.linalg.norm(yb - ys) <= 1e-13 * torch.linalg.norm(ys)
        assert D.dh2_error(M, G) <= 1e-4


def test_batched_fp32_error_bound():
    D = _dev()
    trees, Gs, Gh = _setup(D, torch.complex64)
    Mb = D.dh2_compress_batched(trees, Gs, eps=1e-4)
    for G, M in zip(Gh, Mb):
        G128 = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda").t()
        assert D.dh2_error(M, G128) <= 1e-4


def test_batched_rejects_mixed_dtypes():
    D = _dev()
    trees, Gs, _ = _setup(D, torch.complex128)
    Gs[1] = Gs[1].to(torch.complex64)
    with pytest.raises(TypeError):
        D.dh2_compress_batched(trees[:2], Gs[:2])


def test_batched_mixed_equals_single():
    """The mixed mode's batch (row scales, tensor-core Gram matrices, factor launches over all
    problems) equals each problem's own compression."""
    D = _dev()
    trees, Gs, Gh = _setup(D, torch.complex64)
    mode = D.MODE_MIXED_BF16X3
    Mb = D.dh2_compress_batched(trees, Gs, eps=1e-4, mode=mode)
    for T, G, G64h, M in zip(trees, Gs, Gh, Mb):
        Ms = D.dh2_compress(T, G, eps=1e-4, mode=mode)
        for side in (0, 1):
            assert np.array_equal(M.ranks(side), Ms.ranks(side))
        assert M.storage() == Ms.storage()
        G128 = torch.from_numpy(np.ascontiguousarray(G64h.T)).to("cuda").t()
        eb, es = D.dh2_error(M, G128), D.dh2_error(Ms, G128)
        assert eb <= 1e-4 and abs(eb - es) <= 1e-12 * es
