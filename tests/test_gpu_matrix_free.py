"""Matrix-free compression (entries generated in the kernels) against the
compression of the materialised matrix, and against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import dh2_oracle as O
from synth import (dlp_matrix, ellipsoid_normals, fibonacci_sphere, helmholtz_matrix, mean_nn_distance,
                   random_complex_vectors, random_ellipsoid)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_07087_gb300 as D
    return D


def _ranks(D, T, M):
    out = {}
    for side in (0, 1):
        pr = T.pairs(side)
        rk = M.ranks(side)
        out[side] = {(int(pr["cluster"][p]), int(pr["dir"][p])): int(rk[p]) for p in range(len(rk))}
    return out


def _matvec(D, M, x, dt):
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).to("cuda", dt).t()
    yd = torch.empty_like(xd.t().contiguous()).t()
    D.dh2_matvec(M, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,kappa,leaf", [(2048, 4.0, 32), (4096, 12.0, 32)])
def test_matrix_free_fp64_matches_dense_and_oracle(n, kappa, leaf):
    D = _dev()
    pts = fibonacci_sphere(n)
    h = mean_nn_distance(pts)
    diag = 1.0 / (4.0 * math.pi * h)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa, h)[np.ix_(perm, perm)]
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda").t()
    Md = D.dh2_compress(T, Gd, eps=1e-4, mode=D.MODE_FP64)
    Mf = D.dh2_compress_kernel(T, pts, kappa, diag, eps=1e-4, mode=D.MODE_FP64)
    rd, rf = _ranks(D, T, Md), _ranks(D, T, Mf)
    diff = sum(rd[s][k] != rf[s][k] for s in (0, 1) for k in rd[s])
    assert diff <= 2, diff
    # oracle at the matrix-free ranks
    tr = O.build_tree(pts, O.TreeParams(leaf_size=leaf, kappa=kappa))
    cp = O.CompressParams(eps=1e-4)
    w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
    V = O.compress(tr, G, cp, "row", w, rank_override=rf[0])
    W = O.compress(tr, G, cp, "col", w, rank_override=rf[1])
    S = O.project(tr, G, V, W)
    x = random_complex_vectors(n, 2, seed=21)
    y_ref = O.matvec(tr, G, V, W, S, x)
    y = _matvec(D, Mf, x, torch.complex128)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) <= 1e-11
    e_gen = D.dh2_error(Mf)            # reference generated in FP64
    e_dense = D.dh2_error(Mf, Gd)      # reference = the numpy matrix
    assert e_gen <= 1e-4
    assert abs(e_gen - e_dense) <= 1e-6 * e_dense


def test_matrix_free_fp32():
    D = _dev()
    n, kappa, leaf = 8192, 16.0, 32
    pts = fibonacci_sphere(n)
    h = mean_nn_distance(pts)
    T = D.dh2_tree_build(pts, leaf, kappa)
    Mf = D.dh2_compress_kernel(T, pts, kappa, 1.0 / (4.0 * math.pi * h), eps=1e-4, mode=D.MODE_FP32)
    err = D.dh2_error(Mf)
    assert err <= 1e-4, err
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa, h, dtype=np.complex64)[np.ix_(perm, perm)]
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda").t()
    Md = D.dh2_compress(T, Gd, eps=1e-4)
    rd, rf = _ranks(D, T, Md), _ranks(D, T, Mf)
    total = sum(len(rd[s]) for s in (0, 1))
    diff = sum(rd[s][k] != rf[s][k] for s in (0, 1) for k in rd[s])
    assert diff <= 0.02 * total, (diff, total)


@pytest.mark.parametrize("fp64", [True, False])
def test_matrix_free_double_layer_matches_dense(fp64):
    """1/2 I + double layer on an ellipsoid, generated in the kernels from points and normals,
    against the compression of the materialised (non-symmetric) matrix and the oracle."""
    D = _dev()
    n, kappa, leaf, eps = 2048, 8.0, 32, 1e-4
    pts = random_ellipsoid(n)
    nrm = ellipsoid_normals(pts)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = dlp_matrix(pts, nrm, kappa)[np.ix_(perm, perm)]
    mode = D.MODE_FP64 if fp64 else D.MODE_FP32
    dt = torch.complex128 if fp64 else torch.complex64
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", dt).t()
    G128 = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", torch.complex128).t()
    Md = D.dh2_compress(T, Gd, eps=eps, mode=mode)
    Mf = D.dh2_compress_kernel_dlp(T, pts, nrm, kappa, eps=eps, mode=mode)
    rd, rf = _ranks(D, T, Md), _ranks(D, T, Mf)
    total = sum(len(rd[s]) for s in (0, 1))
    diff = sum(rd[s][k] != rf[s][k] for s in (0, 1) for k in rd[s])
    assert diff <= (2 if fp64 else 0.02 * total), (diff, total)
    e_gen = D.dh2_error(Mf)            # reference generated in FP64 from points and normals
    e_dense = D.dh2_error(Mf, G128)    # reference = the numpy matrix
    assert e_gen <= eps and e_dense <= eps
    assert abs(e_gen - e_dense) <= 1e-6 * e_dense
    if fp64:
        tr = O.build_tree(pts, O.TreeParams(leaf_size=leaf, kappa=kappa))
        cp = O.CompressParams(eps=eps)
        w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
        V = O.compress(tr, G, cp, "row", w, rank_override=rf[0])
        W = O.compress(tr, G, cp, "col", w, rank_override=rf[1])
        S = O.project(tr, G, V, W)
        x = random_complex_vectors(n, 2, seed=23)
        y_ref = O.matvec(tr, G, V, W, S, x)
        y = _matvec(D, Mf, x, torch.complex128)
        assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) <= 1e-11


def test_matrix_free_rejects_view_nearfield():
    D = _dev()
    pts = fibonacci_sphere(256)
    T = D.dh2_tree_build(pts, 16, 4.0)
    from paper_1510_07087_gb300 import _binding as B
    p = B.CompressParams(1e-4, 2.0 / 3.0, 0, D.MODE_FP64, 1, 0)
    h = B.c_void_p()
    st = B._lib().dh2_compress_kernel(T.handle, B._ptr(np.ascontiguousarray(pts)), 4.0, 1.0, B.byref(p),
                                      B.c_void_p(torch.cuda.current_stream().cuda_stream), B.byref(h))
    assert st == 1 and not h.value
