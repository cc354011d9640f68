"""The mixed mode (DH2_MODE_MIXED_BF16X3): leaf Gram matrices on the tensor
cores from exact bf16 slice products, pivoted Cholesky in double-float.

  * exactness: the kernel's Gram matrix of a leaf pair equals the Gram matrix
    of the sliced leaf matrix, computed here in integer arithmetic from the
    slicing rule stated in include/dh2.h (row scale 2^e above the row's
    largest |re|, |im|; a = 2^(e-6) (s1 + 2^-8 s2 + 2^-16 s3), each slice the
    nearest integer), up to the double-float rounding of the result;
  * parity: ranks, error and products against the FP64 oracle under the same
    criteria as the FP32 mode, at leaf sizes 32 and 64 (every row class);
  * a device wait bounded by spin_limit = 1 runs out: DH2_ETIMEOUT, no handle.
"""
import ctypes
import math

import numpy as np
import pytest

from gpu_cases import Case, check_reduced, colmajor, dev
from synth import fibonacci_sphere, helmholtz_matrix, random_ellipsoid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DH2_ETIMEOUT = 4


def _sliced_gram_exact(A32: np.ndarray) -> np.ndarray:
    """Gram matrix of the three-slice fixed-point form of a complex64 matrix whose
    entries are already weighted: integer slice products summed exactly (int64),
    combined exactly, then scaled (float64 rounding only at the end)."""
    X = A32.real.astype(np.float32)
    Y = A32.imag.astype(np.float32)
    mx = np.maximum(np.abs(X).max(axis=1), np.abs(Y).max(axis=1))
    e = np.zeros(len(mx), dtype=np.int64)
    nz = mx > 0
    e[nz] = np.frexp(mx[nz])[1]
    sc = np.ldexp(np.float32(1.0), (6 - e).astype(np.int32)).astype(np.float32)[:, None]

    def slices(M):
        x = (M * sc).astype(np.float32)  # exact: power-of-two scale
        out = []
        for _ in range(3):
            s = np.rint(x).astype(np.float32)
            out.append(s.astype(np.int64))
            x = ((x - s) * np.float32(256.0)).astype(np.float32)
        return out

    xs, ys = slices(X), slices(Y)

    def prod(p, q):  # A_p A_q^* as exact integer (re, im)
        return xs[p] @ xs[q].T + ys[p] @ ys[q].T, ys[p] @ xs[q].T - xs[p] @ ys[q].T

    # 2^32 H / 2^(e_i + e_j - 12) as exact integers: sum over slice pairs of 2^(32 - 8 (p + q)) A_p A_q^*
    Hr = np.zeros((len(mx), len(mx)), dtype=object)
    Hi = np.zeros((len(mx), len(mx)), dtype=object)
    for p in range(3):
        for q in range(3):
            re, im = prod(p, q)
            w = 1 << (32 - 8 * (p + q))
            Hr = Hr + re.astype(object) * w
            Hi = Hi + im.astype(object) * w
    scale = np.ldexp(1.0, (e[:, None] + e[None, :] - 44).astype(np.int64))
    return (Hr.astype(np.float64) + 1j * Hi.astype(np.float64)) * scale


def _leaf_matrix_as_gpu(c: Case, M, side: int, pair: int) -> np.ndarray:
    """The leaf matrix G^omega_tc exactly as the GPU forms it: complex64 entries of G
    times the FP32 weights 1/omega_b (the library's own), conjugated for the column side."""
    T = c.T
    invw = M.block_weights()
    off, ids = T.pair_blocks(side)
    cl = T.clusters()
    blk = T.blocks()
    pr = T.pairs(side)
    t = int(pr["cluster"][pair])
    r0, m = int(cl["start"][t]), int(cl["size"][t])
    G32 = c.G.astype(np.complex64)
    cols = []
    for b in ids[off[pair]:off[pair + 1]]:
        bt, bs = int(blk[b, 0]), int(blk[b, 1])
        w = np.float32(invw[b])
        if side == 0:
            blkm = G32[r0:r0 + m, cl["start"][bs]:cl["start"][bs] + cl["size"][bs]]
        else:
            blkm = G32[cl["start"][bt]:cl["start"][bt] + cl["size"][bt], r0:r0 + m].T.conj()
        cols.append((blkm.real.astype(np.float32) * w) + 1j * (blkm.imag.astype(np.float32) * w))
    return np.concatenate(cols, axis=1).astype(np.complex64)


@pytest.mark.parametrize("leaf,kappa,n,pts_kind", [(32, 8.0, 2048, "sphere"), (64, 12.0, 6144, "ellipsoid")])
def test_mixed_gram_is_exact(leaf, kappa, n, pts_kind):
    D = dev()
    pts = fibonacci_sphere(n) if pts_kind == "sphere" else random_ellipsoid(n)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa)[np.ix_(perm, perm)]

    class _C:
        pass

    c = _C()
    c.T, c.G = T, G
    M = D.dh2_compress(T, colmajor(G, torch.complex64), mode=D.MODE_MIXED_BF16X3, keep_gram=1)
    checked = 0
    for side in (0, 1):
        pr = T.pairs(side)
        leaves = np.flatnonzero(pr["leaf"])
        rng = np.random.default_rng(7 + side)
        # the widest pairs (several exact windows) and a seeded sample
        pick = list(leaves[np.argsort(-pr["ncols"][leaves])[:3]]) + list(rng.choice(leaves, 12, replace=False))
        for p in pick:
            A = _leaf_matrix_as_gpu(c, M, side, int(p))
            H = M.leaf_gram(side, int(p))
            Hx = _sliced_gram_exact(A)
            scale = np.max(np.abs(np.diag(Hx)))
            # exact up to the double-float rounding (2^-48) and the FP32 sum of the products of weight
            # 2^-40 and below (its rounding stays under 2^-44 of the diagonal)
            assert np.max(np.abs(H - Hx)) <= 2.0 ** -40 * scale, (side, p, np.max(np.abs(H - Hx)) / scale)
            # and close to the Gram matrix of A itself (slicing keeps 2^-23 of each row's largest entry)
            A64 = A.astype(np.complex128)
            assert np.max(np.abs(H - A64 @ A64.conj().T)) <= 1e-4 * scale
            checked += 1
    assert checked == 30


def test_mixed_parity_leaf32():
    c = Case(2048, 4.0, 32, 1e-4, dev().MODE_MIXED_BF16X3)
    assert c.launches[c.D.KC_LEAF_GRAM + 0] >= 1
    check_reduced(c, max_bad_frac=0.01, max_diff=1)


def test_mixed_parity_leaf64_all_classes():
    D = dev()
    pts = random_ellipsoid(6144)
    c = Case(6144, 12.0, 64, 1e-4, D.MODE_MIXED_BF16X3, pts=pts)
    for k in range(4):
        assert c.launches[D.KC_LEAF_GRAM + k] >= 1, k
        assert c.launches[D.KC_LEAF_FACTOR + k] >= 1, k
    check_reduced(c, max_bad_frac=0.01, max_diff=1)


def test_mixed_config2():
    check_reduced(Case(8192, 16.0, 32, 1e-4, dev().MODE_MIXED_BF16X3), max_bad_frac=0.01, max_diff=1)


def test_mixed_paper_parameters():
    c = Case(4096, 12.0, 64, 1e-4, dev().MODE_MIXED_BF16X3, eta1=20.0, eta2=5.0)
    check_reduced(c, max_bad_frac=0.01, max_diff=1)


def test_mixed_below_1e5_takes_the_fp32_leaf_step():
    """The Gram path squares the singular values, so below eps = 1e-5 it no longer resolves the
    tail sums: there the mixed mode runs the FP32 mode's leaf step (its ranks and storage are the
    FP32 mode's), unless keep_gram asks for the Gram matrices; at 1e-5 it keeps the Gram path."""
    D = dev()
    pts = fibonacci_sphere(4096)
    T = D.dh2_tree_build(pts, 32, 12.0)
    G = helmholtz_matrix(pts, 12.0)[np.ix_(T.perm(), T.perm())]
    Gd = colmajor(G, torch.complex64)
    Mm = D.dh2_compress(T, Gd, eps=1e-5, mode=D.MODE_MIXED_BF16X3)
    assert Mm.leaf_split_ms()[0] > 0  # the Gram launches ran
    Mm = D.dh2_compress(T, Gd, eps=1e-6, mode=D.MODE_MIXED_BF16X3)
    Mf = D.dh2_compress(T, Gd, eps=1e-6, mode=D.MODE_FP32)
    assert Mm.leaf_split_ms()[0] == 0
    for side in (0, 1):
        assert np.array_equal(Mm.ranks(side), Mf.ranks(side))
    assert Mm.storage() == Mf.storage()
    Mk = D.dh2_compress(T, Gd, eps=1e-6, mode=D.MODE_MIXED_BF16X3, keep_gram=1)
    assert Mk.leaf_split_ms()[0] > 0


def test_mixed_wait_bound_reports_timeout():
    D = dev()
    from paper_1510_07087_gb300 import _binding as B

    pts = fibonacci_sphere(2048)
    T = D.dh2_tree_build(pts, 32, 4.0)
    G = helmholtz_matrix(pts, 4.0)[np.ix_(T.perm(), T.perm())]
    Gd = colmajor(G, torch.complex64)
    p = B._params(1e-4, 2.0 / 3.0, 0, D.MODE_MIXED_BF16X3, 0, 0, spin_limit=1)
    h = ctypes.c_void_p(0xBEEF)
    st = B._lib().dh2_compress(T.handle, ctypes.c_void_p(Gd.data_ptr()), B.DH2_C64, B._colmajor_ld(Gd),
                               ctypes.byref(p), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               ctypes.byref(h))
    assert st == DH2_ETIMEOUT and h.value is None
    M = D.dh2_compress(T, Gd, mode=D.MODE_MIXED_BF16X3)  # default bound: completes
    assert max(M.ranks(0)) > 0


def test_mixed_mode_rejects_matrix_free_and_wide_leaves():
    D = dev()
    pts = fibonacci_sphere(1024)
    T = D.dh2_tree_build(pts, 32, 4.0)
    with pytest.raises(D.DH2Error):
        D.dh2_compress_kernel(T, pts, 4.0, 1.0, mode=D.MODE_MIXED_BF16X3)
    T128 = D.dh2_tree_build(pts, 128, 4.0)  # leaves of 128 points
    assert T128.stats().max_leaf > 64
    G = helmholtz_matrix(pts, 4.0)[np.ix_(T128.perm(), T128.perm())]
    with pytest.raises(D.DH2Error):
        D.dh2_compress(T128, colmajor(G, torch.complex64), mode=D.MODE_MIXED_BF16X3)
