"""The captured schedule (dh2_plan_*) and batches of many small problems.

  * a plan replays the kernel sequence of dh2_compress / dh2_compress_batched
    as one CUDA graph: its ranks, singular values and storage equal the direct
    call's on the same matrices, for one problem (FP32, FP64 and the mixed
    mode) and for a batch;
  * a replay on another matrix of the same shape gives that matrix's
    compression, and a replay on the first matrix gives the first result again;
  * sixteen small problems of uneven size in one batched call each meet the
    FP64 parity criteria against the oracle (ranks outside ties, products,
    errors and storage).
"""
import math

import numpy as np
import pytest

from gpu_cases import Case, check_fp64, colmajor, dev
from synth import (fibonacci_sphere, helmholtz_matrix, random_cube_surface, random_ellipsoid, random_sphere,
                   SEED)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _same(Ma, Mb, T, pairs_checked=40):
    for side in (0, 1):
        ra, rb = Ma.ranks(side), Mb.ranks(side)
        assert np.array_equal(ra, rb), side
        rng = np.random.default_rng(3 + side)
        for p in rng.choice(len(ra), min(pairs_checked, len(ra)), replace=False):
            assert np.array_equal(Ma.sigma(side, int(p)), Mb.sigma(side, int(p))), (side, p)
    assert Ma.storage() == Mb.storage()


def _problem(n, kappa, leaf, dtype, pts=None, kappa_matrix=None):
    D = dev()
    pts = fibonacci_sphere(n) if pts is None else pts
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa if kappa_matrix is None else kappa_matrix)[np.ix_(perm, perm)]
    return T, G, colmajor(G, dtype)


@pytest.mark.parametrize("kind", ["fp32", "fp64", "mixed"])
def test_plan_equals_direct_call(kind):
    D = dev()
    if kind == "mixed":
        T, G, Gd = _problem(4096, 12.0, 64, torch.complex64, pts=random_ellipsoid(4096))
        mode = D.MODE_MIXED_BF16X3
    else:
        dt = torch.complex64 if kind == "fp32" else torch.complex128
        T, G, Gd = _problem(2048, 4.0, 32, dt)
        mode = D.MODE_FP32 if kind == "fp32" else D.MODE_FP64
    P = D.Plan([T], [Gd], eps=1e-4, mode=mode)
    P.run()
    P.wait()
    Mp = P.matrices()[0]
    Md = D.dh2_compress(T, Gd, eps=1e-4, mode=mode)
    _same(Mp, Md, T)
    assert Mp.launch_count() == Md.launch_count()
    G128 = colmajor(G, torch.complex128)
    ep, ed = D.dh2_error(Mp, G128), D.dh2_error(Md, G128)
    assert ep <= 1e-4 and abs(ep - ed) <= 1e-12 * ed


def test_plan_replays_on_new_matrices():
    D = dev()
    T, G1, Gd1 = _problem(2048, 6.0, 32, torch.complex64)
    _, G2, Gd2 = _problem(2048, 6.0, 32, torch.complex64, kappa_matrix=7.0)  # same tree, another matrix
    P = D.Plan([T], [Gd1], eps=1e-4)
    P.run()
    P.wait()
    r1 = [P.matrices()[0].ranks(s) for s in (0, 1)]
    P.run([Gd2])
    P.wait()
    M2 = D.dh2_compress(T, Gd2, eps=1e-4)
    _same(P.matrices()[0], M2, T)
    assert any(not np.array_equal(r1[s], M2.ranks(s)) for s in (0, 1))  # the inputs really differ
    P.run([Gd1])
    P.wait()
    M1 = D.dh2_compress(T, Gd1, eps=1e-4)
    _same(P.matrices()[0], M1, T)
    # a matrix of another leading dimension is refused before anything runs
    wide = torch.zeros((2048, 2050), dtype=torch.complex64, device="cuda").t()[:2048]  # column-major, ld 2050
    assert wide.stride() == (1, 2050)
    with pytest.raises(ValueError):
        P.run([wide])


def _batch(n_prob, lo, hi, dtype, seed_off=0):
    D = dev()
    rng = np.random.default_rng(SEED + seed_off)
    gens = [(random_sphere, 2.0), (random_ellipsoid, 2.0), (random_cube_surface, math.sqrt(3.0))]
    out = []
    for i in range(n_prob):
        g, diam = gens[i % 3]
        n = int(rng.integers(lo, hi + 1))
        kappa = float(rng.uniform(8.0, 40.0)) / diam
        pts = g(n, seed=SEED + seed_off + i)
        out.append((pts, kappa))
    return out


def test_plan_of_a_batch_equals_batched_call():
    D = dev()
    trees, Gs = [], []
    for pts, kappa in _batch(6, 1024, 3072, torch.complex64):
        T = D.dh2_tree_build(pts, 32, kappa)
        G = helmholtz_matrix(pts, kappa)[np.ix_(T.perm(), T.perm())]
        trees.append(T)
        Gs.append(colmajor(G, torch.complex64))
    P = D.Plan(trees, Gs, eps=1e-4)
    P.run()
    P.wait()
    Mb = D.dh2_compress_batched(trees, Gs, eps=1e-4)
    for T, Mp, M in zip(trees, P.matrices(), Mb):
        _same(Mp, M, T, pairs_checked=10)


def test_sixteen_small_problems_in_one_batch_against_the_oracle():
    D = dev()
    cases = []
    for pts, kappa in _batch(16, 400, 1100, torch.complex128, seed_off=100):
        cases.append(Case(len(pts), kappa, 24, 1e-4, D.MODE_FP64, pts=pts, compress=False))
    Mb = D.dh2_compress_batched([c.T for c in cases], [c.Gd for c in cases], eps=1e-4)
    for c, M in zip(cases, Mb):
        c.attach(M)
        check_fp64(c)
