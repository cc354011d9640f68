"""Shared set-up of the GPU parity tests: one compression through the C ABI
beside the FP64 oracle on the same seeded input, and the parity criteria.

Parity rules (ranks, subspaces and products are compared; Q, E and S are
unique only up to unitary changes and are never compared entrywise):
  * FP64 mode: ranks equal to the oracle's except at truncation ties
    (|sum_{i>=k} sigma_i^2 - eps_l^2| <= 1e-8 eps_l^2 for a k between the two);
    with the oracle re-run at the GPU's ranks, y = G~ x agrees to 1e-11
    relative for three seeded right-hand sides; blockwise error, storage
    counts and coupling norms agree with the oracle's.
  * Reduced-precision modes (complex64 input): singular values carry absolute
    errors of a few u_32 * sigma_1, so a rank can differ from the FP64
    oracle's where a tail sum lies near the threshold.  The tests bound the
    fraction of ranks that differ outside ties of 1e-3 eps_l^2 and the size of
    a difference, require |G - G~|_F <= eps |G|_F against the complex128
    matrix, and bound the matrix-vector product against the FP64 oracle at the
    GPU's ranks by the triangle inequality: both products approximate G x to
    eps |G|_F |x|, so they differ by at most 2 eps |G|_F |x|.
"""
import math

import numpy as np
import pytest

from oracle import dh2_oracle as O
from synth import fibonacci_sphere, helmholtz_matrix, random_complex_vectors

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_07087_gb300 as D
    return D


def colmajor(G: np.ndarray, dtype):
    """Column-major device copy: memory of G^T row-major == G column-major."""
    return torch.from_numpy(np.ascontiguousarray(G.T)).to(device="cuda", dtype=dtype).t()


def leaf_class(m: int) -> int:
    """Row class of a leaf pair (the library's leaf launches): <=32, <=40, <=48, <=64, more."""
    return 0 if m <= 32 else 1 if m <= 40 else 2 if m <= 48 else 3 if m <= 64 else 4


def level_class(p: int) -> int:
    """Row class of a non-leaf pair by k_t1c' + k_t2c': <=32, <=48, <=64, more."""
    return 0 if p <= 32 else 1 if p <= 48 else 2 if p <= 64 else 3


class Case:
    """One compression of a seeded Helmholtz (or given) matrix on the GPU and by the oracle."""

    def __init__(self, n, kappa, leaf, eps, mode, eta1=2 * math.sqrt(2), eta2=1.0, G=None, dir_rule=0,
                 nearfield=0, pts=None, compress=True):
        D = dev()
        self.D = D
        pts = fibonacci_sphere(n) if pts is None else pts
        self.tp = O.TreeParams(leaf_size=leaf, kappa=kappa, eta1=eta1, eta2=eta2, dir_rule=dir_rule)
        self.cp = O.CompressParams(eps=eps)
        self.tr = O.build_tree(pts, self.tp)
        if G is None:
            G = helmholtz_matrix(pts, kappa)
        self.G = G[np.ix_(self.tr.perm, self.tr.perm)]
        self.T = D.dh2_tree_build(pts, leaf, kappa, eta1, eta2, dir_rule)
        assert np.array_equal(self.T.perm(), self.tr.perm)
        dt = torch.complex128 if mode == D.MODE_FP64 else torch.complex64
        self.Gd = colmajor(self.G, dt)
        self.mode = mode
        w = O.block_weights(self.tr, O.block_norms(self.tr, self.G), self.cp.zeta)
        self.w = w
        self.V = O.compress(self.tr, self.G, self.cp, "row", w)
        self.W = O.compress(self.tr, self.G, self.cp, "col", w)
        if compress:
            self.attach(D.dh2_compress(self.T, self.Gd, eps=eps, mode=mode, nearfield=nearfield))

    def attach(self, M):
        """Take M (a compression of this case's tree and matrix) as the GPU result: its ranks, and the
        oracle re-run at them."""
        self.M = M
        self.launches = self.M.class_launches()
        self.rank = {}
        self.pid = {}
        for side in (0, 1):
            pr = self.T.pairs(side)
            rk = self.M.ranks(side)
            self.rank[side] = {(int(pr["cluster"][p]), int(pr["dir"][p])): int(rk[p]) for p in range(len(rk))}
            for p in range(len(rk)):
                self.pid[(side, int(pr["cluster"][p]), int(pr["dir"][p]))] = p
        w = self.w
        self.Vg = O.compress(self.tr, self.G, self.cp, "row", w, rank_override=self.rank[0])
        self.Wg = O.compress(self.tr, self.G, self.cp, "col", w, rank_override=self.rank[1])
        self.Sg = O.project(self.tr, self.G, self.Vg, self.Wg)

    def gpu_matvec(self, x: np.ndarray) -> np.ndarray:
        dt = self.Gd.dtype
        xd = torch.from_numpy(np.ascontiguousarray(x.T)).to(device="cuda", dtype=dt).t()
        yd = torch.empty_like(xd.t().contiguous()).t()
        self.D.dh2_matvec(self.M, xd, yd)
        torch.cuda.synchronize()
        return yd.cpu().numpy().astype(np.complex128)

    def leaf_classes(self) -> set:
        """Row classes of the leaf pairs of both sides (from the oracle's tree)."""
        out = set()
        for B in (self.V, self.W):
            for t in range(self.tr.nclusters()):
                if self.tr.is_leaf(t) and B.F[t]:
                    out.add(leaf_class(self.tr.size[t]))
        return out

    def level_classes(self) -> set:
        """Row classes of the non-leaf pairs of both sides at the GPU's ranks."""
        out = set()
        for side, B in ((0, self.V), (1, self.W)):
            for (t, c) in B.rank:
                if self.tr.sons[t]:
                    cs = int(self.tr.sd[self.tr.level[t]][c])
                    out.add(level_class(sum(self.rank[side][(s, cs)] for s in self.tr.sons[t])))
        return out


def tie(sig, k1, k2, eps2, tol):
    s2 = np.concatenate([np.asarray(sig, dtype=np.float64) ** 2, [0.0]])
    tails = np.cumsum(s2[::-1])[::-1]
    lo, hi = min(k1, k2), max(k1, k2)
    return any(abs(tails[min(k, len(tails) - 1)] - eps2) <= tol * eps2 for k in range(lo, hi + 1))


def rank_report(c: Case, tol):
    """(ranks differing outside ties, ties, total, largest |difference|)."""
    bad, ties, total, dmax = 0, 0, 0, 0
    for side, B in ((0, c.V), (1, c.W)):
        for key, ko in B.rank.items():
            kg = c.rank[side][key]
            total += 1
            dmax = max(dmax, abs(kg - ko))
            if kg != ko:
                if tie(B.sigma[key], kg, ko, B.eps_level[c.tr.level[key[0]]] ** 2, tol):
                    ties += 1
                else:
                    bad += 1
    return bad, ties, total, dmax


def check_fp64(c: Case, mv_tol=1e-11):
    bad, ties, total, _ = rank_report(c, 1e-8)
    assert bad == 0, f"{bad} rank mismatches outside ties ({ties} ties) of {total}"
    x = random_complex_vectors(c.tr.n, 3, seed=11)
    y_ref = O.matvec(c.tr, c.G, c.Vg, c.Wg, c.Sg, x)
    y = c.gpu_matvec(x)
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert rel <= mv_tol, rel
    err_gpu = c.D.dh2_error(c.M, c.Gd)
    err_ora = O.error_fro(c.tr, c.G, c.Vg, c.Wg, c.Sg)
    assert err_gpu <= c.cp.eps
    assert abs(err_gpu - err_ora) <= 1e-6 * err_ora + 1e-14
    st = c.M.storage()
    so = O.storage(c.tr, c.Vg, c.Wg, c.Sg)
    for k in ("V", "W", "S", "near"):
        assert st[k] == so[k], k
    assert st["E_V"] == so["E_V"] and st["E_W"] == so["E_W"]


def check_reduced(c: Case, max_bad_frac, max_diff, seed=12, mv_tol=1e-5):
    """Reduced-precision criteria (module docstring); returns the report for printing.

    Besides the triangle-inequality bound, the product at equal ranks must
    agree with the FP64 oracle to mv_tol: the two differ only by rounding in
    the stored complex64 representation and in the subspaces, measured at
    3e-7 to 1.3e-6 relative (a few u_32 times the number of terms) on the
    cases of the suite."""
    bad, ties, total, dmax = rank_report(c, 1e-3)
    x = random_complex_vectors(c.tr.n, 3, seed=seed)
    y_ref = O.matvec(c.tr, c.G, c.Vg, c.Wg, c.Sg, x)
    y = c.gpu_matvec(x)
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    bound = 2.0 * c.cp.eps * np.linalg.norm(c.G) * np.linalg.norm(x) / np.linalg.norm(y_ref)
    err = c.D.dh2_error(c.M, colmajor(c.G, torch.complex128))
    rep = dict(bad=bad, ties=ties, total=total, max_diff=dmax, matvec_rel=rel, matvec_bound=bound, err=err)
    print(f"reduced-precision report (eps={c.cp.eps:g}): {rep}")
    assert bad <= max_bad_frac * total, rep
    assert dmax <= max_diff, rep
    assert rel <= bound, rep
    assert rel <= mv_tol, rep
    assert err <= c.cp.eps, rep
    return rep


def fp64_case(n, kappa, leaf, eps, **kw):
    return Case(n, kappa, leaf, eps, dev().MODE_FP64, **kw)


def fp32_case(n, kappa, leaf, eps, **kw):
    return Case(n, kappa, leaf, eps, dev().MODE_FP32, **kw)
