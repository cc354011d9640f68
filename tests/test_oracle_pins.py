"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than the oracle
itself: brute-force enumeration, a different library routine, an identity the
paper proves (Pythagoras split Eq. error_nonleaf, the Error-estimate theorem,
best approximation by orthogonal projection), a closed form, or a special case
(planted low rank, near-exact tolerance, kappa = 0).
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import dh2_oracle as O
from synth import fibonacci_sphere, helmholtz_matrix, planted_separable_matrix, random_sphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _setup(n, kappa, leaf, eps=1e-4, pts=None, G=None, dir_rule=0, eta2=1.0, err_mode=0,
           eta1=2 * math.sqrt(2)):
    if pts is None:
        pts = fibonacci_sphere(n)
    if G is None:
        G = helmholtz_matrix(pts, kappa)
    tp = O.TreeParams(leaf_size=leaf, kappa=kappa, dir_rule=dir_rule, eta2=eta2, eta1=eta1)
    cp = O.CompressParams(eps=eps, err_mode=err_mode)
    tr, V, W, S, Gp = O.run(pts, G, tp, cp)
    return dict(tr=tr, V=V, W=W, S=S, G=Gp, cp=cp, tp=tp, pts=pts)


@pytest.fixture(scope="module")
def small():
    return _setup(1024, 6.0, 16)


@pytest.fixture(scope="module")
def medium():
    return _setup(2048, 4.0, 32)


@pytest.fixture(scope="module")
def paper_params():
    """The paper's parameter set (Section 7): eta1 = 20, eta2 = 5, many coarse admissible blocks."""
    return _setup(2048, 8.0, 16, eta1=20.0, eta2=5.0)


# ---------------------------------------------------------------- trees

def test_cluster_tree_partitions(small):
    tr = small["tr"]
    assert sorted(tr.perm.tolist()) == list(range(tr.n))
    pts = small["pts"][tr.perm]
    for t in range(tr.nclusters()):
        idx = slice(tr.start[t], tr.start[t] + tr.size[t])
        P = pts[idx]
        # Def. 1: sons partition the father (contiguous in the permuted order)
        if tr.sons[t]:
            s1, s2 = tr.sons[t]
            assert tr.start[s1] == tr.start[t]
            assert tr.start[s2] == tr.start[s1] + tr.size[s1]
            assert tr.size[s1] + tr.size[s2] == tr.size[t]
            assert tr.level[s1] == tr.level[t] + 1
        else:
            assert tr.size[t] <= tr.tp_leaf if hasattr(tr, "tp_leaf") else tr.size[t] <= small["tp"].leaf_size
        # bounding boxes contain the supports (here: the points)
        assert np.all(P >= np.array(tr.lo[t]) - 0.0) and np.all(P <= np.array(tr.hi[t]) + 0.0)


def test_block_leaves_partition_index_pairs():
    """Def. 2: the leaves of the block tree partition I x I (brute force)."""
    d = _setup(512, 5.0, 16)
    tr = d["tr"]
    cover = np.zeros((tr.n, tr.n), dtype=np.int32)
    for t, s, adm, c in tr.blocks:
        cover[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]] += 1
        assert tr.level[t] == tr.level[s]
    assert np.all(cover == 1)


def _gap_dist(tr, t, s):
    # independent restatement: per-axis gap between the intervals
    g = []
    for a in range(3):
        lo = max(tr.lo[t][a], tr.lo[s][a])
        hi = min(tr.hi[t][a], tr.hi[s][a])
        g.append(max(lo - hi, 0.0))
    return float(np.linalg.norm(g))


def test_admissibility_conditions(small):
    tr, tp = small["tr"], small["tp"]
    pts = small["pts"][tr.perm]
    for t, s, adm, c in tr.blocks:
        md = max(tr.diam[t], tr.diam[s])
        d = _gap_dist(tr, t, s)
        if adm:
            # Eqs. (adm_standard) and (adm_parabolic)
            assert md <= tp.eta2 * d * (1 + 1e-14)
            assert tp.kappa * md * md <= tp.eta2 * d * (1 + 1e-14)
            # box distance never exceeds the point distance
            P = pts[tr.start[t]:tr.start[t] + tr.size[t]]
            Qp = pts[tr.start[s]:tr.start[s] + tr.size[s]]
            dmin = np.sqrt(((P[:, None, :] - Qp[None, :, :]) ** 2).sum(-1)).min()
            assert d <= dmin * (1 + 1e-14)
            # Eq. (adm_directional) holds by the covering property of D_l
            u = (np.array(tr.center[t]) - np.array(tr.center[s]))
            u /= np.linalg.norm(u)
            D = tr.dirs[tr.level[t]]
            assert np.linalg.norm(u - D[c]) <= tp.eta1 / (tp.kappa * tr.delta[tr.level[t]]) + 1e-12
            assert np.linalg.norm(u - D[c]) <= np.linalg.norm(u - D, axis=1).min() + 1e-15
        else:
            assert tr.is_leaf(t) or tr.is_leaf(s)


def test_directions_golden_m2():
    ref = np.loadtxt(os.path.join(GOLDEN, "cube_directions_m2.txt"))
    got = O.cube_directions(2)
    assert got.shape == (24, 3)
    np.testing.assert_allclose(got, ref, atol=2e-16, rtol=0)
    np.testing.assert_allclose(O.cube_directions(1),
                               [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], atol=0)


@pytest.mark.parametrize("kappa,delta,eta1", [(4.0, 3.4, 2 * math.sqrt(2)), (16.0, 1.7, 2 * math.sqrt(2)),
                                              (30.0, 2.0, 20.0), (7.0, 0.9, 1.0)])
def test_direction_covering_radius(kappa, delta, eta1):
    """Section 3: every unit z lies within eta1/(kappa delta) of D_l (Lemma Projection)."""
    D = O.level_directions(kappa, delta, eta1, 0)
    np.testing.assert_allclose(np.linalg.norm(D, axis=1), 1.0, atol=1e-15)
    # D = -D (up to rounding): the construction is symmetric
    for c in D:
        assert np.min(np.linalg.norm(D + c, axis=1)) < 1e-14
    z = np.random.default_rng(1).standard_normal((20000, 3))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    near = np.sqrt(((z[:, None, :] - D[None, :, :]) ** 2).sum(-1)).min(1)
    assert near.max() <= eta1 / (kappa * delta)


def test_son_map_is_nearest(small):
    tr = small["tr"]
    for l in range(tr.depth):
        D0, D1 = tr.dirs[l], tr.dirs[l + 1]
        for i in range(0, len(D0), max(1, len(D0) // 40)):
            best = min(range(len(D1)), key=lambda j: (float(np.sum((D0[i] - D1[j]) ** 2)), j))
            assert np.isclose(np.linalg.norm(D0[i] - D1[tr.sd[l][i]]), np.linalg.norm(D0[i] - D1[best]),
                              rtol=0, atol=1e-15)


def test_column_sets_disjoint_and_nested(small):
    """F_tc are disjoint over c (proof of the compression-complexity theorem) and
    F_tc is contained in F_{t'c'} for each son t' (Section 6, Ghat from R)."""
    tr = small["tr"]
    for side in ("row", "col"):
        F = O.column_sets(tr, side)
        for t in range(tr.nclusters()):
            seen = set()
            total = 0
            for c, bl in F[t].items():
                assert not (seen & set(bl))
                seen |= set(bl)
                for b in bl:
                    bt, bs, _, _ = tr.blocks[b]
                    total += tr.size[bs] if side == "row" else tr.size[bt]
                for son in tr.sons[t]:
                    cs = int(tr.sd[tr.level[t]][c])
                    assert set(bl) <= set(F[son][cs])
            assert total <= tr.n


# ---------------------------------------------------------------- compression

def test_leaf_basis_is_truncated_svd_subspace(medium):
    """Leaf step: Q_tc spans the leading left singular vectors of G^omega_tc,
    checked against a Hermitian eigensolver (scipy eigh) of G G^*."""
    tr, V, G, cp = medium["tr"], medium["V"], medium["G"], medium["cp"]
    w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
    checked = 0
    for (t, c), Q in V.Q.items():
        A = np.concatenate([G[tr.start[t]:tr.start[t] + tr.size[t],
                              tr.start[tr.blocks[b][1]]:tr.start[tr.blocks[b][1]] + tr.size[tr.blocks[b][1]]] / w[b]
                            for b in V.F[t][c]], axis=1)
        lam, U = scipy.linalg.eigh(A @ A.conj().T)
        lam, U = lam[::-1], U[:, ::-1]
        k = Q.shape[1]
        eps2 = V.eps_level[tr.level[t]] ** 2
        tail = np.clip(lam, 0, None)
        # rank: tail after k within tolerance, tail after k-1 above (up to Gram rounding)
        slack = 1e-12 * lam[0]
        assert tail[k:].sum() <= eps2 + slack
        if k > 0:
            assert tail[k - 1:].sum() > eps2 - slack
        # Eckart-Young: the residual of span Q is the smallest possible for rank k
        res = np.linalg.norm(A - Q @ (Q.conj().T @ A)) ** 2
        assert abs(res - tail[k:].sum()) <= slack + 1e-9 * eps2
        # the well-separated dominant eigenvectors of A A^* lie in span Q
        for j in range(k, 0, -1):
            if lam[j - 1] - lam[j] > 1e-4 * lam[0]:
                Uj = U[:, :j]
                assert np.linalg.norm(Uj - Q @ (Q.conj().T @ Uj)) < 1e-9
                checked += 1
                break
    assert checked > 20


def test_orthonormal_bases(medium):
    tr, V, W = medium["tr"], medium["V"], medium["W"]
    for B in (V, W):
        for Q in B.Q.values():
            assert np.linalg.norm(Q.conj().T @ Q - np.eye(Q.shape[1])) < 1e-13
        cache = {}
        for (t, c) in B.rank:
            X = O.expand_basis(tr, B, t, c, cache)
            assert X.shape == (tr.size[t], B.rank[(t, c)])
            assert np.linalg.norm(X.conj().T @ X - np.eye(X.shape[1])) < 1e-12
            if tr.sons[t]:
                # Eq. (nested): V_tc restricted to t' equals V_t'c' E_t'c
                cs = int(tr.sd[tr.level[t]][c])
                for son in tr.sons[t]:
                    r = slice(tr.start[son] - tr.start[t], tr.start[son] - tr.start[t] + tr.size[son])
                    np.testing.assert_allclose(X[r], cache[(son, cs)] @ B.E[(son, c)], atol=1e-14)


def _Gw(tr, G, w, t, c, F, side):
    return np.concatenate([O._block_matrix(tr, G, side, b, t) / w[b] for b in F[t][c]], axis=1)


@pytest.mark.parametrize("side", ["row", "col"])
@pytest.mark.parametrize("which", ["medium", "paper_params"])
def test_pythagoras_split_and_error_estimate(which, side, request):
    """Eq. (error_nonleaf) as an equality for every non-leaf (t, c), and the
    Error-estimate theorem |G_tc - QQ^*G_tc|^2 <= sum_{r in desc(t)} eps_r^2."""
    medium = request.getfixturevalue(which)
    tr, G, cp = medium["tr"], medium["G"], medium["cp"]
    w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
    B = O.compress(tr, G, cp, side, w, keep_R=True)
    cache = {}
    ndesc_eps2 = {}
    for t in reversed(range(tr.nclusters())):
        e = B.eps_level[tr.level[t]] ** 2
        ndesc_eps2[t] = e + sum(ndesc_eps2[s] for s in tr.sons[t])
    nonleaf = 0
    for (t, c), k in B.rank.items():
        A = _Gw(tr, G, w, t, c, B.F, side)
        X = O.expand_basis(tr, B, t, c, cache)
        err = np.linalg.norm(A - X @ (X.conj().T @ A)) ** 2
        assert err <= ndesc_eps2[t] * (1 + 1e-9) + 1e-28
        if tr.sons[t]:
            cs = int(tr.sd[tr.level[t]][c])
            rhs = 0.0
            parts = []
            for son in tr.sons[t]:
                Xs = O.expand_basis(tr, B, son, cs, cache)
                r = slice(tr.start[son] - tr.start[t], tr.start[son] - tr.start[t] + tr.size[son])
                As = A[r]
                rhs += np.linalg.norm(As - Xs @ (Xs.conj().T @ As)) ** 2
                parts.append(Xs.conj().T @ As)
            Gh = np.concatenate(parts, axis=0)
            Qh = np.concatenate([B.E[(son, c)] for son in tr.sons[t]], axis=0)
            rhs += np.linalg.norm(Gh - Qh @ (Qh.conj().T @ Gh)) ** 2
            assert abs(err - rhs) <= 1e-10 * max(err, 1e-30) + 1e-26
            # R recursion: R_tc = Qhat^* Ghat equals Q_tc^* G^omega_tc
            np.testing.assert_allclose(B.R[(t, c)][0], X.conj().T @ A, atol=1e-11 * np.abs(A).max())
            nonleaf += 1
    assert nonleaf >= 5


@pytest.mark.parametrize("which", ["medium", "paper_params"])
def test_block_error_bounds_and_closed_form(which, request):
    """Best approximation by orthogonal projection: |G_b - V S_b W^*|^2 = |G_b|^2 - |S_b|^2;
    per block |G_b - V V^* G_b| <= eps_hat |G_b| / sqrt(1 - 2 zeta^2) (Remark "Error control")."""
    medium = request.getfixturevalue(which)
    tr, V, W, S, G, cp = medium["tr"], medium["V"], medium["W"], medium["S"], medium["G"], medium["cp"]
    eh = O.eps_hat(cp)
    bound = eh / math.sqrt(1 - 2 * cp.zeta ** 2)
    cv, cw = {}, {}
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        if not adm:
            continue
        Gb = G[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]]
        Vt = O.expand_basis(tr, V, t, c, cv)
        Ws = O.expand_basis(tr, W, s, c, cw)
        nb = np.linalg.norm(Gb)
        e2 = np.linalg.norm(Gb - Vt @ S[b] @ Ws.conj().T) ** 2
        assert abs(e2 - (nb ** 2 - np.linalg.norm(S[b]) ** 2)) <= 1e-11 * nb ** 2
        assert np.linalg.norm(Gb - Vt @ (Vt.conj().T @ Gb)) <= bound * nb * (1 + 1e-9)
        assert np.linalg.norm(Gb - (Gb @ Ws) @ Ws.conj().T) <= bound * nb * (1 + 1e-9)


@pytest.mark.parametrize("n,kappa,leaf,eps", [(2048, 4.0, 32, 1e-4), (2048, 8.0, 32, 1e-6), (1024, 12.0, 16, 1e-3)])
def test_global_error_bound(n, kappa, leaf, eps):
    d = _setup(n, kappa, leaf, eps=eps)
    err = O.error_fro(d["tr"], d["G"], d["V"], d["W"], d["S"])
    assert err <= eps
    Gt = O.dense_approximation(d["tr"], d["G"], d["V"], d["W"], d["S"])
    np.testing.assert_allclose(np.linalg.norm(d["G"] - Gt) / np.linalg.norm(d["G"]), err, rtol=1e-6)


def test_near_exact_tolerance():
    d = _setup(1024, 6.0, 16, eps=1e-15)
    assert O.error_fro(d["tr"], d["G"], d["V"], d["W"], d["S"]) <= 1e-13


def test_planted_low_rank():
    pts = fibonacci_sphere(1024)
    G = planted_separable_matrix(pts, rank=3)
    d = _setup(1024, 6.0, 16, eps=1e-10, pts=pts, G=G)
    assert max(d["V"].rank.values()) <= 3 and max(d["W"].rank.values()) <= 3
    assert O.error_fro(d["tr"], d["G"], d["V"], d["W"], d["S"]) <= 1e-10


def test_kappa_zero_standard_h2():
    """kappa = 0 with the zero-direction rule: one direction per level (standard H^2)."""
    pts = fibonacci_sphere(1024)
    G = helmholtz_matrix(pts, 0.0)
    d = _setup(1024, 0.0, 16, pts=pts, G=G, dir_rule=1, eta2=1.0)
    tr = d["tr"]
    assert all(len(D) == 1 and np.all(D == 0) for D in tr.dirs)
    assert all(c == 0 for (_, _, adm, c) in tr.blocks if adm)
    assert O.error_fro(tr, d["G"], d["V"], d["W"], d["S"]) <= 1e-4


def test_small_n_no_admissible_blocks():
    d = _setup(24, 4.0, 32)
    assert not any(adm for (_, _, adm, _) in d["tr"].blocks)
    Gt = O.dense_approximation(d["tr"], d["G"], d["V"], d["W"], d["S"])
    assert np.array_equal(Gt, d["G"])


def test_row_column_symmetry(medium):
    """For complex-symmetric G and D = -D, span W_{s,-c} = conj(span V_{s,c})."""
    tr, V, W = medium["tr"], medium["V"], medium["W"]
    assert np.allclose(medium["G"], medium["G"].T)
    checked = 0
    for (t, c), Q in V.Q.items():
        D = tr.dirs[tr.level[t]]
        neg = np.linalg.norm(D + D[c], axis=1)
        cm = int(np.argmin(neg))
        if neg[cm] > 1e-14 or (t, cm) not in W.Q:
            continue
        mirrored = {(tr.blocks[b][1], tr.blocks[b][0]) for b in V.F[t][c]}
        if mirrored != {(tr.blocks[b][0], tr.blocks[b][1]) for b in W.F[t][cm]}:
            continue  # a tie in the nearest-direction choice broke the mirror image
        sig = V.sigma[(t, c)]
        k = V.rank[(t, c)]
        eps2 = V.eps_level[tr.level[t]] ** 2
        tail = np.sum(sig[k:] ** 2)
        if abs(tail - eps2) < 1e-6 * eps2 or W.rank[(t, cm)] != k:
            # only an exact tie may differ
            assert abs(np.sum(sig[min(k, W.rank[(t, cm)]):] ** 2) - eps2) < 1e-3 * eps2
            continue
        P1 = Q @ Q.conj().T
        Wq = W.Q[(t, cm)].conj()
        P2 = Wq @ Wq.conj().T
        if k and (sig[k - 1] - (sig[k] if k < len(sig) else 0)) > 1e-4 * sig[0]:
            assert np.linalg.norm(P1 - P2) < 1e-7
        checked += 1
    assert checked > 20


def test_fast_matvec_equals_assembled(medium):
    tr, V, W, S, G = medium["tr"], medium["V"], medium["W"], medium["S"], medium["G"]
    x = np.random.default_rng(3).standard_normal((tr.n, 2)) + 1j * np.random.default_rng(4).standard_normal((tr.n, 2))
    y = O.matvec(tr, G, V, W, S, x)
    Gt = O.dense_approximation(tr, G, V, W, S)
    ref = Gt @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-14


def test_storage_count(medium):
    tr, V, W, S = medium["tr"], medium["V"], medium["W"], medium["S"]
    st = O.storage(tr, V, W, S)
    nq = sum(tr.size[t] * V.rank[(t, c)] for (t, c) in V.Q)
    assert st["V"] == nq
    assert st["S"] == sum(V.rank[(t, c)] * W.rank[(s, c)] for (t, s, adm, c) in tr.blocks if adm)
    assert st["near"] + sum(tr.size[t] * tr.size[s] for (t, s, adm, c) in tr.blocks if adm) == tr.n ** 2


def test_random_points_bound():
    pts = random_sphere(1024)
    d = _setup(1024, 8.0, 16, pts=pts)
    assert O.error_fro(d["tr"], d["G"], d["V"], d["W"], d["S"]) <= 1e-4


def test_planted_mistake_breaks_pythagoras(medium, monkeypatch):
    """A dropped conjugate in the column side's block matrix must be caught by a pin."""
    tr, G, cp = medium["tr"], medium["G"], medium["cp"]
    w = O.block_weights(tr, O.block_norms(tr, G), cp.zeta)
    orig = O._block_matrix

    def broken(tr_, G_, side, b, r):
        M = orig(tr_, G_, side, b, r)
        return M.conj() if side == "col" else M

    monkeypatch.setattr(O, "_block_matrix", broken)
    B = O.compress(tr, G, cp, "col", w)
    monkeypatch.setattr(O, "_block_matrix", orig)
    V = O.compress(tr, G, cp, "row", w)
    S = O.project(tr, G, V, B)
    # the column basis now approximates the wrong matrix: the global bound fails
    assert O.error_fro(tr, G, V, B, S) > cp.eps


# ---------------------------------------------------------------- split rule (Def. 1), by hand

def _son_sets(tr, t):
    return [sorted(tr.perm[tr.start[s]:tr.start[s] + tr.size[s]].tolist()) for s in tr.sons[t]]


def test_split_rule_midpoint_of_longest_side_by_hand():
    """Geometrically regular subdivision: halve the bounding box across its longest
    side; a point on the cutting plane goes to the first son.  The point set is
    chosen so that a median split, another axis or a strict '<' all differ."""
    P = np.array([
        [3.0, 0.0, 0.0],   # 0
        [0.0, 1.0, 0.0],   # 1
        [2.0, 0.0, 1.0],   # 2: on the plane x = 2 of the root's box [0,4]x[0,1]x[0,1]
        [4.0, 1.0, 1.0],   # 3
        [0.5, 0.0, 0.0],   # 4
        [1.5, 1.0, 0.0],   # 5
        [3.5, 0.0, 1.0],   # 6
        [1.0, 0.2, 0.7],   # 7: on the plane x = 1 of the first son's box [0,2]x[0,1]x[0,1]
    ])
    tr = O.build_tree(P, O.TreeParams(leaf_size=4, kappa=0.0))
    assert _son_sets(tr, 0) == [[1, 2, 4, 5, 7], [0, 3, 6]]
    s1, s2 = tr.sons[0]
    assert tr.sons[s2] == []                      # 3 points: a leaf
    assert _son_sets(tr, s1) == [[1, 4, 7], [2, 5]]
    assert tr.level[tr.sons[s1][0]] == 2 and tr.depth == 2
    # boxes are the points' bounding boxes, diameters their diagonals
    assert tr.lo[s1] == [0.0, 0.0, 0.0] and tr.hi[s1] == [2.0, 1.0, 1.0]
    assert tr.diam[s2] == pytest.approx(math.sqrt(1.0 + 1.0 + 1.0))


def test_split_rule_lowest_axis_on_ties_by_hand():
    """Equal extents along x and y: the cut is across x (the first axis)."""
    P = np.array([[0.0, 0.0, 0.0], [2.0, 2.0, 1.0], [0.5, 1.9, 0.0], [1.5, 0.1, 0.0]])
    tr = O.build_tree(P, O.TreeParams(leaf_size=2, kappa=0.0))
    assert _son_sets(tr, 0) == [[0, 2], [1, 3]]   # across y it would be [[0, 3], [1, 2]]


def test_single_point_clusters_and_duplicates_stop():
    """Coincident points cannot be separated by a cut: the cluster stays a leaf."""
    P = np.zeros((5, 3))
    tr = O.build_tree(P, O.TreeParams(leaf_size=2, kappa=0.0))
    assert tr.nclusters() == 1 and tr.size[0] == 5


# ---------------------------------------------------------------- weights (Remark "Error control")

def _single_block_leaf_pairs(tr, B):
    """Leaf pairs (t, c) whose F_tc holds exactly one block, that block's row cluster being t."""
    out = []
    for t, cmap in B.F.items():
        if not tr.is_leaf(t):
            continue
        for c, blocks in cmap.items():
            if len(blocks) == 1:
                bt, bs, _, _ = tr.blocks[blocks[0]]
                if (bt if B.side == "row" else bs) == t:
                    out.append((t, c, blocks[0]))
    return out


@pytest.mark.parametrize("side", ["row", "col"])
def test_weights_make_leaf_truncation_block_relative(medium, side):
    """With omega_b = |G_b| zeta^-level(t) and eps_r ~ zeta^level(r), a leaf pair whose
    only block is b = (t, s) is truncated block-relatively and level-free: its rank is
    the least k with sum_{i>k} sigma_i(G_b)^2 <= eps_hat^2 |G_b|^2, sigma_i taken here
    from G_b itself.  A wrong norm power or exponent sign changes these ranks."""
    tr, G, cp = medium["tr"], medium["G"], medium["cp"]
    B = medium["V"] if side == "row" else medium["W"]
    eh = O.eps_hat(cp)
    pairs = _single_block_leaf_pairs(tr, B)
    checked = 0
    for t, c, b in pairs:
        bt, bs, _, _ = tr.blocks[b]
        Gb = G[tr.start[bt]:tr.start[bt] + tr.size[bt], tr.start[bs]:tr.start[bs] + tr.size[bs]]
        if side == "col":
            Gb = Gb.conj().T
        sig = scipy.linalg.svdvals(Gb)
        thr = (eh * np.linalg.norm(Gb)) ** 2
        tails = np.array([np.sum(sig[k:] ** 2) for k in range(len(sig) + 1)])
        k = int(np.argmax(tails <= thr))
        if abs(tails[k] - thr) < 1e-6 * thr or (k > 0 and abs(tails[k - 1] - thr) < 1e-6 * thr):
            continue  # a tie at the threshold: either rank is right
        assert B.rank[(t, c)] == k, (t, c, B.rank[(t, c)], k)
        checked += 1
    assert checked >= 10, (len(pairs), checked)


def test_block_scaling_by_powers_of_two_leaves_bases_unchanged(medium):
    """omega_b proportional to |G_b|: scaling one admissible block by 2^j leaves every
    G^omega_tc, hence every rank and basis, bit-identical."""
    tr, G, cp = medium["tr"], medium["G"], medium["cp"]
    rng = np.random.default_rng(11)
    adm = [b for b, (t, s, a, c) in enumerate(tr.blocks) if a]
    G2 = G.copy()
    for b, j in zip(rng.choice(adm, 6, replace=False), (3, -5, 7, 1, -2, 9)):
        t, s, _, _ = tr.blocks[b]
        G2[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]] *= 2.0 ** j
    for side, ref in (("row", medium["V"]), ("col", medium["W"])):
        B = O.compress(tr, G2, cp, side)
        assert B.rank == ref.rank
        for key, Q in ref.Q.items():
            assert np.array_equal(B.Q[key], Q)
        for key, E in ref.E.items():
            assert np.array_equal(B.E[key], E)


# ---------------------------------------------------------------- storage of the transfer matrices

def test_transfer_matrix_shapes_and_storage(medium):
    """Def. of the directional cluster basis: E_{t'c} maps the rank k_tc of the father
    to the rank k_{t'c'} of the son t' at c' = sd(c); storage counts those entries."""
    tr, V, W, S = medium["tr"], medium["V"], medium["W"], medium["S"]
    for B, key in ((V, "E_V"), (W, "E_W")):
        total = 0
        for t in range(tr.nclusters()):
            if not tr.sons[t]:
                continue
            for c in B.F[t]:
                cs = int(tr.sd[tr.level[t]][c])
                for son in tr.sons[t]:
                    assert B.E[(son, c)].shape == (B.rank[(son, cs)], B.rank[(t, c)])
                    total += B.rank[(son, cs)] * B.rank[(t, c)]
        assert O.storage(tr, V, W, S)[key] == total
        assert total > 0
