"""Plain FP64 CPU oracle of directional H^2-matrix compression.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference arm may import or run this module.  It is slow on
purpose and shares no code with the CUDA library: the cluster tree, the
direction sets, the block tree, the column sets F_tc, the weights, the
compression recursion, the projection, the matrix-vector product and the error
are all restated here, step by step, from the paper (S. Boerm, "Directional
H^2-matrix compression for high-frequency problems", 2015).  All arithmetic is
complex128 / float64; numpy.linalg.svd is used as a library primitive for the
singular value decompositions the algorithm asks for.

Readings of the paper taken where it is silent or ambiguous (each also listed
in the design notes of the repository):
  * cluster tree: bisection of the tight bounding box at the midpoint of its
    longest side (lowest axis index on ties), coordinates <= midpoint go to the
    first son, stable order; a cluster with at most `leaf_size` indices is a
    leaf (Def. 1, "geometrically regular subdivision" of Section 7);
  * directions: midpoints of an m x m subdivision of each face of [-1,1]^3,
    projected to the sphere, with m = max(1, ceil(sqrt2 * kappa * delta_l /
    eta1)) so that each square has diameter <= 2 eta1/(kappa delta_l)
    (Section 3); faces in the order +x,-x,+y,-y,+z,-z, squares row-major;
    `dir_rule=1` replaces D_l by {0} when kappa * delta_l <= eta1 (Def. 3
    allows the zero direction);
  * son maps sd_l(c) = nearest direction of level l+1 (Def. 3), block
    direction c_b = nearest direction to (m_t - m_s)/|m_t - m_s| (Eq.
    adm_directional); lowest index on ties;
  * block tree: standard recursion with Eqs. (adm_parabolic) and
    (adm_standard) using one eta2; a block with t or s a leaf that is not
    admissible is an inadmissible leaf (Section 3);
  * weights (Remark "Error control"): omega_b = |G_b|_F * zeta^(-level(t)),
    tolerances eps_r = eps_hat * zeta^level(r); with at most 2^j descendants at
    relative depth j the Error-estimate theorem then gives
    |G_b - Q Q^* G_b|_F <= eps_hat |G_b|_F / sqrt(1 - 2 zeta^2);
    err_mode 0 takes eps_hat = eps * sqrt(1 - 2 zeta^2) / sqrt(2) so that the
    row and column errors together give |G - G~|_F <= eps |G|_F; err_mode 1
    takes eps_hat = eps;
  * truncation: k = min{k : sum_{i>k} sigma_i^2 <= eps_level(t)^2} (Frobenius
    norm throughout, which makes Eq. error_nonleaf an equality);
  * ranks are adaptive, so Ghat_tc has k_{t1c'} + k_{t2c'} rows (the paper
    writes 2k for a fixed rank).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "TreeParams", "CompressParams", "OracleTree", "build_tree", "block_norms",
    "compress", "expand_basis", "project", "matvec", "dense_approximation",
    "error_fro", "storage", "eps_hat",
]


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------

@dataclass
class TreeParams:
    leaf_size: int = 32
    kappa: float = 4.0
    eta1: float = 2.0 * math.sqrt(2.0)
    eta2: float = 1.0
    dir_rule: int = 0          # 0: cube directions, 1: {0} when kappa*delta <= eta1


@dataclass
class CompressParams:
    eps: float = 1e-4
    zeta: float = 2.0 / 3.0
    err_mode: int = 0          # 0: global Frobenius guarantee, 1: eps_hat = eps


def eps_hat(p: CompressParams) -> float:
    """Base tolerance eps_hat of eps_r = eps_hat * zeta^level(r) (Remark "Error control")."""
    if p.err_mode == 0:
        q = 1.0 - 2.0 * p.zeta * p.zeta
        if q <= 0.0:
            raise ValueError("err_mode 0 needs zeta < 1/sqrt(2)")
        return p.eps * math.sqrt(q) / math.sqrt(2.0)
    return p.eps


# --------------------------------------------------------------------------
# cluster tree, directions, block tree (Def. 1, Def. 2, Def. 3, Section 3)
# --------------------------------------------------------------------------

@dataclass
class OracleTree:
    n: int
    params: TreeParams
    perm: np.ndarray                 # perm[i] = original index of permuted index i
    start: list = field(default_factory=list)
    size: list = field(default_factory=list)
    level: list = field(default_factory=list)
    parent: list = field(default_factory=list)
    sons: list = field(default_factory=list)
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    center: list = field(default_factory=list)
    diam: list = field(default_factory=list)
    depth: int = 0
    delta: list = field(default_factory=list)     # delta_l = max diam on level l
    dirs: list = field(default_factory=list)      # D_l as (|D_l|, 3) arrays
    sd: list = field(default_factory=list)        # sd_l as int arrays into D_{l+1}
    blocks: list = field(default_factory=list)    # (t, s, admissible, c_b or -1)

    def is_leaf(self, t: int) -> bool:
        return len(self.sons[t]) == 0

    def nclusters(self) -> int:
        return len(self.start)


def _box_dist(lo_t, hi_t, lo_s, hi_s) -> float:
    """Euclidean distance of two axis-parallel boxes (0 if they intersect)."""
    acc = 0.0
    for a in range(3):
        g = max(0.0, max(lo_s[a] - hi_t[a], lo_t[a] - hi_s[a]))
        acc = acc + g * g
    return math.sqrt(acc)


def cube_directions(m: int) -> np.ndarray:
    """Section 3: midpoints of m x m squares on each face of [-1,1]^3, normalised."""
    out = []
    for face in range(6):
        ax = face // 2
        sgn = 1.0 if face % 2 == 0 else -1.0
        others = [d for d in range(3) if d != ax]
        for a in range(m):
            u = -1.0 + (2.0 * a + 1.0) / m
            for b in range(m):
                v = -1.0 + (2.0 * b + 1.0) / m
                p = [0.0, 0.0, 0.0]
                p[ax] = sgn
                p[others[0]] = u
                p[others[1]] = v
                nrm = math.sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])
                out.append((p[0] / nrm, p[1] / nrm, p[2] / nrm))
    return np.array(out, dtype=np.float64)


def level_directions(kappa: float, delta: float, eta1: float, dir_rule: int) -> np.ndarray:
    """D_l for a level with maximal diameter delta (Section 3 / Def. 3)."""
    if dir_rule == 1 and kappa * delta <= eta1:
        return np.zeros((1, 3), dtype=np.float64)
    x = math.sqrt(2.0) * kappa * delta / eta1
    m = max(1, int(math.ceil(x)))
    return cube_directions(m)


def _nearest(U: np.ndarray, D: np.ndarray) -> np.ndarray:
    """argmin_j |U_i - D_j|^2 with the lowest j on ties, exact elementwise IEEE arithmetic."""
    out = np.empty(U.shape[0], dtype=np.int64)
    step = max(1, 4_000_000 // max(1, D.shape[0]))
    for s in range(0, U.shape[0], step):
        u = U[s:s + step]
        d0 = u[:, None, 0] - D[None, :, 0]
        d1 = u[:, None, 1] - D[None, :, 1]
        d2 = u[:, None, 2] - D[None, :, 2]
        dd = d0 * d0 + d1 * d1 + d2 * d2
        out[s:s + step] = np.argmin(dd, axis=1)
    return out


def build_tree(points: np.ndarray, params: TreeParams) -> OracleTree:
    pts = np.asarray(points, dtype=np.float64)
    n = pts.shape[0]
    tr = OracleTree(n=n, params=params, perm=np.zeros(n, dtype=np.int64))
    offset = [0]

    # Def. 1: sons partition the father; bisection of the bounding box.
    def make(idx: np.ndarray, lvl: int, parent: int) -> int:
        cid = len(tr.start)
        P = pts[idx]
        lo = [float(v) for v in P.min(axis=0)]
        hi = [float(v) for v in P.max(axis=0)]
        tr.start.append(offset[0])
        tr.size.append(len(idx))
        tr.level.append(lvl)
        tr.parent.append(parent)
        tr.sons.append([])
        tr.lo.append(lo)
        tr.hi.append(hi)
        tr.center.append([(lo[a] + hi[a]) * 0.5 for a in range(3)])
        dx, dy, dz = hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]
        tr.diam.append(math.sqrt(dx * dx + dy * dy + dz * dz))
        split = False
        if len(idx) > params.leaf_size:
            ext = [hi[a] - lo[a] for a in range(3)]
            ax = 0
            for a in (1, 2):
                if ext[a] > ext[ax]:
                    ax = a
            mid = (lo[ax] + hi[ax]) * 0.5
            first = idx[P[:, ax] <= mid]
            second = idx[P[:, ax] > mid]
            if len(first) > 0 and len(second) > 0:
                split = True
        if split:
            s1 = make(first, lvl + 1, cid)
            s2 = make(second, lvl + 1, cid)
            tr.sons[cid] = [s1, s2]
        else:
            tr.perm[offset[0]:offset[0] + len(idx)] = idx
            offset[0] += len(idx)
        return cid

    make(np.arange(n, dtype=np.int64), 0, -1)
    tr.depth = max(tr.level)

    # delta_l and the direction families of Section 3.
    tr.delta = [0.0] * (tr.depth + 1)
    for t in range(tr.nclusters()):
        lv = tr.level[t]
        if tr.diam[t] > tr.delta[lv]:
            tr.delta[lv] = tr.diam[t]
    tr.dirs = [level_directions(params.kappa, tr.delta[l], params.eta1, params.dir_rule)
               for l in range(tr.depth + 1)]
    tr.sd = [_nearest(tr.dirs[l], tr.dirs[l + 1]) for l in range(tr.depth)]

    # Def. 2 block tree by the standard recursion with (adm_parabolic) and
    # (adm_standard); admissible leaves get their block direction.
    raw = []

    def recurse(t: int, s: int) -> None:
        md = max(tr.diam[t], tr.diam[s])
        d = _box_dist(tr.lo[t], tr.hi[t], tr.lo[s], tr.hi[s])
        adm = d > 0.0 and md <= params.eta2 * d and params.kappa * (md * md) <= params.eta2 * d
        if adm:
            raw.append((t, s, True))
        elif tr.is_leaf(t) or tr.is_leaf(s):
            raw.append((t, s, False))
        else:
            for t2 in tr.sons[t]:
                for s2 in tr.sons[s]:
                    recurse(t2, s2)

    recurse(0, 0)

    # block directions, one vectorised argmin per level
    cb = [-1] * len(raw)
    by_level: dict = {}
    for i, (t, s, adm) in enumerate(raw):
        if adm:
            by_level.setdefault(tr.level[t], []).append(i)
    for lv, ids in by_level.items():
        U = np.empty((len(ids), 3))
        for j, i in enumerate(ids):
            t, s, _ = raw[i]
            dv = [tr.center[t][a] - tr.center[s][a] for a in range(3)]
            nd = math.sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2])
            U[j] = [dv[0] / nd, dv[1] / nd, dv[2] / nd]
        near = _nearest(U, tr.dirs[lv])
        for j, i in enumerate(ids):
            cb[i] = int(near[j])
    tr.blocks = [(t, s, adm, cb[i]) for i, (t, s, adm) in enumerate(raw)]
    return tr


# --------------------------------------------------------------------------
# F_tc, used directions, weights (Section 6 definitions, Remark "Error control")
# --------------------------------------------------------------------------

def _side_blocks(tr: OracleTree, side: str):
    """Admissible blocks as (block id, r, q, c_b) with r the cluster whose basis is built.

    Row basis: r = t (blocks of G).  Column basis: the same procedure on G^*
    (Section 6, after the spectral-norm split), so r = s and the block of G^*
    is (s, t) with the same block direction (Def. "Directional H^2-matrix").
    """
    out = []
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        if adm:
            out.append((b, t, s, c) if side == "row" else (b, s, t, c))
    return out


def column_sets(tr: OracleTree, side: str) -> dict:
    """F_tc by its definition: blocks (t+, s) with t in desc(t+) and c in dscd_{t+}(c_b).

    Returns {t: {c: [block ids]}}; the list order is the column order of
    G_tc used by this oracle (nearest ancestor first, then the block order).
    """
    rows: dict = {}
    for b, r, q, c in _side_blocks(tr, side):
        rows.setdefault(r, []).append((b, c))
    F: dict = {t: {} for t in range(tr.nclusters())}
    for t in range(tr.nclusters()):
        anc = t
        while anc >= 0:
            lst = rows.get(anc, [])
            if lst:
                cs = np.array([c for _, c in lst], dtype=np.int64)
                for lv in range(tr.level[anc], tr.level[t]):
                    cs = tr.sd[lv][cs]
                for (b, _), c in zip(lst, cs):
                    F[t].setdefault(int(c), []).append(b)
            anc = tr.parent[anc]
    return F


def block_norms(tr: OracleTree, G: np.ndarray) -> np.ndarray:
    """|G|_{t x s}|_F for every block (0 for inadmissible ones, unused)."""
    out = np.zeros(len(tr.blocks))
    for b, (t, s, adm, _) in enumerate(tr.blocks):
        if adm:
            blk = G[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]]
            out[b] = math.sqrt(float(np.sum(blk.real ** 2 + blk.imag ** 2)))
    return out


def block_weights(tr: OracleTree, norms: np.ndarray, zeta: float) -> np.ndarray:
    """omega_b = |G_b|_F * zeta^(-level(t)) (1 for a zero block)."""
    w = np.ones(len(tr.blocks))
    for b, (t, s, adm, _) in enumerate(tr.blocks):
        if adm and norms[b] > 0.0:
            w[b] = norms[b] * zeta ** (-tr.level[t])
    return w


# --------------------------------------------------------------------------
# compression: procedure basis() of Section 6 (figure "Construction of an
# orthogonal directional cluster basis")
# --------------------------------------------------------------------------

@dataclass
class Basis:
    side: str
    F: dict                      # {t: {c: [block ids]}}
    rank: dict                   # (t, c) -> k
    Q: dict                      # leaf (t, c) -> (m_t, k) orthonormal
    E: dict                      # (t', c) -> transfer matrix E_{t'c} (k_{t'c'} x k_{tc}), t' a son
    sigma: dict                  # (t, c) -> singular values of the matrix truncated at (t, c)
    eps_level: list


def _truncation_rank(sig: np.ndarray, eps_l: float) -> int:
    """k = min{k : sum_{i>k} sigma_i^2 <= eps_l^2}, tail summed from the smallest value."""
    s2 = sig.astype(np.float64) ** 2
    tail = 0.0
    k = len(s2)
    for i in range(len(s2) - 1, -1, -1):
        if tail + s2[i] <= eps_l * eps_l:
            tail += s2[i]
            k = i
        else:
            break
    return k


def _block_matrix(tr: OracleTree, G: np.ndarray, side: str, b: int, r: int) -> np.ndarray:
    """Rows of r-hat (r a descendant of the block's basis cluster) times the block's other index set."""
    t, s, _, _ = tr.blocks[b]
    rr = slice(tr.start[r], tr.start[r] + tr.size[r])
    if side == "row":
        return G[rr, tr.start[s]:tr.start[s] + tr.size[s]]
    return G[tr.start[t]:tr.start[t] + tr.size[t], rr].conj().T


def compress(tr: OracleTree, G: np.ndarray, cp: CompressParams, side: str = "row",
             weights: np.ndarray | None = None, rank_override: dict | None = None,
             keep_R: bool = False) -> Basis:
    """Build the orthogonal directional cluster basis of one side.

    side="row" approximates G; side="col" applies the same procedure to G^*
    (Section 6).  `rank_override` maps (t, c) to a rank used instead of the
    truncation rule (used to compare against another implementation's ranks).
    """
    if weights is None:
        weights = block_weights(tr, block_norms(tr, G), cp.zeta)
    eh = eps_hat(cp)
    eps_level = [eh * cp.zeta ** l for l in range(tr.depth + 1)]
    F = column_sets(tr, side)
    out = Basis(side=side, F=F, rank={}, Q={}, E={}, sigma={}, eps_level=eps_level)
    R: dict = {}        # (t, c) -> (matrix, {block id: column slice})
    kept: dict = {}

    def colmap(blocks, widths):
        m, off = {}, 0
        for b, w in zip(blocks, widths):
            m[b] = slice(off, off + w)
            off += w
        return m

    def width(b):
        t, s, _, _ = tr.blocks[b]
        return tr.size[s] if side == "row" else tr.size[t]

    def truncate(A, t, c):
        U, sig, _ = np.linalg.svd(A, full_matrices=False)
        out.sigma[(t, c)] = sig
        if rank_override is not None and (t, c) in rank_override:
            k = int(rank_override[(t, c)])
        else:
            k = _truncation_rank(sig, eps_level[tr.level[t]])
        out.rank[(t, c)] = k
        return U[:, :k]

    def basis(t: int) -> None:
        if tr.is_leaf(t):
            for c, blocks in F[t].items():
                # G^omega_tc: the blocks of F_tc restricted to the rows of t, scaled by 1/omega_b
                A = np.concatenate([_block_matrix(tr, G, side, b, t) / weights[b] for b in blocks], axis=1)
                Qtc = truncate(A, t, c)
                out.Q[(t, c)] = Qtc
                R[(t, c)] = (Qtc.conj().T @ A, colmap(blocks, [width(b) for b in blocks]))
        else:
            for son in tr.sons[t]:
                basis(son)
            lv = tr.level[t]
            for c, blocks in F[t].items():
                cs = int(tr.sd[lv][c])
                parts, ks = [], []
                for son in tr.sons[t]:
                    Rs, cm = R[(son, cs)]
                    # R_{t'c'} restricted to the columns of F_tc (copy, no arithmetic)
                    parts.append(np.concatenate([Rs[:, cm[b]] for b in blocks], axis=1))
                    ks.append(Rs.shape[0])
                Ghat = np.concatenate(parts, axis=0)
                Qhat = truncate(Ghat, t, c)
                off = 0
                for son, kk in zip(tr.sons[t], ks):
                    out.E[(son, c)] = Qhat[off:off + kk, :]
                    off += kk
                R[(t, c)] = (Qhat.conj().T @ Ghat, colmap(blocks, [width(b) for b in blocks]))
            if not keep_R:
                for son in tr.sons[t]:
                    for c in F[son]:
                        R.pop((son, c), None)

    basis(0)
    if keep_R:
        out.R = R
    return out


def leaf_pair_basis(A: np.ndarray, eps_l: float):
    """Leaf step for one explicit matrix A = G^omega_tc (Section 6): the
    singular values, the rank by the truncation rule and Q = leading left
    singular vectors.  Used to check sampled pairs of large problems."""
    U, sig, _ = np.linalg.svd(A, full_matrices=False)
    k = _truncation_rank(sig, eps_l)
    return U[:, :k], sig, k


def expand_basis(tr: OracleTree, B: Basis, t: int, c: int, cache: dict | None = None) -> np.ndarray:
    """Explicit Q_tc from leaf matrices and transfer matrices by Eq. (nested)."""
    if cache is not None and (t, c) in cache:
        return cache[(t, c)]
    if tr.is_leaf(t):
        V = B.Q[(t, c)]
    else:
        cs = int(tr.sd[tr.level[t]][c])
        V = np.concatenate([expand_basis(tr, B, son, cs, cache) @ B.E[(son, c)] for son in tr.sons[t]], axis=0)
    if cache is not None:
        cache[(t, c)] = V
    return V


def project(tr: OracleTree, G: np.ndarray, V: Basis, W: Basis) -> dict:
    """S_b = V_tc^* G|_{t x s} W_sc with c = c_b, from the unweighted G (Section 6, Def. Orthogonality)."""
    S = {}
    cv, cw = {}, {}
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        if not adm:
            continue
        Vt = expand_basis(tr, V, t, c, cv)
        Ws = expand_basis(tr, W, s, c, cw)
        Gb = G[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]]
        S[b] = Vt.conj().T @ Gb @ Ws
    return S


# --------------------------------------------------------------------------
# use and verification (Section 4 matrix-vector product, errors, storage)
# --------------------------------------------------------------------------

def matvec(tr: OracleTree, G: np.ndarray, V: Basis, W: Basis, S: dict, x: np.ndarray) -> np.ndarray:
    """y = G~ x by forward transformation, coupling, backward transformation
    (Section 4, Eqs. mvm1-mvm3 and the recursions of the figure "Fast forward
    and backward transformation") plus the nearfield blocks."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.zeros_like(x)
    xh: dict = {}

    def forward(s: int) -> None:
        if tr.is_leaf(s):
            for c in W.F[s]:
                xh[(s, c)] = W.Q[(s, c)].conj().T @ x[tr.start[s]:tr.start[s] + tr.size[s]]
        else:
            for son in tr.sons[s]:
                forward(son)
            cs_map = tr.sd[tr.level[s]]
            for c in W.F[s]:
                acc = np.zeros((W.rank[(s, c)],) + x.shape[1:], dtype=np.complex128)
                for son in tr.sons[s]:
                    acc = acc + W.E[(son, c)].conj().T @ xh[(son, int(cs_map[c]))]
                xh[(s, c)] = acc

    forward(0)
    yh: dict = {(t, c): np.zeros((V.rank[(t, c)],) + x.shape[1:], dtype=np.complex128)
                for t in range(tr.nclusters()) for c in V.F[t]}
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        if adm:
            yh[(t, c)] = yh[(t, c)] + S[b] @ xh[(s, c)]
        else:
            y[tr.start[t]:tr.start[t] + tr.size[t]] += (
                G[tr.start[t]:tr.start[t] + tr.size[t], tr.start[s]:tr.start[s] + tr.size[s]]
                @ x[tr.start[s]:tr.start[s] + tr.size[s]])

    def backward(t: int) -> None:
        if tr.is_leaf(t):
            for c in V.F[t]:
                y[tr.start[t]:tr.start[t] + tr.size[t]] += V.Q[(t, c)] @ yh[(t, c)]
        else:
            cs_map = tr.sd[tr.level[t]]
            for c in V.F[t]:
                for son in tr.sons[t]:
                    key = (son, int(cs_map[c]))
                    yh[key] = yh[key] + V.E[(son, c)] @ yh[(t, c)]
            for son in tr.sons[t]:
                backward(son)

    backward(0)
    return y


def dense_approximation(tr: OracleTree, G: np.ndarray, V: Basis, W: Basis, S: dict) -> np.ndarray:
    """Assemble G~ explicitly: V_tc S_b W_sc^* on admissible leaves, G_b on the others."""
    Gt = np.zeros_like(G, dtype=np.complex128)
    cv, cw = {}, {}
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        rr = slice(tr.start[t], tr.start[t] + tr.size[t])
        cc = slice(tr.start[s], tr.start[s] + tr.size[s])
        if adm:
            Gt[rr, cc] = expand_basis(tr, V, t, c, cv) @ S[b] @ expand_basis(tr, W, s, c, cw).conj().T
        else:
            Gt[rr, cc] = G[rr, cc]
    return Gt


def error_fro(tr: OracleTree, G: np.ndarray, V: Basis, W: Basis, S: dict) -> float:
    """|G - G~|_F / |G|_F, block by block."""
    num = 0.0
    cv, cw = {}, {}
    for b, (t, s, adm, c) in enumerate(tr.blocks):
        if not adm:
            continue
        rr = slice(tr.start[t], tr.start[t] + tr.size[t])
        cc = slice(tr.start[s], tr.start[s] + tr.size[s])
        D = G[rr, cc] - expand_basis(tr, V, t, c, cv) @ S[b] @ expand_basis(tr, W, s, c, cw).conj().T
        num += float(np.sum(D.real ** 2 + D.imag ** 2))
    den = float(np.sum(G.real ** 2 + G.imag ** 2))
    return math.sqrt(num / den) if den > 0 else 0.0


def storage(tr: OracleTree, V: Basis, W: Basis, S: dict) -> dict:
    """Entries stored by the representation (Def. "DH^2-matrix representation")."""
    out = {"V": 0, "W": 0, "E_V": 0, "E_W": 0, "S": 0, "near": 0}
    for key, Q in V.Q.items():
        out["V"] += Q.size
    for key, Q in W.Q.items():
        out["W"] += Q.size
    for key, E in V.E.items():
        out["E_V"] += E.size
    for key, E in W.E.items():
        out["E_W"] += E.size
    for b, Sb in S.items():
        out["S"] += Sb.size
    for (t, s, adm, c) in tr.blocks:
        if not adm:
            out["near"] += tr.size[t] * tr.size[s]
    out["total"] = sum(out.values())
    return out


def run(points: np.ndarray, G: np.ndarray, tp: TreeParams, cp: CompressParams,
        rank_override_row: dict | None = None, rank_override_col: dict | None = None):
    """Convenience: tree, both bases and the coupling matrices.

    `G` is given in the original index order; the returned tuple holds the
    matrix permuted to the tree's order as its last element.
    """
    tr = build_tree(points, tp)
    G = np.asarray(G)[np.ix_(tr.perm, tr.perm)]
    w = block_weights(tr, block_norms(tr, G), cp.zeta)
    V = compress(tr, G, cp, "row", w, rank_override_row)
    W = compress(tr, G, cp, "col", w, rank_override_col)
    S = project(tr, G, V, W)
    return tr, V, W, S, G
