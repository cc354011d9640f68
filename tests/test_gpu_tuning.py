"""The autotuner and its table (dh2_autotune, dh2_tuning_set/get).

  * dh2_autotune times every candidate of each knob (the R grid, then per leaf
    class the narrow Jacobi launch and the Jacobi width), installs the fastest
    value of each and returns the installed table and the timed candidates;
  * the R grid changes no result (bit-identical products);
  * under other Jacobi widths and launch shapes (which change the rounding
    order of the rotation sums only) the FP64 mode still meets the FP64 parity
    criteria against the oracle and the mixed mode its reduced-precision ones.
"""
import numpy as np
import pytest

from gpu_cases import Case, check_fp64, check_reduced, colmajor, dev
from synth import helmholtz_matrix, random_ellipsoid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _restore_table():
    D = dev()
    saved = D.tuning()
    yield
    D.set_tuning(saved)


def _leaf64_problem(n=4096, kappa=12.0):
    D = dev()
    pts = random_ellipsoid(n)
    T = D.dh2_tree_build(pts, 64, kappa)
    G = helmholtz_matrix(pts, kappa)[np.ix_(T.perm(), T.perm())]
    return T, G, colmajor(G, torch.complex64)


def test_autotune_installs_the_fastest_candidates():
    D = dev()
    T, _, Gd = _leaf64_problem()
    table, log = D.autotune(T, Gd, eps=1e-4, mode=D.MODE_MIXED_BF16X3, reps=3)
    assert D.tuning() == table
    assert all(r["ms"] > 0 for r in log)
    ten = [r for r in log if r["knob"] == "rq_tensor"]
    assert [r["value"] for r in ten] == [0, 1]
    assert table["rq_tensor"] == min(ten, key=lambda r: r["ms"])["value"]
    rq = [r for r in log if r["knob"] == "rq_ctas_per_sm"]
    assert [r["value"] for r in rq] == [0, 1, 2]
    assert table["rq_ctas_per_sm"] == min(rq, key=lambda r: r["ms"])["value"]
    classes = sorted({r["cls"] for r in log if r["knob"] == "jacobi_tpp"})
    assert classes, log  # a leaf-64 tree has leaves in several classes
    for c in classes:
        nar = [r for r in log if r["knob"] == "jacobi_narrow" and r["cls"] == c]
        tpp = [r for r in log if r["knob"] == "jacobi_tpp" and r["cls"] == c]
        assert [r["value"] for r in nar] == [0, 1, 2] and [r["value"] for r in tpp] == [32, 16, 8]
        assert table["jacobi_narrow"][c] == min(nar, key=lambda r: r["ms"])["value"]
        assert table["jacobi_tpp"][c] == min(tpp, key=lambda r: r["ms"])["value"]
    print("autotuned table:", table)


def test_r_grid_changes_no_result():
    """The persistent R kernel's CTAs per SM only change which CTA takes a tile: the ranks, the
    stored bases and every coupling matrix S_b (formed from R) are bit-identical."""
    D = dev()
    T, _, Gd = _leaf64_problem(2048, 8.0)
    adm = np.flatnonzero(T.blocks()[:, 2] == 1)
    rng = np.random.default_rng(9)
    sample = rng.choice(adm, min(60, len(adm)), replace=False)
    res = []
    for rq in (0, 1, 2):
        t = D.tuning()
        t["rq_ctas_per_sm"] = rq
        t["rq_tensor"] = 0  # the grid of the FP32-pipe R kernel
        D.set_tuning(t)
        M = D.dh2_compress(T, Gd, eps=1e-4, mode=D.MODE_MIXED_BF16X3)
        res.append(([M.ranks(0), M.ranks(1)], [M.coupling(int(b)) for b in sample],
                    [M.pair_basis(s, p) for s in (0, 1) for p in range(0, len(M.ranks(s)), 97)]))
    for r, S, V in res[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(r, res[0][0]))
        assert all(np.array_equal(a, b) for a, b in zip(S, res[0][1]))
        assert all(np.array_equal(a, b) for a, b in zip(V, res[0][2]))


@pytest.mark.parametrize("tpp,narrow,tensor", [(8, 2, 1), (16, 0, 0)])
def test_other_choices_keep_parity(tpp, narrow, tensor):
    D = dev()
    D.set_tuning({"jacobi_tpp": [tpp] * 5, "jacobi_narrow": [narrow] * 4, "rq_ctas_per_sm": 1,
                  "rq_tensor": tensor})
    check_fp64(Case(2048, 6.0, 64, 1e-4, D.MODE_FP64, pts=random_ellipsoid(2048)))
    c = Case(4096, 12.0, 64, 1e-4, D.MODE_MIXED_BF16X3, pts=random_ellipsoid(4096))
    check_reduced(c, max_bad_frac=0.01, max_diff=1)


def test_tensor_core_r_agrees_with_the_fp32_pipes():
    """The mixed mode's leaf R on the tensor cores (three bf16 slices per operand, six products,
    FP32 accumulation) and on the FP32 pipes agree to FP32 rounding: the leaf ranks (which R does
    not enter) are equal, the level ranks equal outside near-ties, and the coupling matrices agree
    to 1e-4 of their norm."""
    D = dev()
    T, _, Gd = _leaf64_problem()
    adm = np.flatnonzero(T.blocks()[:, 2] == 1)
    sample = np.random.default_rng(4).choice(adm, min(80, len(adm)), replace=False)
    out = []
    for tensor in (0, 1):
        t = D.tuning()
        t["rq_tensor"] = tensor
        D.set_tuning(t)
        M = D.dh2_compress(T, Gd, eps=1e-4, mode=D.MODE_MIXED_BF16X3)
        assert M.class_launches()[D.KC_LEAF_R_TC] == tensor
        out.append((M, [M.ranks(0), M.ranks(1)], [M.coupling(int(b)) for b in sample]))
    (M0, r0, S0), (M1, r1, S1) = out
    for side in (0, 1):
        leaf = T.pairs(side)["leaf"].astype(bool)
        assert np.array_equal(r0[side][leaf], r1[side][leaf])
        assert np.mean(r0[side] != r1[side]) <= 0.005
    checked = 0
    for a, b in zip(S0, S1):
        if a.shape == b.shape and a.size:
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(a)
            checked += 1
    assert checked >= len(sample) // 2


@pytest.mark.parametrize("kind", ["fp64", "mixed"])
def test_wide_level_pairs_by_column_segments(kind):
    """Non-leaf pairs wider than twice level_seg_cols are factored by column segments (each
    segment's LQ factor L_i, then the pair's factor from [L_1 ... L_S]): with segments of 256
    columns the paper's parameters (eta1 = 20, eta2 = 5) split pairs on several levels, and the
    FP64 mode still meets the FP64 parity criteria against the oracle (ranks outside ties,
    products to 1e-11), the mixed mode its reduced-precision ones."""
    D = dev()
    t = D.tuning()
    t["level_seg_cols"] = 0
    D.set_tuning(t)
    mode = D.MODE_FP64 if kind == "fp64" else D.MODE_MIXED_BF16X3
    n, kappa, leaf = (2048, 8.0, 16) if kind == "fp64" else (4096, 12.0, 32)
    c = Case(n, kappa, leaf, 1e-4, mode, eta1=20.0, eta2=5.0, compress=False)
    plain = D.dh2_compress(c.T, c.Gd, eps=1e-4, mode=mode).class_launches()
    t["level_seg_cols"] = 256
    D.set_tuning(t)
    M = D.dh2_compress(c.T, c.Gd, eps=1e-4, mode=mode)
    split = M.class_launches()
    assert split[D.KC_CLASSIFY] > plain[D.KC_CLASSIFY]  # levels with segment launches
    pr = [c.T.pairs(s) for s in (0, 1)]
    assert max(int(p["ncols"][~p["leaf"].astype(bool)].max(initial=0)) for p in pr) > 512
    c.attach(M)
    if kind == "fp64":
        check_fp64(c)
    else:
        check_reduced(c, max_bad_frac=0.01, max_diff=1)
