"""Host-side parity of the library's tree builder with the oracle (no GPU).

The cluster tree, the direction families, the son maps, the block tree, the
block directions and the column sets F_tc are integer results decided by
floating-point comparisons evaluated in the same order on both sides, so they
must agree exactly.
"""
import math
import os
import re

import numpy as np
import pytest

from oracle import dh2_oracle as O
from synth import fibonacci_sphere, random_cube_surface, random_ellipsoid, random_sphere

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    from paper_1510_07087_gb300 import _binding
    if not os.path.exists(_binding.LIB_PATH):
        pytest.skip("libdh2.so not built")
    return _binding


def test_library_exports_every_declared_symbol():
    b = _lib_or_skip()
    header = open(os.path.join(ROOT, "include", "dh2.h")).read()
    declared = set(re.findall(r"^\s*(?:dh2_status|void|const char\*)\s+(dh2_\w+)\s*\(", header, re.M))
    assert declared, "no declarations parsed"
    lib = b._lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(b.exported_symbols())
    assert b.dh2_version().startswith("dh2")


CASES = [
    ("fib", 2048, 4.0, 32, 2 * math.sqrt(2), 1.0, 0),
    ("fib", 4096, 12.0, 16, 2 * math.sqrt(2), 1.0, 0),
    ("fib", 2048, 8.0, 16, 20.0, 5.0, 0),
    ("sphere", 1500, 6.0, 24, 2 * math.sqrt(2), 1.0, 0),
    ("ellipsoid", 1200, 10.0, 20, 2 * math.sqrt(2), 2.0, 0),
    ("cube", 1800, 9.0, 32, 2 * math.sqrt(2), 1.0, 0),
    ("fib", 1024, 0.0, 16, 2 * math.sqrt(2), 1.0, 1),
    ("fib", 20, 4.0, 32, 2 * math.sqrt(2), 1.0, 0),
]


def _points(kind, n):
    return {"fib": fibonacci_sphere, "sphere": random_sphere, "ellipsoid": random_ellipsoid,
            "cube": random_cube_surface}[kind](n)


@pytest.mark.parametrize("kind,n,kappa,leaf,eta1,eta2,rule", CASES)
def test_tree_matches_oracle(kind, n, kappa, leaf, eta1, eta2, rule):
    b = _lib_or_skip()
    pts = _points(kind, n)
    T = b.dh2_tree_build(pts, leaf, kappa, eta1, eta2, rule)
    ot = O.build_tree(pts, O.TreeParams(leaf_size=leaf, kappa=kappa, eta1=eta1, eta2=eta2, dir_rule=rule))
    assert np.array_equal(T.perm(), ot.perm)
    cl = T.clusters()
    assert np.array_equal(cl["start"], ot.start)
    assert np.array_equal(cl["size"], ot.size)
    assert np.array_equal(cl["level"], ot.level)
    assert np.array_equal(cl["parent"], ot.parent)
    assert np.array_equal(cl["lo"], np.array(ot.lo)) and np.array_equal(cl["hi"], np.array(ot.hi))
    st = T.stats()
    assert st.depth == ot.depth
    for l in range(ot.depth + 1):
        D, sd = T.directions(l)
        assert np.array_equal(D, ot.dirs[l])
        if l < ot.depth:
            assert np.array_equal(sd, ot.sd[l])
    blk = T.blocks()
    ob = np.array([(t, s, int(a), c) for (t, s, a, c) in ot.blocks], dtype=np.int64)
    assert np.array_equal(blk, ob)
    # used pairs and F_tc (as sets of blocks) on both sides
    for side, name in ((0, "row"), (1, "col")):
        F = O.column_sets(ot, name)
        pr = T.pairs(side)
        off, ids = T.pair_blocks(side)
        got = {}
        for p in range(len(pr["cluster"])):
            got[(int(pr["cluster"][p]), int(pr["dir"][p]))] = sorted(ids[off[p]:off[p + 1]].tolist())
            width = 0
            for bb in ids[off[p]:off[p + 1]]:
                t, s, _, _ = ot.blocks[bb]
                width += ot.size[s] if side == 0 else ot.size[t]
            assert width == pr["ncols"][p]
            assert bool(pr["leaf"][p]) == ot.is_leaf(int(pr["cluster"][p]))
        want = {(t, c): sorted(bl) for t in F for c, bl in F[t].items()}
        assert got == want


def test_invalid_arguments_rejected():
    b = _lib_or_skip()
    pts = fibonacci_sphere(100)
    with pytest.raises(b.DH2Error):
        b.dh2_tree_build(pts, 0, 4.0)
    with pytest.raises(b.DH2Error):
        b.dh2_tree_build(pts, 16, -1.0)
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(b.DH2Error):
        b.dh2_tree_build(bad, 16, 4.0)


def test_tuning_table_set_get_and_validation():
    """dh2_tuning_set installs a table that dh2_tuning_get returns; a value outside a knob's set
    (a Jacobi width that is not a power of two up to 32, a narrow choice outside 0..2, more than 4
    R CTAs per SM, an R kernel choice other than 0/1, a segment width that is not 0 or a multiple of
    64 in 256..8192) is refused with DH2_EINVAL and leaves the
    table as it was; dh2_autotune checks its arguments before any device work."""
    b = _lib_or_skip()
    saved = b.tuning()
    try:
        t = {"jacobi_tpp": [32, 16, 8, 4, 32], "jacobi_narrow": [1, 0, 1, 0], "rq_ctas_per_sm": 2,
             "rq_tensor": 0, "level_seg_cols": 512}
        b.set_tuning(t)
        assert b.tuning() == t
        for bad in ({"jacobi_tpp": [32, 12, 8, 4, 32]}, {"jacobi_tpp": [64, 16, 8, 4, 32]},
                    {"jacobi_narrow": [3, 0, 0, 0]}, {"rq_ctas_per_sm": 5}, {"rq_ctas_per_sm": -1},
                    {"rq_tensor": 2}, {"level_seg_cols": 100}, {"level_seg_cols": 1000},
                    {"level_seg_cols": 16384}):
            with pytest.raises(b.DH2Error) as ei:
                b.set_tuning({**t, **bad})
            assert ei.value.status == 1
            assert b.tuning() == t
        lib = b._lib()
        T = b.dh2_tree_build(fibonacci_sphere(64), 16, 4.0)
        p = b.CompressParams(1e-4, 2.0 / 3.0, 0, b.MODE_FP32, 0, 0)
        out = b.Tuning()
        nrec = b.c_int32(7)
        for reps in (0, 16):  # outside 1..15
            assert lib.dh2_autotune(T.handle, b.c_void_p(1), b.DH2_C64, 64, b.byref(p), None, reps, b.byref(out),
                                    None, 0, b.byref(nrec)) == 1
            assert nrec.value == 0
        assert lib.dh2_autotune(T.handle, None, b.DH2_C64, 64, b.byref(p), None, 3, b.byref(out), None, 0,
                                None) == 1
        assert b.tuning() == t
    finally:
        b.set_tuning(saved)


def test_host_input_arguments_rejected_before_any_device_work():
    """dh2_compress_host checks its arguments on the host first: view mode (the staging buffer
    is reused), ld < n, an unknown dtype and null pointers return DH2_EINVAL with no handle."""
    b = _lib_or_skip()
    n = 64
    T = b.dh2_tree_build(fibonacci_sphere(n), 16, 4.0)
    host = np.zeros(2 * n * n, dtype=np.float32)
    lib = b._lib()

    def call(G, dtype, ld, nearfield, params=True):
        p = b.CompressParams(1e-4, 2.0 / 3.0, 0, b.MODE_FP32, nearfield, 0)
        h = b.c_void_p(12345)
        st = lib.dh2_compress_host(T.handle, G, dtype, ld, b.byref(p) if params else None, None, b.byref(h))
        return st, h.value

    ptr = b._ptr(host)
    assert call(ptr, b.DH2_C64, n, 1) == (1, None)          # view mode
    assert call(ptr, b.DH2_C64, n - 1, 0) == (1, None)      # ld < n
    assert call(ptr, 7, n, 0) == (1, None)                  # unknown dtype
    assert call(None, b.DH2_C64, n, 0) == (1, None)         # no matrix
    assert call(ptr, b.DH2_C64, n, 0, params=False) == (1, None)


@pytest.mark.parametrize("kind,n,kappa,leaf,eta1,eta2,rule", CASES)
def test_host_input_panels(kind, n, kappa, leaf, eta1, eta2, rule):
    """Schedule of dh2_compress_host: panels are unions of whole clusters; every admissible
    block's column cluster lies in one panel; a column-basis leaf pair's blocks (own and
    inherited) lie in the panel of its cluster; a row-basis leaf pair runs after the last panel
    its blocks' columns touch."""
    b = _lib_or_skip()
    T = b.dh2_tree_build(_points(kind, n), leaf, kappa, eta1, eta2, rule)
    col, row_panel = T.panels()
    cl = T.clusters()
    start, size = cl["start"].astype(np.int64), cl["size"].astype(np.int64)
    assert col[0] == 0 and col[-1] == n and np.all(np.diff(col) > 0)
    assert set(col[1:-1].tolist()) <= set(start.tolist())
    panel = lambda j: int(np.searchsorted(col, j, side="right") - 1)  # noqa: E731
    blk = T.blocks()
    s_first = np.array([panel(j) for j in start[blk[:, 1]]])
    s_last = np.array([panel(j) for j in start[blk[:, 1]] + size[blk[:, 1]] - 1])
    adm = blk[:, 2] == 1
    assert np.array_equal(s_first[adm], s_last[adm])
    for side in (0, 1):
        pr = T.pairs(side)
        off, ids = T.pair_blocks(side)
        for p in range(len(pr["cluster"])):
            bl = ids[off[p]:off[p + 1]]
            if side == 1:
                if pr["leaf"][p] and len(bl):
                    assert set(s_first[bl].tolist()) == {panel(start[pr["cluster"][p]])}
            elif pr["leaf"][p]:
                assert row_panel[p] == (int(s_last[bl].max()) if len(bl) else 0)
            else:
                assert row_panel[p] == -1


def test_build_reads_every_tuning_macro():
    """Every integer macro with a default behind an #ifndef in the CUDA and C++ sources is one the
    build reads from the environment, and the build reads no other: a tuning choice cannot be set
    by a name that the sources ignore, nor exist without a way to set it."""
    from paper_1510_07087_gb300 import build as B
    found = set()
    for f in sorted(os.listdir(B.CSRC)):
        if f.endswith((".cu", ".cuh", ".cpp", ".h")):
            src = open(os.path.join(B.CSRC, f)).read()
            found |= set(re.findall(r"^#ifndef (DH2_\w+)\s*\n#define \1 -?\d+\b", src, re.M))
    assert found, "no tuning macros parsed"
    assert found == set(B.TUNING_MACROS)
