"""Every row class of the factor and R kernels against the FP64 oracle.

The library launches the leaf factorisations and the leaf R = Q^* A by the
leaf's row count (<= 32, <= 40, <= 48, <= 64 rows; each class has its own CTA
size) and the non-leaf factorisations by k_t1c' + k_t2c' (<= 32, <= 48,
<= 64, more).  At leaf size 64 the headline workload runs mostly in the 33-64
row classes, so each case below asserts from the tree that pairs of every
class exist and, from the library's per-class launch counts, that each class
was launched, before the parity criteria of gpu_cases.py apply.

Inputs: uniform random points on the 2:1:1 ellipsoid (ragged leaves of 24 to
64 points) with the parameter set P-lit (eta1 = 2 sqrt 2,
eta2 = 1), and the Fibonacci sphere with the paper's eta1 = 20, eta2 = 5
(Section 7), whose admissible blocks on coarse levels give non-leaf pairs of
many ranks; eps = 1e-8 there gives non-leaf factors of more than 64 rows.
"""
import math

import pytest

from gpu_cases import Case, check_fp64, check_reduced, dev
from synth import fibonacci_sphere, random_ellipsoid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P_LIT = dict(eta1=2 * math.sqrt(2), eta2=1.0)
P_PAPER = dict(eta1=20.0, eta2=5.0)


def _launched(c: Case, leaf=(), level=()):
    D = c.D
    L = c.launches
    print("launches by class:", {"leaf factor": L[D.KC_LEAF_FACTOR:D.KC_LEAF_FACTOR + 5].tolist(),
                                 "leaf R": L[D.KC_LEAF_R:D.KC_LEAF_R + 5].tolist(),
                                 "level factor": L[D.KC_LEVEL_FACTOR:D.KC_LEVEL_FACTOR + 4].tolist(),
                                 "level R": int(L[D.KC_LEVEL_R])})
    for k in leaf:
        assert k in c.leaf_classes(), f"the tree has no leaf pair of row class {k}"
        assert L[D.KC_LEAF_FACTOR + k] >= 1, f"leaf factor class {k} not launched"
        assert L[D.KC_LEAF_R + k] >= 1, f"leaf R class {k} not launched"
    for k in level:
        assert k in c.level_classes(), f"no non-leaf pair of row class {k} at the GPU's ranks"
        assert L[D.KC_LEVEL_FACTOR + k] >= 1, f"non-leaf factor class {k} not launched"


def _ellipsoid(mode, eps=1e-4):
    pts = random_ellipsoid(6144)
    return Case(6144, 12.0, 64, eps, mode, pts=pts, **P_LIT)


def _sphere_paper(mode, eps):
    return Case(4096, 12.0, 64, eps, mode, pts=fibonacci_sphere(4096), **P_PAPER)


def test_fp64_leaf64_all_leaf_classes():
    c = _ellipsoid(dev().MODE_FP64)
    _launched(c, leaf=(0, 1, 2, 3))
    check_fp64(c)


def test_fp64_leaf64_paper_parameters_level_classes():
    c = _sphere_paper(dev().MODE_FP64, 1e-4)
    _launched(c, leaf=(0, 1, 2, 3), level=(0, 1, 2))
    check_fp64(c)


def test_fp64_leaf64_level_factors_above_64_rows():
    c = _sphere_paper(dev().MODE_FP64, 1e-8)
    _launched(c, level=(2, 3))
    check_fp64(c)


def test_fp32_leaf64_all_leaf_classes():
    c = _ellipsoid(dev().MODE_FP32)
    _launched(c, leaf=(0, 1, 2, 3))
    check_reduced(c, max_bad_frac=0.01, max_diff=1)


def test_fp32_leaf64_paper_parameters_level_classes():
    c = _sphere_paper(dev().MODE_FP32, 1e-4)
    _launched(c, leaf=(0, 1, 2, 3), level=(0, 1, 2))
    check_reduced(c, max_bad_frac=0.01, max_diff=1)
