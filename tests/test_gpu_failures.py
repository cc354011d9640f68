"""Failure paths of the compression, raised on the host or by the kernels'
own status checks (no GPU fault is involved):

  * a Jacobi sweep cap of 1 ends the factorisations with rotations still
    pending: the kernels set the non-convergence bit and the call returns
    DH2_ENOCONV;
  * non-finite entries in G reach the tail sums: the kernels set the
    non-finite bit and the call returns DH2_ENOCONV;
  * a refused device allocation (dh2_debug_fail_alloc) returns DH2_ENOMEM;
in each case the output handle is NULL (nothing is leaked to the caller) and
the next call on the same tree succeeds.
"""
import ctypes

import numpy as np
import pytest

from gpu_cases import colmajor, dev
from synth import fibonacci_sphere, helmholtz_matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DH2_ENOMEM = 2
DH2_ENOCONV = 5


def _setup(n=1024, kappa=6.0, leaf=32, dtype=None):
    D = dev()
    pts = fibonacci_sphere(n)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa)[np.ix_(perm, perm)]
    return D, T, G, colmajor(G, dtype or torch.complex128)


def _raw_compress(D, T, Gd, mode, max_sweeps=0):
    """dh2_compress through ctypes with a sentinel in the output handle."""
    from paper_1510_07087_gb300 import _binding as B

    p = B.CompressParams(1e-4, 2.0 / 3.0, 0, mode, 0, max_sweeps)
    h = ctypes.c_void_p(0xDEAD)
    st = B._lib().dh2_compress(T.handle, ctypes.c_void_p(Gd.data_ptr()), B._dtype_code(Gd), B._colmajor_ld(Gd),
                               ctypes.byref(p), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                               ctypes.byref(h))
    return st, h.value


@pytest.mark.parametrize("mode_name", ["fp64", "fp32"])
def test_sweep_cap_reports_no_convergence(mode_name):
    dt = torch.complex128 if mode_name == "fp64" else torch.complex64
    D, T, G, Gd = _setup(dtype=dt)
    mode = D.MODE_FP64 if mode_name == "fp64" else D.MODE_FP32
    st, h = _raw_compress(D, T, Gd, mode, max_sweeps=1)
    assert st == DH2_ENOCONV and h is None
    M = D.dh2_compress(T, Gd, mode=mode)  # the default cap converges
    assert max(M.ranks(0)) > 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_entries_report_no_convergence(bad):
    D, T, G, Gd = _setup()
    # an entry inside an admissible block
    blk = T.blocks()
    cl = T.clusters()
    b = int(np.flatnonzero(blk[:, 2])[0])
    i, j = int(cl["start"][blk[b, 0]]), int(cl["start"][blk[b, 1]])
    Gbad = Gd.clone()
    Gbad[i, j] = complex(bad, 0.0)
    st, h = _raw_compress(D, T, Gbad, D.MODE_FP64)
    assert st == DH2_ENOCONV and h is None
    M = D.dh2_compress(T, Gd, mode=D.MODE_FP64)
    assert max(M.ranks(0)) > 0


@pytest.mark.parametrize("nth", [1, 2, 3])
def test_refused_allocation_reports_no_memory(nth):
    D, _, G, Gd = _setup()
    pts = fibonacci_sphere(1024)
    T = D.dh2_tree_build(pts, 32, 6.0)  # fresh tree: its device upload is the first allocation
    D.dh2_debug_fail_alloc(nth)
    try:
        st, h = _raw_compress(D, T, Gd, D.MODE_FP64)
    finally:
        D.dh2_debug_fail_alloc(0)
    assert st == DH2_ENOMEM and h is None
    M = D.dh2_compress(T, Gd, mode=D.MODE_FP64)
    assert max(M.ranks(0)) > 0
    x = torch.ones((1024,), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    D.dh2_debug_fail_alloc(1)
    try:
        with pytest.raises(D.DH2Error) as ei:
            D.dh2_matvec(M, x, y)  # its coefficient buffer is refused
    finally:
        D.dh2_debug_fail_alloc(0)
    assert ei.value.status == DH2_ENOMEM
    D.dh2_matvec(M, x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(y)).all()


def test_matvec_operands_checked_before_the_call():
    D, T, G, Gd = _setup()
    M = D.dh2_compress(T, Gd, mode=D.MODE_FP64)
    n = Gd.shape[0]
    good = torch.ones((n,), dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        D.dh2_matvec(M, good.to(torch.complex64), good.to(torch.complex64))
    with pytest.raises(ValueError):
        D.dh2_matvec(M, good[: n - 1], torch.empty_like(good[: n - 1]))
    with pytest.raises(ValueError):
        D.dh2_matvec(M, good, torch.empty((n, 2), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        D.dh2_matvec(M, good.cpu(), good.cpu())
