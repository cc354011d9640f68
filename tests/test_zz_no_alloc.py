"""The allocation-free matrix-vector product against dh2_matvec.

dh2_matvec_noalloc serves callers that may not allocate device memory during
a call; it must give the same product as dh2_matvec (same kernels, scratch
taken from a fixed library array), also on a second call that reuses the
array, and refuse a product whose coefficient vectors do not fit.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

from synth import fibonacci_sphere, helmholtz_matrix, random_complex_vectors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mode_name", ["fp64", "fp32"])
def test_noalloc_matvec_matches_matvec(mode_name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_07087_gb300 as D

    n, kappa, leaf = 2048, 4.0, 32
    pts = fibonacci_sphere(n)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa)[np.ix_(perm, perm)]
    dt = torch.complex128 if mode_name == "fp64" else torch.complex64
    tol = 1e-12 if mode_name == "fp64" else 1e-5
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", dt).t()
    M = D.dh2_compress(T, Gd, eps=1e-4)
    for call in range(2):
        x = random_complex_vectors(n, 3, seed=100 + call)
        xd = torch.from_numpy(np.ascontiguousarray(x.T)).to("cuda", dt).t()
        y_ref = torch.empty_like(xd.t().contiguous()).t()
        y_new = torch.full_like(xd.t().contiguous(), float("nan")).t()
        D.dh2_matvec(M, xd, y_ref)
        D.dh2_matvec_noalloc(M, xd, y_new)
        torch.cuda.synchronize()
        a = y_ref.cpu().numpy()
        b = y_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a)
    # coefficient vectors beyond the fixed array are refused, and nothing is written
    big = 4096
    xb = torch.zeros((n, big), dtype=dt, device="cuda").t().contiguous().t()
    yb = torch.zeros_like(xb.t().contiguous()).t()
    with pytest.raises(D.DH2Error):
        D.dh2_matvec_noalloc(M, xb, yb)
    torch.cuda.synchronize()
    assert not torch.any(torch.view_as_real(yb) != 0)
