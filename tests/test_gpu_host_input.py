"""Compression of a host-resident G (dh2_compress_host): the library copies G
to the device in column panels and overlaps each panel's column-basis leaf
work with the next copy.  Every kernel sees the same entries as with a
device-resident G, so the results must agree exactly."""
import numpy as np
import pytest

from synth import fibonacci_sphere, helmholtz_matrix, mean_nn_distance, random_complex_vectors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1510_07087_gb300 as D
    return D


def _matvec(D, M, x, dt):
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).to("cuda", dt).t()
    yd = torch.empty_like(xd.t().contiguous()).t()
    D.dh2_matvec(M, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,kappa,leaf,fp64,pad", [(8192, 16.0, 32, False, 0), (4096, 12.0, 32, True, 3),
                                                   (2048, 4.0, 32, False, 1)])
def test_host_input_equals_device_input(n, kappa, leaf, fp64, pad):
    D = _dev()
    pts = fibonacci_sphere(n)
    h = mean_nn_distance(pts)
    T = D.dh2_tree_build(pts, leaf, kappa)
    perm = T.perm()
    G = helmholtz_matrix(pts, kappa, h)[np.ix_(perm, perm)]
    cdt = torch.complex128 if fp64 else torch.complex64
    mode = D.MODE_FP64 if fp64 else D.MODE_FP32
    # host copy, column-major with leading dimension n + pad, page-locked
    Gh = torch.zeros((n, n + pad), dtype=cdt, pin_memory=True)
    Gh[:, :n] = torch.from_numpy(np.ascontiguousarray(G.T))
    Gh_cm = Gh[:, :n].t()
    assert Gh_cm.stride() == (1, n + pad)
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", cdt).t()
    Md = D.dh2_compress(T, Gd, eps=1e-4, mode=mode)
    Mh = D.dh2_compress_host(T, Gh_cm, eps=1e-4, mode=mode)
    # the same kernels on the same entries: ranks, singular values, bases and
    # couplings agree bit for bit (sampled)
    for sd in (0, 1):
        assert np.array_equal(Md.ranks(sd), Mh.ranks(sd))
        npairs = len(Md.ranks(sd))
        for pid in range(0, npairs, max(1, npairs // 40)):
            assert np.array_equal(Md.sigma(sd, pid), Mh.sigma(sd, pid))
            assert np.array_equal(Md.pair_basis(sd, pid), Mh.pair_basis(sd, pid))
    adm = np.flatnonzero(T.blocks()[:, 2])
    for b in adm[:: max(1, len(adm) // 40)]:
        assert np.array_equal(Md.coupling(int(b)), Mh.coupling(int(b)))
    # the matrix-vector product accumulates with atomics: equal up to rounding
    x = random_complex_vectors(n, 2, seed=29)
    yd = _matvec(D, Md, x, cdt)
    yh = _matvec(D, Mh, x, cdt)
    tol = 1e-12 if fp64 else 1e-5
    assert np.linalg.norm(yh - yd) <= tol * np.linalg.norm(yd)
    G128 = torch.from_numpy(np.ascontiguousarray(G.T)).to("cuda", torch.complex128).t()
    assert D.dh2_error(Mh, G128) <= 1e-4
    # a second call on the same tree reuses the staging buffer
    Mh2 = D.dh2_compress_host(T, Gh_cm, eps=1e-4, mode=mode)
    for b in adm[:: max(1, len(adm) // 10)]:
        assert np.array_equal(Mh2.coupling(int(b)), Mh.coupling(int(b)))


def test_host_input_rejects_view_mode_and_device_memory():
    D = _dev()
    from paper_1510_07087_gb300 import _binding as B
    n = 256
    pts = fibonacci_sphere(n)
    T = D.dh2_tree_build(pts, 16, 4.0)
    Gh = torch.zeros((n, n), dtype=torch.complex64, pin_memory=True)
    p = B.CompressParams(1e-4, 2.0 / 3.0, 0, D.MODE_FP32, 1, 0)  # nearfield = view
    h = B.c_void_p()
    st = B._lib().dh2_compress_host(T.handle, B.c_void_p(Gh.data_ptr()), B.DH2_C64, n, B.byref(p),
                                    B.c_void_p(torch.cuda.current_stream().cuda_stream), B.byref(h))
    assert st == 1 and not h.value
    with pytest.raises(ValueError):
        D.dh2_compress_host(T, torch.zeros((n, n), dtype=torch.complex64, device="cuda").t())
