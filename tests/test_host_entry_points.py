"""Host-only entry points of the library, exercised without a GPU: the DCT-II
temporal basis (App. E.2.1), the restricted eigensolve's defaults, and the
argument checks of a problem given by its operator, which refuse a malformed
CSR before any device call."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp


@pytest.fixture(scope="module")
def sdf():
    from paper_2606_17971_b300 import sdf as S
    return S


def test_dct2_basis_matches_oracle_and_scipy(sdf):
    from scipy.fft import dct
    from oracle import spacetime_oracle as ST
    for n, r in ((8, 8), (16, 5), (1, 1), (13, 13)):
        w = sdf.dct2_basis(n, r)
        np.testing.assert_allclose(w, ST.dct2_basis(n, r), atol=1e-15)
        ref = dct(np.eye(n), type=2, norm="ortho", axis=0)[:r].T
        np.testing.assert_allclose(w, ref, atol=1e-14)
    # out-of-range requests leave the output untouched
    w = np.full((4, 5), 7.0, order="F")
    sdf._lib.sdf_dct2_basis(4, 5, w.ctypes.data)
    assert np.all(w == 7.0)


def test_restricted_eigensolve_defaults(sdf):
    o = sdf.EigOpts()
    sdf._lib.sdf_default_restricted_eig_opts(10, ctypes.byref(o))
    assert (o.degree, o.guard, o.tol) == (200, 32, 1e-8)
    sdf._lib.sdf_default_restricted_eig_opts(100, ctypes.byref(o))
    assert o.guard == 50


def _create(sdf, K, **kw):
    rp = np.ascontiguousarray(K.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(K.indices, dtype=np.int32)
    v = np.ascontiguousarray(K.data, dtype=np.float64)
    h = ctypes.c_void_p()
    st = sdf._lib.sdf_problem_create_csr(K.shape[0], rp.ctypes.data, ci.ctypes.data,
                                         v.ctypes.data, kw.get("mass", 1.0),
                                         kw.get("alpha", 1e-4), kw.get("kscale", 1.0),
                                         ctypes.byref(h))
    if h.value:
        sdf._lib.sdf_problem_destroy(h)
    return st


def test_malformed_csr_operators_are_refused_on_the_host(sdf):
    K = sp.random(50, 50, density=0.1, format="csr", random_state=3) + sp.identity(50)
    K = K.tocsr()
    bad = K.copy()
    bad.indices[3] = 60  # a column outside [0, n)
    assert _create(sdf, bad) == 1
    bad = K.copy()
    bad.data[5] = np.nan  # a non-finite value
    assert _create(sdf, bad) == 1
    assert _create(sdf, K, alpha=0.0) == 1  # alpha must be positive
    assert _create(sdf, K, mass=-1.0) == 1
