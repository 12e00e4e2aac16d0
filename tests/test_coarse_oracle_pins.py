"""Pins of the coarse-grid basis oracle (oracle/coarse_oracle.py) against
closed forms: injection at coincident nodes, second-order interpolation of a
smooth function, the Kronecker structure against a direct bilinear
interpolation, kappa injection, and the deflating property of the basis."""
import numpy as np

from oracle import coarse_oracle as C
from oracle import oracle as O


def test_prolongation_is_injection_at_coincident_nodes_and_linear_between():
    nc, c = 7, 4
    n = c * (nc + 1) - 1           # fine nodes include every coarse node
    P = C.p1d(n, nc)
    for j in range(nc):
        i = c * (j + 1) - 1
        assert P[i, j] == 1.0 and P[i].sum() == 1.0
    # midpoint between coarse nodes 2 and 3
    i = c * 3 + c // 2 - 1
    np.testing.assert_allclose(P[i, 2:4], [0.5, 0.5])


def test_prolongation_interpolates_smooth_functions_to_second_order():
    errs = []
    for nc in (15, 31, 63):
        n = 2 * nc + 5
        xc = (np.arange(nc) + 1) / (nc + 1)
        xf = (np.arange(n) + 1) / (n + 1)
        f = lambda x: np.sin(np.pi * x) * np.exp(x)
        errs.append(np.abs(C.p1d(n, nc) @ f(xc) - f(xf)).max())
    assert errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_kronecker_prolongation_matches_direct_bilinear_interpolation():
    n, nc = (9, 7), (4, 3)
    P = C.prolongation(n, nc)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(nc[0] * nc[1])
    U = np.zeros((nc[1] + 2, nc[0] + 2))     # with the zero boundary
    U[1:-1, 1:-1] = u.reshape(nc[1], nc[0])
    out = np.zeros(n[0] * n[1])
    for jy in range(n[1]):
        ty = (jy + 1) / (n[1] + 1) * (nc[1] + 1)
        y0 = int(np.floor(ty)); wy = ty - y0
        for ix in range(n[0]):
            tx = (ix + 1) / (n[0] + 1) * (nc[0] + 1)
            x0 = int(np.floor(tx)); wx = tx - x0
            out[jy * n[0] + ix] = ((1 - wy) * ((1 - wx) * U[y0, x0] + wx * U[y0, x0 + 1]) +
                                   wy * ((1 - wx) * U[y0 + 1, x0] + wx * U[y0 + 1, x0 + 1]))
    np.testing.assert_allclose(P @ u, out, atol=1e-14)


def test_coarse_kappa_injection():
    n, nc = (8, 6), (4, 3)
    kap = np.arange(48, dtype=float)           # kappa = node index
    kc = C.coarse_kappa(kap, n, nc)
    # coarse node (ic, jc) sits nearest fine node (round(x_c 9) - 1, round(y_c 7) - 1)
    for jc in range(3):
        for ic in range(4):
            i = int(np.rint((ic + 1) / 5 * 9)) - 1
            j = int(np.rint((jc + 1) / 4 * 7)) - 1
            assert kc[jc * 4 + ic] == j * 8 + i
    assert np.all(C.coarse_kappa(np.ones(48), n, nc) == 1.0)


def test_qr_discard_drops_dependent_columns():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 4))
    A = np.column_stack([A, A[:, 0] + A[:, 1]])      # dependent fifth column
    Q = C.qr_discard(A, 1e-8)
    assert Q.shape == (50, 4)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-13)


def test_coarse_basis_deflates_the_fine_solve():
    n = (40, 36)
    Phi, lam = C.coarse_modes(2, n, 2, 16)
    assert Phi.shape == (1440, 16)
    np.testing.assert_allclose(Phi.T @ Phi, np.eye(16), atol=1e-12)
    P = O.Problem(2, n, alpha=1e-4)
    _, rhs = P.desired_state(2.0, (0.4, 0.6), 0.1)
    act = np.zeros(P.N, np.uint8)
    psi = np.full(P.N, 10.0)
    plain = P.inner_solve(act, rhs, psi, None, deflate=False)
    defl = P.inner_solve(act, rhs, psi, Phi)
    assert defl["iters"] < 0.7 * plain["iters"]
    np.testing.assert_allclose(defl["x"], plain["x"], rtol=0, atol=1e-6 * np.abs(plain["x"]).max())
