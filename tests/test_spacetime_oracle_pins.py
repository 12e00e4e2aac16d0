"""Pins of the space-time oracle (App. E.2, App. F.5) against the
definitions it restates: the spatial operator against the pinned steady
assembly, F against the implicit Euler sweep, the block-tridiagonal SPD
structure and a closed-form spectrum, the desired state's temporal ramp,
the Kronecker and constant-in-time bases, a complete basis converging at
once, parity with a sparse direct solve, and the paper's finding that the
Kronecker basis deflates far better than the constant-in-time lift."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import oracle as O
from oracle import spacetime_oracle as ST


def test_spatial_operator_is_the_steady_assembly():
    for n in (5, 9):
        rp, ci, v = O.Problem(2, n).csr_A()
        A_c = sp.csr_matrix((v, ci, rp), shape=(n * n, n * n))
        assert abs(ST.laplacian_2d(n) - A_c).max() < 1e-9 * abs(A_c).max()


def test_forward_operator_is_implicit_euler():
    n, n_t = 7, 5
    A_s = ST.laplacian_2d(n, 0.3)
    F = ST.forward_operator(A_s, n_t, T=2.0)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(n * n * n_t)
    y = ST.time_steps(u, A_s, n_t, T=2.0)
    assert np.linalg.norm(F @ y - u) <= 1e-11 * np.linalg.norm(u)
    # causality: a source at the last step leaves earlier steps at zero
    u2 = np.zeros_like(u)
    u2[-n * n:] = 1.0
    y2 = spla.spsolve(F.tocsc(), u2)
    assert np.all(y2[: -n * n] == 0.0) and np.all(y2[-n * n:] > 0)


def test_schur_is_block_tridiagonal_spd_with_closed_form_single_step_spectrum():
    n, n_t, alpha = 6, 4, 1e-3
    F = ST.forward_operator(ST.laplacian_2d(n), n_t)
    S = ST.schur(F, alpha).toarray()
    Ns = n * n
    assert np.allclose(S, S.T, atol=0)
    for i in range(n_t):
        for j in range(n_t):
            if abs(i - j) >= 2:
                assert not np.any(S[i * Ns:(i + 1) * Ns, j * Ns:(j + 1) * Ns])
    assert np.linalg.eigvalsh(S).min() >= 1.0 - 1e-12
    # one time step: S = I + alpha (I/dt + A)^2 with A's eigenvalues
    # mu_i + mu_j, mu_q = 4 (n+1)^2 sin^2(q pi / (2 (n+1)))
    S1 = ST.schur(ST.forward_operator(ST.laplacian_2d(n), 1, T=0.5), alpha).toarray()
    mu = 4.0 * (n + 1) ** 2 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    lam = np.sort((1.0 + alpha * (2.0 + mu[:, None] + mu[None, :]) ** 2).ravel())
    np.testing.assert_allclose(np.linalg.eigvalsh(S1), lam, rtol=1e-12)


def test_desired_state_ramp_and_profile():
    n, n_t, tau = 9, 6, 0.2
    yd, rhs = ST.desired_state(n, n_t, 2.0, (0.5, 0.5), sigma=0.12, tau=tau, mass=1.5)
    Ns = n * n
    slabs = yd.reshape(n_t, Ns)
    t = (np.arange(n_t) + 1) / n_t
    ramp = 1.0 - np.exp(-t / tau)
    for l in range(n_t):
        np.testing.assert_allclose(slabs[l], slabs[-1] * ramp[l] / ramp[-1], rtol=1e-13)
    # the centre node of an odd grid sits at c: amplitude a there
    assert slabs[-1][(n // 2) * n + n // 2] == pytest.approx(2.0 * ramp[-1], rel=1e-14)
    np.testing.assert_allclose(rhs, 1.5 * yd, rtol=0)


def test_bases_are_orthonormal_with_the_stated_support():
    n, n_t, r = 6, 4, 5
    Z_s = O.analytic_modes(2, n, r, 1e-3)[0]
    K = ST.kron_basis(Z_s, n_t)
    C = ST.constant_lift(Z_s, n_t)
    Ns = n * n
    np.testing.assert_allclose(K.T @ K, np.eye(r * n_t), atol=1e-13)
    np.testing.assert_allclose(C.T @ C, np.eye(r), atol=1e-13)
    for l in range(n_t):
        for j in range(r):
            col = K[:, l * r + j]
            assert np.all(np.delete(col.reshape(n_t, Ns), l, axis=0) == 0.0)
            np.testing.assert_array_equal(col[l * Ns:(l + 1) * Ns], Z_s[:, j])


def test_complete_kronecker_basis_converges_at_once_and_solve_matches_direct():
    n, n_t, alpha = 4, 3, 1e-3
    P, S = ST.problem(n, n_t, alpha)
    Ns = n * n
    Z_s = np.linalg.eigh(ST.laplacian_2d(n).toarray())[1]   # complete spatial basis
    Z = ST.kron_basis(Z_s, n_t)
    yd, rhs = ST.desired_state(n, n_t, 3.0, (0.5, 0.5), sigma=0.2)
    big = np.full(P.N, 10.0)
    r = P.solve(rhs, big, Z)
    assert r["outer_iters"] == 1 and r["cg_iters"] == [0]
    # a binding bound: the final active set's restricted system, directly
    n2, nt2 = 10, 6
    P2, S2 = ST.problem(n2, nt2, 1e-4)
    yd2, rhs2 = ST.desired_state(n2, nt2, 3.0, (0.45, 0.55))
    psi = np.full(P2.N, 1.0)
    Zs2 = O.analytic_modes(2, n2, 8, 1e-4)[0]
    res = P2.solve(rhs2, psi, ST.kron_basis(Zs2, nt2))
    act = res["active"]
    assert res["status"] == 0 and act.sum() > 0
    I = np.flatnonzero(~act)
    A_ = np.flatnonzero(act)
    S2c = S2.tocsr()
    b = rhs2[I] - S2c[I][:, A_] @ psi[A_]
    x = spla.spsolve(S2c[I][:, I].tocsc(), b)
    assert np.linalg.norm(res["y"][I] - x) <= 1e-6 * np.linalg.norm(x)
    np.testing.assert_array_equal(res["y"][A_], psi[A_])
    assert np.all(res["y"] <= psi + 1e-10)


def test_kronecker_basis_deflates_far_better_than_constant_lift():
    # App. E.2.1 / Sec. 4.3: the constant-in-time lift reduces CG iterations
    # by a few percent (1-19 % in the paper's table), the Kronecker basis by
    # more than half (56-85 %)
    n, n_t, r = 16, 8, 16
    P, _ = ST.problem(n, n_t, 1e-4)
    yd, rhs = ST.desired_state(n, n_t, 2.0, (0.5, 0.5))
    psi = np.full(P.N, 10.0)   # inactive: one clean solve each
    Z_s = O.analytic_modes(2, n, r, 1e-4)[0]
    cold = P.solve(rhs, psi, None, deflate=False)["cg_iters"][0]
    const = P.solve(rhs, psi, ST.constant_lift(Z_s, n_t))["cg_iters"][0]
    kron = P.solve(rhs, psi, ST.kron_basis(Z_s, n_t))["cg_iters"][0]
    assert kron < 0.5 * cold, (cold, const, kron)
    assert const > 0.8 * cold, (cold, const, kron)


def test_schur_solution_minimises_the_reduced_objective():
    # S_st y = y_d is the optimality condition of
    # J(y) = 1/2 ||y - y_d||^2 + alpha/2 ||F y||^2 (u = F y); J is quadratic, so
    # its central difference at the minimiser vanishes along every direction
    n, n_t, alpha = 6, 5, 1e-3
    F = ST.forward_operator(ST.laplacian_2d(n), n_t)
    S = ST.schur(F, alpha)
    yd, _ = ST.desired_state(n, n_t, 2.0, (0.4, 0.6))
    y = spla.spsolve(S.tocsc(), yd)

    def J(v):
        return 0.5 * np.sum((v - yd) ** 2) + 0.5 * alpha * np.sum((F @ v) ** 2)

    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(y.size)
        v /= np.linalg.norm(v)
        eps = 1e-3
        d = (J(y + eps * v) - J(y - eps * v)) / (2 * eps)
        assert abs(d) <= 1e-7 * np.linalg.norm(yd), d


def test_desired_state_slabs_are_the_steady_desired_state_ramped():
    n, n_t, tau, a, c, sigma = 11, 4, 0.2, 2.5, (0.35, 0.6), 0.12
    yd, _ = ST.desired_state(n, n_t, a, c, sigma=sigma, tau=tau)
    steady = O.Problem(2, n).desired_state(a, c, sigma)[0]
    t = (np.arange(n_t) + 1) / n_t
    for l in range(n_t):
        np.testing.assert_allclose(yd[l * n * n:(l + 1) * n * n],
                                   (1.0 - np.exp(-t[l] / tau)) * steady, rtol=1e-13, atol=1e-300)


def test_dct2_basis_is_scipys_orthonormal_dct():
    from scipy.fft import dct
    for n_t, r_t in ((8, 8), (16, 5), (7, 3)):
        W = ST.dct2_basis(n_t, r_t)
        # the orthonormal DCT-II of the identity: row a is basis vector a
        ref = dct(np.eye(n_t), type=2, norm="ortho", axis=0)[:r_t].T
        np.testing.assert_allclose(W, ref, atol=1e-14)
        np.testing.assert_allclose(W.T @ W, np.eye(r_t), atol=1e-14)


def test_full_cosine_basis_equals_kronecker_and_truncation_degrades():
    # App. E.2.1: W_t (x) Z_s with r_t = n_t spans the Kronecker basis' space,
    # so A-DEF2 (invariant under Z -> Z G) takes the same iterations; with
    # r_t < n_t it deflates less
    n, n_t, r = 16, 8, 16
    P, _ = ST.problem(n, n_t, 1e-4)
    yd, rhs = ST.desired_state(n, n_t, 2.0, (0.5, 0.5))
    psi = np.full(P.N, 10.0)
    Z_s = O.analytic_modes(2, n, r, 1e-4)[0]
    kron = P.solve(rhs, psi, ST.kron_basis(Z_s, n_t))
    full = P.solve(rhs, psi, ST.temporal_basis(ST.dct2_basis(n_t, n_t), Z_s))
    half = P.solve(rhs, psi, ST.temporal_basis(ST.dct2_basis(n_t, n_t // 2), Z_s))
    assert abs(full["cg_iters"][0] - kron["cg_iters"][0]) <= 1
    assert np.linalg.norm(full["y"] - kron["y"]) <= 1e-7 * np.linalg.norm(kron["y"])
    assert half["cg_iters"][0] > kron["cg_iters"][0] + 5
    np.testing.assert_array_equal(ST.temporal_basis(np.eye(n_t), Z_s), ST.kron_basis(Z_s, n_t))
