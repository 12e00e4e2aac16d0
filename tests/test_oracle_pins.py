"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks it against an
independent construction (dense first-principles matrices, dense LAPACK
solves, closed forms, a different but equivalent algorithm) or against numbers
the paper prints (tests/golden/paper_tables.json).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_17971_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


# --------------------------------------------------------------------------
# independent first-principles operators (dense, numpy)

def lap1d(n):
    h = 1.0 / (n + 1)
    return (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / h**2


def laplacian_kron(dim, n):
    """L_h as a Kronecker sum of 1D second differences (App. A, Sec. 2.2.8)."""
    L1, I = lap1d(n), np.eye(n)
    if dim == 2:
        return np.kron(I, L1) + np.kron(L1, I)
    return np.kron(np.kron(I, I), L1) + np.kron(np.kron(I, L1), I) + np.kron(np.kron(L1, I), I)


def flux_operator_2d(n, kappa, eps=1.0, b=(0.0, 0.0)):
    """-eps div(kappa grad) by face fluxes with harmonic face means (Eq.
    harmonic), boundary faces taking the node value, plus first-order upwind
    b.grad; assembled face by face rather than row by row."""
    h = 1.0 / (n + 1)
    N = n * n
    A = np.zeros((N, N))
    k = kappa.reshape(n, n)  # [y, x]
    idx = np.arange(N).reshape(n, n)
    for y in range(n):
        for x in range(n):
            p = idx[y, x]
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                yy, xx = y + dy, x + dx
                if 0 <= yy < n and 0 <= xx < n:
                    kf = 2 * k[y, x] * k[yy, xx] / (k[y, x] + k[yy, xx])
                    A[p, p] += eps * kf / h**2
                    A[p, idx[yy, xx]] -= eps * kf / h**2
                else:
                    A[p, p] += eps * k[y, x] / h**2
    # upwind convection via 1D one-sided difference matrices
    Dm = (np.eye(n) - np.eye(n, k=-1)) / h   # backward difference
    Dp = (np.eye(n, k=1) - np.eye(n)) / h    # forward difference
    I = np.eye(n)
    bx, by = b
    A += bx * np.kron(I, Dm if bx > 0 else Dp) + by * np.kron(Dm if by > 0 else Dp, I)
    return A


# --------------------------------------------------------------------------
# P1: operator assembly

@pytest.mark.parametrize("dim,n", [(2, 7), (3, 4)])
def test_S_equals_identity_plus_alpha_L_squared(dim, n):
    alpha = 3e-4
    P = O.Problem(dim, n, alpha=alpha)
    L = laplacian_kron(dim, n)
    S_ref = np.eye(n**dim) + alpha * L.T @ L
    S = P.dense_S()
    assert np.max(np.abs(S - S_ref)) <= 1e-13 * np.max(np.abs(S_ref))
    assert np.array_equal(S, S.T)
    assert np.linalg.eigvalsh(S).min() >= 1.0 - 1e-12  # Sec. 2.1.2: lambda_min >= 1


def test_S_variable_kappa_and_upwind_convection():
    n, alpha = 6, 1e-4
    rng = np.random.default_rng(5)
    kappa = 10.0 ** rng.uniform(-1, 1, n * n)
    b = (0.6, -0.8)
    A_ref = flux_operator_2d(n, kappa, eps=1e-2, b=b)
    P = O.Problem(2, n, kappa=kappa, diff_scale=1e-2, b=np.array(b), alpha=alpha)
    rp, ci, v = P.csr_A()
    A = np.zeros((n * n, n * n))
    A[np.repeat(np.arange(n * n), np.diff(rp)), ci] = v
    assert np.max(np.abs(A - A_ref)) <= 1e-12 * np.max(np.abs(A_ref))
    S_ref = np.eye(n * n) + alpha * A_ref.T @ A_ref
    S = P.dense_S()
    assert np.max(np.abs(S - S_ref)) <= 1e-12 * np.max(np.abs(S_ref))
    assert np.max(np.abs(S - S.T)) <= 1e-12 * np.max(np.abs(S))


@pytest.mark.parametrize("dim,n,k", [(2, 12, 6), (2, 20, 16), (3, 6, 10)])
def test_analytic_modes_are_eigenpairs_of_S(dim, n, k):
    alpha = 1e-4
    P = O.Problem(dim, n, alpha=alpha)
    S = P.dense_S()
    Phi, lam, _ = O.analytic_modes(dim, n, k, alpha)
    w, V = np.linalg.eigh(S)
    tol = GOLD["analytic_vs_iterative_eig_max_rel_err"]["value"]
    assert np.max(np.abs(lam - w[:k]) / w[:k]) <= tol
    assert np.max(np.abs(S @ Phi - Phi * lam)) <= 1e-10 * np.max(lam)
    assert np.max(np.abs(Phi.T @ Phi - np.eye(k))) <= 1e-12
    if w[k] > w[k - 1] * (1 + 1e-9):  # clean cut: same subspace (0 deg angles)
        s = np.linalg.svd(V[:, :k].T @ Phi, compute_uv=False)
        assert s.min() >= 1 - 1e-10


# --------------------------------------------------------------------------
# P2: Cauchy interlacing of the restricted operator

def test_cauchy_interlacing_of_S_II():
    n = 8
    P = O.Problem(2, n, alpha=1e-3)
    S = P.dense_S()
    rng = np.random.default_rng(1)
    act = rng.random(n * n) < 0.3
    I = ~act
    lam = np.linalg.eigvalsh(S)
    mu = np.linalg.eigvalsh(S[np.ix_(I, I)])
    N, m = n * n, I.sum()
    for j in range(m):
        assert lam[j] <= mu[j] * (1 + 1e-12)
        assert mu[j] <= lam[j + N - m] * (1 + 1e-12)


# --------------------------------------------------------------------------
# P3: separable closed form

@pytest.mark.parametrize("dim,n", [(2, 24), (3, 10)])
@pytest.mark.parametrize("deflate", [False, True])
def test_separable_desired_state_closed_form(dim, n, deflate):
    """y_d = a prod sin(pi x_l) sampled at the nodes is an eigenvector of L_h
    with eigenvalue dim*mu_1, hence of S; with an inactive bound the solve
    returns y_d / (alpha (dim mu_1)^2 + 1) (discrete form of App. C.1 2d_sym)."""
    alpha, a = 1e-3, 1.1
    P = O.Problem(dim, n, alpha=alpha)
    h = 1.0 / (n + 1)
    s = np.sin(np.pi * (np.arange(n) + 1) * h)
    yd = a * (np.multiply.outer(s, s) if dim == 2 else np.multiply.outer(s, np.multiply.outer(s, s))).ravel()
    mu1 = 4 / h**2 * np.sin(np.pi / (2 * (n + 1))) ** 2
    y_exact = yd / (alpha * (dim * mu1) ** 2 + 1)
    Phi = O.analytic_modes(dim, n, 8, alpha)[0] if deflate else None
    r = P.solve(yd, np.full(n**dim, 10.0), Phi, deflate=deflate, rtol=1e-12)
    assert r["status"] == 0 and r["outer_iters"] == 1 and not r["active"].any()
    assert np.linalg.norm(r["y"] - y_exact) <= 1e-10 * np.linalg.norm(y_exact)
    if dim == 2:  # continuum factor of the paper, 1/(1 + 4 pi^4 alpha), as h -> 0
        assert abs(1 / (alpha * (2 * mu1) ** 2 + 1) - 1 / (1 + 4 * np.pi**4 * alpha)) < 2e-3


# --------------------------------------------------------------------------
# P4: inner solves

def _restricted_dense(P, act, rhs, psi):
    S = P.dense_S()
    I = ~act
    b = rhs[I] - S[np.ix_(I, act)] @ psi[act]
    return S, I, b


@pytest.mark.parametrize("deflate", [False, True])
def test_inner_solve_matches_dense_cholesky(deflate):
    n = 16
    P = O.Problem(2, n, alpha=1e-4)
    rng = np.random.default_rng(3)
    act = np.zeros(n * n, bool)
    act.reshape(n, n)[5:9, 4:11] = True
    act |= rng.random(n * n) < 0.05
    rhs = rng.standard_normal(n * n)
    psi = 0.5 + rng.random(n * n)
    S, I, b = _restricted_dense(P, act, rhs, psi)
    x_ref = np.linalg.solve(np.linalg.cholesky(S[np.ix_(I, I)]).T,
                            np.linalg.solve(np.linalg.cholesky(S[np.ix_(I, I)]), b))
    Phi = O.dense_modes(P, 12)[0] if deflate else None
    r = P.inner_solve(act, rhs, psi, Phi, deflate=deflate, rtol=1e-12)
    assert r["status"] == 0 and r["fallback"] == 0
    assert np.linalg.norm(r["x"][I] - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert np.array_equal(r["x"][act], psi[act])


def test_full_coarse_space_solves_in_zero_iterations():
    """With Z spanning all of R^{n_I} the coarse correction Q b alone is the
    solution (Eq. coarse), so A-DEF2 stops before its first iteration."""
    n = 6
    P = O.Problem(2, n, alpha=1e-3)
    act = np.zeros(n * n, bool)
    act[[7, 8, 14]] = True
    I = np.flatnonzero(~act)
    Phi = np.zeros((n * n, I.size))
    Phi[I, np.arange(I.size)] = 1.0
    Phi = Phi @ np.linalg.qr(np.random.default_rng(0).standard_normal((I.size, I.size)))[0]
    rhs = np.random.default_rng(2).standard_normal(n * n)
    psi = np.ones(n * n)
    S, Im, b = _restricted_dense(P, act, rhs, psi)
    r = P.inner_solve(act, rhs, psi, Phi, deflate=True, rtol=1e-10)
    assert r["iters"] == 0 and r["fallback"] == 0
    assert np.allclose(r["x"][Im], np.linalg.solve(S[np.ix_(Im, Im)], b), rtol=1e-10, atol=0)


def def1_with_final_correction(S, b, Z, rtol, maxit=100000):
    """DEF1 of Tang et al.: CG on the left-deflated, Jacobi-preconditioned
    system and the final correction x = Q b + P^T x_tilde -- a different
    algorithm whose iterates share A-DEF2's spectrum."""
    E = Z.T @ S @ Z
    Einv = np.linalg.inv(E)
    Pd = np.eye(len(b)) - S @ Z @ Einv @ Z.T   # Tang's P = I - A Q
    d = np.diag(S)
    x = np.zeros_like(b)
    r = Pd @ b
    z = r / d
    p = z.copy()
    rho = r @ z
    it = 0
    Qb = Z @ (Einv @ (Z.T @ b))
    bn = np.linalg.norm(b)
    while True:
        xt = Qb + Pd.T @ x
        if np.linalg.norm(b - S @ xt) <= rtol * bn or it >= maxit:
            return xt, it
        q = Pd @ (S @ p)
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        z = r / d
        rn = r @ z
        p = z + (rn / rho) * p
        rho = rn
        it += 1


def test_adef2_matches_def1_with_correction():
    n = 14
    P = O.Problem(2, n, alpha=1e-4)
    act = np.zeros(n * n, bool)
    act.reshape(n, n)[4:8, 6:10] = True
    rng = np.random.default_rng(4)
    rhs = rng.standard_normal(n * n)
    psi = np.ones(n * n)
    S, I, b = _restricted_dense(P, act, rhs, psi)
    Phi = O.analytic_modes(2, n, 10, 1e-4)[0]
    Z = np.linalg.qr(Phi[I])[0]
    x1, it1 = def1_with_final_correction(S[np.ix_(I, I)], b, Z, 1e-10)
    r = P.inner_solve(act, rhs, psi, Phi, deflate=True, rtol=1e-10)
    plain = P.inner_solve(act, rhs, psi, None, deflate=False, rtol=1e-10)
    assert abs(r["iters"] - it1) <= 2
    assert r["iters"] < plain["iters"]
    assert np.linalg.norm(r["x"][I] - x1) <= 1e-8 * np.linalg.norm(x1)


def test_guard_falls_back_to_plain_pcg():
    n = 10
    P = O.Problem(2, n, alpha=1e-4)
    rhs = np.random.default_rng(6).standard_normal(n * n)
    psi = np.ones(n * n)
    act = np.zeros(n * n, bool)
    Phi = O.analytic_modes(2, n, 6, 1e-4)[0]
    plain = P.inner_solve(act, rhs, psi, None, deflate=False, rtol=1e-10)
    forced = P.inner_solve(act, rhs, psi, Phi, deflate=True, rtol=1e-10, tau_cond=1.0)
    assert forced["fallback"] == 1 and forced["iters"] == plain["iters"]
    assert np.array_equal(forced["x"], plain["x"])
    # a mode that vanishes on I makes the restriction rank deficient
    Phi2 = Phi.copy()
    Phi2[:, 0] = 0.0
    Phi2[3, 0] = 1.0
    act2 = act.copy()
    act2[3] = True
    r2 = P.inner_solve(act2, rhs, psi, Phi2, deflate=True, rtol=1e-10)
    assert r2["fallback"] == 1 and r2["status"] == 0


# --------------------------------------------------------------------------
# P5: the outer loop, replayed with dense solves

def dense_primal_active_set(S, rhs, psi, tau=1e-10, kmax=30):
    """App. B.1 Algorithm pdas with np.linalg.solve as the inner solve."""
    N = len(rhs)
    act = np.zeros(N, bool)
    seq = []
    for _ in range(kmax):
        I = ~act
        y = np.where(act, psi, 0.0)
        if I.any():
            y[I] = np.linalg.solve(S[np.ix_(I, I)], rhs[I] - S[np.ix_(I, act)] @ psi[act])
        new = y > psi - tau
        seq.append(int(act.sum()))
        if np.array_equal(new, act):
            return y, act, seq
        act = new
    return y, act, seq


def test_outer_loop_matches_dense_replay_on_32x32_workload():
    w = W.WORKLOADS["diff2d_32"]
    P = O.Problem(2, w.n, alpha=w.alpha)
    S = P.dense_S()
    Phi = O.dense_modes(P, w.k)[0]
    psi = W.psi_vector(w)
    lo, hi = GOLD["outer_iterations_range"]["min"], GOLD["outer_iterations_range"]["max"]
    nonempty = 0
    for ins in W.draw_instances(w):
        _, rhs = P.desired_state(ins.a, ins.c[:2], w.sigma)
        r = P.solve(rhs, psi, Phi, deflate=True, rtol=1e-8)
        y_d, act_d, seq = dense_primal_active_set(S, rhs, psi)
        assert r["status"] == 0
        assert np.array_equal(r["active"], act_d)
        assert r["n_active"] == seq
        assert np.linalg.norm(r["y"] - y_d) <= 1e-6 * np.linalg.norm(y_d)  # Eq. accuracy_rel_err
        assert np.all(r["y"] <= psi + 1e-12)
        lam = r["lam"]
        assert np.max(np.abs(lam[~r["active"]])) <= 1e-6 * np.linalg.norm(rhs)
        assert np.max(np.abs(lam * (r["y"] - psi))) <= 1e-6 * np.linalg.norm(rhs)
        if r["active"].any():
            nonempty += 1
            assert lo <= r["outer_iters"] <= hi
    assert nonempty >= 3


def test_pdas_rule_reaches_kkt_point():
    """Full PDAS (lambda_i + c (y_i - psi_i) > 0, App. B.1) ends at a KKT point
    with lambda >= 0; the primal rule need not (App. B.1 remark)."""
    w = W.WORKLOADS["diff2d_32"]
    P = O.Problem(2, w.n, alpha=w.alpha)
    psi = W.psi_vector(w)
    ins = max(W.draw_instances(w), key=lambda i: i.a)
    _, rhs = P.desired_state(ins.a, ins.c[:2], w.sigma)
    r = P.solve(rhs, psi, None, deflate=False, rtol=1e-12, rule=1)
    assert r["status"] == 0 and r["active"].any()
    tol = 1e-8 * np.linalg.norm(rhs)
    assert r["lam"][r["active"]].min() >= -tol
    assert np.all(r["y"] <= psi + 1e-9)
    primal = P.solve(rhs, psi, None, deflate=False, rtol=1e-12)
    assert primal["min_lambda_active"] < 0  # monotone primal rule overshoots


# --------------------------------------------------------------------------
# P9: scaling invariance of (K, M) -> (h^d K, h^d I)

def test_mass_and_stiffness_scaling_leave_the_solution_unchanged():
    w = W.WORKLOADS["diff2d_32"]
    h2 = (1.0 / (w.n + 1)) ** 2
    P1 = O.Problem(2, w.n, alpha=w.alpha)
    P2 = O.Problem(2, w.n, alpha=w.alpha, kscale=h2, mass=h2)
    psi = W.psi_vector(w)
    ins = max(W.draw_instances(w), key=lambda i: i.a)
    _, rhs1 = P1.desired_state(ins.a, ins.c[:2], w.sigma)
    _, rhs2 = P2.desired_state(ins.a, ins.c[:2], w.sigma)
    assert np.allclose(rhs2, h2 * rhs1, rtol=1e-15)
    r1 = P1.solve(rhs1, psi, None, deflate=False)
    r2 = P2.solve(rhs2, psi, None, deflate=False)
    assert np.array_equal(r1["active"], r2["active"])
    assert all(abs(a - b) <= 1 for a, b in zip(r1["cg_iters"], r2["cg_iters"]))
    assert np.linalg.norm(r1["y"] - r2["y"]) <= 1e-7 * np.linalg.norm(r1["y"])


# --------------------------------------------------------------------------
# P10: the paper's printed iteration counts (tests/golden/paper_tables.json)

def _suite_100(name):
    n = 100
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, x)
    if name == "2d_sym":
        return (lambda a: (a * np.sin(np.pi * X) * np.sin(np.pi * Y)).ravel()), 0.8, 1.2
    if name == "2d_nonsep":
        return (lambda a: (a * np.sin(2 * np.pi * X * Y)).ravel()), 0.8, 1.2

    def asym(t):  # App. C.1: four Gaussians rotating about (0.5, 0.5)
        r = np.sqrt(0.08)
        s = np.zeros_like(X)
        for k in range(4):
            ph = 5 * np.pi / 4 + k * np.pi / 2
            s += np.exp(-((X - 0.5 - r * np.cos(ph + t)) ** 2 + (Y - 0.5 - r * np.sin(ph + t)) ** 2)
                        / (2 * 0.1**2))
        return s.ravel()
    return asym, 0.0, np.pi / 2


def _calibrated_psi(P, f, lo, hi):
    un = P.inner_solve(np.zeros(P.N, np.uint8), f(0.5 * (lo + hi)), np.ones(P.N), None,
                       deflate=False, rtol=1e-10)
    return np.full(P.N, np.quantile(un["x"], 0.80))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["2d_sym", "2d_asym", "2d_nonsep"])
def test_cold_cg_iterations_match_paper_table(name):
    gold = GOLD["cold_cg_mean_iters_100x100"][name]
    P = O.Problem(2, 100, alpha=1e-3)
    f, lo, hi = _suite_100(name)
    psi = _calibrated_psi(P, f, lo, hi)
    its, frac = [], []
    for p in np.linspace(lo, hi, 30):
        r = P.solve(f(p), psi, None, deflate=False, rtol=1e-10, max_cg=10**6)
        assert r["status"] == 0
        its.append(r["cg_iters"][-1])
        frac.append(r["active"].mean())
    assert abs(np.mean(its) - gold) <= 0.005 * gold
    if name in GOLD["mean_active_fraction"]:
        assert abs(np.mean(frac) - GOLD["mean_active_fraction"][name]) <= 0.02


@pytest.mark.slow
def test_raw_eig100_deflated_iterations_match_paper_table():
    """Typical final-set A-DEF2 count with 100 restricted reference modes on
    2d_asym at 100^2 (the table's mean is dominated by typical instances
    there; we compare the median of every third instance)."""
    gold = GOLD["eig100_iters_2d_asym_100x100"]["value"]
    P = O.Problem(2, 100, alpha=1e-3)
    f, lo, hi = _suite_100("2d_asym")
    psi = _calibrated_psi(P, f, lo, hi)
    Phi = O.analytic_modes(2, 100, 100, 1e-3)[0]
    its = []
    for p in np.linspace(lo, hi, 30)[::3]:
        r = P.solve(f(p), psi, Phi, deflate=True, rtol=1e-10, max_cg=3000)
        its.append(r["cg_iters"][-1])
    assert abs(np.median(its) - gold) <= 0.1 * gold


def test_ritz_reselection_recovers_the_exact_modes_in_a_pool():
    # pool = the 8 lowest eigenvectors of S (A = {}) plus 8 random vectors:
    # the 8 smallest Ritz values of the pool are the 8 smallest eigenvalues
    # (Cauchy interlacing, attained on the exact vectors), so Ritz
    # re-selection must deflate exactly as the 8 exact modes do
    P = O.Problem(2, (24, 20), alpha=1e-4)
    V, lam = O.dense_modes(P, 8)
    rng = np.random.default_rng(11)
    pool = np.asfortranarray(np.column_stack([V, rng.standard_normal((P.N, 8))]))
    _, rhs = P.desired_state(2.0, (0.45, 0.55), 0.1)
    act = np.zeros(P.N, np.uint8)
    psi = np.full(P.N, 10.0)
    exact = P.inner_solve(act, rhs, psi, V)
    try:
        O.Problem.set_ritz(8)
        ritz = P.inner_solve(act, rhs, psi, pool)
    finally:
        O.Problem.set_ritz(0)
    assert abs(ritz["iters"] - exact["iters"]) <= 1, (ritz["iters"], exact["iters"])
    np.testing.assert_allclose(ritz["x"], exact["x"], rtol=0, atol=1e-7 * np.abs(exact["x"]).max())
    # the guard sees the selected Galerkin matrix: cond = lambda_8 / lambda_1
    np.testing.assert_allclose(ritz["cond_E"], lam[-1] / lam[0], rtol=1e-6)


def test_schur_from_operator_is_the_grid_assembly():
    # S from a state operator K (a problem given without a grid) against the
    # C assembly of the same grid operator, mass and kscale included
    import scipy.sparse as sp
    from paper_2606_17971_b300 import workloads as W
    w = W.scaled(W.WORKLOADS["block2d_1024"], 20)
    for mass, kscale in ((1.0, 1.0), (2.5, 0.7)):
        P = O.Problem(2, w.n, kappa=W.kappa_field(w), alpha=1e-3, mass=mass, kscale=kscale)
        rp, ci, v = P.csr_A()
        A = sp.csr_matrix((v, ci, rp), shape=(P.N, P.N))
        S = O.schur_from_operator(A, alpha=1e-3, mass=mass, kscale=kscale).toarray()
        np.testing.assert_allclose(S, P.dense_S(), rtol=1e-13, atol=1e-10)
    # a nonsymmetric operator (upwind convection): K^T K, not K K^T
    P = O.Problem(2, 14, diff_scale=1e-2, b=(0.8, -0.6), alpha=1e-3)
    rp, ci, v = P.csr_A()
    A = sp.csr_matrix((v, ci, rp), shape=(P.N, P.N))
    assert abs(A - A.T).max() > 1.0
    S = O.schur_from_operator(A, alpha=1e-3).toarray()
    np.testing.assert_allclose(S, P.dense_S(), rtol=1e-13, atol=1e-10)


# --------------------------------------------------------------------------
# true residual and attainable-accuracy floor of an inner solve (App. B.2)

def _dense_S_and_inactive(P, active):
    S = P.dense_S()
    I = np.flatnonzero(~active)
    return S, I


def test_floor_uses_the_entrywise_absolute_value_of_S_II():
    # Independent route to || |S_II| |x| ||: A is an M-matrix that couples
    # nearest neighbours only, so every entry of S = I + alpha A^T A has the
    # checkerboard sign s_i s_j and |S| = D S D with D = diag(s).  A planted
    # |S| x (no absolute value on S) or S |x| fails this on a convective,
    # variable-kappa operator with a non-empty active set.
    n = 14
    rng = np.random.default_rng(8)
    kappa = 10.0 ** rng.uniform(-1, 1, n * n)
    P = O.Problem(2, n, kappa=kappa, b=np.array([0.7, -0.4]), alpha=1e-4)
    rhs = P.desired_state(3.0, (0.4, 0.6), 0.12)[1]
    psi = np.full(P.N, 0.6)
    r = P.solve(rhs, psi, None, deflate=False, rtol=1e-10)
    assert r["status"] == 0 and r["outer_iters"] >= 2
    active = r["active"]
    # the last inner solve ran on the final active set (no change at exit)
    S, I = _dense_S_and_inactive(P, active)
    jj, ii = np.divmod(np.arange(P.N), n)
    d = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    SII = S[np.ix_(I, I)]
    x = r["y"][I]
    via_signs = (d[I][:, None] * SII * d[I][None, :]) @ np.abs(x)
    assert np.allclose(via_signs, np.abs(SII) @ np.abs(x), rtol=1e-14, atol=0)
    b = rhs[I] - S[np.ix_(I, np.flatnonzero(active))] @ psi[active]
    want = 10.0 * 2.0 ** -53 * np.linalg.norm(via_signs) / np.linalg.norm(b)
    assert r["relres_floor"][-1] == pytest.approx(want, rel=1e-12)
    assert r["true_relres_each"][-1] == pytest.approx(
        np.linalg.norm(b - SII @ x) / np.linalg.norm(b), rel=1e-6)


def test_floor_is_where_the_fp64_residual_of_the_exact_solution_lies():
    # The exact solution of S y = b, found by iterative refinement with
    # residuals in extended precision and rounded to FP64, has an FP64 true
    # residual that no FP64 method can beat.  It lies below the floor
    # 10 u || |S||y| || / ||b|| and within two decades of it (a floor of the
    # right size: neither vacuous nor unattainable).
    n = 22
    w = W.scaled(W.WORKLOADS["lognormal2d_2048"], n)
    P = O.Problem(2, n, kappa=W.kappa_field(w), alpha=1e-4)
    rhs = P.desired_state(2.0, (0.5, 0.5), 0.1)[1]
    S = P.dense_S()
    Sl = S.astype(np.longdouble)
    y = np.linalg.solve(S, rhs)
    for _ in range(6):
        res = rhs.astype(np.longdouble) - Sl @ y.astype(np.longdouble)
        y = (y.astype(np.longdouble) + np.linalg.solve(S, res.astype(np.float64))).astype(np.float64)
    r64 = np.linalg.norm(rhs - P.apply_S(y)) / np.linalg.norm(rhs)
    floor = 10.0 * 2.0 ** -53 * np.linalg.norm(np.abs(S) @ np.abs(y)) / np.linalg.norm(rhs)
    assert floor > 1e-13  # an ill-conditioned case: the floor is far above u
    assert floor / 100.0 <= r64 <= floor
    # the oracle's plain solve at a tight rtol reports that floor for its own y
    r = P.solve(rhs, np.full(P.N, 1e30), None, deflate=False, rtol=1e-14, max_cg=20000)
    assert r["relres_floor"][0] == pytest.approx(floor, rel=1e-6)
    assert r["true_relres_each"][0] <= 2 * floor
