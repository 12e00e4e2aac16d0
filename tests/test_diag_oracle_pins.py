"""Pins of the spectral-diagnostics oracle against what the definitions and
the mathematics fix: brute-force counts, the weighted distance collapsing to
the plain one under a complete orthonormal basis, a closed-form drift,
Cauchy interlacing (App. A.2), the closed-form spectrum for an empty active
set, rotations by known angles, and the Davis-Kahan bound (Prop. dk)."""
import numpy as np
import pytest

from oracle import diag_oracle as D
from oracle import oracle as O


def _brute_counts(ar, am):
    sym = 0
    act = 0
    for x, y in zip(ar.tolist(), am.tolist()):
        sym += int(bool(x) != bool(y))
        act += int(bool(y))
    return sym, act


def test_counts_match_brute_force_and_metric_properties():
    rng = np.random.default_rng(5)
    N = 257
    masks = [(rng.random(N) < p).astype(np.uint8) for p in (0.0, 0.1, 0.5, 0.9, 1.0)]
    for ar in masks:
        for am in masks:
            assert D.active_set_counts(ar, am) == _brute_counts(ar, am)
            assert D.delta(ar, am) == D.delta(am, ar)
    # identical sets, complementary sets, triangle inequality
    a, b, c = masks[1], masks[2], masks[3]
    assert D.delta(a, a) == 0.0
    assert D.delta(a, 1 - a) == 1.0
    assert D.delta(a, c) <= D.delta(a, b) + D.delta(b, c) + 1e-15
    assert D.rho(masks[0]) == 0.0 and D.rho(masks[4]) == 1.0
    assert D.rho(b) == np.count_nonzero(b) / N


def test_weighted_distance_is_plain_distance_for_a_complete_basis():
    # the rows of an orthogonal N x N matrix have unit norm: w_j = 1, so
    # delta_w reduces to delta
    P = O.Problem(2, 6)
    Phi, _ = O.dense_modes(P, P.N)
    rng = np.random.default_rng(2)
    ar = (rng.random(P.N) < 0.3).astype(np.uint8)
    am = (rng.random(P.N) < 0.4).astype(np.uint8)
    assert D.delta_w(ar, am, Phi, P.N) == pytest.approx(D.delta(ar, am), rel=1e-13)
    # weights concentrated off the changed nodes give zero
    Phi1 = np.zeros((P.N, 1))
    same = np.flatnonzero(ar == am)
    Phi1[same[0], 0] = 1.0
    assert D.delta_w(ar, am, Phi1, 1) == 0.0


def test_drift_of_a_rescaled_operator_matches_closed_form():
    # S_m = I + alpha c^2 A^2 against S_ref = I + alpha A^2 (A the constant-
    # coefficient Laplacian): ||S_ref - S_m|| = alpha |c^2 - 1| mu_max^2,
    # ||S_ref|| = 1 + alpha mu_max^2, mu_max = sum_d (4/h^2) sin^2(n pi / (2(n+1)))
    n, alpha, c = 12, 1e-3, 1.3
    ref = O.Problem(2, n, alpha=alpha)
    m = O.Problem(2, n, alpha=alpha, kscale=c)
    mu = 2 * 4.0 * (n + 1) ** 2 * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    eps, nref = D.drift(ref.dense_S(), m.dense_S())
    assert nref == pytest.approx(1 + alpha * mu * mu, rel=1e-12)
    assert eps == pytest.approx(alpha * abs(c * c - 1) * mu * mu / (1 + alpha * mu * mu), rel=1e-12)
    assert D.drift(ref.dense_S(), ref.dense_S())[0] == 0.0


def test_restricted_eigenvalues_interlace_and_reduce_to_closed_form():
    n, k = 10, 12
    P = O.Problem(2, n, alpha=1e-3)
    S = P.dense_S()
    lam_full = np.linalg.eigvalsh(S)
    # empty active set: the closed-form spectrum
    w0, V0 = D.restricted_modes(S, np.zeros(P.N, np.uint8), k)
    lam_cf = O.analytic_modes(2, n, k, 1e-3)[1]
    np.testing.assert_allclose(w0, np.sort(lam_cf), rtol=1e-12)
    # an active disc: Cauchy interlacing lambda_j(S) <= lambda_j(S_II) <= lambda_{j+|A|}(S)
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    gy, gx = np.meshgrid(x, x, indexing="ij")
    act = (((gx - 0.6) ** 2 + (gy - 0.4) ** 2) < 0.05).ravel().astype(np.uint8)
    nA = int(act.sum())
    assert 0 < nA < P.N - k
    w, V = D.restricted_modes(S, act, k)
    for j in range(k):
        assert lam_full[j] <= w[j] * (1 + 1e-13)
        assert w[j] <= lam_full[j + nA] * (1 + 1e-13)
    assert np.all(V[act.astype(bool)] == 0.0)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)


def test_cutoff_angles_of_known_rotations():
    t = 0.3
    e = np.eye(6)
    Phi = e[:, :3]
    V = e[:, :3].copy()
    V[:, 2] = np.cos(t) * e[:, 2] + np.sin(t) * e[:, 3]
    th = D.cutoff_angles(Phi, V)
    np.testing.assert_allclose(th, [0.0, 0.0, t], atol=1e-12)
    # swapping the order of the first two reference vectors: at r = 1 the
    # spans are orthogonal, at r = 2 they coincide
    th2 = D.cutoff_angles(Phi[:, [1, 0, 2]], e[:, :3])
    np.testing.assert_allclose(th2, [np.pi / 2, 0.0, 0.0], atol=1e-12)


def test_exact_modes_have_zero_angles_at_clean_cuts():
    # n = 10 square grid: eigenvalue groups of size 1, 2, 1, 2, ... ; cuts at
    # r = 1, 3, 4, 6 do not split a group, and there the closed-form modes span
    # the restricted (here: full) invariant subspace exactly
    n, k = 10, 6
    P = O.Problem(2, n, alpha=1e-3)
    Phi = O.analytic_modes(2, n, k, 1e-3)[0]
    _, V = D.restricted_modes(P.dense_S(), np.zeros(P.N, np.uint8), k)
    th = D.cutoff_angles(Phi, V)
    for r in (1, 3, 4, 6):
        assert th[r - 1] < 1e-7, (r, th)


def test_davis_kahan_bound_holds_under_convection_drift():
    # full-domain operators (A = empty): sin theta_r <= ||S_ref - S_m|| / gap_r
    n, k = 12, 8
    ref = O.Problem(2, n, alpha=1e-3, diff_scale=1e-2, b=(0.0, 0.0))
    Sref = ref.dense_S()
    lam = np.linalg.eigvalsh(Sref)
    _, Vref = D.restricted_modes(Sref, np.zeros(ref.N, np.uint8), k)
    for th in (0.4, 2.0):
        m = O.Problem(2, n, alpha=1e-3, diff_scale=1e-2, b=(np.cos(th), np.sin(th)))
        Sm = m.dense_S()
        eps, nref = D.drift(Sref, Sm)
        assert eps > 0
        _, Vm = D.restricted_modes(Sm, np.zeros(m.N, np.uint8), k)
        ang = D.cutoff_angles(Vref, Vm)
        for r in range(1, k + 1):
            gap = lam[r] - lam[r - 1]
            if gap > 1e-9 * nref:
                assert np.sin(ang[r - 1]) <= eps * nref / gap * (1 + 1e-9), (th, r)


def test_sorted_principal_angles_of_known_rotations_and_their_largest_is_the_nested_last():
    e = np.eye(7)
    Phi = e[:, :3]
    t1, t2 = 0.2, 1.1
    V = np.column_stack([e[:, 0],
                         np.cos(t1) * e[:, 1] + np.sin(t1) * e[:, 4],
                         np.cos(t2) * e[:, 2] + np.sin(t2) * e[:, 5]])
    np.testing.assert_allclose(D.principal_angles(Phi, V), [0.0, t1, t2], atol=1e-12)
    # the span of a reordered basis is the same set of angles
    np.testing.assert_allclose(D.principal_angles(Phi[:, ::-1], V[:, [2, 0, 1]]), [0.0, t1, t2],
                               atol=1e-12)
    # the largest principal angle between the full spans is the nested angle at r = k
    rng = np.random.default_rng(8)
    A, B = rng.standard_normal((30, 6)), rng.standard_normal((30, 6))
    assert D.principal_angles(A, B)[-1] == pytest.approx(D.cutoff_angles(A, B)[-1], abs=1e-12)
