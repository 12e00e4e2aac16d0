"""Pins of the safe-merge oracle (oracle/merge_oracle.py, Algorithm safe)
built from exact eigenvectors of S_II, where every outcome is known: a
dependent candidate is skipped, an ill-conditioning candidate stops the merge
(later candidates are not considered), and the merged basis is orthonormal
with E = diag of the chosen eigenvalues."""
import numpy as np

from oracle import merge_oracle as M
from oracle import oracle as O


def _setup():
    P = O.Problem(2, (16, 14), alpha=1e-4)
    act = np.zeros(P.N, np.uint8)
    act[:20] = 1   # a small active set: S_II is a proper submatrix
    S_II, idx = M.restricted(P, act)
    lam, V = np.linalg.eigh(S_II)
    return P, act, S_II, idx, lam, V


def test_dependent_candidates_are_skipped():
    _, _, S_II, _, lam, V = _setup()
    eig = V[:, :4]
    pod = np.column_stack([eig[:, 1] + eig[:, 2], eig[:, 0]])
    Z, acc = M.safe_merge(S_II, eig, pod)
    assert acc == 0 and Z.shape[1] == 4


def test_ill_conditioning_stops_the_merge():
    _, _, S_II, _, lam, V = _setup()
    eig = V[:, :4]
    # candidate 1: the 5th mode (kept), candidate 2: the top mode
    # (cond = lam_max / lam_0 > tau_safe: stop), candidate 3: the 6th mode
    # (fine on its own, but never considered after the stop)
    pod = np.column_stack([V[:, 4], V[:, -1], V[:, 5]])
    tau = 0.5 * (lam[4] / lam[0] + lam[-1] / lam[0])
    assert lam[5] / lam[0] < tau < lam[-1] / lam[0]
    Z, acc = M.safe_merge(S_II, eig, pod, tau_safe=tau)
    assert acc == 1 and Z.shape[1] == 5
    np.testing.assert_allclose(Z.T @ Z, np.eye(5), atol=1e-12)
    E = Z.T @ S_II @ Z
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(E)), lam[:5], rtol=1e-10)


def test_merged_basis_keeps_the_solution():
    P, act, S_II, idx, lam, V = _setup()
    eig = V[:, :6]
    rng = np.random.default_rng(3)
    pod = np.linalg.qr(V[:, 6:12] + 0.05 * rng.standard_normal((len(idx), 6)))[0]
    Z, acc = M.safe_merge(S_II, eig, pod)
    assert acc >= 1
    _, rhs = P.desired_state(2.0, (0.5, 0.45), 0.1)
    psi = np.full(P.N, 10.0)
    ref = P.inner_solve(act, rhs, psi, M.to_full(eig, idx, P.N))
    mer = P.inner_solve(act, rhs, psi, M.to_full(Z, idx, P.N))
    np.testing.assert_allclose(mer["x"], ref["x"], rtol=0, atol=1e-6 * np.abs(ref["x"]).max())
