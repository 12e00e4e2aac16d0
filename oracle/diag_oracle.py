"""Plain FP64 oracle of the spectral diagnostics (numpy / scipy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py import this module.  It shares
no code with the CUDA path.

App. A.1 (sources of spectral variation), Sec. 4.1 and App. D (spectral
coherence diagnostics), each written out from its definition:

* Eq. delta: the active-set distance delta_m = |A_ref sym-diff A_m| / N.
* Eq. rho: the active fraction rho_m = |A_m| / N.
* The eigenmode-weighted distance delta_w (App. D.6):
  sum_j w_j |A_ref(j) - A_m(j)| / sum_j w_j with w_j = sum_{q<r} phi_q(j)^2.
* Eq. epsilon: the operator drift eps_m = ||M_ref - M_m||_2 / ||M_ref||_2 of
  the full-domain Schur complements (dense 2-norms).
* The restricted eigenpairs: the k smallest eigenpairs of M_II (dense eigh),
  the eigenvectors embedded in the full grid with zeros on A.
* Principal angles, two readings.  The paper's reported theta_r (Sec. 4.1,
  App. D: "the principal angle at the deflation cutoff", angles "stratified
  by mode quintile") is the r-th smallest principal angle between the
  K-dimensional spans of the restricted reference modes Phi_I and of the K
  lowest eigenvectors of M_II; theta_max is the largest.  The nested
  quantity of Prop. dk (App. A.3) with S = {1..r} is the largest principal
  angle between span(Phi_I[:, :r]) and span(V[:, :r]).  The first reading
  reproduces the paper's two-regime numbers; both are reported.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import subspace_angles


def active_set_counts(active_ref, active):
    """Eq. delta and Eq. rho numerators: (|A_ref sym-diff A_m|, |A_m|)."""
    ar = np.asarray(active_ref).astype(bool)
    am = np.asarray(active).astype(bool)
    return int(np.count_nonzero(ar != am)), int(np.count_nonzero(am))


def delta(active_ref, active):
    """Eq. delta: normalised Hamming distance of the two active sets."""
    return active_set_counts(active_ref, active)[0] / np.asarray(active).size


def rho(active):
    """Eq. rho: the active fraction."""
    a = np.asarray(active).astype(bool)
    return np.count_nonzero(a) / a.size


def mode_weights(Phi, r):
    """w_j = sum over the first r reference modes of phi_q(j)^2."""
    P = np.asarray(Phi, np.float64)[:, :r]
    return np.sum(P * P, axis=1)


def delta_w(active_ref, active, Phi, r):
    """Eigenmode-weighted active-set distance."""
    w = mode_weights(Phi, r)
    d = (np.asarray(active_ref).astype(bool) != np.asarray(active).astype(bool))
    return float(np.sum(w * d) / np.sum(w))


def drift(S_ref, S_m):
    """Eq. epsilon: ||S_ref - S_m||_2 / ||S_ref||_2 (dense 2-norms) and
    ||S_ref||_2."""
    S_ref = np.asarray(S_ref, np.float64)
    nref = np.linalg.norm(S_ref, 2)
    return float(np.linalg.norm(S_ref - np.asarray(S_m, np.float64), 2) / nref), float(nref)


def restricted_modes(S, active, k):
    """The k smallest eigenpairs of S_II (dense eigh): eigenvalues ascending
    and eigenvectors embedded in the full grid (zeros on A), each signed so
    that its entry of largest magnitude is positive."""
    idx = np.flatnonzero(np.asarray(active) == 0)
    w, V = np.linalg.eigh(np.asarray(S)[np.ix_(idx, idx)])
    V = V[:, :k]
    piv = np.argmax(np.abs(V), axis=0)
    V = V * np.sign(V[piv, np.arange(V.shape[1])])
    Vf = np.zeros((np.asarray(S).shape[0], V.shape[1]))
    Vf[idx] = V
    return w[:k], np.asfortranarray(Vf)


def restrict(Phi, active):
    """Phi_I: the reference modes with their rows on A set to zero."""
    P = np.array(Phi, np.float64, copy=True)
    P[np.asarray(active).astype(bool)] = 0.0
    return P


def principal_angles(Phi_I, V):
    """The principal angles (radians, ascending) between span(Phi_I) and
    span(V): theta_r of the paper's diagnostics is entry r - 1."""
    return np.sort(subspace_angles(np.asarray(Phi_I, np.float64), np.asarray(V, np.float64)))


def cutoff_angles(Phi_I, V, k=None):
    """theta_r for r = 1..k (radians): the largest principal angle between
    span(Phi_I[:, :r]) and span(V[:, :r])."""
    k = min(Phi_I.shape[1], V.shape[1]) if k is None else k
    return np.array([float(np.max(subspace_angles(Phi_I[:, :r], V[:, :r])))
                     for r in range(1, k + 1)])
