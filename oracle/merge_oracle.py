"""Plain FP64 oracle of the conditioning-based safe merge (numpy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py import this module.  It shares
no code with the CUDA path.

Sec. 2.2.5, Algorithm safe, followed step by step in the restricted space:
  Z <- orth(Phi_eig restricted to I); E <- Z^T S_II Z;
  for each POD candidate in order: orthogonalise it against Z (twice); if its
  norm is below tau_dep skip it; normalise; if cond(Z_trial^T S_II Z_trial) >
  tau_safe stop; else accept.
Reading: "orthogonalise" is classical Gram-Schmidt applied twice; cond is the
ratio of the extreme eigenvalues of the symmetric E_trial.
"""
from __future__ import annotations

import numpy as np


def safe_merge(S_II, Phi_eig_I, Phi_pod_I, tau_safe=1e4, tau_dep=1e-10):
    """Returns Z (n_I x k', orthonormal) and the number of accepted POD modes."""
    Z, _ = np.linalg.qr(np.asarray(Phi_eig_I, np.float64))
    accepted = 0
    for j in range(Phi_pod_I.shape[1]):
        z = np.array(Phi_pod_I[:, j], np.float64)
        for _ in range(2):
            z -= Z @ (Z.T @ z)
        nz = np.linalg.norm(z)
        if nz < tau_dep:
            continue
        z /= nz
        Zt = np.column_stack([Z, z])
        Et = Zt.T @ (S_II @ Zt)
        ev = np.linalg.eigvalsh(0.5 * (Et + Et.T))
        if ev[-1] / ev[0] > tau_safe or ev[0] <= 0:
            break
        Z = Zt
        accepted += 1
    return Z, accepted


def restricted(prob, active):
    """Dense S_II and the index list of I (small problems only)."""
    S = prob.dense_S()
    idx = np.flatnonzero(np.asarray(active) == 0)
    return S[np.ix_(idx, idx)], idx


def to_full(Z_I, idx, N):
    """Full-grid columns (zero on the active set) of a restricted basis."""
    Z = np.zeros((N, Z_I.shape[1]))
    Z[idx] = Z_I
    return np.asfortranarray(Z)
