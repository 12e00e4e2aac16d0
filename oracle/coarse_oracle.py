"""Plain FP64 oracle of the coarse-grid reference basis (numpy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py import this module.  It shares
no code with the CUDA path.

Algorithm (coarse), Sec. 2.2.7 "Coarse-grid eigenmode prolongation":
  1. coarse grid of n_c = floor(n / c) interior nodes per direction;
  2. the r_pool smallest eigenpairs of the coarse S_c (= those of the coarse A_c);
  3. prolongation of each coarse eigenvector by P = P_1D (x) ... (x) P_1D,
     P_1D the 1D linear interpolation from coarse to fine interior nodes
     (Eq. prolong), the boundary values being zero;
  4. economy QR of the prolongated block, columns with |R_jj| < tau_sv
     discarded; the basis is the remaining columns of Q.

Readings (the paper is silent on them):
  * the coarse kappa is the fine kappa injected at the fine node nearest to
    each coarse node, i_f = round(x_c (n + 1)) - 1 per direction;
  * the QR is Gram-Schmidt column by column (each column orthogonalised twice
    against the kept ones), R_jj > 0; a column whose remaining norm R_jj is
    below tau_sv times the largest column norm is discarded and takes no
    part in later columns.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def p1d(n: int, nc: int) -> np.ndarray:
    """1D prolongation (n x nc): fine interior node i at x = (i+1)/(n+1) takes
    the linear interpolant of the coarse values at x_c = (j+1)/(nc+1), with
    zero at x = 0 and x = 1."""
    P = np.zeros((n, nc))
    for i in range(n):
        t = (i + 1) / (n + 1) * (nc + 1) - 1.0   # coarse index coordinate
        j0 = int(np.floor(t))
        w = t - j0
        if 0 <= j0 < nc:
            P[i, j0] += 1.0 - w
        if 0 <= j0 + 1 < nc:
            P[i, j0 + 1] += w
    return P


def prolongation(n, nc) -> np.ndarray:
    """P = P_1D (x) ... (x) P_1D for lexicographic ordering with x fastest."""
    P = p1d(n[0], nc[0])
    for d in range(1, len(n)):
        P = np.kron(p1d(n[d], nc[d]), P)
    return P


def coarse_kappa(kappa, n, nc):
    """Injection of the node kappa to the coarse nodes."""
    if kappa is None:
        return None
    kap = np.asarray(kappa, np.float64).reshape(tuple(reversed(n)))
    idx = [np.clip(np.rint((np.arange(m) + 1) / (m + 1) * (nf + 1)).astype(int) - 1, 0, nf - 1)
           for m, nf in zip(nc, n)]
    if len(n) == 2:
        out = kap[np.ix_(idx[1], idx[0])]
    else:
        out = kap[np.ix_(idx[2], idx[1], idx[0])]
    return np.ascontiguousarray(out).ravel()


def coarse_modes(dim, n, c, r_pool, kappa=None, alpha=1e-4, diff_scale=1.0, tau_sv=1e-8):
    """The coarse-grid candidate basis (N x r', r' <= r_pool) and the coarse
    eigenvalues of S_c."""
    n = tuple(n)
    nc = tuple(m // c for m in n)
    Pc = O.Problem(dim, nc, kappa=coarse_kappa(kappa, n, nc), alpha=alpha, diff_scale=diff_scale)
    Phic, lam = O.dense_modes(Pc, r_pool)
    Pt = prolongation(n, nc) @ Phic
    return qr_discard(Pt, tau_sv), lam


def qr_discard(A, tau_sv):
    """Gram-Schmidt QR (twice per column) keeping the columns with R_jj >=
    tau_sv * max_j ||a_j||."""
    scale = np.linalg.norm(A, axis=0).max()
    qs = []
    for j in range(A.shape[1]):
        v = A[:, j].copy()
        for _ in range(2):
            for q in qs:
                v -= q * (q @ v)
        r = np.linalg.norm(v)
        if r >= tau_sv * scale:
            qs.append(v / r)
    return np.stack(qs, axis=1)
