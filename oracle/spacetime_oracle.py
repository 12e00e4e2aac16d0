"""Plain FP64 oracle of the space-time extension (numpy / scipy.sparse).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py import this module.  It shares
no code with the CUDA path.

App. E.2 and App. F.5 (space-time), written out from their definitions:

* State equation y_t - div(kappa grad y) = u on (0, T], y(., 0) = 0, with
  implicit Euler on n_t steps of dt = T / n_t:
  (y^l - y^(l-1)) / dt + A y^l = u^l for l = 1..n_t.  All at once, F y = u
  with F block lower bidiagonal: I/dt + A on the diagonal, -I/dt below it.
* Reduced problem (u = F y, as u = A y in the steady case):
  S_st = mass I + (alpha / mass) F^T F, block tridiagonal and SPD.
* Desired state with a temporal ramp (App. F.5):
  y_d(x, t_l) = (1 - exp(-t_l / tau)) a exp(-|x - c|^2 / (2 sigma^2)) at the
  interior nodes x_j = (j + 1) h and t_l = l dt, l = 1..n_t; rhs = mass y_d.
* Deflation bases (App. E.2.1): the Kronecker expansion
  Z_st = I_{n_t} (x) Z_s (Eq. kron_basis), the cosine basis W_t (x) Z_s with
  W_t the first r_t columns of the orthonormal DCT-II matrix, and the
  constant-in-time lift 1_{n_t} (x) Z_s / sqrt(n_t).
* The primal active-set loop and A-DEF2 are the C oracle's (the same
  algorithm as the steady problem), run on S_st given as CSR.

Node order: x fastest, then y, then the time step, so that time step l is
the contiguous slab [l N_s, (l + 1) N_s).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (sp.linalg.spsolve)

from oracle import oracle as O


def laplacian_2d(n, diff_scale=1.0):
    """A = diff_scale (-Laplace) on the n x n interior grid of the unit
    square, 5-point, zero Dirichlet values: kron(I, T) + kron(T, I) with
    T = tridiag(-1, 2, -1) / h^2, h = 1 / (n + 1)."""
    h = 1.0 / (n + 1)
    T = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2
    I = sp.identity(n)
    return (diff_scale * (sp.kron(I, T) + sp.kron(T, I))).tocsr()


def forward_operator(A_s, n_t, T=1.0):
    """F: block lower bidiagonal, I/dt + A_s on the diagonal, -I/dt below."""
    dt = T / n_t
    Ns = A_s.shape[0]
    I_s = sp.identity(Ns)
    sub = sp.diags([np.ones(n_t - 1)], [-1], shape=(n_t, n_t))
    return (sp.kron(sp.identity(n_t), I_s / dt + A_s) - sp.kron(sub, I_s / dt)).tocsr()


def schur(F, alpha, mass=1.0):
    """S_st = mass I + (alpha / mass) F^T F."""
    return (mass * sp.identity(F.shape[0]) + (alpha / mass) * (F.T @ F)).tocsr()


def time_steps(u, A_s, n_t, T=1.0):
    """The implicit Euler sweep: y^l = (I/dt + A_s)^-1 (u^l + y^(l-1) / dt),
    y^0 = 0, one sparse direct solve per step (the time-stepping definition
    that F encodes)."""
    dt = T / n_t
    Ns = A_s.shape[0]
    M = (sp.identity(Ns) / dt + A_s).tocsc()
    y = np.zeros(Ns * n_t)
    prev = np.zeros(Ns)
    for l in range(n_t):
        prev = sp.linalg.spsolve(M, u[l * Ns:(l + 1) * Ns] + prev / dt)
        y[l * Ns:(l + 1) * Ns] = prev
    return y


def desired_state(n, n_t, a, c, sigma=0.12, tau=0.2, T=1.0, mass=1.0):
    """(y_d, rhs) on the space-time grid (x fastest, then y, then t)."""
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    gy, gx = np.meshgrid(x, x, indexing="ij")
    g = a * np.exp(-((gx - c[0]) ** 2 + (gy - c[1]) ** 2) / (2.0 * sigma**2)).ravel()
    t = (np.arange(n_t) + 1) * (T / n_t)
    yd = np.concatenate([(1.0 - np.exp(-tl / tau)) * g for tl in t])
    return yd, mass * yd


def kron_basis(Z_s, n_t):
    """Z_st = I_{n_t} (x) Z_s (Eq. kron_basis): column l r + j is spatial
    mode j on time step l."""
    return np.asfortranarray(np.kron(np.identity(n_t), np.asarray(Z_s, np.float64)))


def dct2_basis(n_t, r_t):
    """The first r_t orthonormal DCT-II basis vectors of length n_t (columns):
    W[l, a] = sqrt((2 - [a = 0]) / n_t) cos(pi (l + 1/2) a / n_t)."""
    l = np.arange(n_t)[:, None] + 0.5
    a = np.arange(r_t)[None, :]
    return np.sqrt(np.where(a == 0, 1.0, 2.0) / n_t) * np.cos(np.pi * l * a / n_t)


def temporal_basis(W_t, Z_s):
    """W_t (x) Z_s: column a r + j is spatial mode j weighted by W_t[l, a] on
    time step l (the Kronecker basis is W_t = I, the cosine basis the DCT-II)."""
    return np.asfortranarray(np.kron(np.asarray(W_t, np.float64), np.asarray(Z_s, np.float64)))


def constant_lift(Z_s, n_t):
    """1_{n_t} (x) Z_s / sqrt(n_t): each spatial mode constant in time."""
    return np.asfortranarray(np.kron(np.ones((n_t, 1)) / np.sqrt(n_t), np.asarray(Z_s, np.float64)))


def problem(n, n_t, alpha=1e-4, diff_scale=1.0, T=1.0, mass=1.0):
    """The oracle problem handle of S_st (the C oracle's solves on its CSR)
    and S_st itself."""
    S = schur(forward_operator(laplacian_2d(n, diff_scale), n_t, T), alpha, mass)
    return O.Problem.from_csr(S), S
