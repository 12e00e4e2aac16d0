"""Plain FP64 CPU oracle of the online-spectral-deflation active-set solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this module.
It shares no code with the CUDA path (``paper_2606_17971_b300``); the only
module both sides use is the seeded input generator
``paper_2606_17971_b300.workloads``, which holds none of the method's
arithmetic.

What lives here:
  * ``Problem``: ctypes wrapper of ``sdf_oracle.c`` -- CSR assembly of
    S = M + alpha K^T M^-1 K (Sec. 2.1.2 Eq. schur; App. A; App. B.3), the
    desired state, the primal active-set loop (App. B.1 Algorithm pdas), plain
    Jacobi-PCG (App. B.2) and A-DEF2 (Sec. 2.2.1 Algorithm adef2 in the cited
    standard form).
  * ``analytic_modes``: closed-form Kronecker sine eigenmodes of
    alpha L^2 + I on a tensor grid (Sec. 2.2.8).
  * ``dense_modes``: the k smallest eigenpairs of a (small) S by a dense
    symmetric eigensolver (Sec. 2.2.2 Eq. eig, with LAPACK in place of ARPACK).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsdf_oracle.so")

MAX_OUTER = 64

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOMEM", 5: "CG_MAXIT", 6: "OUTER_MAXIT",
          7: "BREAKDOWN", 8: "NONFINITE"}


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("outer_iters", ctypes.c_int32),
        ("cg_iters", ctypes.c_int32 * MAX_OUTER),
        ("n_active", ctypes.c_int32 * MAX_OUTER),
        ("fallback", ctypes.c_int32 * MAX_OUTER),
        ("cond_E", ctypes.c_double * MAX_OUTER),
        ("relres", ctypes.c_double * MAX_OUTER),
        ("true_relres", ctypes.c_double),
        ("min_margin", ctypes.c_double),
        ("min_lambda_active", ctypes.c_double),
        ("true_relres_each", ctypes.c_double * MAX_OUTER),
        ("relres_floor", ctypes.c_double * MAX_OUTER),
    ]


class Opts(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("tau_cond", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("max_cg", ctypes.c_int32),
        ("deflate", ctypes.c_int32),
        ("rule", ctypes.c_int32),
        ("pdas_c", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile sdf_oracle.c into oracle/_build/libsdf_oracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        up = ctypes.POINTER(ctypes.c_ubyte)
        _lib.orc_create.restype = P
        _lib.orc_create.argtypes = [ctypes.c_int] * 4 + [dp, ctypes.c_double, dp,
                                                          ctypes.c_double, ctypes.c_double,
                                                          ctypes.c_double]
        _lib.orc_create_csr.restype = P
        _lib.orc_create_csr.argtypes = [ctypes.c_int, ip, ip, dp]
        _lib.orc_destroy.argtypes = [P]
        for f in ("orc_size", "orc_nnz_A", "orc_nnz_S"):
            getattr(_lib, f).argtypes = [P]
            getattr(_lib, f).restype = ctypes.c_int
        _lib.orc_get_A.argtypes = [P, ip, ip, dp]
        _lib.orc_get_S.argtypes = [P, ip, ip, dp]
        _lib.orc_apply_S.argtypes = [P, dp, dp]
        _lib.orc_apply_S_rows.argtypes = [P, dp, ip, ctypes.c_int, dp]
        _lib.orc_desired_state.argtypes = [P, ctypes.c_double, dp, ctypes.c_double, dp, dp]
        _lib.orc_inner_solve.restype = ctypes.c_int
        _lib.orc_inner_solve.argtypes = [P, up, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, dp, ip, dp, dp, ip]
        _lib.orc_last_timing.argtypes = [dp, dp]
        _lib.orc_last_residuals.argtypes = [dp, dp]
        _lib.orc_solve.restype = ctypes.c_int
        _lib.orc_solve.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(Opts), dp, dp, dp, up,
                                   ctypes.POINTER(Stats)]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """S = mass*I + alpha*kscale^2/mass * A^T A on an interior tensor grid.

    A = diff_scale * (-div(kappa grad)) [5/7-point, harmonic faces] plus
    first-order upwind convection with velocity ``b`` (App. A; the upwind
    scheme is the convection-diffusion workload's choice).  ``kappa`` holds node
    values in x-fastest order or is None (kappa = 1)."""

    def __init__(self, dim, n, kappa=None, diff_scale=1.0, b=None, kscale=1.0,
                 mass=1.0, alpha=1e-4):
        L = lib()
        n = list(n) if hasattr(n, "__len__") else [n] * dim
        while len(n) < 3:
            n.append(1)
        self.dim, self.n = dim, tuple(n[:dim])
        self.kappa = _f64(kappa)
        self.b = _f64(b)
        self.mass, self.alpha, self.kscale = mass, alpha, kscale
        self._h = L.orc_create(dim, n[0], n[1], n[2], _dp(self.kappa), diff_scale,
                               _dp(self.b), kscale, mass, alpha)
        if not self._h:
            raise ValueError("orc_create failed")
        self.N = L.orc_size(self._h)

    @classmethod
    def from_csr(cls, S):
        """A problem given by its Schur complement S (scipy.sparse, N x N;
        copied), for operators assembled outside the C file: the solves and
        the S products only (no grid, no A, no desired state)."""
        S = S.tocsr()
        S.sort_indices()
        rp = np.ascontiguousarray(S.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(S.indices, dtype=np.int32)
        v = np.ascontiguousarray(S.data, dtype=np.float64)
        self = cls.__new__(cls)
        self._h = lib().orc_create_csr(S.shape[0], _ip(rp), _ip(ci), _dp(v))
        if not self._h:
            raise ValueError("orc_create_csr failed")
        self.dim, self.n, self.N = 1, (S.shape[0],), S.shape[0]
        self.kappa = self.b = None
        self.mass, self.alpha, self.kscale = 1.0, None, 1.0
        return self

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def _csr(self, which):
        L = lib()
        nnz = (L.orc_nnz_A if which == "A" else L.orc_nnz_S)(self._h)
        rp = np.zeros(self.N + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz, np.float64)
        (L.orc_get_A if which == "A" else L.orc_get_S)(self._h, _ip(rp), _ip(ci), _dp(v))
        return rp, ci, v

    def csr_A(self):
        return self._csr("A")

    def csr_S(self):
        return self._csr("S")

    def dense_S(self):
        rp, ci, v = self.csr_S()
        S = np.zeros((self.N, self.N))
        S[np.repeat(np.arange(self.N), np.diff(rp)), ci] = v
        return S

    def apply_S(self, x):
        x = _f64(x)
        y = np.empty(self.N)
        lib().orc_apply_S(self._h, _dp(x), _dp(y))
        return y

    def apply_S_rows(self, x, rows):
        x = _f64(x)
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty(len(rows))
        lib().orc_apply_S_rows(self._h, _dp(x), _ip(rows), len(rows), _dp(out))
        return out

    def desired_state(self, a, c, sigma):
        c = _f64(np.asarray(c, dtype=np.float64).reshape(-1))
        yd = np.empty(self.N)
        rhs = np.empty(self.N)
        lib().orc_desired_state(self._h, float(a), _dp(c), float(sigma), _dp(yd), _dp(rhs))
        return yd, rhs

    @staticmethod
    def set_ritz(r: int):
        """Ritz re-selection (Sec. 2.2.3) in every later A-DEF2 solve: the r
        smallest Ritz vectors of the restricted pool (0: off)."""
        lib().orc_set_ritz(int(r))

    def inner_solve(self, active, rhs, psi, Phi=None, deflate=True, rtol=1e-8,
                    maxit=100000, tau_cond=1e10, x0=None):
        """Solve S_II x_I = rhs_I - S_IA psi_A on the given active set."""
        active = np.ascontiguousarray(active, dtype=np.uint8)
        rhs, psi = _f64(rhs), _f64(psi)
        x = np.zeros(self.N) if x0 is None else _f64(x0).copy()
        k, ld, ph = 0, self.N, None
        if Phi is not None:
            ph = np.asfortranarray(Phi, dtype=np.float64)
            k, ld = ph.shape[1], ph.shape[0]
        it = ctypes.c_int(0)
        fb = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        ce = ctypes.c_double(0)
        st = lib().orc_inner_solve(self._h, _up(active), _dp(rhs), _dp(psi),
                                   _dp(ph) if ph is not None else None, k, ld,
                                   int(bool(deflate and k > 0)), rtol, maxit, tau_cond,
                                   _dp(x), ctypes.byref(it), ctypes.byref(rr),
                                   ctypes.byref(ce), ctypes.byref(fb))
        ts, tl = ctypes.c_double(0), ctypes.c_double(0)
        lib().orc_last_timing(ctypes.byref(ts), ctypes.byref(tl))
        tr, fl = ctypes.c_double(0), ctypes.c_double(0)
        lib().orc_last_residuals(ctypes.byref(tr), ctypes.byref(fl))
        return dict(x=x, status=st, iters=it.value, relres=rr.value, cond_E=ce.value,
                    fallback=fb.value, t_setup=ts.value, t_loop=tl.value,
                    true_relres=tr.value, relres_floor=fl.value)

    def solve(self, rhs, psi, Phi=None, deflate=True, rtol=1e-8, tau=1e-10,
              tau_cond=1e10, max_outer=30, max_cg=100000, rule=0, pdas_c=1.0,
              x0=None):
        """Primal active-set loop (App. B.1) with the inner solve of
        Algorithm online_deflation (A-DEF2 or plain Jacobi-PCG)."""
        rhs, psi = _f64(rhs), _f64(psi)
        k, ld, ph = 0, self.N, None
        if Phi is not None:
            ph = np.asfortranarray(Phi, dtype=np.float64)
            k, ld = ph.shape[1], ph.shape[0]
        o = Opts(rtol=rtol, tau=tau, tau_cond=tau_cond, max_outer=max_outer,
                 max_cg=max_cg, deflate=int(bool(deflate and k > 0)), rule=rule,
                 pdas_c=pdas_c)
        y = np.empty(self.N)
        lam = np.empty(self.N)
        act = np.empty(self.N, np.uint8)
        st = Stats()
        x0a = _f64(x0)
        lib().orc_solve(self._h, _dp(rhs), _dp(psi), _dp(ph) if ph is not None else None,
                        k, ld, ctypes.byref(o), _dp(x0a), _dp(y), _dp(lam), _up(act),
                        ctypes.byref(st))
        no = st.outer_iters
        return dict(
            y=y, lam=lam, active=act.astype(bool), status=st.status,
            outer_iters=no, cg_iters=list(st.cg_iters[:no]),
            n_active=list(st.n_active[:no]), fallback=list(st.fallback[:no]),
            cond_E=list(st.cond_E[:no]), relres=list(st.relres[:no]),
            true_relres=st.true_relres, min_margin=st.min_margin,
            min_lambda_active=st.min_lambda_active,
            true_relres_each=list(st.true_relres_each[:no]),
            relres_floor=list(st.relres_floor[:no]))


def analytic_modes(dim, n, k, alpha=1e-4, diff_scale=1.0):
    """The k smallest eigenpairs of S_ref = alpha (diff_scale L_h)^2 + I on an
    n^dim interior grid (Sec. 2.2.8, with the node index in place of x_l):

        phi_{i_1..i_d}(j_1..j_d) = prod_l sqrt(2/(n+1)) sin(i_l pi j_l / (n+1)),
        lambda = alpha (diff_scale sum_l mu_{i_l})^2 + 1,
        mu_q = (4/h^2) sin^2(q pi / (2(n+1))),  h = 1/(n+1).

    Ties in lambda are broken lexicographically by (i_d, ..., i_1) so that a
    degenerate group cut by k is cut reproducibly.  Returns (Phi[N, k]
    column-major in x-fastest node order, lambda[k])."""
    h = 1.0 / (n + 1)
    q = np.arange(1, n + 1)
    mu = (4.0 / h**2) * np.sin(q * np.pi / (2.0 * (n + 1))) ** 2
    # enumerate candidate multi-indices with small sums (enough for k modes)
    m = min(n, int(np.ceil((4.0 * k) ** (1.0 / dim))) + 4)
    grids = np.meshgrid(*([np.arange(m)] * dim), indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)  # columns: i_1..i_d (0-based)
    # summing the sorted per-direction values makes permuted multi-indices
    # produce bit-identical sums, so exact ties stay ties
    lam_sum = np.sort(mu[idx], axis=1).sum(axis=1)
    keys = [idx[:, d] for d in range(dim)] + [lam_sum]  # lexsort: last key primary
    order = np.lexsort(keys)[:k]
    sel = idx[order]
    j = np.arange(1, n + 1)
    s1 = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, q[:m]) * np.pi / (n + 1))  # [j, i]
    Phi = np.empty((n**dim, k))
    for c, ii in enumerate(sel):
        v = s1[:, ii[0]]
        for d in range(1, dim):
            v = np.multiply.outer(s1[:, ii[d]], v)  # slower index outermost
        Phi[:, c] = v.reshape(-1)
    lam = alpha * (diff_scale * lam_sum[order]) ** 2 + 1.0
    return np.asfortranarray(Phi), lam, sel + 1


def schur_from_operator(K, alpha=1e-4, mass=1.0, kscale=1.0):
    """S = mass I + (alpha kscale^2 / mass) K^T K for a state operator K
    given as a scipy.sparse matrix (Sec. 2.1.2 Eq. schur with M = mass I),
    as a CSR matrix: the operator of a problem given without a grid."""
    import scipy.sparse as sp
    K = sp.csr_matrix(K, dtype=np.float64)
    n = K.shape[0]
    return (mass * sp.identity(n) + (alpha * kscale * kscale / mass) * (K.T @ K)).tocsr()


def dense_modes(prob: Problem, k: int):
    """k smallest eigenpairs of the full S (Eq. eig) by a dense symmetric
    eigensolver; for small N only.  Signs are fixed so that the entry of
    largest magnitude of each mode is positive."""
    S = prob.dense_S()
    w, V = np.linalg.eigh(S)
    V = V[:, :k]
    piv = np.argmax(np.abs(V), axis=0)
    V = V * np.sign(V[piv, np.arange(k)])
    return np.asfortranarray(V), w[:k]
