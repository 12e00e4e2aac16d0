"""Python binding of the C ABI in include/sdf.h (argument marshalling only).

Every step of the solve runs in the CUDA library libsdf_b300.so; PyTorch only
provides device memory (tensors whose data pointers are passed through) and
the current CUDA stream.  Importing this module raises if the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsdf_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2606_17971_b300.build` "
                      "(the solver has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

SDF_MAX_K = 128
SDF_MAX_OUTER = 32
F64, F32, BF16 = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "WORKSPACE", 3: "CUDA", 4: "NOT_SPD", 5: "CG_MAXIT",
          6: "OUTER_MAXIT", 7: "BREAKDOWN", 8: "NONFINITE", 9: "TIMEOUT", 10: "UNSUPPORTED"}
_TORCH_DTYPE = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("alpha", ctypes.c_double),
                ("mass", ctypes.c_double), ("kscale", ctypes.c_double),
                ("diff_scale", ctypes.c_double), ("has_kappa", ctypes.c_int32),
                ("convection", ctypes.c_int32), ("yd_sigma", ctypes.c_double),
                ("time_axis", ctypes.c_int32), ("t_final", ctypes.c_double),
                ("ramp_tau", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("tau", ctypes.c_double), ("tau_cond", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("max_cg", ctypes.c_int32),
                ("deflate", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("max_blocks", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("replace_every", ctypes.c_int32),
                ("max_launches", ctypes.c_int64), ("ritz_r", ctypes.c_int32),
                ("safe_r", ctypes.c_int32), ("tau_safe", ctypes.c_double),
                ("tau_dep", ctypes.c_double), ("floor_c", ctypes.c_double),
                ("column_depth", ctypes.c_int32), ("column_pairs", ctypes.c_int32),
                ("graph", ctypes.c_int32)]


SDF_NPROF = 9
PROFILE_NAMES = ("expand", "spmv", "update", "setup", "coarse", "active", "lambda", "resid",
                 "project")
PREC_F64, PREC_MIXED = 0, 1


class EigOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("degree", ctypes.c_int32), ("guard", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class EigStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("max_rel_resid", ctypes.c_double), ("matvecs", ctypes.c_int64),
                ("seconds", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * SDF_NPROF), ("samples", ctypes.c_int64 * SDF_NPROF),
                ("launches", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32 * SDF_MAX_OUTER),
                ("n_active", ctypes.c_int32 * SDF_MAX_OUTER),
                ("fallback", ctypes.c_int32 * SDF_MAX_OUTER),
                ("floor_stop", ctypes.c_int32 * SDF_MAX_OUTER),
                ("cond_E", ctypes.c_double * SDF_MAX_OUTER),
                ("relres", ctypes.c_double * SDF_MAX_OUTER),
                ("true_relres", ctypes.c_double * SDF_MAX_OUTER),
                ("relres_floor", ctypes.c_double * SDF_MAX_OUTER)]


_vp, _sz = ctypes.c_void_p, ctypes.c_size_t
_i32, _i64 = ctypes.c_int, ctypes.c_int64
_sigs = {
    "sdf_default_opts": (None, [ctypes.POINTER(Opts)]),
    "sdf_problem_create": (_i32, [ctypes.POINTER(ProblemDesc), _vp, ctypes.POINTER(_vp)]),
    "sdf_problem_device_bytes": (_i32, [_vp, ctypes.POINTER(_sz)]),
    "sdf_problem_create_csr": (_i32, [_i64, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(_vp)]),
    "sdf_solve_batch_rhs": (_i32, [_vp, _vp, _vp, _i32, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp,
                                   _vp, _vp, _vp, _vp]),
    "sdf_problem_bind": (_i32, [_vp, _vp, _sz, _vp]),
    "sdf_set_reference_modes": (_i32, [_vp, _vp, _i32, _i64, _i32]),
    "sdf_analytic_modes": (_i32, [_vp, _i32, _vp, _i64, _i32, _vp, _vp]),
    "sdf_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(Opts), ctypes.POINTER(_sz)]),
    "sdf_host_io_bytes": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_solve_batch": (_i32, [_vp, _vp, _i32, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp, _vp, _vp,
                               _vp, _vp]),
    "sdf_solve_batch_host": (_i32, [_vp, _vp, _i32, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp, _vp,
                                    _vp, _vp, _vp]),
    "sdf_apply_S": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp]),
    "sdf_project": (_i32, [_vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "sdf_project_noalloc": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sdf_get_profile": (_i32, [_vp, ctypes.POINTER(Profile)]),
    "sdf_reset_profile": (_i32, [_vp]),
    "sdf_last_error": (ctypes.c_char_p, [_vp]),
    "sdf_problem_destroy": (None, [_vp]),
    "sdf_solve_batch_x0": (_i32, [_vp, _vp, _i32, _vp, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp,
                                  _vp, _vp, _vp, _vp]),
    "sdf_mlp_param_count": (_i64, [_vp]),
    "sdf_mlp_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_mlp_forward": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _sz, _vp]),
    "sdf_mlp_loss_grad": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
    "sdf_adam_step": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, _vp]),
    "sdf_pod_workspace_size": (_i32, [_i64, _i32, ctypes.POINTER(_sz)]),
    "sdf_pod": (_i32, [_vp, _i32, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "sdf_warm_expand_workspace_size": (_i32, [_i32, _i32, ctypes.POINTER(_sz)]),
    "sdf_warm_expand": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _i32, _vp, _vp, _sz, _vp]),
    "sdf_aux_last_error": (ctypes.c_char_p, []),
    "sdf_warm_fit_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_warm_fit": (_i32, [_vp, _vp, _vp, _i32, _i32, ctypes.c_float, _vp, _vp, _sz, _vp]),
    "sdf_warm_predict_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_warm_predict": (_i32, [_vp, _vp, _i32, _vp, _vp, _sz, _vp]),
    "sdf_learned_host_io_bytes": (_i32, [_vp, _vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_solve_batch_learned_host": (_i32, [_vp, _vp, _vp, _i32, _vp, ctypes.POINTER(Opts), _vp,
                                            _sz, _vp, _vp, _vp, _vp, _vp]),
    "sdf_autotune_choice": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]),
    "sdf_autotune": (_i32, [_vp, _vp, _i32, _vp, ctypes.POINTER(Opts), _vp, _sz, _vp, _vp, _vp,
                            ctypes.POINTER(_i32)]),
    "sdf_default_eig_opts": (None, [_vp]),
    "sdf_eig_workspace_size": (_i32, [_vp, _i32, _vp, ctypes.POINTER(_sz)]),
    "sdf_reference_modes_eig": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "sdf_coarse_modes_workspace_size": (_i32, [_vp, _i32, _i32, _vp, ctypes.POINTER(_sz)]),
    "sdf_reference_modes_coarse": (_i32, [_vp, _i32, _i32, _vp, ctypes.c_double, _vp, _i64,
                                          ctypes.POINTER(_i32), _vp, _vp, _vp, _sz, _vp]),
    "sdf_spacetime_kron_modes": (_i32, [_vp, _vp, _i32, _i64, _i32, _vp, _i64, _vp]),
    "sdf_spacetime_modes": (_i32, [_vp, _vp, _i32, _vp, _i32, _i64, _i32, _vp, _i64, _vp]),
    "sdf_dct2_basis": (None, [_i32, _i32, _vp]),
    "sdf_diag_sets_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_diag_active_sets": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                    _vp]),
    "sdf_diag_drift_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_diag_drift": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _sz, _vp]),
    "sdf_default_restricted_eig_opts": (None, [_i32, _vp]),
    "sdf_restricted_eig_workspace_size": (_i32, [_vp, _i32, _vp, ctypes.POINTER(_sz)]),
    "sdf_restricted_modes_eig": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _sz,
                                        _vp]),
    "sdf_diag_angles_workspace_size": (_i32, [_vp, _i32, ctypes.POINTER(_sz)]),
    "sdf_diag_relres_workspace_size": (_i32, [_vp, ctypes.POINTER(_sz)]),
    "sdf_diag_relres": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "sdf_diag_angles": (_i32, [_vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp, _sz, _vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


class SdfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.sdf_default_opts(ctypes.byref(o))
    names = {f[0] for f in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"sdf_opts has no field {k!r}")
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def stats_dict(s: Stats) -> dict:
    n = s.outer_iters
    return dict(status=s.status, outer_iters=n, cg_iters=list(s.cg_iters[:n]),
                n_active=list(s.n_active[:n]), fallback=list(s.fallback[:n]),
                cond_E=list(s.cond_E[:n]), relres=list(s.relres[:n]),
                true_relres=list(s.true_relres[:n]), relres_floor=list(s.relres_floor[:n]),
                floor_stop=list(s.floor_stop[:n]))


class Problem:
    """Handle over sdf_problem: operator data bound to a device tensor."""

    def __init__(self, dim, n, alpha=1e-4, kappa=None, mass=1.0, kscale=1.0, diff_scale=1.0,
                 convection=False, yd_sigma=0.1, time_axis=False, t_final=1.0, ramp_tau=0.2,
                 device="cuda"):
        """time_axis=True: the space-time problem on an (n_x, n_y, n_t) grid
        (dim = 3; sdf_problem_desc.time_axis)."""
        n = list(n) if hasattr(n, "__len__") else [n] * dim
        while len(n) < 3:
            n.append(1)
        d = ProblemDesc(dim=dim, alpha=alpha, mass=mass, kscale=kscale, diff_scale=diff_scale,
                        has_kappa=int(kappa is not None), convection=int(bool(convection)),
                        yd_sigma=yd_sigma, time_axis=int(bool(time_axis)), t_final=t_final,
                        ramp_tau=ramp_tau)
        for i in range(3):
            d.n[i] = n[i]
        self.dim, self.n = dim, tuple(n[:dim])
        self.N = int(np.prod(self.n))
        self.device = torch.device(device)
        kap = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
        h = ctypes.c_void_p()
        st = _lib.sdf_problem_create(ctypes.byref(d), kap.ctypes.data if kap is not None else None,
                                     ctypes.byref(h))
        if st != 0:
            raise SdfError(st, "sdf_problem_create")
        self._h = h
        nb = _sz()
        self._check(_lib.sdf_problem_device_bytes(self._h, ctypes.byref(nb)))
        self._buf = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        self._check(_lib.sdf_problem_bind(self._h, _ptr(self._buf), self._buf.numel(), _stream()))
        self._phi = None
        self._ws = None

    @classmethod
    def csr(cls, K, alpha=1e-4, mass=1.0, kscale=1.0, device="cuda"):
        """sdf_problem_create_csr: a problem given by its operator K (a
        scipy.sparse matrix, n x n); S = mass I + alpha kscale^2/mass K^T K
        is assembled by the library.  Solve with solve_rhs."""
        K = K.tocsr()
        n = K.shape[0]
        rp = np.ascontiguousarray(K.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(K.indices, dtype=np.int32)
        v = np.ascontiguousarray(K.data, dtype=np.float64)
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        st = _lib.sdf_problem_create_csr(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, mass,
                                         alpha, kscale, ctypes.byref(h))
        if st != 0:
            raise SdfError(st, "sdf_problem_create_csr")
        self._h = h
        self.dim, self.n, self.N = 0, (n,), n
        self.device = torch.device(device)
        nb = _sz()
        self._check(_lib.sdf_problem_device_bytes(self._h, ctypes.byref(nb)))
        self._buf = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        self._check(_lib.sdf_problem_bind(self._h, _ptr(self._buf), self._buf.numel(), _stream()))
        self._phi = None
        self._ws = None
        return self

    def _check(self, st):
        if st != 0:
            raise SdfError(st, _lib.sdf_last_error(self._h).decode())
        return st

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.sdf_problem_destroy(self._h)
            self._h = None

    # reference modes ------------------------------------------------------
    def set_modes(self, phi: torch.Tensor):
        """phi: (k, N) contiguous device tensor (mode j = row j), i.e. the
        column-major N x k layout of the C ABI with ld = N."""
        assert phi.is_cuda and phi.is_contiguous() and phi.shape[1] == self.N
        dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[phi.dtype]
        self._check(_lib.sdf_set_reference_modes(self._h, _ptr(phi), phi.shape[0], self.N, dt))
        self._phi = phi
        return self

    def analytic_modes(self, k, dtype=F64):
        phi = torch.empty((k, self.N), dtype=_TORCH_DTYPE[dtype], device=self.device)
        ev = np.zeros(k)
        self._check(_lib.sdf_analytic_modes(self._h, k, _ptr(phi), self.N, dtype,
                                            ev.ctypes.data, _stream()))
        return phi, ev

    def spacetime_kron_modes(self, zs: torch.Tensor):
        """sdf_spacetime_kron_modes: I_nt (x) Z_s for spatial modes zs
        (r, N_s) (row j = mode j); returns (r n_t, N) of zs's dtype."""
        assert zs.is_cuda and zs.is_contiguous()
        r, Ns = zs.shape
        nt = self.n[2] if len(self.n) > 2 else 1
        dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[zs.dtype]
        phi = torch.empty((r * nt, self.N), dtype=zs.dtype, device=self.device)
        self._check(_lib.sdf_spacetime_kron_modes(self._h, _ptr(zs), r, Ns, dt, _ptr(phi),
                                                  self.N, _stream()))
        return phi

    def spacetime_modes(self, wt: np.ndarray, zs: torch.Tensor):
        """sdf_spacetime_modes: W_t (x) Z_s for a temporal factor wt (n_t, r_t)
        (host) and spatial modes zs (r, N_s); returns (r_t r, N) of zs's dtype."""
        assert zs.is_cuda and zs.is_contiguous()
        wt = np.asfortranarray(wt, dtype=np.float64)
        r, Ns = zs.shape
        rt = wt.shape[1]
        dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[zs.dtype]
        phi = torch.empty((rt * r, self.N), dtype=zs.dtype, device=self.device)
        self._check(_lib.sdf_spacetime_modes(self._h, wt.ctypes.data, rt, _ptr(zs), r, Ns, dt,
                                             _ptr(phi), self.N, _stream()))
        return phi

    def eig_modes(self, k, **kw):
        """k smallest eigenpairs of A (those of S) by Chebyshev-filtered
        subspace iteration (sdf_reference_modes_eig): returns Phi (k, N)
        float64 (row j = mode j), lambda_S, lambda_A and the solver stats."""
        o = EigOpts()
        _lib.sdf_default_eig_opts(ctypes.byref(o))
        for key, v in kw.items():
            setattr(o, key, v)
        nb = _sz()
        self._check(_lib.sdf_eig_workspace_size(self._h, k, ctypes.byref(o), ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        phi = torch.empty((k, self.N), dtype=torch.float64, device=self.device)
        ls, la = np.zeros(k), np.zeros(k)
        st = EigStats()
        rc = _lib.sdf_reference_modes_eig(self._h, k, ctypes.byref(o), _ptr(phi), self.N,
                                          ls.ctypes.data, la.ctypes.data, ctypes.byref(st),
                                          _ptr(ws), ws.numel(), _stream())
        if rc not in (0, 5):
            self._check(rc)
        stats = dict(iters=st.iters, converged=bool(st.converged), max_rel_resid=st.max_rel_resid,
                     matvecs=st.matvecs, seconds=st.seconds, status=rc)
        return phi, ls, la, stats

    def coarse_modes(self, c, r_pool, tau_sv=1e-8, **kw):
        """Coarse-grid reference basis (sdf_reference_modes_coarse): returns
        Phi (r, N) float64 with r <= r_pool kept columns, the coarse
        eigenvalues of S_c and the coarse eigensolve's stats."""
        o = EigOpts()
        _lib.sdf_default_eig_opts(ctypes.byref(o))
        for key, v in kw.items():
            setattr(o, key, v)
        nb = _sz()
        self._check(_lib.sdf_coarse_modes_workspace_size(self._h, c, r_pool, ctypes.byref(o),
                                                         ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        phi = torch.empty((r_pool, self.N), dtype=torch.float64, device=self.device)
        lam = np.zeros(r_pool)
        r = ctypes.c_int(0)
        st = EigStats()
        self._check(_lib.sdf_reference_modes_coarse(self._h, c, r_pool, ctypes.byref(o), tau_sv,
                                                    _ptr(phi), self.N, ctypes.byref(r),
                                                    lam.ctypes.data, ctypes.byref(st), _ptr(ws),
                                                    ws.numel(), _stream()))
        stats = dict(iters=st.iters, converged=bool(st.converged), max_rel_resid=st.max_rel_resid,
                     matvecs=st.matvecs, seconds=st.seconds)
        return phi[:r.value].contiguous(), lam, stats

    # spectral diagnostics -----------------------------------------------------
    def _scratch(self, size_fn, *args):
        nb = _sz()
        self._check(size_fn(self._h, *args, ctypes.byref(nb)))
        return torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)

    def diag_active_sets(self, active_ref: torch.Tensor, active: torch.Tensor, r=0):
        """sdf_diag_active_sets: active-set distances (Eq. delta, Eq. rho and
        the mode-weighted delta_w over the first r registered modes) of the
        B masks `active` (B, N) uint8 from `active_ref` (N,) uint8."""
        assert active_ref.dtype == torch.uint8 and active.dtype == torch.uint8
        act = active.reshape(-1, self.N).contiguous()
        B = act.shape[0]
        ws = self._scratch(_lib.sdf_diag_sets_workspace_size, B)
        sym, na = np.zeros(B, np.int64), np.zeros(B, np.int64)
        dl, rh, dw = np.zeros(B), np.zeros(B), np.zeros(B)
        self._check(_lib.sdf_diag_active_sets(self._h, _ptr(active_ref.contiguous()), _ptr(act), B,
                                              r, sym.ctypes.data, na.ctypes.data, dl.ctypes.data,
                                              rh.ctypes.data, dw.ctypes.data if r > 0 else None,
                                              _ptr(ws), ws.numel(), _stream()))
        return dict(sym_diff=sym, n_active=na, delta=dl, rho=rh, delta_w=dw if r > 0 else None)

    def diag_drift(self, inst_ref: torch.Tensor, inst: torch.Tensor, steps=200):
        """sdf_diag_drift: eps_b = ||S(ref) - S(b)||_2 / ||S(ref)||_2 (Eq.
        epsilon) by Lanczos; returns (eps (B,), ||S(ref)||_2)."""
        inst = inst.reshape(-1, 7).contiguous()
        B = inst.shape[0]
        ws = self._scratch(_lib.sdf_diag_drift_workspace_size, steps)
        eps = np.zeros(B)
        nref = ctypes.c_double(0.0)
        self._check(_lib.sdf_diag_drift(self._h, _ptr(inst_ref.contiguous()), _ptr(inst), B, steps,
                                        eps.ctypes.data, ctypes.byref(nref), _ptr(ws), ws.numel(),
                                        _stream()))
        return eps, nref.value

    def restricted_modes(self, inst: torch.Tensor, active: torch.Tensor, k, **kw):
        """sdf_restricted_modes_eig: the k smallest eigenpairs of S_II on the
        inactive set of `active` (N,) uint8 for one instance (7,); returns
        V (k, N) float64 (row j = eigenvector j, zero on A), lambda, stats."""
        o = EigOpts()
        _lib.sdf_default_restricted_eig_opts(k, ctypes.byref(o))
        for key, v in kw.items():
            setattr(o, key, v)
        nb = _sz()
        self._check(_lib.sdf_restricted_eig_workspace_size(self._h, k, ctypes.byref(o),
                                                           ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        V = torch.empty((k, self.N), dtype=torch.float64, device=self.device)
        lam = np.zeros(k)
        st = EigStats()
        rc = _lib.sdf_restricted_modes_eig(self._h, _ptr(inst.contiguous()),
                                           _ptr(active.contiguous()), k, ctypes.byref(o), _ptr(V),
                                           self.N, lam.ctypes.data, ctypes.byref(st), _ptr(ws),
                                           ws.numel(), _stream())
        if rc not in (0, 5):
            self._check(rc)
        stats = dict(iters=st.iters, converged=bool(st.converged), max_rel_resid=st.max_rel_resid,
                     matvecs=st.matvecs, seconds=st.seconds, status=rc)
        return V, lam, stats

    def diag_relres(self, out, inst: torch.Tensor = None):
        """sdf_diag_relres: the true relative residual of each instance's
        final inner solve, from a solve's outputs (y, lam, active; lam must
        have been requested)."""
        y, lam, act = out["y"], out["lam"], out["active"]
        assert lam is not None, "solve with want_lambda=True"
        B = y.shape[0]
        nb = _sz()
        self._check(_lib.sdf_diag_relres_workspace_size(self._h, ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        rel = np.zeros(B)
        self._check(_lib.sdf_diag_relres(self._h, _ptr(inst), B, _ptr(y), _ptr(lam), _ptr(act),
                                         rel.ctypes.data, _ptr(ws), ws.numel(), _stream()))
        return rel

    def diag_angles(self, active: torch.Tensor, V: torch.Tensor, k=None, sorted_angles=False):
        """sdf_diag_angles for V (k, N) float64 against the registered modes
        restricted to the inactive set: the nested angles theta_r (radians),
        r = 1..k (Prop. dk with S = {1..r}); with sorted_angles=True also the
        ascending principal angles between the k-dimensional spans (the
        paper's theta_r is entry r - 1)."""
        k = V.shape[0] if k is None else k
        assert V.dtype == torch.float64 and V.is_contiguous() and V.shape[1] == self.N
        ws = self._scratch(_lib.sdf_diag_angles_workspace_size, k)
        th, srt = np.zeros(k), np.zeros(k)
        self._check(_lib.sdf_diag_angles(self._h, _ptr(active.contiguous()), _ptr(V), self.N, k,
                                         th.ctypes.data, srt.ctypes.data, _ptr(ws), ws.numel(),
                                         _stream()))
        return (th, srt) if sorted_angles else th

    # workspace --------------------------------------------------------------
    def workspace(self, batch, opts=None, host_io=False):
        opts = opts or default_opts()
        nb = _sz()
        self._check(_lib.sdf_workspace_size(self._h, batch, ctypes.byref(opts), ctypes.byref(nb)))
        need = int(nb.value)
        if host_io:
            io = _sz()
            self._check(_lib.sdf_host_io_bytes(self._h, batch, ctypes.byref(io)))
            need = ((need + 255) // 256) * 256 + int(io.value)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._ws

    # solves ---------------------------------------------------------------
    def solve(self, inst: torch.Tensor, psi: torch.Tensor, opts=None, want_lambda=True,
              out=None, raise_on_fail=False):
        """inst: (B, 7) float64 device tensor; psi: (N,) float64 device tensor."""
        opts = opts or default_opts()
        B = inst.shape[0]
        assert inst.dtype == torch.float64 and inst.is_contiguous() and inst.shape[1] == 7
        ws = self.workspace(B, opts)
        if out is None:
            out = dict(y=torch.empty((B, self.N), dtype=torch.float64, device=self.device),
                       lam=torch.empty((B, self.N), dtype=torch.float64, device=self.device)
                       if want_lambda else None,
                       active=torch.empty((B, self.N), dtype=torch.uint8, device=self.device))
        stats = (Stats * B)()
        st = _lib.sdf_solve_batch(self._h, _ptr(inst), B, _ptr(psi), ctypes.byref(opts),
                                  _ptr(ws), ws.numel(), _stream(), _ptr(out["y"]),
                                  _ptr(out["lam"]), _ptr(out["active"]), stats)
        if st not in (0, 5, 6, 7, 8) or (raise_on_fail and st != 0):
            self._check(st)
        out["status"] = st
        out["stats"] = [stats_dict(s) for s in stats]
        return out

    def autotune(self, inst: torch.Tensor, psi: torch.Tensor, opts=None):
        """sdf_autotune: pick the column depth of the mixed 3D kernels for
        this batch size by timing short solves; returns the choice (0: none)."""
        opts = opts or default_opts()
        B = inst.shape[0]
        ws = self.workspace(B, opts)
        y = torch.empty((B, self.N), dtype=torch.float64, device=self.device)
        a = torch.empty((B, self.N), dtype=torch.uint8, device=self.device)
        ch = ctypes.c_int(0)
        self._check(_lib.sdf_autotune(self._h, _ptr(inst), B, _ptr(psi), ctypes.byref(opts),
                                      _ptr(ws), ws.numel(), _stream(), _ptr(y), _ptr(a),
                                      ctypes.byref(ch)))
        return ch.value

    def autotune_choice(self, batch):
        """sdf_autotune_choice: (column depth, pairing) kept for a batch size
        (depth 0 / pairing -1: not tuned)."""
        d, pr = ctypes.c_int(0), ctypes.c_int(0)
        self._check(_lib.sdf_autotune_choice(self._h, batch, ctypes.byref(d), ctypes.byref(pr)))
        return d.value, pr.value

    def solve_x0(self, inst: torch.Tensor, psi: torch.Tensor, x0: torch.Tensor, opts=None,
                 want_lambda=False, out=None):
        """sdf_solve_batch_x0: every inner solve starts from x0 (B, N) float64
        restricted to its inactive set."""
        opts = opts or default_opts()
        B = inst.shape[0]
        assert x0.dtype == torch.float64 and x0.is_contiguous() and x0.shape == (B, self.N)
        ws = self.workspace(B, opts)
        if out is None:
            out = dict(y=torch.empty((B, self.N), dtype=torch.float64, device=self.device),
                       lam=torch.empty((B, self.N), dtype=torch.float64, device=self.device)
                       if want_lambda else None,
                       active=torch.empty((B, self.N), dtype=torch.uint8, device=self.device))
        stats = (Stats * B)()
        st = _lib.sdf_solve_batch_x0(self._h, _ptr(inst), B, _ptr(psi), _ptr(x0),
                                     ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(),
                                     _ptr(out["y"]), _ptr(out["lam"]), _ptr(out["active"]), stats)
        if st not in (0, 5, 6, 7, 8):
            self._check(st)
        out["status"] = st
        out["stats"] = [stats_dict(s) for s in stats]
        return out

    def solve_rhs(self, rhs: torch.Tensor, psi: torch.Tensor, opts=None, inst=None,
                  want_lambda=False, out=None):
        """sdf_solve_batch_rhs: rhs (B, N) float64 device tensor in place of
        the instances' mass y_d; inst (B, 7) only for per-instance convection."""
        opts = opts or default_opts()
        assert rhs.dtype == torch.float64 and rhs.is_contiguous() and rhs.shape[1] == self.N
        B = rhs.shape[0]
        ws = self.workspace(B, opts)
        if out is None:
            out = dict(y=torch.empty((B, self.N), dtype=torch.float64, device=self.device),
                       lam=torch.empty((B, self.N), dtype=torch.float64, device=self.device)
                       if want_lambda else None,
                       active=torch.empty((B, self.N), dtype=torch.uint8, device=self.device))
        stats = (Stats * B)()
        st = _lib.sdf_solve_batch_rhs(self._h, _ptr(inst), _ptr(rhs), B, _ptr(psi),
                                      ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(),
                                      _ptr(out["y"]), _ptr(out["lam"]), _ptr(out["active"]), stats)
        if st not in (0, 5, 6, 7, 8):
            self._check(st)
        out["status"] = st
        out["stats"] = [stats_dict(s) for s in stats]
        return out

    def solve_host(self, inst: np.ndarray, psi: np.ndarray, opts=None, y=None, lam=None,
                   active=None):
        """Host-memory variant (sdf_solve_batch_host): numpy in, numpy out."""
        opts = opts or default_opts()
        inst = np.ascontiguousarray(inst, dtype=np.float64)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        B = inst.shape[0]
        ws = self.workspace(B, opts, host_io=True)
        y = np.empty((B, self.N)) if y is None else y
        active = np.empty((B, self.N), np.uint8) if active is None else active
        stats = (Stats * B)()
        st = _lib.sdf_solve_batch_host(self._h, inst.ctypes.data, B, psi.ctypes.data,
                                       ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(),
                                       y.ctypes.data, None if lam is None else lam.ctypes.data,
                                       active.ctypes.data, stats)
        if st not in (0, 5, 6, 7, 8):
            self._check(st)
        return dict(y=y, lam=lam, active=active, status=st, stats=[stats_dict(s) for s in stats])

    def solve_learned_host(self, model, inst: np.ndarray, psi: np.ndarray, opts=None, y=None,
                           lam=None, active=None):
        """The learned pipeline from host buffers (sdf_solve_batch_learned_host):
        numpy in, x0 predicted by `model` (a WarmModel) and the solve on the
        device, numpy out."""
        opts = opts or default_opts()
        inst = np.ascontiguousarray(inst, dtype=np.float64)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        B = inst.shape[0]
        nb, xb = _sz(), _sz()
        self._check(_lib.sdf_workspace_size(self._h, B, ctypes.byref(opts), ctypes.byref(nb)))
        self._check(_lib.sdf_learned_host_io_bytes(self._h, ctypes.byref(model.desc), B,
                                                   ctypes.byref(xb)))
        need = ((int(nb.value) + 255) // 256) * 256 + int(xb.value)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        ws = self._ws
        y = np.empty((B, self.N)) if y is None else y
        active = np.empty((B, self.N), np.uint8) if active is None else active
        stats = (Stats * B)()
        st = _lib.sdf_solve_batch_learned_host(
            self._h, ctypes.byref(model.desc), inst.ctypes.data, B, psi.ctypes.data,
            ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(), y.ctypes.data,
            None if lam is None else lam.ctypes.data, active.ctypes.data, stats)
        if st not in (0, 5, 6, 7, 8):
            self._check(st)
        return dict(y=y, lam=lam, active=active, status=st, stats=[stats_dict(s) for s in stats])

    # tracing ----------------------------------------------------------------
    def profile(self):
        pr = Profile()
        self._check(_lib.sdf_get_profile(self._h, ctypes.byref(pr)))
        mean = {n: (pr.ms[i] / pr.samples[i] if pr.samples[i] else None)
                for i, n in enumerate(PROFILE_NAMES)}
        return dict(mean_ms=mean, samples={n: pr.samples[i] for i, n in enumerate(PROFILE_NAMES)},
                    launches=pr.launches)

    def reset_profile(self):
        self._check(_lib.sdf_reset_profile(self._h))

    # building blocks --------------------------------------------------------
    def apply_S(self, inst: torch.Tensor, u: torch.Tensor, active: torch.Tensor = None, mode=0):
        out = torch.empty_like(u)
        self._check(_lib.sdf_apply_S(self._h, _ptr(inst), _ptr(active), _ptr(u), _ptr(out), mode,
                                     None, 0, _stream()))
        return out

    def project(self, active: torch.Tensor, v: torch.Tensor):
        k = self._phi.shape[0]
        out = torch.empty(k, dtype=torch.float64, device=self.device)
        ws = torch.empty(1 << 20, dtype=torch.uint8, device=self.device)
        self._check(_lib.sdf_project(self._h, _ptr(active), _ptr(v), _ptr(out), _ptr(ws),
                                     ws.numel(), _stream()))
        return out

    def project_noalloc(self, active: torch.Tensor, v: torch.Tensor, out: torch.Tensor):
        """Phi_I^T v into the caller's `out` (k doubles) using the library's
        built-in scratch array instead of a workspace (sdf_project_noalloc)."""
        self._check(_lib.sdf_project_noalloc(self._h, _ptr(active), _ptr(v), _ptr(out),
                                              _stream()))
        return out


# ---------------------------------------------------------------------------
# learned warm start: MLP (tensor-core products), Adam, POD, expansion

SDF_MLP_MAX_LAYERS = 8
SDF_POD_MAX_R = 64


class MlpDesc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("width", ctypes.c_int32 * (SDF_MLP_MAX_LAYERS + 1))]


def _aux_check(st):
    if st != 0:
        raise SdfError(st, _lib.sdf_aux_last_error().decode())


class Mlp:
    """Widths (w0, ..., wL); parameters are one flat FP32 device tensor laid
    out as W_1, b_1, ..., W_L, b_L (W row-major out x in)."""

    def __init__(self, widths, device="cuda"):
        self.widths = tuple(int(w) for w in widths)
        self.desc = MlpDesc(n_layers=len(self.widths) - 1)
        for i, w in enumerate(self.widths):
            self.desc.width[i] = w
        self.n_params = int(_lib.sdf_mlp_param_count(ctypes.byref(self.desc)))
        if self.n_params < 0:
            raise SdfError(1, "bad MLP widths")
        self.device = torch.device(device)
        self._ws = None

    def _workspace(self, batch):
        nb = _sz()
        _aux_check(_lib.sdf_mlp_workspace_size(ctypes.byref(self.desc), batch, ctypes.byref(nb)))
        if self._ws is None or self._ws.numel() < nb.value:
            self._ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        return self._ws

    def forward(self, theta: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        B = x.shape[0]
        y = torch.empty((B, self.widths[-1]), dtype=torch.float32, device=self.device)
        ws = self._workspace(B)
        _aux_check(_lib.sdf_mlp_forward(ctypes.byref(self.desc), _ptr(theta), _ptr(x), B, _ptr(y),
                                        _ptr(ws), ws.numel(), _stream()))
        return y

    def loss_grad(self, theta: torch.Tensor, x: torch.Tensor, t: torch.Tensor, grad=None,
                  loss=None):
        x, t = x.contiguous(), t.contiguous()
        B = x.shape[0]
        grad = torch.empty_like(theta) if grad is None else grad
        loss = torch.empty(1, dtype=torch.float64, device=self.device) if loss is None else loss
        ws = self._workspace(B)
        _aux_check(_lib.sdf_mlp_loss_grad(ctypes.byref(self.desc), _ptr(theta), _ptr(x), _ptr(t),
                                          B, _ptr(grad), _ptr(loss), _ptr(ws), ws.numel(),
                                          _stream()))
        return loss, grad


def dct2_basis(n, r):
    """sdf_dct2_basis: the first r orthonormal DCT-II vectors of length n,
    as an (n, r) float64 array."""
    w = np.zeros((n, r), order="F")
    _lib.sdf_dct2_basis(n, r, w.ctypes.data)
    return w


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _aux_check(_lib.sdf_adam_step(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(), step,
                                  lr, beta1, beta2, eps, _stream()))


def pod(Y: torch.Tensor, r: int):
    """POD of the rows of Y (m, N) float64 device tensor; returns ybar (N,),
    psi_rm (N, r) bf16 node-major, psi_cm (r, N) float64 (column j = row j),
    singular values (r,) and coefficients (m, r) as numpy arrays."""
    Y = Y.contiguous()
    m, N = Y.shape
    nb = _sz()
    _aux_check(_lib.sdf_pod_workspace_size(N, m, ctypes.byref(nb)))
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device=Y.device)
    ybar = torch.empty(N, dtype=torch.float64, device=Y.device)
    psi_rm = torch.empty((N, r), dtype=torch.bfloat16, device=Y.device)
    psi_cm = torch.empty((r, N), dtype=torch.float64, device=Y.device)
    sing = np.zeros(r)
    coef = np.zeros((m, r))
    _aux_check(_lib.sdf_pod(_ptr(Y), m, N, r, _ptr(ybar), _ptr(psi_rm), _ptr(psi_cm),
                            sing.ctypes.data, coef.ctypes.data, _ptr(ws), ws.numel(), _stream()))
    return ybar, psi_rm, psi_cm, sing, coef


def warm_expand(psi_rm: torch.Tensor, ybar: torch.Tensor, cstd: torch.Tensor,
                cmean: torch.Tensor, cscale: torch.Tensor) -> torch.Tensor:
    """x0[b] = ybar + psi (cstd[b] * cscale + cmean), (B, N) float64."""
    N, r = psi_rm.shape
    B = cstd.shape[0]
    nb = _sz()
    _aux_check(_lib.sdf_warm_expand_workspace_size(B, r, ctypes.byref(nb)))
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device=psi_rm.device)
    x0 = torch.empty((B, N), dtype=torch.float64, device=psi_rm.device)
    _aux_check(_lib.sdf_warm_expand(_ptr(psi_rm), _ptr(ybar), N, r, _ptr(cstd.contiguous()),
                                    _ptr(cmean), _ptr(cscale), B, _ptr(x0), _ptr(ws), ws.numel(),
                                    _stream()))
    return x0


class WarmModelDesc(ctypes.Structure):
    _fields_ = [("mlp", MlpDesc), ("r", ctypes.c_int32), ("n", ctypes.c_int64),
                ("in_lo", ctypes.c_double * 8), ("in_hi", ctypes.c_double * 8),
                ("theta", _vp), ("ybar", _vp), ("psi", _vp), ("cmean", _vp), ("cscale", _vp)]


class WarmModel:
    """Learned warm start (sdf_warm_fit / sdf_warm_predict): device tensors for
    the MLP parameters and the POD basis; theta0 (FP32 tensor) is the
    caller's initial parameter vector."""

    def __init__(self, widths, n, in_lo, in_hi, theta0: torch.Tensor):
        self.mlp = Mlp(widths, theta0.device)
        r = int(widths[-1])
        dev = theta0.device
        assert theta0.numel() == self.mlp.n_params and theta0.dtype == torch.float32
        self.theta = theta0.clone().contiguous()
        self.ybar = torch.empty(n, dtype=torch.float64, device=dev)
        self.psi = torch.empty((r, n), dtype=torch.float64, device=dev)  # column-major n x r
        self.cmean = torch.empty(r, dtype=torch.float32, device=dev)
        self.cscale = torch.empty(r, dtype=torch.float32, device=dev)
        d = WarmModelDesc(mlp=self.mlp.desc, r=r, n=n)
        for i, (a, b) in enumerate(zip(in_lo, in_hi)):
            d.in_lo[i], d.in_hi[i] = float(a), float(b)
        d.theta, d.ybar, d.psi = _ptr(self.theta), _ptr(self.ybar), _ptr(self.psi)
        d.cmean, d.cscale = _ptr(self.cmean), _ptr(self.cscale)
        self.desc = d
        self.device = dev

    def fit(self, Y: torch.Tensor, inst: torch.Tensor, epochs=500, lr0=1e-3):
        m = Y.shape[0]
        nb = _sz()
        _aux_check(_lib.sdf_warm_fit_workspace_size(ctypes.byref(self.desc), m, ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        loss = np.zeros(epochs)
        _aux_check(_lib.sdf_warm_fit(ctypes.byref(self.desc), _ptr(Y.contiguous()),
                                     _ptr(inst.contiguous()), m, epochs, lr0, loss.ctypes.data,
                                     _ptr(ws), ws.numel(), _stream()))
        return loss

    def predict(self, inst: torch.Tensor) -> torch.Tensor:
        B = inst.shape[0]
        nb = _sz()
        _aux_check(_lib.sdf_warm_predict_workspace_size(ctypes.byref(self.desc), B,
                                                        ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        x0 = torch.empty((B, self.desc.n), dtype=torch.float64, device=self.device)
        _aux_check(_lib.sdf_warm_predict(ctypes.byref(self.desc), _ptr(inst.contiguous()), B,
                                         _ptr(x0), _ptr(ws), ws.numel(), _stream()))
        return x0
