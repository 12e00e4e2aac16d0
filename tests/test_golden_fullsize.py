"""The committed 128^3 golden states against closed forms (no GPU).

tests/golden/diff3d_128_oracle_states.npz holds the oracle's full-size solves
of two instances of the 3D diffusion workload (written by
oracle/full_size_reference.py; each took about 25 minutes on 8 cores).  Both
solves end with an empty active set after one outer iteration, so each state
is the solution of S y = rhs with S = I + alpha L^2 (L the 7-point Laplacian,
kappa = 1, Sec. 2.1.2 Eq. schur) and rhs = y_d (mass 1).

For constant kappa the sine modes phi_q (App. A, the analytic modes of
Sec. 2.2.8) diagonalise S with eigenvalues 1 + alpha mu_q^2, and the desired
state a exp(-|x - c|^2 / (2 sigma^2)) is separable, so the exact solution's
coefficient on every mode is closed-form:

    phi_q^T y = a (s_q1^T g_z)(s_q2^T g_y)(s_q3^T g_x) / (1 + alpha mu_q^2).

The stored states must carry these coefficients on the 512 lowest sine modes
per direction triple (q_l <= 8), up to what the stored data allow: the solve's
true residual r (||r|| <= true_relres ||rhs||, and lambda_min(S) >= 1, so
|phi_q^T e| <= ||e|| <= true_relres ||rhs||) plus the float32 rounding of the
stored state (|phi_q^T d| <= ||d|| <= 2^-24 ||y||).  Measured: 1e-10 of the
largest coefficient."""
import json
import os

import numpy as np
import pytest

from paper_2606_17971_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    g = json.load(open(os.path.join(HERE, "golden", "diff3d_128_oracle.json")))
    s = np.load(os.path.join(HERE, "golden", "diff3d_128_oracle_states.npz"))
    return g, s


def _sines(n, m):
    j = np.arange(1, n + 1)
    q = np.arange(1, m + 1)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, q) * np.pi / (n + 1)), q


def test_golden_instances_are_the_workload_draws(golden):
    g, _ = golden
    w = W.WORKLOADS["diff3d_128"]
    assert g["workload"] == w.name and g["k"] == w.k and g["rtol"] == 1e-8
    insts = W.draw_instances(w, count=max(i["index"] for i in g["instances"]) + 1)
    for gi in g["instances"]:
        ins = insts[gi["index"]]
        assert ins.a == gi["a"] and list(ins.c) == gi["c"]


def test_golden_states_carry_the_closed_form_spectral_coefficients(golden):
    g, s = golden
    w = W.WORKLOADS["diff3d_128"]
    n, m = w.n, 8
    h = 1.0 / (n + 1)
    S1, q = _sines(n, m)
    mu = (4.0 / h**2) * np.sin(q * np.pi / (2 * (n + 1))) ** 2
    lam = 1.0 + w.alpha * (mu[:, None, None] + mu[None, :, None] + mu[None, None, :]) ** 2
    x = np.arange(1, n + 1) * h
    for gi in g["instances"]:
        i, a, c = gi["index"], gi["a"], gi["c"]
        assert gi["outer_iters"] == 1 and gi["active_count"] == 0
        y = s[f"y{i}"].astype(np.float64)
        assert y.size == n**3
        act = np.unpackbits(s[f"active{i}"])[: y.size]
        assert not act.any()
        assert np.linalg.norm(y) == pytest.approx(gi["y_norm"], rel=1e-6)
        gx, gy, gz = (np.exp(-(x - cc) ** 2 / (2 * w.sigma**2)) for cc in c)
        rhs_c = a * np.einsum("a,b,c->abc", S1.T @ gz, S1.T @ gy, S1.T @ gx)
        exact = rhs_c / lam
        Y = y.reshape(n, n, n)  # [z, y, x], x fastest
        got = np.einsum("za,yb,xc,zyx->abc", S1, S1, S1, Y, optimize=True)
        rhs_norm = a * np.linalg.norm(gx) * np.linalg.norm(gy) * np.linalg.norm(gz)
        bound = gi["true_relres"] * rhs_norm + 2.0**-24 * np.linalg.norm(y)
        err = np.abs(got - exact).max()
        assert err <= bound, (i, err, bound)
        # and the coefficients are far from trivial: the lowest mode carries
        # a sizeable part of the state
        assert abs(exact[0, 0, 0]) > 0.1 * np.linalg.norm(y)
