"""GPU reference eigensolve (Chebyshev-filtered subspace iteration) against
the oracle's dense eigenpairs, the closed-form spectrum of the constant-kappa
operator, and the eigen-residual through the library's own S."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2606_17971_b300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def sdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_17971_b300 import sdf as S
    return S


def _sin_max_angle(A, B):
    """sine of the largest principal angle between the column spans of A and B
    (both with orthonormal columns)."""
    s = np.linalg.svd(A.T @ B, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))


def test_block_kappa_modes_match_dense_eigenpairs(sdf):
    n = (48, 40)
    w = W.scaled(W.WORKLOADS["block2d_1024"], 48)
    kap = np.ascontiguousarray(W.kappa_field(w).reshape(48, 48)[:40, :]).ravel()
    P = O.Problem(2, n, kappa=kap, alpha=w.alpha)
    k = 12
    Phi_o, lam_o = O.dense_modes(P, k)[:2]
    G = sdf.Problem(2, n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    phi, ls, la, st = G.eig_modes(k, tol=1e-9)
    assert st["converged"], st
    np.testing.assert_allclose(ls, np.sort(lam_o)[:k], rtol=1e-9)
    Pg = phi.cpu().numpy().T
    np.testing.assert_allclose(Pg.T @ Pg, np.eye(k), atol=1e-12)
    assert _sin_max_angle(Pg, Phi_o) < 1e-6


def test_constant_kappa_spectrum_matches_closed_form_3d(sdf):
    n = (10, 9, 8)   # unequal sides: no multiplet at the cut
    k = 20
    G = sdf.Problem(3, n, alpha=1e-4, yd_sigma=0.1)
    phi, ls, la, st = G.eig_modes(k, tol=1e-10)
    assert st["converged"], st
    # closed form: lambda_A = sum_d (4/h_d^2) sin^2(i_d pi / (2 (n_d + 1)))
    mus = [(4.0 * (nd + 1) ** 2) * np.sin(np.arange(1, nd + 1) * np.pi / (2 * (nd + 1))) ** 2
           for nd in n]
    lam = np.sort((mus[0][:, None, None] + mus[1][None, :, None] + mus[2][None, None, :]).ravel())
    np.testing.assert_allclose(la, lam[:k], rtol=1e-10)
    np.testing.assert_allclose(ls, 1.0 + 1e-4 * lam[:k] ** 2, rtol=1e-10)


def test_eigen_residual_through_S_and_deflated_solve(sdf):
    w = W.scaled(W.WORKLOADS["lognormal2d_2048"], 64)
    kap = W.kappa_field(w)
    G = sdf.Problem(2, w.n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    k = 24
    phi, ls, la, st = G.eig_modes(k, tol=1e-8)
    assert st["converged"], st
    inst = torch.as_tensor(W.instances_array(W.draw_instances(w, count=1)), device="cuda")
    for j in range(k):
        Sphi = G.apply_S(inst, phi[j].contiguous(), mode=1)
        r = (Sphi - ls[j] * phi[j]).norm().item()
        assert r <= 1e-6 * ls[j], (j, r, ls[j])
    # the modes deflate the solve: same solution as the oracle, fewer iterations than plain
    P = O.Problem(2, w.n, kappa=kap, alpha=w.alpha)
    insts = W.draw_instances(w, count=3)
    G.set_modes(phi)
    out = G.solve(torch.as_tensor(W.instances_array(insts), device="cuda"),
                  torch.ones(w.N, dtype=torch.float64, device="cuda"), want_lambda=False)
    plain = G.solve(torch.as_tensor(W.instances_array(insts), device="cuda"),
                    torch.ones(w.N, dtype=torch.float64, device="cuda"),
                    sdf.default_opts(deflate=0), want_lambda=False)
    for b, inst_b in enumerate(insts):
        ref = P.solve(P.desired_state(inst_b.a, inst_b.c[:2], w.sigma)[1], np.ones(P.N),
                      phi.cpu().numpy().T)
        y = out["y"][b].cpu().numpy()
        assert np.linalg.norm(y - ref["y"]) <= 1e-6 * np.linalg.norm(ref["y"])
        assert sum(out["stats"][b]["cg_iters"]) < sum(plain["stats"][b]["cg_iters"])


def test_convection_is_refused(sdf):
    G = sdf.Problem(2, 24, alpha=1e-4, diff_scale=1e-2, convection=True, yd_sigma=0.1)
    with pytest.raises(sdf.SdfError):
        G.eig_modes(4)


def test_coarse_grid_basis_matches_oracle_and_deflates(sdf):
    from oracle import coarse_oracle as C
    n = (48, 40)
    w = W.scaled(W.WORKLOADS["block2d_1024"], 48)
    kap = np.ascontiguousarray(W.kappa_field(w).reshape(48, 48)[:40, :]).ravel()
    r_pool = 12
    Q_o, lam_o = C.coarse_modes(2, n, 2, r_pool, kappa=kap, alpha=w.alpha)
    G = sdf.Problem(2, n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    phi, lam_c, st = G.coarse_modes(2, r_pool, tol=1e-10)
    assert st["converged"]
    np.testing.assert_allclose(lam_c, np.sort(lam_o)[:r_pool], rtol=1e-9)
    Pg = phi.cpu().numpy().T
    assert Pg.shape == Q_o.shape
    np.testing.assert_allclose(Pg.T @ Pg, np.eye(r_pool), atol=1e-12)
    assert _sin_max_angle(Pg, Q_o) < 1e-6
    # a 3D grid with every column kept deflates the fine solve
    G3 = sdf.Problem(3, (30, 28, 26), alpha=1e-4, yd_sigma=0.1)
    phi3, _, _ = G3.coarse_modes(2, 16)
    assert phi3.shape[0] == 16
    G3.set_modes(phi3)
    inst = torch.as_tensor([[2.0, 0.45, 0.5, 0.55, 0, 0, 0]], dtype=torch.float64, device="cuda")
    psi = torch.full((G3.N,), 10.0, dtype=torch.float64, device="cuda")
    defl = G3.solve(inst, psi, want_lambda=False)
    plain = G3.solve(inst, psi, sdf.default_opts(deflate=0), want_lambda=False)
    assert defl["stats"][0]["cg_iters"][0] < 0.8 * plain["stats"][0]["cg_iters"][0]
    assert (defl["y"] - plain["y"]).abs().max().item() < 1e-6 * plain["y"].abs().max().item()
