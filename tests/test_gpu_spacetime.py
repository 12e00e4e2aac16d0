"""GPU space-time path (App. E.2, App. F.5) against the space-time oracle:
the operator S_st = I + alpha F^T F, the Kronecker basis I_nt (x) Z_s, and
whole primal active-set solves (FP64 A-DEF2 with the Kronecker basis, the
constant-in-time lift, and plain PCG) compared state by state and active set
by active set."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from oracle import spacetime_oracle as ST  # noqa: E402
from paper_2606_17971_b300 import workloads as W  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def sdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_17971_b300 import sdf as S
    return S


def _gpu_problem(sdf, w, n, n_t):
    return sdf.Problem(3, (n, n, n_t), alpha=w.alpha, yd_sigma=w.sigma, time_axis=True,
                       t_final=w.extra["t_final"], ramp_tau=w.extra["ramp_tau"])


def test_space_time_operator_matches_oracle(sdf):
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t = 12, 6
    G = _gpu_problem(sdf, w, n, n_t)
    _, S = ST.problem(n, n_t, w.alpha, T=w.extra["t_final"])
    rng = np.random.default_rng(7)
    u = rng.standard_normal(G.N)
    inst = torch.as_tensor([[1.0, 0.5, 0.5, 0, 0, 0, 0]], dtype=torch.float64, device=DEV)
    out = G.apply_S(inst, torch.as_tensor(u, device=DEV), mode=1).cpu().numpy()
    ref = S @ u
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)
    # b_z of an instance is ignored on the time axis (b_x, b_y too without convection)
    inst2 = torch.as_tensor([[1.0, 0.5, 0.5, 0, 0.3, -0.2, 5.0]], dtype=torch.float64, device=DEV)
    out2 = G.apply_S(inst2, torch.as_tensor(u, device=DEV), mode=1).cpu().numpy()
    np.testing.assert_array_equal(out2, out)


def test_kronecker_basis_matches_oracle(sdf):
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = 10, 5, 6
    G2 = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma)
    G = _gpu_problem(sdf, w, n, n_t)
    for dt in (sdf.F64, sdf.BF16):
        zs, _ = G2.analytic_modes(r, dt)
        phi = G.spacetime_kron_modes(zs)
        ref = ST.kron_basis(zs.to(torch.float64).cpu().numpy().T, n_t)
        np.testing.assert_array_equal(phi.to(torch.float64).cpu().numpy().T, ref)
    with pytest.raises(sdf.SdfError):
        G.analytic_modes(4)
    with pytest.raises(sdf.SdfError):
        G2.spacetime_kron_modes(zs)


@pytest.mark.parametrize("basis", ["kron", "const", "plain"])
def test_space_time_solves_match_oracle(sdf, basis):
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = 24, 8, 8
    G = _gpu_problem(sdf, w, n, n_t)
    P, _ = ST.problem(n, n_t, w.alpha, T=w.extra["t_final"])
    zs, _ = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma).analytic_modes(r)
    Zs = zs.cpu().numpy().T
    if basis == "kron":
        phi = G.spacetime_kron_modes(zs)
        Phi = ST.kron_basis(Zs, n_t)
    elif basis == "const":
        Phi = ST.constant_lift(Zs, n_t)
        phi = torch.as_tensor(np.ascontiguousarray(Phi.T), device=DEV)
    else:
        phi, Phi = None, None
    if phi is not None:
        G.set_modes(phi)
    insts = W.draw_instances(W.scaled(w, n), count=6)
    psi = np.ones(G.N)
    gpu = G.solve(torch.as_tensor(W.instances_array(insts), device=DEV),
                  torch.as_tensor(psi, device=DEV),
                  sdf.default_opts(deflate=int(phi is not None)), want_lambda=False)
    assert gpu["status"] == 0
    some_active = False
    for b, ins in enumerate(insts):
        _, rhs = ST.desired_state(n, n_t, ins.a, ins.c[:2], sigma=w.sigma,
                                  tau=w.extra["ramp_tau"], T=w.extra["t_final"])
        orc = P.solve(rhs, psi, Phi, deflate=Phi is not None)
        st = gpu["stats"][b]
        assert st["status"] == 0 == orc["status"]
        act = gpu["active"][b].cpu().numpy().astype(bool)
        assert np.array_equal(act, orc["active"]), b
        some_active |= bool(act.any())
        assert st["outer_iters"] == orc["outer_iters"] and st["n_active"] == orc["n_active"]
        y = gpu["y"][b].cpu().numpy()
        assert np.linalg.norm(y - orc["y"]) <= 1e-6 * np.linalg.norm(orc["y"]), b
        # the constant lift deflates almost nothing: its count is that of a
        # slowly converging PCG tail, which summation order moves by a few
        # percent (2.6 % seen); the others within max(3, 2 %)
        rel = 0.03 if basis == "const" else 0.02
        for ig, io in zip(st["cg_iters"], orc["cg_iters"]):
            assert abs(ig - io) <= max(3, rel * io), (b, st["cg_iters"], orc["cg_iters"])
    assert some_active


def test_kronecker_basis_cuts_gpu_iterations(sdf):
    # App. E.2.1 / Sec. 4.3 on the GPU: Kronecker basis well over half, the
    # constant-in-time lift almost nothing
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = w.n, w.extra["n_t"], w.k
    G = _gpu_problem(sdf, w, n, n_t)
    zs, _ = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma).analytic_modes(r)
    inst = torch.as_tensor(W.instances_array(W.draw_instances(w, count=4)), device=DEV)
    psi = torch.full((G.N,), 10.0, dtype=torch.float64, device=DEV)  # inactive: one solve
    plain = G.solve(inst, psi, sdf.default_opts(deflate=0), want_lambda=False)
    G.set_modes(G.spacetime_kron_modes(zs))
    kron = G.solve(inst, psi, want_lambda=False)
    lift = torch.as_tensor(np.ascontiguousarray(ST.constant_lift(zs.cpu().numpy().T, n_t).T),
                           device=DEV)
    G.set_modes(lift)
    const = G.solve(inst, psi, want_lambda=False)
    for b in range(4):
        c0 = plain["stats"][b]["cg_iters"][0]
        assert kron["stats"][b]["cg_iters"][0] < 0.5 * c0
        assert const["stats"][b]["cg_iters"][0] > 0.8 * c0
    assert (kron["y"] - plain["y"]).abs().max().item() <= 1e-6 * plain["y"].abs().max().item()


def test_mixed_path_refuses_space_time(sdf):
    w = W.WORKLOADS["spacetime2d_64"]
    G = _gpu_problem(sdf, w, 8, 4)
    inst = torch.as_tensor([[1.0, 0.5, 0.5, 0, 0, 0, 0]], dtype=torch.float64, device=DEV)
    with pytest.raises(sdf.SdfError):
        G.solve(inst, torch.ones(G.N, dtype=torch.float64, device=DEV),
                sdf.default_opts(precision=sdf.PREC_MIXED), raise_on_fail=True)


def test_cosine_temporal_basis_matches_oracle(sdf):
    # App. E.2.1: W_t (x) Z_s with W_t the DCT-II columns
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = 20, 8, 6
    for rt in (8, 3):
        np.testing.assert_allclose(sdf.dct2_basis(n_t, rt), ST.dct2_basis(n_t, rt), atol=1e-15)
    G = _gpu_problem(sdf, w, n, n_t)
    zs, _ = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma).analytic_modes(r)
    Zs = zs.cpu().numpy().T
    Wt = sdf.dct2_basis(n_t, 3)
    phi = G.spacetime_modes(Wt, zs)
    np.testing.assert_array_equal(phi.cpu().numpy().T, ST.temporal_basis(Wt, Zs))
    np.testing.assert_array_equal(G.spacetime_modes(np.eye(n_t), zs).cpu().numpy(),
                                  G.spacetime_kron_modes(zs).cpu().numpy())
    # a truncated cosine basis: the whole solve against the oracle
    P, _ = ST.problem(n, n_t, w.alpha, T=w.extra["t_final"])
    G.set_modes(phi)
    insts = W.draw_instances(W.scaled(w, n), count=4)
    psi = np.ones(G.N)
    gpu = G.solve(torch.as_tensor(W.instances_array(insts), device=DEV),
                  torch.as_tensor(psi, device=DEV), want_lambda=False)
    for b, ins in enumerate(insts):
        _, rhs = ST.desired_state(n, n_t, ins.a, ins.c[:2], sigma=w.sigma,
                                  tau=w.extra["ramp_tau"], T=w.extra["t_final"])
        orc = P.solve(rhs, psi, ST.temporal_basis(Wt, Zs))
        st = gpu["stats"][b]
        assert np.array_equal(gpu["active"][b].cpu().numpy().astype(bool), orc["active"])
        assert st["outer_iters"] == orc["outer_iters"]
        y = gpu["y"][b].cpu().numpy()
        assert np.linalg.norm(y - orc["y"]) <= 1e-6 * np.linalg.norm(orc["y"])
        for ig, io in zip(st["cg_iters"], orc["cg_iters"]):
            assert abs(ig - io) <= max(3, 0.02 * io), (b, st["cg_iters"], orc["cg_iters"])


def test_full_cosine_basis_deflates_like_kronecker_on_gpu(sdf):
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = 32, 8, 16
    G = _gpu_problem(sdf, w, n, n_t)
    zs, _ = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma).analytic_modes(r)
    inst = torch.as_tensor(W.instances_array(W.draw_instances(W.scaled(w, n), count=2)), device=DEV)
    psi = torch.full((G.N,), 10.0, dtype=torch.float64, device=DEV)
    its = {}
    for name, phi in (("kron", G.spacetime_kron_modes(zs)),
                      ("full", G.spacetime_modes(sdf.dct2_basis(n_t, n_t), zs)),
                      ("half", G.spacetime_modes(sdf.dct2_basis(n_t, n_t // 2), zs))):
        G.set_modes(phi)
        its[name] = [s["cg_iters"][0] for s in G.solve(inst, psi, want_lambda=False)["stats"]]
    for b in range(2):
        assert abs(its["full"][b] - its["kron"][b]) <= max(3, 0.02 * its["kron"][b]), its
        assert its["half"][b] > its["kron"][b] + 5, its


def test_space_time_eigenmodes_span_the_kronecker_basis(sdf):
    # App. E.2.1 compares eigenmodes of the space-time operator with the
    # Kronecker basis.  With constant kappa and no convection the spatial
    # sines diagonalise S_st, and here its r n_t lowest eigenvectors span
    # I_nt (x) Z_s(r) exactly, so the two bases deflate alike
    w = W.WORKLOADS["spacetime2d_64"]
    n, n_t, r = 24, 8, 4
    G = _gpu_problem(sdf, w, n, n_t)
    zs, _ = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma).analytic_modes(r)
    kron = G.spacetime_kron_modes(zs)
    G.set_modes(kron)
    inst = torch.as_tensor([[2.0, 0.45, 0.55, 0, 0, 0, 0]], dtype=torch.float64, device=DEV)
    act = torch.zeros(G.N, dtype=torch.uint8, device=DEV)
    V, lam, st = G.restricted_modes(inst[0], act, r * n_t)
    assert st["converged"], st
    _, srt = G.diag_angles(act, V, sorted_angles=True)
    assert srt.max() < 1e-5, srt.max()
    _, S = ST.problem(n, n_t, w.alpha, T=w.extra["t_final"])
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(S.toarray())[:r * n_t], rtol=1e-9)
    psi = torch.full((G.N,), 10.0, dtype=torch.float64, device=DEV)
    it_kron = G.solve(inst, psi, want_lambda=False)["stats"][0]["cg_iters"][0]
    G.set_modes(V)
    it_eig = G.solve(inst, psi, want_lambda=False)["stats"][0]["cg_iters"][0]
    assert abs(it_eig - it_kron) <= 3, (it_eig, it_kron)
