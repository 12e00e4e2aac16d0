"""GPU spectral diagnostics against the oracle: active-set distances (exact
counts, weighted distance over F64 and BF16 modes), operator drift by
Lanczos against dense 2-norms, restricted eigenpairs of S_II against dense
eigh (with and without convection), and the cutoff principal angles."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import diag_oracle as D  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2606_17971_b300 import workloads as W  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def sdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_17971_b300 import sdf as S
    return S


def _disc(n, c, r2):
    """Active set shaped like a constrained peak: the nodes within a disc."""
    nx, ny = n
    x = (np.arange(nx) + 1) / (nx + 1)
    y = (np.arange(ny) + 1) / (ny + 1)
    gy, gx = np.meshgrid(y, x, indexing="ij")
    return (((gx - c[0]) ** 2 + (gy - c[1]) ** 2) < r2).ravel().astype(np.uint8)


def _block_problem(n=(48, 40)):
    w = W.scaled(W.WORKLOADS["block2d_1024"], 48)
    kap = np.ascontiguousarray(W.kappa_field(w).reshape(48, 48)[: n[1], : n[0]]).ravel()
    return w, kap


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_active_set_distances_match_oracle(sdf, dtype):
    n = (48, 40)
    w, kap = _block_problem(n)
    G = sdf.Problem(2, n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    k = 24
    phi, _ = G.analytic_modes(k, sdf.BF16 if dtype == "bf16" else sdf.F64)
    G.set_modes(phi)
    Phi_stored = phi.to(torch.float64).cpu().numpy().T  # the modes as stored
    ref = _disc(n, (0.5, 0.5), 0.04)
    masks = [ref, np.zeros_like(ref), np.ones_like(ref), _disc(n, (0.55, 0.45), 0.05),
             _disc(n, (0.3, 0.7), 0.01), 1 - ref]
    act = torch.as_tensor(np.stack(masks), device=DEV)
    for r in (0, 1, 7, k):
        out = G.diag_active_sets(torch.as_tensor(ref, device=DEV), act, r=r)
        for b, m in enumerate(masks):
            sym, na = D.active_set_counts(ref, m)
            assert out["sym_diff"][b] == sym and out["n_active"][b] == na
            assert out["delta"][b] == D.delta(ref, m) and out["rho"][b] == D.rho(m)
            if r > 0:
                assert out["delta_w"][b] == pytest.approx(D.delta_w(ref, m, Phi_stored, r),
                                                          rel=1e-12, abs=1e-15)
    with pytest.raises(sdf.SdfError):
        G.diag_active_sets(torch.as_tensor(ref, device=DEV), act, r=k + 1)


def test_active_set_counts_full_size_batch(sdf):
    # 512^2, 256 masks: counts exact against numpy
    w = W.WORKLOADS["convdiff2d_512"]
    G = sdf.Problem(2, w.n, alpha=w.alpha, diff_scale=w.diff_scale, convection=True,
                    yd_sigma=w.sigma)
    rng = np.random.default_rng(3)
    ref = (rng.random(w.N) < 0.05).astype(np.uint8)
    act = (rng.random((256, w.N)) < rng.random((256, 1)) * 0.2).astype(np.uint8)
    out = G.diag_active_sets(torch.as_tensor(ref, device=DEV), torch.as_tensor(act, device=DEV))
    np.testing.assert_array_equal(out["sym_diff"], np.count_nonzero(act != ref[None], axis=1))
    np.testing.assert_array_equal(out["n_active"], np.count_nonzero(act, axis=1))


def test_drift_matches_dense_two_norms(sdf):
    # convection-diffusion on 16^2 (N = 256): steps >= N makes Lanczos exact
    n, alpha, eps_d = 16, 1e-3, 1e-2
    G = sdf.Problem(2, n, alpha=alpha, diff_scale=eps_d, convection=True, yd_sigma=0.1)
    thetas = [0.0, 0.4, 2.0, np.pi]
    rows = [[1.0, 0.5, 0.5, 0, np.cos(t), np.sin(t), 0] for t in thetas] + [[1.0, 0.5, 0.5, 0, 0, 0, 0]]
    inst = torch.as_tensor(rows, dtype=torch.float64, device=DEV)
    ref_row = torch.as_tensor([1.0, 0.5, 0.5, 0, 0, 0, 0], dtype=torch.float64, device=DEV)
    eps, nref = G.diag_drift(ref_row, inst, steps=300)
    Sref = O.Problem(2, n, alpha=alpha, diff_scale=eps_d, b=(0.0, 0.0)).dense_S()
    for b, t in enumerate(thetas):
        Sm = O.Problem(2, n, alpha=alpha, diff_scale=eps_d, b=(np.cos(t), np.sin(t))).dense_S()
        e_o, n_o = D.drift(Sref, Sm)
        assert eps[b] == pytest.approx(e_o, rel=1e-10), (t, eps[b], e_o)
        assert nref == pytest.approx(n_o, rel=1e-12)
    assert eps[-1] == 0.0  # the reference itself: no drift, exactly


def test_drift_lanczos_lower_bound_and_zero_without_convection(sdf):
    n, alpha, eps_d = 24, 1e-3, 1e-2
    G = sdf.Problem(2, n, alpha=alpha, diff_scale=eps_d, convection=True, yd_sigma=0.1)
    inst = torch.as_tensor([[1.0, 0.5, 0.5, 0, np.cos(1.0), np.sin(1.0), 0]],
                           dtype=torch.float64, device=DEV)
    ref_row = torch.as_tensor([1.0, 0.5, 0.5, 0, 0, 0, 0], dtype=torch.float64, device=DEV)
    eps, _ = G.diag_drift(ref_row, inst, steps=120)
    Sref = O.Problem(2, n, alpha=alpha, diff_scale=eps_d, b=(0.0, 0.0)).dense_S()
    Sm = O.Problem(2, n, alpha=alpha, diff_scale=eps_d, b=(np.cos(1.0), np.sin(1.0))).dense_S()
    e_o, _ = D.drift(Sref, Sm)
    # fewer steps than the dimension (576): a lower bound, here converged
    assert eps[0] <= e_o * (1 + 1e-12) and eps[0] >= e_o * (1 - 1e-6)
    # a 3D diffusion problem has no instance-dependent part: eps = 0 exactly
    G3 = sdf.Problem(3, 12, alpha=1e-4, yd_sigma=0.1)
    i3 = torch.as_tensor(W.instances_array(W.draw_instances(W.scaled(W.WORKLOADS["diff3d_128"], 12),
                                                            count=3)), device=DEV)
    e3, n3 = G3.diag_drift(i3[0], i3, steps=16)
    assert np.all(e3 == 0.0) and n3 > 0


@pytest.mark.parametrize("conv", [False, True])
def test_restricted_modes_match_dense_eigh_and_interlace(sdf, conv):
    if conv:
        n, kap, alpha, ds = (40, 36), None, 1e-3, 1e-2
        b = (np.cos(0.7), np.sin(0.7))
        P = O.Problem(2, n, alpha=alpha, diff_scale=ds, b=b)
        G = sdf.Problem(2, n, alpha=alpha, diff_scale=ds, convection=True, yd_sigma=0.1)
        inst = torch.as_tensor([1.0, 0.5, 0.5, 0, b[0], b[1], 0], dtype=torch.float64, device=DEV)
    else:
        n = (48, 40)
        w, kap = _block_problem(n)
        alpha = w.alpha
        P = O.Problem(2, n, kappa=kap, alpha=alpha)
        G = sdf.Problem(2, n, alpha=alpha, kappa=kap, yd_sigma=w.sigma)
        inst = torch.as_tensor([1.0, 0.5, 0.5, 0, 0, 0, 0], dtype=torch.float64, device=DEV)
    act = _disc(n, (0.6, 0.4), 0.03)
    k = 12
    V, lam, st = G.restricted_modes(inst, torch.as_tensor(act, device=DEV), k)
    assert st["converged"], st
    S = P.dense_S()
    lam_o, V_o = D.restricted_modes(S, act, k)
    np.testing.assert_allclose(lam, lam_o, rtol=1e-9)
    Vg = V.cpu().numpy().T
    assert np.all(Vg[act.astype(bool)] == 0.0)
    np.testing.assert_allclose(Vg.T @ Vg, np.eye(k), atol=1e-12)
    for j in range(k):  # simple eigenvalues here: each vector up to sign
        assert abs(Vg[:, j] @ V_o[:, j]) > 1 - 1e-8, j
    # Cauchy interlacing against the full spectrum (App. A.2)
    lf = np.linalg.eigvalsh(S)
    nA = int(act.sum())
    # margin: Rayleigh-Ritz rounding is about eps ||S|| (8e-11 here)
    assert np.all(lf[:k] <= lam * (1 + 1e-9)) and np.all(lam <= lf[nA:nA + k] * (1 + 1e-9))


def test_cutoff_angles_match_oracle(sdf):
    n = (48, 40)
    w, kap = _block_problem(n)
    P = O.Problem(2, n, kappa=kap, alpha=w.alpha)
    G = sdf.Problem(2, n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    k = 16
    phi, _, _, st = G.eig_modes(k, tol=1e-10)  # reference modes of the full operator
    assert st["converged"]
    G.set_modes(phi)
    inst = torch.as_tensor([1.0, 0.5, 0.5, 0, 0, 0, 0], dtype=torch.float64, device=DEV)
    for act in (np.zeros(P.N, np.uint8), _disc(n, (0.6, 0.4), 0.03), _disc(n, (0.4, 0.5), 0.08)):
        a_t = torch.as_tensor(act, device=DEV)
        V, _, st = G.restricted_modes(inst, a_t, k)
        assert st["converged"]
        th, srt = G.diag_angles(a_t, V, sorted_angles=True)
        Phi_I = D.restrict(phi.cpu().numpy().T, act)
        th_o = D.cutoff_angles(Phi_I, V.cpu().numpy().T)
        np.testing.assert_allclose(th, th_o, atol=2e-6)
        np.testing.assert_allclose(srt, D.principal_angles(Phi_I, V.cpu().numpy().T), atol=2e-6)
        assert srt[-1] == pytest.approx(th[-1], abs=2e-6)
        if act.sum() == 0:
            assert th.max() < 1e-5  # the same operator: aligned at every cut
        else:
            assert th.max() > 1e-3  # restriction rotates the modes


def test_diagnostics_refuse_bad_arguments(sdf):
    G = sdf.Problem(2, 16, alpha=1e-3, yd_sigma=0.1)
    inst = torch.as_tensor([1.0, 0.5, 0.5, 0, 0, 0, 0], dtype=torch.float64, device=DEV)
    act = torch.zeros(G.N, dtype=torch.uint8, device=DEV)
    with pytest.raises(sdf.SdfError):
        G.diag_drift(inst, inst, steps=0)
    with pytest.raises(sdf.SdfError):
        G.diag_drift(inst, inst, steps=2000)
    nearly_all = torch.ones(G.N, dtype=torch.uint8, device=DEV)
    nearly_all[:10] = 0
    with pytest.raises(sdf.SdfError):  # |I| = 10 < k + guard
        G.restricted_modes(inst, nearly_all, 4)
    with pytest.raises(sdf.SdfError):  # no registered modes
        G.diag_angles(act, torch.zeros((4, G.N), dtype=torch.float64, device=DEV))


def test_two_regime_spectral_coherence_on_a_sweep(sdf):
    # Sec. 4.1: over instances whose active sets differ by up to ~20 % of the
    # nodes, the r-th smallest principal angle between the restricted
    # reference modes and S_II's lowest eigenvectors stays small while the
    # largest approaches 90 degrees; deflation stays effective
    n, K, r = 48, 40, 20
    w = W.scaled(W.WORKLOADS["diff2d_32"], n)
    G = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma)
    phiK, _ = G.analytic_modes(K)
    insts = W.draw_instances(w, count=4)
    inst = torch.as_tensor(W.instances_array(insts), device=DEV)
    psi = torch.full((G.N,), 0.5, dtype=torch.float64, device=DEV)
    G.set_modes(phiK[:r].contiguous())
    defl = G.solve(inst, psi, want_lambda=False)
    cold = G.solve(inst, psi, sdf.default_opts(deflate=0), want_lambda=False)
    G.set_modes(phiK)
    P = O.Problem(2, n, alpha=w.alpha)
    S = P.dense_S()
    Phi = phiK.cpu().numpy().T
    for b in range(4):
        act = defl["active"][b].contiguous()
        assert 0 < int(act.sum().item()) < G.N // 4
        V, _, st = G.restricted_modes(inst[b], act, K)
        assert st["converged"]
        _, srt = G.diag_angles(act, V, sorted_angles=True)
        assert np.degrees(srt[r - 1]) < 5.0 and np.degrees(srt[-1]) > 60.0, np.degrees(srt)
        # the same angles from the oracle's dense restricted eigenvectors
        a_np = act.cpu().numpy()
        _, V_o = D.restricted_modes(S, a_np, K)
        srt_o = D.principal_angles(D.restrict(Phi, a_np), V_o)
        assert abs(np.degrees(srt[r - 1]) - np.degrees(srt_o[r - 1])) < 0.05
        eff = 1 - sum(defl["stats"][b]["cg_iters"]) / sum(cold["stats"][b]["cg_iters"])
        assert eff > 0.5


def test_true_relative_residual_matches_dense_recomputation(sdf):
    # App. B.2: the solve stops on the recurrence residual; the diagnostic
    # recomputes ||b_I - S_II y_I|| / ||b_I|| from the solve's outputs
    n = (48, 40)
    w, kap = _block_problem(n)
    P = O.Problem(2, n, kappa=kap, alpha=w.alpha)
    G = sdf.Problem(2, n, alpha=w.alpha, kappa=kap, yd_sigma=w.sigma)
    Phi = O.dense_modes(P, 16)[0]
    G.set_modes(torch.as_tensor(np.ascontiguousarray(Phi.T), device=DEV))
    insts = W.draw_instances(w, count=5)
    inst = torch.as_tensor(W.instances_array(insts), device=DEV)
    psi_np = np.ones(P.N)
    out = G.solve(inst, torch.as_tensor(psi_np, device=DEV), want_lambda=True)
    rel = G.diag_relres(out, inst)
    S = P.dense_S()
    some_active = False
    for b, ins in enumerate(insts):
        rhs = P.desired_state(ins.a, ins.c[:2], w.sigma)[1]
        act = out["active"][b].cpu().numpy().astype(bool)
        some_active |= bool(act.any())
        y = out["y"][b].cpu().numpy()
        bI = (rhs - S @ (psi_np * act))[~act]
        rI = (rhs - S @ y)[~act]
        want = np.linalg.norm(rI) / np.linalg.norm(bI)
        # r = rhs - S y cancels to 1e-8 of terms as large as ||S|| |y|, so
        # two FP64 summation orders agree to a few digits only (3e-5 seen)
        assert rel[b] == pytest.approx(want, rel=1e-3, abs=1e-14)
        assert rel[b] <= 1.5e-8
    assert some_active
