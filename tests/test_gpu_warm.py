"""GPU parity of the learned warm start against the oracle (oracle/warm_oracle.py):
the tensor-core MLP forward pass and gradient, Adam, the POD, the expansion
x0 = ybar + Psi c, and the solver started from x0."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import warm_oracle as WO  # noqa: E402


@pytest.fixture(scope="module")
def sdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_17971_b300 import sdf as S
    return S


def _theta(widths, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(widths) - 1):
        fi, fo = widths[i], widths[i + 1]
        parts.append(rng.standard_normal(fo * fi) * scale / np.sqrt(fi))
        parts.append(rng.standard_normal(fo) * 0.1)
    return np.concatenate(parts).astype(np.float32)


@pytest.mark.parametrize("widths,batch", [((4, 256, 256, 256, 64), 200),
                                          ((3, 48, 256, 16), 37),
                                          ((4, 256, 256, 256, 64), 300)])
def test_mlp_forward_matches_oracle(sdf, widths, batch):
    # ragged batches (not multiples of 128) and widths that are not multiples of 16
    theta = _theta(widths, 1)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (batch, widths[0])).astype(np.float32)
    mlp = sdf.Mlp(widths)
    y = mlp.forward(torch.from_numpy(theta).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    _, A = WO.forward(theta.astype(np.float64), X.astype(np.float64), widths)
    want = A[-1]
    err = np.abs(y - want).max() / np.abs(want).max()
    assert err < 2e-3, err
    # and BF16 operands keep it within a few 2^-8 of the exact FP64 network
    _, Ae = WO.forward(theta.astype(np.float64), X.astype(np.float64), widths, exact=True)
    assert np.linalg.norm(y - Ae[-1]) / np.linalg.norm(Ae[-1]) < 3e-2


@pytest.mark.parametrize("batch", [200, 128])
def test_mlp_loss_gradient_matches_oracle(sdf, batch):
    widths = (4, 256, 256, 256, 64)
    theta = _theta(widths, 3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (batch, 4)).astype(np.float32)
    T = rng.standard_normal((batch, 64)).astype(np.float32)
    mlp = sdf.Mlp(widths)
    loss, g = mlp.loss_grad(torch.from_numpy(theta).cuda(), torch.from_numpy(X).cuda(),
                            torch.from_numpy(T).cuda())
    loss, g = loss.item(), g.cpu().numpy().astype(np.float64)
    lw, gw = WO.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                              T.astype(np.float64), widths)
    assert abs(loss - lw) < 1e-4 * lw
    off = 0
    for li in range(len(widths) - 1):
        n = widths[li + 1] * widths[li] + widths[li + 1]
        a, b = g[off:off + n], gw[off:off + n]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-2, li
        off += n
    assert np.linalg.norm(g - gw) / np.linalg.norm(gw) < 5e-3


def test_adam_matches_oracle(sdf):
    rng = np.random.default_rng(5)
    n = 10007
    theta = rng.standard_normal(n).astype(np.float32)
    m = np.zeros(n)
    v = np.zeros(n)
    th = torch.from_numpy(theta.copy()).cuda()
    md = torch.zeros(n, device="cuda")
    vd = torch.zeros(n, device="cuda")
    t64 = theta.astype(np.float64)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        lr = WO.cosine_lr(step, 3, 1e-2)
        sdf.adam_step(th, torch.from_numpy(g).cuda(), md, vd, step, float(lr))
        t64, m, v = WO.adam(t64, g.astype(np.float64), m, v, step, lr)
    np.testing.assert_allclose(th.cpu().numpy(), t64, rtol=0, atol=1e-5)


def test_pod_matches_oracle(sdf):
    rng = np.random.default_rng(6)
    m, N, r = 40, 5003, 16
    # decaying spectrum, distinct singular values
    U = np.linalg.qr(rng.standard_normal((N, m)))[0]
    s = 10.0 ** -np.linspace(0, 3, m)
    Y = (U * s) @ rng.standard_normal((m, m)).T + 0.3
    Y = Y.T.copy()  # m x N
    ybar, psi_rm, psi_cm, sing, coef = sdf.pod(torch.from_numpy(Y).cuda(), r)
    yb, Psi, sw, cw = WO.pod(Y, r)
    np.testing.assert_allclose(ybar.cpu().numpy(), yb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(sing, sw, rtol=1e-9)
    np.testing.assert_allclose(psi_cm.cpu().numpy().T, Psi, rtol=0, atol=1e-8)
    np.testing.assert_allclose(coef, cw, rtol=0, atol=1e-8 * np.abs(cw).max())
    # the BF16 node-major copy is the rounded FP64 basis
    np.testing.assert_array_equal(psi_rm.float().cpu().numpy().astype(np.float64),
                                  WO.bf16(psi_cm.cpu().numpy().T))


def test_warm_expand_matches_numpy(sdf):
    rng = np.random.default_rng(7)
    N, r, B = 3001, 64, 21   # ragged node count and batch
    psi = WO.bf16(rng.standard_normal((N, r)) / np.sqrt(N))
    ybar = rng.standard_normal(N)
    cstd = rng.standard_normal((B, r)).astype(np.float32)
    cmean = rng.standard_normal(r).astype(np.float32)
    cscale = rng.uniform(0.5, 2, r).astype(np.float32)
    x0 = sdf.warm_expand(torch.from_numpy(psi).to(torch.bfloat16).cuda(),
                         torch.from_numpy(ybar).cuda(), torch.from_numpy(cstd).cuda(),
                         torch.from_numpy(cmean).cuda(), torch.from_numpy(cscale).cuda())
    c = WO.bf16(cstd.astype(np.float32) * cscale + cmean)
    want = ybar[None, :] + c @ psi.T
    err = np.abs(x0.cpu().numpy() - want).max() / np.abs(want).max()
    assert err < 1e-5, err


def _diff2d(sdf):
    from paper_2606_17971_b300 import workloads as W
    w = W.WORKLOADS["diff2d_32"]
    G = sdf.Problem(2, w.n, alpha=w.alpha, yd_sigma=w.sigma)
    phi, _ = G.analytic_modes(w.k)
    G.set_modes(phi)
    psi = torch.full((w.N,), w.psi, dtype=torch.float64, device="cuda")
    return W, w, G, psi


def test_zero_start_reproduces_cold_solve(sdf):
    W, w, G, psi = _diff2d(sdf)
    inst = torch.as_tensor(W.instances_array(W.draw_instances(w, count=8)), device="cuda")
    x0 = torch.zeros((8, w.N), dtype=torch.float64, device="cuda")
    # the first inner solve from x0 = 0 is the cold one, bit for bit
    one = sdf.default_opts(max_outer=1)
    cold1, warm1 = G.solve(inst, psi, one, want_lambda=False), G.solve_x0(inst, psi, x0, one)
    assert torch.equal(cold1["y"], warm1["y"])
    assert [s["cg_iters"] for s in cold1["stats"]] == [s["cg_iters"] for s in warm1["stats"]]
    # later solves continue from the previous iterate: same active sets and states
    cold = G.solve(inst, psi, want_lambda=False)
    warm = G.solve_x0(inst, psi, x0)
    assert torch.equal(cold["active"], warm["active"])
    assert (warm["y"] - cold["y"]).abs().max().item() < 1e-6
    assert [s["outer_iters"] for s in cold["stats"]] == [s["outer_iters"] for s in warm["stats"]]


def test_close_start_keeps_active_sets_and_saves_iterations(sdf):
    W, w, G, psi = _diff2d(sdf)
    inst = torch.as_tensor(W.instances_array(W.draw_instances(w, count=8)), device="cuda")
    cold = G.solve(inst, psi, want_lambda=False)
    rng = np.random.default_rng(8)
    pert = torch.from_numpy(1e-3 * rng.standard_normal((8, w.N))).cuda()
    x0 = cold["y"] * (1.0 + pert)
    warm = G.solve_x0(inst, psi, x0)
    assert torch.equal(cold["active"], warm["active"])
    assert (warm["y"] - cold["y"]).abs().max().item() < 1e-6
    ic = sum(sum(s["cg_iters"]) for s in cold["stats"])
    iw = sum(sum(s["cg_iters"]) for s in warm["stats"])
    assert iw < ic


def test_fitted_model_gives_same_active_sets_with_fewer_iterations(sdf):
    W, w, G, psi = _diff2d(sdf)
    train = W.draw_instances(w, count=256, seed=w.seed + 100)
    held = W.draw_instances(w, count=16, seed=w.seed + 200)
    it = torch.as_tensor(W.instances_array(train), device="cuda")
    ih = torch.as_tensor(W.instances_array(held), device="cuda")
    # training states: the first (unconstrained) inner solve of each instance
    Y = G.solve(it, psi, sdf.default_opts(max_outer=1), want_lambda=False)["y"]
    widths = (3, 256, 256, 256, 32)
    lo, hi = W.input_box(w)
    model = sdf.WarmModel(widths, w.N, lo, hi, torch.from_numpy(W.mlp_init(widths)).cuda())
    loss = model.fit(Y, it, epochs=2000, lr0=1e-3)
    assert np.isfinite(loss).all() and loss[-1] < 1e-3 * loss[0]
    x0 = model.predict(ih)
    cold = G.solve(ih, psi, want_lambda=False)
    warm = G.solve_x0(ih, psi, x0)
    assert torch.equal(cold["active"], warm["active"])
    assert (warm["y"] - cold["y"]).abs().max().item() < 1e-6
    ic = sum(sum(s["cg_iters"]) for s in cold["stats"])
    iw = sum(sum(s["cg_iters"]) for s in warm["stats"])
    first = G.solve(ih, psi, sdf.default_opts(max_outer=1), want_lambda=False)["y"]
    rel = (x0 - first).norm() / first.norm()
    print(f"warm-start gain: {iw} vs {ic} CG iterations, prediction error {rel.item():.3g}")
    # the prediction is a few percent off; the CG iterations this saves grow
    # only with log(1 / error)
    assert iw < ic, (iw, ic, rel.item())
    assert rel.item() < 5e-2


def test_fit_on_more_states_than_the_pod_takes(sdf):
    # 600 training states: the basis is the POD of the first 384 (compared
    # with the oracle's POD of those), the MLP is fit to the coefficients of
    # all 600 on it, and the fitted model predicts held-out first solves
    W, w, G, psi = _diff2d(sdf)
    train = W.draw_instances(w, count=600, seed=w.seed + 300)
    it = torch.as_tensor(W.instances_array(train), device="cuda")
    Y = G.solve(it, psi, sdf.default_opts(max_outer=1), want_lambda=False)["y"]
    widths = (3, 256, 256, 256, 32)
    lo, hi = W.input_box(w)
    model = sdf.WarmModel(widths, w.N, lo, hi, torch.from_numpy(W.mlp_init(widths)).cuda())
    loss = model.fit(Y, it, epochs=1000, lr0=1e-3)
    assert np.isfinite(loss).all() and loss[-1] < 1e-3 * loss[0]
    yb, Psi, _, _ = WO.pod(Y[:384].cpu().numpy(), 32)
    np.testing.assert_allclose(model.ybar.cpu().numpy(), yb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(model.psi.cpu().numpy().T, Psi, rtol=0, atol=1e-8)
    held = torch.as_tensor(W.instances_array(W.draw_instances(w, count=16, seed=w.seed + 400)),
                           device="cuda")
    first = G.solve(held, psi, sdf.default_opts(max_outer=1), want_lambda=False)["y"]
    rel = ((model.predict(held) - first).norm() / first.norm()).item()
    assert rel < 5e-2, rel


def test_learned_host_entry_matches_the_device_pipeline(sdf):
    # sdf_solve_batch_learned_host (host mu in, x0 predicted and the solve on
    # the device, host y / lambda / A out) against predict + solve_x0 on
    # device buffers: the same kernels in the same order, so bit for bit
    W, w, G, psi = _diff2d(sdf)
    train = W.draw_instances(w, count=128, seed=w.seed + 500)
    it = torch.as_tensor(W.instances_array(train), device="cuda")
    Y = G.solve(it, psi, sdf.default_opts(max_outer=1), want_lambda=False)["y"]
    widths = (3, 256, 256, 256, 32)
    lo, hi = W.input_box(w)
    model = sdf.WarmModel(widths, w.N, lo, hi, torch.from_numpy(W.mlp_init(widths)).cuda())
    model.fit(Y, it, epochs=300, lr0=1e-3)
    held = W.instances_array(W.draw_instances(w, count=11, seed=w.seed + 600))
    hd = torch.as_tensor(held, device="cuda")
    dev = G.solve_x0(hd, psi, model.predict(hd), want_lambda=True)
    lam = np.empty((11, w.N))
    host = G.solve_learned_host(model, held, psi.cpu().numpy(), lam=lam)
    assert host["status"] == 0
    assert np.array_equal(host["y"], dev["y"].cpu().numpy())
    assert np.array_equal(host["active"], dev["active"].cpu().numpy())
    assert np.array_equal(lam, dev["lam"].cpu().numpy())
    assert [s["cg_iters"] for s in host["stats"]] == [s["cg_iters"] for s in dev["stats"]]
