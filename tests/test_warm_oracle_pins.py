"""Pins of the learned-warm-start oracle (oracle/warm_oracle.py) against what
mathematics and independent library routines fix: BF16 rounding against
torch's conversion, GELU against its closed form and torch, the backward pass
against central finite differences and torch autograd, Adam against
torch.optim.Adam, and the POD against the method of snapshots."""
import numpy as np
import pytest
import torch

from oracle import warm_oracle as WO


def test_bf16_rounding_is_round_to_nearest_even():
    one = 1.0
    ulp = 2.0 ** -7                      # BF16 spacing just above 1
    cases = {
        one: one,
        one + ulp / 2: one,                 # tie -> even (mantissa 0)
        one + 3 * ulp / 2: one + 2 * ulp,   # tie -> even (mantissa 2)
        one + 0.51 * ulp: one + ulp,
        -(one + 0.49 * ulp): -one,
    }
    for x, want in cases.items():
        assert WO.bf16(np.array([x]))[0] == want
    rng = np.random.default_rng(1)
    x = rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(WO.bf16(x), want)


def test_gelu_closed_form_and_library():
    # Phi(1) = 0.841344746068543 (standard normal CDF)
    assert abs(WO.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(WO.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    assert WO.gelu(np.array([0.0]))[0] == 0.0
    z = np.linspace(-8, 8, 1001)
    want = torch.nn.functional.gelu(torch.from_numpy(z), approximate="none").numpy()
    np.testing.assert_allclose(WO.gelu(z), want, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (WO.gelu(z + h) - WO.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(WO.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_backward_matches_central_differences():
    widths = (4, 8, 8, 3)
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(WO.n_params(widths)) * 0.5
    X = rng.uniform(-1, 1, (6, 4))
    T = rng.standard_normal((6, 3))
    _, g = WO.loss_and_grad(theta, X, T, widths, exact=True)
    h = 1e-6
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        lp, _ = WO.loss_and_grad(theta + e, X, T, widths, exact=True)
        lm, _ = WO.loss_and_grad(theta - e, X, T, widths, exact=True)
        assert abs((lp - lm) / (2 * h) - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_backward_matches_torch_autograd_at_full_width():
    rng = np.random.default_rng(3)
    widths = WO.WIDTHS
    theta = rng.standard_normal(WO.n_params(widths)) * 0.05
    X = rng.uniform(-1, 1, (40, 4))
    T = rng.standard_normal((40, 64))
    loss, g = WO.loss_and_grad(theta, X, T, widths, exact=True)
    th = torch.tensor(theta, requires_grad=True)
    a = torch.from_numpy(X)
    o = 0
    for li in range(len(widths) - 1):
        fi, fo = widths[li], widths[li + 1]
        W = th[o:o + fo * fi].view(fo, fi)
        o += fo * fi
        b = th[o:o + fo]
        o += fo
        a = a @ W.T + b
        if li < len(widths) - 2:
            a = torch.nn.functional.gelu(a, approximate="none")
    lt = ((a - torch.from_numpy(T)) ** 2).mean()
    lt.backward()
    assert abs(lt.item() - loss) < 1e-12 * abs(loss)
    np.testing.assert_allclose(g, th.grad.numpy(), rtol=1e-9, atol=1e-14)


def test_bf16_rounded_gradient_stays_close_to_exact():
    # the rounded variant differs from the exact one by BF16 operand rounding
    # only: relative error a few times 2^-8
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(WO.n_params()) * 0.05
    X = rng.uniform(-1, 1, (64, 4))
    T = rng.standard_normal((64, 64))
    _, ge = WO.loss_and_grad(theta, X, T, exact=True)
    _, gr = WO.loss_and_grad(theta, X, T, exact=False)
    assert np.linalg.norm(gr - ge) / np.linalg.norm(ge) < 2e-2


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.standard_normal(50)
        theta, m, v = WO.adam(theta, g, m, v, step, 1e-2)
        p.grad = torch.from_numpy(g.copy())
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_pod_matches_method_of_snapshots():
    rng = np.random.default_rng(6)
    m, N, r = 12, 300, 5
    Y = rng.standard_normal((m, 3)) @ rng.standard_normal((3, N)) + 0.01 * rng.standard_normal((m, N))
    ybar, Psi, s, coef = WO.pod(Y, r)
    np.testing.assert_allclose(ybar, Y.mean(axis=0))
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(r), atol=1e-12)
    # method of snapshots: eigenvalues of the centred Gram are s^2
    Yc = Y - Y.mean(axis=0)
    lam = np.sort(np.linalg.eigvalsh(Yc @ Yc.T))[::-1]
    np.testing.assert_allclose(s ** 2, lam[:r], rtol=1e-10)
    np.testing.assert_allclose(coef, Yc @ Psi, atol=1e-12)
    # full rank m-1 reconstructs the snapshots
    ybar, Psi, s, coef = WO.pod(Y, m - 1)
    np.testing.assert_allclose(ybar + coef @ Psi.T, Y, atol=1e-10)
    # sign rule: largest-magnitude entry of each column is positive
    for j in range(Psi.shape[1]):
        assert Psi[np.argmax(np.abs(Psi[:, j])), j] > 0


def test_scaling_maps_box_to_unit_cube():
    lo = np.array([1.0, 0.25, 0.25, 0.25])
    hi = np.array([3.0, 0.75, 0.75, 0.75])
    np.testing.assert_allclose(WO.scale_inputs(lo[None], lo, hi), -np.ones((1, 4)))
    np.testing.assert_allclose(WO.scale_inputs(hi[None], lo, hi), np.ones((1, 4)))
    np.testing.assert_allclose(WO.scale_inputs(((lo + hi) / 2)[None], lo, hi), np.zeros((1, 4)))


def test_cosine_schedule_endpoints():
    assert WO.cosine_lr(1, 100, 1e-3) == pytest.approx(1e-3)
    assert WO.cosine_lr(51, 100, 1e-3) == pytest.approx(5e-4)
    assert WO.cosine_lr(101, 100, 1e-3) == pytest.approx(0.0, abs=1e-18)
