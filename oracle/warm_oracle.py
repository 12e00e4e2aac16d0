"""Plain FP64 oracle of the learned warm start (numpy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py import this module.  It shares
no code with the CUDA path.

The paper has no learned component (its introduction lists learned
initialisations as related work only); the warm start is the target
configuration's fourth part, read as follows:

* POD of solved states (the paper's own POD, Sec. 2.2.4 "Online POD
  enrichment", mean-centred): y_i = ybar + Psi c_i, Psi the leading left
  singular vectors of the centred snapshot matrix.
* MLP mu -> c with widths 4-256-256-256-64, exact GELU
  g(z) = z/2 (1 + erf(z / sqrt 2)) between layers, identity after the last.
  Inputs min-max scaled to [-1, 1] over the parameter box; the targets (the
  fit's business, not this module's) are the coefficients centred per
  coefficient and divided by one common scale.
* Loss: mean squared error over the batch and the coefficients.  Adam with
  bias correction (Kingma & Ba), learning rate given per step.
* Precision: the kernels multiply BF16 operands (weights, layer inputs and
  back-propagated errors) with FP32 accumulation.  The oracle rounds the
  same quantities to BF16 (round to nearest even, ``bf16``) at the same
  points and does the rest in FP64, so that the two differ only by
  accumulation order.  ``exact=True`` skips the rounding (plain FP64).

Parameters are laid out as the kernels' master copy: for each layer W
(out x in, row-major) followed by b (out).
"""
from __future__ import annotations

import numpy as np
from math import sqrt
from scipy.special import erf

WIDTHS = (4, 256, 256, 256, 64)


def bf16(x):
    """Round FP64 values to BF16 (round to nearest, ties to even), returned as
    FP64.  Values are first rounded to FP32, as the kernels hold them."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * np.exp(-0.5 * z * z) / sqrt(2.0 * np.pi)


def n_params(widths=WIDTHS):
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def unpack(theta, widths=WIDTHS):
    """Split the flat parameter vector into [(W, b), ...] views."""
    out, o = [], 0
    for i in range(len(widths) - 1):
        fi, fo = widths[i], widths[i + 1]
        W = theta[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = theta[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def forward(theta, X, widths=WIDTHS, exact=False):
    """Layer pre-activations Z_l and activations A_l (A_0 = X)."""
    rnd = (lambda a: a) if exact else bf16
    layers = unpack(np.asarray(theta, np.float64), widths)
    A = [np.asarray(X, np.float64)]
    Z = []
    for li, (W, b) in enumerate(layers):
        z = rnd(A[-1]) @ rnd(W).T + b
        Z.append(z)
        A.append(gelu(z) if li < len(layers) - 1 else z)
    return Z, A


def loss_and_grad(theta, X, T, widths=WIDTHS, exact=False):
    """MSE loss mean((f(X) - T)^2) and its gradient with respect to theta.

    Backward pass by the chain rule: dZ_L = 2 (f - T) / (m c);
    dW_l = dZ_l^T A_{l-1}, db_l = sum_rows dZ_l,
    dZ_{l-1} = (dZ_l W_l) * g'(Z_{l-1}).  BF16 rounding (unless exact) of
    dZ_l, A_{l-1} and W_l where the kernels round them."""
    rnd = (lambda a: a) if exact else bf16
    layers = unpack(np.asarray(theta, np.float64), widths)
    Z, A = forward(theta, X, widths, exact)
    m, c = T.shape
    diff = A[-1] - T
    loss = float(np.mean(diff * diff))
    dZ = 2.0 * diff / (m * c)
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        dW = rnd(dZ).T @ rnd(A[li])
        db = dZ.sum(axis=0)
        grads.append((dW, db))
        if li > 0:
            dZ = (rnd(dZ) @ rnd(W)) * gelu_grad(Z[li - 1])
    grads.reverse()
    return loss, np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])


def adam(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_lr(step, total, lr0=1e-3):
    """Cosine decay from lr0 to 0 over `total` steps (step counts from 1)."""
    return 0.5 * lr0 * (1.0 + np.cos(np.pi * (step - 1) / max(1, total)))


def pod(Y, r):
    """POD of snapshots Y (m x N, one state per row): mean, the r leading
    left singular vectors of the centred snapshot matrix (N x r, columns
    sign-normalised so that each column's largest-magnitude entry is
    positive), singular values and the snapshots' coefficients (m x r)."""
    Y = np.asarray(Y, np.float64)
    ybar = Y.mean(axis=0)
    Yc = Y - ybar
    U, s, Vt = np.linalg.svd(Yc.T, full_matrices=False)
    Psi = U[:, :r].copy()
    for j in range(Psi.shape[1]):
        if Psi[np.argmax(np.abs(Psi[:, j])), j] < 0:
            Psi[:, j] = -Psi[:, j]
    coef = Yc @ Psi
    return ybar, Psi, s[:r], coef


def scale_inputs(mu, lo, hi):
    """Min-max scaling of each parameter to [-1, 1]."""
    mu = np.asarray(mu, np.float64)
    return 2.0 * (mu - lo) / (hi - lo) - 1.0
