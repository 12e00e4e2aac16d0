"""The seeded input generators against the input recipe they state (no GPU).

Every input of the tests and of the bench comes from
paper_2606_17971_b300/workloads.py.  These checks hold it to the laws its
docstring names: the lognormal coefficient's Gaussian field has the
exponential covariance sigma^2 exp(-r/ell) with ell = 0.1 and sigma = 1; the
block coefficient is constant on 4 x 4 equal blocks with log10 kappa in
[-1, 1]; instance parameters follow their uniform laws, with unit convection
velocities; draws are reproducible from the seed; the initial MLP weights have
variance 1/fan_in and zero biases."""
import numpy as np
import pytest

from paper_2606_17971_b300 import workloads as W


def test_gaussian_field_has_the_stated_exponential_covariance():
    # 400 seeded draws on a 48^2 grid (h = 1/49): the sample covariance at a
    # lag of j nodes along x, along y and along the diagonal against
    # exp(-r/0.1).  About 40,000 independent patches enter each estimate,
    # so its sampling error is below 0.01; the bar is 0.04.
    n, ell = 48, 0.1
    h = 1.0 / (n + 1)
    F = np.stack([W.gaussian_field_2d(n, ell, 1.0, np.random.default_rng(s))
                  for s in range(400)])
    assert abs(F.mean()) < 0.03
    assert F.var() == pytest.approx(1.0, abs=0.04)
    for j in (1, 2, 4, 8):
        cx = np.mean(F[:, :, j:] * F[:, :, :-j])
        cy = np.mean(F[:, j:, :] * F[:, :-j, :])
        cd = np.mean(F[:, j:, j:] * F[:, :-j, :-j])
        assert cx == pytest.approx(np.exp(-j * h / ell), abs=0.04), (j, cx)
        assert cy == pytest.approx(np.exp(-j * h / ell), abs=0.04), (j, cy)
        assert cd == pytest.approx(np.exp(-np.sqrt(2.0) * j * h / ell), abs=0.04), (j, cd)
    # sigma scales the field: the same draw with sigma = 2 is twice as large
    a = W.gaussian_field_2d(n, ell, 1.0, np.random.default_rng(5))
    b = W.gaussian_field_2d(n, ell, 2.0, np.random.default_rng(5))
    np.testing.assert_allclose(b, 2.0 * a, rtol=1e-12, atol=1e-12)


def test_lognormal_kappa_is_the_exponential_of_the_field():
    w = W.scaled(W.WORKLOADS["lognormal2d_2048"], 40)
    kap = W.kappa_field(w)
    assert kap.shape == (w.N,) and np.all(kap > 0)
    again = W.kappa_field(w)
    np.testing.assert_array_equal(kap, again)  # one seeded draw
    g = np.log(kap)
    assert abs(g.mean()) < 1.0 and 0.2 < g.std() < 2.0


@pytest.mark.parametrize("dim,n", [(2, 30), (2, 33), (3, 13)])
def test_block_kappa_is_constant_on_4x4_blocks(dim, n):
    w = W.scaled(W.WORKLOADS["block2d_1024"], n, dim=dim)
    kap = W.kappa_field(w).reshape((n,) * dim)
    lk = np.log10(kap)
    assert lk.min() >= -1.0 and lk.max() <= 1.0
    # node j (0-based) sits at x = (j + 1) / (n + 1), in block floor(4x)
    blk = np.minimum((4 * (np.arange(n) + 1)) // (n + 1), 3)
    seen = {}
    for idx in np.ndindex(*kap.shape):
        key = tuple(blk[i] for i in idx)
        seen.setdefault(key, set()).add(kap[idx])
    assert len(seen) == 4 ** dim
    assert all(len(v) == 1 for v in seen.values())
    assert len({next(iter(v)) for v in seen.values()}) == 4 ** dim


def test_constant_kappa_is_none():
    assert W.kappa_field(W.WORKLOADS["diff3d_128"]) is None


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_instance_laws(name):
    w = W.WORKLOADS[name]
    insts = W.draw_instances(w, count=4000, seed=w.seed + 17)
    a = np.array([i.a for i in insts])
    c = np.array([i.c for i in insts])
    lo, hi = w.a_range
    assert a.min() >= lo and a.max() <= hi
    # mean of U[lo, hi] within 5 standard errors
    assert abs(a.mean() - 0.5 * (lo + hi)) < 5 * (hi - lo) / np.sqrt(12 * len(a))
    assert c.shape == (len(insts), 3)
    assert np.all(c[:, :w.dim] >= w.c_range[0]) and np.all(c[:, :w.dim] <= w.c_range[1])
    assert np.all(c[:, w.dim:] == 0.0)
    b = np.array([i.b for i in insts])
    if w.convection:
        np.testing.assert_allclose(np.hypot(b[:, 0], b[:, 1]), 1.0, rtol=1e-12)
        theta = np.mod(np.arctan2(b[:, 1], b[:, 0]), 2 * np.pi)
        # uniform angle: each quadrant holds about a quarter
        q = np.bincount((theta // (np.pi / 2)).astype(int), minlength=4) / len(theta)
        assert np.all(np.abs(q - 0.25) < 0.03), q
    else:
        assert np.all(b == 0.0)


def test_draws_are_reproducible_and_offsets_continue_the_stream():
    w = W.WORKLOADS["diff3d_128"]
    first = W.draw_instances(w, count=10)
    assert W.instances_array(first).tolist() == W.instances_array(W.draw_instances(w, count=10)).tolist()
    tail = W.draw_instances(w, count=4, offset=6)
    assert W.instances_array(tail).tolist() == W.instances_array(first[6:]).tolist()
    other = W.draw_instances(w, count=10, seed=w.seed + 1000)
    assert W.instances_array(other).tolist() != W.instances_array(first).tolist()
    seeds = [v.seed for v in W.WORKLOADS.values()]
    assert len(set(seeds)) == len(seeds)


def test_instances_array_layout():
    w = W.WORKLOADS["convdiff2d_512"]
    insts = W.draw_instances(w, count=3)
    arr = W.instances_array(insts)
    assert arr.shape == (3, 7) and arr.dtype == np.float64
    for row, i in zip(arr, insts):
        assert row.tolist() == [i.a, *i.c, *i.b]


def test_mlp_init_scale():
    widths = W.WARM_WIDTHS
    theta = W.mlp_init(widths, seed=3).astype(np.float64)
    assert theta.size == sum(widths[i + 1] * (widths[i] + 1) for i in range(len(widths) - 1))
    off = 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        Wl = theta[off:off + fo * fi]
        off += fo * fi
        bl = theta[off:off + fo]
        off += fo
        assert np.all(bl == 0.0)
        # variance 1/fan_in, within 5 standard errors of the sample variance
        assert abs(Wl.var() * fi - 1.0) < 5 * np.sqrt(2.0 / Wl.size), (fi, fo, Wl.var() * fi)
    lo, hi = W.input_box(W.WORKLOADS["diff3d_128"])
    assert lo == [1.0, 0.25, 0.25, 0.25] and hi == [3.0, 0.75, 0.75, 0.75]
