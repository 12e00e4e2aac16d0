"""Full-size parity at 128^3 (k = 60 closed-form modes), in the launch
configuration of the bench: one batch of 128 instances on the mixed path with
BF16 modes and the autotuned column depth, plus one instance on the plain
FP64 path.

The oracle's own full-size solves of the first two instances
(tests/golden/diff3d_128_oracle.json and diff3d_128_oracle_states.npz, written
by oracle/full_size_reference.py) fix the outer iterations, the active sets and
every node of the state (stored in float32: relative rounding 6e-8).  The GPU
states must be within relative L2 1e-5 (mixed path) and 1e-6 (FP64 path) of
them over every node (Eq. accuracy_rel_err).  The residual bound stays as a
second check: with S = mass I + wgt A^T A and the active set empty,
||S^-1|| <= 1/mass = 1, so for two approximations with relative residuals
r1, r2 of S y = rhs, |y1_i - y2_i| <= ||y1 - y2||_2 <= (r1 + r2) ||rhs||.  The
true residual on the inactive set is recomputed in FP64 through the library's
S for sampled instances of the batch, and y <= psi + tau holds for all of them."""
import json
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DEV = "cuda"


@pytest.fixture(scope="module")
def sdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_17971_b300 import sdf as S
    return S


@pytest.fixture(scope="module")
def setup():
    from oracle import oracle as O
    from paper_2606_17971_b300 import workloads as W
    gold = json.load(open(os.path.join(HERE, "golden", "diff3d_128_oracle.json")))
    states = np.load(os.path.join(HERE, "golden", "diff3d_128_oracle_states.npz"))
    w = W.WORKLOADS["diff3d_128"]
    assert gold["k"] == w.k and gold["rtol"] == 1e-8
    insts = W.draw_instances(w, count=128)
    for g in gold["instances"]:
        i = insts[g["index"]]
        assert i.a == g["a"] and list(i.c) == g["c"]
    P = O.Problem(w.dim, w.n, alpha=w.alpha)
    return dict(W=W, w=w, gold=gold, insts=insts, P=P, psi=W.psi_vector(w), states=states)


def _check_full_state(states, i, y, active, tol):
    """Every node: relative L2 error against the oracle's stored state, and the
    stored active set bit for bit."""
    ref = states[f"y{i}"].astype(np.float64)
    yy = y.cpu().numpy()
    err = np.linalg.norm(yy - ref) / np.linalg.norm(ref)
    assert err <= tol, (i, err)
    act_ref = np.unpackbits(states[f"active{i}"])[:ref.size].astype(bool)
    assert np.array_equal(active.cpu().numpy().astype(bool), act_ref), i
    return err


def _true_relres(G, inst_row, y, active, rhs, psi):
    """||(rhs - S y)_I|| / ||rhs_I - (S psi_A)_I||: the relative residual of
    S_II y_I = rhs_I - S_IA psi_A, in FP64 through the library's S."""
    inact = (active == 0).to(torch.float64)
    psiA = psi * (1.0 - inact)
    r = (rhs - G.apply_S(inst_row, y, mode=1)) * inact
    b = (rhs - G.apply_S(inst_row, psiA.contiguous(), mode=1)) * inact
    return (r.norm() / b.norm()).item()


def _check_against_golden(g, y, relres_gpu, rhs_norm, idx):
    # |y_gpu - y_orc| <= ||e||_2 <= (r_gpu + r_orc) ||rhs|| (lambda_min(S) >= 1);
    # 1.01 covers the rounding of the norms themselves
    bound = 1.01 * (relres_gpu + g["true_relres"]) * rhs_norm
    assert abs(y.norm().item() - g["y_norm"]) <= bound, (y.norm().item(), g["y_norm"], bound)
    err = np.abs(y[idx].cpu().numpy() - np.array(g["y_sample"]))
    assert err.max() <= bound, (err.max(), bound)


def test_full_size_batch_matches_the_oracle_solves(sdf, setup):
    s = setup
    w, gold, insts, P = s["w"], s["gold"], s["insts"], s["P"]
    G = sdf.Problem(3, w.n, alpha=w.alpha, yd_sigma=w.sigma)
    phi, _ = G.analytic_modes(w.k, sdf.BF16)
    G.set_modes(phi)
    psi = torch.as_tensor(s["psi"], device=DEV)
    inst_t = torch.as_tensor(s["W"].instances_array(insts), device=DEV)
    o = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED)
    G.autotune(inst_t, psi, o)
    out = G.solve(inst_t, psi, o, want_lambda=False)
    assert out["status"] == 0
    # feasibility on every instance of the batch
    assert out["y"].max().item() <= w.psi + o.tau
    idx = torch.as_tensor(np.array(gold["sample_index"]), device=DEV)
    golden = {g["index"]: g for g in gold["instances"]}
    for b in sorted(set(golden) | {17, 40, 63, 100, 127}):
        st = out["stats"][b]
        assert st["status"] == 0 and all(r <= 1e-8 for r in st["relres"]), (b, st)
        rhs_np = P.desired_state(insts[b].a, insts[b].c, w.sigma)[1]
        rhs = torch.as_tensor(rhs_np, device=DEV)
        act = out["active"][b]
        rel = _true_relres(G, inst_t[b:b + 1].contiguous(), out["y"][b].contiguous(), act, rhs,
                           psi)
        # the mixed path stops on an FP64 residual of the FP64 iterate
        assert rel <= 1.05e-8, (b, rel)
        if b in golden:
            g = golden[b]
            assert st["outer_iters"] == g["outer_iters"] and st["n_active"] == g["n_active"]
            assert int(act.sum().item()) == g["active_count"] == 0
            # FP32 arithmetic and BF16 modes against FP64: a few percent more
            assert abs(sum(st["cg_iters"]) - sum(g["cg_iters"])) <= 0.05 * sum(g["cg_iters"])
            _check_against_golden(g, out["y"][b], rel, np.linalg.norm(rhs_np), idx)
            _check_full_state(s["states"], b, out["y"][b], act, 1e-5)


def test_full_size_plain_fp64_instance_matches_the_oracle(sdf, setup):
    s = setup
    w, gold, insts, P = s["w"], s["gold"], s["insts"], s["P"]
    g = gold["instances"][0]
    G = sdf.Problem(3, w.n, alpha=w.alpha, yd_sigma=w.sigma)
    phi, _ = G.analytic_modes(w.k)
    G.set_modes(phi)
    psi = torch.as_tensor(s["psi"], device=DEV)
    inst_t = torch.as_tensor(s["W"].instances_array(insts[:1]), device=DEV)
    out = G.solve(inst_t, psi, sdf.default_opts(check_every=128), want_lambda=False)
    st = out["stats"][0]
    assert st["status"] == 0 and st["outer_iters"] == g["outer_iters"]
    assert int(out["active"][0].sum().item()) == g["active_count"]
    # same arithmetic as the oracle, other summation order
    assert abs(st["cg_iters"][0] - g["cg_iters"][0]) <= max(3, 0.01 * g["cg_iters"][0])
    rhs_np = P.desired_state(insts[0].a, insts[0].c, w.sigma)[1]
    rel = _true_relres(G, inst_t, out["y"][0].contiguous(), out["active"][0],
                       torch.as_tensor(rhs_np, device=DEV), psi)
    assert rel <= 1.05e-8
    _check_against_golden(g, out["y"][0], rel, np.linalg.norm(rhs_np),
                          torch.as_tensor(np.array(gold["sample_index"]), device=DEV))
    _check_full_state(s["states"], 0, out["y"][0], out["active"][0], 1e-6)
