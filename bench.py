#!/usr/bin/env python
"""Benchmark: instances/sec to the converged active set at rtol 1e-8.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--path PATH]

One step solves one batch of synthetic instances of the workload (seeded
inputs from paper_2606_17971_b300.workloads) through the C ABI: the primal
active-set loop around A-DEF2-deflated Jacobi-PCG until every instance's active
set is converged.  The timed region is bracketed by a barrier and
cuda.synchronize on both sides, timed with CUDA events on the solve's stream,
max over ranks; rank 0 prints one JSON line.  Multi-GPU runs are replicas:
each rank solves its own instances (the path shards by instance with no
collective), so scaling is weak.

--impl reference times the CPU oracle (oracle/) on the host cores on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "instances/sec to converged active set at rtol 1e-8, batched+learned vs plain"
UNIT = "instances/s"
FP64_PEAK_TFLOPS = 1.25  # nominal B300 FP64 of the profiling recipe (probe measured 1.20)
KSRC = [os.path.join(ROOT, "paper_2606_17971_b300", "csrc", f)
        for f in ("sdf.cu", "sdf_device.cuh", "tc_device.cuh")]


def source_hash() -> str:
    h = hashlib.sha256()
    for f in KSRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# algorithmic work per dof and per launch

def stencil_flops(dim):
    # A u in flux form: 2*dim differences + 2*dim FMAs (2 flops); same for A^T w;
    # mass*u + wgt*A^T w: 3 flops
    return 2 * (2 * dim + 4 * dim) + 3


def kernel_work(name, dim, k, phi_bytes, vec_bytes=8, mixed=False, batch=1):
    """(flops, bytes) per dof and instance of one launch of a CG kernel.

    Mixed path (FP32 vectors; Phi shared by the batch, so its bytes are
    divided by the batch size):
      update  k_update_v: r, q, p, mask, x_lo read; r_out, v, x_lo written
      expand  k_expand_b: mask, r, p read, p written, Phi (shared)
      spmv    k_spmv:     p read, q written
      project k_proj_gemm: v read, Phi (shared)
    FP64 path: see the per-kernel comments below."""
    if mixed:
        if name == "update":
            return stencil_flops(dim) + 9, 4 * 4 + 1 + 8 + 4 + 4
        if name == "expand":
            return 2 * k + 4, 1 + 4 + 8 + k * phi_bytes / batch
        if name == "spmv":
            return stencil_flops(dim) + 2, 4 + 4 + 1
        if name == "project":
            return 2 * k, 4 + k * phi_bytes / batch
    if name == "update":   # r,q,p,dinv read, r written; x (FP64) read+written; Phi; S z; Phi^T S z
        return 2 * k + stencil_flops(dim) + 9, 5 * vec_bytes + 16 + 1 + k * phi_bytes
    if name == "expand":   # r,dinv,p read; p written; Phi read; Phi c
        return 2 * k + 4, 4 * vec_bytes + 1 + k * phi_bytes
    if name == "spmv":     # p read, q written
        return stencil_flops(dim) + 2, 2 * vec_bytes + 1
    raise ValueError(name)


def profile_traffic(kernel, workload):
    """DRAM traffic per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"k_{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != source_hash():
        return None
    return float(t.group(1))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        load = [v for v in sm if v > 0.5 * (smax or max(sm))] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# multi-process aggregation (one process per GPU, instances sharded by rank)

def shard(items, rank, world):
    """The instances of this rank: every world-th one, starting at rank (no
    collective in the data path: ranks solve disjoint instances)."""
    return items[rank::world]


def max_over_ranks(value, device, world):
    """The largest of the ranks' values (the job's wall time is the slowest
    rank's); world == 1 returns the value itself."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_problem(w, sdf, device, phi_dtype=0):
    from paper_2606_17971_b300 import workloads as W
    kap = W.kappa_field(w)
    G = sdf.Problem(w.dim, w.n, alpha=w.alpha, kappa=kap, diff_scale=w.diff_scale,
                    convection=w.convection, yd_sigma=w.sigma, device=device)
    phi, _ = G.analytic_modes(w.k, phi_dtype)  # closed-form reference modes on the GPU (Sec. 2.2.8)
    G.set_modes(phi)
    return G, phi


def cpu_sample(w, inst, m_iters=20):
    """Bounded oracle sample: one restricted A-DEF2 solve at the full size,
    truncated at m_iters CG iterations; returns (setup seconds, seconds per
    CG iteration, threads)."""
    from oracle import oracle as O
    from paper_2606_17971_b300 import workloads as W
    P = O.Problem(w.dim, w.n, kappa=W.kappa_field(w), diff_scale=w.diff_scale, alpha=w.alpha)
    Phi = O.analytic_modes(w.dim, w.n, w.k, w.alpha, diff_scale=w.diff_scale)[0]
    _, rhs = P.desired_state(inst.a, inst.c[: w.dim], w.sigma)
    r = P.inner_solve(np.zeros(P.N, np.uint8), rhs, np.full(P.N, w.psi), Phi, maxit=m_iters)
    return r["t_setup"], r["t_loop"] / max(1, r["iters"]), os.cpu_count()


def spacetime_leg(w, sdf, dev):
    """The space-time workload (App. E.2) on the FP64 path: one batch of
    its instances with the Kronecker basis I_nt (x) Z_s, with the
    constant-in-time lift 1_nt (x) Z_s / sqrt(n_t), and with plain PCG, each
    timed with CUDA events after one warm-up solve (not part of the metric)."""
    import torch
    from paper_2606_17971_b300 import workloads as W
    n_t = w.extra["n_t"]
    G = sdf.Problem(3, (w.n, w.n, n_t), alpha=w.alpha, yd_sigma=w.sigma, time_axis=True,
                    t_final=w.extra["t_final"], ramp_tau=w.extra["ramp_tau"], device=dev)
    zs, _ = sdf.Problem(2, w.n, alpha=w.alpha, yd_sigma=w.sigma, device=dev).analytic_modes(w.k)
    kron = G.spacetime_kron_modes(zs)
    # the constant-in-time lift is W_t (x) Z_s with W_t = 1_nt / sqrt(n_t)
    lift = G.spacetime_modes(np.full((n_t, 1), 1.0 / np.sqrt(n_t)), zs)
    inst = torch.as_tensor(W.instances_array(W.draw_instances(w, count=w.batch)), device=dev)
    psi = torch.full((G.N,), w.psi, dtype=torch.float64, device=dev)
    res = {"workload": w.name, "grid": [w.n, w.n], "n_t": n_t, "N": G.N, "instances": w.batch,
           "spatial_modes": w.k, "path": "FP64 A-DEF2 (primal active-set loop)"}
    stream = torch.cuda.current_stream()
    for name, phi in (("kronecker", kron), ("constant_lift", lift), ("plain", None)):
        o = sdf.default_opts(check_every=128, deflate=int(phi is not None))
        if phi is not None:
            G.set_modes(phi)
        G.solve(inst[:1].contiguous(), psi, o, want_lambda=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = G.solve(inst, psi, o, want_lambda=False)
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = {"instances_per_s": w.batch / (e0.elapsed_time(e1) * 1e-3),
                     "cg_iters_per_instance": float(np.mean([sum(s["cg_iters"]) for s in r["stats"]])),
                     "outer_iters_per_instance": float(np.mean([s["outer_iters"] for s in r["stats"]])),
                     "rank": 0 if phi is None else int(phi.shape[0]),
                     "statuses": sorted(set(s["status"] for s in r["stats"]))}
    c0 = res["plain"]["cg_iters_per_instance"]
    res["iteration_reduction"] = {k: 1.0 - res[k]["cg_iters_per_instance"] / c0
                                  for k in ("kronecker", "constant_lift")}
    return res


def diag_sweep_leg(n, count, sdf, dev, K=40, r=20, psi_value=0.5):
    """The spectral-coherence sweep of Sec. 4.1 on the GPU: instances of the
    2D diffusion family on an n x n grid with psi = psi_value (calibrated for
    a sizeable active set, as the paper calibrates psi), each solved with r
    reference modes and cold; then delta and rho against the first
    instance's active set, the K lowest eigenpairs of S_II, and the
    principal angles between them and the K restricted reference modes
    (theta_r the r-th smallest, theta_max the largest, and the nested angle
    of Prop. dk at r).  Timed per stage; not part of the metric."""
    import torch
    from paper_2606_17971_b300 import workloads as W
    w = W.scaled(W.WORKLOADS["diff2d_32"], n)
    G = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma, device=dev)
    phiK, _ = G.analytic_modes(K)
    phir = phiK[:r].contiguous()
    insts = W.draw_instances(w, count=count)
    inst = torch.as_tensor(W.instances_array(insts), device=dev)
    psi = torch.full((G.N,), psi_value, dtype=torch.float64, device=dev)
    t = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.set_modes(phir)
    defl = G.solve(inst, psi, want_lambda=False)
    cold = G.solve(inst, psi, sdf.default_opts(deflate=0), want_lambda=False)
    torch.cuda.synchronize()
    t["solves_s"] = time.perf_counter() - t0
    G.set_modes(phiK)
    t0 = time.perf_counter()
    sets = G.diag_active_sets(defl["active"][0].clone(), defl["active"], r=r)
    t["sets_s"] = time.perf_counter() - t0
    rows, t_eig, t_ang = [], 0.0, 0.0
    for b in range(count):
        act = defl["active"][b].contiguous()
        t0 = time.perf_counter()
        V, _, est = G.restricted_modes(inst[b], act, K)
        t_eig += time.perf_counter() - t0
        t0 = time.perf_counter()
        nested, srt = G.diag_angles(act, V, sorted_angles=True)
        t_ang += time.perf_counter() - t0
        n_d = sum(defl["stats"][b]["cg_iters"])
        n_c = sum(cold["stats"][b]["cg_iters"])
        q = np.array_split(np.degrees(srt), 5)  # mean angle per mode quintile (App. D.6)
        rows.append({"a": insts[b].a, "delta": float(sets["delta"][b]), "rho": float(sets["rho"][b]),
                     "delta_w": float(sets["delta_w"][b]),
                     "quintile_mean_deg": [float(x.mean()) for x in q],
                     "theta_r_deg": float(np.degrees(srt[r - 1])),
                     "theta_max_deg": float(np.degrees(srt[-1])),
                     "nested_theta_r_deg": float(np.degrees(nested[r - 1])),
                     "cg_deflated": n_d, "cg_cold": n_c, "eff": 1.0 - n_d / n_c,
                     "eig_converged": bool(est["converged"]), "eig_passes": est["iters"]})
    t["restricted_eig_s"] = t_eig
    t["angles_s"] = t_ang
    d = np.array([x["delta"] for x in rows])
    dw = np.array([x["delta_w"] for x in rows])
    e = np.array([x["eff"] for x in rows])

    def corr(a, c):
        return float(np.corrcoef(a, c)[0, 1]) if a.std() > 0 and c.std() > 0 else None

    return {"grid": [n, n], "instances": count, "psi": psi_value, "K": K, "r": r, "seconds": t,
            "delta_max": float(d.max()), "theta_r_max_deg": max(x["theta_r_deg"] for x in rows),
            "theta_max_min_deg": min(x["theta_max_deg"] for x in rows),
            "eff_mean": float(e.mean()), "eff_std": float(e.std()),
            "corr_delta_eff": corr(d, e), "corr_delta_w_eff": corr(dw, e),
            "quintile_mean_deg": [float(np.mean([x["quintile_mean_deg"][i] for x in rows]))
                                  for i in range(5)],
            "rows": rows}


def csr_leg(n, sdf, dev, batch=8, k=16):
    """A problem given by its operator: K = the 5-point -Laplace on an n x n
    grid, built here with scipy as a caller would, solved through
    sdf_problem_create_csr / sdf_solve_batch_rhs, against the grid path on the
    same operator and the same family of right-hand sides (mass y_d of the
    same instances, evaluated here as a caller would), FP64, k closed-form
    modes; not part of the metric."""
    import scipy.sparse as sp
    import torch
    from paper_2606_17971_b300 import workloads as W
    w = W.scaled(W.WORKLOADS["diff2d_32"], n)
    h = 1.0 / (n + 1)
    T1 = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h**2
    K = (sp.kron(sp.identity(n), T1) + sp.kron(T1, sp.identity(n))).tocsr()
    Gg = sdf.Problem(2, n, alpha=w.alpha, yd_sigma=w.sigma, device=dev)
    phi, _ = Gg.analytic_modes(k)
    Gg.set_modes(phi)
    t0 = time.perf_counter()
    Gc = sdf.Problem.csr(K, alpha=w.alpha, device=dev)
    t_create = time.perf_counter() - t0
    Gc.set_modes(phi)
    insts = W.draw_instances(w, count=batch)
    inst = torch.as_tensor(W.instances_array(insts), device=dev)
    psi = torch.full((Gg.N,), w.psi, dtype=torch.float64, device=dev)
    # the caller's right-hand sides: the same Gaussian family at the nodes
    x = (np.arange(n) + 1) * h
    gy, gx = np.meshgrid(x, x, indexing="ij")
    rhs = torch.as_tensor(np.stack([
        i.a * np.exp(-((gx - i.c[0]) ** 2 + (gy - i.c[1]) ** 2).ravel() / (2 * w.sigma**2))
        for i in insts]), device=dev).contiguous()
    res = {"grid": [n, n], "instances": batch, "k": k, "nnz_K": int(K.nnz),
           "host_assembly_s": t_create}
    stream = torch.cuda.current_stream()
    for name, run in (("grid", lambda: Gg.solve(inst, psi, want_lambda=False)),
                      ("csr", lambda: Gc.solve_rhs(rhs, psi))):
        run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = run()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = {"instances_per_s": batch / (e0.elapsed_time(e1) * 1e-3),
                     "cg_iters_per_instance": float(np.mean([sum(s["cg_iters"]) for s in r["stats"]])),
                     "statuses": sorted(set(s["status"] for s in r["stats"]))}
    return res


def oracle_counts(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    inst = d.get("instances", [])
    if not inst:
        return None
    return (float(np.mean([i["outer_iters"] for i in inst])),
            float(np.mean([sum(i["cg_iters"]) for i in inst])))


def run_reference(args, w):
    from paper_2606_17971_b300 import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    counts = oracle_counts(w.name)
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no full-size oracle iteration counts for {w.name} (tests/golden)"}))
        return
    n_outer, iters = counts
    insts = W.draw_instances(w, count=args.warmup + args.steps)
    for i in range(args.warmup):
        cpu_sample(w, insts[i], 5)
    per_inst = []
    t0 = time.time()
    for i in range(args.steps):
        ts, ti, cores = cpu_sample(w, insts[args.warmup + i], 10)
        per_inst.append(n_outer * ts + iters * ti)
    wall = time.time() - t0
    val = 1.0 / float(np.mean(per_inst))
    sample = (f"oracle A-DEF2 at the full {w.n}^{w.dim} size, one restricted solve per step "
              f"truncated at 10 CG iterations; instances/s = 1/(outer*t_setup + iters*t_iter) "
              f"with outer={n_outer:.2f}, iters={iters:.0f} from the oracle's own full-size "
              f"solves (tests/golden/{w.name}_oracle.json)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w.name, "path": "CPU oracle (plain C, FP64)"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diff3d_128")
    ap.add_argument("--n", type=int, default=0, help="grid override (profiling captures only)")
    ap.add_argument("--max-cg", type=int, default=0, help="CG cap (profiling captures only)")
    ap.add_argument("--path", default="mixed", choices=["plain", "mixed"],
                    help="plain: FP64 A-DEF2 per instance; mixed: FP32/BF16 with FP64 refinement")
    ap.add_argument("--phi", default="bf16", choices=["f32", "bf16"], help="mode storage (mixed)")
    ap.add_argument("--batch", type=int, default=0,
                    help="instances per step and GPU (default: 64 mixed, 1 plain)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-learned", action="store_true",
                    help="mixed path without the learned warm start")
    ap.add_argument("--train", type=int, default=128,
                    help="training instances of the learned warm start (first solves)")
    ap.add_argument("--epochs", type=int, default=2000, help="Adam epochs of the warm-start MLP")
    ap.add_argument("--eig", default="", help="also time the reference eigensolve (Sec. 2.2.2) "
                    "of this variable-kappa workload, separately (e.g. block2d_1024)")
    ap.add_argument("--eig-degree", type=int, default=240)
    ap.add_argument("--eig-coarse", type=int, default=2,
                    help="also time the coarse-grid basis (Sec. 2.2.7) with this factor (0: off)")
    ap.add_argument("--spacetime", default="spacetime2d_64",
                    help="also time the space-time workload (App. E.2) with the Kronecker "
                         "basis, the constant-in-time lift and plain PCG ('' : off)")
    ap.add_argument("--no-diag", action="store_true",
                    help="skip timing the active-set diagnostics on the last batch")
    ap.add_argument("--diag-sweep", type=int, default=0,
                    help="also run the spectral-coherence sweep of Sec. 4.1 over this many "
                         "instances of the 2D diffusion family (0: off)")
    ap.add_argument("--diag-n", type=int, default=128, help="grid of the diagnostics sweep")
    ap.add_argument("--csr-n", type=int, default=0,
                    help="also time the CSR operator path against the grid path on an n x n "
                         "diffusion problem (0: off)")
    args = ap.parse_args()

    from paper_2606_17971_b300 import workloads as W
    w = W.WORKLOADS[args.workload]
    if args.n:
        w = W.scaled(w, args.n)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import torch.distributed as dist
    from paper_2606_17971_b300 import sdf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    mixed = args.path == "mixed"
    phi_dt = (sdf.BF16 if args.phi == "bf16" else sdf.F32) if mixed else sdf.F64
    G, phi = make_problem(w, sdf, dev, phi_dt)
    B = args.batch or (64 if mixed else 1)
    steps, warm = args.steps, args.warmup
    insts = W.draw_instances(w, count=(steps + warm) * B * world)
    mine = shard(insts, rank, world)
    inst_t = [torch.as_tensor(W.instances_array(mine[i * B:(i + 1) * B]), device=dev)
              for i in range(steps + warm)]
    psi = torch.full((w.N,), w.psi, dtype=torch.float64, device=dev)
    opts = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED if mixed else sdf.PREC_F64)
    opts_lambda = False
    if args.max_cg:
        opts.max_cg = args.max_cg
    out = {"y": torch.empty((B, w.N), dtype=torch.float64, device=dev), "lam": None,
           "active": torch.empty((B, w.N), dtype=torch.uint8, device=dev)}

    # ---- learned warm start: trained before the timed region ----
    learned = mixed and not args.no_learned
    model, train_info = None, None
    if learned:
        t0 = time.perf_counter()
        ntr = args.train
        tr = W.draw_instances(w, count=ntr, seed=w.seed + 1000 + rank)
        it_tr = torch.as_tensor(W.instances_array(tr), device=dev)
        o1 = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED, max_outer=1)
        Ytr = torch.empty((ntr, w.N), dtype=torch.float64, device=dev)
        tb = min(128, ntr)
        for j in range(0, ntr, tb):
            Ytr[j:j + tb] = G.solve(it_tr[j:j + tb].contiguous(), psi, o1, want_lambda=False)["y"]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        widths = (1 + w.dim, 256, 256, 256, 64)
        lo, hi = W.input_box(w)
        model = sdf.WarmModel(widths, w.N, lo, hi, torch.from_numpy(W.mlp_init(widths)).to(dev))
        loss = model.fit(Ytr, it_tr, epochs=args.epochs, lr0=1e-3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del Ytr
        train_info = {"instances": ntr, "solve_s": t1 - t0, "fit_s": t2 - t1,
                      "epochs": args.epochs, "loss_first": float(loss[0]),
                      "loss_last": float(loss[-1]), "widths": list(widths), "pod_rank": 64,
                      "note": "first (unconstrained) solves of separate training instances; "
                              "not part of the timed region"}

    # autotuned column depth of the stencil kernels (short capped solves, untimed)
    tuned_zc = G.autotune(inst_t[0], psi, opts) if mixed else 0

    def one_step(inst):
        if model is not None:
            x0 = model.predict(inst)
            return G.solve_x0(inst, psi, x0, opts, out=out, want_lambda=opts_lambda)
        return G.solve(inst, psi, opts, out=out, want_lambda=opts_lambda)

    for i in range(warm):
        one_step(inst_t[i])
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    opts.profile = 1
    G.reset_profile()
    stats = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # NVTX range: lets a profiler capture exactly the timed launches
        torch.cuda.nvtx.range_push("timed_region")
        e0.record(stream)
        for i in range(steps):
            res = one_step(inst_t[warm + i])
            stats.extend(res["stats"])
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    prof = G.profile()
    ms = max_over_ranks(e0.elapsed_time(e1), dev, world)
    value = steps * B * world / (ms * 1e-3)

    # ---- e2e: host buffers in, host buffers out, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        opts.profile = 0
        inst_h = [torch.from_numpy(W.instances_array(mine[i * B:(i + 1) * B])).pin_memory()
                  for i in range(steps + warm)]
        psi_h = torch.full((w.N,), w.psi, dtype=torch.float64).pin_memory()
        y_h = torch.empty((B, w.N), dtype=torch.float64).pin_memory()
        a_h = torch.empty((B, w.N), dtype=torch.uint8).pin_memory()
        if model is None:
            def e2e_step(i):
                G.solve_host(inst_h[i].numpy(), psi_h.numpy(), opts, y=y_h.numpy(),
                             active=a_h.numpy())
        else:
            # the learned pipeline through the binding: copy mu and psi in, predict
            # x0 (tensor-core MLP + FP64 expansion), solve, copy y and A out
            def e2e_step(i):
                inst_d = inst_h[i].to(dev, non_blocking=True)
                psi_d = psi_h.to(dev, non_blocking=True)
                x0 = model.predict(inst_d)
                r = G.solve_x0(inst_d, psi_d, x0, opts, out=out, want_lambda=False)
                y_h.copy_(r["y"], non_blocking=True)
                a_h.copy_(r["active"], non_blocking=True)
                torch.cuda.current_stream().synchronize()
        e2e_step(0)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            e2e_step(warm + i)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dev, world)
        e2e = {"value": steps * B * world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(inst_h[0].numel() * 8 + psi_h.numel() * 8),
               "d2h_bytes_per_step": int(y_h.numel() * 8 + a_h.numel()),
               "path": "learned pipeline through the Python binding" if model is not None
               else "sdf_solve_batch_host"}

    # ---- the same batch without the learned start (untimed comparison) ----
    cold_cmp = None
    if model is not None:
        opts.profile = 0
        ec0, ec1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ec0.record(stream)
        rc = G.solve(inst_t[warm], psi, opts, out=out, want_lambda=False)
        ec1.record(stream)
        torch.cuda.synchronize()
        cold_cmp = {"ms": ec0.elapsed_time(ec1),
                    "cg_iters_per_instance": float(np.mean([sum(s["cg_iters"]) for s in rc["stats"]])),
                    "learned_cg_iters_per_instance":
                        float(np.mean([sum(s["cg_iters"]) for s in stats[:B]])),
                    "note": "first timed batch solved again from x0 = 0"}

    # ---- roofline of the dominant kernel ----
    names = ("expand", "spmv", "update") + (("project",) if mixed else ())
    tot = {n: (prof["mean_ms"][n] or 0.0) * prof["samples"][n] for n in names}
    dom = max(names, key=lambda n: tot[n])
    phi_bytes = 8 if not mixed else (2 if args.phi == "bf16" else 4)
    flops_dof, bytes_dof = kernel_work(dom, w.dim, w.k, phi_bytes, 4 if mixed else 8, mixed, B)
    units = w.N * B
    mean_s = prof["mean_ms"][dom] * 1e-3
    hbm = peaks().get("hbm_gbs")
    if mixed:  # FP32 arithmetic: the streaming kernels are HBM-bound by design
        achieved = bytes_dof * units / mean_s / 1e9
        roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm,
                "traffic": profile_traffic(dom + "_mixed", w.name),
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        achieved = flops_dof * units / mean_s / 1e12
        roof = {"kernel": f"k_{dom}", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": profile_traffic(dom, w.name),
                "peak_source": "nominal FP64 of the profiling recipe (1.25 TFLOP/s; probe measured 1.20)"}
    roof.update({
            "algorithmic_flops_per_launch": flops_dof * units,
            "algorithmic_bytes_per_launch": bytes_dof * units,
            "hbm_gbs_at_algorithmic_bytes": bytes_dof * units / mean_s / 1e9,
            "hbm_peak_gbs": hbm, "mean_launch_ms": prof["mean_ms"][dom],
            "timed_launches": prof["samples"][dom],
            "kernel_mean_ms": {n: prof["mean_ms"][n] for n in names + ("resid",)},
            "units_per_launch": units})

    cg = [sum(s["cg_iters"]) for s in stats]
    outer = [s["outer_iters"] for s in stats]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": [w.n] * w.dim, "k": w.k, "alpha": w.alpha,
                   "instances_per_step": B * world, "batch_per_gpu": B,
                   "path": ("mixed FP32/%s A-DEF2, FP64 x, reductions and residual replacement"
                            % args.phi if mixed else "plain FP64 A-DEF2 per instance")
                           + (", learned warm start" if learned else "")
                           + " (primal active-set loop)",
                   "modes": "closed-form sines on the GPU (Sec. 2.2.8)",
                   "l2": "inputs larger than L2: Phi is %.2f GB, read twice per CG iteration"
                         % (w.N * w.k * phi_bytes / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "autotuned_column_depth": tuned_zc},
        "cg_iters_per_instance": float(np.mean(cg)), "outer_iters_per_instance": float(np.mean(outer)),
        "statuses": sorted(set(s["status"] for s in stats)),
        "roofline": roof, "clocks": clk.summary(), "e2e": e2e,
        # the solver's launches plus the warm-start prediction's per step: per
        # layer one weight conversion and one product, then input conversion,
        # input scaling and the expansion
        "gpu_launches": int(prof["launches"]) + (steps * (2 * 4 + 3) if model is not None else 0),
    }
    if model is not None:
        line["learned"] = {"training": train_info, "same_batch_cold": cold_cmp}
    if mixed and not args.no_plain:
        # the metric compares against the plain per-instance FP64 path: one
        # instance of the same workload after one warm-up solve
        Gp, _ = make_problem(w, sdf, dev, sdf.F64)
        op = sdf.default_opts(check_every=128)
        one = inst_t[0][:1].contiguous()
        Gp.solve(one, psi, op, want_lambda=False)
        torch.cuda.synchronize()
        ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ep0.record(stream)
        rp = Gp.solve(inst_t[1][:1].contiguous(), psi, op, want_lambda=False)
        ep1.record(stream)
        torch.cuda.synchronize()
        pv = 1e3 / ep0.elapsed_time(ep1)
        line["plain_fp64_per_instance"] = {
            "value": pv, "unit": UNIT, "instances_timed": 1,
            "cg_iters": sum(rp["stats"][0]["cg_iters"]), "note": "same workload, same run"}
        line["speedup_vs_plain"] = value / pv
        del Gp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ts, ti, cores = cpu_sample(w, mine[0], 20)
        per = np.mean(outer) * ts + np.mean(cg) * ti
        line["cpu_baseline"] = {
            "value": 1.0 / per, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle A-DEF2 at the full {w.n}^{w.dim} size on instance 0, one restricted "
                       f"solve truncated at 20 CG iterations (set-up {ts:.2f} s, {ti * 1e3:.1f} ms "
                       f"per iteration); instances/s = 1/(outer*t_setup + iters*t_iter) with this "
                       f"run's mean outer={np.mean(outer):.2f}, iters={np.mean(cg):.0f}")}
    if args.eig and rank == 0:
        # the offline eigensolve, timed on its own (not part of the metric)
        we = W.WORKLOADS[args.eig]
        Ge = sdf.Problem(we.dim, we.n, alpha=we.alpha, kappa=W.kappa_field(we), yd_sigma=we.sigma,
                         device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ls, la, est = Ge.eig_modes(we.k, degree=args.eig_degree, max_iter=2000)
        torch.cuda.synchronize()
        line["eigensolve"] = {"workload": we.name, "k": we.k, "N": we.N,
                              "seconds": time.perf_counter() - t0, "passes": est["iters"],
                              "converged": est["converged"], "max_rel_resid": est["max_rel_resid"],
                              "block_matvecs": est["matvecs"],
                              "method": "Chebyshev-filtered subspace iteration on A, FP64"}
        if args.eig_coarse >= 2:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            phc, _, cst = Ge.coarse_modes(args.eig_coarse, we.k, degree=args.eig_degree,
                                          max_iter=2000)
            torch.cuda.synchronize()
            line["eigensolve"]["coarse_grid"] = {
                "factor": args.eig_coarse, "seconds": time.perf_counter() - t0,
                "columns_kept": int(phc.shape[0]), "coarse_passes": cst["iters"],
                "method": "eigenpairs on the grid coarsened by the factor, linear prolongation, QR"}
        del Ge
    if not args.no_diag and rank == 0:
        # Eq. delta / Eq. rho / the mode-weighted distance of the last timed
        # batch's active sets from its first instance's (not part of the metric)
        ref = out["active"][0].clone()
        G.diag_active_sets(ref, out["active"], r=w.k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dg = G.diag_active_sets(ref, out["active"], r=w.k)
        td = time.perf_counter() - t0
        line["diagnostics"] = {
            "active_sets": B, "N": w.N, "r": w.k, "ms": 1e3 * td,
            "mask_and_mode_gb_per_s": (B * w.N + w.N + w.N * w.k * phi_bytes * ((B + 7) // 8))
                                      / td / 1e9,
            "delta_max": float(dg["delta"].max()), "rho_mean": float(dg["rho"].mean()),
            "note": "sdf_diag_active_sets, host round trip included"}
    if args.spacetime and rank == 0:
        line["spacetime"] = spacetime_leg(W.WORKLOADS[args.spacetime], sdf, dev)
    if args.csr_n and rank == 0:
        line["csr_path"] = csr_leg(args.csr_n, sdf, dev)
    if args.diag_sweep and rank == 0:
        line["diagnostics_sweep"] = diag_sweep_leg(args.diag_n, args.diag_sweep, sdf, dev)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
