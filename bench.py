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


HBM_FALLBACK_GBS = 6400.0  # an earlier B300 copy measurement, used only without the file


def hbm_peak():
    """(HBM copy bandwidth in GB/s, where it comes from): the measured-peaks
    file of the machine, else the fallback figure, labelled as such."""
    v = peaks().get("hbm_gbs")
    if v:
        return float(v), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return HBM_FALLBACK_GBS, "fallback (no measured-peaks file: 6.4 TB/s, an earlier B300 copy)"


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
      update  k_update_v: r, q, p, x_lo (4 B each) and mask (1 B) read;
              r_out, v, x_lo written (the FP64 x fold, once per replacement
              period, is not counted)
      expand  k_expand_b: mask, r, p read, p written, Phi (shared)
      spmv    k_spmv:     p read, q written
      project k_proj_gemm: v read, Phi (shared)
    FP64 path: see the per-kernel comments below."""
    if mixed:
        if name == "update":
            return stencil_flops(dim) + 9, 4 * 4 + 1 + 3 * 4
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


def resolve_mode(args):
    """The workload's benchmark mode (MODES) with the command line's overrides."""
    mode = dict(MODES[args.workload])
    if args.path:
        mode["path"] = args.path
    if args.phi:
        mode["phi"] = args.phi
    if args.modes:
        mode["modes"] = args.modes
    if args.batch:
        mode["batch"] = args.batch
    if args.no_learned:
        mode["learned"] = False
    if mode["path"] == "plain":
        mode["learned"] = False
    return mode


def workload_config(w, mode, world, args):
    """The `config` object of a line: the workload measured (grid, modes,
    instances per step, held-out set) and how its inputs relate to L2.  Both
    arms print this same object; how each arm computes (GPU path, CPU oracle)
    is in the line's `path` key."""
    mixed = mode["path"] == "mixed"
    B = mode["batch"]
    units = w.N * B
    cfg = {"workload": w.name, "grid": [w.n] * w.dim, "k": w.k, "alpha": w.alpha,
           "instances_per_step": B * world, "batch_per_gpu": B}
    if mode.get("learned"):
        phi_bytes = 2 if mode.get("phi") == "bf16" else 4
        n_held = args.held_out or w.extra.get("held_out", 1024)
        cfg["held_out"] = n_held  # per rank: shard() deals n_held * world instances
        cfg["held_out_batches"] = max(1, n_held // B)
        cfg["l2"] = ("inputs larger than L2: Phi is %.2f GB and each vector %.2f GB"
                     % (w.N * w.k * phi_bytes / 1e9, units * 4 / 1e9))
    else:
        cfg["l2"] = ("inputs larger than L2 (%.2f GB of vectors per batch)"
                     % (8 * units * (4 if mixed else 8) / 1e9))
    cfg["parallelism"] = f"replicas x{world}" if world > 1 else "1 GPU"
    return cfg


def run_reference(args, w, mode, world):
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
        "data": "synthetic", "config": workload_config(w, mode, world, args),
        "path": "CPU oracle (plain C, FP64)",
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))




# ---------------------------------------------------------------------------
# how each workload is benchmarked (the configurations the metric is quoted on)

MODES = {
    # config 0: the plain method, FP64, the 20-instance batch
    "diff2d_32": dict(path="plain", batch=20, modes="eig"),
    # config 1: FP64, one instance per launch, k = 64 reference eigenmodes
    "block2d_1024": dict(path="plain", batch=1, modes="eig"),
    # config 2: FP64, 256 instances in one batched solve, shared k = 48 modes
    "convdiff2d_512": dict(path="plain", batch=256, modes="analytic"),
    # config 3: FP32 stencil and projections (FP32 or BF16 modes), FP64
    # scalars, coarse operator and residual replacement; --path plain for FP64
    "lognormal2d_2048": dict(path="mixed", phi="f32", batch=32, modes="eig"),
    # config 4 (the headline): batched + mixed + learned warm start
    "diff3d_128": dict(path="mixed", phi="bf16", batch=128, modes="analytic", learned=True),
}


def loop_roofline(prof, w, k, mixed, phi_bytes, B, units, chunk=100):
    """Roofline of the whole CG iteration: the algorithmic bytes (mixed path)
    or FP64 flops (FP64 path) of one iteration per dof and instance, times
    the units of one launch, over the summed mean kernel times of one
    iteration (the FP64 residual replacement amortised over its period).
    Bytes per unit: x, r, p each read and written once, q written and read
    once, the active-set mask as bits, and the modes read twice per
    iteration, shared by the batch: 8 s_v + 1/8 + 2 k s_Phi / B."""
    names = ("expand", "spmv", "update", "project")
    ms = sum((prof["mean_ms"][n] or 0.0) for n in names)
    if mixed:
        ms += (prof["mean_ms"]["resid"] or 0.0) / chunk
    sv = 4 if mixed else 8
    bpu = 8 * sv + 1.0 / 8 + 2.0 * k * phi_bytes / B
    fpu = 2 * stencil_flops(w.dim) + 20 + 4 * k
    out = {"ms_per_iter": ms, "units": units, "bytes_per_unit": bpu, "flops_per_unit": fpu,
           "kernels": [n for n in names if prof["mean_ms"][n]]}
    if ms <= 0:
        return out
    if mixed:
        hbm, src = hbm_peak()
        ach = bpu * units / (ms * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": src})
    else:
        ach = fpu * units / (ms * 1e-3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS,
                    "peak_source": "nominal FP64 rate of the profiling recipe (1.25 TFLOP/s)",
                    "hbm_gbs_at_algorithmic_bytes": bpu * units / (ms * 1e-3) / 1e9})
    return out


def dominant_roofline(prof, w, k, mixed, phi_bytes, B, units, fb):
    """The kernel with the largest share of the timed CG time, against its own
    bound: HBM for the FP32 kernels (algorithmic bytes / CUDA-event mean),
    the FP64 pipe for the FP64 ones."""
    names = [n for n in ("expand", "spmv", "update", "project") if prof["samples"][n]]
    tot = {n: (prof["mean_ms"][n] or 0.0) * prof["samples"][n] for n in names}
    dom = max(names, key=lambda n: tot[n])
    mean_s = prof["mean_ms"][dom] * 1e-3
    if mixed:
        hbm, src = hbm_peak()
        flops, byts = kernel_work(dom, w.dim, k, phi_bytes, 4, True, B)
        ach = byts * units / mean_s / 1e9
        roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": profile_traffic(dom + "_mixed", w.name),
                "peak_source": src}
    else:
        flops, byts = kernel_work_fp64(dom, w.dim, k, fb, B)
        ach = flops * units / mean_s / 1e12
        roof = {"kernel": f"k_{dom}", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": profile_traffic(dom + "_fp64", w.name),
                "peak_source": "nominal FP64 rate of the profiling recipe (1.25 TFLOP/s)"}
    roof.update({"algorithmic_flops_per_launch": flops * units,
                 "algorithmic_bytes_per_launch": byts * units,
                 "hbm_gbs_at_algorithmic_bytes": byts * units / mean_s / 1e9,
                 "mean_launch_ms": prof["mean_ms"][dom], "timed_launches": prof["samples"][dom],
                 "kernel_mean_ms": {n: prof["mean_ms"][n] for n in names + ["resid"]},
                 "units_per_launch": units})
    return roof


def kernel_work_fp64(name, dim, k, batched, B):
    """(flops, bytes) per dof and instance of one launch of an FP64-path CG
    kernel.  Batched (8 or more instances): the update writes v = S z - r and
    one GEMM projects the batch (modes read once per tile of the batch); one
    instance at a time: the update projects S z - r itself and the expansion
    reads the modes per instance."""
    share = B if batched else 1
    if name == "update":   # r, q, p, x read; r, x written (+ v); mask; stencil
        f = stencil_flops(dim) + 9 + (0 if batched else 2 * k)
        b = 7 * 8 + 1 + (8 if batched else k * 8)
        return f, b
    if name == "expand":   # r, p read; p written; mask; modes (once per group of 32)
        groups = -(-B // 32) if batched else 1
        return 2 * k + 4, 3 * 8 + 1 + k * 8 * groups / share
    if name == "spmv":     # p read, q written, mask
        return stencil_flops(dim) + 2, 2 * 8 + 1
    if name == "project":  # v read; modes shared by the batch
        return 2 * k, 8 + k * 8 / share
    raise ValueError(name)


def reference_modes(w, G, sdf, mode, dtype, args):
    """Reference modes Phi of the workload on the GPU, as the configuration
    names them: closed-form sines (Sec. 2.2.8; the b = 0 reference of the
    convection workload) or the k smallest eigenpairs of A by the library's
    Chebyshev-filtered subspace iteration (Sec. 2.2.2), timed separately."""
    import torch
    info = {"source": mode}
    if mode == "analytic":
        phi, _ = G.analytic_modes(w.k, dtype)
        info["method"] = "closed-form Kronecker sines on the GPU (Sec. 2.2.8)"
        return phi, info
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi, _, _, est = G.eig_modes(w.k, degree=args.eig_degree, max_iter=4000)
    torch.cuda.synchronize()
    info.update({"seconds": time.perf_counter() - t0, "passes": est["iters"],
                 "converged": bool(est["converged"]), "max_rel_resid": est["max_rel_resid"],
                 "block_matvecs": est["matvecs"],
                 "method": "Chebyshev-filtered subspace iteration on A, FP64, timed separately"})
    if dtype == sdf.F32:
        phi = phi.float().contiguous()
    elif dtype == sdf.BF16:
        phi = phi.to(torch.bfloat16).contiguous()
    return phi, info


def timed_steps(G, steps, run_step, world, dev):
    """Time exactly `steps` calls of run_step(i) on the device: barrier and
    synchronize on both sides, CUDA events on the solve's stream, clocks
    sampled meanwhile; returns (ms, per-step results, clock summary)."""
    import torch
    import torch.distributed as dist
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        torch.cuda.nvtx.range_push("timed_region")
        e0.record(stream)
        for i in range(steps):
            # each solve returns a fresh statistics list (the output buffers
            # are reused between steps)
            res.append({"stats": run_step(i)["stats"]})
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    return max_over_ranks(e0.elapsed_time(e1), dev, world), res, clk.summary()


def mean_stat(stats, f):
    return float(np.mean([f(s) for s in stats])) if stats else None


def cpu_leg(w, inst, stats):
    """The oracle on a bounded sample of this workload (one restricted A-DEF2
    solve at the full size truncated at a few CG iterations, closed-form modes
    of the same k), scaled to the run's mean outer and CG iterations."""
    outer = mean_stat(stats, lambda s: s["outer_iters"])
    iters = mean_stat(stats, lambda s: sum(s["cg_iters"]))
    m_iters = 20 if w.N * w.k <= 2e8 else 5
    ts, ti, cores = cpu_sample(w, inst, m_iters)
    per = outer * ts + iters * ti
    return {"value": 1.0 / per, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle A-DEF2 at the full {w.n}^{w.dim} size on one instance, one "
                       f"restricted solve truncated at {m_iters} CG iterations (set-up {ts:.2f} s, "
                       f"{ti * 1e3:.1f} ms per iteration); instances/s = 1/(outer*t_setup + "
                       f"iters*t_iter) with this run's mean outer={outer:.2f}, iters={iters:.0f}")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="diff3d_128", choices=sorted(MODES))
    ap.add_argument("--n", type=int, default=0,
                    help="grid override (profiling captures and reduced-size runs)")
    ap.add_argument("--max-cg", type=int, default=0, help="CG cap (profiling captures only)")
    ap.add_argument("--path", default="", choices=["", "plain", "mixed"],
                    help="plain: FP64 A-DEF2; mixed: FP32/BF16 with FP64 refinement "
                         "(default: the workload's configuration)")
    ap.add_argument("--phi", default="", choices=["", "f32", "bf16"], help="mode storage (mixed)")
    ap.add_argument("--modes", default="", choices=["", "analytic", "eig"])
    ap.add_argument("--eig-degree", type=int, default=240)
    ap.add_argument("--batch", type=int, default=0, help="instances per step and GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="steps of the end-to-end (host-buffer) measurement")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-deflate", action="store_true",
                    help="plain Jacobi-PCG (no deflation) on the same workload and path")
    ap.add_argument("--plain-instances", type=int, default=8,
                    help="instances of the plain per-instance FP64 comparison")
    ap.add_argument("--no-learned", action="store_true",
                    help="the headline workload without the learned warm start")
    ap.add_argument("--train", type=int, default=0,
                    help="training instances of the learned warm start (default: the workload's)")
    ap.add_argument("--train-rtol", type=float, default=1e-3,
                    help="CG tolerance of the training solves")
    ap.add_argument("--held-out", type=int, default=0,
                    help="held-out instances cycled by the timed steps (default: the workload's)")
    ap.add_argument("--epochs", type=int, default=2000, help="Adam epochs of the warm-start MLP")
    ap.add_argument("--spacetime", default="",
                    help="also time this space-time workload (App. E.2) with the Kronecker "
                         "basis, the constant-in-time lift and plain PCG")
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
    mode = resolve_mode(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, w, mode, world)

    import torch
    import torch.distributed as dist
    from paper_2606_17971_b300 import sdf

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    if mode.get("learned"):
        line = headline_run(args, w, mode, sdf, dev, world, rank)
    else:
        line = workload_run(args, w, mode, sdf, dev, world, rank)
    if rank == 0:
        if args.spacetime:
            line["spacetime"] = spacetime_leg(W.WORKLOADS[args.spacetime], sdf, dev)
        if args.csr_n:
            line["csr_path"] = csr_leg(args.csr_n, sdf, dev)
        if args.diag_sweep:
            line["diagnostics_sweep"] = diag_sweep_leg(args.diag_n, args.diag_sweep, sdf, dev)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def base_line(w, mode, B, world, steps, warm, ms, mixed):
    return {
        "metric": METRIC, "value": steps * B * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic (seeded draws of the workload's parameter law)"}


def workload_run(args, w, mode, sdf, dev, world, rank):
    """One batch per step of a workload without the learned start: configs 0-3
    (and the space-time workload), on the FP64 or the mixed path."""
    import torch
    from paper_2606_17971_b300 import workloads as W
    mixed = mode["path"] == "mixed"
    phi_dt = (sdf.BF16 if mode.get("phi") == "bf16" else sdf.F32) if mixed else sdf.F64
    phi_bytes = (2 if phi_dt == sdf.BF16 else 4) if mixed else 8
    B = mode["batch"]
    steps, warm = args.steps, args.warmup
    kap = W.kappa_field(w)
    G = sdf.Problem(w.dim, w.n, alpha=w.alpha, kappa=kap, diff_scale=w.diff_scale,
                    convection=w.convection, yd_sigma=w.sigma, device=dev)
    phi, modes_info = reference_modes(w, G, sdf, mode["modes"], phi_dt, args)
    G.set_modes(phi)
    insts = W.draw_instances(w, count=max(w.instances, (steps + warm) * B * world))
    mine = shard(insts, rank, world)
    batches = [torch.as_tensor(W.instances_array(mine[(i * B) % len(mine):][:B]), device=dev)
               for i in range(steps + warm)]
    psi = torch.full((w.N,), w.psi, dtype=torch.float64, device=dev)
    opts = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED if mixed else sdf.PREC_F64,
                            max_cg=1000000, deflate=0 if args.no_deflate else 1)
    if args.max_cg:
        opts.max_cg = args.max_cg
    out = {"y": torch.empty((B, w.N), dtype=torch.float64, device=dev), "lam": None,
           "active": torch.empty((B, w.N), dtype=torch.uint8, device=dev)}
    tuned = G.autotune(batches[0], psi, opts) if (mixed and w.dim == 3) else 0
    for i in range(warm):
        G.solve(batches[i], psi, opts, out=out, want_lambda=False)
    opts.profile = 1
    G.reset_profile()
    ms, res, clk = timed_steps(G, steps, lambda i: G.solve(batches[warm + i], psi, opts, out=out,
                                                           want_lambda=False), world, dev)
    prof = G.profile()
    stats = [s for r in res for s in r["stats"]]
    line = base_line(w, mode, B, world, steps, warm, ms, mixed)
    units = w.N * B
    fb = (not mixed) and B >= 8
    roof = dominant_roofline(prof, w, w.k, mixed, phi_bytes, B, units, fb)
    roof["loop"] = loop_roofline(prof, w, w.k, mixed, phi_bytes, B, units)
    line["config"] = workload_config(w, mode, world, args)
    line["path"] = (("mixed FP32 / %s modes, FP64 x, reductions, coarse operator and residual "
                     "replacement" % mode.get("phi") if mixed else
                     ("FP64 A-DEF2, shared-Phi batch kernels" if fb else
                      "FP64 A-DEF2, one instance per launch")) + " (primal active-set loop)"
                    + (", deflation off (plain Jacobi-PCG)" if args.no_deflate else ""))
    line["modes"] = modes_info
    if tuned:
        line["autotuned"] = {"column_depth": tuned, "instance_pairs": G.autotune_choice(B)[1]}
    line.update({
        "cg_iters_per_instance": mean_stat(stats, lambda s: sum(s["cg_iters"])),
        "outer_iters_per_instance": mean_stat(stats, lambda s: s["outer_iters"]),
        "statuses": sorted(set(s["status"] for s in stats)),
        "floor_stops": int(sum(sum(s["floor_stop"]) for s in stats)),
        "max_true_relres": float(max(s["true_relres"][-1] for s in stats)),
        "max_relres_floor": float(max(max(s["relres_floor"]) for s in stats)),
        "roofline": roof, "clocks": clk, "gpu_launches": int(prof["launches"])})
    if not args.no_e2e:
        ne = min(steps, args.e2e_steps)
        inst_h = [b.cpu().pin_memory() for b in batches[warm:warm + ne]]
        psi_h = torch.full((w.N,), w.psi, dtype=torch.float64).pin_memory()
        y_h = torch.empty((B, w.N), dtype=torch.float64).pin_memory()
        a_h = torch.empty((B, w.N), dtype=torch.uint8).pin_memory()
        opts.profile = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(ne):
            G.solve_host(inst_h[i].numpy(), psi_h.numpy(), opts, y=y_h.numpy(), active=a_h.numpy())
        te = max_over_ranks(time.perf_counter() - t0, dev, world)
        line["e2e"] = {"value": ne * B * world / te, "unit": UNIT,
                       "h2d_bytes_per_step": int(inst_h[0].numel() * 8 + psi_h.numel() * 8),
                       "d2h_bytes_per_step": int(y_h.numel() * 8 + a_h.numel()),
                       "steps": ne, "path": "sdf_solve_batch_host (C ABI, host buffers)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_leg(w, mine[0], stats)
    return line


def headline_run(args, w, mode, sdf, dev, world, rank):
    """Config 4: the batched + mixed + learned form on held-out batches, against
    the plain per-instance FP64 path and against the same batches solved
    cold.  Training (untimed): the first (unconstrained) solve of each
    training instance by the batched solver, POD of the states, full-batch
    Adam of the MLP on the tensor cores."""
    import torch
    from paper_2606_17971_b300 import workloads as W
    mixed = True
    phi_dt = sdf.BF16 if mode.get("phi") == "bf16" else sdf.F32
    phi_bytes = 2 if phi_dt == sdf.BF16 else 4
    B = mode["batch"]
    steps, warm = args.steps, args.warmup
    G = sdf.Problem(w.dim, w.n, alpha=w.alpha, kappa=W.kappa_field(w), yd_sigma=w.sigma,
                    device=dev)
    phi, modes_info = reference_modes(w, G, sdf, mode["modes"], phi_dt, args)
    G.set_modes(phi)
    psi = torch.full((w.N,), w.psi, dtype=torch.float64, device=dev)
    # held-out instances, in batches of B, cycled by the timed steps
    n_held = args.held_out or w.extra.get("held_out", 1024)
    held = shard(W.draw_instances(w, count=n_held * world), rank, world)
    nb = max(1, len(held) // B)
    batches = [torch.as_tensor(W.instances_array(held[i * B:(i + 1) * B]), device=dev)
               for i in range(nb)]
    opts = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED, max_cg=1000000)
    if args.max_cg:
        opts.max_cg = args.max_cg
    out = {"y": torch.empty((B, w.N), dtype=torch.float64, device=dev), "lam": None,
           "active": torch.empty((B, w.N), dtype=torch.uint8, device=dev)}

    # ---- training (untimed) ----
    t0 = time.perf_counter()
    ntr = args.train or w.extra.get("train", 2000)
    tr = W.draw_instances(w, count=ntr, seed=w.seed + 1000 + rank)
    it_tr = torch.as_tensor(W.instances_array(tr), device=dev)
    o1 = sdf.default_opts(check_every=128, precision=sdf.PREC_MIXED, max_outer=1,
                          rtol=args.train_rtol)
    Ytr = torch.empty((ntr, w.N), dtype=torch.float64, device=dev)
    for j in range(0, ntr, B):
        Ytr[j:j + B] = G.solve(it_tr[j:j + B].contiguous(), psi, o1, want_lambda=False)["y"]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    widths = (1 + w.dim, 256, 256, 256, 64)
    lo, hi = W.input_box(w)
    model = sdf.WarmModel(widths, w.N, lo, hi, torch.from_numpy(W.mlp_init(widths)).to(dev))
    loss = model.fit(Ytr, it_tr, epochs=args.epochs, lr0=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del Ytr
    torch.cuda.empty_cache()
    train_info = {"instances": ntr, "rtol": args.train_rtol, "solve_s": t1 - t0, "fit_s": t2 - t1,
                  "epochs": args.epochs, "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
                  "widths": list(widths), "pod_rank": 64, "pod_snapshots": min(ntr, 384),
                  "note": "first (unconstrained) solves of separate training instances; "
                          "not part of the timed region"}

    # ---- plain per-instance FP64 path on the first held-out instances ----
    plain = None
    if not args.no_plain:
        Gp = sdf.Problem(w.dim, w.n, alpha=w.alpha, kappa=W.kappa_field(w), yd_sigma=w.sigma,
                         device=dev)
        php, _ = reference_modes(w, Gp, sdf, mode["modes"], sdf.F64, args)
        Gp.set_modes(php)
        op = sdf.default_opts(check_every=128, max_cg=1000000)
        npl = min(args.plain_instances, B)
        Gp.solve(batches[0][:1].contiguous(), psi, op, want_lambda=False)  # warm-up instance
        stream = torch.cuda.current_stream()
        ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ep0.record(stream)
        pst = []
        for i in range(npl):
            pst += Gp.solve(batches[0][i:i + 1].contiguous(), psi, op, want_lambda=False)["stats"]
        ep1.record(stream)
        torch.cuda.synchronize()
        plain = {"value": npl / (ep0.elapsed_time(ep1) * 1e-3), "unit": UNIT,
                 "instances_timed": npl,
                 "cg_iters_per_instance": mean_stat(pst, lambda s: sum(s["cg_iters"])),
                 "statuses": sorted(set(s["status"] for s in pst)),
                 "note": "same workload and held-out instances, one instance per launch, "
                         "after one warm-up instance"}
        del Gp, php
        torch.cuda.empty_cache()

    tuned = G.autotune(batches[0], psi, opts)

    def learned_step(inst):
        x0 = model.predict(inst)
        return G.solve_x0(inst, psi, x0, opts, out=out, want_lambda=False)

    def timed_solve(fn):
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), {"stats": r["stats"]}

    # ---- warm-up: one learned step, then cold solves of held-out batches
    # (each held-out batch is solved cold once, for the comparison) ----
    cold = {}
    learned_step(batches[0])
    for i in range(warm - 1):
        b = i % nb
        if b not in cold:
            cold[b] = timed_solve(lambda: G.solve(batches[b], psi, opts, out=out,
                                                  want_lambda=False))
        else:
            learned_step(batches[b])
    torch.cuda.synchronize()

    # ---- timed region: learned steps over the held-out batches ----
    opts.profile = 1
    G.reset_profile()
    ms, res, clk = timed_steps(G, steps, lambda i: learned_step(batches[i % nb]), world, dev)
    prof = G.profile()
    opts.profile = 0
    stats = [s for r in res for s in r["stats"]]

    # ---- the other held-out batches, cold, on their first 32 instances
    # (untimed; iteration counts per instance against the learned step's) ----
    nsl = min(32, B)
    cold_slices = {}
    for b in range(nb):
        if b not in cold:
            cold_slices[b] = timed_solve(lambda: G.solve(batches[b][:nsl].contiguous(), psi, opts,
                                                         want_lambda=False))
    # learned against cold iterations and ms per held-out batch
    per_batch = []
    for b in range(nb):
        i = next((i for i in range(steps) if i % nb == b), None)
        if i is not None:
            lst = res[i]["stats"]
            lrn_ms = ms / steps
        else:
            lrn_ms, rl = timed_solve(lambda: learned_step(batches[b]))
            lst = rl["stats"]
        full = b in cold
        cms, rc = cold[b] if full else cold_slices[b]
        cst = rc["stats"]
        lst = lst[:len(cst)]
        # the learned start changes the CG iterations only: the outer
        # iterations and the active-set sizes of every solve equal the cold ones
        same = all(a["outer_iters"] == c["outer_iters"] and a["n_active"] == c["n_active"]
                   for a, c in zip(lst, cst))
        per_batch.append({"batch": b, "instances_compared": len(cst),
                          "cold_ms": cms if full else None,
                          "learned_ms": lrn_ms if full else None,
                          "cold_cg_iters": mean_stat(cst, lambda s: sum(s["cg_iters"])),
                          "learned_cg_iters": mean_stat(lst, lambda s: sum(s["cg_iters"])),
                          "outer_and_active_sizes_equal": same})
    # relative error of the prediction against the first (unconstrained)
    # solve, on 16 held-out instances
    sl = batches[0][:16].contiguous()
    first = G.solve(sl, psi, sdf.default_opts(precision=sdf.PREC_MIXED, max_outer=1),
                    want_lambda=False)["y"]
    pred_err = ((model.predict(sl) - first).norm() / first.norm()).item()

    line = base_line(w, mode, B, world, steps, warm, ms, mixed)
    units = w.N * B
    roof = dominant_roofline(prof, w, w.k, True, phi_bytes, B, units, False)
    roof["loop"] = loop_roofline(prof, w, w.k, True, phi_bytes, B, units)
    line["config"] = workload_config(w, mode, world, args)
    line["path"] = ("mixed FP32 / %s modes, FP64 x, reductions, coarse operator and residual "
                    "replacement, learned warm start (primal active-set loop)" % mode.get("phi"))
    line["modes"] = modes_info
    line["autotuned"] = {"column_depth": tuned, "instance_pairs": G.autotune_choice(B)[1]}
    cold_ms = float(np.mean([c[0] for c in cold.values()]))
    cold_it = float(np.mean([p["cold_cg_iters"] for p in per_batch]))
    lrn_cmp = float(np.mean([p["learned_cg_iters"] for p in per_batch]))
    lrn_it = mean_stat(stats, lambda s: sum(s["cg_iters"]))
    line.update({
        "cg_iters_per_instance": lrn_it,
        "outer_iters_per_instance": mean_stat(stats, lambda s: s["outer_iters"]),
        "statuses": sorted(set(s["status"] for s in stats)),
        "floor_stops": int(sum(sum(s["floor_stop"]) for s in stats)),
        "max_true_relres": float(max(s["true_relres"][-1] for s in stats)),
        "roofline": roof, "clocks": clk,
        # the solver's launches plus the prediction's per step: per layer one
        # weight conversion and one product, then input conversion, input
        # scaling and the expansion
        "gpu_launches": int(prof["launches"]) + steps * (2 * 4 + 3),
        "learned": {"training": train_info,
                    "cold": {"ms_per_batch": cold_ms, "cg_iters_per_instance": cold_it,
                             "instances_per_s": B / (cold_ms * 1e-3)},
                    "learned_vs_cold": {"cg_iters": lrn_cmp / cold_it,
                                        "ms": (ms / steps) / cold_ms,
                                        "note": "iterations: the same instances, every held-out "
                                                "batch; ms: the timed steps against the full "
                                                "cold batches solved during warm-up"},
                    "prediction_rel_error_first_solve": pred_err,
                    "per_batch": per_batch}})
    if plain:
        line["plain_fp64_per_instance"] = plain
        line["speedup_vs_plain"] = line["value"] / plain["value"]
    if not args.no_e2e:
        ne = min(steps, args.e2e_steps)
        inst_h = [batches[i % nb].cpu().pin_memory() for i in range(ne)]
        psi_h = torch.full((w.N,), w.psi, dtype=torch.float64).pin_memory()
        y_h = torch.empty((B, w.N), dtype=torch.float64).pin_memory()
        a_h = torch.empty((B, w.N), dtype=torch.uint8).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(ne):
            G.solve_learned_host(model, inst_h[i].numpy(), psi_h.numpy(), opts, y=y_h.numpy(),
                                 active=a_h.numpy())
        te = max_over_ranks(time.perf_counter() - t0, dev, world)
        line["e2e"] = {"value": ne * B * world / te, "unit": UNIT,
                       "h2d_bytes_per_step": int(inst_h[0].numel() * 8 + psi_h.numel() * 8),
                       "d2h_bytes_per_step": int(y_h.numel() * 8 + a_h.numel()), "steps": ne,
                       "path": "sdf_solve_batch_learned_host (C ABI: host mu in, prediction "
                               "and solve on the device, host y and A out)"}
    if not args.no_diag and rank == 0:
        ref = out["active"][0].clone()
        G.diag_active_sets(ref, out["active"], r=w.k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dg = G.diag_active_sets(ref, out["active"], r=w.k)
        td = time.perf_counter() - t0
        line["diagnostics"] = {"active_sets": B, "N": w.N, "r": w.k, "ms": 1e3 * td,
                               "delta_max": float(dg["delta"].max()),
                               "rho_mean": float(dg["rho"].mean()),
                               "note": "sdf_diag_active_sets, host round trip included"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_leg(w, held[0], stats)
    return line


if __name__ == "__main__":
    main()
