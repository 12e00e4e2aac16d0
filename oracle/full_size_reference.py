"""Write tests/golden/diff3d_128_oracle.json and diff3d_128_oracle_states.npz:
full-size oracle solves of the first instances of the 128^3 diffusion
workload (k = 60 closed-form reference modes, rtol 1e-8, psi = 1).  The JSON
holds the statistics and the state at 64 sampled nodes; the npz holds every
node of each final state, rounded to float32 (relative rounding 6e-8, far
below the 1e-6 / 1e-5 parity bars) and zlib-compressed.  Calls only the
oracle; takes tens of minutes per instance on a few CPU cores, so it is run
once and its output committed.

TEST INFRASTRUCTURE ONLY: it writes a stored expected value for tests/ and
calls nothing outside oracle/ and the seeded input generators.

Usage: python -m oracle.full_size_reference [count]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2606_17971_b300 import workloads as W  # noqa: E402


def main(count=2, name="diff3d_128"):
    w = W.WORKLOADS[name]
    P = O.Problem(w.dim, w.n, alpha=w.alpha)
    Phi = O.analytic_modes(w.dim, w.n, w.k, w.alpha)[0]
    psi = W.psi_vector(w)
    rng = np.random.default_rng(12345)
    sample = np.sort(rng.choice(w.N, size=64, replace=False))
    out_path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.json")
    npz_path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle_states.npz")
    states = {}
    res = {"workload": name, "rtol": 1e-8, "k": w.k, "modes": "closed-form sines (Sec. 2.2.8)",
           "sample_index": sample.tolist(), "instances": []}
    for i, ins in enumerate(W.draw_instances(w, count=count)):
        _, rhs = P.desired_state(ins.a, ins.c[: w.dim], w.sigma)
        t = time.time()
        r = P.solve(rhs, psi, Phi, rtol=1e-8, max_cg=200000)
        res["instances"].append({
            "index": i, "a": ins.a, "c": list(ins.c), "status": r["status"],
            "outer_iters": r["outer_iters"], "cg_iters": r["cg_iters"], "n_active": r["n_active"],
            "y_norm": float(np.linalg.norm(r["y"])), "y_sample": r["y"][sample].tolist(),
            "active_count": int(r["active"].sum()), "true_relres": r["true_relres"],
            "true_relres_each": r["true_relres_each"], "relres_floor": r["relres_floor"],
            "seconds": time.time() - t, "threads": os.cpu_count()})
        states[f"y{i}"] = r["y"].astype(np.float32)
        states[f"active{i}"] = np.packbits(r["active"].astype(np.uint8))
        with open(out_path, "w") as f:
            json.dump(res, f, indent=1)
        np.savez_compressed(npz_path, **states)
        print(i, r["cg_iters"], r["n_active"], "%.0fs" % (time.time() - t), flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
