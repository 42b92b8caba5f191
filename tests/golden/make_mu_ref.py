"""Write the oracle's reference cut values mu_ref of the benchmark workloads
into tests/golden/mu_ref.json.

Time-to-cut (the benchmark's second metric) is the time until the sweep cut
after an IRLS step comes within 1e-6 relative of mu_ref, the value of the
sweep cut (Section 3.3) of the FP64 oracle's last iterate of the same
workload: x^(0) (W^(0) = C) and T IRLS steps (Section 2.1), eps_l =
max(0.1 * 2^-(l-1), 1e-6), each reduced system (Eq. reduced-laplacian-system)
solved by the oracle's Jacobi-PCG to ||r|| <= 1e-12 ||b||, warm-started from
the previous iterate.  This script calls only the oracle and the seeded input
generators; the PCG runs in the oracle's C restatement over every host core.

    python tests/golden/make_mu_ref.py [grid64] [grid2048] [vol256]

The sequence of related 128^3 volume problems (capacities of problem k+1 =
those of problem k times exp(N(0, 0.01)) per edge, seed 5) gets one mu_ref per
evaluation problem (the second half, problems 100-199) in
tests/golden/mu_ref_seq128.json: x^(0) from zero and T = 30 IRLS steps per
problem, each system solved by the oracle's Jacobi-PCG to ||r|| <= 1e-3 ||b||
(the sequence's tolerance, as in the paper's warm-start experiment), each
warm-started from the previous iterate; the file is rewritten after every
problem, and a rerun continues after the last problem written.

    python tests/golden/make_mu_ref.py seq128
    python tests/golden/make_mu_ref.py seq128 A B    # problems A..B-1 into a part file
    python tests/golden/make_mu_ref.py seq128-merge  # fold the part files in
"""
from __future__ import annotations

import datetime
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle as O  # noqa: E402
from oracle import pcg_omp  # noqa: E402

OUT = os.path.join(HERE, "mu_ref.json")
OUT_SEQ = os.path.join(HERE, "mu_ref_seq128.json")
SEQ_PROBLEMS, SEQ_T, SEQ_TOL = 200, 30, 1e-3
# workload -> (generator number, IRLS steps T)
WORKLOADS = {"grid64": (1, 50), "grid2048": (2, 50), "vol256": (3, 30)}
TOL = 1e-12


def run(name):
    k, T = WORKLOADS[name]
    t0 = time.time()
    g = gen.config_graph(k)
    prob = O.Problem.from_graph(g)
    eps = O.eps_schedule(T)
    nt = prob.nonterminals
    steps = []
    x = None
    for l in range(T + 1):
        gl = O.initial_conductance(prob) if l == 0 else O.reweight(prob, x, eps[l - 1])
        Lt, b = O.reduced_system(prob, O.laplacian(prob, gl))
        v, it, rel = pcg_omp.pcg_jacobi(Lt, b, None if x is None else x[nt], tol=TOL, maxit=10 ** 7)
        if rel > TOL:
            raise RuntimeError(f"{name} step {l}: PCG stopped at {rel:.3e}")
        x = prob.full_x(v)
        mu = O.sweep_cut(prob, x)["value"]
        steps.append({"step": l, "eps": eps[l - 1] if l else 0.0, "pcg_iters": it,
                      "rel_residual": rel, "sweep_value": mu})
        print(f"{name} step {l}: {it} PCG iterations, sweep {mu:.12g} ({time.time() - t0:.0f} s)",
              flush=True)
    mu_ref = steps[-1]["sweep_value"]
    first = next(s["step"] for s in steps
                 if all(abs(t["sweep_value"] - mu_ref) <= 1e-6 * mu_ref for t in steps[s["step"]:]))
    return {
        "workload": g.name, "generator": f"gen.config_graph({k})", "T": T,
        "eps": "max(0.1 * 2^-(l-1), 1e-6)", "pcg": f"oracle Jacobi-PCG, tol {TOL}, warm start",
        "mu_ref": mu_ref,
        "first_step_within_1e-6_for_good": first,
        "steps": steps,
        "seconds": time.time() - t0,
        "host": f"{platform.machine()}, {pcg_omp.max_threads()} OpenMP threads",
        "date": datetime.date.today().isoformat(),
        "command": "python tests/golden/make_mu_ref.py " + name,
    }


def irls_sweeps(prob, T, tol):
    """x^(0) from zero, then T warm-started IRLS steps; the sweep value after
    each step and the PCG iterations of each solve."""
    eps = O.eps_schedule(T)
    nt = prob.nonterminals
    x, sweeps, iters = None, [], []
    for l in range(T + 1):
        gl = O.initial_conductance(prob) if l == 0 else O.reweight(prob, x, eps[l - 1])
        Lt, b = O.reduced_system(prob, O.laplacian(prob, gl))
        v, it, rel = pcg_omp.pcg_jacobi(Lt, b, None if x is None else x[nt], tol=tol, maxit=10 ** 7)
        if rel > tol:
            raise RuntimeError(f"step {l}: PCG stopped at {rel:.3e}")
        x = prob.full_x(v)
        sweeps.append(O.sweep_cut(prob, x)["value"])
        iters.append(it)
    return sweeps, iters


def run_sequence(lo=None, hi=None, base=None, problems=SEQ_PROBLEMS, T=SEQ_T, tol=SEQ_TOL,
                 main=OUT_SEQ):
    """The sequence's evaluation problems lo..hi-1 (default: the second half)
    into ``main``, or into a part file next to it when a range is given.
    ``base`` (default: the 128^3 volume, gen.config_graph(5)), ``problems``,
    ``T`` and ``tol`` are there so that a test can run a small sequence."""
    lo = problems // 2 if lo is None else lo
    hi = problems if hi is None else hi
    out = main if (lo, hi) == (problems // 2, problems) else main[:-5] + f".part{lo}-{hi}.json"
    data = {"workload": "seq128", "generator": "gen.config_graph(5), gen.capacity_sequence(seed=5, sigma=0.01)",
            "problems": problems, "evaluation": [problems // 2, problems - 1], "T": T,
            "eps": "max(0.1 * 2^-(l-1), 1e-6)",
            "pcg": f"oracle Jacobi-PCG, tol {tol}, x^(0) from zero, steps warm-started",
            "command": "python tests/golden/make_mu_ref.py seq128", "mu_ref": {}}
    if os.path.exists(out):
        with open(out) as f:
            data = json.load(f)
    base = gen.config_graph(5) if base is None else base
    t0 = time.time()
    for k, c in enumerate(gen.capacity_sequence(base, problems, seed=5, sigma=0.01)):
        if k >= hi:
            break
        if k < lo or str(k) in data["mu_ref"]:
            continue
        prob = O.Problem.from_graph(gen.Graph(base.n, base.row_ptr, base.col, c, base.s, base.t))
        sweeps, iters = irls_sweeps(prob, T, tol)
        mu = sweeps[-1]
        first = next(l for l in range(len(sweeps))
                     if all(abs(v - mu) <= 1e-6 * mu for v in sweeps[l:]))
        data["mu_ref"][str(k)] = {"mu_ref": mu, "first_step_within_1e-6_for_good": first,
                                  "pcg_iters": int(sum(iters)), "pcg_iters_x0": int(iters[0])}
        data["host"] = f"{platform.machine()}, {pcg_omp.max_threads()} OpenMP threads"
        data["date"] = datetime.date.today().isoformat()
        with open(out, "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")
        print(f"seq128 problem {k}: mu_ref {mu:.12g}, step {first}, {sum(iters)} PCG iterations "
              f"({time.time() - t0:.0f} s)", flush=True)


def merge_sequence_parts(main=OUT_SEQ):
    """Fold the part files of run_sequence into ``main``
    (tests/golden/mu_ref_seq128.json)."""
    import glob
    with open(main) as f:
        data = json.load(f)
    parts = sorted(glob.glob(main[:-5] + ".part*.json"))
    for path in parts:
        with open(path) as f:
            data["mu_ref"].update(json.load(f)["mu_ref"])
    data["mu_ref"] = {k: data["mu_ref"][k] for k in sorted(data["mu_ref"], key=int)}
    with open(main, "w") as f:
        json.dump(data, f, indent=1)
        f.write("\n")
    for path in parts:
        os.remove(path)
    print(f"seq128: {len(data['mu_ref'])} problems")


def main(argv):
    if argv and argv[0] == "seq128":
        run_sequence(*[int(a) for a in argv[1:3]])
        return 0
    if argv == ["seq128-merge"]:
        merge_sequence_parts()
        return 0
    names = argv or list(WORKLOADS)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        data[name] = run(name)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1)
            f.write("\n")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
