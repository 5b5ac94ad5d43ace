"""Writes oracle_iters_to_tol.json: iterations the FP64 oracle needs to reach a
relative residual of 1e-3 on the benchmark workloads (used to scale timed
oracle samples to whole solves).  Calls only the oracle and the input generators.

Steps follow the library's recipe: Jacobi scaling from the closed-form diagonal
of the dual Hessian and lambda = 1 / (1.02 * largest eigenvalue of the scaled
Hessian), the eigenvalue by power iteration with Algorithm 1.

    python tests/golden/make_oracle_iters_to_tol.py [barcelona|tiny] ...
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.harness import closed_form_steps, oracle_build, oracle_power_lambda  # noqa: E402

TOL = 1e-3
CAP = 200000


def run(name):
    P = {"barcelona": synth.barcelona, "tiny": synth.tiny, "large": synth.large}[name](0)
    tree, fac, cu = oracle_build(P)
    unit = closed_form_steps(fac, tree, 1.0)
    L = oracle_power_lambda(fac, tree, unit, iters=100)
    steps = closed_form_steps(fac, tree, 1.0 / (1.02 * L))
    t0 = time.time()
    R = oracle.apg(fac, tree, cu, P["cost"], P["p"], steps, CAP, tol=TOL)
    return {"iterations": int(len(R.rho_rel)), "rho_rel": float(R.rho_rel[-1]), "tol": TOL,
            "lambda_scaled": 1.0 / (1.02 * L), "seconds": time.time() - t0, "nodes": tree.n}


if __name__ == "__main__":
    path = os.path.join(HERE, "oracle_iters_to_tol.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in sys.argv[1:] or ["barcelona"]:
        out[name] = run(name)
        json.dump(out, open(path, "w"), indent=1)
        print(name, out[name], flush=True)
