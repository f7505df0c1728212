"""Writes oracle/workload_iters.json: the FP64 oracle's own N-GMRES iteration
count, f and ||g||/P at convergence for the named workloads (dense_small,
dense_256, sparse_20000, dense_4way_96; the first two by default).  The CPU-baseline
leg of bench.py uses the count to turn a timed sample of oracle iterations
into solves per second.  Calls only the oracle and the input generators."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import cp_oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_iters.json")


def run(name, prob, u0, R, tol=1e-7):
    X = O.SparseTensor(prob.coords, prob.vals, prob.dims) if name.startswith("sparse") else O.DenseTensor(prob.T)
    t0 = time.time()
    _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=tol))
    return dict(iters=rep.iters, fg_evals=rep.fg_evals, restarts=rep.restarts,
                ls_failures=rep.ls_failures, f=rep.f, gnorm_over_P=rep.gnorm_over_P,
                converged=rep.converged, seconds=time.time() - t0)


if __name__ == "__main__":
    which = sys.argv[1:] or ["dense_small", "dense_256"]
    res = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in which:
        if name == "dense_small":
            prob, u0 = synth.workload_dense_small()
            res[name] = run(name, prob, u0, 3)
        elif name == "dense_256":
            prob, u0 = synth.workload_dense_256()
            res[name] = run(name, prob, u0, 16)
        elif name == "sparse_20000":
            prob, u0 = synth.workload_sparse()
            res[name] = run(name, prob, u0, 10)
        elif name == "dense_4way_96":
            prob, u0 = synth.workload_dense_4way()
            res[name] = run(name, prob, u0, 32)
        json.dump(res, open(OUT, "w"), indent=1, sort_keys=True)
        print(name, res[name], flush=True)
