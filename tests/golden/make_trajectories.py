"""Writes tests/golden/trajectories.json: the FP64 oracle's first iterations of
Algorithm 1 (N-GMRES accelerated ALS, Section 2.1) on the full-size
workloads, for the GPU's fixed-iteration trajectory tests.

Calls only the oracle and the seeded input generators.  For each workload and
each iteration j = 1..k it stores the oracle's f and ||g||/P after j
iterations, its counters (iterations, restarts, ALS sweeps, line-search
trials, failed searches), a first-order bound on how far rounding alone can
move the iterate (the ALS sweep bound and the line search's step bound,
accumulated over the iterations done),
and 2000 seeded entries and the norm of the iterate after k iterations.

    python tests/golden/make_trajectories.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import cp_oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "trajectories.json")

# name: (generator, dense?, iterations k)
WORKLOADS = {
    "dense_256": (synth.workload_dense_256, True, 4),
    "sparse_20000": (synth.workload_sparse, False, 3),
    "dense_4way_96": (synth.workload_dense_4way, True, 2),
}


def sweep_bound(X, u, R):
    """First-order bound on the relative change of one ALS sweep's result
    when its sums are rounded differently: mode n solves A^(n) Gammabar^(n) =
    M^(n), so an input perturbation e moves A^(n) by kappa(Gammabar^(n)) e;
    the inputs carry eta = (Kbar + 2R) 2^-53 of summation error plus the
    error of the factors updated before (once in M, twice in the Grams)."""
    F = [A.copy() for A in O.unpack(np.array(u, dtype=np.float64), X.dims, R)]
    K = int(np.prod(X.dims)) if hasattr(X, "T") else len(X.vals)
    errs = []
    for n in range(len(F)):
        Gb = O.gamma_bar(F, n)
        kbar = K // X.dims[n] if hasattr(X, "T") else max(K, max(X.dims))
        errs.append(np.linalg.cond(Gb) * ((kbar + 2 * R) * 2.0 ** -53 + 3.0 * sum(errs)))
        F[n] = O.als_mode_solve(X.mttkrp(F, n), Gb)
    return 3.0 * max(errs)


def step_bound(X, R, ubar, d, beta):
    """First-order bound on the relative move of x = ubar + beta d by rounding
    in the line search's inputs and step:
      * d = uhat - ubar is the difference of two normalised iterates, each
        entry carrying about four roundings of the normalisation (scale,
        root, product), so d is off by up to 4 2^-53 (|ubar| + |uhat|) and x
        by beta times that;
      * the step beta solves phi'(beta) = 0 (or sits where phi' crosses the
        curvature bound); phi'(beta) = g(x) . d is a sum of P products, off
        by at most P 2^-53 sum |g_i d_i| (recursive summation), which moves
        beta by that over |phi''(beta)| (phi'' from a central difference of
        phi'), and x by |delta beta| ||d||."""
    if not beta > 0:
        return 0.0
    P = ubar.size
    x = ubar + beta * d
    _, g = O.fg(X, x, R)
    h = 1e-4 * beta
    _, gp = O.fg(X, ubar + (beta + h) * d, R)
    _, gm = O.fg(X, ubar + (beta - h) * d, R)
    phi2 = abs(float(gp @ d) - float(gm @ d)) / (2 * h)
    noise = P * 2.0 ** -53 * float(np.sum(np.abs(g * d)))
    nx = float(np.linalg.norm(x))
    from_d = beta * 4 * 2.0 ** -53 * (float(np.linalg.norm(ubar)) + float(np.linalg.norm(ubar + d))) / nx
    if phi2 == 0.0:
        return float("inf")
    return from_d + noise / phi2 * float(np.linalg.norm(d)) / nx


def run(name):
    gen, dense, k = WORKLOADS[name]
    prob, u0 = gen()
    R = prob.R
    X = O.DenseTensor(prob.T) if dense else O.SparseTensor(prob.coords, prob.vals, prob.dims)
    P = O.n_params(prob.dims, R)
    # one solve of k iterations; per-iteration counters from the calls it makes
    per_iter, iterates = [], []
    real_ng, real_mt = O.ngmres_step, O.more_thuente

    def ng(U, G, ubar, gbar, eps=1e-12):
        per_iter.append({"restart": True, "ls_trials": 0, "ls_failed": False})
        iterates.append(np.array(U[-1]))   # the iterate u_i this iteration starts from
        return real_ng(U, G, ubar, gbar, eps)

    def mt(phi, f0, g0, opts=O.LSOpts()):
        out = real_mt(phi, f0, g0, opts)
        cells = dict(zip(phi.__code__.co_freevars, (c.cell_contents for c in phi.__closure__)))
        per_iter[-1].update(restart=False, ls_trials=out[4], ls_failed=out[5] != 1,
                            line=(np.array(cells["ubar"]), np.array(cells["d"]), out[0]))
        return out
    O.ngmres_step, O.more_thuente = ng, mt
    t0 = time.time()
    try:
        u, g, rep = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7), max_iters=k)
    finally:
        O.ngmres_step, O.more_thuente = real_ng, real_mt
    t_solve = time.time() - t0
    assert rep.iters == k == len(per_iter)
    # the window's newest point at iteration i is u_i (Algorithm 1), so
    # iterates[i] is u_i; the sweep bound accumulates over u_0 .. u_{j-1}
    bounds, acc = [], 0.0
    for i in range(k):
        acc += sweep_bound(X, iterates[i], R)
        if "line" in per_iter[i]:
            acc += step_bound(X, R, *per_iter[i]["line"])
        bounds.append(acc)
    steps = []
    counts = dict(iters=0, restarts=0, als_sweeps=0, ls_trials=0, ls_failures=0)
    for j in range(1, k + 1):
        it = per_iter[j - 1]
        counts = dict(iters=j, restarts=counts["restarts"] + int(it["restart"]), als_sweeps=j,
                      ls_trials=counts["ls_trials"] + it["ls_trials"],
                      ls_failures=counts["ls_failures"] + int(it["ls_failed"]))
        f, gn = rep.history[j]
        steps.append(dict(counts, f=f, gnorm_over_P=gn, u_bound=bounds[j - 1]))
    F = O.unpack(u, prob.dims, R)
    mnorm = float(np.sqrt(sum(np.sum(X.mttkrp(F, n) ** 2) for n in range(len(F)))))
    out = dict(dims=list(prob.dims), R=R, k=k, P=P, normT2=X.norm2, f0=rep.history[0][0],
               gnorm0=rep.history[0][1], steps=steps, mnorm_final=mnorm,
               u_norm=float(np.linalg.norm(u)), oracle_seconds=t_solve)
    out.update(sample_iterate(u, P))
    return out


def sample_iterate(u, P):
    """2000 seeded entries of the iterate (all of it when P <= 2000)."""
    idx = np.arange(P) if P <= 2000 else np.sort(np.random.default_rng(2000).choice(P, 2000, replace=False))
    return {"u_index": [int(i) for i in idx], "u_sample": [float(u[i]) for i in idx]}


if __name__ == "__main__":
    names = sys.argv[1:] or list(WORKLOADS)
    res = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        res[name] = run(name)
        json.dump(res, open(OUT, "w"), indent=0, sort_keys=True)
        print(name, {k: v for k, v in res[name].items() if k not in ("u_final", "u_index", "u_sample")},
              flush=True)
