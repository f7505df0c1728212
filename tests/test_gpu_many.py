"""cp_solve_many (many small 3-way dense solves in one persistent launch, one
thread-block cluster per request at a time) against the FP64 oracle, through
the C ABI.

FP64 requests must follow the oracle's Algorithm 1: the same iterations and
restarts, f within 1e-10 |f| + 1e-14 ||T||^2 (the whole-solve tolerance of
the single-request path), the oracle's gradient at the returned iterate below
tol, and the iterate within 1e-6 of the oracle's (the solution is fixed only
to the tolerance).  Fixed-iteration runs pin the first iterations one by
one.  Mixed requests (FP32 products) must end certified by the oracle's FP64
gradient.  A request's result must not depend on the others in its launch
(bit-identical alone and in a mix) or on the cluster size beyond rounding."""
import numpy as np
import pytest
import torch

import synth
from oracle import cp_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10

# (dims, R, collinearity, noise, dtype): ragged sides, several fiber chunks
# per CTA, both tensor dtypes
CASES = [
    ((20, 20, 20), 3, 0.5, 0.10, np.float64),
    ((12, 10, 8), 4, 0.5, 0.05, np.float32),
    ((24, 16, 20), 5, 0.5, 0.02, np.float32),
    ((9, 31, 14), 2, 0.5, 0.10, np.float64),
    ((33, 17, 40), 6, 0.5, 0.05, np.float32),
]


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1105_5331_gb300 as cp
    return cp


@pytest.fixture(scope="module")
def ctx(cp):
    c = cp.cp_ctx_create(0, torch.cuda.current_stream())
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def problem(k, case):
    dims, R, c, eta, dtype = case
    rng = synth.rng_for(11, k)
    prob = synth.dense_problem(rng, dims, R, c, eta=eta, dtype=dtype)
    return prob, synth.initial_guess(rng, dims, R)


@pytest.fixture(scope="module")
def oracle_solves():
    out = []
    for k, case in enumerate(CASES):
        prob, u0 = problem(k, case)
        X = O.DenseTensor(prob.T.astype(np.float64))
        uo, go, rep = O.cp_solve(X, u0, O.SolveOpts(R=case[1], tol=1e-7))
        out.append((prob, u0, X, uo, rep))
    return out


def opts_for(cp, R, prec="fp64", maxit=None):
    o = cp.cp_solve_opts_default(R)
    o.prec = 0 if prec == "fp64" else 1
    if maxit is not None:
        o.maxit = maxit
    return o


@pytest.mark.parametrize("cluster", [0, 1, 2, 4])
def test_fp64_requests_follow_the_oracle(cp, ctx, oracle_solves, cluster):
    tensors, us, opts = [], [], []
    for (prob, u0, X, uo, rep), case in zip(oracle_solves, CASES):
        tensors.append(cp.cp_tensor_dense(ctx, dev(prob.T)))
        us.append(dev(u0))
        opts.append(opts_for(cp, case[1]))
    reps = cp.cp_solve_many(ctx, tensors, opts, us, cluster=cluster)
    for k, ((prob, u0, X, uo, rep_o), r, ud) in enumerate(zip(oracle_solves, reps, us)):
        R = CASES[k][1]
        u = ud.cpu().numpy()
        print(k, "iters", r["iters"], rep_o.iters, "restarts", r["restarts"], rep_o.restarts, "f", r["f"], rep_o.f)
        assert r["converged"] and rep_o.converged, k
        assert (r["iters"], r["restarts"]) == (rep_o.iters, rep_o.restarts), k
        assert abs(r["f"] - rep_o.f) <= TOL * abs(rep_o.f) + 1e-14 * X.norm2, k
        f, g = O.fg(X, u, R)
        assert np.linalg.norm(g) / O.n_params(prob.dims, R) < 1e-7, k
        assert abs(f - r["f"]) <= TOL * abs(f) + 1e-14 * X.norm2, k
        assert rel(u, uo) <= 1e-6, k
    for t in tensors:
        t.close()


def test_fixed_iterations_follow_the_oracle(cp, ctx):
    """The 20^3 R=3 workload, maxit = 1..6: f, ||g||/P and the counters after
    each iteration against the oracle's run with the same limit."""
    prob, u0 = synth.workload_dense_small()
    R = 3
    X = O.DenseTensor(prob.T)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    P = O.n_params(prob.dims, R)
    js = list(range(1, 7))
    us = [dev(u0) for _ in js]
    reps = cp.cp_solve_many(ctx, [t] * len(js), [opts_for(cp, R, maxit=j) for j in js], us, cluster=2)
    for j, r, ud in zip(js, reps, us):
        uo, go, ro = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7), max_iters=j)
        got = (r["iters"], r["restarts"], r["als_sweeps"], r["ls_failures"])
        want = (ro.iters, ro.restarts, ro.als_sweeps, ro.ls_failures)
        assert got == want, (j, got, want)
        assert abs(r["f"] - ro.f) <= TOL * abs(ro.f) + 1e-14 * X.norm2, j
        gn = np.linalg.norm(go) / P
        assert abs(r["gnorm_over_P"] - gn) <= TOL * gn + 1e-14 * X.norm2 / P, j
        assert rel(ud.cpu().numpy(), uo) <= 1e-8, j
    t.close()


def test_zero_iterations_return_the_normalised_start(cp, ctx):
    prob, u0 = problem(1, CASES[1])
    R = CASES[1][1]
    X = O.DenseTensor(prob.T.astype(np.float64))
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    (r,) = cp.cp_solve_many(ctx, [t], [opts_for(cp, R, maxit=0)], [ud])
    un, _, _ = O.normalize(u0, prob.dims, R)
    f, g = O.fg(X, un, R)
    assert r["iters"] == 0 and not r["converged"]
    assert rel(ud.cpu().numpy(), un) <= 1e-14
    assert abs(r["f"] - f) <= TOL * abs(f) + 1e-14 * X.norm2
    assert abs(r["gnorm_over_P"] - np.linalg.norm(g) / O.n_params(prob.dims, R)) <= 1e-10 * np.linalg.norm(g)
    t.close()


def serving_like(n, seed=3):
    """Small requests shaped like the serving stream's (random sides, ranks,
    collinearity, noise and tolerance), kept small for the oracle."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        dims = tuple(int(x) for x in rng.integers(16, 49, size=3))
        R = int(rng.integers(2, 13))
        c = float(rng.choice([0.5, 0.9]))
        eta = float(rng.uniform(0.01, 0.10))
        tol = float(rng.choice([1e-5, 1e-7]))
        prng = synth.rng_for(12, k)
        prob = synth.dense_problem(prng, dims, R, c, eta=eta, dtype=np.float32)
        out.append((prob, synth.initial_guess(prng, dims, R), R, tol))
    return out


def test_mixed_requests_are_certified_by_the_fp64_gradient(cp, ctx):
    reqs = serving_like(12)
    tensors = [cp.cp_tensor_dense(ctx, dev(p.T)) for p, _, _, _ in reqs]
    us = [dev(u0) for _, u0, _, _ in reqs]
    opts = []
    for _, _, R, tol in reqs:
        o = opts_for(cp, R, prec="mixed")
        o.tol = tol
        opts.append(o)
    reps = cp.cp_solve_many(ctx, tensors, opts, us)
    for (prob, u0, R, tol), r, ud in zip(reqs, reps, us):
        X = O.DenseTensor(prob.T.astype(np.float64))
        f, g = O.fg(X, ud.cpu().numpy(), R)
        gn = np.linalg.norm(g) / O.n_params(prob.dims, R)
        print(prob.dims, R, tol, "mixed", r["mixed_iters"], "fp64", r["fp64_iters"], "gn", gn)
        assert r["converged"]
        assert gn < tol
        assert abs(f - r["f"]) <= TOL * abs(f) + 1e-14 * X.norm2
    for t in tensors:
        t.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_result_alone_equals_result_in_a_mix(cp, ctx, prec):
    reqs = serving_like(5, seed=7)
    tensors = [cp.cp_tensor_dense(ctx, dev(p.T)) for p, _, _, _ in reqs]
    opts = [opts_for(cp, R, prec=prec) for _, _, R, _ in reqs]
    us = [dev(u0) for _, u0, _, _ in reqs]
    mix = cp.cp_solve_many(ctx, tensors, opts, us, cluster=2)
    for k in (0, 3):
        ud = dev(reqs[k][1])
        (alone,) = cp.cp_solve_many(ctx, [tensors[k]], [opts[k]], [ud], cluster=2)
        assert torch.equal(ud, us[k]), k
        for key in ("iters", "restarts", "ls_trials", "f", "gnorm_over_P", "mixed_iters", "fp64_iters"):
            assert alone[key] == mix[k][key], (k, key)
    for t in tensors:
        t.close()


def test_cluster_sizes_agree_to_rounding(cp, ctx, oracle_solves):
    prob, u0, X, uo, rep = oracle_solves[4]
    R = CASES[4][1]
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    res = []
    for cl in (1, 2, 8):
        ud = dev(u0)
        (r,) = cp.cp_solve_many(ctx, [t], [opts_for(cp, R, maxit=5)], [ud], cluster=cl)
        res.append((r, ud.cpu().numpy()))
    for r, u in res[1:]:
        assert r["iters"] == res[0][0]["iters"] and r["restarts"] == res[0][0]["restarts"]
        assert abs(r["f"] - res[0][0]["f"]) <= TOL * abs(res[0][0]["f"])
        assert rel(u, res[0][1]) <= 1e-9
    t.close()


def test_unsupported_requests_are_refused(cp, ctx):
    rng = np.random.default_rng(0)
    T4 = rng.standard_normal((4, 5, 6, 3))
    t4 = cp.cp_tensor_dense(ctx, dev(T4))
    with pytest.raises(cp.CpError) as ei:
        cp.cp_solve_many(ctx, [t4], [opts_for(cp, 2)], [dev(synth.initial_guess(rng, (4, 5, 6, 3), 2))])
    assert ei.value.status == 11
    T = rng.standard_normal((6, 5, 4))
    t = cp.cp_tensor_dense(ctx, dev(T))
    with pytest.raises(cp.CpError) as ei:
        cp.cp_solve_many(ctx, [t], [opts_for(cp, 33)], [dev(synth.initial_guess(rng, (6, 5, 4), 33))])
    assert ei.value.status == 11
    t4.close()
    t.close()


def test_plan_is_tuned_once_per_bucket(cp, ctx):
    """cp_many_plan: a size in {1, 2, 4, 8}, the same on the second call and
    for another request of the same bucket (entries and rank within the same
    powers of two, same precision)."""
    reqs = serving_like(3, seed=9)
    prob, u0, R, _ = reqs[0]
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    o = opts_for(cp, R, prec="mixed")
    c1 = cp.cp_many_plan(ctx, t, o, dev(u0))
    assert c1 in (1, 2, 4, 8)
    assert cp.cp_many_plan(ctx, t, o, dev(u0)) == c1
    # same bucket: one side trimmed by one (entries stay within the power of two)
    dims = prob.dims
    K = int(np.prod(dims))
    lk = int(np.ceil(np.log2(K)))
    T2 = prob.T[:-1]
    if int(np.ceil(np.log2(T2.size))) == lk:
        t2 = cp.cp_tensor_dense(ctx, dev(T2))
        u2 = synth.initial_guess(np.random.default_rng(1), T2.shape, R)
        assert cp.cp_many_plan(ctx, t2, o, dev(u2)) == c1
        t2.close()
    t.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_parking_between_launches_changes_nothing(cp, ctx, prec):
    """Launches of 20 us: every cluster stops after about one iteration and
    leaves its request's state in device memory, and the next launch resumes
    it (window, carried contraction, phase, counters); the results must be
    bit-identical to launches long enough to finish every solve."""
    reqs = serving_like(4, seed=13)
    tensors = [cp.cp_tensor_dense(ctx, dev(p.T)) for p, _, _, _ in reqs]
    opts = []
    for _, _, R, tol in reqs:
        o = opts_for(cp, R, prec=prec)
        o.tol = tol
        opts.append(o)
    us_long = [dev(u0) for _, u0, _, _ in reqs]
    long_ = cp.cp_solve_many(ctx, tensors, opts, us_long, cluster=2)
    try:
        cp.cp_many_set_round(ctx, 20e-6)
        us_short = [dev(u0) for _, u0, _, _ in reqs]
        short = cp.cp_solve_many(ctx, tensors, opts, us_short, cluster=2)
    finally:
        cp.cp_many_set_round(ctx, 0.5)
    for a, b, ua, ub in zip(long_, short, us_long, us_short):
        assert torch.equal(ua, ub)
        for key in ("iters", "restarts", "ls_trials", "ls_failures", "f", "gnorm_over_P", "mixed_iters", "fp64_iters",
                    "converged"):
            assert a[key] == b[key], key
    for t in tensors:
        t.close()


def test_not_spd_request_is_reported(cp, ctx):
    """A zero tensor: the first ALS update zeroes A^(1), so Gammabar^(2) is 0
    and stays singular after the ridge retry (ridge = 1e-12 trace / R = 0):
    the request ends with CP_ERR_NOT_SPD, as the oracle's mode solve raises."""
    T = np.zeros((10, 9, 8), dtype=np.float32)
    rng = np.random.default_rng(3)
    u0 = synth.initial_guess(rng, T.shape, 2)
    X = O.DenseTensor(T.astype(np.float64))
    with pytest.raises(O.NotSPD):
        O.cp_solve(X, u0, O.SolveOpts(R=2, tol=1e-7))
    t = cp.cp_tensor_dense(ctx, dev(T))
    with pytest.raises(cp.CpError) as ei:
        cp.cp_solve_many(ctx, [t], [opts_for(cp, 2)], [dev(u0)], cluster=2)
    assert ei.value.status == 5
    t.close()
