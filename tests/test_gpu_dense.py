"""GPU parity of the FP64 dense path against the FP64 oracle, through the C ABI.

Tolerance: 1e-10 relative (Frobenius) for every FP64 per-call result; integer
outcomes of the line search (nfev, info) must be identical."""
import numpy as np
import pytest
import torch

import synth
from oracle import cp_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


SHAPES = [
    ((20, 20, 20), 3, np.float64),
    ((7, 5, 3), 1, np.float32),
    ((13, 9, 11, 2), 17, np.float32),
    ((40, 3), 64, np.float64),
    ((3, 1, 5), 5, np.float64),
    ((65, 70, 33), 33, np.float32),
    ((300, 2, 17), 16, np.float32),
]


def make(shape, R, dtype, seed=0):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal(shape).astype(dtype)
    u = synth.initial_guess(rng, shape, R)
    return T, u


@pytest.mark.parametrize("shape,R,dtype", SHAPES)
def test_mttkrp_fp64_parity(cp, ctx, shape, R, dtype):
    T, u = make(shape, R, dtype)
    t = cp.cp_tensor_dense(ctx, dev(T))
    F = O.unpack(u, shape, R)
    ud = dev(u)
    for n in range(len(shape)):
        out = torch.empty(shape[n] * R, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, R, ud, n, out)
        cp.cp_ctx_sync(ctx)
        ref = O.mttkrp_dense(T.astype(np.float64), F, n)
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL, (shape, R, n)


def test_tensor_norm_and_host_upload(cp, ctx):
    T, _ = make((17, 5, 9), 2, np.float32)
    t_host = cp.cp_tensor_dense(ctx, T)          # host pointer path
    t_dev = cp.cp_tensor_dense(ctx, dev(T))
    n_host = cp.cp_tensor_info(t_host)[2]
    n_dev = cp.cp_tensor_info(t_dev)[2]
    ref = float(np.sum(T.astype(np.float64) ** 2))
    assert abs(n_host - ref) <= 1e-13 * ref and n_host == n_dev


@pytest.mark.parametrize("shape,R,dtype", SHAPES)
def test_fg_parity(cp, ctx, shape, R, dtype):
    T, u = make(shape, R, dtype, seed=1)
    t = cp.cp_tensor_dense(ctx, dev(T))
    ud = dev(u)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(ud)
    cp.cp_fg(ctx, t, R, ud, f, g)
    cp.cp_ctx_sync(ctx)
    fo, go = O.fg(O.DenseTensor(T), u, R)
    assert abs(f.item() - fo) <= TOL * abs(fo)
    assert rel(g.cpu().numpy(), go) <= TOL
    # f without g
    f2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    cp.cp_fg(ctx, t, R, ud, f2, None)
    cp.cp_ctx_sync(ctx)
    assert abs(f2.item() - fo) <= TOL * abs(fo)


ALS_SHAPES = [
    ((20, 20, 20), 3, np.float64),
    ((7, 5, 3), 1, np.float32),
    ((13, 9, 11, 20), 7, np.float32),
    ((65, 70, 33), 33, np.float32),
    ((300, 2, 17), 2, np.float32),
]


def als_sweep_tolerance(X, u, R):
    """Forward-error bound for two FP64 evaluations of one ALS sweep that
    differ only in rounding (order of sums, Gauss-Jordan against Cholesky).
    Mode n solves A^(n) Gammabar^(n) = M^(n); a relative perturbation e of
    its inputs moves A^(n) by at most kappa(Gammabar^(n)) e to first order.
    Its inputs carry the summation error of M and the Grams, at most
    eta = (Kbar + 2R) u relative with u = 2^-53 (recursive summation of Kbar
    products, R-term Hadamard and solve), plus the error of every factor
    updated before it, which enters M once and the Grams twice:
    e_n = kappa_n (eta + 3 sum_{m<n} e_m).  The sweep is held to
    max(1e-10, 3 max_n e_n); the kappa_n are those of the oracle's sweep."""
    u_ = 2.0 ** -53
    F = [A.copy() for A in O.unpack(np.array(u, dtype=np.float64), X.dims, R)]
    errs = []
    for n in range(len(F)):
        Gb = O.gamma_bar(F, n)
        kappa = np.linalg.cond(Gb)
        Kbar = int(np.prod([d for m, d in enumerate(X.dims) if m != n]))
        eta = (Kbar + 2 * R) * u_
        errs.append(kappa * (eta + 3.0 * sum(errs)))
        F[n] = O.als_mode_solve(X.mttkrp(F, n), Gb)
    return max(TOL, 3.0 * max(errs))


@pytest.mark.parametrize("shape,R,dtype", ALS_SHAPES)
@pytest.mark.parametrize("normalize", [False, True])
def test_als_sweep_parity(cp, ctx, shape, R, dtype, normalize):
    rng = synth.rng_for(11)
    T = rng.standard_normal(shape).astype(dtype)
    u = synth.initial_guess(rng, shape, R)
    X = O.DenseTensor(T)
    try:
        ref = O.als_sweep(X, u, R)
    except O.NotSPD:
        pytest.skip("Gammabar singular for this shape")
    if normalize:
        ref, _, _ = O.normalize(ref, shape, R)
    t = cp.cp_tensor_dense(ctx, dev(T))
    ud = dev(u)
    cp.cp_als_sweep(ctx, t, R, ud, normalize)
    cp.cp_ctx_sync(ctx)
    tol = als_sweep_tolerance(X, u, R)
    err = rel(ud.cpu().numpy(), ref)
    print("ALS sweep", shape, R, "error", err, "tolerance", tol)
    assert err <= tol


def test_als_sweep_parity_well_conditioned(cp, ctx):
    prob, u = synth.workload_dense_small()
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u)
    cp.cp_als_sweep(ctx, t, 3, ud, True)
    cp.cp_ctx_sync(ctx)
    ref, _, _ = O.normalize(O.als_sweep(O.DenseTensor(prob.T), u, 3), prob.dims, 3)
    assert rel(ud.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("shape,R", [((20, 20, 20), 3), ((5, 7, 4, 3), 9), ((30, 2), 1), ((6, 6, 6), 40)])
def test_normalize_parity(cp, ctx, shape, R):
    rng = np.random.default_rng(5)
    u = synth.initial_guess(rng, shape, R) * rng.uniform(0.2, 5.0)
    g = rng.standard_normal(u.size)
    uo, go, lo = O.normalize(u, shape, R, g)
    ud, gd = dev(u), dev(g)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    cp.cp_normalize(ctx, shape, R, ud, gd, lam)
    cp.cp_ctx_sync(ctx)
    assert rel(ud.cpu().numpy(), uo) <= TOL
    assert rel(gd.cpu().numpy(), go) <= TOL
    assert rel(lam.cpu().numpy(), lo) <= TOL


def test_normalize_zero_column(cp, ctx):
    shape, R = (4, 5, 3), 3
    u = synth.initial_guess(np.random.default_rng(6), shape, R)
    F = O.unpack(u, shape, R)
    F[1][:, 0] = 0.0
    u = O.pack(F)
    uo, _, lo = O.normalize(u, shape, R)
    ud = dev(u)
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    cp.cp_normalize(ctx, shape, R, ud, None, lam)
    cp.cp_ctx_sync(ctx)
    assert np.array_equal(lam.cpu().numpy() == 0, lo == 0)
    assert rel(ud.cpu().numpy(), uo) <= TOL


@pytest.mark.parametrize("m,P", [(1, 1), (1, 100), (5, 1000), (20, 12345), (64, 777)])
def test_ngmres_step_parity(cp, ctx, m, P):
    rng = np.random.default_rng(m * 1000 + P)
    U, G = rng.standard_normal((m, P)), rng.standard_normal((m, P))
    ub, gb = rng.standard_normal(P), rng.standard_normal(P)
    if P < m:
        pytest.skip("P < m makes P^T P singular")
    uo, ao = O.ngmres_step(U, G, ub, gb, 1e-12)
    uh = torch.empty(P, dtype=torch.float64, device="cuda")
    al = torch.empty(m, dtype=torch.float64, device="cuda")
    cp.ngmres_step(ctx, dev(U), dev(G), dev(ub), dev(gb), 1e-12, uh, al)
    cp.cp_ctx_sync(ctx)
    assert rel(al.cpu().numpy(), ao) <= 1e-9
    assert rel(uh.cpu().numpy(), uo) <= TOL


def test_ngmres_step_zero_residual_differences(cp, ctx):
    P, m = 50, 3
    rng = np.random.default_rng(3)
    gb = rng.standard_normal(P)
    G = np.tile(gb, (m, 1))
    U = rng.standard_normal((m, P))
    ub = rng.standard_normal(P)
    uh = torch.empty(P, dtype=torch.float64, device="cuda")
    al = torch.empty(m, dtype=torch.float64, device="cuda")
    cp.ngmres_step(ctx, dev(U), dev(G), dev(ub), dev(gb), 1e-12, uh, al)
    cp.cp_ctx_sync(ctx)
    assert np.all(al.cpu().numpy() == 0) and np.array_equal(uh.cpu().numpy(), ub)


@pytest.mark.parametrize("direction", ["steepest", "als"])
def test_linesearch_parity(cp, ctx, direction):
    prob, u0 = synth.workload_dense_small()
    R = 3
    X = O.DenseTensor(prob.T)
    x0, _, _ = O.normalize(u0, prob.dims, R)
    f0, g0 = O.fg(X, x0, R)
    if direction == "steepest":
        d = -g0 * 1e-3
    else:
        d = O.als_sweep(X, x0, R) - x0
        if g0 @ d >= 0:
            d = -g0 * 1e-3

    def phi(beta):
        x = x0 + beta * d
        fx, gx = O.fg(X, x, R)
        return fx, float(gx @ d), (x, gx)

    b, fo, _, extra, nfo, info_o = O.more_thuente(phi, f0, float(g0 @ d))
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    x = torch.empty(x0.size, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    f, stp, nfev, info = cp.linesearch(ctx, t, R, dev(x0), f0, dev(g0), dev(d), x, g)
    assert (nfev, info) == (nfo, info_o)
    assert abs(stp - b) <= TOL * abs(b)
    assert abs(f - fo) <= TOL * abs(fo)
    assert rel(x.cpu().numpy(), extra[0]) <= TOL
    assert rel(g.cpu().numpy(), extra[1]) <= TOL


def solve_line_searches(X, u0, R):
    """(ubar, d, f(ubar), g(ubar)) of every line search of the oracle's
    solve of the 20x20x20 workload (Algorithm 1, Step III)."""
    found = []
    real = O.more_thuente

    def capture(phi, f0, g0, opts=O.LSOpts()):
        cells = dict(zip(phi.__code__.co_freevars, (c.cell_contents for c in phi.__closure__)))
        found.append((cells["ubar"], cells["d"]))
        return real(phi, f0, g0, opts)
    O.more_thuente = capture
    try:
        O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7))
    finally:
        O.more_thuente = real
    return [(ub, d, *O.fg(X, ub, R)) for ub, d in found]


def mt_events(phi, f0, g0, opts):
    """Run the oracle's search and name what chose each trial after the
    first: 'sel' (the trial selection's step), 'bisect' (midpoint of a
    bracket that shrank too slowly) or 'fallback' (the best point, when no
    further progress is possible); also return info."""
    real, pending, events = O.mt_trial, {}, []

    def spy(lo, hi, t, brackt, stmin, stmax):
        pending["sel"] = real(lo, hi, t, brackt, stmin, stmax)
        return pending["sel"]

    def rec(a):
        if "sel" in pending:
            lo, hi, nxt, _ = pending.pop("sel")
            if a == min(max(nxt, opts.stpmin), opts.stpmax):
                events.append("sel")
            elif a == lo[0]:
                events.append("fallback")
            elif a == lo[0] + 0.5 * (hi[0] - lo[0]):
                events.append("bisect")
        return phi(a)
    O.mt_trial = spy
    try:
        out = O.more_thuente(rec, f0, g0, opts)
    finally:
        O.mt_trial = real
    return out, events


# (line search of the solve, options, what must happen): options under which
# the workload's own line searches take each driver rule and each exit code
LS_CASES = [
    (11, dict(gtol=1e-6, stp0=9.827, stpmax=12.653), "bisect"),
    (10, dict(ftol=0.1, stp0=43.869, stpmax=15.443), "bisect"),
    (11, dict(ftol=0.3, gtol=0.9, xtol=1e-6, stp0=0.423, stpmin=0.1, stpmax=0.3), "bisect"),
    (1, dict(xtol=0.8), "fallback"),
    (1, dict(xtol=0.8), "info2"),
    (0, dict(maxfev=2, gtol=1e-6), "info3"),
    (0, dict(stpmin=1e3, stp0=1e3), "info4"),
    (0, dict(stpmax=0.05), "info5"),
    (2, dict(ftol=0.45, gtol=1e-8, xtol=1e-10, stp0=0.1962), "info6"),
    (10, dict(ftol=0.45, gtol=1e-8, xtol=1e-6, stp0=0.5303, stpmax=10.0), "info6"),
]


@pytest.mark.parametrize("k,opt,what", LS_CASES, ids=[f"{c[2]}-ls{c[0]}" for c in LS_CASES])
def test_linesearch_parity_every_driver_rule(cp, ctx, k, opt, what):
    """The GPU search (on the line polynomial of phi) against the oracle's
    search (f and g at every trial) on the solve's own search lines, with
    options that make each More-Thuente driver rule and exit code happen:
    identical nfev and info, stp, f, x and g within 1e-10."""
    prob, u0 = synth.workload_dense_small()
    R = 3
    X = O.DenseTensor(prob.T)
    ub, d, fb, gb = solve_line_searches(X, u0, R)[k]
    ls = O.LSOpts(**opt)

    def phi(beta):
        x = ub + beta * d
        fx, gx = O.fg(X, x, R)
        return fx, float(gx @ d), (x, gx)

    (b, fo, _, extra, nfo, info_o), events = mt_events(phi, fb, float(gb @ d), ls)
    assert (what in events) if what in ("bisect", "fallback") else info_o == int(what[4:]), (events, info_o)
    co = cp.cp_ls_opts()
    for name in ("ftol", "gtol", "xtol", "stpmin", "stpmax", "stp0", "maxfev"):
        setattr(co, name, getattr(ls, name))
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    x = torch.empty(ub.size, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    f, stp, nfev, info = cp.linesearch(ctx, t, R, dev(ub), fb, dev(gb), dev(d), x, g, co)
    assert (nfev, info) == (nfo, info_o)
    assert abs(stp - b) <= TOL * abs(b)
    assert abs(f - fo) <= TOL * abs(fo)
    assert rel(x.cpu().numpy(), extra[0]) <= TOL
    assert rel(g.cpu().numpy(), extra[1]) <= TOL


def test_linesearch_rejects_ascent(cp, ctx):
    prob, u0 = synth.workload_dense_small()
    X = O.DenseTensor(prob.T)
    f0, g0 = O.fg(X, u0, 3)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    x = torch.empty(u0.size, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    with pytest.raises(cp.CpError) as ei:
        cp.linesearch(ctx, t, 3, dev(u0), f0, dev(g0), dev(g0), x, g)
    assert ei.value.status == 7


def test_solve_parity_dense_small(cp, ctx):
    """The 20x20x20, R=3, c=0.5, 10 % noise workload: GPU solve vs oracle solve."""
    prob, u0 = synth.workload_dense_small()
    R = 3
    X = O.DenseTensor(prob.T)
    uo, go, rep_o = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7))
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    opts = cp.cp_solve_opts_default(R)
    rep = cp.cp_solve(ctx, t, opts, ud)
    assert rep["converged"] and rep_o.converged
    u = ud.cpu().numpy()
    f, g = O.fg(X, u, R)
    assert np.linalg.norm(g) / O.n_params(prob.dims, R) < 1e-7
    assert abs(rep["f"] - rep_o.f) <= 1e-10 * rep_o.f + 1e-14 * X.norm2
    assert rel(u, uo) <= 1e-6
    print("iterations gpu/oracle:", rep["iters"], rep_o.iters, "restarts", rep["restarts"], rep_o.restarts)


def test_solve_recovers_noise_free_planted(cp, ctx):
    rng = synth.rng_for(0, 3)
    prob = synth.dense_problem(rng, (12, 10, 14), 4, 0.5)
    u0 = synth.initial_guess(rng, prob.dims, 4)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    opts = cp.cp_solve_opts_default(4)
    opts.tol = 1e-12
    rep = cp.cp_solve(ctx, t, opts, ud)
    assert rep["converged"]
    f = O.f_bruteforce(prob.T, O.unpack(ud.cpu().numpy(), prob.dims, 4))
    assert f <= 1e-12 * float(np.sum(prob.T ** 2))


def test_results_are_deterministic(cp, ctx):
    T, u = make((33, 20, 17), 8, np.float32, seed=9)
    t = cp.cp_tensor_dense(ctx, dev(T))
    ud = dev(u)
    outs = []
    for _ in range(2):
        out = torch.empty(33 * 8, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, 8, ud, 0, out)
        f = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.empty_like(ud)
        cp.cp_fg(ctx, t, 8, ud, f, g)
        cp.cp_ctx_sync(ctx)
        outs.append((out.cpu().numpy(), f.item(), g.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][2], outs[1][2])


def test_argument_errors(cp, ctx):
    T, u = make((4, 5, 6), 2, np.float64)
    t = cp.cp_tensor_dense(ctx, dev(T))
    out = torch.empty(100, dtype=torch.float64, device="cuda")
    for bad in [dict(R=0, mode=0), dict(R=65, mode=0), dict(R=2, mode=3), dict(R=2, mode=-1)]:
        with pytest.raises(cp.CpError) as ei:
            cp.cp_mttkrp(ctx, t, bad["R"], dev(u), bad["mode"], out)
        assert ei.value.status == 1
    with pytest.raises(cp.CpError):
        cp.cp_tensor_dense(ctx, dev(np.zeros((3,))))      # order 1
    with pytest.raises(cp.CpError):
        cp.cp_tensor_dense(ctx, dev(np.zeros((3, 0, 2))))  # empty mode


def test_full_size_dense_256_fp64_mttkrp_parity(cp, ctx):
    """The 256^3, R=16 workload at full size (FP64 path) against the oracle."""
    prob, u0 = synth.workload_dense_256()
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    F = O.unpack(u0, prob.dims, 16)
    for n in range(3):
        out = torch.empty(256 * 16, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, 16, ud, n, out)
        cp.cp_ctx_sync(ctx)
        ref = O.mttkrp_dense(prob.T, F, n)
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL
