"""GPU checks of batched and served solves: every request's result is the
same (bit for bit) alone and in a mix, admission respects the HBM budget,
waiting requests can be cancelled."""
import numpy as np
import pytest
import torch

import synth
from oracle import cp_oracle as O

pytestmark = pytest.mark.gpu


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


def small_requests(n, seed=0):
    """Requests shaped like the serving stream, with sides and ranks scaled
    down so the test runs in seconds."""
    reqs = synth.request_stream(n, rate_per_s=200.0, config=50 + seed, side_range=(8, 40), rank_range=(2, 6))
    out = []
    for r in reqs:
        prob, u0 = synth.request_problem(r, config=50 + seed)
        out.append((r, prob, u0))
    return out


def opts_for(cp, r, prec):
    o = cp.cp_solve_opts_default(r.R)
    o.tol = max(r.tol, 1e-6)
    o.prec = prec
    o.maxit = 3000
    return o


def solo(cp, ctx, prob, u0, o):
    t = cp.cp_tensor_dense(ctx, prob.T)
    u = np.array(u0, copy=True)
    rep = cp.cp_solve(ctx, t, o, u)
    t.close()
    return u, rep


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_batch_equals_solo(cp, ctx, prec_name):
    prec = cp.CP_FP64 if prec_name == "fp64" else cp.CP_MIXED_BF16X3
    items = small_requests(6, seed=1)
    tensors, opts, us = [], [], []
    for r, prob, u0 in items:
        tensors.append(cp.cp_tensor_dense(ctx, prob.T))
        opts.append(opts_for(cp, r, prec))
        us.append(np.array(u0, copy=True))
    reps = cp.cp_solve_batch(ctx, tensors, opts, us)
    for (r, prob, u0), u, rep, o in zip(items, us, reps, opts):
        u_solo, rep_solo = solo(cp, ctx, prob, u0, o)
        assert np.array_equal(u, u_solo)
        assert rep["iters"] == rep_solo["iters"] and rep["f"] == rep_solo["f"]
        if rep["converged"]:
            _, g = O.fg(O.DenseTensor(prob.T), u, r.R)
            assert np.linalg.norm(g) / O.n_params(prob.dims, r.R) < o.tol * 1.0001
    for t in tensors:
        t.close()


def many_solo(cp, ctx, prob, u0, o):
    t = cp.cp_tensor_dense(ctx, prob.T)
    u = np.array(u0, copy=True)
    (rep,) = cp.cp_solve_many(ctx, [t], [o], [u], cluster=0)
    t.close()
    return u, rep


@pytest.mark.parametrize("engine", [False, True])
def test_server_results_equal_solo_and_stats(cp, ctx, engine):
    """Engine off: every request runs on a graph slot and must equal cp_solve;
    engine on (the default): the requests share the cluster engine's rounds
    and must equal cp_solve_many of the request alone (the same tuned
    cluster size)."""
    items = small_requests(12, seed=2)
    srv = cp.cp_server_create(ctx, 8 << 30, 4)
    cp.cp_server_set_engine(srv, engine)
    outs, ids, opts = [], [], []
    for k, (r, prob, u0) in enumerate(items):
        o = opts_for(cp, r, cp.CP_MIXED_BF16X3 if k % 2 else cp.CP_FP64)
        out = np.zeros_like(u0)
        ids.append(cp.cp_server_submit(srv, prob.T, o, u0, out))
        outs.append(out)
        opts.append(o)
    cp.cp_server_drain(srv, 600.0)
    for (r, prob, u0), rid, out, o in zip(items, ids, outs, opts):
        status, rep, lat = cp.cp_server_poll(srv, rid)
        assert status in (0, 8)
        assert lat > 0
        u_solo, rep_solo = (many_solo if engine else solo)(cp, ctx, prob, u0, o)
        assert np.array_equal(out, u_solo)
        assert rep["iters"] == rep_solo["iters"]
        if rep["converged"]:
            _, g = O.fg(O.DenseTensor(prob.T.astype(np.float64)), out, r.R)
            assert np.linalg.norm(g) / O.n_params(prob.dims, r.R) < o.tol
    st = cp.cp_server_stats(srv)
    assert st["completed"] == 12 and 0 < st["p50_s"] <= st["p99_s"] and st["solves_per_s"] > 0
    srv.close()


def test_server_mixes_engine_and_graph_requests(cp, ctx):
    """A 4-way request (outside the engine) and 3-way requests in one
    server: each equals its own path's solo result."""
    items = small_requests(4, seed=6)
    rng = synth.rng_for(0, 21)
    p4 = synth.dense_problem(rng, (9, 8, 7, 6), 3, 0.5, eta=0.05, dtype=np.float32)
    u4 = synth.initial_guess(rng, p4.dims, 3)
    srv = cp.cp_server_create(ctx, 8 << 30, 3)
    o4 = cp.cp_solve_opts_default(3)
    o4.maxit = 3000
    out4 = np.zeros_like(u4)
    id4 = cp.cp_server_submit(srv, p4.T, o4, u4, out4)
    outs, ids, opts = [], [], []
    for r, prob, u0 in items:
        o = opts_for(cp, r, cp.CP_FP64)
        out = np.zeros_like(u0)
        ids.append(cp.cp_server_submit(srv, prob.T, o, u0, out))
        outs.append(out)
        opts.append(o)
    cp.cp_server_drain(srv, 600.0)
    assert cp.cp_server_poll(srv, id4)[0] in (0, 8)
    u_solo, _ = solo(cp, ctx, p4, u4, o4)
    assert np.array_equal(out4, u_solo)
    for (r, prob, u0), rid, out, o in zip(items, ids, outs, opts):
        assert cp.cp_server_poll(srv, rid)[0] in (0, 8)
        u_solo, _ = many_solo(cp, ctx, prob, u0, o)
        assert np.array_equal(out, u_solo)
    srv.close()


def test_server_admission_budget(cp, ctx):
    items = small_requests(5, seed=3)
    # a budget far below the default: requests queue for memory, never exceed it
    biggest = max(prob.T.nbytes for _, prob, _ in items)
    budget = 64 << 20
    srv = cp.cp_server_create(ctx, budget, 4)
    outs = []
    for r, prob, u0 in items:
        out = np.zeros_like(u0)
        cp.cp_server_submit(srv, prob.T, opts_for(cp, r, cp.CP_FP64), u0, out)
        outs.append(out)
    cp.cp_server_drain(srv, 600.0)
    st = cp.cp_server_stats(srv)
    assert st["completed"] == 5 and st["peak_bytes"] <= budget
    assert biggest < budget
    srv.close()


def test_server_rejects_request_above_budget(cp, ctx):
    r, prob, u0 = small_requests(1, seed=4)[0]
    # a budget below the tensor alone (the output buffer stays referenced: an
    # admitted request would write to it)
    srv = cp.cp_server_create(ctx, prob.T.nbytes // 2, 2)
    out = np.zeros_like(u0)
    with pytest.raises(cp.CpError) as ei:
        cp.cp_server_submit(srv, prob.T, opts_for(cp, r, cp.CP_FP64), u0, out)
    assert ei.value.status == 10
    srv.close()


def test_server_cancel_waiting_request(cp, ctx):
    items = small_requests(4, seed=5)
    srv = cp.cp_server_create(ctx, 8 << 30, 1)
    ids, outs = [], []
    for r, prob, u0 in items:
        out = np.zeros_like(u0)
        ids.append(cp.cp_server_submit(srv, prob.T, opts_for(cp, r, cp.CP_FP64), u0, out))
        outs.append(out)
    try:
        cp.cp_server_cancel(srv, ids[-1])
        cancelled = True
    except cp.CpError:
        cancelled = False   # already admitted: nothing to cancel
    cp.cp_server_drain(srv, 600.0)
    status, _, _ = cp.cp_server_poll(srv, ids[-1])
    if cancelled:
        assert status == 1 and np.all(outs[-1] == 0)
    assert cp.cp_server_poll(srv, ids[0])[0] in (0, 8)
    srv.close()


def test_mixed_solve_polish_certifies_fp64_gradient(cp, ctx):
    rng = synth.rng_for(0, 11)
    prob = synth.dense_problem(rng, (40, 36, 30), 5, 0.9, eta=0.1, hetero=0.1, dtype=np.float32)
    u0 = synth.initial_guess(rng, prob.dims, 5)
    o = cp.cp_solve_opts_default(5)
    o.prec = cp.CP_MIXED_BF16X3
    u = np.array(u0, copy=True)
    t = cp.cp_tensor_dense(ctx, prob.T)
    rep = cp.cp_solve(ctx, t, o, u)
    assert rep["converged"]
    _, g = O.fg(O.DenseTensor(prob.T), u, 5)
    assert np.linalg.norm(g) / O.n_params(prob.dims, 5) < 1e-7
    t.close()


def test_server_reports_a_failing_engine_request_beside_good_ones(cp, ctx):
    """A zero tensor (CP_ERR_NOT_SPD after the first sweep) among ordinary
    requests on the cluster engine: its status is reported, the others
    converge to their solo results."""
    items = small_requests(3, seed=8)
    srv = cp.cp_server_create(ctx, 8 << 30, 4)
    T0 = np.zeros((10, 9, 8), dtype=np.float32)
    u00 = synth.initial_guess(np.random.default_rng(3), T0.shape, 2)
    o0 = cp.cp_solve_opts_default(2)
    out0 = np.zeros_like(u00)
    id0 = cp.cp_server_submit(srv, T0, o0, u00, out0)
    outs, ids, opts = [], [], []
    for r, prob, u0 in items:
        o = opts_for(cp, r, cp.CP_FP64)
        out = np.zeros_like(u0)
        ids.append(cp.cp_server_submit(srv, prob.T, o, u0, out))
        outs.append(out)
        opts.append(o)
    cp.cp_server_drain(srv, 600.0)
    assert cp.cp_server_poll(srv, id0)[0] == 5
    for (r, prob, u0), rid, out, o in zip(items, ids, outs, opts):
        assert cp.cp_server_poll(srv, rid)[0] in (0, 8)
        u_solo, _ = many_solo(cp, ctx, prob, u0, o)
        assert np.array_equal(out, u_solo)
    srv.close()
