"""GPU parity of the sparse (COO) path against the oracle, through the C ABI.

Sort and segmentation: bit-exact.  FP64 MTTKRP / f / g: 1e-10 relative.
FP32 products (the mixed setting on COO tensors): 5e-5 relative to FP64."""
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
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


CASES = [
    ((5, 4, 6), 40),
    ((7, 1, 9), 30),
    ((300, 200, 100), 5000),
    ((3, 4, 5, 6), 200),
    ((20000, 20000, 20000), 20000),
    ((2, 3), 6),
    ((1000, 17, 33, 2, 5), 3000),
]


@pytest.mark.parametrize("dims,nnz", CASES)
def test_sort_and_segments_bit_exact(cp, ctx, dims, nnz):
    rng = np.random.default_rng(nnz)
    coords = synth.distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    t = cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    for n in range(len(dims)):
        perm, seg_ptr, seg_row = cp.cp_tensor_sorted_mode(ctx, t, n)
        p_o, s_o, r_o = O.coo_sort_mode(coords, n)
        assert np.array_equal(perm, p_o)
        assert np.array_equal(seg_ptr, s_o)
        assert np.array_equal(seg_row, r_o)


def test_host_buffers_and_norm(cp, ctx):
    dims, nnz = (50, 60, 70), 1000
    rng = np.random.default_rng(1)
    coords = synth.distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    t = cp.cp_tensor_coo(ctx, dims, coords, vals)      # host arrays
    assert cp.cp_tensor_info(t)[2] == pytest.approx(float(np.sum(vals.astype(np.float64) ** 2)), rel=1e-13)
    perm, _, _ = cp.cp_tensor_sorted_mode(ctx, t, 2)
    assert np.array_equal(perm, O.coo_sort_mode(coords, 2)[0])


def test_empty_tensor(cp, ctx):
    dims = (4, 5, 6)
    t = cp.cp_tensor_coo(ctx, dims, np.zeros((0, 3), dtype=np.int64), np.zeros(0, dtype=np.float32))
    perm, seg_ptr, seg_row = cp.cp_tensor_sorted_mode(ctx, t, 1)
    assert perm.size == 0 and list(seg_ptr) == [0] and seg_row.size == 0
    u = dev(synth.initial_guess(np.random.default_rng(2), dims, 3))
    out = torch.full((5 * 3,), 7.0, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp(ctx, t, 3, u, 1, out)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(u)
    cp.cp_fg(ctx, t, 3, u, f, g)
    cp.cp_ctx_sync(ctx)
    assert torch.all(out == 0)
    fo, go = O.fg(O.SparseTensor(np.zeros((0, 3), dtype=np.int64), np.zeros(0), dims), u.cpu().numpy(), 3)
    assert abs(f.item() - fo) <= TOL * abs(fo) and rel(g.cpu().numpy(), go) <= TOL


def test_rejects_duplicates_and_out_of_range(cp, ctx):
    dims = (4, 5, 6)
    coords = np.array([[0, 1, 2], [3, 4, 5], [0, 1, 2]], dtype=np.int64)
    vals = np.ones(3, dtype=np.float32)
    with pytest.raises(cp.CpError) as ei:
        cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    assert ei.value.status == 2
    coords = np.array([[0, 1, 2], [4, 0, 0]], dtype=np.int64)
    with pytest.raises(cp.CpError) as ei:
        cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals[:2]))
    assert ei.value.status == 2
    coords = np.array([[0, -1, 2]], dtype=np.int64)
    with pytest.raises(cp.CpError):
        cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals[:1]))


@pytest.mark.parametrize("dims,nnz", CASES)
@pytest.mark.parametrize("R", [1, 10, 33])
def test_sparse_mttkrp_parity(cp, ctx, dims, nnz, R):
    rng = np.random.default_rng(nnz + R)
    coords = synth.distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    u = synth.initial_guess(rng, dims, R)
    F = O.unpack(u, dims, R)
    t = cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    ud = dev(u)
    for n in range(len(dims)):
        ref = O.mttkrp_sparse(coords, vals.astype(np.float64), dims, F, n)
        out = torch.empty(dims[n] * R, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, R, ud, n, out, cp.CP_FP64)
        out32 = torch.empty_like(out)
        cp.cp_mttkrp(ctx, t, R, ud, n, out32, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL
        assert rel(out32.cpu().numpy().reshape(ref.shape), ref) <= 5e-5


def test_skewed_segment_longer_than_a_work_unit(cp, ctx):
    dims, R = (3, 4000, 50), 6
    rng = np.random.default_rng(5)
    # row 1 of mode 0 holds 5000 nonzeros (many work units), rows 0 and 2 few
    c1 = np.stack([np.ones(5000, dtype=np.int64), rng.permutation(4000 * 50)[:5000] // 50,
                   rng.permutation(4000 * 50)[:5000] % 50], axis=1)
    coords = np.unique(np.concatenate([c1, [[0, 0, 0], [2, 5, 7]]]), axis=0)
    vals = rng.standard_normal(coords.shape[0]).astype(np.float32)
    u = synth.initial_guess(rng, dims, R)
    t = cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    out = torch.empty(3 * R, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp(ctx, t, R, dev(u), 0, out)
    cp.cp_ctx_sync(ctx)
    ref = O.mttkrp_sparse(coords, vals.astype(np.float64), dims, O.unpack(u, dims, R), 0)
    assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL


def test_sparse_fg_parity(cp, ctx):
    dims, nnz, R = (60, 50, 40), 3000, 5
    rng = np.random.default_rng(9)
    coords = synth.distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    u = synth.initial_guess(rng, dims, R)
    t = cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    ud = dev(u)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(ud)
    cp.cp_fg(ctx, t, R, ud, f, g)
    cp.cp_ctx_sync(ctx)
    fo, go = O.fg(O.SparseTensor(coords, vals, dims), u, R)
    assert abs(f.item() - fo) <= TOL * abs(fo)
    assert rel(g.cpu().numpy(), go) <= TOL


def sparse_als_tolerance(X, u, R, nnz):
    """The first-order bound of the dense ALS parity test with the nonzeros
    per row in place of Kbar: e_n = kappa(Gammabar^(n)) (eta + 3 sum_{m<n}
    e_m), eta = (nnz + 2R) 2^-53 (a row sums at most nnz products; the Grams
    sum I_m <= nnz terms), held to max(1e-10, 3 max e_n)."""
    F = [A.copy() for A in O.unpack(np.array(u, dtype=np.float64), X.dims, R)]
    errs = []
    for n in range(len(F)):
        Gb = O.gamma_bar(F, n)
        eta = (max(nnz, max(X.dims)) + 2 * R) * 2.0 ** -53
        errs.append(np.linalg.cond(Gb) * (eta + 3.0 * sum(errs)))
        F[n] = O.als_mode_solve(X.mttkrp(F, n), Gb)
    return max(TOL, 3.0 * max(errs))


def test_sparse_als_sweep_tall_factor(cp, ctx):
    """A factor taller than one Gram row chunk (9000 rows): the Grams take
    the chunked path with its fixed-order cross-block sum."""
    dims, nnz, R = (9000, 50, 40), 40000, 6
    rng = np.random.default_rng(17)
    coords = synth.distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    u = synth.initial_guess(rng, dims, R)
    X = O.SparseTensor(coords, vals, dims)
    try:
        ref = O.als_sweep(X, u, R)
    except O.NotSPD:
        pytest.skip("Gammabar singular for this draw")
    t = cp.cp_tensor_coo(ctx, dims, dev(coords), dev(vals))
    ud = dev(u)
    cp.cp_als_sweep(ctx, t, R, ud, False)
    cp.cp_ctx_sync(ctx)
    tol = sparse_als_tolerance(X, u, R, nnz)
    err = rel(ud.cpu().numpy(), ref)
    print("sparse ALS sweep error", err, "tolerance", tol)
    assert err <= tol


def test_two_way_laplacian_solve_reaches_eckart_young_optimum(cp, ctx):
    """Test Problem II with d = 1: f* = 1/2 sum of the s - R smallest squared
    eigenvalues 2 - 2 cos(k pi / (s + 1)) of the tridiagonal Laplacian."""
    s, R = 12, 3
    lap = synth.laplacian_tensor(1, s)
    t = cp.cp_tensor_coo(ctx, lap.dims, dev(lap.coords), dev(lap.vals))
    lam = np.sort(2 - 2 * np.cos(np.arange(1, s + 1) * np.pi / (s + 1)))
    fstar = 0.5 * float(np.sum(lam[: s - R] ** 2))
    ud = dev(synth.initial_guess(synth.rng_for(97), lap.dims, R))
    opts = cp.cp_solve_opts_default(R)
    opts.tol = 1e-10
    opts.maxit = 2000
    rep = cp.cp_solve(ctx, t, opts, ud)
    assert rep["converged"]
    assert abs(rep["f"] - fstar) <= 1e-8 * fstar


def test_laplacian_4way_solve_parity(cp, ctx):
    """Test Problem II, d = 2, s = 5, R = 3: GPU solve vs oracle solve."""
    lap = synth.laplacian_tensor(2, 5)
    R = 3
    u0 = synth.initial_guess(synth.rng_for(4, 1), lap.dims, R)
    X = O.SparseTensor(lap.coords, lap.vals, lap.dims)
    uo, _, rep_o = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7, maxit=3000))
    t = cp.cp_tensor_coo(ctx, lap.dims, dev(lap.coords), dev(lap.vals))
    ud = dev(u0)
    opts = cp.cp_solve_opts_default(R)
    opts.maxit = 3000
    rep = cp.cp_solve(ctx, t, opts, ud)
    assert rep["converged"] and rep_o.converged
    f, g = O.fg(X, ud.cpu().numpy(), R)
    assert np.linalg.norm(g) / O.n_params(lap.dims, R) < 1e-7
    assert abs(rep["f"] - rep_o.f) <= 1e-10 * rep_o.f + 1e-14 * X.norm2
    print("iterations gpu/oracle", rep["iters"], rep_o.iters)


# Test Problem II at the paper's shapes (Section 4, Tables 4-6): the 2d-way
# Laplacian tensor on an s^d grid, N = 2d.
TP2_SHAPES = [(2, 8, 6), (2, 16, 3), (3, 4, 2), (3, 8, 5), (4, 4, 2)]


@pytest.mark.parametrize("d,s,R", TP2_SHAPES)
def test_sparse_mttkrp_parity_test_problem_2(cp, ctx, d, s, R):
    """Every mode's sparse MTTKRP of the N = 4, 6, 8 Laplacian tensors:
    FP64 within 1e-10 of the oracle, FP32 products within 5e-5."""
    lap = synth.laplacian_tensor(d, s)
    u = synth.initial_guess(synth.rng_for(4, 100 + 10 * d + s), lap.dims, R)
    F = O.unpack(u, lap.dims, R)
    t = cp.cp_tensor_coo(ctx, lap.dims, dev(lap.coords), dev(lap.vals))
    ud = dev(u)
    for n in range(2 * d):
        ref = O.mttkrp_sparse(lap.coords, lap.vals.astype(np.float64), lap.dims, F, n)
        out = torch.empty(s * R, dtype=torch.float64, device="cuda")
        out32 = torch.empty_like(out)
        cp.cp_mttkrp(ctx, t, R, ud, n, out, cp.CP_FP64)
        cp.cp_mttkrp(ctx, t, R, ud, n, out32, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL, n
        assert rel(out32.cpu().numpy().reshape(ref.shape), ref) <= 5e-5, n


@pytest.mark.parametrize("d,s,R", TP2_SHAPES)
def test_laplacian_solve_paper_shapes(cp, ctx, d, s, R):
    """GPU solve against the oracle's solve on Test Problem II at the paper's
    shapes, from the same seeded start, to ||g||/P < 1e-7: both converge,
    f agrees within 1e-10 f + 1e-14 ||T||^2, and the oracle's gradient at the
    GPU's solution meets the tolerance."""
    lap = synth.laplacian_tensor(d, s)
    u0 = synth.initial_guess(synth.rng_for(4, 10 * d + s), lap.dims, R)
    X = O.SparseTensor(lap.coords, lap.vals, lap.dims)
    uo, _, rep_o = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-7, maxit=5000))
    t = cp.cp_tensor_coo(ctx, lap.dims, dev(lap.coords), dev(lap.vals))
    ud = dev(u0)
    opts = cp.cp_solve_opts_default(R)
    opts.maxit = 5000
    rep = cp.cp_solve(ctx, t, opts, ud)
    print("Test Problem II d=%d s=%d R=%d: iterations gpu/oracle %d/%d, f %.17g / %.17g"
          % (d, s, R, rep["iters"], rep_o.iters, rep["f"], rep_o.f))
    assert rep["converged"] and rep_o.converged
    f, g = O.fg(X, ud.cpu().numpy(), R)
    assert np.linalg.norm(g) / O.n_params(lap.dims, R) < 1e-7
    assert abs(rep["f"] - rep_o.f) <= 1e-10 * rep_o.f + 1e-14 * X.norm2


def test_full_size_sparse_sort_and_mttkrp(cp, ctx):
    """The 20000^3, 2e6-nonzero workload at full size: bit-exact sort and
    segmentation of every mode, FP64 MTTKRP parity."""
    prob, u0 = synth.workload_sparse()
    t = cp.cp_tensor_coo(ctx, prob.dims, dev(prob.coords), dev(prob.vals))
    F = O.unpack(u0, prob.dims, prob.R)
    ud = dev(u0)
    for n in range(3):
        perm, seg_ptr, seg_row = cp.cp_tensor_sorted_mode(ctx, t, n)
        p_o, s_o, r_o = O.coo_sort_mode(prob.coords, n)
        assert np.array_equal(perm, p_o) and np.array_equal(seg_ptr, s_o) and np.array_equal(seg_row, r_o)
        out = torch.empty(prob.dims[n] * prob.R, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, prob.R, ud, n, out)
        cp.cp_ctx_sync(ctx)
        ref = O.mttkrp_sparse(prob.coords, prob.vals.astype(np.float64), prob.dims, F, n)
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= TOL
