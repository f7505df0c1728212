"""GPU checks of the mixed-precision dense MTTKRP (tcgen05, bf16x3 split
products, FP32 accumulation) against the FP64 oracle, through the C ABI.

Stated bounds:
  * element by element, |M_gpu - M| <= c (|T_(n)| |Phibar|) with
    c = 3.01 2^-16 + (2N - 2) 2^-24 + (n_mma + 1) 2^-22: the split products
    drop at most 3.01 u^2 |ab| (u = 2^-8), the FP32 copies of T and of the
    factors and the FP32 Khatri-Rao products add (2N - 2) 2^-24, and every
    tensor-core MMA that adds into an FP32 accumulator is charged two FP32
    ulps (2^-22) of the CTA's share of |T_(n)| |Phibar|, n_mma of them along
    one accumulator (12 MMAs per 64-element contraction tile: four 16-deep
    steps of three split products), one more for the epilogue and the FP32
    partial;
  * relative Frobenius error of M^(n) <= 5e-5 (the split errors have random
    signs and add to ~5e-6 of ||M||);
  * f and g built from these MTTKRPs are held to the same relative bound
    against their FP64 values (g relative to ||M||, the scale at which its
    terms cancel)."""
import numpy as np
import pytest
import torch

import synth
from oracle import cp_oracle as O

pytestmark = pytest.mark.gpu

MIXED_TOL = 5e-5


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


def split_k_tiles_per_cta(I, Kbar):
    """Contraction tiles (64 elements) one CTA adds for a single-mode launch:
    the rows form ceil(I / 128) groups and the SMs are shared among them."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ktiles = -(-Kbar // 64)
    groups = -(-I // 128)
    target = max(1, sms // groups)
    return -(-ktiles // target)


def elementwise_bound(T, F, n, rows=None):
    """c (|T_(n)| |Phibar|) for the rows of mode n listed (all if None),
    |T_(n)| |Phibar| computed by the oracle's MTTKRP of |T| and |A|."""
    N = T.ndim
    Tabs = np.abs(np.asarray(T, dtype=np.float64))
    Fabs = [np.abs(A) for A in F]
    if rows is not None:
        Tabs = np.take(Tabs, rows, axis=n)
        Fabs[n] = Fabs[n][rows]
    B = O.mttkrp_dense(Tabs, Fabs, n)
    Kbar = int(np.prod([T.shape[m] for m in range(N) if m != n]))
    n_mma = 12 * split_k_tiles_per_cta(T.shape[n], Kbar)
    c = 3.01 * 2.0 ** -16 + (2 * N - 2) * 2.0 ** -24 + (n_mma + 1) * 2.0 ** -22
    return c * B


def check_elementwise(got, ref, bound, what):
    excess = np.abs(got - ref) - bound
    worst = np.unravel_index(np.argmax(excess), excess.shape)
    assert np.all(excess <= 0.0), (what, worst, got[worst], ref[worst], bound[worst])


SHAPES = [
    ((20, 20, 20), 3, np.float64),        # tiny, one k-tile group per CTA
    ((7, 5, 3), 1, np.float32),           # K-bar below one tile
    ((130, 33, 17), 16, np.float32),      # two M tiles, ragged rows and k
    ((96, 40, 30, 5), 32, np.float32),    # 4-way, R = 32
    ((300, 20, 9), 20, np.float32),       # 3 M tiles -> two row groups
    ((64, 64, 64), 48, np.float32),       # padded rank 48
    ((17, 256, 12), 64, np.float32),      # R = 64
]


@pytest.mark.parametrize("shape,R,dtype", SHAPES)
def test_mixed_mttkrp_error_bound(cp, ctx, shape, R, dtype):
    rng = np.random.default_rng(R)
    T = rng.standard_normal(shape).astype(dtype)
    u = synth.initial_guess(rng, shape, R)
    F = O.unpack(u, shape, R)
    t = cp.cp_tensor_dense(ctx, dev(T))
    ud = dev(u)
    for n in range(len(shape)):
        out = torch.empty(shape[n] * R, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, R, ud, n, out, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        ref = O.mttkrp_dense(T.astype(np.float64), F, n)
        got = out.cpu().numpy().reshape(ref.shape)
        err = rel(got, ref)
        assert err <= MIXED_TOL, (shape, R, n, err)
        check_elementwise(got, ref, elementwise_bound(T, F, n), (shape, R, n))


def test_mixed_mttkrp_deterministic(cp, ctx):
    rng = np.random.default_rng(3)
    T = rng.standard_normal((130, 70, 33)).astype(np.float32)
    u = dev(synth.initial_guess(rng, T.shape, 16))
    t = cp.cp_tensor_dense(ctx, dev(T))
    outs = []
    for _ in range(2):
        out = torch.empty(70 * 16, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, 16, u, 1, out, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_mixed_fg_error_bound(cp, ctx):
    prob, u0 = synth.workload_dense_small()
    X = O.DenseTensor(prob.T)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(ud)
    cp.cp_fg(ctx, t, 3, ud, f, g, cp.CP_MIXED_BF16X3)
    cp.cp_ctx_sync(ctx)
    fo, go = O.fg(X, u0, 3)
    F = O.unpack(u0, prob.dims, 3)
    Mscale = np.sqrt(sum(np.sum(O.mttkrp_dense(prob.T, F, n) ** 2) for n in range(3)))
    assert abs(f.item() - fo) <= MIXED_TOL * (X.norm2 + abs(fo))
    assert np.linalg.norm(g.cpu().numpy() - go) <= MIXED_TOL * Mscale


def test_full_size_dense_256_mixed_mttkrp(cp, ctx):
    """The 256^3, R=16 workload at full size in the launch configuration the
    bench times: every mode against the FP64 oracle."""
    prob, u0 = synth.workload_dense_256()
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    F = O.unpack(u0, prob.dims, 16)
    for n in range(3):
        out = torch.empty(256 * 16, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, 16, ud, n, out, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        ref = O.mttkrp_dense(prob.T, F, n)
        got = out.cpu().numpy().reshape(ref.shape)
        assert rel(got, ref) <= MIXED_TOL
        check_elementwise(got, ref, elementwise_bound(prob.T, F, n), n)


def test_full_size_dense_4way_96_mixed_mttkrp_sampled_rows(cp, ctx):
    """The 96^4, R=32 workload at full size in the bench's launch
    configuration: every mode's mixed MTTKRP on the GPU, checked on sampled
    rows (first, last and six random) that the oracle computes from the
    tensor sliced along that mode, element by element and in norm."""
    prob, u0 = synth.workload_dense_4way()
    R = prob.R
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    ud = dev(u0)
    F = O.unpack(u0, prob.dims, R)
    rng = np.random.default_rng(96)
    for n in range(4):
        out = torch.empty(prob.dims[n] * R, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp(ctx, t, R, ud, n, out, cp.CP_MIXED_BF16X3)
        cp.cp_ctx_sync(ctx)
        rows = np.unique(np.concatenate([[0, prob.dims[n] - 1], rng.integers(0, prob.dims[n], 6)]))
        Fs = list(F)
        Fs[n] = F[n][rows]
        ref = O.mttkrp_dense(np.take(prob.T, rows, axis=n), Fs, n)
        got = out.cpu().numpy().reshape(prob.dims[n], R)[rows]
        assert rel(got, ref) <= MIXED_TOL
        check_elementwise(got, ref, elementwise_bound(prob.T, F, n, rows), n)


# Khatri-Rao variant MTTKRPs (the line search's pass): shapes where every
# listed mode goes into one tensor-core launch, a 4-way tensor with 8 variants
# of rank 32 (256 columns), rank 60 (4 x 60 = 240 columns), and a 4-way rank
# too wide for one launch (8 x 40 > 256: one MTTKRP per variant), in FP64 and
# mixed precision.
VARIANT_CASES = [
    ((20, 20, 20), 3, np.float64, "fp64"),
    ((20, 20, 20), 3, np.float64, "mixed"),
    ((130, 33, 17), 16, np.float32, "mixed"),
    ((24, 12, 10, 6), 5, np.float32, "mixed"),
    ((24, 12, 10, 6), 5, np.float32, "fp64"),
    ((40, 30, 20, 9), 32, np.float32, "mixed"),
    ((9, 8, 7), 60, np.float32, "mixed"),
    ((12, 10, 8, 6), 40, np.float32, "mixed"),
    ((70, 90), 4, np.float32, "mixed"),       # 2-way: two variants, one other mode
    ((70, 90), 4, np.float64, "fp64"),
    ((33, 17, 9), 1, np.float32, "mixed"),    # rank 1
]


def variant_factors(A, D, n, v):
    """Factor m is D's when m != n and bit j of v is set, j being m's index
    among the modes other than n."""
    others = [m for m in range(len(A)) if m != n]
    return [D[m] if m != n and (v >> others.index(m)) & 1 else A[m] for m in range(len(A))]


@pytest.mark.parametrize("shape,R,dtype,prec_name", VARIANT_CASES)
def test_mttkrp_variants_parity(cp, ctx, shape, R, dtype, prec_name):
    rng = np.random.default_rng(R + len(shape))
    T = rng.standard_normal(shape).astype(dtype)
    u = synth.initial_guess(rng, shape, R)
    d = synth.initial_guess(rng, shape, R) - u
    N = len(shape)
    nvar = 2 ** (N - 1)
    modes = list(reversed(range(N)))
    out = torch.empty(sum(nvar * shape[n] * R for n in modes), dtype=torch.float64, device="cuda")
    prec = cp.CP_MIXED_BF16X3 if prec_name == "mixed" else cp.CP_FP64
    t = cp.cp_tensor_dense(ctx, dev(T))
    cp.cp_mttkrp_variants(ctx, t, R, dev(u), dev(d), modes, out, prec)
    cp.cp_ctx_sync(ctx)
    got = out.cpu().numpy()
    A, D = O.unpack(u, shape, R), O.unpack(d, shape, R)
    tol = MIXED_TOL if prec_name == "mixed" else 1e-10
    off = 0
    for n in modes:
        for v in range(nvar):
            ref = O.mttkrp_dense(T.astype(np.float64), variant_factors(A, D, n, v), n)
            assert rel(got[off:off + ref.size].reshape(ref.shape), ref) <= tol, (shape, R, n, v)
            off += ref.size


def test_mttkrp_variants_one_mode_and_argument_errors(cp, ctx):
    """One listed mode gives that mode's variants alone (the same values as
    when all modes are listed); a repeated mode, a mode out of range and an
    empty list are argument errors."""
    rng = np.random.default_rng(23)
    shape, R = (30, 20, 10), 6
    T = rng.standard_normal(shape).astype(np.float32)
    u = dev(synth.initial_guess(rng, shape, R))
    d = dev(0.5 * synth.initial_guess(rng, shape, R))
    t = cp.cp_tensor_dense(ctx, dev(T))
    one = torch.empty(4 * 20 * R, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp_variants(ctx, t, R, u, d, [1], one, cp.CP_FP64)
    full = torch.empty(4 * sum(shape) * R, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp_variants(ctx, t, R, u, d, [0, 1, 2], full, cp.CP_FP64)
    cp.cp_ctx_sync(ctx)
    off = 4 * 30 * R
    assert np.array_equal(one.cpu().numpy(), full.cpu().numpy()[off:off + 4 * 20 * R])
    for modes in ([0, 0], [3], []):
        with pytest.raises(cp.CpError):
            cp.cp_mttkrp_variants(ctx, t, R, u, d, modes, full, cp.CP_FP64)


def test_full_size_dense_256_variants_multilinear(cp, ctx):
    """The 256^3, R=16 workload, all three modes' variants in the one launch
    the solve's line search makes: sum_v beta^popcount(v) M_v^(n) equals the
    FP64 oracle's M^(n)(u + beta d) within the mixed bound."""
    prob, u0 = synth.workload_dense_256()
    rng = np.random.default_rng(11)
    d = 0.1 * rng.standard_normal(u0.size)
    beta = 0.7
    R, N = 16, 3
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    out = torch.empty(3 * 4 * 256 * R, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp_variants(ctx, t, R, dev(u0), dev(d), [2, 0, 1], out, cp.CP_MIXED_BF16X3)
    cp.cp_ctx_sync(ctx)
    got = out.cpu().numpy().reshape(3, 4, 256, R)
    X = O.unpack(u0 + beta * d, prob.dims, R)
    for k, n in enumerate([2, 0, 1]):
        if n == 1:
            continue
        line = sum(beta ** bin(v).count("1") * got[k, v] for v in range(4))
        ref = O.mttkrp_dense(prob.T, X, n)
        assert rel(line, ref) <= MIXED_TOL, n


def test_mixed_solve_4way_against_oracle(cp, ctx):
    """A 4-way dense problem (planted R = 8, collinearity 0.5, 5 % noise, FP32
    data) solved with the mixed-precision MTTKRP (every mode's line-search
    variants in one launch: 8 x 8 columns) and the FP64 polish.  By the FP64
    oracle's own evaluation at the result, the gradient meets the tolerance
    and f is the one reported; f equals the FP64 solve's, and the rank-one
    terms match the FP64 solve's up to order and sign (greedy matching by
    congruence, the product over modes of the column cosines)."""
    rng = synth.rng_for(60)
    dims, R = (24, 20, 16, 12), 8
    prob = synth.dense_problem(rng, dims, R, 0.5, eta=0.05, dtype=np.float32)
    u0 = synth.initial_guess(rng, dims, R)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    sols = {}
    for name, prec in (("mixed", cp.CP_MIXED_BF16X3), ("fp64", cp.CP_FP64)):
        opts = cp.cp_solve_opts_default(R)
        opts.prec = prec
        ud = dev(u0)
        rep = cp.cp_solve(ctx, t, opts, ud)
        assert rep["converged"], (name, rep)
        sols[name] = (ud.cpu().numpy(), rep)
    u, rep = sols["mixed"]
    X = O.DenseTensor(prob.T)
    f, g = O.fg(X, u, R)
    P = O.n_params(dims, R)
    assert np.linalg.norm(g) / P < 1.0001e-7
    assert abs(rep["f"] - f) <= 1e-10 * abs(f) + 1e-14 * X.norm2
    assert abs(rep["f"] - sols["fp64"][1]["f"]) <= 1e-6 * abs(f)
    A, B = O.unpack(u, dims, R), O.unpack(sols["fp64"][0], dims, R)
    perm = match_terms(A, B)
    for a, b in zip(A, B):
        bp = b[:, perm]
        s = np.sign(np.sum(a * bp, axis=0))
        s[s == 0] = 1.0
        assert np.linalg.norm(a - bp * s) / np.linalg.norm(b) <= 1e-3
    print("iterations mixed/fp64:", rep["iters"], sols["fp64"][1]["iters"], "fp64 polish", rep["fp64_iters"],
          "order", perm)


def match_terms(A, B):
    """perm[r] = the term of B matched to term r of A, greedily by the largest
    congruence prod_n |cos(a_r^(n), b_s^(n))|."""
    R = A[0].shape[1]
    C = np.ones((R, R))
    for a, b in zip(A, B):
        an = a / np.linalg.norm(a, axis=0)
        bn = b / np.linalg.norm(b, axis=0)
        C *= np.abs(an.T @ bn)
    perm = [-1] * R
    used = set()
    for idx in np.argsort(-C, axis=None):
        r, s = divmod(int(idx), R)
        if perm[r] < 0 and s not in used:
            perm[r] = s
            used.add(s)
    return perm


# Dimension tree (3-way): W = T x_c A^(c) in one tensor-core pass, then the
# MTTKRPs of the two other modes from W.  W's split products involve T and one
# FP32 factor; its tensor-core accumulation runs over the I_c / 64
# contraction tiles of a 128-row tile (n_mma = 12 I_c / 64, the kernel keeps
# each tile's whole contraction in one accumulator); the contraction of W
# with the other factor's FP32 copy sums I_m products in FP32 (m the mode
# summed out).  So c = 3.01 2^-16 + 3 2^-24 + (n_mma + 1) 2^-22 + I_m 2^-24,
# applied to |T_(n)| |Phibar| as for the MTTKRP.
DIMTREE_CASES = [((20, 20, 20), 3), ((130, 33, 17), 16), ((96, 80, 70), 16), ((17, 65, 200), 5),
                 ((40, 30, 20), 64)]


def dimtree_bound(T, F, n, contracted):
    Tabs = np.abs(np.asarray(T, dtype=np.float64))
    B = O.mttkrp_dense(Tabs, [np.abs(A) for A in F], n)
    n_mma = 12 * -(-T.shape[contracted] // 64)
    summed = [m for m in range(3) if m not in (n, contracted)][0]
    c = 3.01 * 2.0 ** -16 + 3 * 2.0 ** -24 + (n_mma + 1) * 2.0 ** -22 + T.shape[summed] * 2.0 ** -24
    return c * B


@pytest.mark.parametrize("shape,R", DIMTREE_CASES)
@pytest.mark.parametrize("contracted", [0, 2])
def test_dimtree_mttkrps_error_bound(cp, ctx, shape, R, contracted):
    rng = np.random.default_rng(R + contracted)
    T = rng.standard_normal(shape).astype(np.float32)
    u = synth.initial_guess(rng, shape, R)
    F = O.unpack(u, shape, R)
    t = cp.cp_tensor_dense(ctx, dev(T))
    others = [m for m in range(3) if m != contracted]
    out = torch.empty(sum(shape[m] for m in others) * R, dtype=torch.float64, device="cuda")
    cp.cp_mttkrp_dimtree(ctx, t, R, dev(u), contracted, out)
    cp.cp_ctx_sync(ctx)
    got_all = out.cpu().numpy()
    off = 0
    for n in others:
        ref = O.mttkrp_dense(T.astype(np.float64), F, n)
        got = got_all[off:off + shape[n] * R].reshape(ref.shape)
        off += shape[n] * R
        assert rel(got, ref) <= MIXED_TOL, (shape, R, contracted, n)
        check_elementwise(got, ref, dimtree_bound(T, F, n, contracted), (shape, R, contracted, n))


def test_dimtree_full_size_dense_256(cp, ctx):
    """Both dimension-tree pairs of the 256^3 R=16 workload against the
    oracle's MTTKRPs, element by element."""
    prob, u0 = synth.workload_dense_256()
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    F = O.unpack(u0, prob.dims, 16)
    for contracted in (0, 2):
        out = torch.empty(2 * 256 * 16, dtype=torch.float64, device="cuda")
        cp.cp_mttkrp_dimtree(ctx, t, 16, dev(u0), contracted, out)
        cp.cp_ctx_sync(ctx)
        got_all = out.cpu().numpy()
        for k, n in enumerate(m for m in range(3) if m != contracted):
            ref = O.mttkrp_dense(prob.T, F, n)
            got = got_all[k * 4096:(k + 1) * 4096].reshape(ref.shape)
            assert rel(got, ref) <= MIXED_TOL
            check_elementwise(got, ref, dimtree_bound(prob.T, F, n, contracted), (contracted, n))


def test_dimtree_rejects_other_cases(cp, ctx):
    rng = np.random.default_rng(4)
    T4 = rng.standard_normal((5, 4, 3, 2)).astype(np.float32)
    t4 = cp.cp_tensor_dense(ctx, dev(T4))
    out = torch.empty(1000, dtype=torch.float64, device="cuda")
    u = dev(synth.initial_guess(rng, T4.shape, 2))
    with pytest.raises(cp.CpError) as ei:
        cp.cp_mttkrp_dimtree(ctx, t4, 2, u, 0, out)
    assert ei.value.status == 11
    T3 = rng.standard_normal((5, 4, 3)).astype(np.float32)
    t3 = cp.cp_tensor_dense(ctx, dev(T3))
    u3 = dev(synth.initial_guess(rng, T3.shape, 2))
    with pytest.raises(cp.CpError) as ei:
        cp.cp_mttkrp_dimtree(ctx, t3, 2, u3, 1, out)
    assert ei.value.status == 1
    with pytest.raises(cp.CpError) as ei:
        cp.cp_mttkrp_dimtree(ctx, t3, 2, u3, 0, out, cp.CP_FP64)
    assert ei.value.status == 11


@pytest.mark.parametrize("dimtree", [0, 1])
def test_mixed_solve_with_and_without_dimension_tree(cp, ctx, dimtree):
    """The mixed-precision solve of a 3-way problem with the sweep's and
    ubar's MTTKRP pairs from the dimension tree (1) and from plain passes
    (0): both meet ||g||/P < 1e-7 by the oracle's own FP64 gradient at the
    returned point."""
    rng = synth.rng_for(0, 51)
    prob = synth.dense_problem(rng, (60, 50, 40), 6, 0.5, eta=0.05, dtype=np.float32)
    u0 = synth.initial_guess(rng, prob.dims, 6)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    u = dev(u0)
    o = cp.cp_solve_opts_default(6)
    o.prec = cp.CP_MIXED_BF16X3
    o.dimtree = dimtree
    rep = cp.cp_solve(ctx, t, o, u)
    print("dimtree", dimtree, rep)
    assert rep["converged"]
    f, g = O.fg(O.DenseTensor(prob.T), u.cpu().numpy(), 6)
    assert np.linalg.norm(g) / O.n_params(prob.dims, 6) < 1e-7 * 1.01
    assert abs(f - rep["f"]) <= 1e-10 * f


def test_small_dense_tensors_solve_in_fp64_when_mixed_is_asked(cp, ctx):
    """Below 4096 entries a mixed-precision request runs in FP64 (the bf16x3
    noise in f costs more iterations there than the tensor cores save);
    mixed_min_entries = -1 keeps it mixed.  Both meet the tolerance by the
    oracle's own gradient."""
    rng = synth.rng_for(0, 7)
    prob = synth.dense_problem(rng, (9, 8, 7), 3, 0.5, eta=0.05)
    u0 = synth.initial_guess(rng, prob.dims, 3)
    t = cp.cp_tensor_dense(ctx, dev(prob.T))
    X = O.DenseTensor(prob.T)
    for floor, mixed_expected in ((0, False), (-1, True)):
        o = cp.cp_solve_opts_default(3)
        o.prec = cp.CP_MIXED_BF16X3
        o.tol = 1e-8
        o.mixed_min_entries = floor
        u = dev(u0)
        rep = cp.cp_solve(ctx, t, o, u)
        assert rep["converged"]
        assert (rep["mixed_iters"] > 0) == mixed_expected, rep
        _, g = O.fg(X, u.cpu().numpy(), 3)
        assert np.linalg.norm(g) / O.n_params(prob.dims, 3) < 1e-8 * 1.01
