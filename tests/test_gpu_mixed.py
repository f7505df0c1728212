"""GPU checks of the mixed-precision dense MTTKRP (tcgen05, bf16x3 split
products, FP32 accumulation) against the FP64 oracle, through the C ABI.

Stated bound: relative Frobenius error of M^(n) <= 5e-5 (each split product
carries ~2^-17 relative error, the accumulation is FP32); f and g built from
these MTTKRPs are held to the same relative bound against their FP64 values
(g is compared relative to ||M||, the scale at which its terms cancel)."""
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
        err = rel(out.cpu().numpy().reshape(ref.shape), ref)
        assert err <= MIXED_TOL, (shape, R, n, err)


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
        assert rel(out.cpu().numpy().reshape(ref.shape), ref) <= MIXED_TOL


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
