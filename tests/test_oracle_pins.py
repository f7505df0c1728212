"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(brute force, closed forms, invariants, hand-worked examples), independent of
the oracle's own formulas.  CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import cp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_factors(rng, dims, R):
    return [rng.standard_normal((I, R)) for I in dims]


# --------------------------------------------------------------------------
# MTTKRP
# --------------------------------------------------------------------------

def explicit_matricize(T, n):
    """T_(n) built element by element: column index runs over the other
    modes in increasing order with the LAST one fastest (pure Python loops)."""
    dims = T.shape
    others = [m for m in range(T.ndim) if m != n]
    cols = list(itertools.product(*[range(dims[m]) for m in others]))
    Tn = np.zeros((dims[n], len(cols)))
    for i in range(dims[n]):
        for c, idx in enumerate(cols):
            full = [0] * T.ndim
            full[n] = i
            for m, v in zip(others, idx):
                full[m] = v
            Tn[i, c] = T[tuple(full)]
    return Tn, cols, others


def explicit_khatri_rao(factors, cols, others, R):
    """Phibar with rows in the same column order as explicit_matricize."""
    Phi = np.ones((len(cols), R))
    for c, idx in enumerate(cols):
        for m, v in zip(others, idx):
            for r in range(R):
                Phi[c, r] *= factors[m][v, r]
    return Phi


@pytest.mark.parametrize("dims,R", [((3, 4), 2), ((2, 3, 4), 3), ((3, 2, 4, 2), 2), ((5, 1, 3), 4)])
def test_mttkrp_equals_explicit_matricization_times_khatri_rao(dims, R):
    rng = np.random.default_rng(1)
    T = rng.standard_normal(dims)
    factors = rand_factors(rng, dims, R)
    for n in range(len(dims)):
        Tn, cols, others = explicit_matricize(T, n)
        Phi = explicit_khatri_rao(factors, cols, others, R)
        np.testing.assert_allclose(O.mttkrp_dense(T, factors, n), Tn @ Phi, rtol=1e-13, atol=1e-13)


def test_mttkrp_golden_hand_example():
    g = json.load(open(os.path.join(GOLDEN, "mttkrp_2x2x2.json")))
    T = np.array(g["T"], dtype=float)
    F = [np.array(g[k], dtype=float) for k in ("A", "B", "C")]
    for n in range(3):
        np.testing.assert_array_equal(O.mttkrp_dense(T, F, n), np.array(g["M"][n], dtype=float))


def test_mttkrp_rank_one_closed_form():
    rng = np.random.default_rng(2)
    a, b, c = rng.standard_normal(4), rng.standard_normal(5), rng.standard_normal(3)
    T = np.multiply.outer(np.multiply.outer(a, b), c)
    B, C = rng.standard_normal((5, 2)), rng.standard_normal((3, 2))
    A = rng.standard_normal((4, 2))
    M1 = O.mttkrp_dense(T, [A, B, C], 0)
    expect = np.outer(a, (b @ B) * (c @ C))
    np.testing.assert_allclose(M1, expect, rtol=1e-13)


def test_mttkrp_two_way_is_matrix_product():
    rng = np.random.default_rng(3)
    T = rng.standard_normal((6, 4))
    A, B = rng.standard_normal((6, 3)), rng.standard_normal((4, 3))
    np.testing.assert_allclose(O.mttkrp_dense(T, [A, B], 0), T @ B, rtol=1e-13)
    np.testing.assert_allclose(O.mttkrp_dense(T, [A, B], 1), T.T @ A, rtol=1e-13)


def test_sparse_mttkrp_matches_loop_over_nonzeros():
    rng = np.random.default_rng(4)
    dims = (5, 4, 6)
    coords = synth.distinct_coords(rng, dims, 40)
    vals = rng.standard_normal(40)
    F = rand_factors(rng, dims, 3)
    for n in range(3):
        ref = np.zeros((dims[n], 3))
        for k in range(40):
            for r in range(3):
                p = vals[k]
                for m in range(3):
                    if m != n:
                        p *= F[m][coords[k, m], r]
                ref[coords[k, n], r] += p
        np.testing.assert_allclose(O.mttkrp_sparse(coords, vals, dims, F, n), ref, rtol=1e-13, atol=1e-14)
        dense = np.zeros(dims)
        dense[tuple(coords.T)] = vals
        np.testing.assert_allclose(O.mttkrp_dense(dense, F, n), ref, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------
# f and g
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims,R", [((4, 5, 3), 2), ((3, 3, 2, 4), 3), ((6, 7), 2)])
def test_f_expansion_equals_bruteforce(dims, R):
    rng = np.random.default_rng(5)
    T = rng.standard_normal(dims)
    u = synth.initial_guess(rng, dims, R)
    X = O.DenseTensor(T)
    f, _ = O.fg(X, u, R)
    ref = 0.0
    F = O.unpack(u, dims, R)
    for idx in itertools.product(*[range(d) for d in dims]):
        model = sum(math.prod(F[n][idx[n], r] for n in range(len(dims))) for r in range(R))
        ref += 0.5 * (T[idx] - model) ** 2
    assert abs(f - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("dims,R", [((4, 3, 5), 2), ((3, 2, 3, 2), 3)])
def test_gradient_central_differences(dims, R):
    rng = np.random.default_rng(6)
    T = rng.standard_normal(dims)
    X = O.DenseTensor(T)
    u = synth.initial_guess(rng, dims, R)
    _, g = O.fg(X, u, R)
    fd = np.zeros_like(u)
    for k in range(u.size):
        h = 1e-6 * max(1.0, abs(u[k]))
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        fd[k] = (O.f_bruteforce(T, O.unpack(up, dims, R)) - O.f_bruteforce(T, O.unpack(um, dims, R))) / (2 * h)
    assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g)


@pytest.mark.parametrize("dims,R", [((5, 4, 3), 2), ((4, 3, 3, 2), 3)])
def test_f_along_a_line_is_a_polynomial_of_degree_2N(dims, R):
    """phi(beta) = f(u + beta d) is a polynomial of degree 2N (the model is
    multilinear in the factors; Section 2.1's line search sees this
    function): the interpolant through 2N + 1 values predicts phi elsewhere,
    its derivative is g(u + beta d) . d, and its leading coefficient is
    1/2 sum_{r,s} prod_n (D_n^T D_n)[r, s]."""
    rng = np.random.default_rng(13)
    N = len(dims)
    X = O.DenseTensor(rng.standard_normal(dims))
    u = synth.initial_guess(rng, dims, R)
    d = 0.3 * synth.initial_guess(rng, dims, R)
    b = np.linspace(-1.0, 1.5, 2 * N + 1)
    coef = np.polyfit(b, [O.fg(X, u + t * d, R)[0] for t in b], 2 * N)
    D = O.unpack(d, dims, R)
    lead = 0.5 * np.sum(np.prod([Dn.T @ Dn for Dn in D], axis=0))
    assert abs(coef[0] - lead) <= 1e-6 * abs(lead)
    for t in (-0.7, 0.2, 1.3):
        f, g = O.fg(X, u + t * d, R)
        assert abs(np.polyval(coef, t) - f) <= 1e-8 * (abs(f) + X.norm2)
        assert abs(np.polyval(np.polyder(coef), t) - g @ d) <= 1e-6 * (abs(g @ d) + X.norm2)


@pytest.mark.parametrize("dims,R", [((5, 4, 3), 2), ((4, 3, 3, 2), 3)])
def test_mttkrp_is_multilinear_along_a_line(dims, R):
    """M^(n)(u + beta d) = sum over the 2^(N-1) choices of A or D for the
    other modes of beta^(number of D) times that MTTKRP (the Khatri-Rao
    variants the line search's single pass makes), for every mode."""
    rng = np.random.default_rng(17)
    N = len(dims)
    T = rng.standard_normal(dims)
    A = rand_factors(rng, dims, R)
    D = rand_factors(rng, dims, R)
    beta = 0.37
    X = [a + beta * dd for a, dd in zip(A, D)]
    for n in range(N):
        others = [m for m in range(N) if m != n]
        acc = np.zeros((dims[n], R))
        for v in range(2 ** (N - 1)):
            F = [D[m] if m != n and (v >> others.index(m)) & 1 else A[m] for m in range(N)]
            acc += beta ** bin(v).count("1") * O.mttkrp_dense(T, F, n)
        ref = O.mttkrp_dense(T, X, n)
        assert np.abs(acc - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_line_search_on_the_polynomial_visits_the_same_trials(seed):
    """More-Thuente on phi(beta) = f(x0 + beta d) evaluated through f and g at
    every trial, and on the degree-2N polynomial that interpolates phi (its
    derivative for phi'), end at the same step after the same number of trials
    with the same termination code: a search on the exact polynomial is the
    search Section 2.1 runs."""
    rng = np.random.default_rng(seed)
    dims, R = (6, 5, 4), 3
    X = O.DenseTensor(rng.standard_normal(dims))
    x0 = synth.initial_guess(rng, dims, R)
    f0, g0 = O.fg(X, x0, R)
    d = -g0 * 0.05 + 0.1 * rng.standard_normal(x0.size)
    if g0 @ d >= 0:
        d = -g0 * 0.05
    N = len(dims)

    def phi_true(b):
        f, g = O.fg(X, x0 + b * d, R)
        return f, float(g @ d), None

    b = np.linspace(-1.0, 2.0, 2 * N + 1)
    coef = np.polyfit(b, [O.fg(X, x0 + t * d, R)[0] for t in b], 2 * N)
    dcoef = np.polyder(coef)

    def phi_poly(t):
        return float(np.polyval(coef, t)), float(np.polyval(dcoef, t)), None

    st, ft, _, _, nt, it = O.more_thuente(phi_true, f0, float(g0 @ d))
    sp, fp, _, _, np_, ip = O.more_thuente(phi_poly, *phi_poly(0.0)[:2])
    assert (nt, it) == (np_, ip)
    assert abs(st - sp) <= 1e-8 * abs(st)
    assert abs(ft - fp) <= 1e-8 * (abs(ft) + X.norm2)


def test_exact_decomposition_has_zero_f_and_g():
    rng = np.random.default_rng(7)
    dims, R = (5, 4, 6), 3
    F = rand_factors(rng, dims, R)
    T = O.cp_full(F)
    X = O.DenseTensor(T)
    f, g = O.fg(X, O.pack(F), R)
    assert abs(f) <= 1e-12 * X.norm2
    assert np.linalg.norm(g) <= 1e-12 * X.norm2
    for n in range(3):  # M^(n) = A^(n) Gammabar^(n) at an exact decomposition
        np.testing.assert_allclose(O.mttkrp_dense(T, F, n), F[n] @ O.gamma_bar(F, n), rtol=1e-12, atol=1e-12)


def test_sparse_fg_equals_dense_fg():
    rng = np.random.default_rng(8)
    dims, R = (6, 5, 7), 3
    coords = synth.distinct_coords(rng, dims, 50)
    vals = rng.standard_normal(50)
    dense = np.zeros(dims)
    dense[tuple(coords.T)] = vals
    u = synth.initial_guess(rng, dims, R)
    fs, gs = O.fg(O.SparseTensor(coords, vals, dims), u, R)
    fd, gd = O.fg(O.DenseTensor(dense), u, R)
    assert abs(fs - fd) <= 1e-12 * abs(fd)
    np.testing.assert_allclose(gs, gd, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# ALS
# --------------------------------------------------------------------------

def test_als_mode_updates_decrease_f_and_zero_the_mode_gradient():
    rng = np.random.default_rng(9)
    prob = synth.dense_problem(rng, (8, 7, 6), 3, 0.5, eta=0.1)
    X = O.DenseTensor(prob.T)
    R = 3
    u = synth.initial_guess(rng, prob.dims, R)
    F = [A.copy() for A in O.unpack(u, prob.dims, R)]
    f_prev = O.f_bruteforce(prob.T, F)
    for sweep in range(4):
        for n in range(3):
            M = O.mttkrp_dense(prob.T, F, n)
            F[n] = O.als_mode_solve(M, O.gamma_bar(F, n))
            f_now = O.f_bruteforce(prob.T, F)
            assert f_now <= f_prev * (1 + 1e-12)
            f_prev = f_now
            _, g = O.fg(X, O.pack(F), R)
            Gn = O.unpack(g, prob.dims, R)[n]
            assert np.linalg.norm(Gn) <= 1e-9 * np.linalg.norm(M)
    # the sweep function reproduces the hand-rolled sweep
    u1 = O.als_sweep(X, u, R)
    F2 = [A.copy() for A in O.unpack(u, prob.dims, R)]
    for n in range(3):
        F2[n] = O.als_mode_solve(O.mttkrp_dense(prob.T, F2, n), O.gamma_bar(F2, n))
    np.testing.assert_allclose(u1, O.pack(F2), rtol=1e-12)


def test_gradient_vanishes_at_an_als_fixed_point():
    """Plain ALS (one sweep and a normalisation per step) run until it stops
    moving reaches a point where every mode solve returns its own factor, so
    each G^(n) = -M^(n) + A^(n) Gammabar^(n) is zero there: the gradient, built
    independently of the ALS solves, must vanish up to rounding."""
    rng = synth.rng_for(88)
    prob = synth.dense_problem(rng, (9, 8, 7), 3, 0.5, eta=0.1)
    X = O.DenseTensor(prob.T)
    R = 3
    u, _, _ = O.normalize(synth.initial_guess(rng, prob.dims, R), prob.dims, R)
    for _ in range(2000):
        v, _, _ = O.normalize(O.als_sweep(X, u, R), prob.dims, R)
        step = np.linalg.norm(v - u) / np.linalg.norm(u)
        u = v
        if step < 1e-14:
            break
    assert step < 1e-14
    _, g = O.fg(X, u, R)
    F = O.unpack(u, prob.dims, R)
    Mnorm = np.linalg.norm(O.pack([X.mttkrp(F, n) for n in range(3)]))
    assert np.linalg.norm(g) <= 1e-12 * Mnorm


def test_als_recovers_noise_free_planted_tensor():
    rng = np.random.default_rng(10)
    prob = synth.dense_problem(rng, (10, 9, 8), 3, 0.3)
    X = O.DenseTensor(prob.T)
    u = synth.initial_guess(rng, prob.dims, 3)
    for _ in range(400):
        u = O.als_sweep(X, u, 3)
    f, g = O.fg(X, u, 3)
    assert f <= 1e-16 * X.norm2 * 1e4
    # congruence with the planted factors up to permutation and scaling
    F = O.unpack(u, prob.dims, 3)
    cong = np.ones((3, 3))
    for A, B in zip(F, prob.planted):
        An = A / np.linalg.norm(A, axis=0)
        Bn = B / np.linalg.norm(B, axis=0)
        cong *= np.abs(An.T @ Bn)
    best = max(sum(cong[i, p[i]] for i in range(3)) for p in itertools.permutations(range(3)))
    assert best >= 3 * (1 - 1e-8)


# --------------------------------------------------------------------------
# Normalisation
# --------------------------------------------------------------------------

def test_normalize_invariants_and_exact_gradient_rescale():
    rng = np.random.default_rng(11)
    dims, R = (5, 6, 4), 4
    T = rng.standard_normal(dims)
    X = O.DenseTensor(T)
    u = synth.initial_guess(rng, dims, R) * np.repeat(rng.uniform(0.1, 3, size=R * 0 + 1), 1)
    f, g = O.fg(X, u, R)
    un, gn, lam = O.normalize(u, dims, R, g)
    f2, g2 = O.fg(X, un, R)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    np.testing.assert_allclose(gn, g2, rtol=1e-10, atol=1e-12)
    assert np.all(np.diff(lam) <= 0)
    F = O.unpack(un, dims, R)
    for A in F:
        np.testing.assert_allclose(np.linalg.norm(A, axis=0), lam ** (1 / 3), rtol=1e-12)


def test_normalize_carries_mttkrp_gram_and_inverse_by_scales_and_order():
    """After the normalisation every mode's factor is the old one with columns
    scaled by s_{n,r} = lambda_r^(1/N) / ||a_r^(n)|| and reordered by decreasing
    lambda.  Then M^(n), the Grams and the inverse of Gammabar^(n) at the new
    point follow from the old ones by the same order and the products of the
    other modes' scales; the accelerated iteration reuses them instead of
    recomputing.  M^(n) does not depend on A^(n) at all, which is why the
    sweep's last MTTKRP is the one at the swept point."""
    rng = np.random.default_rng(23)
    dims, R = (5, 4, 6), 4
    N = len(dims)
    T = rng.standard_normal(dims)
    F = [A * rng.uniform(0.2, 4.0, size=R) for A in rand_factors(rng, dims, R)]
    nu = np.stack([np.sqrt(np.sum(A * A, axis=0)) for A in F])
    lam = np.prod(nu, axis=0)
    order = np.argsort(-lam, kind="stable")
    s = lam ** (1.0 / N) / nu
    un, _, lam_sorted = O.normalize(O.pack(F), dims, R)
    np.testing.assert_allclose(lam_sorted, lam[order], rtol=1e-13)
    Fn = O.unpack(un, dims, R)
    for n in range(N):
        np.testing.assert_allclose(Fn[n], (F[n] * s[n])[:, order], rtol=1e-12)
        c = np.prod(np.delete(s, n, axis=0), axis=0)
        M_old = O.mttkrp_dense(T, F, n)
        np.testing.assert_allclose(O.mttkrp_dense(T, Fn, n), (M_old * c)[:, order],
                                   rtol=1e-11, atol=1e-12 * np.abs(M_old).max())
        G_old = F[n].T @ F[n]
        np.testing.assert_allclose(O.grams(Fn)[n],
                                   (G_old * np.outer(s[n], s[n]))[np.ix_(order, order)],
                                   rtol=1e-11, atol=1e-13 * np.abs(G_old).max())
        Gi_old = np.linalg.inv(O.gamma_bar(F, n))
        Gi_new = np.linalg.inv(O.gamma_bar(Fn, n))
        np.testing.assert_allclose(Gi_new, (Gi_old / np.outer(c, c))[np.ix_(order, order)],
                                   rtol=1e-8, atol=1e-10 * np.abs(Gi_new).max())
        F_other = [A.copy() for A in F]
        F_other[n] = rng.standard_normal(F[n].shape)
        np.testing.assert_array_equal(O.mttkrp_dense(T, F_other, n), M_old)


def test_normalize_zero_column_left_unscaled():
    dims, R = (3, 3), 2
    u = np.arange(1.0, 13.0)
    F = O.unpack(u.copy(), dims, R)
    F[0][:, 1] = 0.0
    un, _, lam = O.normalize(O.pack(F), dims, R)
    assert lam[-1] == 0.0
    Fn = O.unpack(un, dims, R)
    np.testing.assert_array_equal(Fn[1][:, 1], F[1][:, 1])


# --------------------------------------------------------------------------
# N-GMRES Step II: in the linear case it is GMRES (Lemma 1)
# --------------------------------------------------------------------------

def arnoldi_gmres(A, b, x0, Minv, k):
    """Right-preconditioned GMRES by Arnoldi: minimise ||b - A x|| over
    x in x0 + Minv K_k(A Minv, r0) (textbook algorithm, independent of the oracle)."""
    n = b.size
    r0 = b - A @ x0
    beta = np.linalg.norm(r0)
    V = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    V[:, 0] = r0 / beta
    for j in range(k):
        w = A @ (Minv @ V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return x0 + Minv @ (V[:, :k] @ y)


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_ngmres_step_is_gmres_in_the_linear_case(k):
    rng = np.random.default_rng(12)
    n = 30
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    Minv = np.diag(1.0 / np.diag(A))        # Jacobi preconditioner
    grad = lambda x: A @ x - b               # g(u) of f = 1/2 u^T A u - b^T u
    us = [rng.standard_normal(n)]
    for _ in range(k):                       # stationary iteration (Eq. stat)
        us.append(us[-1] + Minv @ (b - A @ us[-1]))
    U = np.array(us[:k])
    G = np.array([grad(x) for x in us[:k]])
    ubar = us[k]
    uhat, alpha = O.ngmres_step(U, G, ubar, grad(ubar), eps=0.0)
    ref = arnoldi_gmres(A, b, us[0], Minv, k)
    np.testing.assert_allclose(uhat, ref, rtol=1e-8, atol=1e-10)


def test_ngmres_single_vector_closed_form():
    rng = np.random.default_rng(13)
    P = 50
    u0, g0, ub, gb = (rng.standard_normal(P) for _ in range(4))
    uhat, alpha = O.ngmres_step(u0[None], g0[None], ub, gb, eps=1e-12)
    p = gb - g0
    delta = 1e-12 * (p @ p)
    a = -(p @ gb) / (p @ p + delta)
    assert abs(alpha[0] - a) <= 1e-14 * abs(a)
    np.testing.assert_allclose(uhat, ub + a * (ub - u0), rtol=1e-14)


# --------------------------------------------------------------------------
# More-Thuente line search
# --------------------------------------------------------------------------

def quad_phi(g0, c):
    return lambda a: (g0 * a + 0.5 * c * a * a, g0 + c * a, None)


def test_linesearch_accepts_unit_step_on_matching_quadratic():
    beta, f, g, _, nfev, info = O.more_thuente(quad_phi(-2.0, 2.0), 0.0, -2.0)
    assert (beta, nfev, info) == (1.0, 1, 1)


def strong_wolfe(phi, beta, f0, g0, mu, eta):
    f, g, _ = phi(beta)
    return f <= f0 + mu * beta * g0 + 1e-15 * abs(f0) and abs(g) <= eta * abs(g0)


def mt_test_functions():
    """Test functions of More and Thuente's Section 5 (definitions only)."""
    def f1(a, b=2.0):
        return -a / (a * a + b), (a * a - b) / (a * a + b) ** 2

    def f2(a, b=0.004):
        return (a + b) ** 5 - 2 * (a + b) ** 4, 5 * (a + b) ** 4 - 8 * (a + b) ** 3

    def f3(a, b=0.01, l=39):
        if a <= 1 - b:
            p, dp = 1 - a, -1.0
        elif a >= 1 + b:
            p, dp = a - 1, 1.0
        else:
            p, dp = (a - 1) ** 2 / (2 * b) + b / 2, (a - 1) / b
        return (p + 2 * (1 - b) / (l * math.pi) * math.sin(l * math.pi * a / 2),
                dp + (1 - b) * math.cos(l * math.pi * a / 2))

    def gamma(b):
        return math.sqrt(1 + b * b) - b

    def yanai(b1, b2):
        def f(a):
            v = gamma(b1) * math.sqrt((1 - a) ** 2 + b2 * b2) + gamma(b2) * math.sqrt(a * a + b1 * b1)
            dv = -gamma(b1) * (1 - a) / math.sqrt((1 - a) ** 2 + b2 * b2) + gamma(b2) * a / math.sqrt(a * a + b1 * b1)
            return v, dv
        return f

    return [(f1, 1e-3, 1e-1), (f2, 1e-1, 1e-1), (f3, 1e-1, 1e-1),
            (yanai(1e-3, 1e-3), 1e-3, 1e-3), (yanai(1e-2, 1e-3), 1e-3, 1e-3),
            (yanai(1e-3, 1e-2), 1e-3, 1e-3)]


@pytest.mark.parametrize("case", range(6))
@pytest.mark.parametrize("a0", [1e-3, 1e-1, 1e1, 1e3])
def test_linesearch_strong_wolfe_on_published_test_functions(case, a0):
    fn, mu, eta = mt_test_functions()[case]
    phi = lambda a: (*fn(a), None)
    f0, g0 = fn(0.0)
    opts = O.LSOpts(ftol=mu, gtol=eta, stp0=a0, maxfev=40, xtol=1e-12)
    beta, f, g, _, nfev, info = O.more_thuente(phi, f0, g0, opts)
    assert info == 1, (case, a0, info, nfev)
    assert strong_wolfe(phi, beta, f0, g0, mu, eta)
    assert nfev <= 20


def record_trials(phi):
    trials = []

    def rec(a):
        out = phi(a)
        trials.append(a)
        return out
    return rec, trials


def test_linesearch_extrapolates_by_four_steps_until_maxfev_or_stpmax():
    """On phi(b) = -b the slope never flattens, so every trial extrapolates
    to the upper limit a_t + 4 (a_t - a_l): trials (4^k - 1) / 3 until
    maxfev ends the search (info 3), or stpmax is reached with sufficient
    decrease and the slope still below ftol phi'(0) (info 5)."""
    lin = lambda a: (-a, -1.0, None)
    rec, trials = record_trials(lin)
    beta, _, _, _, nfev, info = O.more_thuente(rec, 0.0, -1.0, O.LSOpts(maxfev=5))
    assert trials == [1.0, 5.0, 21.0, 85.0, 341.0] and (beta, nfev, info) == (341.0, 5, 3)
    rec, trials = record_trials(lin)
    beta, _, _, _, nfev, info = O.more_thuente(rec, 0.0, -1.0, O.LSOpts(stpmax=100.0))
    assert trials == [1.0, 5.0, 21.0, 85.0, 100.0] and (beta, nfev, info) == (100.0, 5, 5)


def test_linesearch_extrapolates_at_least_1_1_steps():
    """phi(b) = (b - 1.05)^2 - 1.05^2: after the unit trial both the cubic and
    the secant step point to the minimiser 1.05, inside the unbracketed lower
    limit a_t + 1.1 (a_t - a_l) = 2.1, so the next trial is 2.1."""
    phi = lambda a: ((a - 1.05) ** 2 - 1.05 ** 2, 2 * (a - 1.05), None)
    rec, trials = record_trials(phi)
    O.more_thuente(rec, 0.0, -2.1)
    assert trials[:2] == [1.0, pytest.approx(2.1, rel=1e-15)]


def test_linesearch_first_stage_works_on_psi():
    """phi(b) = -b + a b^2 + c b^3 with phi(1) between phi(0) + ftol phi'(0)
    and phi(0): phi is lower at 1 than at 0 (case 3 for phi, extrapolation
    beyond 2.1) but psi(b) = phi(b) - phi(0) - ftol b phi'(0) is higher
    (case 1 for psi), so the first stage must bracket in (0, 1) with the case-1
    step of psi."""
    mu = 1e-4
    c = 0.5 - 2 * (1 - 0.5e-4)
    a = (1 - 0.5e-4) - c
    phi = lambda b: (-b + a * b * b + c * b ** 3, -1 + 2 * a * b + 3 * c * b * b, None)
    f1, g1, _ = phi(1.0)
    assert f1 == pytest.approx(-0.5e-4) and g1 == pytest.approx(-0.5)
    rec, trials = record_trials(phi)
    O.more_thuente(rec, 0.0, -1.0, O.LSOpts(ftol=mu))
    lo = (0.0, 0.0, -1.0 + mu)
    t = (1.0, f1 + mu, g1 + mu)
    ac = hermite_cubic_min(*lo, *t)
    aq = quad_fgf_min(*lo, t[0], t[1])
    want = ac if abs(ac) < abs(aq) else ac + 0.5 * (aq - ac)
    assert 0 < want < 1 and trials[1] == pytest.approx(want, rel=1e-12)


def psi_step_quartic():
    """The quartic with phi(0) = 0, phi'(0) = -1, phi(1) = -0.2, phi'(1) = -0.5,
    phi(5) = -0.25, searched with ftol = gtol = 0.1: the unit trial lies
    below the sufficient-decrease line and is still steep, so the search
    extrapolates to 5, where phi is above that line but below phi(1); the
    trial after it is chosen in the first stage (psi) with the lower end at 1,
    the one path on which the lower end is mapped back from psi."""
    A = np.array([[1, 0, 0, 0, 0], [0, 1, 0, 0, 0], [1, 1, 1, 1, 1], [0, 1, 2, 3, 4],
                  [1, 5, 25, 125, 625]], dtype=float)
    P = np.polynomial.Polynomial(np.linalg.solve(A, [0, -1, -0.2, -0.5, -0.25]))
    dP = P.deriv()
    return (lambda a: (float(P(a)), float(dP(a)))), 0.1, 0.1


@pytest.mark.parametrize("case", range(7))
@pytest.mark.parametrize("a0", [1e-3, 1e-1, 1e0, 1e1, 1e3])
def test_linesearch_interval_ends_are_evaluated_points(monkeypatch, case, a0):
    """Every point handed to the trial selection (the two ends and the new
    trial) is an evaluated trial or 0 with its own phi and phi' (or, all three
    together, psi and psi' in the first stage)."""
    fn, mu, eta = (mt_test_functions() + [psi_step_quartic()])[case]
    f0, g0 = fn(0.0)
    seen = {0.0: (f0, g0)}

    def phi(a):
        v, d = fn(a)
        seen[a] = (v, d)
        return v, d, None

    real, checked = O.mt_trial, []

    def checking_trial(lo, hi, t, brackt, stmin, stmax):
        forms = []
        for a, v, d in (lo, hi, t):
            fv, fd = seen[a]
            if v == fv and d == fd:
                forms.append("phi")
            elif v == pytest.approx(fv - f0 - a * mu * g0, rel=1e-12, abs=1e-15) and \
                    d == pytest.approx(fd - mu * g0, rel=1e-12, abs=1e-15):
                forms.append("psi")
            else:
                forms.append("neither")
        assert len(set(forms)) == 1 and forms[0] != "neither", (lo, hi, t, forms)
        checked.append(forms[0])
        return real(lo, hi, t, brackt, stmin, stmax)

    monkeypatch.setattr(O, "mt_trial", checking_trial)
    O.more_thuente(phi, f0, g0, O.LSOpts(ftol=mu, gtol=eta, stp0=a0, maxfev=40, xtol=1e-12))


def test_linesearch_interval_checks_reach_the_first_stage():
    """Across the cases above the first stage (psi) and the second (phi) are
    both exercised, and the quartic takes a psi step with its lower end away
    from 0, so the check above covers the mapping back from psi."""
    forms = set()
    for fn, mu, eta in mt_test_functions() + [psi_step_quartic()]:
        for a0 in [1e-3, 1e-1, 1e0, 1e1, 1e3]:
            f0, g0 = fn(0.0)
            real = O.mt_trial
            try:
                def spy(lo, hi, t, brackt, stmin, stmax):
                    a, v, _ = t
                    if v == fn(a)[0]:
                        forms.add("phi")
                    else:
                        forms.add("psi, lower end at 0" if lo[0] == 0.0 else "psi, lower end inside")
                    return real(lo, hi, t, brackt, stmin, stmax)
                O.mt_trial = spy
                O.more_thuente(lambda a: (*fn(a), None), f0, g0,
                               O.LSOpts(ftol=mu, gtol=eta, stp0=a0, maxfev=40, xtol=1e-12))
            finally:
                O.mt_trial = real
    assert forms == {"phi", "psi, lower end at 0", "psi, lower end inside"}


def test_linesearch_rejects_ascent_direction():
    assert O.more_thuente(quad_phi(1.0, 1.0), 0.0, 1.0)[-1] == -1


def poly_phi(coeffs):
    """phi(b) = -b + b^2 (c0 + c1 b + c2 b^2 + ...): phi(0) = 0, phi'(0) = -1."""
    P = np.polynomial.Polynomial([0.0, -1.0] + [float(c) for c in coeffs])
    dP = P.deriv()
    return lambda a: (float(P(a)), float(dP(a)))


def test_linesearch_bisects_a_bracket_that_shrinks_too_slowly():
    """phi = -b + 18 b^2 - 16 b^3 + 20 b^4 - 17 b^5: phi(1) = 4 > phi(0), so
    the unit trial brackets the minimum in [0, 1].  The next two trials are
    lower, still descending points near 0, each becoming the lower end while
    1 stays the upper end.  After the third trial the bracket [a_3, 1] is
    still wider than 0.66 times the bracket two trials earlier ([0, 1]), so
    More and Thuente's safeguard replaces the interpolated step by the
    midpoint of the bracket."""
    fn = poly_phi([18, -16, 20, -17])
    rec, trials = record_trials(lambda a: (*fn(a), None))
    O.more_thuente(rec, 0.0, -1.0)
    a2, a3 = trials[1], trials[2]
    assert fn(1.0)[0] > 0.0
    for prev, a in ((0.0, a2), (a2, a3)):
        assert fn(a)[0] < fn(prev)[0] and fn(a)[1] < 0.0 and 0.0 < a < 1.0
    assert 1.0 - a3 >= 0.66 * 1.0
    assert trials[3] == pytest.approx(a3 + 0.5 * (1.0 - a3), rel=1e-15)


def test_linesearch_returns_the_best_point_once_the_interval_is_below_xtol():
    """phi = -b + 5 b^6 with xtol = 0.8: phi(1) = 4 > 0 brackets the minimum
    in [0, 1]; the second trial is lower and still descending, so the bracket
    becomes [a_2, 1], whose width 1 - a_2 is below xtol times its upper end.
    No further progress is allowed: the next trial is the best point a_2
    itself, and the search ends there with info 2."""
    fn = poly_phi([0, 0, 0, 5])
    rec, trials = record_trials(lambda a: (*fn(a), None))
    beta, _, _, _, nfev, info = O.more_thuente(rec, 0.0, -1.0, O.LSOpts(xtol=0.8))
    a2 = trials[1]
    assert fn(a2)[0] < 0.0 and fn(a2)[1] < 0.0 and 1.0 - a2 <= 0.8
    assert trials == [1.0, a2, a2] and (beta, nfev, info) == (a2, 3, 2)


def test_linesearch_first_stage_cannot_return_after_the_switch():
    """The second stage starts at the first trial with psi <= 0 and
    phi' >= min(ftol, gtol) phi'(0).  Such a trial lies past a minimiser and
    on or below the sufficient-decrease line, and it closes the bracket on
    that side, so every later trial that is no higher than the best point is
    also on or below the line: the first stage's step on psi (taken only for
    trials above the line) cannot occur after the switch.  Checked on random
    quintics and step options: after the switch, no trial is both no higher
    than the lower end and above the line."""
    rng = np.random.default_rng(20)
    switched_cases = 0
    for _ in range(400):
        fn = poly_phi(rng.normal(size=4) * rng.choice([1.0, 5.0, 20.0]))
        mu, eta = float(rng.choice([1e-4, 0.1, 0.3])), float(rng.choice([1e-3, 1e-2, 0.1, 0.9]))
        opts = O.LSOpts(ftol=mu, gtol=eta, stp0=float(10 ** rng.uniform(-2, 1)), maxfev=30)
        seen, state = [], {"switched": False}
        real = O.mt_trial

        def spy(lo, hi, t, brackt, stmin, stmax):
            seen.append((lo, t, state["switched"]))
            return real(lo, hi, t, brackt, stmin, stmax)

        def phi(a):
            f, g = fn(a)
            if f <= mu * a * -1.0 and g >= min(mu, eta) * -1.0:
                state["switched"] = True
            return f, g, None
        O.mt_trial = spy
        try:
            O.more_thuente(phi, 0.0, -1.0, opts)
        finally:
            O.mt_trial = real
        for lo, t, after in seen:
            a, f = t[0], fn(t[0])[0]
            lo_f = fn(lo[0])[0] if lo[0] != 0.0 else 0.0
            if after and f <= lo_f:
                assert f <= -mu * a, (a, f, lo)
        switched_cases += any(after for _, _, after in seen)
    assert switched_cases >= 20


# Trial selection of More-Thuente, case by case, against interpolants built
# here by solving their interpolation conditions as linear systems.

def hermite_cubic_min(a, fa, ga, b, fb, gb):
    """Local minimiser of the cubic with p(a) = fa, p'(a) = ga, p(b) = fb,
    p'(b) = gb, found from the roots of p' (None if p has none)."""
    x = np.array([0.0, b - a])
    V = np.array([[1, x[0], x[0] ** 2, x[0] ** 3], [0, 1, 2 * x[0], 3 * x[0] ** 2],
                  [1, x[1], x[1] ** 2, x[1] ** 3], [0, 1, 2 * x[1], 3 * x[1] ** 2]])
    c = np.linalg.solve(V, [fa, ga, fb, gb])
    for r in np.roots([3 * c[3], 2 * c[2], c[1]]):
        if abs(r.imag) < 1e-12 and 2 * c[2] + 6 * c[3] * r.real > 0:
            return a + r.real
    return None


def quad_fgf_min(a, fa, ga, b, fb):
    """Stationary point of the quadratic with q(a) = fa, q'(a) = ga, q(b) = fb."""
    h = b - a
    c = np.linalg.solve([[1, 0, 0], [0, 1, 0], [1, h, h * h]], [fa, ga, fb])
    return a - c[1] / (2 * c[2])


def secant_gg_root(a, ga, b, gb):
    """Zero of the straight line through (a, ga) and (b, gb)."""
    m, q = np.linalg.solve([[a, 1], [b, 1]], [ga, gb])
    return -q / m


@pytest.mark.parametrize("t", [(1.0, 0.5, 1.0), (1.0, 0.5, 3.0), (1.0, 3.0, -0.5), (-1.0, 0.7, -1.5)])
def test_mt_trial_case1_higher_value(t):
    """f_t > f_l: the minimum is bracketed; the cubic step if it is nearer
    a_l than the quadratic one, else halfway from the cubic to the quadratic;
    the new trial becomes the upper end."""
    lo = (0.0, 0.0, -1.0) if t[0] > 0 else (0.0, 0.0, 1.0)
    hi = (0.0, 0.0, -1.0)
    nlo, nhi, nxt, brackt = O.mt_trial(lo, hi, t, False, 0.0, 10.0)
    ac = hermite_cubic_min(*lo, *t)
    aq = quad_fgf_min(*lo, t[0], t[1])
    want = ac if abs(ac - lo[0]) < abs(aq - lo[0]) else ac + 0.5 * (aq - ac)
    assert brackt and nlo == lo and nhi == t
    assert nxt == pytest.approx(want, rel=1e-12, abs=1e-14)


def test_mt_trial_case1_takes_both_branches():
    """The case-1 examples above include one that takes the cubic step and
    one that takes the midpoint, with the cubic and quadratic steps apart, so
    that exchanging the two interpolants changes the result."""
    lo = (0.0, 0.0, -1.0)
    near = []
    for t in [(1.0, 0.5, 1.0), (1.0, 0.5, 3.0)]:
        ac, aq = hermite_cubic_min(*lo, *t), quad_fgf_min(*lo, t[0], t[1])
        assert abs(ac - aq) > 1e-3
        near.append(abs(ac - lo[0]) < abs(aq - lo[0]))
    assert sorted(near) == [False, True]


@pytest.mark.parametrize("t", [(1.0, -0.2, 0.5), (1.0, -0.6, 0.1), (2.0, -0.5, 3.0)])
def test_mt_trial_case2_derivative_sign_change(t):
    """f_t <= f_l, g_t g_l < 0: bracketed; of the cubic and secant steps the
    one farther from a_t; a_t becomes the lower end and a_l the upper."""
    lo, hi = (0.0, 0.0, -1.0), (5.0, 9.0, 1.0)
    nlo, nhi, nxt, brackt = O.mt_trial(lo, hi, t, False, 0.0, 10.0)
    ac = hermite_cubic_min(*lo, *t)
    asec = secant_gg_root(lo[0], lo[2], t[0], t[2])
    want = ac if abs(ac - t[0]) >= abs(asec - t[0]) else asec
    assert brackt and nlo == t and nhi == lo
    assert nxt == pytest.approx(want, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("t,brackt", [((1.0, -0.8, -0.3), False), ((1.0, -0.8, -0.3), True),
                                      ((1.0, -0.55, -0.9), False), ((0.5, -0.4, -0.6), True)])
def test_mt_trial_case3_derivative_decreases(t, brackt):
    """f_t <= f_l, same sign, |g_t| <= |g_l|: the cubic step if it lies beyond
    a_t (else the far bound); not bracketed: the farther of cubic and secant,
    clipped to [stmin, stmax]; bracketed: the nearer, at most 0.66 of the way
    to the upper end."""
    lo, hi, stmax = (0.0, 0.0, -1.0), (2.0, 1.0, 1.0), 10.0
    nlo, nhi, nxt, b2 = O.mt_trial(lo, hi, t, brackt, 0.0, stmax)
    ac = hermite_cubic_min(*lo, *t)
    if ac is None or ac <= t[0]:
        ac = stmax
    asec = secant_gg_root(lo[0], lo[2], t[0], t[2])
    if brackt:
        want = ac if abs(ac - t[0]) < abs(asec - t[0]) else asec
        want = min(t[0] + 0.66 * (hi[0] - t[0]), want)
    else:
        want = ac if abs(ac - t[0]) > abs(asec - t[0]) else asec
        want = min(stmax, max(0.0, want))
    assert b2 == brackt and nlo == t and nhi == hi
    assert nxt == pytest.approx(want, rel=1e-12, abs=1e-14)


def test_mt_trial_case4_derivative_does_not_decrease():
    """f_t <= f_l, same sign, |g_t| > |g_l|: not bracketed -> the far bound;
    bracketed -> the cubic step between a_t and the upper end."""
    lo, t = (0.0, 0.0, -1.0), (1.0, -2.0, -1.5)
    assert O.mt_trial(lo, (0.0, 0.0, -1.0), t, False, 0.0, 10.0)[2] == 10.0
    hi = (3.0, 1.0, 2.0)
    nlo, nhi, nxt, brackt = O.mt_trial(lo, hi, t, True, 0.0, 10.0)
    assert nlo == t and nhi == hi and brackt
    assert nxt == pytest.approx(hermite_cubic_min(*t, *hi), rel=1e-12)


# --------------------------------------------------------------------------
# COO sort and segmentation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2])
def test_coo_sort_matches_python_sorted(n):
    rng = np.random.default_rng(14)
    dims = (4, 5, 3)
    coords = synth.distinct_coords(rng, dims, 45)
    perm, seg_ptr, seg_row = O.coo_sort_mode(coords, n)
    key = lambda k: tuple(int(coords[k, (n + j) % 3]) for j in range(3))
    assert list(perm) == sorted(range(45), key=key)
    assert seg_ptr[0] == 0 and seg_ptr[-1] == 45 and np.all(np.diff(seg_ptr) > 0)
    rows = coords[perm, n]
    for s in range(seg_row.size):
        assert np.all(rows[seg_ptr[s]:seg_ptr[s + 1]] == seg_row[s])
    assert len(set(seg_row.tolist())) == seg_row.size


def test_coo_sort_empty():
    perm, seg_ptr, seg_row = O.coo_sort_mode(np.zeros((0, 3), dtype=np.int64), 1)
    assert perm.size == 0 and list(seg_ptr) == [0] and seg_row.size == 0


# --------------------------------------------------------------------------
# Generators
# --------------------------------------------------------------------------

def test_collinear_factor_has_exact_collinearity():
    rng = synth.rng_for(99)
    for c in (0.5, 0.9):
        A = synth.collinear_factor(rng, 40, 5, c)
        np.testing.assert_allclose(A.T @ A, synth.collinearity_matrix(5, c), atol=1e-12)


def test_noise_scaled_to_eta_of_planted_norm():
    rng = synth.rng_for(98)
    prob = synth.dense_problem(rng, (6, 7, 8), 2, 0.5, eta=0.1)
    TR = O.cp_full(prob.planted)
    assert abs(np.linalg.norm(prob.T - TR) - 0.1 * np.linalg.norm(TR)) <= 1e-12 * np.linalg.norm(TR)


def test_laplacian_matches_paper_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "laplacian_d2_s2.json")))
    lap = synth.laplacian_tensor(g["d"], g["s"])
    got = {tuple(int(x) for x in c): float(v) for c, v in zip(lap.coords, lap.vals)}
    want = {tuple(c): float(v) for c, v in g["nonzeros"]}
    assert got == want


@pytest.mark.parametrize("d,s", [(1, 6), (2, 4), (3, 3)])
def test_laplacian_is_the_kronecker_sum_of_1d_laplacians(d, s):
    """With the first d indices as the grid point and the last d as its
    neighbour, the tensor viewed as an s^d x s^d matrix is the Kronecker sum
    of d copies of tridiag(-1, 2, -1), whose eigenvalues are the sums of d
    values 2 - 2 cos(k pi / (s + 1)), k = 1..s."""
    lap = synth.laplacian_tensor(d, s)
    T = np.zeros(lap.dims)
    T[tuple(lap.coords.T)] = lap.vals
    A = T.reshape(s ** d, s ** d)
    L1 = 2 * np.eye(s) - np.eye(s, k=1) - np.eye(s, k=-1)
    K = np.zeros((s ** d, s ** d))
    for k in range(d):
        term = np.ones((1, 1))
        for m in range(d):
            term = np.kron(term, L1 if m == k else np.eye(s))
        K += term
    np.testing.assert_array_equal(A, K)
    mu = 2 - 2 * np.cos(np.arange(1, s + 1) * np.pi / (s + 1))
    sums = np.sort([sum(c) for c in itertools.product(mu, repeat=d)])
    np.testing.assert_allclose(np.linalg.eigvalsh(A), sums, atol=1e-12)


@pytest.mark.parametrize("d,s", [(1, 5), (2, 4), (3, 3)])
def test_laplacian_nnz_count(d, s):
    lap = synth.laplacian_tensor(d, s)
    assert lap.coords.shape[0] == s ** d + 2 * d * (s - 1) * s ** (d - 1)
    assert np.unique(lap.coords, axis=0).shape[0] == lap.coords.shape[0]


# --------------------------------------------------------------------------
# Whole N-GMRES solve
# --------------------------------------------------------------------------

def test_solve_two_way_laplacian_reaches_eckart_young_optimum():
    """Test Problem II with d = 1 is the s x s tridiagonal Laplacian, an SPD
    matrix with eigenvalues 2 - 2 cos(k pi / (s + 1)).  For N = 2 the CP problem
    is best rank-R matrix approximation, whose optimum keeps the R largest
    eigenvalues: f* = 1/2 sum of the other squared eigenvalues."""
    s, R = 12, 3
    lap = synth.laplacian_tensor(1, s)
    X = O.SparseTensor(lap.coords, lap.vals, lap.dims)
    lam = np.sort(2 - 2 * np.cos(np.arange(1, s + 1) * np.pi / (s + 1)))
    fstar = 0.5 * float(np.sum(lam[: s - R] ** 2))
    u0 = synth.initial_guess(synth.rng_for(97), lap.dims, R)
    u, g, rep = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-10, maxit=2000))
    assert rep.converged
    assert abs(rep.f - fstar) <= 1e-8 * fstar


def test_solve_monotone_and_recovers_planted():
    rng = synth.rng_for(96)
    prob = synth.dense_problem(rng, (9, 8, 10), 3, 0.9)
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, prob.dims, 3)
    u, g, rep = O.cp_solve(X, u0, O.SolveOpts(R=3, tol=1e-12, maxit=3000))
    assert rep.converged
    fs = [h[0] for h in rep.history]
    assert all(b <= a * (1 + 1e-10) + 1e-14 for a, b in zip(fs, fs[1:]))
    assert rep.f <= 1e-12 * X.norm2


def test_solve_restarting_every_iteration_is_normalised_als(monkeypatch):
    """When the N-GMRES direction is never a descent direction every iteration
    restarts from the ALS iterate, so the solve reduces to plain ALS (one sweep
    and one normalisation per iteration) and each window holds one point."""
    rng = synth.rng_for(94)
    prob = synth.dense_problem(rng, (6, 5, 7), 2, 0.5)
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, prob.dims, 2)
    windows = []

    def ascent_step(U, G, ubar, gbar, eps=1e-12):
        windows.append(len(U))
        return ubar + gbar, None

    monkeypatch.setattr(O, "ngmres_step", ascent_step)
    iters = 12
    u, g, rep = O.cp_solve(X, u0, O.SolveOpts(R=2, tol=0.0, maxit=iters))
    assert rep.iters == iters and rep.restarts == iters and rep.als_sweeps == iters
    assert windows == [1] * iters
    v, _, _ = O.normalize(u0, prob.dims, 2)
    for _ in range(iters):
        v, _, _ = O.normalize(O.als_sweep(X, v, 2), prob.dims, 2)
    np.testing.assert_allclose(u, v, rtol=1e-12, atol=1e-13 * np.abs(v).max())


def test_solve_with_failing_line_search_is_normalised_als(monkeypatch):
    """A line search that ends without sufficient decrease falls back to
    beta = 0 (R10), i.e. to the ALS iterate, so if it always does the solve's
    iterates are plain normalised ALS; every iteration counts as a restart or
    a line-search failure."""
    rng = synth.rng_for(92)
    prob = synth.dense_problem(rng, (6, 7, 5), 2, 0.5)
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, prob.dims, 2)

    def failing_search(phi, f0, g0, opts=O.LSOpts()):
        _, _, extra = phi(0.5)
        return 0.5, f0 + 1.0, None, extra, 1, 3

    monkeypatch.setattr(O, "more_thuente", failing_search)
    iters = 10
    u, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=2, tol=0.0, maxit=iters))
    assert rep.iters == iters and rep.restarts + rep.ls_failures == iters
    assert rep.ls_failures > 0
    v, _, _ = O.normalize(u0, prob.dims, 2)
    for _ in range(iters):
        v, _, _ = O.normalize(O.als_sweep(X, v, 2), prob.dims, 2)
    np.testing.assert_allclose(u, v, rtol=1e-12, atol=1e-13 * np.abs(v).max())


def test_solve_window_grows_to_w_and_slides(monkeypatch):
    """The window holds the last min(k + 1, w) iterates since the last
    restart, and a restart leaves only the ALS iterate in it."""
    rng = synth.rng_for(93)
    prob = synth.dense_problem(rng, (8, 7, 9), 3, 0.9)
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, prob.dims, 3)
    real = O.ngmres_step
    windows = []

    def recording_step(U, G, ubar, gbar, eps=1e-12):
        windows.append(len(U))
        return real(U, G, ubar, gbar, eps)

    monkeypatch.setattr(O, "ngmres_step", recording_step)
    w, iters = 3, 10
    _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=3, w=w, tol=0.0, maxit=iters))
    assert rep.iters == iters and len(windows) == iters
    assert windows[0] == 1
    resets = 0
    for prev, n in zip(windows, windows[1:]):
        if n == 1:
            resets += 1
        else:
            assert n == min(prev + 1, w)
    assert 2 <= max(windows) <= w
    # A restart in the last iteration leaves no later window to show it.
    assert resets in (rep.restarts, rep.restarts - 1)


def test_solve_loop_structure_of_algorithm_1(monkeypatch):
    """What Algorithm 1 with the readings R6, R8 fixes about the loop, checked
    on every call of Step II and Step III: the window's newest point is the
    iterate the ALS step (Step I) started from, the window slides by one, every
    point in it and every accelerated iterate is normalised (a fixed point of
    the normalisation), and the search starts at the ALS iterate."""
    rng = synth.rng_for(91)
    prob = synth.dense_problem(rng, (8, 7, 9), 3, 0.9)
    dims, R = prob.dims, 3
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, dims, R)
    real_step, real_search = O.ngmres_step, O.more_thuente
    calls, searches = [], []

    def recording_step(U, G, ubar, gbar, eps=1e-12):
        calls.append((np.array(U, copy=True), ubar.copy()))
        return real_step(U, G, ubar, gbar, eps)

    def recording_search(phi, f0, g0, opts=O.LSOpts()):
        f_at_0, _, (x0, _) = phi(0.0)
        _, _, (x1, _) = phi(1.0)
        searches.append((x0, x1, f0, f_at_0))
        return real_search(phi, f0, g0, opts)

    monkeypatch.setattr(O, "ngmres_step", recording_step)
    monkeypatch.setattr(O, "more_thuente", recording_search)
    w, iters = 3, 14
    _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=R, w=w, tol=0.0, maxit=iters))
    assert rep.iters == iters and len(searches) == iters - rep.restarts >= 4

    def is_normalised(v):
        return np.allclose(O.normalize(v, dims, R)[0], v, rtol=1e-11, atol=1e-13 * np.abs(v).max())

    for U, ubar in calls:
        assert all(is_normalised(row) for row in U)
        ubar_from_newest, _, _ = O.normalize(O.als_sweep(X, U[-1], R), dims, R)
        np.testing.assert_allclose(ubar, ubar_from_newest, rtol=1e-12, atol=1e-13 * np.abs(ubar).max())
    slid = 0
    for (U, _), (V, _) in zip(calls, calls[1:]):
        if len(V) == 1:
            continue                                     # a restart
        keep = U[1:] if len(U) == w else U
        np.testing.assert_array_equal(V[:-1], keep)
        slid += len(U) == w
    assert slid >= 1
    ubars = {c[1].tobytes() for c in calls}
    for x0, x1, f0, f_at_0 in searches:
        assert x0.tobytes() in ubars                      # beta = 0 is the ALS iterate
        assert f_at_0 == pytest.approx(f0, rel=1e-13)
        assert is_normalised(x1)                          # beta = 1 is the normalised uhat


@pytest.mark.parametrize("d,s,R", [(3, 4, 2), (4, 4, 2)])
def test_solve_test_problem_2_shapes_reach_an_als_fixed_point(d, s, R):
    """Test Problem II at the paper's N = 6 and N = 8 sizes (s = 4, R = 2,
    Tables 4-6): the solve converges with f non-increasing, and where the
    gradient vanishes every ALS mode solve returns its own factor, so the
    solution is a fixed point of the normalised ALS step."""
    lap = synth.laplacian_tensor(d, s)
    X = O.SparseTensor(lap.coords, lap.vals, lap.dims)
    u0 = synth.initial_guess(synth.rng_for(89), lap.dims, R)
    u, g, rep = O.cp_solve(X, u0, O.SolveOpts(R=R, tol=1e-10, maxit=3000))
    assert rep.converged
    fs = [h[0] for h in rep.history]
    assert all(b <= a * (1 + 1e-12) + 1e-14 for a, b in zip(fs, fs[1:]))
    v, _, _ = O.normalize(O.als_sweep(X, u, R), lap.dims, R)
    assert np.linalg.norm(v - u) <= 1e-9 * np.linalg.norm(u)


def test_ngmres_beats_als_on_collinear_problem():
    rng = synth.rng_for(95)
    prob = synth.dense_problem(rng, (15, 15, 15), 3, 0.9, paper_l1=1, paper_l2=1)
    X = O.DenseTensor(prob.T)
    u0 = synth.initial_guess(rng, prob.dims, 3)
    tol = 1e-9
    _, _, rep = O.cp_solve(X, u0, O.SolveOpts(R=3, tol=tol, maxit=3000))
    assert rep.converged
    u, _, _ = O.normalize(u0, prob.dims, 3)
    P = O.n_params(prob.dims, 3)
    als_it = 0
    while als_it < 3000:
        u, _, _ = O.normalize(O.als_sweep(X, u, 3), prob.dims, 3)
        als_it += 1
        if np.linalg.norm(O.fg(X, u, 3)[1]) / P < tol:
            break
    assert rep.iters < als_it
