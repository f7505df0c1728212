"""Plain, slow, FP64 CPU oracle for N-GMRES-accelerated ALS (De Sterck, arXiv 1105.5331).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module: it is
called by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py`` and nowhere else.  It shares no code with the CUDA path.

Every function restates one passage of the paper in numpy, FP64 throughout,
with library primitives (einsum, matmul, Cholesky, triangular solve, stable
sort) as single steps and no blocking or reordering beyond the definitions.

Iterate layout: u = [A^(1); ...; A^(N)] with each factor row-major I_n x R.

Readings where the paper is silent (the same readings are used by the CUDA path):
  R1  MTTKRP is the index sum M[i,r] = sum over all other indices of
      T[...] * prod_{m != n} A^(m)[i_m, r]; this is T_(n) Phibar^(n) for any
      consistent matricisation (Eq. Phi, Eq. Gn).
  R2  The ALS mode solve uses a Cholesky factorisation of Gammabar^(n).  If it
      fails, one retry with Gammabar + 1e-12 * trace / R * I; then an error.
  R3  Normalisation: a rank-one term with a zero column has lambda_r = 0 and is
      left unscaled.
  R4  Terms are reordered by a stable sort on decreasing lambda (ties keep the
      lower index).  lambda^(1/N) is computed with pow.
  R5  The initial guess is normalised before its gradient is taken.
  R6  The accelerated iterate uhat is normalised before the line search.
  R7  Restart when s = g(ubar)^T (uhat - ubar) >= 0: no line search,
      u_{i+1} = ubar and the window is reset to {(ubar, g(ubar))}.
  R8  The gradient of a normalised iterate is obtained by rescaling column r of
      G^(n) by 1/s_{n,r} (and permuting alike); this is exact because
      prod_n s_{n,r} = 1 (follows from Eq. Gn).
  R9  Stop when ||g(u_i)||_2 / P < tol, P = R * sum_n I_n.
  R10 Line search: More-Thuente with ftol 1e-4, gtol 1e-2, first step 1 and at
      most 20 evaluations (Section 2.4); xtol 1e-15, stpmin 1e-15, stpmax 1e15.
      When it stops without meeting both Wolfe conditions, its last point is
      kept if it meets the sufficient-decrease condition, otherwise beta = 0.
  R11 The normal equations (P^T P + delta I) alpha = -P^T g(ubar) are solved by
      Cholesky, delta = 1e-12 * max diag(P^T P); if P^T P = 0, alpha = 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

# ---------------------------------------------------------------------------
# Iterate layout (Section 2.3: factor matrices stacked into the iterate u)
# ---------------------------------------------------------------------------


def n_params(dims, R: int) -> int:
    return int(R * sum(int(d) for d in dims))


def unpack(u: np.ndarray, dims, R: int) -> list[np.ndarray]:
    """Views A^(n) (I_n x R, row-major) into the packed iterate u."""
    out, off = [], 0
    for I in dims:
        I = int(I)
        out.append(u[off:off + I * R].reshape(I, R))
        off += I * R
    return out


def pack(factors) -> np.ndarray:
    return np.concatenate([np.asarray(A, dtype=np.float64).ravel() for A in factors])


# ---------------------------------------------------------------------------
# Eq. (A), Eq. (fA): the CP model and the objective by brute force
# ---------------------------------------------------------------------------


def cp_full(factors) -> np.ndarray:
    """A_R = sum_r a_r^(1) o ... o a_r^(N) as a dense array (Eq. A)."""
    N = len(factors)
    letters = "abcdefghijklmnopqrstuvwxy"[:N]
    expr = ",".join(ch + "z" for ch in letters) + "->" + letters
    return np.einsum(expr, *factors)


def f_bruteforce(T: np.ndarray, factors) -> float:
    """f = 1/2 ||T - A_R||_F^2 evaluated entry by entry (Eq. fA)."""
    D = np.asarray(T, dtype=np.float64) - cp_full(factors)
    return 0.5 * float(np.sum(D * D))


# ---------------------------------------------------------------------------
# MTTKRP  M^(n) = T_(n) Phibar^(n)   (Eq. Gn, Eq. Phi; reading R1)
# ---------------------------------------------------------------------------


def mttkrp_dense(T: np.ndarray, factors, n: int) -> np.ndarray:
    """M[i,r] = sum_{i_m, m != n} T[i_1..i_N] prod_{m != n} A^(m)[i_m, r]."""
    N = T.ndim
    letters = "abcdefghijklmnopqrstuvwxy"[:N]
    others = [m for m in range(N) if m != n]
    expr = letters + "," + ",".join(letters[m] + "z" for m in others) + "->" + letters[n] + "z"
    return np.einsum(expr, np.asarray(T, dtype=np.float64), *[factors[m] for m in others])


def mttkrp_sparse(coords: np.ndarray, vals: np.ndarray, dims, factors, n: int) -> np.ndarray:
    """The same index sum over the nonzeros only (T is zero elsewhere)."""
    R = factors[0].shape[1]
    w = np.asarray(vals, dtype=np.float64)[:, None] * np.ones((1, R))
    for m in range(len(dims)):
        if m != n:
            w = w * factors[m][coords[:, m]]
    M = np.zeros((int(dims[n]), R))
    np.add.at(M, coords[:, n], w)
    return M


# ---------------------------------------------------------------------------
# Gram-Hadamard matrices (Eq. Gamma)
# ---------------------------------------------------------------------------


def grams(factors) -> list[np.ndarray]:
    return [A.T @ A for A in factors]


def gamma_all(factors) -> np.ndarray:
    """Gamma = (A1^T A1) * ... * (AN^T AN), * elementwise."""
    out = np.ones((factors[0].shape[1],) * 2)
    for G in grams(factors):
        out = out * G
    return out


def gamma_bar(factors, n: int) -> np.ndarray:
    """Gammabar^(n): the same Hadamard product without mode n."""
    out = np.ones((factors[0].shape[1],) * 2)
    for m, A in enumerate(factors):
        if m != n:
            out = out * (A.T @ A)
    return out


# ---------------------------------------------------------------------------
# Objective and gradient (Eq. fA expanded, Eq. Gn)
# ---------------------------------------------------------------------------


class DenseTensor:
    """A dense data tensor with its squared norm (oracle side)."""

    def __init__(self, T: np.ndarray):
        self.T = np.asarray(T, dtype=np.float64)
        self.dims = self.T.shape
        self.norm2 = float(np.sum(self.T * self.T))

    def mttkrp(self, factors, n):
        return mttkrp_dense(self.T, factors, n)


class SparseTensor:
    """A COO data tensor with its squared norm (oracle side)."""

    def __init__(self, coords: np.ndarray, vals: np.ndarray, dims):
        self.coords = np.asarray(coords, dtype=np.int64)
        self.vals = np.asarray(vals, dtype=np.float64)
        self.dims = tuple(int(d) for d in dims)
        self.norm2 = float(np.sum(self.vals * self.vals))

    def mttkrp(self, factors, n):
        return mttkrp_sparse(self.coords, self.vals, self.dims, factors, n)


def fg(X, u: np.ndarray, R: int):
    """f(u) and g(u).

    f = 1/2 (||T||^2 - 2 <T, A_R> + ||A_R||^2) with <T, A_R> = sum_{i,r}
    A^(N)[i,r] M^(N)[i,r] and ||A_R||^2 = sum_{r,s} Gamma[r,s]   (Eq. fA);
    G^(n) = -M^(n) + A^(n) Gammabar^(n)                              (Eq. Gn).
    """
    factors = unpack(u, X.dims, R)
    N = len(factors)
    Ms = [X.mttkrp(factors, n) for n in range(N)]
    inner = float(np.sum(factors[N - 1] * Ms[N - 1]))
    model2 = float(np.sum(gamma_all(factors)))
    f = 0.5 * (X.norm2 - 2.0 * inner + model2)
    g = pack([-Ms[n] + factors[n] @ gamma_bar(factors, n) for n in range(N)])
    return f, g


# ---------------------------------------------------------------------------
# ALS (Section 2.3: block nonlinear Gauss-Seidel on G^(n) = 0)
# ---------------------------------------------------------------------------


class NotSPD(RuntimeError):
    pass


def _cholesky_lower(S: np.ndarray) -> np.ndarray:
    """Plain Cholesky S = L L^T (reading R2: one ridge retry)."""
    try:
        return np.linalg.cholesky(S)
    except np.linalg.LinAlgError:
        R = S.shape[0]
        ridge = 1e-12 * np.trace(S) / R
        try:
            return np.linalg.cholesky(S + ridge * np.eye(R))
        except np.linalg.LinAlgError as exc:
            raise NotSPD(str(exc)) from exc


def als_mode_solve(M: np.ndarray, Gb: np.ndarray) -> np.ndarray:
    """A^(n) = M Gammabar^-1: solve Gammabar X^T = M^T with Gammabar = L L^T."""
    L = _cholesky_lower(Gb)
    Y = solve_triangular(L, M.T, lower=True)
    return solve_triangular(L.T, Y, lower=False).T


def als_sweep(X, u: np.ndarray, R: int) -> np.ndarray:
    """One ALS iteration M(u): for n = 1..N solve G^(n) = 0 for A^(n) with the
    factors of modes < n already updated (Eq. foopt)."""
    factors = [A.copy() for A in unpack(np.array(u, dtype=np.float64), X.dims, R)]
    for n in range(len(factors)):
        M = X.mttkrp(factors, n)
        factors[n] = als_mode_solve(M, gamma_bar(factors, n))
    return pack(factors)


# ---------------------------------------------------------------------------
# Normalisation and reordering (Section 2.3; readings R3, R4, R8)
# ---------------------------------------------------------------------------


def normalize(u: np.ndarray, dims, R: int, g: np.ndarray | None = None):
    """Unit-normalise every column, give each mode lambda_r^(1/N), order terms
    by decreasing lambda_r.  Returns (u', g' or None, lambda sorted)."""
    factors = [A.copy() for A in unpack(np.array(u, dtype=np.float64), dims, R)]
    grads = None if g is None else [G.copy() for G in unpack(np.array(g, dtype=np.float64), dims, R)]
    N = len(factors)
    nu = np.stack([np.sqrt(np.sum(A * A, axis=0)) for A in factors])  # N x R
    lam = np.prod(nu, axis=0)
    for r in range(R):
        if np.any(nu[:, r] == 0.0):
            lam[r] = 0.0
            continue
        root = pow(float(lam[r]), 1.0 / N)
        for n in range(N):
            s = root / nu[n, r]
            factors[n][:, r] *= s
            if grads is not None:
                grads[n][:, r] /= s
    order = np.argsort(-lam, kind="stable")
    factors = [A[:, order] for A in factors]
    u2 = pack(factors)
    g2 = None if grads is None else pack([G[:, order] for G in grads])
    return u2, g2, lam[order]


# ---------------------------------------------------------------------------
# N-GMRES Step II (Eq. accel, Eq. linearize, Eq. normal; delta I of Section 2.1)
# ---------------------------------------------------------------------------


def ngmres_step(U: np.ndarray, G: np.ndarray, ubar: np.ndarray, gbar: np.ndarray, eps: float = 1e-12):
    """Accelerated iterate from a window of m previous iterates.

    U, G: m x P (rows u_j and g(u_j), oldest first).  p_j = g(ubar) - g(u_j),
    (P^T P + delta I) alpha = -P^T g(ubar), delta = eps * max diag(P^T P),
    uhat = ubar + sum_j alpha_j (ubar - u_j).  Returns (uhat, alpha).
    """
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    G = np.atleast_2d(np.asarray(G, dtype=np.float64))
    Pm = gbar[None, :] - G                  # rows are p_j
    H = Pm @ Pm.T
    rhs = -(Pm @ gbar)
    dmax = float(np.max(np.diag(H)))
    if dmax == 0.0:
        alpha = np.zeros(U.shape[0])
    else:
        L = np.linalg.cholesky(H + eps * dmax * np.eye(H.shape[0]))
        alpha = solve_triangular(L.T, solve_triangular(L, rhs, lower=True), lower=False)
    uhat = ubar + (alpha[:, None] * (ubar[None, :] - U)).sum(axis=0)
    return uhat, alpha


# ---------------------------------------------------------------------------
# More-Thuente line search (Step III; Section 2.4 parameters; the method of
# J. J. More and D. J. Thuente, ACM TOMS 20(3):286-307, 1994)
# ---------------------------------------------------------------------------


@dataclass
class LSOpts:
    ftol: float = 1e-4     # sufficient decrease parameter mu
    gtol: float = 1e-2     # curvature parameter eta
    xtol: float = 1e-15    # relative width of the interval of uncertainty
    stpmin: float = 1e-15
    stpmax: float = 1e15
    stp0: float = 1.0
    maxfev: int = 20


def _cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic interpolating f and f' at a and b, or None if the
    cubic has no real local minimiser (textbook interpolation formula)."""
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = np.copysign(np.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def _quad_min(a, fa, da, b, fb):
    """Minimiser of the quadratic through f(a), f'(a), f(b)."""
    h = b - a
    den = 2.0 * (fb - fa - da * h)
    if den == 0.0:
        return None
    return a - da * h * h / den


def _secant_min(a, da, b, db):
    """Minimiser of the quadratic through f'(a), f'(b)."""
    if db == da:
        return None
    return b - db * (b - a) / (db - da)


def mt_trial(lo, hi, t, brackt, stmin, stmax):
    """Trial value selection and interval update of More-Thuente (Section 4 of
    their paper): lo = (a_l, f_l, g_l) best point, hi = (a_u, f_u, g_u) other
    endpoint, t = (a_t, f_t, g_t) the newest trial.  Returns (lo, hi, a_next, brackt)."""
    al, fl, gl = lo
    au, fu, gu = hi
    at, ft, gt = t
    if ft > fl:
        # Case 1: higher function value -> the minimum is bracketed.
        ac = _cubic_min(al, fl, gl, at, ft, gt)
        aq = _quad_min(al, fl, gl, at, ft)
        if ac is None:
            ac = aq
        if aq is None:
            aq = ac
        if ac is None:
            nxt = al + 0.5 * (at - al)
        else:
            nxt = ac if abs(ac - al) < abs(aq - al) else ac + 0.5 * (aq - ac)
        brackt = True
    elif gt * gl < 0.0:
        # Case 2: lower value, derivatives of opposite sign -> bracketed.
        ac = _cubic_min(al, fl, gl, at, ft, gt)
        asec = _secant_min(al, gl, at, gt)
        if ac is None:
            ac = asec
        if asec is None:
            asec = ac
        if ac is None:
            nxt = al + 0.5 * (at - al)
        else:
            nxt = ac if abs(ac - at) >= abs(asec - at) else asec
        brackt = True
    elif abs(gt) <= abs(gl):
        # Case 3: lower value, same sign, derivative magnitude decreases.
        ac = _cubic_min(al, fl, gl, at, ft, gt)
        forward = (at - al)
        if ac is None or (ac - at) * forward <= 0.0:
            ac = stmax if at > al else stmin
        asec = _secant_min(al, gl, at, gt)
        if asec is None:
            asec = ac
        if brackt:
            nxt = ac if abs(ac - at) < abs(asec - at) else asec
            if at > al:
                nxt = min(at + 0.66 * (au - at), nxt)
            else:
                nxt = max(at + 0.66 * (au - at), nxt)
        else:
            nxt = ac if abs(ac - at) > abs(asec - at) else asec
            nxt = min(stmax, max(stmin, nxt))
    else:
        # Case 4: lower value, same sign, derivative magnitude does not decrease.
        if brackt:
            ac = _cubic_min(at, ft, gt, au, fu, gu)
            nxt = ac if ac is not None else at + 0.5 * (au - at)
        else:
            nxt = stmax if at > al else stmin
    # Updating rules U1-U3.
    if ft > fl:
        hi = t
    else:
        if gt * (al - at) < 0.0:
            hi = lo
        lo = t
    return lo, hi, nxt, brackt


def more_thuente(phi, f0: float, g0: float, opts: LSOpts = LSOpts()):
    """Search for beta with phi(beta) <= phi(0) + ftol beta phi'(0) and
    |phi'(beta)| <= gtol |phi'(0)|.  ``phi(beta)`` returns (value, derivative, extra).

    Stage 1 works on psi(a) = phi(a) - phi(0) - ftol a phi'(0) until a point
    with psi <= 0 and phi' >= min(ftol, gtol) phi'(0) is seen; then phi itself.
    Unbracketed trials extrapolate into [a_t + 1.1 (a_t - a_l), a_t + 4 (a_t - a_l)];
    bracketed intervals that fail to shrink by 0.66 over two trials are bisected.

    Returns (beta, value, derivative, extra, nfev, info); info 1 = both
    conditions met, 2 = interval below xtol, 3 = maxfev, 4 = at stpmin,
    5 = at stpmax, 6 = rounding prevents progress, -1 = not a descent direction.
    """
    if not (g0 < 0.0):
        return 0.0, f0, g0, None, 0, -1
    ftol, gtol, xtol = opts.ftol, opts.gtol, opts.xtol
    lo = (0.0, f0, g0)          # best point so far (a_l)
    hi = (0.0, f0, g0)          # other endpoint (a_u)
    brackt = False
    stage = 1
    width = opts.stpmax - opts.stpmin
    width1 = 2.0 * width
    stp = min(max(opts.stp0, opts.stpmin), opts.stpmax)
    imin, imax = 0.0, stp + 4.0 * stp   # allowed range when stp was chosen
    nfev = 0
    while True:
        f, g, extra = phi(stp)
        nfev += 1
        ftest = f0 + stp * ftol * g0
        info = 0
        if brackt and (stp <= imin or stp >= imax):
            info = 6
        if brackt and imax - imin <= xtol * imax:
            info = 2
        if stp == opts.stpmax and f <= ftest and g <= ftol * g0:
            info = 5
        if stp == opts.stpmin and (f > ftest or g >= ftol * g0):
            info = 4
        if nfev >= opts.maxfev:
            info = 3
        if f <= ftest and abs(g) <= gtol * (-g0):
            info = 1
        if info:
            return stp, f, g, extra, nfev, info
        if stage == 1 and f <= ftest and g >= min(ftol, gtol) * g0:
            stage = 2
        t = (stp, f, g)
        xlo = stp + 1.1 * (stp - lo[0])
        xhi = stp + 4.0 * (stp - lo[0])
        if stage == 1 and f <= lo[1] and f > ftest:
            def psi(p):
                return (p[0], p[1] - f0 - p[0] * ftol * g0, p[2] - ftol * g0)
            lo_m, hi_m, stp, brackt = mt_trial(psi(lo), psi(hi), psi(t), brackt, xlo, xhi)
            lo = (lo_m[0], lo_m[1] + f0 + lo_m[0] * ftol * g0, lo_m[2] + ftol * g0)
            hi = (hi_m[0], hi_m[1] + f0 + hi_m[0] * ftol * g0, hi_m[2] + ftol * g0)
        else:
            lo, hi, stp, brackt = mt_trial(lo, hi, t, brackt, xlo, xhi)
        if brackt:
            if abs(hi[0] - lo[0]) >= 0.66 * width1:
                stp = lo[0] + 0.5 * (hi[0] - lo[0])
            width1 = width
            width = abs(hi[0] - lo[0])
            imin, imax = min(lo[0], hi[0]), max(lo[0], hi[0])
        else:
            imin, imax = xlo, xhi
        stp = min(max(stp, opts.stpmin), opts.stpmax)
        if brackt and (stp <= imin or stp >= imax or imax - imin <= xtol * imax):
            stp = lo[0]


# ---------------------------------------------------------------------------
# The N-GMRES optimisation algorithm (Algorithm 1, Steps I-III, Section 2.1)
# ---------------------------------------------------------------------------


@dataclass
class SolveOpts:
    R: int
    w: int = 20
    tol: float = 1e-7
    maxit: int = 10000
    eps: float = 1e-12
    ls: LSOpts = field(default_factory=LSOpts)


@dataclass
class SolveReport:
    iters: int = 0
    fg_evals: int = 0
    als_sweeps: int = 0
    restarts: int = 0
    ls_failures: int = 0
    f: float = float("nan")
    gnorm_over_P: float = float("nan")
    converged: bool = False
    history: list = field(default_factory=list)


def cp_solve(X, u0: np.ndarray, opts: SolveOpts, max_iters: int | None = None):
    """N-GMRES accelerated ALS (Algorithm 1) with windowed start-up (Section 2.1)
    and the readings R5-R11.  Returns (u, g, report)."""
    R, dims = opts.R, X.dims
    P = n_params(dims, R)
    rep = SolveReport()
    u, _, _ = normalize(u0, dims, R)                       # R5
    f, g = fg(X, u, R)
    rep.fg_evals += 1
    Wu, Wg = [u], [g]
    limit = opts.maxit if max_iters is None else min(opts.maxit, max_iters)
    while True:
        gn = float(np.linalg.norm(g)) / P
        rep.history.append((f, gn))
        if gn < opts.tol:                                   # R9
            rep.converged = True
            break
        if rep.iters >= limit:
            break
        # Step I: preliminary iterate by one ALS sweep, normalised.
        ubar, _, _ = normalize(als_sweep(X, u, R), dims, R)
        rep.als_sweeps += 1
        fbar, gbar = fg(X, ubar, R)
        rep.fg_evals += 1
        # Step II: accelerated iterate from the window.
        uhat, _ = ngmres_step(np.array(Wu), np.array(Wg), ubar, gbar, opts.eps)
        uhat, _, _ = normalize(uhat, dims, R)               # R6
        d = uhat - ubar
        s = float(gbar @ d)
        if s >= 0.0:                                        # R7: restart
            rep.restarts += 1
            u, f, g = ubar, fbar, gbar
            Wu, Wg = [u], [g]
        else:
            # Step III: line search on f(ubar + beta d), beta >= 0.
            def phi(beta):
                x = ubar + beta * d
                fx, gx = fg(X, x, R)
                return fx, float(gx @ d), (x, gx)
            beta, fb, _, extra, nfev, info = more_thuente(phi, fbar, s, opts.ls)
            rep.fg_evals += nfev
            if info != 1:
                rep.ls_failures += 1
            if info == 1 or (extra is not None and fb <= fbar + opts.ls.ftol * beta * s):
                x, gx = extra
                u, g, _ = normalize(x, dims, R, gx)        # R8
                f = fb
            else:                                           # R10: beta = 0
                u, f, g = ubar, fbar, gbar
            Wu.append(u)
            Wg.append(g)
            if len(Wu) > opts.w:
                Wu.pop(0)
                Wg.pop(0)
        rep.iters += 1
    rep.f = f
    rep.gnorm_over_P = float(np.linalg.norm(g)) / P
    return u, g, rep


# ---------------------------------------------------------------------------
# Mode sort and segmentation of a COO tensor (bit-exact reference)
# ---------------------------------------------------------------------------


def coo_sort_mode(coords: np.ndarray, n: int):
    """Permutation that stably sorts the nonzeros by the cyclic key
    (i_n, i_{n+1}, ..., i_N, i_1, ..., i_{n-1}), and the segment pointers of
    runs of equal i_n.  Returns (perm int64, seg_ptr int64, seg_row int64)."""
    N = coords.shape[1]
    key_modes = [(n + k) % N for k in range(N)]
    # np.lexsort sorts by the LAST key first; it is a stable sort.
    perm = np.lexsort(tuple(coords[:, m] for m in reversed(key_modes))).astype(np.int64)
    rows = coords[perm, n]
    if rows.size == 0:
        return perm, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int64)
    starts = np.flatnonzero(np.concatenate([[True], rows[1:] != rows[:-1]]))
    seg_ptr = np.concatenate([starts, [rows.size]]).astype(np.int64)
    return perm, seg_ptr, rows[starts].astype(np.int64)
