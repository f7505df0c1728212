"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the bench.

This module only draws random numbers and assembles input tensors.  It holds
none of the CP method's arithmetic (no MTTKRP, no gradient, no ALS, no N-GMRES,
no line search).  Both sides of every parity test read the bytes produced here.

Generators (paper section / equation in brackets):

* ``collinear_factor`` -- a factor matrix whose columns have unit norm and
  pairwise cosine ``c`` [Section 3, Eq. collin, Test Problem I].  Entries are
  drawn N(0,1), orthonormalised by a thin QR with the sign of diag(R) fixed
  positive, then multiplied on the right by the upper Cholesky factor C of
  K = (1-c) I + c 11^T, so that (QC)^T (QC) = C^T C = K exactly.  When I < R
  no orthonormal basis exists; then the scaled Gaussian G / sqrt(I) is used and
  the collinearity holds only in expectation.
* ``dense_problem`` -- a planted rank-R tensor T_R = [[A1..AN]] (Eq. A) plus
  Gaussian noise scaled to a fraction eta of ||T_R||_F, or the paper's own
  two-level noise l1/l2 [Test Problem I], or the heteroscedastic variant.
* ``sparse_planted`` -- distinct uniform coordinates, values of a planted
  rank-R model with U(0,1) factors evaluated there, plus 1 % Gaussian noise.
* ``laplacian_tensor`` -- Test Problem II (Section 4): the 2d-way finite
  difference Laplacian tensor on an s^d grid, values 2d and -1.
* ``initial_guess`` -- N(0,1) factor entries, packed in the iterate layout.
* ``request_stream`` -- a Poisson stream of small dense 3-way requests.

Every generator takes a ``numpy.random.Generator``; ``rng_for`` makes the
seeded PCG64 one (seed = 11055331 + 100 * config + request_id).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 11055331


def rng_for(config: int, request_id: int = 0) -> np.random.Generator:
    """Seeded PCG64 generator for workload ``config`` and request ``request_id``."""
    return np.random.Generator(np.random.PCG64(BASE_SEED + 100 * int(config) + int(request_id)))


def collinearity_matrix(R: int, c: float) -> np.ndarray:
    """K with ones on the diagonal and ``c`` elsewhere (Test Problem I)."""
    return (1.0 - c) * np.eye(R) + c * np.ones((R, R))


def collinear_factor(rng: np.random.Generator, I: int, R: int, c: float) -> np.ndarray:
    """I x R factor with unit columns and pairwise cosine c (Eq. collin)."""
    G = rng.standard_normal((I, R))
    C = np.linalg.cholesky(collinearity_matrix(R, c)).T  # upper, C^T C = K
    if I >= R:
        Q, Rq = np.linalg.qr(G, mode="reduced")
        sgn = np.sign(np.diag(Rq))
        sgn[sgn == 0] = 1.0
        return (Q * sgn[None, :]) @ C
    return (G / np.sqrt(I)) @ C


def _outer_sum(factors: list[np.ndarray]) -> np.ndarray:
    """Dense tensor sum_r a_r^(1) o ... o a_r^(N) (the planted model, Eq. A)."""
    R = factors[0].shape[1]
    dims = [A.shape[0] for A in factors]
    # Build the first-mode-major Khatri-Rao product of all but the first factor
    # by repeated row-wise broadcasting, then one matrix product.
    right = factors[-1]
    for A in reversed(factors[1:-1]):
        right = (A[:, None, :] * right[None, :, :]).reshape(-1, R)
    full = factors[0] @ right.T
    return full.reshape(dims)


def planted_model_at(factors: list[np.ndarray], coords: np.ndarray) -> np.ndarray:
    """Values of the planted model sum_r prod_n A_n[coords[:, n], r] at given coordinates."""
    prod = np.ones((coords.shape[0], factors[0].shape[1]))
    for n, A in enumerate(factors):
        prod *= A[coords[:, n]]
    return prod.sum(axis=1)


@dataclass
class DenseProblem:
    T: np.ndarray                  # the data tensor (storage dtype)
    planted: list[np.ndarray]      # the planted factors (float64)
    dims: tuple
    R: int
    meta: dict = field(default_factory=dict)


def dense_problem(rng: np.random.Generator, dims, R: int, c: float, *, eta: float = 0.0,
                  hetero: float = 0.0, paper_l1: float | None = None, paper_l2: float | None = None,
                  dtype=np.float64) -> DenseProblem:
    """Planted rank-R dense tensor with collinearity c and noise.

    * ``eta``: T = T_R + eta ||T_R|| N / ||N||   (Gaussian noise at eta of ||T_R||_F)
    * ``hetero``: adds hetero ||T_R|| (N2 o sqrt(U)) / ||N2 o sqrt(U)||, U ~ U(0,1)
      (per-entry variance scaled by a uniform draw).
    * ``paper_l1``, ``paper_l2``: Test Problem I's two noise levels in percent.
    """
    dims = tuple(int(d) for d in dims)
    planted = [collinear_factor(rng, I, R, c) for I in dims]
    TR = _outer_sum(planted)
    nTR = np.linalg.norm(TR)
    T = TR.copy()
    if eta > 0:
        N1 = rng.standard_normal(dims)
        T += eta * nTR * N1 / np.linalg.norm(N1)
    if hetero > 0:
        N2 = rng.standard_normal(dims) * np.sqrt(rng.uniform(0.0, 1.0, dims))
        T += hetero * nTR * N2 / np.linalg.norm(N2)
    if paper_l1:
        N1 = rng.standard_normal(dims)
        T = T + (100.0 / paper_l1 - 1.0) ** -0.5 * nTR * N1 / np.linalg.norm(N1)
    if paper_l2:
        N2 = rng.standard_normal(dims) * T
        T = T + (100.0 / paper_l2 - 1.0) ** -0.5 * np.linalg.norm(T) * N2 / np.linalg.norm(N2)
    return DenseProblem(T=np.ascontiguousarray(T.astype(dtype)), planted=planted, dims=dims, R=R,
                        meta=dict(c=c, eta=eta, hetero=hetero, l1=paper_l1, l2=paper_l2))


def initial_guess(rng: np.random.Generator, dims, R: int) -> np.ndarray:
    """N(0,1) initial factors packed as u = [A1; ...; AN], each row-major I_n x R."""
    return np.concatenate([rng.standard_normal((int(I), R)).ravel() for I in dims])


@dataclass
class SparseProblem:
    coords: np.ndarray   # nnz x N int64, distinct, in sampled order
    vals: np.ndarray     # nnz float32
    dims: tuple
    R: int
    planted: list[np.ndarray] | None = None


def distinct_coords(rng: np.random.Generator, dims, nnz: int) -> np.ndarray:
    """``nnz`` distinct uniform int64 coordinates, kept in the order first sampled."""
    dims = np.asarray(dims, dtype=np.int64)
    total = int(np.prod(dims.astype(object)))
    if nnz > total:
        raise ValueError("more nonzeros than entries")
    have = np.empty((0, len(dims)), dtype=np.int64)
    while have.shape[0] < nnz:
        need = nnz - have.shape[0]
        draw = np.stack([rng.integers(0, d, size=max(need + need // 8, 16), dtype=np.int64)
                         for d in dims], axis=1)
        cand = np.concatenate([have, draw], axis=0)
        # Linearised key (exact in int64 only when the index space fits; fall back to rows).
        _, first = np.unique(cand, axis=0, return_index=True)
        keep = np.sort(first)
        have = cand[keep][:nnz]
    return np.ascontiguousarray(have[:nnz])


def sparse_planted(rng: np.random.Generator, dims, nnz: int, R: int, noise: float = 0.01) -> SparseProblem:
    """Sparse COO tensor: planted rank-R model (U(0,1) factors) at distinct
    uniform coordinates, plus ``noise`` * ||m|| * n / ||n|| Gaussian noise; FP32 values."""
    coords = distinct_coords(rng, dims, nnz)
    planted = [rng.uniform(0.0, 1.0, (int(I), R)) for I in dims]
    m = planted_model_at(planted, coords)
    n = rng.standard_normal(nnz)
    v = m + noise * np.linalg.norm(m) * n / np.linalg.norm(n)
    return SparseProblem(coords=coords, vals=v.astype(np.float32), dims=tuple(int(d) for d in dims),
                         R=R, planted=planted)


def laplacian_tensor(d: int, s: int) -> SparseProblem:
    """Test Problem II: the finite-difference Laplacian on an s^d grid as a
    2d-way sparse tensor of size s x ... x s.  Entry (p, p) = 2d, and
    (p, p +- e_k) = -1 for grid neighbours inside the grid."""
    grid = np.stack(np.meshgrid(*[np.arange(s)] * d, indexing="ij"), axis=-1).reshape(-1, d)
    rows = [np.concatenate([grid, grid], axis=1)]
    vals = [np.full(grid.shape[0], 2.0 * d)]
    for k in range(d):
        for step in (-1, 1):
            nb = grid.copy()
            nb[:, k] += step
            ok = (nb[:, k] >= 0) & (nb[:, k] < s)
            rows.append(np.concatenate([grid[ok], nb[ok]], axis=1))
            vals.append(np.full(int(ok.sum()), -1.0))
    coords = np.concatenate(rows, axis=0).astype(np.int64)
    return SparseProblem(coords=np.ascontiguousarray(coords), vals=np.concatenate(vals).astype(np.float32),
                         dims=(s,) * (2 * d), R=0)


@dataclass
class Request:
    request_id: int
    arrival_s: float
    dims: tuple
    R: int
    c: float
    eta: float
    tol: float


def request_stream(n_requests: int, rate_per_s: float = 200.0, config: int = 5,
                   side_range=(16, 192), rank_range=(2, 32)) -> list[Request]:
    """Poisson arrivals of small dense 3-way requests with random shapes,
    ranks, collinearity, noise and tolerance (parameters only; tensors are
    built per request with ``rng_for(config, request_id)``)."""
    rng = rng_for(config, 0)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for k in range(n_requests):
        dims = tuple(int(x) for x in rng.integers(side_range[0], side_range[1] + 1, size=3))
        R = int(rng.integers(rank_range[0], rank_range[1] + 1))
        c = float(rng.choice([0.5, 0.9]))
        eta = float(rng.uniform(0.01, 0.10))
        tol = float(rng.choice([1e-5, 1e-7]))
        out.append(Request(k + 1, float(t[k]), dims, R, c, eta, tol))
    return out


def request_problem(req: Request, config: int = 5, dtype=np.float32):
    """Tensor and initial guess of one streamed request."""
    rng = rng_for(config, req.request_id)
    prob = dense_problem(rng, req.dims, req.R, req.c, eta=req.eta, dtype=dtype)
    u0 = initial_guess(rng, req.dims, req.R)
    return prob, u0


# The five named workloads -------------------------------------------------

def workload_dense_small():
    """20x20x20 FP64, R=3, c=0.5, 10 % noise, N(0,1) start."""
    rng = rng_for(1)
    prob = dense_problem(rng, (20, 20, 20), 3, 0.5, eta=0.10, dtype=np.float64)
    return prob, initial_guess(rng, prob.dims, 3)


def workload_dense_256(dims=(256, 256, 256), R=16):
    """256^3 FP32, R=16, c=0.9, 10 % homoscedastic + 10 % heteroscedastic noise."""
    rng = rng_for(2)
    prob = dense_problem(rng, dims, R, 0.9, eta=0.10, hetero=0.10, dtype=np.float32)
    return prob, initial_guess(rng, prob.dims, R)


def workload_dense_4way(dims=(96, 96, 96, 96), R=32):
    """96^4 FP32, R=32, c=0.5, 5 % noise."""
    rng = rng_for(3)
    prob = dense_problem(rng, dims, R, 0.5, eta=0.05, dtype=np.float32)
    return prob, initial_guess(rng, prob.dims, R)


def workload_sparse(dims=(20000, 20000, 20000), nnz=2_000_000, R=10):
    """Sparse 20000^3 COO, 2e6 distinct nonzeros, planted rank 10 + 1 % noise."""
    rng = rng_for(4)
    prob = sparse_planted(rng, dims, nnz, R, noise=0.01)
    return prob, initial_guess(rng, prob.dims, R)
