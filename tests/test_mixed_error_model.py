"""Where the stated bound of the mixed-precision MTTKRP comes from, checked on
the CPU on the inputs of the GPU parity tests (no GPU code involved).

The tensor-core path computes every product a b of a tensor entry a and a
Khatri-Rao entry b (FP32 products of FP32 factor copies) from bf16 splits
x = x_h + x_l + r_x, x_h = bf16(x), x_l = bf16(x - x_h), as
a_h b_h + a_h b_l + a_l b_h, each bf16 product exact in FP32.  With u = 2^-8
(bf16 round to nearest): |x_l| <= (1 + u) u |x| and |r_x| <= u^2 |x|, so the
dropped part a_l b_l + r_a (b_h + b_l) + r_b (a_h + a_l) + r_a r_b is at most
3.01 u^2 |a b|.  The FP32 copies add (2N - 2) 2^-24 relative to each product.
Elementwise, |dM| <= (3.01 * 2^-16 + (2N - 2) 2^-24) (|T_(n)| |Phibar|).

The split errors of different products have independent signs, so relative
to ||M|| (where the terms of M cancel) they add up to about 2^-17.5 ~ 5e-6,
whatever the contraction length.  The GPU tests hold the mixed MTTKRP to a
relative Frobenius error of 5e-5: this model of the split arithmetic (sums in
FP64, or in FP32 as a stand-in for the FP32 accumulation) stays at least five
times inside it on every one of those inputs."""
import numpy as np
import pytest

import synth
from oracle import cp_oracle as O

STATED = 5e-5            # the GPU tests' bound (relative Frobenius)
U2 = 2.0 ** -16


def bf16(x):
    """Round FP32 values to bf16 (round to nearest even), returned as FP32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = bf16(x)
    return hi, bf16((x - hi).astype(np.float32))


def khatri_rao_fp32(F, others):
    """Rows in matricisation order (last listed mode fastest), products in FP32."""
    B = np.ones((1, F[0].shape[1]), dtype=np.float32)
    for m in others:
        A = F[m].astype(np.float32)
        B = (B[:, None, :] * A[None, :, :]).reshape(-1, A.shape[1]).astype(np.float32)
    return B


def model_errors(T, F, n):
    N = T.ndim
    others = [m for m in range(N) if m != n]
    Tn = np.moveaxis(T.astype(np.float32), n, 0).reshape(T.shape[n], -1)
    B = khatri_rao_fp32(F, others)
    (th, tl), (bh, bl) = split(Tn), split(B)
    th64, tl64, bh64, bl64 = (a.astype(np.float64) for a in (th, tl, bh, bl))
    m64 = th64 @ bh64 + th64 @ bl64 + tl64 @ bh64
    m32 = (th @ bh) + (th @ bl) + (tl @ bh)
    ref = O.mttkrp_dense(T.astype(np.float64), F, n)
    scale = np.abs(Tn.astype(np.float64)) @ np.abs(B.astype(np.float64))
    coef = 3.01 * U2 + (2 * N - 2) * 2.0 ** -24
    nref = np.linalg.norm(ref)
    return (np.max(np.abs(m64 - ref) - coef * scale),
            np.linalg.norm(m64 - ref) / nref, np.linalg.norm(m32.astype(np.float64) - ref) / nref)


# the shapes, ranks, dtypes and seeds of the GPU parity test of the mixed MTTKRP
PARITY_SHAPES = [
    ((20, 20, 20), 3, np.float64),
    ((7, 5, 3), 1, np.float32),
    ((130, 33, 17), 16, np.float32),
    ((96, 40, 30, 5), 32, np.float32),
    ((300, 20, 9), 20, np.float32),
    ((64, 64, 64), 48, np.float32),
    ((17, 256, 12), 64, np.float32),
]


@pytest.mark.parametrize("shape,R,dtype", PARITY_SHAPES)
def test_split_products_within_the_derived_bounds(shape, R, dtype):
    rng = np.random.default_rng(R)
    T = rng.standard_normal(shape).astype(dtype)
    u = synth.initial_guess(rng, shape, R)
    F = O.unpack(u, shape, R)
    for n in range(len(shape)):
        excess, rel64, rel32 = model_errors(T, F, n)
        assert excess <= 1e-12, (shape, n, excess)
        assert rel64 <= STATED / 5 and rel32 <= STATED / 5, (shape, n, rel64, rel32)


@pytest.mark.slow
def test_split_products_on_the_dense_256_workload():
    prob, u0 = synth.workload_dense_256()
    F = O.unpack(u0, prob.dims, 16)
    for n in range(3):
        excess, rel64, rel32 = model_errors(prob.T, F, n)
        assert excess <= 1e-9, (n, excess)
        assert rel64 <= STATED / 5 and rel32 <= STATED / 5, (n, rel64, rel32)
