"""The MTTKRP entry point that allocates no device memory.

Some callers cannot allocate device memory while they run: code that enqueues
work inside a stream capture it does not own, serving loops with a fixed
memory budget in which cudaMalloc may stall or fail, or programs whose device
memory is owned by another allocator.  cp_mttkrp_noalloc uses a fixed scratch
array inside the library instead.  This test calls it through the C ABI and
compares it with cp_mttkrp, twice in a row, so that leftovers of the first call
in the shared scratch cannot go unnoticed.  It lives in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import cp_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the FP64 parity tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1105_5331_gb300 as cp
    return cp


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,R,dtype", [((96, 80, 70), 16, np.float32), ((20, 20, 20), 3, np.float64),
                                           ((13, 9, 11, 20), 7, np.float32)])
def test_noalloc_matches_cp_mttkrp_twice(cp, shape, R, dtype):
    ctx = cp.cp_ctx_create(0, torch.cuda.current_stream())
    rng = np.random.default_rng(sum(shape) + R)
    T = rng.standard_normal(shape).astype(dtype)
    u = torch.from_numpy(synth.initial_guess(rng, shape, R)).cuda()
    t = cp.cp_tensor_dense(ctx, torch.from_numpy(T).cuda())
    for call in range(2):
        # second call: another mode first, so the scratch holds other data
        for n in (range(len(shape)) if call == 0 else reversed(range(len(shape)))):
            ref = torch.empty(shape[n] * R, dtype=torch.float64, device="cuda")
            got = torch.full_like(ref, float("nan"))
            cp.cp_mttkrp(ctx, t, R, u, n, ref)
            cp.cp_mttkrp_noalloc(ctx, t, R, u, n, got)
            cp.cp_ctx_sync(ctx)
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            assert rel(a, b) <= TOL, (call, n)
            oracle = O.mttkrp_dense(T.astype(np.float64), O.unpack(u.cpu().numpy(), shape, R), n)
            assert rel(a, oracle.ravel()) <= TOL
    t.close()
    ctx.close()


def test_noalloc_fewer_ctas_when_the_scratch_is_the_limit(cp):
    """4000 rows at R = 64 make one partial block 2 048 000 bytes, so only
    four blocks fit the 8 MiB scratch: the split-K grid shrinks to four CTAs,
    each taking a quarter of the contraction, instead of two per SM."""
    ctx = cp.cp_ctx_create(0, torch.cuda.current_stream())
    shape, R = (4000, 40, 40), 64
    assert (8 << 20) // (shape[0] * R * 8) == 4
    rng = np.random.default_rng(4000)
    T = rng.standard_normal(shape).astype(np.float32)
    u = torch.from_numpy(synth.initial_guess(rng, shape, R)).cuda()
    t = cp.cp_tensor_dense(ctx, torch.from_numpy(T).cuda())
    oracle = O.mttkrp_dense(T.astype(np.float64), O.unpack(u.cpu().numpy(), shape, R), 0).ravel()
    for call in range(2):
        ref = torch.empty(shape[0] * R, dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        cp.cp_mttkrp(ctx, t, R, u, 0, ref)
        cp.cp_mttkrp_noalloc(ctx, t, R, u, 0, got)
        cp.cp_ctx_sync(ctx)
        a = got.cpu().numpy()
        assert rel(a, ref.cpu().numpy()) <= TOL, call
        assert rel(a, oracle) <= TOL, call
    t.close()
    ctx.close()


def test_noalloc_rejects_rows_beyond_the_scratch(cp):
    ctx = cp.cp_ctx_create(0, torch.cuda.current_stream())
    # one partial block of I x R doubles must fit in the 8 MiB scratch
    shape, R = (20000, 2, 2), 64
    t = cp.cp_tensor_dense(ctx, torch.zeros(shape, dtype=torch.float32, device="cuda"))
    u = torch.zeros(sum(shape) * R, dtype=torch.float64, device="cuda")
    out = torch.empty(20000 * R, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CpError) as ei:
        cp.cp_mttkrp_noalloc(ctx, t, R, u, 0, out)
    assert ei.value.status == 2
    assert "scratch" in cp.cp_last_error()
    t.close()
    ctx.close()
