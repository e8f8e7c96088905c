"""The allocation-free residual norm (irk_residual_norm_noalloc) against the
context-scratch entry point irk_residual_norm, through the C ABI, on two calls
in a row.  Collected last so that a first-failure run has run everything else."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11377_gb300.build import build
    build()
    from paper_2010_11377_gb300 import binding
    return binding


def _ctx(B, N, s):
    from paper_2010_11377_gb300 import problems
    prob = problems.heat(N)
    A, b, c = B.irk_butcher_table("radau_iia", s)
    ctx = B.irk_setup(prob["rowptr"], prob["col"], prob["valM"], prob["valF"], (A, b, c), 1 / 64)
    return ctx, prob["n"]


def test_noalloc_matches_scratch_entry_point(B):
    ctx, n = _ctx(B, 61, 3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for seed in (1, 2):                       # two calls in a row, different data
        k = torch.tensor(synth.random_stage_block(n, 3, seed).ravel(), dtype=torch.float64, device="cuda")
        rhs = torch.tensor(synth.random_stage_block(n, 3, seed + 10).ravel(), dtype=torch.float64, device="cuda")
        ref = B.irk_residual_norm(ctx, k, rhs)
        B.irk_residual_norm_noalloc(ctx, k, rhs, out)
        got = float(out.item())
        assert abs(got - ref) <= 1e-13 * ref, (seed, got, ref)
    # after the first call on the device, a call changes neither the device's
    # free memory nor the caching allocator's allocation count
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    B.irk_residual_norm_noalloc(ctx, k, rhs, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
    assert abs(float(out.item()) - ref) <= 1e-13 * ref
    ctx.close()


def test_noalloc_rejects_oversize(B):
    from paper_2010_11377_gb300._abi import IrkError
    ctx, n = _ctx(B, 1026, 1)                  # 1025^2 = 1,050,625 rows > 2^20
    assert n > 1048576
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(IrkError) as ei:
        B.irk_residual_norm_noalloc(ctx, z, z, out)
    assert ei.value.status == 9 and "exceeds the maximum" in str(ei.value)
    ctx.close()
