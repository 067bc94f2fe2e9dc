"""aafwi_misfit_noalloc: the misfit for callers that cannot allocate device
memory while they run (a framework that owns the whole device budget through
its own allocator, or a loop that must not pay cudaMalloc's device-wide
synchronisation).  Its scratch is a static array inside the library, so the
test checks that two calls in a row, sharing that array, both reproduce the
plan-based aafwi_misfit, and that oversized inputs are refused before any
launch.  Collected last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2008_11778_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2008_11778_gb300 import aafwi, build
    build.build()
    aafwi.load()
    assert torch.cuda.is_available()
    return aafwi


def test_noalloc_misfit_matches_plan_misfit_twice(lib):
    import torch
    # 3 shots x 1000 steps x 300 receivers = 900,000 samples: 13 full chunks
    # of the static partial-sum array plus a ragged tail
    p = synth.small_problem(nz=36, nx=300, nb=8, nt=1000, S=3)
    plan = lib.Plan(p.geom, c_max=3000.0)
    n = plan.trace_count
    assert n == 900_000
    rng = np.random.default_rng(5)
    for call in range(2):
        a = torch.as_tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
        b = torch.as_tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
        r_plan = torch.empty(n, device="cuda")
        r_static = torch.full((n,), float("nan"), device="cuda")
        J_plan = plan.misfit(a, b, r_plan)
        J_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        J_static = lib.misfit_noalloc(a, b, r_static, J_dev=J_dev)
        assert J_static == pytest.approx(J_plan, rel=1e-12), call
        assert float(J_dev.item()) == J_static
        assert torch.equal(r_static, r_plan)
        e = (a - b).double()
        assert J_static == pytest.approx(0.5 * float((e * e).sum()), rel=1e-12)


def test_noalloc_misfit_refuses_oversized_input(lib):
    import torch
    a = torch.zeros(8, device="cuda")
    for n in (lib.MISFIT_NOALLOC_MAX_SAMPLES + 1, 0):
        with pytest.raises(lib.AafwiError) as e:
            lib.misfit_noalloc(a, a, n=n)
        assert e.value.code == 1
        assert "static scratch" in str(e.value)
