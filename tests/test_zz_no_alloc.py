"""mgr_vcycle_noalloc: the allocation-free V-cycle entry point.

Callers that cannot allocate device memory where they run (all device memory
handed to their own pool up front, or no allocation allowed after start-up)
use this entry point; it takes its workspace from a fixed buffer compiled into
the library.  Its result must equal that of mgr_vcycle (the same kernels with
the handle's workspace) bit for bit, on two calls in a row, which also shows
that what one call leaves in the shared buffer does not leak into the next;
and after a start-up call neither the library's memory pool nor the device's
free memory may change across the calls.  This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1904_05960_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_05960_gb300 import mgr  # noqa: E402

@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("precision", [mgr.MGR_FP64, mgr.MGR_MIXED])
def test_noalloc_vcycle_matches_vcycle_on_two_calls(precision):
    p = synth.two_phase(12, 10, 7, seed=4)
    s = mgr.Solver(p, precision=precision)
    g = torch.Generator(device="cpu").manual_seed(11)
    # start-up call: under lazy module loading the runtime maps the fixed
    # buffer when the entry point is first used on the device
    n0 = mgr.mgr_get_csr_dims(s.h, mgr.Q_AMG_A, 2, 0)[0]
    mgr.mgr_vcycle_noalloc(s.h, 2, torch.zeros(n0, dtype=torch.float64, device="cuda"),
                           torch.empty(n0, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    for slot in (0, 2):                 # A_uu AMG and the pressure AMG
        n = mgr.mgr_get_csr_dims(s.h, mgr.Q_AMG_A, slot, 0)[0]
        for call in range(2):
            b = torch.randn(n, generator=g, dtype=torch.float64).cuda()
            ref = torch.empty_like(b)
            mgr.mgr_vcycle(s.h, slot, b, ref)
            out = torch.full_like(b, float("nan"))
            torch.cuda.synchronize()
            pool_before = mgr.mgr_memory_usage()
            free_before = torch.cuda.mem_get_info()[0]
            mgr.mgr_vcycle_noalloc(s.h, slot, b, out)
            torch.cuda.synchronize()
            assert mgr.mgr_memory_usage() == pool_before
            assert torch.cuda.mem_get_info()[0] == free_before
            assert torch.isfinite(out).all()
            assert torch.equal(out, ref), (slot, call, _rel(out, ref))
    s.close()


def test_noalloc_rejects_workspace_beyond_the_fixed_buffer():
    # 64x64x32 cells: the A_uu V-cycle needs ~11 MB of FP64 level vectors
    # (418,275 + 113,389 + ... rows), the pressure V-cycle ~4 MB
    p = synth.two_phase(64, 64, 32)
    s = mgr.Solver(p)
    n = mgr.mgr_get_csr_dims(s.h, mgr.Q_AMG_A, 0, 0)[0]
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(mgr.MgrError) as e:
        mgr.mgr_vcycle_noalloc(s.h, 0, b, x)
    assert e.value.code == -1
    assert torch.count_nonzero(x) == 0          # nothing was launched
    # the pressure AMG of the same problem fits and still works
    n2 = mgr.mgr_get_csr_dims(s.h, mgr.Q_AMG_A, 2, 0)[0]
    b2 = torch.randn(n2, dtype=torch.float64, device="cuda")
    ref, out = torch.empty_like(b2), torch.empty_like(b2)
    mgr.mgr_vcycle(s.h, 2, b2, ref)
    mgr.mgr_vcycle_noalloc(s.h, 2, b2, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    s.close()
