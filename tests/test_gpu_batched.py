"""Batched ensemble entry points (mgr_setup_batched / fgmres_solve_batched).

Every system keeps the hierarchy and the FGMRES iteration of its single-system
solve, so the batched solutions must equal the single-system solutions bit for
bit, with the same iteration counts; one member is also checked against the
oracle (Sec. 6 solver settings, iterations +-2, solution 1e-6).  Members are
drawn by the ensemble recipe (cubic side, sigma in [1, 3], dt log-uniform in
[0.1, 10]) with small sides so the oracle and the test stay fast.
"""
import numpy as np
import pytest

from paper_1904_05960_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_05960_gb300 import mgr  # noqa: E402

SIDES = (8, 14)
NSYS = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def members():
    return [synth.ensemble_member(i, SIDES) for i in range(NSYS)]


def _solve_single(p, A, precision, ortho=mgr.MGR_ORTHO_AUTO):
    h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=precision))
    b = torch.from_numpy(p.rhs).cuda()
    x = torch.zeros_like(b)
    r = mgr.fgmres_solve(h, A, b, x, mgr.fgmres_options_default(ortho=ortho))
    mgr.mgr_destroy(h)
    return x, r


@pytest.mark.parametrize("precision", [mgr.MGR_MIXED, mgr.MGR_FP64])
@pytest.mark.parametrize("workers", [0, 3, -1], ids=["autotuned", "3-workers", "lockstep"])
@pytest.mark.parametrize("ortho", [mgr.MGR_ORTHO_MGS, mgr.MGR_ORTHO_CGS2], ids=["mgs", "cgs2"])
def test_batched_equals_single_solves(members, precision, workers, ortho):
    As = [mgr.DeviceMatrix(p) for p in members]
    bh = mgr.mgr_setup_batched(As, mgr.mgr_options_default(True, precision=precision),
                               workers=workers)
    info = mgr.mgr_batch_info(bh)
    assert info["workers"] == -1 or 1 <= info["workers"] <= min(16, NSYS)
    if workers:
        assert info["workers"] == workers and not info["tune_ms"]
    else:
        # every worker count and the lockstep graph were timed
        assert info["tune_ms"] and info["workers"] in info["tune_ms"] and -1 in info["tune_ms"]
    bs = [torch.from_numpy(p.rhs).cuda() for p in members]
    xs = [torch.full_like(b, float("nan")) for b in bs]
    fo = mgr.fgmres_options_default(ortho=ortho)
    st, infos = mgr.fgmres_solve_batched(bh, As, bs, xs, fo)
    assert st == mgr.MGR_SUCCESS
    torch.cuda.synchronize()
    for i, (p, A) in enumerate(zip(members, As)):
        assert infos[i]["converged"] and infos[i]["relres"] <= 1e-8
        x1, r1 = _solve_single(p, A, precision, ortho)
        assert infos[i]["iters"] == r1["iters"], i
        assert torch.equal(xs[i], x1), i
    # a second solve on the same batch gives the same answer
    xs2 = [torch.zeros_like(b) for b in bs]
    mgr.fgmres_solve_batched(bh, As, bs, xs2, fo)
    for i in range(NSYS):
        assert torch.equal(xs2[i], xs[i])
    mgr.mgr_destroy_batched(bh)


def test_lockstep_with_sliced_jacobians_equals_single_solves():
    """Two systems large enough (31M non-zeros each) for the solves to read
    sliced copies of their Jacobians: the lockstep schedule's row-parallel
    product over those copies gives every system its single-system bits."""
    probs = [synth.two_phase(64, 64, 32, seed=q, sigma=2.0) for q in (0, 1)]
    As = [mgr.DeviceMatrix(p) for p in probs]
    bs = [torch.from_numpy(p.rhs).cuda() for p in probs]
    opts = mgr.mgr_options_default(True, precision=mgr.MGR_MIXED)
    bh = mgr.mgr_setup_batched(As, opts, workers=-1)
    xs = [torch.zeros_like(b) for b in bs]
    st, infos = mgr.fgmres_solve_batched(bh, As, bs, xs)
    assert st == mgr.MGR_SUCCESS
    mgr.mgr_destroy_batched(bh)
    for p, A, b, x, inf in zip(probs, As, bs, xs, infos):
        h = mgr.mgr_setup(A, opts)
        x1 = torch.zeros_like(b)
        r = mgr.fgmres_solve(h, A, b, x1)
        assert mgr.mgr_jacobian_product(h, A, b, torch.empty_like(b), refresh=False)
        mgr.mgr_destroy(h)
        assert r["iters"] == inf["iters"] and torch.equal(x1, x)


def test_lockstep_launches_per_round(members):
    """Lockstep: each FGMRES round is one launch per phase for all systems
    (the preconditioner applications of all of them in one graph launch), so
    the host issues the same dozen-odd launches per round whatever the number
    of systems, where the systems solved one by one issue a dozen or more per
    iteration each (classical Gram-Schmidt, whose launches per iteration are
    fixed)."""
    As = [mgr.DeviceMatrix(p) for p in members]
    opts = mgr.mgr_options_default(True, precision=mgr.MGR_MIXED)
    fo = mgr.fgmres_options_default(ortho=mgr.MGR_ORTHO_CGS2)
    bs = [torch.from_numpy(p.rhs).cuda() for p in members]
    xs = [torch.zeros_like(b) for b in bs]
    bh = mgr.mgr_setup_batched(As, opts, workers=-1)
    h0, k0 = mgr.mgr_host_launch_count(), mgr.mgr_launch_count()
    st, infos = mgr.fgmres_solve_batched(bh, As, bs, xs, fo)
    lock_host = mgr.mgr_host_launch_count() - h0
    lock_kernels = mgr.mgr_launch_count() - k0
    mgr.mgr_destroy_batched(bh)
    assert st == mgr.MGR_SUCCESS
    rounds = max(i["iters"] for i in infos)
    total = sum(i["iters"] for i in infos)
    hs = [mgr.mgr_setup(A, opts) for A in As]
    h0, k0 = mgr.mgr_host_launch_count(), mgr.mgr_launch_count()
    for h, A, b in zip(hs, As, bs):
        mgr.fgmres_solve(h, A, b, torch.zeros_like(b), fo)
    single_host = mgr.mgr_host_launch_count() - h0
    single_kernels = mgr.mgr_launch_count() - k0
    for h in hs:
        mgr.mgr_destroy(h)
    assert single_host >= 12 * total
    # a fixed number of launches per round, plus the cycle starts and ends
    assert lock_host <= 20 * rounds + 30 * (sum(i["restarts"] for i in infos) + NSYS), lock_host
    assert lock_host < single_host / 2
    # the preconditioner graphs run the same kernels either way; the Krylov
    # phases are one kernel for all systems instead of one per system
    assert lock_kernels < single_kernels


def test_batched_member_matches_oracle(members):
    import oracle
    As = [mgr.DeviceMatrix(p) for p in members[:3]]
    bh = mgr.mgr_setup_batched(As, mgr.mgr_options_default(True), workers=2)
    bs = [torch.from_numpy(p.rhs).cuda() for p in members[:3]]
    xs = [torch.zeros_like(b) for b in bs]
    st, infos = mgr.fgmres_solve_batched(bh, As, bs, xs)
    mgr.mgr_destroy_batched(bh)
    assert st == mgr.MGR_SUCCESS
    p = members[0]
    ref = oracle.Oracle(p).fgmres(p.rhs)
    assert ref["status"] == 0
    assert abs(infos[0]["iters"] - ref["iters"]) <= 2
    x = xs[0].cpu().numpy()
    assert np.linalg.norm(x - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])


def test_batched_inspection_handle(members):
    As = [mgr.DeviceMatrix(p) for p in members[:2]]
    bh = mgr.mgr_setup_batched(As, mgr.mgr_options_default(True), workers=1)
    h1 = mgr.mgr_batch_handle(bh, 1)
    hs = mgr.mgr_setup(As[1], mgr.mgr_options_default(True))
    for kind, slot, lvl in ((mgr.Q_MGR_S, 1, 0), (mgr.Q_AMG_P, 0, 0), (mgr.Q_AMG_A, 2, 1)):
        a = mgr.mgr_get_csr(h1, kind, slot, lvl)
        b = mgr.mgr_get_csr(hs, kind, slot, lvl)
        assert a is not None and b is not None
        for u, v in zip(a[2:], b[2:]):
            assert np.array_equal(u, v)
    mgr.mgr_destroy(hs)
    with pytest.raises(mgr.MgrError):
        mgr.mgr_batch_handle(bh, 2)
    mgr.mgr_destroy_batched(bh)


def test_batched_argument_errors(members):
    As = [mgr.DeviceMatrix(p) for p in members[:2]]
    with pytest.raises(mgr.MgrError) as e:
        mgr.mgr_setup_batched([], mgr.mgr_options_default(True))
    assert e.value.code == -1
    for bad in (17, -2):
        with pytest.raises(mgr.MgrError) as e:
            mgr.mgr_setup_batched(As, mgr.mgr_options_default(True), workers=bad)
        assert e.value.code == -1
    bh = mgr.mgr_setup_batched(As, mgr.mgr_options_default(True), workers=1)
    bs = [torch.from_numpy(p.rhs).cuda() for p in members[:2]]
    xs = [torch.zeros_like(b) for b in bs]
    with pytest.raises(mgr.MgrError) as e:          # systems given in the wrong order
        mgr.fgmres_solve_batched(bh, As[::-1], bs[::-1], xs[::-1])
    assert e.value.code == -1
    mgr.mgr_destroy_batched(bh)
    for workers in (1, -1):                         # an unknown orthogonalisation
        bh = mgr.mgr_setup_batched(As, mgr.mgr_options_default(True), workers=workers)
        with pytest.raises(mgr.MgrError) as e:
            mgr.fgmres_solve_batched(bh, As, bs, xs, mgr.fgmres_options_default(ortho=3))
        assert e.value.code == -1
        mgr.mgr_destroy_batched(bh)
