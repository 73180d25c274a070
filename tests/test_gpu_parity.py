"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Bars (written here, derived in the design notes):
  * integer work -- C/F marks, strength graphs, CSR patterns of W_p, A_cor,
    G(A_cor), S_l, P, R and every Galerkin operator: bit-exact;
  * FP64 setup values (W_p, A_cor, S_l, P, RAP): <= 1e-12 relative to the
    largest magnitude of the matrix (both sides use the same rounded
    operations in the same order, so in practice they are equal);
  * one FP64 preconditioner application / V-cycle: <= 1e-10 relative (same
    operator, different summation order inside the sparse products and an
    explicit coarsest inverse instead of an LU solve);
  * FGMRES to 1e-8: iteration counts within +-2 and the solution within 1e-6
    relative of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1904_05960_gb300 import synth
from tests.helpers import labeled_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_05960_gb300 import mgr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _same_pattern(a, b, what):
    assert a.shape == b.shape, f"{what}: shape {a.shape} vs {b.shape}"
    assert np.array_equal(a.indptr, b.indptr), f"{what}: row pointers differ"
    assert np.array_equal(a.indices, b.indices), f"{what}: column indices differ"


def _close_values(a, b, what, rtol=1e-12):
    scale = max(np.abs(a.data).max() if a.nnz else 0.0, 1e-300)
    d = np.abs(a.data - b.data).max() if a.nnz else 0.0
    assert d <= rtol * scale, f"{what}: max diff {d:.3e} vs scale {scale:.3e}"


def compare_hierarchy(o, h, L):
    for l in range(L):
        for kind, name in ((mgr.Q_MGR_W, "W_p"), (mgr.Q_MGR_COR, "A_cor"),
                           (mgr.Q_MGR_CORKEPT, "G(A_cor)"), (mgr.Q_MGR_S, "S")):
            a = o.scipy(kind, l)
            b = mgr.mgr_get_scipy(h, kind, l)
            _same_pattern(a, b, f"level {l} {name}")
            _close_values(a, b, f"level {l} {name}")
    for slot in range(L + 1):
        no = o.amg_levels(slot)
        assert mgr.mgr_amg_levels(h, slot) == no, f"AMG slot {slot} depth"
        for k in range(no):
            a = o.scipy(oracle.Q_AMG_A, slot, k)
            b = mgr.mgr_get_scipy(h, mgr.Q_AMG_A, slot, k)
            _same_pattern(a, b, f"AMG {slot}/{k} A")
            _close_values(a, b, f"AMG {slot}/{k} A")
            if k + 1 < no:
                cf_o, cf_g = o.cf(slot, k), mgr.mgr_get_cf(h, slot, k)
                assert np.array_equal(cf_o, cf_g), f"AMG {slot}/{k} C/F marks"
                for kind, name in ((mgr.Q_AMG_S, "S"), (mgr.Q_AMG_P, "P"), (mgr.Q_AMG_R, "R")):
                    a = o.scipy(kind, slot, k)
                    b = mgr.mgr_get_scipy(h, kind, slot, k)
                    if name == "S":
                        a.sort_indices()
                        b.sort_indices()
                        _same_pattern(a, b, f"AMG {slot}/{k} strength")
                    else:
                        _same_pattern(a, b, f"AMG {slot}/{k} {name}")
                        _close_values(a, b, f"AMG {slot}/{k} {name}")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _maxrel(a, b):
    """Element-wise: the largest entry difference over the largest entry."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _spmv_bound_ok(p, x, y_gpu, y_orc, rtol=1e-12):
    """Every entry of the FP64 product within rtol of its own scale
    sum_j |a_ij x_j| (summation order is the only difference)."""
    A = p.to_scipy()
    scale = abs(A) @ np.abs(x)
    bad = np.abs(y_gpu - y_orc) > rtol * scale
    return not bad.any(), int(bad.sum())


SMALL = [
    ("single_phase_8", lambda: synth.config(1)),
    ("two_phase_10x9x6", lambda: synth.two_phase(10, 9, 6)),
    ("two_phase_13x11x7_ragged", lambda: synth.two_phase(13, 11, 7, seed=3, sigma=1.5)),
    ("two_phase_24x20x12", lambda: synth.two_phase(24, 20, 12, seed=5, corr=(6.0, 6.0, 2.0))),
]


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_hierarchy_bit_exact_small(name, make):
    p = make()
    o = oracle.Oracle(p)
    s = mgr.Solver(p)
    compare_hierarchy(o, s.h, o.num_levels)
    s.close()


@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_apply_and_vcycles_match_oracle(name, make):
    p = make()
    o = oracle.Oracle(p)
    s = mgr.Solver(p)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(p.n)
    z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    zo = o.apply(v)
    assert _rel(z, zo) <= 1e-10 and _maxrel(z, zo) <= 1e-10
    for slot in range(o.num_levels + 1):
        if o.amg_levels(slot) == 0:
            continue
        nA = o.scipy(oracle.Q_AMG_A, slot, 0).shape[0]
        b = rng.standard_normal(nA)
        x = torch.zeros(nA, dtype=torch.float64, device="cuda")
        mgr.mgr_vcycle(s.h, slot, torch.from_numpy(b).cuda(), x)
        torch.cuda.synchronize()
        xg, xo = x.cpu().numpy(), o.vcycle(slot, b)
        assert _rel(xg, xo) <= 1e-10 and _maxrel(xg, xo) <= 1e-10, (slot, _maxrel(xg, xo))
    s.close()


@pytest.mark.parametrize("name,make", SMALL + [
    ("two_phase_4x4x3_tiny", lambda: synth.two_phase(4, 4, 3)),
    ("channels_20x18x16", lambda: synth.channels(20, 18, 16, seed=2))],
    ids=[s[0] for s in SMALL] + ["two_phase_4x4x3_tiny", "channels_20x18x16"])
def test_jacobian_spmv_matches_oracle_elementwise(name, make):
    """The FP64 Jacobian product of every FGMRES iteration (w = A z_j),
    through the C ABI, against the oracle's row sums: every entry within
    1e-12 of its own scale sum_j |a_ij x_j|."""
    p = make()
    A = mgr.DeviceMatrix(p)
    rng = np.random.default_rng(3)
    for x in (rng.standard_normal(p.n), np.abs(rng.standard_normal(p.n)) + 1.0):
        y = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
        mgr.mgr_spmv(A, torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        ok, nbad = _spmv_bound_ok(p, x, y.cpu().numpy(), oracle.csr_spmv(p.row_ptr, p.col, p.val, x))
        assert ok, f"{nbad} entries outside the bound"


@pytest.mark.parametrize("name,make", SMALL[1:] + [("config2_64x64x32", lambda: synth.config(2))],
                         ids=[s[0] for s in SMALL[1:]] + ["config2_64x64x32"])
def test_mixed_precision_apply_within_fp32_bound(name, make):
    """One application of the FP32 preconditioner (MGR_MIXED) and each of its
    V-cycles against the oracle's FP64 ones, element-wise.  Bound 1e-4 of the
    largest entry: every stored value and intermediate vector carries an FP32
    rounding (unit roundoff 6e-8), and the smoothers' and coarse solves'
    conditioning (below ~1e3 on these operators) amplifies it.  At 64x64x32
    the displacement and pressure operators are applied through their shared
    row patterns with the FP32 values sliced by 32 rows."""
    p = make()
    o = oracle.Oracle(p)
    s = mgr.Solver(p, precision=mgr.MGR_MIXED)
    if p.nnz > 2 ** 24:
        assert mgr.mgr_row_patterns(s.h, 0, 0) > 0
    rng = np.random.default_rng(17)
    v = rng.standard_normal(p.n)
    z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    err = _maxrel(z, o.apply(v))
    assert err <= 1e-4, err
    assert err > 0.0          # it really ran in FP32
    for slot in range(o.num_levels + 1):
        if o.amg_levels(slot) == 0:
            continue
        nA = o.scipy(oracle.Q_AMG_A, slot, 0).shape[0]
        b = rng.standard_normal(nA)
        x = torch.zeros(nA, dtype=torch.float64, device="cuda")
        mgr.mgr_vcycle(s.h, slot, torch.from_numpy(b).cuda(), x)
        torch.cuda.synchronize()
        assert _maxrel(x.cpu().numpy(), o.vcycle(slot, b)) <= 1e-4
    s.close()


@pytest.mark.parametrize("name,make", SMALL[1:] + [("config2_64x64x32", lambda: synth.config(2))],
                         ids=[s[0] for s in SMALL[1:]] + ["config2_64x64x32"])
def test_bf16_smoother_diagonals_solution_matches_oracle(name, make):
    """diag_bf16 (MGR_MIXED): the l1-Jacobi diagonals, D_FF^-1 and the 2x2
    block inverses read in BF16.  The preconditioner changes by the BF16
    rounding of those values (unit roundoff 2^-9 ~ 2e-3), which flexible GMRES
    absorbs: the solution stays within 1e-6 of the oracle's and the
    iterations within +-2 of the oracle's.  One application differs from the
    oracle's FP64 one by the diagonal rounding, below 5e-2 of its largest
    entry (a few 2e-3 perturbations per level, damped by the smoothers)."""
    p = make()
    o = oracle.Oracle(p)
    ref = o.fgmres(p.rhs)
    s = mgr.Solver(p, precision=mgr.MGR_MIXED, diag_bf16=1)
    v = np.random.default_rng(23).standard_normal(p.n)
    z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    err = _maxrel(z, o.apply(v))
    assert 0.0 < err <= 5e-2, err
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_f16_values_solution_matches_oracle():
    """values_f16 (MGR_MIXED) on the 64x64x32 workload: the patterned
    operators (A_uu and the pressure operator) read FP16 values scaled per
    row.  Each value carries a relative rounding of 2^-11 ~ 5e-4 of its row's
    largest magnitude; one application stays within 5e-2 of the oracle's FP64
    one (as for the BF16 diagonals), and flexible GMRES absorbs the change:
    iterations within +-2 of the oracle's, solution within 1e-6."""
    p = synth.config(2)
    o = oracle.Oracle(p)
    ref = o.fgmres(p.rhs)
    s = mgr.Solver(p, precision=mgr.MGR_MIXED, values_f16=1)
    assert mgr.mgr_row_patterns(s.h, 0, 0) > 0
    v = np.random.default_rng(29).standard_normal(p.n)
    z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    err = _maxrel(z, o.apply(v))
    assert 0.0 < err <= 5e-2, err
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_directed_star_hierarchy_matches_oracle():
    """Scalar matrix whose strength graph is a directed star (the PMIS weight
    pin): C/F marks, strength, P, R and the Galerkin operator bit-exact."""
    from tests.test_oracle_pins import directed_star_matrix
    from tests.helpers import scalar_problem
    p = scalar_problem(directed_star_matrix())
    o = oracle.Oracle(p, num_levels=0, amg_max_coarse=1)
    s = mgr.Solver(p, num_levels=0, amg_max_coarse=1)
    compare_hierarchy(o, s.h, 0)
    assert mgr.mgr_get_cf(s.h, 0, 0).tolist() == [1] + [-1] * 7
    s.close()


@pytest.mark.parametrize("ortho", [mgr.MGR_ORTHO_MGS, mgr.MGR_ORTHO_CGS2], ids=["mgs", "cgs2"])
@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_fgmres_matches_oracle(name, make, ortho):
    """Either orthogonalisation reaches the oracle's (modified Gram-Schmidt)
    iteration count to +-2 and its solution to 1e-6."""
    p = make()
    ref = oracle.Oracle(p).fgmres(p.rhs)
    s = mgr.Solver(p)
    r = s.solve(torch.from_numpy(p.rhs).cuda(), ortho=ortho)
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_restart_path_matches_oracle():
    p = synth.two_phase(8, 8, 4)
    ref = oracle.Oracle(p).fgmres(p.rhs, restart=5)
    s = mgr.Solver(p)
    r = s.solve(torch.from_numpy(p.rhs).cuda(), restart=5)
    assert r["converged"] and r["restarts"] >= 1
    assert abs(r["iters"] - ref["iters"]) <= 2
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


MGS_CASES = SMALL + [
    # 3 * 49 * 49 * 33 + 2 * 48 * 48 * 32 = 385,161 unknowns: more KB-entry
    # tiles than Gram-Schmidt blocks, so the blocks sweep several tiles in both
    # directions and the last tile is ragged
    ("two_phase_48x48x32", lambda: synth.two_phase(48, 48, 32, seed=6)),
]


@pytest.mark.parametrize("name,make", MGS_CASES, ids=[s[0] for s in MGS_CASES])
def test_modified_gram_schmidt_matches_oracle(name, make):
    """FGMRES with modified Gram-Schmidt (the oracle's orthogonalisation):
    the residual history agrees step by step -- to 1e-6 of each estimate plus
    1e-12 of ||b||, the rounding the Arnoldi recurrence accumulates relative to
    the starting residual -- and the solution to 1e-6; a short restart takes
    the restart path too."""
    p = make()
    restart = 12 if p.n < 100000 else 50
    ref = oracle.Oracle(p).fgmres(p.rhs, restart=restart, hist_cap=1001)
    s = mgr.Solver(p)
    r = s.solve(torch.from_numpy(p.rhs).cuda(), restart=restart, hist_cap=1001,
                ortho=mgr.MGR_ORTHO_MGS)
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 1, (r["iters"], ref["iters"])
    k = min(len(r["hist"]), len(ref["hist"])) - 1
    h_gpu, h_orc = np.asarray(r["hist"][:k]), ref["hist"][:k]
    assert np.all(np.abs(h_gpu - h_orc) <= 1e-6 * h_orc + 1e-12), name
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_exact_two_level_identity_on_gpu():
    """With ideal components the GPU preconditioner is A^-1 (Sec. 5.1)."""
    p = labeled_system(seed=13, two_phase=False, diag_uu=True, n_nodes=30, n_cells=40)
    s = mgr.Solver(p, nmax_drop=[-1], amg_max_coarse=1000)
    A = p.to_scipy()
    x = np.random.default_rng(0).standard_normal(p.n)
    z = s.apply(torch.from_numpy(A @ x).cuda()).cpu().numpy()
    assert _rel(z, x) <= 1e-10
    s.close()


def test_nmax_variants_bit_exact():
    p = synth.two_phase(9, 8, 5, seed=2)
    for nmax in (0, 1, 7):
        o = oracle.Oracle(p, nmax_drop=[nmax, -1])
        s = mgr.Solver(p, nmax_drop=[nmax, -1])
        compare_hierarchy(o, s.h, 2)
        s.close()


def test_splitmix64_device_matches_published_vectors():
    xs = np.array([0, 0x9E3779B97F4A7C15, 0x3C6EF372FE94F82A, 12345], dtype=np.uint64)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    mgr.mgr_splitmix64_device(torch.from_numpy(xs.view(np.int64)).cuda(), out)
    got = out.cpu().numpy().view(np.uint64)
    assert [int(g) for g in got] == [oracle.splitmix64(int(x)) for x in xs]
    assert int(got[0]) == 0xE220A8397B1DCDAF


def test_mixed_precision_solution_within_1e6():
    p = synth.two_phase(16, 16, 8)
    ref = oracle.Oracle(p).fgmres(p.rhs)
    s = mgr.Solver(p, precision=mgr.MGR_MIXED)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_invalid_arguments_are_rejected():
    p = synth.two_phase(4, 4, 3)
    A = mgr.DeviceMatrix(p)
    with pytest.raises(mgr.MgrError) as e:
        mgr.mgr_setup(A, mgr.mgr_options_default(True, num_levels=9))
    assert e.value.code == -1
    with pytest.raises(mgr.MgrError) as e:   # F = every label: empty C set
        mgr.mgr_setup(A, mgr.mgr_options_default(True, f_label_mask=[0b111, 0b10]))
    assert e.value.code == -1
    for bad in (dict(global_smoother=[0, 3]), dict(ilu_solve_sweeps=-1), dict(diag_bf16=1),
                dict(diag_bf16=2, precision=mgr.MGR_MIXED), dict(values_f16=1),
                dict(values_f16=2, precision=mgr.MGR_MIXED)):
        with pytest.raises(mgr.MgrError) as e:
            mgr.mgr_setup(A, mgr.mgr_options_default(True, **bad))
        assert e.value.code == -1
    s = mgr.Solver(p)
    with pytest.raises(mgr.MgrError) as e:
        s.solve(torch.zeros(p.n, dtype=torch.float64, device="cuda"), ortho=3)
    assert e.value.code == -1
    s.close()


def test_memory_pool_trim_keeps_handles_valid():
    """The library's pool keeps freed memory for the next setup; trimming it
    returns that memory and leaves live handles working."""
    p = synth.two_phase(10, 9, 6, seed=4)
    o = oracle.Oracle(p)
    ref = o.fgmres(p.rhs)
    s1 = mgr.Solver(p)
    s1.close()
    s2 = mgr.Solver(p)
    mgr.mgr_trim_memory(0)
    r = s2.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and abs(r["iters"] - ref["iters"]) <= 2
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s2.close()
    mgr.mgr_trim_memory(0)


def test_zero_diagonal_reported():
    p = synth.two_phase(4, 4, 3)
    v = p.val.copy()
    r0, r1 = p.row_ptr[5], p.row_ptr[6]
    cols = p.col[r0:r1]
    v[r0 + int(np.nonzero(cols == 5)[0][0])] = 0.0
    p.val = v
    with pytest.raises(mgr.MgrError) as e:
        mgr.Solver(p)
    assert e.value.code == -4


def test_full_size_workload_hierarchy_and_solve():
    """The 64x64x32 two-phase workload (680,419 unknowns): the whole integer
    hierarchy bit-exact and the FP64 solve within the bars."""
    p = synth.config(2)
    o = oracle.Oracle(p)
    s = mgr.Solver(p)
    compare_hierarchy(o, s.h, 2)
    # the displacement operator is applied through shared row patterns (the
    # mesh stencil: a few hundred distinct column-offset rows), with the
    # V-cycle still the oracle's to the apply bar, element-wise
    npat = mgr.mgr_row_patterns(s.h, 0, 0)
    assert 0 < npat <= 4096, npat
    b = np.random.default_rng(31).standard_normal(p.meta["n_u"])
    x = torch.zeros(p.meta["n_u"], dtype=torch.float64, device="cuda")
    mgr.mgr_vcycle(s.h, 0, torch.from_numpy(b).cuda(), x)
    torch.cuda.synchronize()
    assert _maxrel(x.cpu().numpy(), o.vcycle(0, b)) <= 1e-10
    ref = o.fgmres(p.rhs)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and abs(r["iters"] - ref["iters"]) <= 2
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_jacobian_sliced_product_and_solve():
    """The 64x64x32 two-phase Jacobian (31.35M non-zeros) is multiplied by
    FGMRES over a sliced copy made at every solve: each entry of the product
    within 1e-12 of its own scale sum |a_ij x_j| of the oracle's CSR product;
    changing A's values in place and refreshing gives the new product; the
    solve meets the oracle's iterations and solution."""
    p = synth.config(2)
    A = mgr.DeviceMatrix(p)
    h = mgr.mgr_setup(A, mgr.mgr_options_default(True))
    xh = np.random.default_rng(41).standard_normal(p.n)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty_like(x)
    assert mgr.mgr_jacobian_product(h, A, x, y, refresh=True)
    ok, nbad = _spmv_bound_ok(p, xh, y.cpu().numpy(), oracle.csr_spmv(p.row_ptr, p.col, p.val, xh))
    assert ok, nbad
    y2 = torch.empty_like(x)
    assert mgr.mgr_jacobian_product(h, A, x, y2, refresh=False)   # the same copy, the same bits
    torch.cuda.synchronize()
    assert torch.equal(y, y2)
    # values changed in place: a refresh picks them up
    A.val.mul_(0.5)
    assert mgr.mgr_jacobian_product(h, A, x, y2, refresh=True)
    torch.cuda.synchronize()
    assert torch.allclose(y2, 0.5 * y, rtol=1e-14, atol=0.0)
    A.val.mul_(2.0)
    # the solve over the sliced copy: the oracle's iterations and solution
    ref = oracle.Oracle(p).fgmres(p.rhs)
    b = torch.from_numpy(p.rhs).cuda()
    xs = torch.zeros_like(b)
    r = mgr.fgmres_solve(h, A, b, xs)
    assert r["converged"] and abs(r["iters"] - ref["iters"]) <= 2
    assert _rel(xs.cpu().numpy(), ref["x"]) <= 1e-6
    mgr.mgr_destroy(h)


def test_large_workload_against_oracle_fingerprint():
    """128x128x64 cells (5,342,147 unknowns), both precisions, against the
    oracle's solution of the same system (one oracle run of ~13 minutes,
    stored as a fingerprint by tests/golden/make_oracle_fingerprint.py): the
    exact error over 4096 seeded sample entries and the probe estimate of the
    full relative error within 1e-6, iterations within +-2 of the oracle's.
    Also properties at this size: the true residual recomputed with the
    oracle's own sparse product, FP32 and FP64 preconditioners reaching the
    same solution, PMIS invariants and P's rows on the displacement AMG's
    first coarsening."""
    from oracle import fingerprint
    from tests.test_oracle_pins import _pmis_invariants
    fp = fingerprint.load("two_phase_128x128x64")
    p = synth.two_phase(128, 128, 64, seed=0, sigma=2.0, E_sigma=1.5)
    assert p.n == fp["n"] and p.nnz == fp["nnz"]
    sols = {}
    for prec in (mgr.MGR_MIXED, mgr.MGR_FP64):
        s = mgr.Solver(p, precision=prec)
        r = s.solve(torch.from_numpy(p.rhs).cuda())
        x = r["x"].cpu().numpy()
        assert r["converged"]
        assert abs(r["iters"] - fp["iters"]) <= 2, (r["iters"], fp["iters"])
        ax = oracle.csr_spmv(p.row_ptr, p.col, p.val, x)
        assert np.linalg.norm(p.rhs - ax) <= 1e-8 * np.linalg.norm(p.rhs) * 1.001
        c = fingerprint.compare(x, fp)
        assert c["sample_rel"] <= 1e-6 and c["probe_rel"] <= 1e-6, c
        sols[prec] = x
        if prec == mgr.MGR_FP64:
            S = mgr.mgr_get_scipy(s.h, mgr.Q_AMG_S, 0, 0)
            cf = mgr.mgr_get_cf(s.h, 0, 0)
            _pmis_invariants(S, cf)
            P = mgr.mgr_get_scipy(s.h, mgr.Q_AMG_P, 0, 0)
            assert np.diff(P.indptr).max() <= 4
            cidx = np.cumsum(cf == 1) - 1
            Pc = P[cf == 1]
            assert np.array_equal(Pc.indices, cidx[cf == 1]) and np.all(Pc.data == 1.0)
        s.close()
    assert _rel(sols[mgr.MGR_MIXED], sols[mgr.MGR_FP64]) <= 1e-6


def test_headline_workload_properties():
    """256x256x96 cells with permeability channels and stiff/soft layers
    (31,803,171 unknowns, 1.56e9 non-zeros), MGR_MIXED with one level of
    aggressive coarsening in the displacement AMG (Sec. 6), the configuration
    the benchmark times.  The oracle cannot solve it inside a test, so: the
    true residual of the GPU solution recomputed with the oracle's sparse
    product; W_p = -D_FF^-1 A_FC on 2000 seeded sample rows (the paper's
    definition, Eq. "injective_rp", against the input matrix); the PMIS
    invariants on seeded sample points of the displacement AMG's second
    coarsening; and the library's device memory within the GPU."""
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    mgr.mgr_trim_memory(0)
    p = synth.channels(256, 256, 96, seed=0)
    assert p.n == 31803171
    s = mgr.Solver(p, precision=mgr.MGR_MIXED, agg_levels=[1, 0, 0])
    used, _ = mgr.mgr_memory_usage()
    assert used < 0.6 * torch.cuda.get_device_properties(0).total_memory
    rng = np.random.default_rng(77)
    nu = p.meta["n_u"]
    # W_p rows: F = displacement dofs (a prefix), C = cell dofs
    rows = np.sort(rng.choice(nu, 2000, replace=False))
    W = mgr.mgr_get_csr(s.h, mgr.Q_MGR_W, 0)
    _, nC, wrp, wci, wv = W
    for i in rows:
        a0, a1 = p.row_ptr[i], p.row_ptr[i + 1]
        cols, vals = p.col[a0:a1], p.val[a0:a1]
        d = vals[cols == i][0]
        c = cols >= nu
        want_c, want_v = cols[c] - nu, -(vals[c] / d)
        got_c, got_v = wci[wrp[i]:wrp[i + 1]], wv[wrp[i]:wrp[i + 1]]
        assert np.array_equal(got_c, want_c)
        assert np.all(np.abs(got_v - want_v) <= 1e-15 * np.abs(want_v))
    # PMIS on the displacement AMG's second level (the first is coarsened in
    # two stages, so its C points need not be neighbours of every F point in
    # the first-stage strength graph), at sample points
    S = mgr.mgr_get_scipy(s.h, mgr.Q_AMG_S, 0, 1)
    cf = mgr.mgr_get_cf(s.h, 0, 1)
    assert np.all((cf == 1) | (cf == -1))
    St = None
    for i in rng.choice(S.shape[0], 2000, replace=False):
        row = S.indices[S.indptr[i]:S.indptr[i + 1]]
        if cf[i] == -1 and len(row):
            assert np.any(cf[row] == 1), f"F point {i} without a strong C point"
        if cf[i] == 1:
            for j in row[cf[row] == 1]:          # no two C points strongly coupled both ways
                rj = S.indices[S.indptr[j]:S.indptr[j + 1]]
                assert i not in rj
    del S, St
    r = s.solve(torch.from_numpy(p.rhs).cuda(), max_iter=4000)
    assert r["converged"] and r["relres"] <= 1e-8
    x = r["x"].cpu().numpy()
    s.close()
    ax = oracle.csr_spmv(p.row_ptr, p.col, p.val, x)
    assert np.linalg.norm(p.rhs - ax) <= 1e-8 * np.linalg.norm(p.rhs) * 1.001


# Operator variants of Sec. 5.1 (Jacobi restriction with the full triple
# product, F-relaxation after the correction, point-block D_FF), each against
# the oracle: hierarchy bit-exact, one application, FGMRES.
VARIANTS = [
    ("jacobi_restriction", dict(restrict_jacobi=[1, 1])),
    ("post_smoothing", dict(frelax_post=[1, 1])),
    ("point_block_dff", dict(dff_block=[1, 1])),
    ("all_three", dict(restrict_jacobi=[1, 0], frelax_post=[1, 0], dff_block=[1, 1])),
]


@pytest.mark.parametrize("name,kw", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_operator_variants_match_oracle(name, kw):
    p = synth.two_phase(10, 9, 6, seed=4, E_sigma=1.0)
    o = oracle.Oracle(p, **kw)
    s = mgr.Solver(p, **kw)
    compare_hierarchy(o, s.h, 2)
    for l in range(2):
        for key, kind, what in (("restrict_jacobi", mgr.Q_MGR_WR, "W_r"),
                                ("dff_block", mgr.Q_MGR_BD, "D_FF^-1")):
            if kw.get(key, [0, 0])[l]:
                a = o.scipy(kind, l)
                b = mgr.mgr_get_scipy(s.h, kind, l)
                _same_pattern(a, b, f"level {l} {what}")
                _close_values(a, b, f"level {l} {what}")
            else:
                assert mgr.mgr_get_scipy(s.h, kind, l) is None
    rng = np.random.default_rng(11)
    v = rng.standard_normal(p.n)
    z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(z, o.apply(v)) <= 1e-10
    ref = o.fgmres(p.rhs)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()
    sm = mgr.Solver(p, precision=mgr.MGR_MIXED, **kw)
    rm = sm.solve(torch.from_numpy(p.rhs).cuda())
    assert rm["converged"] and rm["relres"] <= 1e-8
    assert _rel(rm["x"].cpu().numpy(), ref["x"]) <= 1e-6
    sm.close()


@pytest.mark.parametrize("precision", [mgr.MGR_FP64, mgr.MGR_MIXED])
def test_multicolour_gauss_seidel_smoother_matches_oracle(precision):
    """Global smoother option 1 (multicolour point-block Gauss-Seidel at the
    second reduction): colouring bit-exact, application and FGMRES as the
    oracle's."""
    p = synth.two_phase(13, 11, 7, seed=3, sigma=1.5)
    kw = dict(global_smoother=[0, 1])
    o = oracle.Oracle(p, **kw)
    s = mgr.Solver(p, precision=precision, **kw)
    assert mgr.mgr_get_block_colors(s.h, 0) is None
    cg, ncg = mgr.mgr_get_block_colors(s.h, 1)
    co, nco = o.block_colors(1)
    assert ncg == nco and np.array_equal(cg, co)
    if precision == mgr.MGR_FP64:
        compare_hierarchy(o, s.h, 2)
        v = np.random.default_rng(5).standard_normal(p.n)
        z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
        assert _rel(z, o.apply(v)) <= 1e-10
    ref = o.fgmres(p.rhs)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


@pytest.mark.parametrize("precision", [mgr.MGR_FP64, mgr.MGR_MIXED])
def test_aggressive_coarsening_matches_oracle(precision):
    """One level of two-stage aggressive coarsening in the A_uu AMG: hierarchy
    bit-exact (C/F marks, strength, P = P1 P2 truncated, Galerkin products),
    FGMRES as the oracle's."""
    p = synth.two_phase(13, 11, 7, seed=3, sigma=1.5)
    kw = dict(agg_levels=[1, 0, 0])
    o = oracle.Oracle(p, **kw)
    s = mgr.Solver(p, precision=precision, **kw)
    if precision == mgr.MGR_FP64:
        compare_hierarchy(o, s.h, 2)
        base = oracle.Oracle(p)
        assert o.amg_levels(0) < base.amg_levels(0) or \
            o.scipy(oracle.Q_AMG_A, 0, 1).shape[0] < base.scipy(oracle.Q_AMG_A, 0, 1).shape[0]
    ref = o.fgmres(p.rhs)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


@pytest.mark.parametrize("precision", [mgr.MGR_FP64, mgr.MGR_MIXED])
@pytest.mark.parametrize("level,sweeps,solve", [(1, 1, 3), (1, 2, 1), (1, 1, 0), (0, 1, 2)],
                         ids=["l1-s1-j3", "l1-s2-j1", "l1-s1-j0", "l0-s1-j2"])
def test_ilu1_smoother_matches_oracle(precision, level, sweeps, solve):
    """Global smoother option 2 (pointwise ILU(1), Sec. 6): the incomplete
    factors on the level-1 fill pattern as the oracle's (pattern bit-exact,
    values to 1e-12), the smoother's application and FGMRES as the
    oracle's."""
    p = synth.two_phase(13, 11, 7, seed=3, sigma=1.5)
    gsm, gsw = [0, 0], [0, 0]
    gsm[level], gsw[level] = 2, sweeps
    if level == 0:
        gsw[1] = 3
    kw = dict(global_smoother=gsm, global_sweeps=gsw, ilu_solve_sweeps=solve)
    o = oracle.Oracle(p, **kw)
    s = mgr.Solver(p, precision=precision, **kw)
    if precision == mgr.MGR_FP64:
        compare_hierarchy(o, s.h, 2)
        fo = o.scipy(oracle.Q_MGR_ILU, level)
        fg = mgr.mgr_get_scipy(s.h, mgr.Q_MGR_ILU, level)
        _same_pattern(fo, fg, "ILU(1) factors")
        _close_values(fo, fg, "ILU(1) factors")
        assert mgr.mgr_get_csr_dims(s.h, mgr.Q_MGR_ILU, 1 - level) is None
        v = np.random.default_rng(5).standard_normal(p.n)
        z = s.apply(torch.from_numpy(v).cuda()).cpu().numpy()
        assert _rel(z, o.apply(v)) <= 1e-10
    ref = o.fgmres(p.rhs)
    r = s.solve(torch.from_numpy(p.rhs).cuda())
    assert r["converged"] and r["relres"] <= 1e-8
    assert abs(r["iters"] - ref["iters"]) <= 2, (r["iters"], ref["iters"])
    assert _rel(r["x"].cpu().numpy(), ref["x"]) <= 1e-6
    s.close()


def test_solve_from_host_buffers_matches_device_path():
    """mgr_solve_host (host CSR, rhs and solution) gives the device path's
    solution bit for bit and the oracle's to the solution bar."""
    p = synth.two_phase(11, 9, 6, seed=8)
    o = oracle.Oracle(p)
    ref = o.fgmres(p.rhs)
    s = mgr.Solver(p)
    rd = s.solve(torch.from_numpy(p.rhs).cuda())
    s.close()
    for pin in (True, False):
        Ah = mgr.HostMatrix(p, pin=pin)
        bh = torch.from_numpy(p.rhs.copy())
        xh = torch.zeros(p.n, dtype=torch.float64)
        r = mgr.mgr_solve_host(Ah, bh, xh, mgr.mgr_options_default(True))
        assert r["converged"] and r["iters"] == rd["iters"]
        assert np.array_equal(xh.numpy(), rd["x"].cpu().numpy())
        assert abs(r["iters"] - ref["iters"]) <= 2
        assert _rel(xh.numpy(), ref["x"]) <= 1e-6
