"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself: an
exact algebraic identity of the paper (Sec. 5.1 two-level exactness), a dense
triple product, a brute-force enumeration of a definition on a tiny input, a
textbook invariant, a published test vector, or a library direct solver.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
from oracle import Q_AMG_A, Q_AMG_P, Q_AMG_R, Q_AMG_S, Q_MGR_COR, Q_MGR_CORKEPT, Q_MGR_S, Q_MGR_W
from paper_1904_05960_gb300 import synth
from tests.helpers import labeled_system, poisson3d, scalar_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(p):
    return p.to_scipy().toarray()


# ---------------------------------------------------------------- splitmix64
def test_splitmix64_published_vectors():
    """The PMIS weight hash equals the published SplitMix64 outputs."""
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert rows
    for x, out in rows:
        assert oracle.splitmix64(int(x, 16)) == int(out, 16)


# ------------------------------------------------- reduction operators (5.1)
@pytest.mark.parametrize("two_phase", [False, True])
def test_wp_and_coarse_grid_equal_dense_triple_product(two_phase):
    """With no dropping, S_1 = R~ A P~ = A_CC - A_CF D_FF^-1 A_FC (Sec. 5.2),
    with R~ = [0 I] and P~ = [W_p; I], W_p = -D_FF^-1 A_FC (Eq. injective_rp)."""
    p = labeled_system(seed=3, two_phase=two_phase)
    o = oracle.Oracle(p, nmax_drop=[-1, -1])
    A = dense(p)
    F = np.nonzero(p.dof_label == 0)[0]
    Cc = np.nonzero(p.dof_label != 0)[0]
    D = np.diag(A[np.ix_(F, F)])
    Wp = -A[np.ix_(F, Cc)] / D[:, None]
    assert np.allclose(o.scipy(Q_MGR_W, 0).toarray(), Wp, rtol=1e-13, atol=1e-14)
    Pt = np.zeros((len(p.rhs), len(Cc)))
    Pt[F] = Wp
    Pt[Cc, np.arange(len(Cc))] = 1.0
    Rt = np.zeros((len(Cc), len(p.rhs)))
    Rt[np.arange(len(Cc)), Cc] = 1.0
    S_dense = Rt @ A @ Pt
    S = o.scipy(Q_MGR_S, 0).toarray()
    assert np.abs(S - S_dense).max() <= 1e-12 * np.abs(S_dense).max()


def test_second_reduction_is_pressure_schur_complement():
    """S_2 = A~_pp - A~_ps D_ss^-1 A~_sp with no dropping (Eq. coarse_grid_pressure)."""
    p = labeled_system(seed=5, two_phase=True)
    o = oracle.Oracle(p)
    S1 = o.scipy(Q_MGR_S, 0).toarray()
    s_idx = np.arange(0, S1.shape[0], 2)
    p_idx = np.arange(1, S1.shape[0], 2)
    Dss = np.diag(S1[np.ix_(s_idx, s_idx)])
    S2_dense = S1[np.ix_(p_idx, p_idx)] - S1[np.ix_(p_idx, s_idx)] @ (S1[np.ix_(s_idx, p_idx)] / Dss[:, None])
    S2 = o.scipy(Q_MGR_S, 1).toarray()
    assert np.abs(S2 - S2_dense).max() <= 1e-12 * np.abs(S2_dense).max()


def test_drop_nmax_zero_keeps_only_point_diagonal_blocks():
    """N_max = 0 leaves A_cor with diagonal field sub-blocks only (Sec. 5.2)."""
    p = labeled_system(seed=7, two_phase=True, density=0.3)
    o = oracle.Oracle(p, nmax_drop=[0, -1])
    kept = o.scipy(Q_MGR_CORKEPT, 0).tocoo()
    cnode = p.dof_node[p.dof_label != 0]
    assert kept.nnz > 0
    assert np.all(cnode[kept.row] == cnode[kept.col])
    full = o.scipy(Q_MGR_COR, 0).tocoo()
    same = cnode[full.row] == cnode[full.col]
    assert same.sum() == kept.nnz


@pytest.mark.parametrize("nmax", [1, 4])
def test_drop_rule_brute_force(nmax):
    """G keeps the own-point entries plus the nmax others of largest |value|."""
    p = labeled_system(seed=11, two_phase=True, density=0.35)
    o = oracle.Oracle(p, nmax_drop=[nmax, -1])
    A = dense(p)
    F = np.nonzero(p.dof_label == 0)[0]
    Cc = np.nonzero(p.dof_label != 0)[0]
    D = np.diag(A[np.ix_(F, F)])
    cor_dense = A[np.ix_(Cc, F)] @ (A[np.ix_(F, Cc)] / D[:, None])
    cor = o.scipy(Q_MGR_COR, 0)
    kept = o.scipy(Q_MGR_CORKEPT, 0)
    assert np.allclose(cor.toarray(), cor_dense, rtol=1e-12, atol=1e-13)
    cnode = p.dof_node[Cc]
    for i in range(len(Cc)):
        cols = cor.indices[cor.indptr[i]:cor.indptr[i + 1]]
        own = [c for c in cols if cnode[c] == cnode[i]]
        rest = [c for c in cols if cnode[c] != cnode[i]]
        rest.sort(key=lambda c: (-abs(cor_dense[i, c]), c))
        want = sorted(own + rest[:nmax])
        got = sorted(kept.indices[kept.indptr[i]:kept.indptr[i + 1]].tolist())
        assert got == want


# ---------------------------------------- MGR exactness identities (Sec. 5.1)
def test_two_level_mgr_is_exact_with_ideal_components():
    """A_FF diagonal makes Jacobi interpolation ideal; with exact F-relaxation
    and an exact coarse solve, I - M^-1 A = 0 (Eqs. MGR-mul1 / MGR-pre)."""
    p = labeled_system(seed=13, two_phase=False, diag_uu=True, n_nodes=30, n_cells=40)
    o = oracle.Oracle(p, nmax_drop=[-1], amg_max_coarse=1000)
    A = dense(p)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(p.n)
        z = o.apply(A @ x)
        assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)


def test_three_level_mgr_is_exact_with_ideal_components():
    """Same identity applied recursively (Algorithm 2): A_uu and A_ss diagonal,
    no dropping, no global smoother, exact coarsest solve."""
    p = labeled_system(seed=17, two_phase=True, diag_uu=True, diag_ss=True, n_nodes=25,
                       n_cells=30)
    o = oracle.Oracle(p, nmax_drop=[-1, -1], global_sweeps=[0, 0], amg_max_coarse=1000)
    A = dense(p)
    x = np.random.default_rng(1).standard_normal(p.n)
    z = o.apply(A @ x)
    assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)


def test_dropping_breaks_exactness():
    """The same setting with N_max = 0 is no longer exact (a control for the
    exactness tests: G does change the coarse grid)."""
    p = labeled_system(seed=13, two_phase=False, diag_uu=True, n_nodes=30, n_cells=40,
                       density=0.3)
    o = oracle.Oracle(p, nmax_drop=[0], amg_max_coarse=1000)
    A = dense(p)
    x = np.random.default_rng(0).standard_normal(p.n)
    z = o.apply(A @ x)
    assert np.linalg.norm(z - x) > 1e-6 * np.linalg.norm(x)


def test_block_jacobi_global_smoother_exact_on_block_diagonal():
    """One sweep of cell-block Jacobi solves a block-diagonal flow system
    exactly, so the whole level returns A^-1 v (global relaxation of Alg. 2)."""
    p0 = labeled_system(seed=19, two_phase=True, block_diag_flow=True, n_nodes=1, n_cells=50)
    keep = np.nonzero(p0.dof_label != 0)[0]
    A = p0.to_scipy()[keep][:, keep]
    from tests.helpers import to_problem
    p = to_problem(A, p0.dof_label[keep], p0.dof_node[keep], p0.dof_comp[keep])
    o = oracle.Oracle(p, num_levels=1, f_label_mask=[1 << 1], frelax=[oracle.FRELAX_JACOBI],
                      frelax_sweeps=[1], nmax_drop=[-1], global_sweeps=[1])
    x = np.random.default_rng(2).standard_normal(p.n)
    z = o.apply(A @ x)
    assert np.linalg.norm(z - x) <= 1e-12 * np.linalg.norm(x)


def test_fgmres_one_iteration_with_exact_preconditioner():
    p = labeled_system(seed=13, two_phase=False, diag_uu=True, n_nodes=30, n_cells=40)
    o = oracle.Oracle(p, nmax_drop=[-1], amg_max_coarse=1000)
    r = o.fgmres(p.rhs)
    assert r["status"] == 0 and r["iters"] == 1


# ----------------------------------------------------------------- AMG (Sec. 6)
def _amg_only(A, **kw):
    return oracle.Oracle(scalar_problem(A), num_levels=0, **kw)


def test_strength_brute_force():
    rng = np.random.default_rng(4)
    A = sp.random(60, 60, density=0.2, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k)) + sp.eye(60) * 3
    A = sp.csr_matrix(A)
    A.sort_indices()
    o = _amg_only(A, amg_max_coarse=4)
    S = o.scipy(Q_AMG_S, 0, 0)
    Ad = A.toarray()
    for i in range(60):
        cols = [j for j in A.indices[A.indptr[i]:A.indptr[i + 1]] if j != i]
        negs = [-Ad[i, j] for j in cols]
        m = max(negs) if negs else 0.0
        want = sorted(j for j in cols if m > 0 and -Ad[i, j] >= 0.25 * m)
        got = sorted(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist())
        assert got == want


def test_strength_unknown_approach_ignores_other_components():
    """The A_uu AMG (F-relaxation of the first reduction) sees only couplings
    between equal displacement components (unknown approach, Sec. 6); brute
    force over the definition restricted to equal components."""
    p = synth.single_phase(3, 3, 3)
    o = oracle.Oracle(p, amg_max_coarse=8)
    nu = p.meta["n_u"]
    Auu = p.to_scipy()[:nu, :nu].tocsr()
    comp = p.dof_comp[:nu]
    S = o.scipy(Q_AMG_S, 0, 0)
    Sc = S.tocoo()
    assert Sc.nnz > 0 and np.all(comp[Sc.row] == comp[Sc.col])
    for i in range(nu):
        cols = [j for j in Auu.indices[Auu.indptr[i]:Auu.indptr[i + 1]]
                if j != i and comp[j] == comp[i]]
        vals = {j: Auu[i, j] for j in cols}
        m = max([-v for v in vals.values()], default=0.0)
        want = sorted(j for j in cols if m > 0 and -vals[j] >= 0.25 * m)
        assert sorted(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist()) == want


def _pmis_invariants(S, cf):
    """What the synchronous PMIS rounds guarantee: every point decided; no two
    C points depend strongly on each other (the later one would have been made
    F); isolated points are F; every other F point has a C point in S_i; where
    S is symmetric, C is an independent set."""
    St = S.T.tocsr()
    C = cf == 1
    assert np.all((cf == 1) | (cf == -1))
    M = S.multiply(St).tocoo()            # mutual strong dependence
    assert not np.any(C[M.row] & C[M.col]), "two C points depend on each other"
    if (S != St).nnz == 0:
        Sc = S.tocoo()
        assert not np.any(C[Sc.row] & C[Sc.col]), "C points must be independent"
    for i in range(S.shape[0]):
        row = S.indices[S.indptr[i]:S.indptr[i + 1]]
        trow = St.indices[St.indptr[i]:St.indptr[i + 1]]
        if len(row) == 0 and len(trow) == 0:
            assert not C[i], f"isolated point {i} must be F"
            continue
        if not C[i]:
            assert np.any(C[row]), f"F point {i} has no C point in S_i"


def test_pmis_invariants_poisson():
    A = poisson3d(10, 9, 8)
    o = _amg_only(A, amg_max_coarse=10)
    for k in range(o.amg_levels(0) - 1):
        _pmis_invariants(o.scipy(Q_AMG_S, 0, k), o.cf(0, k))


def test_pmis_invariants_elasticity_hierarchy():
    p = synth.config(1)
    o = oracle.Oracle(p)
    for k in range(o.amg_levels(0) - 1):
        _pmis_invariants(o.scipy(Q_AMG_S, 0, k), o.cf(0, k))


def test_interpolation_structure_and_constant_preservation():
    """Direct interpolation: C rows are unit rows, F rows use strong C
    neighbours only, at most P_max entries, and rows whose matrix row sums to
    zero interpolate constants exactly (also after truncation with row-sum
    rescaling)."""
    A = poisson3d(9, 9, 9)
    o = _amg_only(A, amg_max_coarse=10, amg_pmax=4)
    S = o.scipy(Q_AMG_S, 0, 0)
    P = o.scipy(Q_AMG_P, 0, 0)
    cf = o.cf(0, 0)
    cidx = np.cumsum(cf == 1) - 1
    rowsum = np.asarray(A.sum(axis=1)).ravel()
    Pone = P @ np.ones(P.shape[1])
    for i in range(A.shape[0]):
        cols = P.indices[P.indptr[i]:P.indptr[i + 1]]
        vals = P.data[P.indptr[i]:P.indptr[i + 1]]
        if cf[i] == 1:
            assert cols.tolist() == [cidx[i]] and vals.tolist() == [1.0]
            continue
        assert len(cols) <= 4
        strongC = set(cidx[j] for j in S.indices[S.indptr[i]:S.indptr[i + 1]] if cf[j] == 1)
        assert set(cols.tolist()) <= strongC
        if rowsum[i] == 0 and len(cols):
            assert abs(Pone[i] - 1.0) <= 1e-14


def neumann_elasticity(nx, ny, nz, lam=72.0, mu=72.0):
    """Q1 stiffness of an nx x ny x nz box of unit cells with no boundary
    condition (3 dofs per vertex, vertex-major).  With lam = mu = 72 every
    entry is an integer, so the rigid translations are exact null vectors in
    floating point: within each displacement component every row sums to 0,
    with off-diagonals of both signs."""
    nnx, nny = nx + 1, ny + 1
    K = lam * synth.KLAM + mu * synth.KMU
    rows, cols, vals = [], [], []
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                nodes = [(cx + (a & 1)) + nnx * ((cy + ((a >> 1) & 1)) + nny * (cz + ((a >> 2) & 1)))
                         for a in range(8)]
                for a in range(8):
                    for b in range(8):
                        for i in range(3):
                            for j in range(3):
                                rows.append(3 * nodes[a] + i)
                                cols.append(3 * nodes[b] + j)
                                vals.append(K[3 * a + i, 3 * b + j])
    n = 3 * nnx * nny * (nz + 1)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.eliminate_zeros()
    A.sort_indices()
    return A, np.tile(np.arange(3), n // 3).astype(np.int32)


@pytest.mark.parametrize("pmax", [0, 4])
def test_interpolation_preserves_constants_with_positive_couplings(pmax):
    """Direct interpolation on the elasticity operator (zero row sums within
    each component, off-diagonals of both signs), with a strength graph that
    also marks positive couplings strong.  Where a row has a positive strong C
    neighbour its positive entries are scaled by beta = sum_pos / sum_pos_C;
    where it has none they are lumped into the diagonal.  Both branches must
    interpolate the constant exactly: P 1 = 1 on every F row with a negative
    strong C neighbour, with and without truncation to P_max (rows rescaled to
    keep their sums).  A sign slip in either branch, or a wrong lumping rule,
    breaks this."""
    A, comp = neumann_elasticity(3, 3, 2)
    n = A.shape[0]
    Ac = A.tocoo()
    off = (Ac.row != Ac.col) & (comp[Ac.row] == comp[Ac.col])
    S = sp.csr_matrix((np.ones(off.sum()), (Ac.row[off], Ac.col[off])), shape=(n, n))
    node = np.arange(n) // 3
    cf = np.where(node % 3 == 0, 1, -1).astype(np.int8)
    P = oracle.interp(A, S, cf, comp=comp, pmax=pmax)
    Pone = P @ np.ones(P.shape[1])
    beta_rows = lump_rows = 0
    for i in np.nonzero(cf == -1)[0]:
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        strongC = [(j, v) for j, v in zip(cols, vals)
                   if j != i and comp[j] == comp[i] and cf[j] == 1]
        if not any(v < 0 for _, v in strongC):
            continue
        pos_same = any(v > 0 for j, v in zip(cols, vals) if j != i and comp[j] == comp[i])
        if any(v > 0 for _, v in strongC):
            beta_rows += 1
        elif pos_same:
            lump_rows += 1
        assert abs(Pone[i] - 1.0) <= 1e-13, (i, Pone[i])
    assert beta_rows > 0 and lump_rows > 0, (beta_rows, lump_rows)
    if pmax:
        assert np.diff(P.indptr).max() <= pmax


def test_pmis_weight_counts_the_points_a_point_influences():
    """PMIS weights w_i = |S^T_i| + u_i (the number of points that depend
    strongly on i).  On directed stars -- every leaf depends on its centre,
    the centre on nothing -- the centre has the largest weight, becomes C, and
    every leaf then has a C point in S_i and becomes F: C = the centres.  (A
    weight |S_i| would instead make every leaf C first.)"""
    stars = [7, 4, 1]
    rows, cols, centres = [], [], []
    base = 0
    for k in stars:
        centres.append(base)
        for leaf in range(base + 1, base + 1 + k):
            rows.append(leaf)
            cols.append(base)
        base += k + 1
    S = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(base, base))
    for seed in (0, 1, 12345):
        cf = oracle.pmis(S, seed=seed)
        want = -np.ones(base, dtype=np.int8)
        want[centres] = 1
        assert np.array_equal(cf, want), (seed, cf)


def directed_star_matrix(leaves=7):
    """Scalar matrix whose strength graph is a directed star: each leaf row has
    -1 to the centre (its only negative coupling), the centre row has only
    positive couplings (so S_centre is empty)."""
    n = leaves + 1
    A = sp.lil_matrix((n, n))
    A[0, 0] = 4.0
    for i in range(1, n):
        A[i, i] = 2.0
        A[i, 0] = -1.0
        A[0, i] = 0.25
    return sp.csr_matrix(A)


def test_pmis_through_the_amg_setup_on_a_directed_star():
    """The same closed form through the AMG setup: strength from the matrix,
    PMIS, direct interpolation (each leaf interpolates from the centre with
    weight -a_i0 / a_ii = 1/2)."""
    A = directed_star_matrix()
    o = _amg_only(A, amg_max_coarse=1)
    cf = o.cf(0, 0)
    assert cf[0] == 1 and np.all(cf[1:] == -1)
    P = o.scipy(Q_AMG_P, 0, 0).toarray()
    assert np.array_equal(P[:, 0], np.r_[1.0, np.full(7, 0.5)])


def test_interpolation_without_truncation_keeps_all_strong_c():
    A = poisson3d(7, 7, 7)
    o = _amg_only(A, amg_max_coarse=10, amg_pmax=0)
    S = o.scipy(Q_AMG_S, 0, 0)
    P = o.scipy(Q_AMG_P, 0, 0)
    cf = o.cf(0, 0)
    for i in np.nonzero(cf == -1)[0]:
        nC = sum(cf[j] == 1 for j in S.indices[S.indptr[i]:S.indptr[i + 1]])
        assert P.indptr[i + 1] - P.indptr[i] == nC


def test_galerkin_coarse_operator_is_dense_triple_product():
    p = synth.config(1)
    o = oracle.Oracle(p)
    for slot in (0, 1):
        for k in range(o.amg_levels(slot) - 1):
            A = o.scipy(Q_AMG_A, slot, k).toarray()
            P = o.scipy(Q_AMG_P, slot, k).toarray()
            R = o.scipy(Q_AMG_R, slot, k).toarray()
            assert np.array_equal(R, P.T)
            Ac = o.scipy(Q_AMG_A, slot, k + 1).toarray()
            ref = P.T @ A @ P
            assert np.abs(Ac - ref).max() <= 1e-12 * np.abs(ref).max()


def test_l1_diagonal():
    A = poisson3d(5, 4, 3)
    o = _amg_only(A, amg_max_coarse=5)
    Ad = A.toarray()
    want = np.diag(Ad) + (np.abs(Ad).sum(axis=1) - np.abs(np.diag(Ad)))
    assert np.allclose(o.l1(0, 0), want, rtol=1e-15)


def test_coarsest_level_is_exact_solve():
    A = poisson3d(6, 5, 4)
    o = _amg_only(A, amg_max_coarse=1000)
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x = o.vcycle(0, b)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-12, atol=1e-12)


def test_vcycle_symmetric_and_contracting_on_poisson():
    """With R = P^T and one l1-Jacobi sweep before and after, the V-cycle is a
    symmetric operator B, and the error propagator I - BA contracts."""
    A = poisson3d(8, 8, 8)
    o = _amg_only(A, amg_max_coarse=20)
    assert o.amg_levels(0) >= 3
    n = A.shape[0]
    B = np.column_stack([o.vcycle(0, e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh((B + B.T) / 2).min() > 0
    E = np.eye(n) - B @ A.toarray()
    rho = np.abs(np.linalg.eigvals(E)).max()
    assert rho < 0.9


def test_jacobian_product_equals_library_product():
    """The Arnoldi step's y = A x (with and without a hierarchy) against
    scipy's sparse product, to rounding: |dy_i| <= 1e-14 sum_j |a_ij x_j|."""
    p = synth.two_phase(7, 6, 5, seed=2)
    A = p.to_scipy()
    x = np.random.default_rng(9).standard_normal(p.n)
    ref = A @ x
    bound = 1e-14 * (abs(A) @ np.abs(x))
    for y in (oracle.Oracle(p).matvec(x), oracle.csr_spmv(p.row_ptr, p.col, p.val, x)):
        assert np.all(np.abs(y - ref) <= bound)


# --------------------------------------------------------------- full solves
def test_single_phase_solve_matches_direct_solver():
    p = synth.config(1)
    o = oracle.Oracle(p)
    r = o.fgmres(p.rhs, restart=50, maxit=500, rtol=1e-8)
    assert r["status"] == 0 and r["relres"] <= 1e-8
    x = sla.spsolve(p.to_scipy().tocsc(), p.rhs)
    assert np.linalg.norm(r["x"] - x) <= 1e-6 * np.linalg.norm(x)


def test_two_phase_solve_matches_direct_solver():
    p = synth.two_phase(10, 9, 6)
    o = oracle.Oracle(p)
    r = o.fgmres(p.rhs, restart=50, maxit=500, rtol=1e-8)
    assert r["status"] == 0 and r["relres"] <= 1e-8
    x = sla.spsolve(p.to_scipy().tocsc(), p.rhs)
    assert np.linalg.norm(r["x"] - x) <= 1e-6 * np.linalg.norm(x)
    A = p.to_scipy()
    assert np.linalg.norm(p.rhs - A @ r["x"]) <= 1e-8 * np.linalg.norm(p.rhs) * 1.0001


def test_restarted_fgmres_converges():
    p = synth.two_phase(8, 8, 4)
    o = oracle.Oracle(p)
    r = o.fgmres(p.rhs, restart=5, maxit=500, rtol=1e-8)
    assert r["status"] == 0 and r["relres"] <= 1e-8


# ---------------------------------------------------------------------------
# Operator variants of Sec. 5.1: Jacobi restriction, MGR-post, point-block D_FF
# ---------------------------------------------------------------------------
def _dense_blocks(p, level_mask=1):
    """Dense A and the F / C index sets of the first reduction (F = u)."""
    A = p.to_scipy().toarray()
    F = np.nonzero(((level_mask >> p.dof_label) & 1) == 1)[0]
    C = np.nonzero(((level_mask >> p.dof_label) & 1) == 0)[0]
    return A, F, C


def _point_block_inverse(A, F, node):
    """D_FF^-1 with D_FF = blocks of consecutive F dofs sharing dof_node."""
    nF = len(F)
    Bd = np.zeros((nF, nF))
    f = 0
    while f < nF:
        g = f + 1
        while g < nF and node[F[g]] == node[F[f]]:
            g += 1
        Bd[f:g, f:g] = np.linalg.inv(A[np.ix_(F[f:g], F[f:g])])
        f = g
    return Bd


@pytest.mark.parametrize("block", [0, 1])
def test_jacobi_restriction_gives_the_full_triple_product(block):
    # Sec. 5.1: W_r = -A_CF D^-1, W_p = -D^-1 A_FC; with no dropping the coarse
    # operator must be R~ A P~ = A_CC + W_r A_FC + A_CF W_p + W_r A_FF W_p.
    # lognormal E: the nodal 3x3 blocks of A_uu are not diagonal
    p = synth.two_phase(3, 3, 2, seed=1, E_sigma=1.0)
    o = oracle.Oracle(p, num_levels=1, f_label_mask=[1], frelax=[0], frelax_sweeps=[1],
                      nmax_drop=[-1], global_sweeps=[0], restrict_jacobi=[1], dff_block=[block])
    A, F, C = _dense_blocks(p)
    Aff, Afc, Acf, Acc = (A[np.ix_(F, F)], A[np.ix_(F, C)], A[np.ix_(C, F)], A[np.ix_(C, C)])
    Dinv = _point_block_inverse(A, F, p.dof_node) if block else np.diag(1.0 / np.diag(Aff))
    Wp = -Dinv @ Afc
    Wr = -Acf @ Dinv
    rap = Acc + Wr @ Afc + Acf @ Wp + Wr @ Aff @ Wp
    S = o.scipy(oracle.Q_MGR_S, 0).toarray()
    assert np.abs(S - rap).max() <= 1e-12 * np.abs(rap).max()
    assert np.abs(o.scipy(oracle.Q_MGR_WR, 0).toarray() - Wr).max() <= 1e-14 * np.abs(Wr).max()
    assert np.abs(o.scipy(oracle.Q_MGR_W, 0).toarray() - Wp).max() <= 1e-14 * np.abs(Wp).max()


def test_point_block_dff_interpolation_and_coarse_grid():
    # D_FF as the 3x3 nodal blocks of A_uu (and 1x1 for s): W_p = -Bd A_FC and
    # S = A_CC - A_CF Bd A_FC, Bd = block inverses, with no dropping.
    # lognormal E: with a uniform modulus the free nodes' 3x3 self-blocks are
    # diagonal on this mesh and both choices of D_FF coincide
    p = synth.two_phase(3, 3, 2, seed=2, E_sigma=1.0)
    o = oracle.Oracle(p, num_levels=1, f_label_mask=[1], frelax=[0], frelax_sweeps=[1],
                      nmax_drop=[-1], global_sweeps=[0], dff_block=[1])
    A, F, C = _dense_blocks(p)
    Bd = _point_block_inverse(A, F, p.dof_node)
    assert np.abs(o.scipy(oracle.Q_MGR_BD, 0).toarray() - Bd).max() <= 1e-13 * np.abs(Bd).max()
    Wp = -Bd @ A[np.ix_(F, C)]
    S_ref = A[np.ix_(C, C)] + A[np.ix_(C, F)] @ Wp
    assert np.abs(o.scipy(oracle.Q_MGR_W, 0).toarray() - Wp).max() <= 1e-13 * np.abs(Wp).max()
    assert np.abs(o.scipy(oracle.Q_MGR_S, 0).toarray() - S_ref).max() <= 1e-12 * np.abs(S_ref).max()
    # blocks are 3x3 on u: the interpolation differs from the pointwise one
    o1 = oracle.Oracle(p, num_levels=1, f_label_mask=[1], frelax=[0], frelax_sweeps=[1],
                       nmax_drop=[-1], global_sweeps=[0])
    assert np.abs(o1.scipy(oracle.Q_MGR_W, 0).toarray() - Wp).max() > 1e-6 * np.abs(Wp).max()


@pytest.mark.parametrize("post", [0, 1])
@pytest.mark.parametrize("jac", [0, 1])
def test_mgr_pre_and_post_error_propagation(post, jac):
    # Eqs. MGR-pre / MGR-post with exact components: F-relaxation
    # M_FF^-1 = Q (Q^T A Q)^-1 Q^T and coarse solve (R~ A P~)^-1 (both AMGs are
    # a single dense level on this tiny system, and nothing is dropped), so
    #   pre:  I - M^-1 A = (I - P~ M_CC^-1 R~ A)(I - M_FF^-1 A)
    #   post: I - M^-1 A = (I - M_FF^-1 A)(I - P~ M_CC^-1 R~ A).
    p = synth.two_phase(2, 2, 2, seed=3)
    o = oracle.Oracle(p, num_levels=1, f_label_mask=[1], frelax=[0], frelax_sweeps=[1],
                      nmax_drop=[-1], global_sweeps=[0], amg_max_coarse=200,
                      restrict_jacobi=[jac], frelax_post=[post])
    assert o.amg_levels(0) == 1 and o.amg_levels(1) == 1
    A, F, C = _dense_blocks(p)
    n, nF, nC = p.n, len(F), len(C)
    Dinv = np.diag(1.0 / np.diag(A[np.ix_(F, F)]))
    Pt = np.zeros((n, nC))
    Pt[np.ix_(F, np.arange(nC))] = -Dinv @ A[np.ix_(F, C)]
    Pt[C, np.arange(nC)] = 1.0
    Rt = np.zeros((nC, n))
    Rt[np.arange(nC), C] = 1.0
    if jac:
        Rt[np.ix_(np.arange(nC), F)] = -A[np.ix_(C, F)] @ Dinv
    Mcc_inv = np.linalg.inv(Rt @ A @ Pt)
    Q = np.zeros((n, nF))
    Q[F, np.arange(nF)] = 1.0
    Mff_inv = Q @ np.linalg.inv(Q.T @ A @ Q) @ Q.T
    I = np.eye(n)
    Ecg = I - Pt @ Mcc_inv @ Rt @ A
    Ef = I - Mff_inv @ A
    E_ref = Ef @ Ecg if post else Ecg @ Ef
    MinvA = np.column_stack([o.apply(A[:, j]) for j in range(n)])
    E = I - MinvA
    assert np.abs(E - E_ref).max() <= 1e-9
    # the two orderings are different operators
    E_other = Ecg @ Ef if post else Ef @ Ecg
    assert np.abs(E - E_other).max() > 1e-6


# ---------------------------------------------------------------------------
# Global smoother: point-block Jacobi and multicolour point-block Gauss-Seidel
# ---------------------------------------------------------------------------
def _level1_blocks(o, p):
    """Level-1 operator S_1 (dense) and its point blocks (runs of equal node)."""
    S = o.scipy(oracle.Q_MGR_A, 1).toarray()
    node = p.dof_node[p.dof_label != 0]           # level-1 dofs: s and p of each cell
    blocks, i = [], 0
    while i < len(node):
        j = i + 1
        while j < len(node) and node[j] == node[i]:
            j += 1
        blocks.append(np.arange(i, j))
        i = j
    return S, blocks


def test_multicolour_coloring_is_proper():
    p = synth.two_phase(6, 5, 4, seed=8)
    o = oracle.Oracle(p, global_smoother=[0, 1])
    S, blocks = _level1_blocks(o, p)
    colors, nc = o.block_colors(1)
    assert len(colors) == len(blocks) and colors.min() == 0 and colors.max() == nc - 1
    owner = np.empty(S.shape[0], dtype=np.int64)
    for k, b in enumerate(blocks):
        owner[b] = k
    rows, cols = np.nonzero(S)
    adj = owner[rows] != owner[cols]
    assert np.all(colors[owner[rows[adj]]] != colors[owner[cols[adj]]])
    assert 3 <= nc <= 40


@pytest.mark.parametrize("sweeps", [1, 3])
def test_multicolour_gauss_seidel_is_block_gauss_seidel(sweeps):
    # Forward block Gauss-Seidel in the ordering (colour, block): with the
    # block lower triangle L_D (block diagonal included) of that ordering,
    # z_{k+1} = z_k + L_D^-1 (v - S z_k) from z_0 = 0 -- the textbook sweep.
    p = synth.two_phase(4, 4, 3, seed=9)
    o = oracle.Oracle(p, global_smoother=[0, 1], global_sweeps=[0, sweeps])
    S, blocks = _level1_blocks(o, p)
    colors, _ = o.block_colors(1)
    order = sorted(range(len(blocks)), key=lambda k: (colors[k], k))
    rank = np.empty(len(blocks), dtype=np.int64)
    rank[order] = np.arange(len(blocks))
    owner = np.empty(S.shape[0], dtype=np.int64)
    for k, b in enumerate(blocks):
        owner[b] = k
    LD = np.where(rank[owner][:, None] >= rank[owner][None, :], S, 0.0)
    v = np.random.default_rng(3).standard_normal(S.shape[0])
    z = np.zeros_like(v)
    for _ in range(sweeps):
        z = z + np.linalg.solve(LD, v - S @ z)
    got = o.global_relax(1, v)
    assert np.abs(got - z).max() <= 1e-11 * np.abs(z).max()


def test_block_jacobi_smoother_is_block_jacobi():
    p = synth.two_phase(4, 4, 3, seed=9)
    o = oracle.Oracle(p, global_sweeps=[0, 3])
    S, blocks = _level1_blocks(o, p)
    D = np.zeros_like(S)
    for b in blocks:
        D[np.ix_(b, b)] = S[np.ix_(b, b)]
    v = np.random.default_rng(4).standard_normal(S.shape[0])
    z = np.zeros_like(v)
    for _ in range(3):
        z = z + np.linalg.solve(D, v - S @ z)
    got = o.global_relax(1, v)
    assert np.abs(got - z).max() <= 1e-11 * np.abs(z).max()


# ---------------------------------------------------------------------------
# Aggressive (two-stage) coarsening of the first A_uu AMG level
# ---------------------------------------------------------------------------
def test_aggressive_level_composes_two_stages():
    # With no truncation the aggressive interpolation must be P = P1 P2: P1 is
    # the ordinary first level's interpolation (same first stage), and since
    # P1 has identity rows at its C points, P2 = P[C1 rows]; P2 is the identity
    # on the final C points, C2 is a subset of C1, and the next operator is the
    # Galerkin product P^T A P.
    p = synth.two_phase(8, 7, 5, seed=6)
    base = oracle.Oracle(p, amg_pmax=0)
    agg = oracle.Oracle(p, amg_pmax=0, agg_levels=[1, 0, 0])
    A = agg.scipy(oracle.Q_AMG_A, 0, 0).toarray()
    P1 = base.scipy(oracle.Q_AMG_P, 0, 0).toarray()
    P = agg.scipy(oracle.Q_AMG_P, 0, 0).toarray()
    cf1, cf = base.cf(0, 0), agg.cf(0, 0)
    C1, C = np.nonzero(cf1 == 1)[0], np.nonzero(cf == 1)[0]
    assert set(C) < set(C1) and len(C) < len(C1)
    P2 = P[C1, :]
    assert np.abs(P - P1 @ P2).max() <= 1e-13 * np.abs(P).max()
    pos = {c: t for t, c in enumerate(C1)}
    assert np.array_equal(P2[[pos[c] for c in C], :], np.eye(len(C)))
    Ac = agg.scipy(oracle.Q_AMG_A, 0, 1).toarray()
    assert np.abs(Ac - P.T @ A @ P).max() <= 1e-12 * np.abs(Ac).max()
    # the intermediate Galerkin operator is the ordinary hierarchy's level 1
    A1 = base.scipy(oracle.Q_AMG_A, 0, 1).toarray()
    assert np.abs(A1 - P1.T @ A @ P1).max() <= 1e-12 * np.abs(A1).max()


def test_aggressive_level_truncation_and_hierarchy():
    p = synth.two_phase(8, 7, 5, seed=6)
    base = oracle.Oracle(p)
    agg = oracle.Oracle(p, agg_levels=[1, 0, 0])
    P = agg.scipy(oracle.Q_AMG_P, 0, 0)
    assert np.diff(P.indptr).max() <= 4                        # P_max = 4
    C = np.nonzero(agg.cf(0, 0) == 1)[0]
    Pd = P.toarray()
    assert np.array_equal(Pd[C, :], np.eye(len(C)))
    n0 = [base.scipy(oracle.Q_AMG_A, 0, k).shape[0] for k in range(base.amg_levels(0))]
    n1 = [agg.scipy(oracle.Q_AMG_A, 0, k).shape[0] for k in range(agg.amg_levels(0))]
    assert n1[0] == n0[0] and n1[1] < n0[1] // 3               # one aggressive step
    assert agg.amg_levels(2) == base.amg_levels(2)             # other AMGs untouched
    r = agg.fgmres(p.rhs)
    assert r["status"] == 0 and r["relres"] <= 1e-8


# ---------------------------------------------------------------------------
# ILU(1) global smoother
# ---------------------------------------------------------------------------
def _ilu_parts(o, l):
    F = o.scipy(oracle.Q_MGR_ILU, l)
    Fd = F.toarray()
    n = Fd.shape[0]
    return F, np.tril(Fd, -1) + np.eye(n), np.triu(Fd)


def test_ilu1_pattern_and_defining_property():
    # ILU on a pattern P: (L U)_ij = a_ij for every (i, j) in P, and P for
    # level 1 is pattern(A) + pattern(L_A U_A) (strict triangles of A).
    import scipy.sparse as sp
    p = synth.two_phase(5, 4, 3, seed=7)
    o = oracle.Oracle(p, global_smoother=[0, 2])
    S = o.scipy(oracle.Q_MGR_A, 1)
    F, L, U = _ilu_parts(o, 1)
    pat_a = (abs(S) > 0).astype(np.int8)
    lo = sp.tril(pat_a, -1, format="csr")
    up = sp.triu(pat_a, 1, format="csr")
    want = ((pat_a + (lo @ up)) > 0).astype(np.int8).tocsr()
    want.sort_indices()
    got = sp.csr_matrix((np.ones(F.nnz), F.indices, F.indptr), shape=F.shape)
    assert np.array_equal(got.indptr, want.indptr) and np.array_equal(got.indices, want.indices)
    LU = L @ U
    mask = want.toarray() > 0
    Sd = S.toarray()
    assert np.abs((LU - Sd)[mask]).max() <= 1e-13 * np.abs(Sd).max()
    assert np.abs((LU - Sd)[~mask]).max() > 1e-8 * np.abs(Sd).max()   # incomplete


def test_ilu1_without_fill_is_the_exact_lu():
    # When pattern(L_A U_A) adds nothing to pattern(A), elimination creates
    # no fill at any level, so ILU(1) is the exact LU factorization.  The
    # level-1 operator of a single column of cells (1 x 1 x nz) is banded
    # and has that property.
    p = synth.two_phase(1, 1, 12, seed=1)
    o = oracle.Oracle(p, global_smoother=[0, 2])
    S = o.scipy(oracle.Q_MGR_A, 1)
    F, L, U = _ilu_parts(o, 1)
    assert F.nnz == (abs(S) > 0).sum()
    Sd = S.toarray()
    assert np.abs(L @ U - Sd).max() <= 1e-12 * np.abs(Sd).max()
    assert np.abs(np.linalg.solve(L @ U, np.ones(len(Sd))) -
                  np.linalg.solve(Sd, np.ones(len(Sd)))).max() < 1e-9


@pytest.mark.parametrize("solve_sweeps", [3, 400])
def test_ilu1_smoother_sweep(solve_sweeps):
    # One smoother sweep from zero: z = w with L y = v, U w = y solved by
    # Jacobi iterations y <- v - (L - I) y, w <- D_U^-1 (y - (U - D_U) w),
    # starting from y = v, w = D_U^-1 y; with enough iterations the solves are
    # exact and z = (L U)^-1 v.
    p = synth.two_phase(4, 3, 3, seed=2)
    o = oracle.Oracle(p, global_smoother=[0, 2], global_sweeps=[0, 1],
                      ilu_solve_sweeps=solve_sweeps)
    F, L, U = _ilu_parts(o, 1)
    n = L.shape[0]
    v = np.random.default_rng(1).standard_normal(n)
    got = o.global_relax(1, v)
    if solve_sweeps >= n:
        want = np.linalg.solve(L @ U, v)
    else:
        Ls, D, Us = L - np.eye(n), np.diag(np.diag(U)), U - np.diag(np.diag(U))
        y = v.copy()
        for _ in range(solve_sweeps):
            y = v - Ls @ y
        w = np.linalg.solve(D, y)
        for _ in range(solve_sweeps):
            w = np.linalg.solve(D, y - Us @ w)
        want = w
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_ilu1_two_sweeps_are_a_stationary_iteration():
    # Two sweeps from zero: z1 = B v, z2 = z1 + B (v - A z1), B the one-sweep
    # operator (approximate triangular solves); with exact solves, z2 is two
    # steps of the iteration z <- z + (LU)^-1 (v - A z).
    p = synth.two_phase(4, 3, 3, seed=5)
    o1 = oracle.Oracle(p, global_smoother=[0, 2], global_sweeps=[0, 1], ilu_solve_sweeps=400)
    o2 = oracle.Oracle(p, global_smoother=[0, 2], global_sweeps=[0, 2], ilu_solve_sweeps=400)
    A = o1.scipy(oracle.Q_MGR_A, 1).toarray()
    F, L, U = _ilu_parts(o1, 1)
    n = A.shape[0]
    v = np.random.default_rng(3).standard_normal(n)
    z1 = np.linalg.solve(L @ U, v)
    z2 = z1 + np.linalg.solve(L @ U, v - A @ z1)
    assert np.abs(o1.global_relax(1, v) - z1).max() <= 1e-10 * np.abs(z1).max()
    assert np.abs(o2.global_relax(1, v) - z2).max() <= 1e-10 * np.abs(z2).max()
    # the second sweep reduces the error of the smoother (A z = v) on this SPD-like block
    e1 = np.linalg.norm(v - A @ z1)
    e2 = np.linalg.norm(v - A @ z2)
    assert e2 < e1


def test_fgmres_residual_history_is_the_krylov_minimum():
    # With a fixed preconditioner M, flexible GMRES is right-preconditioned
    # GMRES: after k steps its residual is min ||b - A M^-1 y|| over y in the
    # Krylov space K_k(A M^-1, b).  The minimum is formed here from the dense
    # operator A M^-1 (M^-1 applied to every unit vector) with a QR of the
    # Krylov basis, independently of the oracle's Arnoldi and Givens updates.
    p = synth.two_phase(4, 3, 3, seed=11)
    o = oracle.Oracle(p)
    n = p.n
    A = p.to_scipy().toarray()
    Minv = np.column_stack([o.apply(e) for e in np.eye(n)])
    B = A @ Minv
    b = p.rhs / np.linalg.norm(p.rhs)
    r = o.fgmres(b, restart=50, maxit=30, rtol=1e-12, hist_cap=40)
    hist = r["hist"]
    K = np.empty((n, 0))
    v = b.copy()
    for k in range(1, min(len(hist) - 1, 12) + 1):
        K = np.column_stack([K, v])
        Q, _ = np.linalg.qr(K)            # orthonormal basis of K_k
        Q, _ = np.linalg.qr(Q)
        BQ = B @ Q
        y, *_ = np.linalg.lstsq(BQ, b, rcond=None)
        res = np.linalg.norm(b - BQ @ y)
        assert abs(hist[k] - res) <= 1e-6 * max(res, 1e-8), (k, hist[k], res)
        v = B @ Q[:, -1]
    assert np.all(np.diff(hist[:13]) <= 1e-14)     # non-increasing within a cycle


def test_fingerprint_comparison_recovers_a_known_error():
    """The stored-fingerprint comparison (oracle/fingerprint.py): exact on the
    sample, and the probe estimate within its ~18% spread (16 probes) of the
    true relative error of a planted perturbation."""
    from oracle import fingerprint
    n = 20000
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n)
    idx = np.sort(rng.choice(n, 500, replace=False))
    fp = dict(n=n, norm2=float(np.linalg.norm(x)), iters=1, probe_seed=1000, sample_idx=idx,
              sample_x=x[idx],
              probes=np.array([np.random.default_rng(1000 + k).standard_normal(n) @ x
                               for k in range(16)]))
    assert fingerprint.compare(x, fp)["probe_rel"] <= 1e-13
    e = 1e-7 * rng.standard_normal(n)
    c = fingerprint.compare(x + e, fp)
    true = np.linalg.norm(e) / np.linalg.norm(x)
    assert abs(c["sample_rel"] - np.linalg.norm(e[idx]) / np.linalg.norm(x[idx])) <= 1e-12
    assert 0.5 * true <= c["probe_rel"] <= 1.5 * true
