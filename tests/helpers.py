"""Small seeded test matrices with the field structure of the paper's Jacobian.

These builders hold no solver arithmetic: they only lay out random sparse
blocks so that the algebraic identities of the method (Sec. 5.1) can be tested
on inputs small enough for dense linear algebra.
"""
import numpy as np
import scipy.sparse as sp

from paper_1904_05960_gb300.synth import Problem


def _rand_sparse(rng, nr, nc, density, scale=1.0):
    m = sp.random(nr, nc, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1.0, 1.0, size=k) * scale)
    return m


def to_problem(A, label, node, comp, seed=0, two_phase=True):
    A = sp.csr_matrix(A)
    A.sort_indices()
    A.eliminate_zeros()
    n = A.shape[0]
    return Problem(n=n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32),
                   val=A.data.astype(np.float64), dof_label=np.asarray(label, np.int32),
                   dof_node=np.asarray(node, np.int32), dof_comp=np.asarray(comp, np.int32),
                   rhs=np.random.default_rng(seed + 1).standard_normal(n),
                   meta=dict(two_phase=two_phase))


def labeled_system(seed=0, n_nodes=20, n_cells=16, two_phase=True, diag_uu=False,
                   diag_ss=False, block_diag_flow=False, density=0.15):
    """Random nonsingular system with u (3 per node) then cell dofs (s,p or p).

    diag_uu: A_uu diagonal (then D_FF = A_FF at the first reduction);
    diag_ss: A_ss diagonal and A_us = 0 (then diag of the reduced s-block is
             the whole block at the second reduction);
    block_diag_flow: the flow block couples only the dofs of one cell.
    """
    rng = np.random.default_rng(seed)
    nu = 3 * n_nodes
    ncd = 2 if two_phase else 1
    nf = ncd * n_cells
    if diag_uu:
        Auu = sp.diags(rng.uniform(2.0, 4.0, nu))
    else:
        B = _rand_sparse(rng, nu, nu, density)
        Auu = B @ B.T + sp.diags(np.full(nu, 3.0))
    Auc = _rand_sparse(rng, nu, nf, density)
    Acu = _rand_sparse(rng, nf, nu, density)
    if two_phase:
        Auc = Auc.tolil()
        Auc[:, 0::2] = 0.0            # A_us = 0 (no gravity)
        Auc = Auc.tocsr()
    if block_diag_flow:
        blocks = [rng.uniform(-1, 1, (ncd, ncd)) + 4 * np.eye(ncd) for _ in range(n_cells)]
        Acc = sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")
    else:
        Acc = _rand_sparse(rng, nf, nf, density) + sp.diags(rng.uniform(4.0, 6.0, nf))
        if diag_ss and two_phase:
            Acc = Acc.tolil()
            for i in range(0, nf, 2):
                for j in range(0, nf, 2):
                    if i != j:
                        Acc[i, j] = 0.0
            Acc = Acc.tocsr()
    A = sp.bmat([[Auu, Auc], [Acu, Acc]], format="csr")
    label = np.zeros(nu + nf, np.int32)
    node = np.zeros(nu + nf, np.int32)
    comp = np.zeros(nu + nf, np.int32)
    node[:nu] = np.repeat(np.arange(n_nodes), 3)
    comp[:nu] = np.tile(np.arange(3), n_nodes)
    if two_phase:
        label[nu::2] = 1
        label[nu + 1::2] = 2
        node[nu:] = n_nodes + np.repeat(np.arange(n_cells), 2)
        comp[nu:] = np.tile(np.arange(2), n_cells)
    else:
        label[nu:] = 2
        node[nu:] = n_nodes + np.arange(n_cells)
    # keep structural entries explicit for the dense comparisons
    return to_problem(A, label, node, comp, seed=seed, two_phase=two_phase)


def poisson3d(nx, ny, nz, shift_first=1.0):
    """7-point graph Laplacian (zero row sums) with one diagonal entry shifted
    so the matrix is SPD."""
    def lap1(n):
        return sp.diags([-np.ones(n - 1), np.r_[1, 2 * np.ones(n - 2), 1], -np.ones(n - 1)],
                        [-1, 0, 1])
    Ix, Iy, Iz = sp.eye(nx), sp.eye(ny), sp.eye(nz)
    A = (sp.kron(Iz, sp.kron(Iy, lap1(nx))) + sp.kron(Iz, sp.kron(lap1(ny), Ix))
         + sp.kron(lap1(nz), sp.kron(Iy, Ix))).tocsr()
    A = A + sp.csr_matrix(([shift_first], ([0], [0])), shape=A.shape)
    return A.tocsr()


def scalar_problem(A, seed=0):
    n = A.shape[0]
    return to_problem(A, np.full(n, 2), np.arange(n), np.zeros(n), seed=seed, two_phase=False)
