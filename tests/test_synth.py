"""Pins of the synthetic Jacobian generator against the discretisation's
textbook properties (Sec. 3: Q1 elasticity, TPFA with upwinding, Biot coupling)."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1904_05960_gb300 import synth


def _gauss_element(E=1.0, nu=0.25):
    """Independent 2x2x2 Gauss quadrature of the unit-cube Q1 stiffness."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    Dm = np.zeros((6, 6))
    Dm[:3, :3] = lam
    Dm[np.arange(3), np.arange(3)] += 2 * mu
    Dm[np.arange(3, 6), np.arange(3, 6)] = mu
    K = np.zeros((24, 24))
    for x in g:
        for y in g:
            for z in g:
                B = np.zeros((6, 24))
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    fx = (x if ax else 1 - x); fy = (y if ay else 1 - y); fz = (z if az else 1 - z)
                    dx = (1 if ax else -1) * fy * fz
                    dy = fx * (1 if ay else -1) * fz
                    dz = fx * fy * (1 if az else -1)
                    c = 3 * a
                    B[0, c] = dx; B[1, c + 1] = dy; B[2, c + 2] = dz
                    B[3, c] = dy; B[3, c + 1] = dx
                    B[4, c + 1] = dz; B[4, c + 2] = dy
                    B[5, c] = dz; B[5, c + 2] = dx
                K += B.T @ Dm @ B / 8.0
    return K


def test_element_stiffness_matches_gauss_quadrature():
    nu = 0.25
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    K = lam * synth.KLAM + mu * synth.KMU
    assert np.allclose(K, _gauss_element(1.0, nu), rtol=1e-13, atol=1e-14)


def test_element_rigid_body_modes_exact():
    """Six rigid-body modes span the null space of the exact element matrices."""
    Kl, Km, Q = synth.q1_element_matrices()
    modes = []
    for t in range(3):
        m = [Fraction(0)] * 24
        for a in range(8):
            m[3 * a + t] = Fraction(1)
        modes.append(m)
    for (i, j) in ((0, 1), (1, 2), (2, 0)):       # rotation in the (i, j) plane
        m = [Fraction(0)] * 24
        for a in range(8):
            c = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
            m[3 * a + i] = Fraction(-c[j])
            m[3 * a + j] = Fraction(c[i])
        modes.append(m)
    for K in (Kl, Km):
        for r in range(24):
            for m in modes:
                assert sum(K[r][c] * m[c] for c in range(24)) == 0
    for r in range(24):
        for c in range(24):
            assert Kl[r][c] == Kl[c][r] and Km[r][c] == Km[c][r]
    Kf = np.array([[float(x) for x in row] for row in Km])
    assert np.linalg.matrix_rank(Kf) == 18


def test_divergence_coupling_exact():
    """Q = int grad N: corner values sum to zero per direction and Q applied to
    the field u = x e_x gives the cell volume (int div u = 1)."""
    _, _, Q = synth.q1_element_matrices()
    for i in range(3):
        assert sum(Q[3 * a + i] for a in range(8)) == 0
    ux = [Fraction(a & 1) if i == 0 else Fraction(0) for a in range(8) for i in range(3)]
    assert sum(q * u for q, u in zip(Q, ux)) == 1


def test_config1_sizes_symmetry_and_positivity():
    p = synth.config(1)
    assert (p.n, p.meta["n_u"], p.meta["n_cells"]) == (2699, 2187, 512)
    A = p.to_scipy()
    nu = p.meta["n_u"]
    Auu = A[:nu, :nu]
    assert abs(Auu - Auu.T).max() == 0.0
    assert np.linalg.eigvalsh(Auu.toarray()).min() > 0
    for r in range(p.n):
        cols = p.col[p.row_ptr[r]:p.row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0)


def test_dof_counts_formula():
    for nx, ny, nz in ((64, 64, 32), (128, 128, 64), (256, 256, 96)):
        nu = 3 * (nx + 1) * (ny + 1) * (nz + 1)
        cells = nx * ny * nz
        assert nu + 2 * cells == {64: 680419, 128: 5342147, 256: 31803171}[nx]
    p = synth.two_phase(6, 5, 4)
    assert p.n == 3 * 7 * 6 * 5 + 2 * 120


def test_single_phase_tpfa_rows_sum_to_zero_in_interior():
    p = synth.single_phase(6, 5, 4)
    A = p.to_scipy()
    nu = p.meta["n_u"]
    App = A[nu:, nu:].toarray()
    assert np.allclose(App, App.T)
    cz = np.arange(p.meta["n_cells"]) // (6 * 5)
    interior = cz < 3
    rs = App.sum(axis=1)
    assert np.abs(rs[interior]).max() <= 1e-12 * np.abs(App).max()
    assert np.all(rs[~interior] > 0)


def test_two_phase_flux_jacobian_is_conservative():
    """With accumulation and wells removed, each phase's flux Jacobian has zero
    column sums over all cells (fluxes cancel in pairs)."""
    rng = np.random.default_rng(0)
    nx, ny, nz = 5, 4, 3
    perm = np.exp(rng.standard_normal((nz, ny, nx)))
    sat = rng.uniform(0.2, 0.8, (nz, ny, nx))
    p = synth.build_poromechanics(nx, ny, nz, two_phase=True, perm=perm, sat=sat, phi0=0.0,
                                  inv_N=0.0, wi=0.0, biot=0.0)
    A = p.to_scipy().toarray()
    nu = p.meta["n_u"]
    F = A[nu:, nu:]
    for ph in (0, 1):
        rows = F[ph::2]
        assert np.abs(rows.sum(axis=0)).max() <= 1e-12 * np.abs(F).max()


def test_two_phase_block_structure():
    p = synth.two_phase(6, 5, 4)
    A = p.to_scipy()
    nu = p.meta["n_u"]
    # no gravity: A_us = 0
    assert A[:nu, nu::2].nnz == 0
    assert A[:nu, nu + 1::2].nnz > 0 and A[nu:, :nu].nnz > 0
    assert np.array_equal(p.dof_label[nu:nu + 4], [1, 2, 1, 2])
    assert np.array_equal(p.dof_node[nu:nu + 4], [nu // 3, nu // 3, nu // 3 + 1, nu // 3 + 1])


@pytest.mark.parametrize("cid", [1])
def test_generator_deterministic(cid):
    a, b = synth.config(cid), synth.config(cid)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.col, b.col)
