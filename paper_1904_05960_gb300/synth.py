"""Seeded synthetic Jacobians of (multiphase) poromechanics, for the MGR solver.

This module builds the linear systems the solver is exercised on; it holds none
of the solver's arithmetic.  It produces the Jacobian of the fully implicit
displacement / saturation / pressure formulation (paper Sec. 2-4, Eq. 4.2, the
3x3 field-block system "block_linear_system"):

* displacement: continuous trilinear (Q1) finite elements on unit hexahedra,
  3 dofs per vertex, isotropic linear elasticity (Sec. 3, item (i));
* saturation and pressure: one dof each per cell (piecewise constants), with a
  two-point flux approximation and first-order phase upwinding (Sec. 3, items
  (ii)-(iii)); saturation and pressure of a cell are interleaved, so the flow
  part has dense 2x2 cell blocks (Sec. 5.3, Remark on interleaved ordering);
* Biot coupling b = 1 (stress = C:grad^s u - b p 1, Sec. 2).

Global dof order: all displacement dofs first (node-major, x/y/z interleaved),
then the cell dofs (cell-major; (s, p) interleaved for two-phase, p only for
single-phase).  Labels: 0 = u, 1 = s, 2 = p.

The element integrals of Q1 on the unit cube are products of 1-D integrals of
the linear hat functions, so they are formed exactly in rational arithmetic and
only then scaled by the (floating-point) material constants.

Proposed details that the paper leaves open (the paper's staircase / SPE10 data
are not available; these synthetic meshes stand in for them):
no gravity (so A_us = 0), traction-free top, bottom fixed, roller sides;
mu_w = 1, mu_o = 5, phi0 = 0.2, Biot modulus 1/N = 1e-3 (two-phase), dt = 1;
Corey k_rw = s^2, k_ro = (1-s)^2; TPFA transmissibility = harmonic mean of the
cell permeabilities (unit face area and distance); upwinding on the sign of
p_K - p_L for the frozen state p = 1 - d/d_max (d = Manhattan distance from the
injector cell (0,0,0)); injector at rate (no Jacobian entry); BHP producer at
the opposite corner cell with WI = 1 and p_bh = -1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import os
from fractions import Fraction

import numpy as np

LABEL_U, LABEL_S, LABEL_P = 0, 1, 2


# ---------------------------------------------------------------------------
# Exact Q1 element integrals on the unit cube
# ---------------------------------------------------------------------------
def _corner(a):
    return (a & 1, (a >> 1) & 1, (a >> 2) & 1)


_M1 = [[Fraction(1, 3), Fraction(1, 6)], [Fraction(1, 6), Fraction(1, 3)]]  # int phi_a phi_b
_G1 = [[Fraction(1), Fraction(-1)], [Fraction(-1), Fraction(1)]]            # int phi_a' phi_b'


def _D1(a, b):
    """int_0^1 phi_a'(x) phi_b(x) dx for the linear hats phi_0 = 1-x, phi_1 = x."""
    return Fraction(-1 if a == 0 else 1, 2)


def _int_grad(a, b, p, q):
    """Exact int_cube (d N_a / d x_p) (d N_b / d x_q) dV."""
    ca, cb = _corner(a), _corner(b)
    val = Fraction(1)
    for d in range(3):
        if d == p and d == q:
            f = _G1[ca[d]][cb[d]]
        elif d == p:
            f = _D1(ca[d], cb[d])
        elif d == q:
            f = _D1(cb[d], ca[d])
        else:
            f = _M1[ca[d]][cb[d]]
        val *= f
    return val


def q1_element_matrices():
    """Exact rational K_lambda, K_mu (24x24) and Q (24,) of the unit-cube Q1 element.

    K = lambda * K_lambda + mu * K_mu is the isotropic elastic stiffness
    (bilinear form lambda div u div v + 2 mu eps(u):eps(v)), local dof 3a+i for
    corner a = ax + 2 ay + 4 az and component i.  Q[3a+i] = int d N_a/d x_i dV
    is the divergence (Biot) coupling to the cell's constant pressure.
    """
    Kl = [[Fraction(0)] * 24 for _ in range(24)]
    Km = [[Fraction(0)] * 24 for _ in range(24)]
    for a in range(8):
        for b in range(8):
            lap = sum(_int_grad(a, b, k, k) for k in range(3))
            for i in range(3):
                for j in range(3):
                    Kl[3 * a + i][3 * b + j] = _int_grad(a, b, i, j)
                    Km[3 * a + i][3 * b + j] = _int_grad(a, b, j, i) + (lap if i == j else 0)
    Q = []
    for a in range(8):
        ca = _corner(a)
        for i in range(3):
            v = Fraction(1)
            for d in range(3):
                v *= Fraction(-1 if ca[d] == 0 else 1) if d == i else Fraction(1, 2)
            Q.append(v)
    return Kl, Km, Q


_KL, _KM, _Q = q1_element_matrices()
KLAM = np.array([[float(x) for x in r] for r in _KL])
KMU = np.array([[float(x) for x in r] for r in _KM])
QDIV = np.array([float(x) for x in _Q])


# ---------------------------------------------------------------------------
# Problem container
# ---------------------------------------------------------------------------
@dataclass
class Problem:
    """One square sparse system in CSR with per-dof grouping information."""
    n: int
    row_ptr: np.ndarray        # int64 [n+1]
    col: np.ndarray            # int32 [nnz], ascending within a row
    val: np.ndarray            # float64 [nnz]
    dof_label: np.ndarray      # int32 [n]: 0=u, 1=s, 2=p
    dof_node: np.ndarray       # int32 [n]: vertex id (u) / n_nodes + cell id (s,p)
    dof_comp: np.ndarray       # int32 [n]: x/y/z for u, s=0/p=1 (p=0 single-phase)
    rhs: np.ndarray            # float64 [n]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


# ---------------------------------------------------------------------------
# Random fields
# ---------------------------------------------------------------------------
def _gaussian_field(rng, shape_zyx, corr_zyx):
    """White noise smoothed by a separable Gaussian (std = correlation length in
    cells, periodic), renormalised to zero mean and unit variance."""
    g = rng.standard_normal(shape_zyx)
    if corr_zyx is not None and any(c > 0 for c in corr_zyx):
        from scipy.ndimage import gaussian_filter
        g = gaussian_filter(g, sigma=corr_zyx, mode="wrap")
        g = (g - g.mean()) / g.std()
    return g


def _channel_field(rng, nx, ny, nz, n_channels=8, width=4, thick=2, k_hi=1e3, k_lo=1e-3):
    """Straight x-directed high-permeability channels in a low background."""
    k = np.full((nz, ny, nx), k_lo)
    for _ in range(n_channels):
        y0 = int(rng.integers(0, max(1, ny - width + 1)))
        z0 = int(rng.integers(0, max(1, nz - thick + 1)))
        k[z0:z0 + thick, y0:y0 + width, :] = k_hi
    return k


# ---------------------------------------------------------------------------
# Assembly
# ---------------------------------------------------------------------------
def _compress(cols, vals, valid):
    """Row-wise candidate templates (ascending columns) -> CSR, dropping absent
    candidates and exact zeros."""
    keep = valid & (vals != 0.0)
    counts = keep.sum(axis=1)
    return counts, cols[keep].astype(np.int32), vals[keep]


def _chunks(total, size):
    return [(a, min(a + size, total)) for a in range(0, total, size)]


def build_poromechanics(nx, ny, nz, *, two_phase=True, E=1e4, nu=0.25, biot=1.0,
                        dt=1.0, perm=None, sat=None, inv_N=None, phi0=0.2,
                        mu_w=1.0, mu_o=5.0, wi=1.0, p_bh=-1.0, rhs_seed=1,
                        meta=None, threads=None, chunk_rows=65536):
    """Assemble the fully implicit Jacobian on an nx*ny*nz grid of unit cells.

    E may be a scalar or a per-cell array (nz, ny, nx); perm a per-cell array.
    Rows are assembled in chunks of about chunk_rows points (vertices, then
    cells) on `threads` threads (default: the machine's cores, at most 16), so
    that the working memory stays a small multiple of the final CSR; the result
    does not depend on either setting.
    """
    nnx, nny, nnz_ = nx + 1, ny + 1, nz + 1
    n_nodes = nnx * nny * nnz_
    n_cells = nx * ny * nz
    n_u = 3 * n_nodes
    ncd = 2 if two_phase else 1          # cell dofs
    n = n_u + ncd * n_cells
    if inv_N is None:
        inv_N = 1e-3 if two_phase else 0.0
    if threads is None:
        threads = max(1, min(16, os.cpu_count() or 1))

    Ec = np.broadcast_to(np.asarray(E, dtype=np.float64), (nz, ny, nx))
    nuc = np.broadcast_to(np.asarray(nu, dtype=np.float64), (nz, ny, nx))
    lam_c = Ec * nuc / ((1.0 + nuc) * (1.0 - 2.0 * nuc))
    mu_c = Ec / (2.0 * (1.0 + nuc))
    lam_p = np.zeros((nz + 2, ny + 2, nx + 2))
    mu_p = np.zeros((nz + 2, ny + 2, nx + 2))
    lam_p[1:-1, 1:-1, 1:-1] = lam_c
    mu_p[1:-1, 1:-1, 1:-1] = mu_c
    del lam_c, mu_c

    # --- Dirichlet set: bottom fixed, rollers on the four sides ------------
    # (index 3*node+comp; node order: x fastest)
    fixed = np.zeros((nnz_, nny, nnx, 3), dtype=bool)
    fixed[0, :, :, :] = True
    fixed[:, :, 0, 0] = True
    fixed[:, :, nx, 0] = True
    fixed[:, 0, :, 1] = True
    fixed[:, ny, :, 1] = True
    fixed_dof = fixed.reshape(-1)

    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    eoffs = [(ox, oy, oz) for oz in (-1, 0) for oy in (-1, 0) for ox in (-1, 0)]

    def cell_dof(cid, comp):
        return n_u + ncd * cid + comp

    pcomp = 1 if two_phase else 0

    # ---------------- displacement rows: 27*3 u columns + 8 p columns ------
    Wu = 27 * 3 + 8
    diag_slot = 3 * 13  # offset (0,0,0) is template entry 13

    def u_rows(a0, a1):
        node = np.arange(a0, a1, dtype=np.int64)
        m = a1 - a0
        ix = node % nnx
        iy = (node // nnx) % nny
        iz = node // (nnx * nny)
        ucols = np.zeros((m, 3, Wu), dtype=np.int64)
        uvals = np.zeros((m, 3, Wu))
        uvalid = np.zeros((m, 3, Wu), dtype=bool)
        for t, (dx, dy, dz) in enumerate(offs):
            jx, jy, jz = ix + dx, iy + dy, iz + dz
            inr = (jx >= 0) & (jx < nnx) & (jy >= 0) & (jy < nny) & (jz >= 0) & (jz < nnz_)
            nb = np.where(inr, jx + nnx * (jy + nny * jz), 0)
            blk = np.zeros((m, 3, 3))
            for (ox, oy, oz) in eoffs:
                ax, ay, az = -ox, -oy, -oz
                bx, by, bz = dx - ox, dy - oy, dz - oz
                if not (0 <= bx <= 1 and 0 <= by <= 1 and 0 <= bz <= 1):
                    continue
                a = ax + 2 * ay + 4 * az
                b = bx + 2 * by + 4 * bz
                cl = lam_p[iz + oz + 1, iy + oy + 1, ix + ox + 1]
                cm = mu_p[iz + oz + 1, iy + oy + 1, ix + ox + 1]
                kl = KLAM[3 * a:3 * a + 3, 3 * b:3 * b + 3]
                km = KMU[3 * a:3 * a + 3, 3 * b:3 * b + 3]
                blk += cl[:, None, None] * kl[None] + cm[:, None, None] * km[None]
            for i in range(3):
                for j in range(3):
                    ucols[:, i, 3 * t + j] = 3 * nb + j
                    uvals[:, i, 3 * t + j] = blk[:, i, j]
                    uvalid[:, i, 3 * t + j] = inr
        for t, (ox, oy, oz) in enumerate(eoffs):
            cx, cy, cz = ix + ox, iy + oy, iz + oz
            inr = (cx >= 0) & (cx < nx) & (cy >= 0) & (cy < ny) & (cz >= 0) & (cz < nz)
            cid = cx + nx * (cy + ny * cz)
            a = (-ox) + 2 * (-oy) + 4 * (-oz)
            for i in range(3):
                ucols[:, i, 81 + t] = np.where(inr, cell_dof(cid, pcomp), 0)
                uvals[:, i, 81 + t] = -biot * QDIV[3 * a + i]
                uvalid[:, i, 81 + t] = inr
        ucols = ucols.reshape(3 * m, Wu)
        uvals = uvals.reshape(3 * m, Wu)
        uvalid = uvalid.reshape(3 * m, Wu)
        # Dirichlet: remove fixed columns everywhere, fixed rows become identity.
        uvalid[:, :81] &= ~fixed_dof[ucols[:, :81]]
        rfix = fixed_dof[3 * a0:3 * a1]
        uvalid[rfix, :] = False
        rows_fixed = np.nonzero(rfix)[0]
        comp_fixed = (3 * a0 + rows_fixed) % 3
        uvals[rows_fixed, diag_slot + comp_fixed] = 1.0
        uvalid[rows_fixed, diag_slot + comp_fixed] = True
        return _compress(ucols, uvals, uvalid)

    # ---------------- cell rows ------------------------------------------
    cid_all = np.arange(n_cells, dtype=np.int64)
    cx_ = cid_all % nx
    cy_ = (cid_all // nx) % ny
    cz_ = cid_all // (nx * ny)
    k = np.asarray(perm, dtype=np.float64).reshape(n_cells)
    s = (np.asarray(sat, dtype=np.float64).reshape(n_cells) if two_phase else None)

    # stencil slots sorted by neighbour cell id: -z,-y,-x,self,+x,+y,+z
    nbr_off = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    SELF = 3
    J = {}
    names = [("s", "s"), ("s", "p"), ("p", "s"), ("p", "p")] if two_phase else [("p", "p")]
    for nm in names:
        J[nm] = np.zeros((n_cells, 7))

    d = cx_ + cy_ + cz_
    dmax = max((nx - 1) + (ny - 1) + (nz - 1), 1)
    pst = 1.0 - d / dmax
    del d

    def lam(sv):
        return sv * sv / mu_w, (1.0 - sv) * (1.0 - sv) / mu_o

    def dlam(sv):
        return 2.0 * sv / mu_w, -2.0 * (1.0 - sv) / mu_o

    # Each cell is the K side of at most one face per axis and the L side of
    # at most one, so the index arrays of one update hold no repeats and a
    # plain indexed add is exact.
    for axis, (slot_plus, slot_minus) in enumerate(((4, 2), (5, 1), (6, 0))):
        step = (1, nx, nx * ny)[axis]
        coord = (cx_, cy_, cz_)[axis]
        lim = (nx, ny, nz)[axis]
        K = cid_all[coord < lim - 1]
        L = K + step
        T = 2.0 * k[K] * k[L] / (k[K] + k[L])
        if two_phase:
            dp = pst[K] - pst[L]
            up_is_K = (dp > 0) | ((dp == 0) & (K < L))
            U = np.where(up_is_K, K, L)
            lw, lo = lam(s[U])
            dlw, dlo = dlam(s[U])
            slotU_K = np.where(up_is_K, SELF, slot_plus)   # U as seen from row K
            slotU_L = np.where(up_is_K, slot_minus, SELF)  # U as seen from row L
            for ph, lm, dl in (("s", lw, dlw), ("p", lo, dlo)):
                Jp = J[(ph, "p")]
                Js = J[(ph, "s")]
                Jp[K, SELF] += T * lm
                Jp[K, slot_plus] += -T * lm
                Jp[L, slot_minus] += -T * lm
                Jp[L, SELF] += T * lm
                Js[K, slotU_K] += T * dl * dp
                Js[L, slotU_L] += -T * dl * dp
        else:
            Jp = J[("p", "p")]
            Jp[K, SELF] += T
            Jp[K, slot_plus] += -T
            Jp[L, slot_minus] += -T
            Jp[L, SELF] += T
    if two_phase:
        J[("s", "s")][:, SELF] += phi0 / dt
        J[("s", "p")][:, SELF] += s * inv_N / dt
        J[("p", "s")][:, SELF] += -phi0 / dt
        J[("p", "p")][:, SELF] += (1.0 - s) * inv_N / dt
        wc = n_cells - 1                                    # producer: far corner
        lw, lo = lam(s[wc])
        dlw, dlo = dlam(s[wc])
        J[("s", "p")][wc, SELF] += wi * lw
        J[("p", "p")][wc, SELF] += wi * lo
        J[("s", "s")][wc, SELF] += wi * dlw * (pst[wc] - p_bh)
        J[("p", "s")][wc, SELF] += wi * dlo * (pst[wc] - p_bh)
    else:
        top = cz_ == nz - 1
        J[("p", "p")][top, SELF] += 2.0 * k[top]             # drained top, p = 0
        J[("p", "p")][:, SELF] += inv_N / dt

    # u columns of a cell row: its 8 vertices (ascending node id)
    Wc = 24 + 7 * ncd

    def cell_rows(c0, c1):
        m = c1 - c0
        cx, cy, cz = cx_[c0:c1], cy_[c0:c1], cz_[c0:c1]
        sc = s[c0:c1] if two_phase else None
        ccols = np.zeros((m, ncd, Wc), dtype=np.int64)
        cvals = np.zeros((m, ncd, Wc))
        cvalid = np.zeros((m, ncd, Wc), dtype=bool)
        for a in range(8):
            ax, ay, az = _corner(a)
            nid = (cx + ax) + nnx * ((cy + ay) + nny * (cz + az))
            for i in range(3):
                for r in range(ncd):
                    if two_phase:
                        coef = biot * (sc if r == 0 else (1.0 - sc)) / dt
                    else:
                        coef = np.full(m, biot / dt)
                    ccols[:, r, 3 * a + i] = 3 * nid + i
                    cvals[:, r, 3 * a + i] = coef * QDIV[3 * a + i]
                    cvalid[:, r, 3 * a + i] = ~fixed_dof[3 * nid + i]
        for t, (dx, dy, dz) in enumerate(nbr_off):
            jx, jy, jz = cx + dx, cy + dy, cz + dz
            inr = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
            nb = np.where(inr, jx + nx * (jy + ny * jz), 0)
            if two_phase:
                for r, ph in enumerate(("s", "p")):
                    for q, var in enumerate(("s", "p")):
                        ccols[:, r, 24 + 2 * t + q] = cell_dof(nb, q)
                        cvals[:, r, 24 + 2 * t + q] = J[(ph, var)][c0:c1, t]
                        cvalid[:, r, 24 + 2 * t + q] = inr
            else:
                ccols[:, 0, 24 + t] = cell_dof(nb, 0)
                cvals[:, 0, 24 + t] = J[("p", "p")][c0:c1, t]
                cvalid[:, 0, 24 + t] = inr
        return _compress(ccols.reshape(-1, Wc), cvals.reshape(-1, Wc), cvalid.reshape(-1, Wc))

    jobs = ([(u_rows, a, b) for a, b in _chunks(n_nodes, chunk_rows)]
            + [(cell_rows, a, b) for a, b in _chunks(n_cells, chunk_rows)])
    if threads > 1 and len(jobs) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=threads) as ex:
            parts = list(ex.map(lambda j: j[0](j[1], j[2]), jobs))
    else:
        parts = [f(a, b) for f, a, b in jobs]
    del J
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.concatenate([c for c, _, _ in parts]), out=row_ptr[1:])
    nnz_total = int(row_ptr[-1])
    col = np.empty(nnz_total, dtype=np.int32)
    val = np.empty(nnz_total)
    pos = 0
    for q in range(len(parts)):
        _, cc, vv = parts[q]
        col[pos:pos + len(cc)] = cc
        val[pos:pos + len(vv)] = vv
        pos += len(cc)
        parts[q] = None
    del parts

    dof_label = np.empty(n, dtype=np.int32)
    dof_label[:n_u] = LABEL_U
    dof_node = np.empty(n, dtype=np.int32)
    dof_node[:n_u] = np.repeat(np.arange(n_nodes), 3)
    dof_comp = np.empty(n, dtype=np.int32)
    dof_comp[:n_u] = np.tile(np.arange(3), n_nodes)
    if two_phase:
        dof_label[n_u::2] = LABEL_S
        dof_label[n_u + 1::2] = LABEL_P
        dof_node[n_u:] = n_nodes + np.repeat(np.arange(n_cells), 2)
        dof_comp[n_u:] = np.tile(np.arange(2), n_cells)
    else:
        dof_label[n_u:] = LABEL_P
        dof_node[n_u:] = n_nodes + np.arange(n_cells)
        dof_comp[n_u:] = 0
    rhs = np.random.default_rng(rhs_seed).standard_normal(n)
    m = dict(nx=nx, ny=ny, nz=nz, n_u=n_u, n_cells=n_cells, two_phase=two_phase,
             n_nodes=n_nodes)
    if meta:
        m.update(meta)
    return Problem(n=n, row_ptr=row_ptr, col=col, val=val, dof_label=dof_label,
                   dof_node=dof_node, dof_comp=dof_comp, rhs=rhs, meta=m)


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------
def single_phase(nx=8, ny=8, nz=8, seed=0, sigma=1.0, E=1e4, nu=0.25, dt=1.0):
    """Single-phase poromechanics: Q1 u (E, nu), TPFA p, lognormal uncorrelated k."""
    rng = np.random.default_rng(seed)
    perm = np.exp(sigma * rng.standard_normal((nz, ny, nx)))
    return build_poromechanics(nx, ny, nz, two_phase=False, E=E, nu=nu, dt=dt, perm=perm,
                               rhs_seed=seed + 1,
                               meta=dict(kind="single_phase", seed=seed, sigma=sigma))


def two_phase(nx=64, ny=64, nz=32, seed=0, sigma=2.0, corr=(16.0, 16.0, 2.0), E=1e4,
              E_sigma=0.0, nu=0.25, dt=1.0):
    """Two-phase poromechanics: lognormal k with Gaussian correlation (x, y, z
    lengths in cells), saturation U[0.2, 0.8], optional lognormal E."""
    rng = np.random.default_rng(seed)
    g = _gaussian_field(rng, (nz, ny, nx), (corr[2], corr[1], corr[0]) if corr else None)
    perm = np.exp(sigma * g)
    sat = rng.uniform(0.2, 0.8, size=(nz, ny, nx))
    Ef = E
    if E_sigma > 0:
        Ef = E * np.exp(E_sigma * rng.standard_normal((nz, ny, nx)))
    return build_poromechanics(nx, ny, nz, two_phase=True, E=Ef, nu=nu, dt=dt, perm=perm,
                               sat=sat, rhs_seed=seed + 1,
                               meta=dict(kind="two_phase", seed=seed, sigma=sigma,
                                         corr=corr, E_sigma=E_sigma, dt=dt))


def channels(nx=256, ny=256, nz=96, seed=0):
    """High-contrast channels (1e3 in 1e-3) and alternating stiff/soft layers
    (E = 1e4 / 10 every 8 cells in z, nu = 0.3)."""
    rng = np.random.default_rng(seed)
    perm = _channel_field(rng, nx, ny, nz)
    sat = rng.uniform(0.2, 0.8, size=(nz, ny, nx))
    layer = (np.arange(nz) // 8) % 2
    E = np.where(layer == 0, 1e4, 10.0)[:, None, None] * np.ones((nz, ny, nx))
    return build_poromechanics(nx, ny, nz, two_phase=True, E=E, nu=0.3, perm=perm, sat=sat,
                               rhs_seed=seed + 1, meta=dict(kind="channels", seed=seed))


def ensemble_member(i, side_range=(16, 48)):
    """Member i of the 64-system ensemble: cubic side uniform in side_range
    (inclusive; [16, 48] for the ensemble workload), sigma in [1, 3], dt
    log-uniform in [0.1, 10], seed i."""
    rng = np.random.default_rng(1000 + i)
    side = int(rng.integers(side_range[0], side_range[1] + 1))
    sigma = float(rng.uniform(1.0, 3.0))
    dt = float(10.0 ** rng.uniform(-1.0, 1.0))
    return two_phase(side, side, side, seed=i, sigma=sigma, dt=dt)


CONFIGS = {
    1: dict(fn="single_phase", kw=dict(nx=8, ny=8, nz=8, seed=0)),
    2: dict(fn="two_phase", kw=dict(nx=64, ny=64, nz=32, seed=0, sigma=2.0)),
    3: dict(fn="two_phase", kw=dict(nx=128, ny=128, nz=64, seed=0, sigma=2.0, E_sigma=1.5)),
    5: dict(fn="channels", kw=dict(nx=256, ny=256, nz=96, seed=0)),
}


def config(cid, **override):
    """Build workload `cid` (1, 2, 3 or 5); keyword overrides change its sizes."""
    c = CONFIGS[cid]
    kw = dict(c["kw"])
    kw.update(override)
    return globals()[c["fn"]](**kw)
