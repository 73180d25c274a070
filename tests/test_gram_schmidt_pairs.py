"""The pair form of modified Gram-Schmidt the GPU uses (two projections per
launch) against the one-at-a-time recurrence, on the CPU.

For the basis pair V_2k, V_2k+1 the GPU takes the second projection as
V_2k+1 . w - h_2k g_k with g_k = V_2k . V_2k+1, formed when V_2k+1 is (the
last pass of the iteration that made it, from the unnormalised vector).  In
exact arithmetic that is V_2k+1 . (w - h_2k V_2k), the projection modified
Gram-Schmidt takes; these tests check it to rounding on a basis that has lost
orthogonality the way a long Arnoldi process does, and that dropping the
correction term does not pass.
"""
import numpy as np


def _basis(n, k, drift, seed):
    """k unit vectors whose pairwise inner products are ~drift (a perturbed
    orthonormal basis)."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    v = q + drift * rng.standard_normal((n, k)) / np.sqrt(n)
    return (v / np.linalg.norm(v, axis=0)).T.copy()


def _mgs(V, w):
    h = np.zeros(len(V))
    for i, vi in enumerate(V):
        h[i] = vi @ w
        w = w - h[i] * vi
    return h, w


def _mgs_pairs(V, w, g):
    """Two projections per pass; g[k] = V_2k . V_2k+1."""
    h = np.zeros(len(V))
    for p in range(0, len(V), 2):
        h[p] = V[p] @ w
        if p + 1 < len(V):
            h[p + 1] = V[p + 1] @ w - h[p] * g[p // 2]
            w = w - h[p] * V[p] - h[p + 1] * V[p + 1]
        else:
            w = w - h[p] * V[p]
    return h, w


def _workload(n=20000, k=13, drift=1e-7, seed=3):
    V = _basis(n, k, drift, seed)
    rng = np.random.default_rng(seed + 1)
    # a preconditioned Arnoldi vector: mostly the last basis vector, a little
    # of every other direction
    w = 3.0 * V[-1] + 0.2 * rng.standard_normal(n) / np.sqrt(n) + 0.5 * V[0]
    return V, w


def test_pair_projections_equal_one_at_a_time():
    V, w = _workload()
    g = np.array([V[2 * q] @ V[2 * q + 1] for q in range(len(V) // 2)])
    h1, w1 = _mgs(V, w)
    h2, w2 = _mgs_pairs(V, w, g)
    scale = np.linalg.norm(w)
    assert np.max(np.abs(h1 - h2)) <= 1e-13 * scale
    assert np.linalg.norm(w1 - w2) <= 1e-13 * scale


def test_pair_projections_need_the_gram_correction():
    """With the basis's inner products at 1e-7 the correction is far above
    rounding: leaving it out (classical projection inside a pair) fails."""
    V, w = _workload()
    h1, _ = _mgs(V, w)
    h0, _ = _mgs_pairs(V, w, np.zeros(len(V) // 2))
    assert np.max(np.abs(h1 - h0)) > 1e2 * 1e-13 * np.linalg.norm(w)


def test_gram_entry_from_the_unnormalised_vector():
    """g_k formed at the last pass, (V_2k . w) / ||w|| with w the vector
    before its scaling, is V_2k . V_2k+1 of the stored basis to rounding."""
    V, w = _workload(k=7)
    g = np.array([V[2 * q] @ V[2 * q + 1] for q in range(3)])
    _, wf = _mgs_pairs(V[:7], w, g)   # 7 vectors: V_6 starts the pair (6, 7)
    nrm = np.linalg.norm(wf)
    g_last = (V[6] @ wf) / nrm
    v7 = wf * (1.0 / nrm)
    assert abs(g_last - V[6] @ v7) <= 1e-15
    # and the new vector is orthogonal to the basis to the basis's own drift
    assert np.max(np.abs(V[:7] @ v7)) <= 1e-6
