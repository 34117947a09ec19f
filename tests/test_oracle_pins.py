"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  None of them compares the
oracle with itself: each checks a closed form, a theorem of the paper, a
hand solution, a second formulation of the same tearing, or a printed
example (tests/golden/).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import vtm_oracle as O
from paper_0910_0663_gb300 import workloads as wl


def _net(n, edges, g, ground):
    indptr, indices, data = wl.assemble_nodal(n, np.asarray(edges, np.int64), np.asarray(g, float),
                                              np.asarray(ground, float))
    return O.csr_matrix(indptr, indices, data, n)


# ---------------------------------------------------------------------------
# Two-node circuit: closed forms (Sec. VIII, reflection coefficient; Fig. 4)
# ---------------------------------------------------------------------------

def _two_node(g0a, g0b, g):
    A = _net(2, [[0, 1]], [g], [g0a, g0b])
    return A, np.array([0, 1], np.int32)


@pytest.mark.parametrize("g0,g,W", [(1.0, 1.0, 1.0), (0.3, 2.0, 0.7), (1e-3, 1.5, 4.0)])
def test_two_node_reflection_closed_form(g0, g, W):
    # Tile {node}: its twin hangs on 2g; the node has g0 to ground.  The input
    # admittance seen from the twin is 2g in series with g0: S = 2g g0/(2g+g0),
    # and the reflection coefficient is (W - S)/(W + S).
    A, part = _two_node(g0, g0, g)
    tear = O.tear_midpoint(A, part, 2)
    S_hand = 2 * g * g0 / (2 * g + g0)
    for P in (0, 1):
        S, T = O.reflection_ops(A, tear, P, W)
        assert S.shape == (1, 1)
        assert S[0, 0] == pytest.approx(S_hand, rel=1e-13)
        assert T[0, 0] == pytest.approx((W - S_hand) / (W + S_hand), rel=1e-12)


@pytest.mark.parametrize("W", [0.25, 1.0, 3.0])
def test_two_node_error_contracts_by_reflection(W):
    # Symmetric 2-node circuit: the wave error of each line end is multiplied
    # by T per sweep, so the node-voltage error shrinks by exactly |T| per sweep.
    g0, g = 1.0, 1.0
    A, part = _two_node(g0, g0, g)
    b = np.array([[1.0, 0.0]])
    x_star = np.array([2.0 / 3.0, 1.0 / 3.0])  # hand solution of [[2,-1],[-1,2]] x = [1,0]
    res, its = O.vtm_midpoint(A, part, 2, b, W=W, tol=0, max_sweeps=12, keep_iterates=True)
    S = 2 * g * g0 / (2 * g + g0)
    T = abs((W - S) / (W + S))
    errs = [np.abs(x[0] - x_star).max() for x in its]
    for k in range(2, 9):
        if errs[k - 1] < 1e-13:
            break
        assert errs[k] / errs[k - 1] == pytest.approx(T, rel=1e-8)


def test_two_node_matched_line_exact():
    # W = S on both ends: rho(T1 T2) = 0, the answer arrives with the first
    # reflected wave -> exact at sweep 2 (Sec. VIII, ideal case).
    g0, g = 0.5, 2.0
    A, part = _two_node(g0, g0, g)
    S = 2 * g * g0 / (2 * g + g0)
    b = np.array([[0.7, -0.2]])
    x_star = np.linalg.solve(A.toarray(), b[0])
    _, its = O.vtm_midpoint(A, part, 2, b, W=S, tol=0, max_sweeps=3, keep_iterates=True)
    assert np.abs(its[0][0] - x_star).max() > 1e-3
    assert np.abs(its[1][0] - x_star).max() < 1e-14


def test_two_node_one_side_matched_exact_by_sweep3():
    # Only tile 1 matched (W = S1 != S2): tile 2 is exact at sweep 2, tile 1 at
    # sweep 3 ("if one port is precisely matched ... settle down after 1
    # reflection", Sec. VIII).
    g0a, g0b, g = 0.5, 3.0, 2.0
    A, part = _two_node(g0a, g0b, g)
    S1 = 2 * g * g0a / (2 * g + g0a)
    b = np.array([[0.7, -0.2]])
    x_star = np.linalg.solve(A.toarray(), b[0])
    _, its = O.vtm_midpoint(A, part, 2, b, W=S1, tol=0, max_sweeps=3, keep_iterates=True)
    assert abs(its[1][0][1] - x_star[1]) < 1e-14
    assert abs(its[1][0][0] - x_star[0]) > 1e-6
    assert np.abs(its[2][0] - x_star).max() < 1e-14


# ---------------------------------------------------------------------------
# Fixed point, single partition, convergence (Lemma 2, Theorem 1, Appendix)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("Zc", [0.25, 1.0, 4.0])
def test_fixed_point_is_direct_solution(Zc):
    # u^inf = S^-1 r (end of the Appendix) => x^inf = A^-1 b, for every Zc > 0.
    w = wl.grid2d(12, 12, 4, 4, Zc=Zc, seed=3, ground=0.05)
    A = w.csr()
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / Zc, tol=1e-14, max_sweeps=20000)
    assert res.converged
    x_star = np.linalg.solve(A.toarray(), w.b[0])
    assert np.abs(res.x[0] - x_star).max() <= 1e-11 * np.abs(x_star).max()


def test_single_partition_is_one_direct_solve():
    w = wl.grid2d(10, 10, 10, 10, seed=1)
    assert w.nparts == 1
    A = w.csr()
    res = O.vtm_midpoint(A, w.partition, 1, w.b, W=1.0, tol=1e-12)
    assert res.sweeps == 1 and res.converged
    x_star = np.linalg.solve(A.toarray(), w.b[0])
    assert np.abs(res.x[0] - x_star).max() <= 1e-13 * np.abs(x_star).max()


def _random_resistor_net(rng, n, extra_edges, nparts):
    # spanning path plus random chords; random ground on a few nodes
    perm = rng.permutation(n)
    edges = [(perm[k], perm[k + 1]) for k in range(n - 1)]
    while len(edges) < n - 1 + extra_edges:
        i, j = rng.choice(n, 2, replace=False)
        if (i, j) not in edges and (j, i) not in edges:
            edges.append((i, j))
    edges = np.array(edges, np.int64)
    g = rng.uniform(0.1, 5.0, len(edges))
    ground = np.zeros(n)
    ground[rng.choice(n, max(1, n // 5), replace=False)] = rng.uniform(0.01, 1.0, max(1, n // 5))
    part = rng.integers(0, nparts, n).astype(np.int32)
    part[:nparts] = np.arange(nparts)  # no empty part
    return _net(n, edges, g, ground), part


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("Zc", [0.1, 1.0, 10.0])
def test_theorem1_convergence_random_spd(seed, Zc):
    # Theorem 1: SPD resistor network, SPD line impedance -> VTM converges to
    # the answer of the resistor network.
    rng = np.random.default_rng(100 + seed)
    A, part = _random_resistor_net(rng, 40, 50, 4)
    b = rng.uniform(-1, 1, (2, 40))
    res = O.vtm_midpoint(A, part, 4, b, W=1 / Zc, tol=1e-12, max_sweeps=50000)
    assert res.converged
    x_star = np.linalg.solve(A.toarray(), b.T).T
    assert np.abs(res.x - x_star).max() <= 1e-8 * np.abs(x_star).max()


# ---------------------------------------------------------------------------
# Reflection operator (Sec. VIII; Appendix Lemmas 5-6 and the spectral bound)
# ---------------------------------------------------------------------------

def test_reflection_symmetric_spectrum_in_unit_interval():
    w = wl.grid2d(12, 12, 6, 6, seed=4)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    for Zc in (0.3, 1.0, 3.0):
        W = 1 / Zc
        for P in range(w.nparts):
            S, T = O.reflection_ops(A, tear, P, W)
            assert np.abs(S - S.T).max() < 1e-12
            lam = np.linalg.eigvalsh(S)
            assert lam.min() > 0
            assert np.abs(T - T.T).max() < 1e-12
            mu = np.sort(np.linalg.eigvalsh((T + T.T) / 2))
            assert mu.max() < 1 and mu.min() > -1
            assert np.allclose(mu, np.sort((W - lam) / (W + lam)), atol=1e-12)


def test_floating_tile_has_unit_reflection_eigenvalue():
    # A tile without any ground: S is singular (constant mode), so T has
    # eigenvalue exactly 1; the local matrix stays non-singular.
    edges = wl.grid_edges_2d(4, 8)
    g = np.ones(len(edges))
    ground = np.zeros(32)
    ground[:4] = 1.0  # ground only in the left tile
    A = _net(32, edges, g, ground)
    part = np.array([(k % 8) // 4 for k in range(32)], np.int32)
    tear = O.tear_midpoint(A, part, 2)
    S, T = O.reflection_ops(A, tear, 1, 1.0)
    assert np.linalg.eigvalsh(S).min() == pytest.approx(0.0, abs=1e-12)
    assert np.linalg.eigvalsh((T + T.T) / 2).max() == pytest.approx(1.0, abs=1e-12)


def _augmented(A, tear):
    """Midpoint-augmented system: every torn branch g becomes 2g - m - 2g."""
    n = tear.n
    lines = np.flatnonzero(tear.port_node < tear.port_remote)
    nl = len(lines)
    M = np.zeros((n + nl, n + nl))
    M[:n, :n] = tear.A_in.toarray()
    for k, s in enumerate(lines):
        i, j, g = tear.port_node[s], tear.port_remote[s], tear.port_g[s]
        m = n + k
        M[m, m] = 4 * g
        M[m, i] = M[i, m] = -2 * g
        M[m, j] = M[j, m] = -2 * g
        M[i, i] += g
        M[j, j] += g
    return M, lines


def test_midpoint_augmentation_is_exact():
    # Eliminating every midpoint gives back A (the reading R1 is exact).
    w = wl.grid2d(8, 8, 4, 4, seed=5)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    M, lines = _augmented(A, tear)
    n = w.n
    Ared = M[:n, :n] - M[:n, n:] @ np.linalg.solve(M[n:, n:], M[n:, :n])
    assert np.abs(Ared - A.toarray()).max() < 1e-13


def test_schur_sum_and_excitation_sum_two_tiles():
    # Appendix: S_1 + S_2 = S and r_1 + r_2 = r on the interface of a 2-way
    # tearing (S from the augmented system, S_s from each sub-circuit).
    w = wl.grid2d(6, 8, 6, 4, seed=6)
    A = w.csr()
    assert w.nparts == 2
    tear = O.tear_midpoint(A, w.partition, 2)
    M, lines = _augmented(A, tear)
    n = w.n
    bm = np.concatenate([w.b[0], np.zeros(len(lines))])
    S_full = M[n:, n:] - M[n:, :n] @ np.linalg.solve(M[:n, :n], M[:n, n:])
    r_full = bm[n:] - M[n:, :n] @ np.linalg.solve(M[:n, :n], bm[:n])
    S_sum = np.zeros_like(S_full)
    r_sum = np.zeros(len(lines))
    line_of = {}
    for k, s in enumerate(lines):
        line_of[s] = k
        line_of[tear.twin[s]] = k
    for P in (0, 1):
        S, _ = O.reflection_ops(A, tear, P, 1.0)
        r = O.port_excitation(A, tear, P, w.b)[0]
        idx = np.array([line_of[s] for s in tear.tile_ports[P]])
        S_sum[np.ix_(idx, idx)] += S
        r_sum[idx] += r
    assert np.abs(S_sum - S_full).max() < 1e-12
    assert np.abs(r_sum - r_full).max() < 1e-12


def test_convergence_factor_two_tiles():
    # CF = sqrt(rho(T1 T2)) (Sec. VIII): over two sweeps the residual shrinks
    # by rho(T1 T2) asymptotically.
    w = wl.grid2d(8, 8, 8, 4, seed=7, ground=0.02)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, 2)
    W = 1.0
    _, T1 = O.reflection_ops(A, tear, 0, W)
    _, T2 = O.reflection_ops(A, tear, 1, W)
    p0, p1 = tear.tile_ports
    pos1 = {s: k for k, s in enumerate(p1)}
    Pi = np.zeros((len(p0), len(p1)))  # twin map from tile-2 order to tile-1 order
    for a, s in enumerate(p0):
        Pi[a, pos1[tear.twin[s]]] = 1.0
    rho = O.spectral_radius(T1 @ Pi @ T2 @ Pi.T)
    assert rho < 1
    res = O.vtm_midpoint(A, w.partition, 2, w.b, W=W, tol=0, max_sweeps=400)
    h = res.history[:, 0]
    k = len(h) - 40
    while h[k] < 1e-13 and k > 20:
        k -= 20
    ratio = (h[k] / h[k - 20]) ** (1 / 10)  # per two sweeps
    assert ratio == pytest.approx(rho, rel=2e-3)


def test_boundary_conditions_at_convergence():
    # At the fixed point u_1 = u_2 = u and i_1 = -i_2 (Sec. V, after Eq. 8),
    # and the twin voltage is the midpoint voltage (x_i + x_j)/2.
    w = wl.grid2d(12, 12, 4, 4, seed=8, ground=0.05)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-14, max_sweeps=20000)
    u, cur = res.u[0], res.i[0]
    scale = np.abs(u).max()
    assert np.abs(u - u[tear.twin]).max() < 1e-10 * scale
    assert np.abs(cur + cur[tear.twin]).max() < 1e-10 * np.abs(cur).max()
    mid = 0.5 * (res.x[0][tear.port_node] + res.x[0][tear.port_remote])
    assert np.abs(u - mid).max() < 1e-10 * scale


def test_midpoint_vtm_equals_vertex_separator_vtm():
    # The same method reached two ways: (a) the node-partition oracle and
    # (b) the paper's vertex-separator tearing (Sec. V-VI) of the explicitly
    # augmented system with the midpoints as interfacial nodes, each split in
    # half.  Their iterates agree sweep by sweep.
    w = wl.grid2d(6, 10, 6, 5, seed=9)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, 2)
    M, lines = _augmented(A, tear)
    n = w.n
    inner_sub = np.concatenate([w.partition.astype(np.int64), -np.ones(len(lines), np.int64)])
    bm = np.concatenate([w.b[0], np.zeros(len(lines))])
    ts = O.twin_split(M, bm, inner_sub, alpha=0.5)
    W = 0.8
    out = O.vtm_twin(ts, W * np.eye(len(lines)), 15)
    _, its = O.vtm_midpoint(A, w.partition, 2, w.b, W=W, tol=0, max_sweeps=15, keep_iterates=True)
    for k in range(15):
        xa = its[k][0]
        xb = O.twin_assemble(ts, n + len(lines), out[k])[0][:n]
        assert np.abs(xa - xb).max() < 1e-12 * max(1.0, np.abs(xa).max())


# ---------------------------------------------------------------------------
# The paper's four-node op-amp example (Sec. IX, Eq. 15-21; golden fixture)
# ---------------------------------------------------------------------------

def _golden(name):
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _four_node():
    v = _golden("four_node_opamp.txt")
    A = np.array([[v["g1"], v["g21"], 0, 0],
                  [0, v["g2"], 0, v["g42"]],
                  [v["g13"], 0, v["g3"], 0],
                  [0, 0, v["g34"], v["g4"]]])
    return A, v


def test_four_node_loop_gain_and_jacobi():
    A, v = _four_node()
    gain = v["g13"] * v["g34"] * v["g42"] * v["g21"] / (v["g1"] * v["g3"] * v["g4"] * v["g2"])
    assert gain == v["loop_gain"]
    # The Jacobi matrix is a weighted 4-cycle: lambda^4 = -(loop gain) sign
    # pattern gives |lambda| = |gain|^(1/4) = 10.
    assert O.spectral_radius(O.stationary_iteration_matrix(A, "jacobi")) == pytest.approx(10.0, rel=1e-12)


def test_four_node_classical_methods_diverge():
    A, _ = _four_node()
    for m in ("gs",):
        assert O.spectral_radius(O.stationary_iteration_matrix(A, m)) > 1
    for om in (0.2, 0.5, 1.0, 1.5, 1.9):
        assert O.spectral_radius(O.stationary_iteration_matrix(A, "sor", omega=om)) > 1
        assert O.spectral_radius(O.stationary_iteration_matrix(A, "ssor", omega=om)) > 1
    for blocks in ([[0], [1, 2, 3]], [[0, 1], [2, 3]], [[0, 1, 2], [3]]):
        G = O.stationary_iteration_matrix(A, "bj", blocks=[np.array(b) for b in blocks])
        assert O.spectral_radius(G) > 1


def test_four_node_split_matches_eq16_eq17():
    A, v = _four_node()
    b = np.array([1.0, 2.0, 3.0, 4.0])
    ts = O.twin_split(A, b, np.array([0, -1, -1, 1]), alpha=v["g2a"] / v["g2"])
    # sub-circuit 1 (Eq. 16), unknowns [u2a, u3a | u1]
    M1 = np.block([[ts.C[0], ts.E[0]], [ts.F[0], ts.D[0]]])
    ref1 = np.array([[v["g2a"], 0, 0], [0, v["g3a"], v["g13"]], [v["g21"], 0, v["g1"]]])
    assert np.array_equal(M1, ref1)
    # sub-circuit 2 (Eq. 17), unknowns [u2b, u3b | u4]
    M2 = np.block([[ts.C[1], ts.E[1]], [ts.F[1], ts.D[1]]])
    ref2 = np.array([[v["g2b"], 0, v["g42"]], [0, v["g3b"], 0], [0, v["g34"], v["g4"]]])
    assert np.array_equal(M2, ref2)
    assert np.allclose(ts.f[0] + ts.f[1], b[[1, 2]])


@pytest.mark.parametrize("rhs", ["ones", "random"])
def test_four_node_vtm_converges(rhs):
    A, v = _four_node()
    b = np.ones(4) if rhs == "ones" else np.random.default_rng(0).uniform(-1, 1, 4)
    ts = O.twin_split(A, b, np.array([0, -1, -1, 1]), alpha=0.5)
    out = O.vtm_twin(ts, np.diag([v["W2"], v["W3"]]), 40)
    x_star = np.linalg.solve(A, b)
    err = [np.abs(O.twin_assemble(ts, 4, s)[0] - x_star).max() for s in out]
    assert err[-1] < 1e-12 * np.abs(x_star).max()
    # the two twins of each interfacial node agree at the end
    assert np.abs(out[-1]["u"][0] - out[-1]["u"][1]).max() < 1e-10


def test_ideal_matrix_matching_exact_in_three_sweeps():
    # W = S_1 (full matrix): T_1 = 0, rho(T1 T2) = 0 (Sec. VIII ideal case);
    # the answer is exact once the matched side has seen one reflection.
    rng = np.random.default_rng(11)
    ny, nx = 5, 7
    edges = wl.grid_edges_2d(ny, nx)
    A = _net(ny * nx, edges, rng.uniform(0.5, 2, len(edges)), np.full(ny * nx, 0.1)).toarray()
    col = np.arange(ny * nx) % nx
    inner = np.where(col < 3, 0, np.where(col == 3, -1, 1))  # column 3 separates
    b = rng.uniform(-1, 1, ny * nx)
    ts = O.twin_split(A, b, inner)
    S1, _ = O.twin_schur(ts, 0)
    S2, _ = O.twin_schur(ts, 1)
    W = S1
    T1 = (W - S1) @ np.linalg.inv(W + S1)
    T2 = (W - S2) @ np.linalg.inv(W + S2)
    assert np.abs(T1).max() < 1e-12
    assert O.spectral_radius(T1 @ T2) < 1e-12
    out = O.vtm_twin(ts, W, 3)
    x_star = np.linalg.solve(A, b)
    assert np.abs(O.twin_assemble(ts, ny * nx, out[1], side=0)[0] - x_star).max() > 1e-6
    assert np.abs(O.twin_assemble(ts, ny * nx, out[2], side=0)[0] - x_star).max() < 1e-12


# ---------------------------------------------------------------------------
# Block Jacobi and the adjoint
# ---------------------------------------------------------------------------

def test_block_jacobi_fixed_point():
    w = wl.grid2d(12, 12, 4, 4, seed=12, ground=0.1)
    A = w.csr()
    x, k, conv, hist = O.block_jacobi(A, w.partition, w.nparts, w.b, tol=1e-13)
    assert conv
    x_star = np.linalg.solve(A.toarray(), w.b[0])
    assert np.abs(x[0] - x_star).max() <= 1e-11 * np.abs(x_star).max()
    # its asymptotic rate is the spectral radius of its iteration matrix
    G = O.stationary_iteration_matrix(A.toarray(), "bj",
                                      blocks=[np.flatnonzero(w.partition == P) for P in range(w.nparts)])
    rho = O.spectral_radius(G)
    ratio = (hist[-5, 0] / hist[-25, 0]) ** (1 / 20)
    assert ratio == pytest.approx(rho, rel=2e-2)


def test_adjoint_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    ny = nx = 5
    n = ny * nx
    edges = wl.grid_edges_2d(ny, nx)
    g = rng.uniform(0.5, 2.0, len(edges))
    ground = np.full(n, 0.2)  # well conditioned, so the differences are not rounding noise
    b = rng.uniform(-1, 1, n)
    L, x, lam, dg, dgr, db = O.adjoint_gradients(n, edges, g, ground, b)

    def loss(gg, gr, bb):
        A = _net(n, edges, gg, gr).toarray()
        xx = np.linalg.solve(A, bb)
        return float(xx @ xx)

    h = 1e-4
    for e in rng.choice(len(edges), 6, replace=False):
        gp, gm = g.copy(), g.copy()
        gp[e] += h
        gm[e] -= h
        fd = (loss(gp, ground, b) - loss(gm, ground, b)) / (2 * h)
        assert dg[e] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for i in rng.choice(n, 4, replace=False):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(g, ground, bp) - loss(g, ground, bm)) / (2 * h)
        assert db[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        gp, gm = ground.copy(), ground.copy()
        gp[i] += h
        gm[i] -= h
        fd = (loss(g, gp, b) - loss(g, gm, b)) / (2 * h)
        assert dgr[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


# ---------------------------------------------------------------------------
# Sensitivity: a mistake planted in the oracle is caught by the pins above
# ---------------------------------------------------------------------------

def test_planted_mistake_is_caught(monkeypatch):
    real = O.local_system

    def wrong(A, tear, P, Wp):  # drop the node-side g_s of the torn branch
        M = real(A, tear, P, Wp).tolil()
        ports = tear.tile_ports[P]
        nodes = tear.tile_nodes[P]
        loc = {v: k for k, v in enumerate(nodes)}
        for s in ports:
            k = len(ports) + loc[tear.port_node[s]]
            M[k, k] -= tear.port_g[s]
        return M.tocsc()

    monkeypatch.setattr(O, "local_system", wrong)
    w = wl.grid2d(12, 12, 4, 4, Zc=1.0, seed=3, ground=0.05)
    A = w.csr()
    with np.errstate(all="ignore"):
        res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-12, max_sweeps=3000)
    x_star = np.linalg.solve(A.toarray(), w.b[0])
    assert (not res.converged) or np.abs(res.x[0] - x_star).max() > 1e-6


def test_tearing_counts_for_grid_tiles():
    # 32x32 grid in 4x4 tiles of 8x8: 2*4*3*8 = 192 torn branches, 384 ports,
    # interior tiles 32 ports, edge tiles 24, corner tiles 16.
    w = wl.c1_small_grid()
    tear = O.tear_midpoint(w.csr(), w.partition, w.nparts)
    assert len(tear.port_g) == 384
    assert len(tear.lag_rho) == 0
    sizes = sorted(len(p) for p in tear.tile_ports)
    assert sizes == [16] * 4 + [24] * 8 + [32] * 4
    assert sum(s * s for s in sizes) == 9728


def test_lagged_controlled_sources_keep_the_fixed_point():
    # Cut controlled-source entries are applied with one sweep of delay
    # (reading R2); at the fixed point x^k = x^{k-1}, so the limit is still
    # A^-1 b for the unsymmetric system.
    w = wl.vccs_grid(24, 24, 8, 8, seed=2)
    A = w.csr()
    assert abs(A - A.T).max() > 0
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    assert len(tear.lag_rho) > 0
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-13, max_sweeps=20000)
    assert res.converged
    x_star = O.direct_solve(A, w.b)
    assert np.abs(res.x - x_star).max() <= 1e-9 * np.abs(x_star).max()
    xb, kb, convb, _ = O.block_jacobi(A, w.partition, w.nparts, w.b, tol=1e-13)
    assert convb and np.abs(xb - x_star).max() <= 1e-9 * np.abs(x_star).max()


def test_vccs_recipe_keeps_row_diagonal_dominance():
    w = wl.vccs_grid(32, 32, 8, 8, seed=0)
    A = w.csr().toarray()
    d = np.abs(np.diag(A))
    off = np.abs(A).sum(axis=1) - d
    assert np.all(d > off)
    assert w.meta["vccs"] == round(0.05 * 32 * 32)


def test_multi_rhs_columns_are_independent():
    w = wl.grid2d(12, 12, 4, 4, seed=14, nrhs=3, ground=0.05)
    A = w.csr()
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-12, max_sweeps=20000)
    for r in range(3):
        one = O.vtm_midpoint(A, w.partition, w.nparts, w.b[r:r + 1], W=1.0, tol=0,
                             max_sweeps=res.sweeps)
        assert np.abs(one.x[0] - res.x[r]).max() <= 1e-13 * np.abs(res.x[r]).max()
    x_star = O.direct_solve(A, w.b)
    assert np.abs(res.x - x_star).max() <= 1e-9 * np.abs(x_star).max()


# ---------------------------------------------------------------------------
# Per-line characteristic admittance (Sec. VIII choices of W)
# ---------------------------------------------------------------------------

def test_diagonal_admittance_is_block_jacobi_sweep_by_sweep():
    # W = diag(C) = 2 g on every line: a twin's port row is 4g u - 2g x = w_in,
    # so the wave sent back is 2g x of its node and the node across the line
    # sees the current g (x_j - x_i^(k-1)): exactly the lagged coupling of
    # block Jacobi (Sec. X), iterate by iterate (the paper's VTM_Diag ~ BJ)
    w = wl.grid2d(24, 24, 8, 6, seed=5)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    Wd = O.line_admittance_choice(tear, "diag")
    assert np.allclose(Wd, 2 * tear.port_g)
    res, its = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=Wd, tol=0, max_sweeps=25,
                              keep_iterates=True)
    x_bj, k_bj, _, h_bj = O.block_jacobi(A, w.partition, w.nparts, w.b, tol=0, max_sweeps=25)
    assert k_bj == res.sweeps == 25
    assert np.allclose(res.history, h_bj, rtol=1e-10, atol=0)
    assert np.abs(its[-1] - x_bj).max() <= 1e-12 * np.abs(x_bj).max()


def test_schur_approximation_limits():
    # radius 0: D~ is the 1x1 block of the port's node, D_ll = a_ll + sum of
    # the g of its torn branches -> S~ = 2g - 4g^2 / D_ll (closed form);
    # growing the neighbourhood can only lower S~ (principal submatrices of an
    # M-matrix have smaller inverse diagonals) down to diag(S_P) of the dense
    # input admittance C - E D^-1 F (reflection_ops), all positive
    w = wl.grid2d(24, 24, 8, 6, seed=6)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    g = tear.port_g
    low = tear.port_tile <= tear.port_tile[tear.twin]
    s_at = {}
    for s in range(len(g)):
        s_at.setdefault(int(tear.port_node[s]), []).append(s)
    Dll = np.array([A[tear.port_node[s], tear.port_node[s]] + g[s_at[int(tear.port_node[s])]].sum()
                    for s in range(len(g))])
    S0 = 2 * g - 4 * g ** 2 / Dll
    W0 = O.line_admittance_choice(tear, "sca", radius=0)
    assert np.allclose(W0[low], S0[low], rtol=1e-13)
    assert np.allclose(W0, W0[tear.twin])
    diagS = np.empty(len(g))
    for P in range(w.nparts):
        S, _ = O.reflection_ops(A, tear, P, 1.0)
        diagS[tear.tile_ports[P]] = np.diag(S)
    Wfull = O.line_admittance_choice(tear, "sca", radius=-1)
    assert np.allclose(Wfull[low], diagS[low], rtol=1e-11)
    prev = W0
    for r in (1, 2, 4):
        Wr = O.line_admittance_choice(tear, "sca", radius=r)
        assert np.all(Wr <= prev * (1 + 1e-12))
        assert np.all(Wr >= Wfull * (1 - 1e-12))
        prev = Wr
    assert np.all(Wfull > 0)


@pytest.mark.parametrize("kind,alpha,radius", [("diag", 1.0, -1), ("wob", 0.3, -1), ("sca", 1.0, 2),
                                               ("sca", 1.0, -1), ("alpha", 2.5, -1)])
def test_per_line_admittance_keeps_the_fixed_point(kind, alpha, radius):
    # Lemma 2 / the fixed-point argument holds for any W > 0 per line
    w = wl.c1_small_grid()
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    Wl = O.line_admittance_choice(tear, kind, alpha=alpha, radius=radius)
    assert np.all(Wl > 0) and np.allclose(Wl, Wl[tear.twin])
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=Wl, tol=1e-12, max_sweeps=20000)
    assert res.converged
    x_star = O.direct_solve(A, w.b)
    assert np.abs(res.x - x_star).max() <= 1e-8 * np.abs(x_star).max()


# ---------------------------------------------------------------------------
# Backward-Euler march (the transient an RC workload's G + C/h comes from)
# ---------------------------------------------------------------------------

def test_march_single_rc_node_closed_form():
    # one node, conductance g to ground, capacitance term c = C/h, injection I:
    # x_k = (I + c x_(k-1)) / (g + c)  =>  x_k = I/g + (x0 - I/g) (c/(g+c))^k
    g, c, I, x0 = 0.7, 3.0, 2.0, -1.5
    A = sp.csr_matrix(np.array([[g + c]]))
    X = O.backward_euler_march(A, np.array([c]), np.full((12, 1), I), np.array([x0]))
    k = np.arange(1, 13)
    ref = I / g + (x0 - I / g) * (c / (g + c)) ** k
    assert np.allclose(X[:, 0], ref, rtol=1e-13, atol=0)


def test_march_settles_to_the_dc_solution_and_is_linear():
    # constant injections: x_k -> G^-1 p (G = A - diag(c)); the march is linear
    # in (p, x0)
    w = wl.grid2d(6, 6, 3, 3, seed=41)
    G = w.csr()
    G = G + sp.diags(np.full(w.n, 0.5))          # a stronger ground: fast settling
    c = np.random.default_rng(1).uniform(0.1, 0.3, w.n)
    A = (G + sp.diags(c)).tocsr()
    p = np.tile(w.b[0], (400, 1))
    X = O.backward_euler_march(A, c, p)
    x_dc = np.linalg.solve(G.toarray(), w.b[0])
    assert np.abs(X[-1] - x_dc).max() <= 1e-12 * np.abs(x_dc).max()
    rng = np.random.default_rng(2)
    p1, p2 = rng.uniform(-1, 1, (5, w.n)), rng.uniform(-1, 1, (5, w.n))
    a1, a2 = rng.uniform(-1, 1, w.n), rng.uniform(-1, 1, w.n)
    lhs = O.backward_euler_march(A, c, p1 + p2, a1 + a2)
    rhs = O.backward_euler_march(A, c, p1, a1) + O.backward_euler_march(A, c, p2, a2)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# Stochastic line delays (the asynchronous form of Sec. XI)
# ---------------------------------------------------------------------------

def test_unit_delays_are_the_synchronous_iteration():
    w = wl.grid2d(24, 24, 8, 6, seed=61)
    A = w.csr()
    r1 = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=0, max_sweeps=40)
    r2 = O.vtm_midpoint_delayed(A, w.partition, w.nparts, w.b, W=1.0, tol=0, max_sweeps=40,
                                max_delay=1)
    assert np.allclose(r1.history, r2.history, rtol=1e-12, atol=0)
    assert np.abs(r1.x - r2.x).max() <= 1e-13 * np.abs(r1.x).max()


@pytest.mark.parametrize("max_delay,seed", [(2, 0), (3, 1), (4, 2)])
def test_stochastic_delays_keep_the_fixed_point(max_delay, seed):
    # whatever the delays, a converged state satisfies the twin-row and node
    # equations of Eq. 11 with equal waves both ways, i.e. A x = b
    w = wl.power_grid(64, 64, 16, 16, Zc=1.0, seed=62)
    A = w.csr()
    r = O.vtm_midpoint_delayed(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-11, max_sweeps=20000,
                               max_delay=max_delay, seed=seed)
    assert r.converged
    x_star = O.direct_solve(A, w.b)
    assert np.abs(r.x - x_star).max() <= 1e-8 * np.abs(x_star).max()
    sync = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0, tol=1e-11)
    assert r.sweeps >= sync.sweeps  # delays slow the exchange down


# ---------------------------------------------------------------------------
# Weighted overlapped block admittance (Sec. VIII choice 4) by its dynamics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("g0,g", [(0.5, 2.0), (3.0, 0.25)])
def test_weighted_overlapped_block_admittance_on_two_nodes(g0, g):
    # W = alpha C with C = 2g (the twin's share of the torn branch).  The error
    # contracts by |(W - S)/(W + S)| per sweep with S = 2g g0/(2g + g0) the
    # input admittance of each side (hand-solved), and the weight that makes
    # alpha 2g = S matches the line: exact by sweep 2.  A weight on g instead of
    # 2g, or a dropped alpha, breaks both.
    A, part = _two_node(g0, g0, g)
    tear = O.tear_midpoint(A, part, 2)
    S = 2 * g * g0 / (2 * g + g0)
    b = np.array([[0.7, -0.2]])
    x_star = np.linalg.solve(A.toarray(), b[0])
    alpha_match = S / (2 * g)
    Wm = O.line_admittance_choice(tear, "wob", alpha=alpha_match)
    _, its = O.vtm_midpoint(A, part, 2, b, W=Wm, tol=0, max_sweeps=3, keep_iterates=True)
    assert np.abs(its[0][0] - x_star).max() > 1e-3
    assert np.abs(its[1][0] - x_star).max() < 1e-14
    for alpha in (0.3, 1.7):
        Wa = O.line_admittance_choice(tear, "wob", alpha=alpha)
        _, its = O.vtm_midpoint(A, part, 2, b, W=Wa, tol=0, max_sweeps=10, keep_iterates=True)
        errs = [np.abs(x[0] - x_star).max() for x in its]
        rate = abs((alpha * 2 * g - S) / (alpha * 2 * g + S))
        for k in range(2, 8):
            if errs[k - 1] < 1e-12:
                break
            assert errs[k] / errs[k - 1] == pytest.approx(rate, rel=1e-7)


def test_weighted_overlapped_block_with_unit_weight_is_block_jacobi():
    # alpha = 1 gives W = C, the overlapped-block choice: the same iteration as
    # block Jacobi over the same sub-circuits, sweep by sweep
    w = wl.grid2d(16, 16, 8, 8, seed=7)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    W1 = O.line_admittance_choice(tear, "wob", alpha=1.0)
    res = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=W1, tol=0, max_sweeps=15)
    _, _, _, h_bj = O.block_jacobi(A, w.partition, w.nparts, w.b, tol=0, max_sweeps=15)
    assert np.allclose(res.history, h_bj, rtol=1e-10, atol=0)


# ---------------------------------------------------------------------------
# Classical iteration matrices (Sec. IX comparison) against plain sweeps and
# Young's theorem
# ---------------------------------------------------------------------------

def _gs_sweep(A, x, omega, order):
    # one relaxation sweep of A x = 0, node by node in `order`, written out
    x = x.copy()
    for i in order:
        s = sum(A[i, j] * x[j] for j in range(len(x)) if j != i)
        x[i] = (1 - omega) * x[i] + omega * (-s / A[i, i])
    return x


@pytest.mark.parametrize("seed", [0, 1])
def test_stationary_matrices_equal_elementwise_sweeps(seed):
    # G x equals one sweep of the update each method performs on A x = 0:
    # Gauss-Seidel (forward, omega = 1), SOR (forward), SSOR (forward then
    # backward); a wrong splitting or a transposed triangle fails at once
    rng = np.random.default_rng(seed)
    m = 6
    A = rng.uniform(-1, 1, (m, m))
    A[np.arange(m), np.arange(m)] = np.abs(A).sum(axis=1) + rng.uniform(0.5, 1.5, m)
    x = rng.uniform(-1, 1, m)
    fwd, bwd = list(range(m)), list(range(m - 1, -1, -1))
    G = O.stationary_iteration_matrix(A, "gs")
    assert np.allclose(G @ x, _gs_sweep(A, x, 1.0, fwd), rtol=1e-13, atol=1e-14)
    for om in (0.7, 1.3):
        G = O.stationary_iteration_matrix(A, "sor", omega=om)
        assert np.allclose(G @ x, _gs_sweep(A, x, om, fwd), rtol=1e-13, atol=1e-14)
        G = O.stationary_iteration_matrix(A, "ssor", omega=om)
        assert np.allclose(G @ x, _gs_sweep(A, _gs_sweep(A, x, om, fwd), om, bwd), rtol=1e-13, atol=1e-14)
    Gj = O.stationary_iteration_matrix(A, "jacobi")
    xj = np.array([-sum(A[i, j] * x[j] for j in range(m) if j != i) / A[i, i] for i in range(m)])
    assert np.allclose(Gj @ x, xj, rtol=1e-13, atol=1e-14)


def test_stationary_radii_follow_youngs_theorem():
    # The 1-D Laplacian tridiag(-1, 2, -1) of order m is consistently ordered:
    # rho_J = cos(pi/(m+1)), rho_GS = rho_J^2, and SOR at
    # omega_opt = 2/(1 + sqrt(1 - rho_J^2)) has rho = omega_opt - 1 (as has
    # every omega above it); SSOR at omega = 1 is symmetric Gauss-Seidel, whose
    # matrix is I - M^-1 A with M = (D - L) D^-1 (D - U)
    m = 12
    A = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    rj = np.cos(np.pi / (m + 1))
    assert O.spectral_radius(O.stationary_iteration_matrix(A, "jacobi")) == pytest.approx(rj, rel=1e-12)
    assert O.spectral_radius(O.stationary_iteration_matrix(A, "gs")) == pytest.approx(rj ** 2, rel=1e-10)
    w_opt = 2 / (1 + np.sqrt(1 - rj ** 2))
    # at omega_opt the SOR matrix has one defective eigenvalue: eigvals carry
    # ~sqrt(eps) of rounding there
    assert O.spectral_radius(O.stationary_iteration_matrix(A, "sor", omega=w_opt)) == \
        pytest.approx(w_opt - 1, rel=1e-6)
    for om in (1.8, 1.9):
        assert O.spectral_radius(O.stationary_iteration_matrix(A, "sor", omega=om)) == \
            pytest.approx(om - 1, rel=1e-6)
    D = np.diag(np.diag(A))
    Lm, Um = -np.tril(A, -1), -np.triu(A, 1)
    M = (D - Lm) @ np.linalg.solve(D, D - Um)
    G_sgs = np.eye(m) - np.linalg.solve(M, A)
    assert np.allclose(O.stationary_iteration_matrix(A, "ssor", omega=1.0), G_sgs, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------
# The multi-process form of the oracle iteration (the timed CPU baseline)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["grid", "lagged"])
def test_multiprocess_oracle_repeats_the_oracle_bitwise(case):
    # the same sub-circuit solves, spread over worker processes that exchange
    # the waves through shared memory with one sweep of delay: the same
    # history and iterate, bit for bit
    from oracle.vtm_oracle_mp import vtm_midpoint_mp
    if case == "grid":
        w = wl.grid2d(24, 24, 8, 6, Zc=0.5, seed=21, nrhs=2)
    else:
        w = wl.vccs_grid(24, 24, 8, 8, seed=3)
    A = w.csr()
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=1e-10, max_sweeps=3000)
    got = vtm_midpoint_mp(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=1e-10, max_sweeps=3000, workers=3)
    assert got.sweeps == ref.sweeps and got.converged == ref.converged
    assert np.array_equal(got.history, ref.history)
    assert np.array_equal(got.x, ref.x)
    assert np.array_equal(got.w_in, ref.w_in)
