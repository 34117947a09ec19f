"""Plain FP64 CPU oracle of the Virtual Transmission Method (VTM).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or run anything in this package.  The CUDA library never calls it, and it
never calls the CUDA library: the two share no code, tables or helpers.

Everything here is slow and literal on purpose.  Each function follows one
passage of Wei & Yang, "Transmission Line Inspires A New Distributed
Algorithm to Solve the Linear System of Circuit" (arXiv 0910.0663):

* ``tear_midpoint``      Sec. V (wire tearing, four steps; Fig. 4) applied to a
                         disjoint node partition by tearing every cut branch at
                         its midpoint (reading R1, see ``tear_midpoint``).
* ``vtm_midpoint``       Sec. VI, Eq. 11 / Eq. 14: every sub-circuit solves its
                         own system with ``C + W`` on the twin rows and the
                         delayed waves ``W u_twin - i_twin`` on the right-hand
                         side; zero initial boundary values.
* ``vtm_midpoint_delayed``  VTM with stochastic line delays (Sec. XI, the
                         asynchronous/chaotic form).
* ``reflection_ops``     Sec. VIII: input admittance ``S = C - E D^-1 F`` and
                         voltage reflection matrix ``T = (W - S)(W + S)^-1``.
* ``line_admittance_choice``  Sec. VIII choices of W (alpha I, diagonal,
                         weighted overlapped block, Schur complement
                         approximation) as one admittance per virtual line.
* ``twin_split`` /
  ``vtm_twin``           Sec. V-VI with a vertex-separator interface (Example
                         1/2, the four-node example of Sec. IX, Eq. 15-21) and
                         a full characteristic-admittance matrix ``W``.
* ``direct_solve``       the reference answer ``x = A^-1 b`` (Eq. 1).
* ``backward_euler_march``  a transient of x_k = A^-1 (p_k + C/h x_(k-1)) by
                         direct solves (the time march of an RC network).
* ``block_jacobi``       the block Jacobi comparison method (Sec. X).
* ``stationary_*``       Jacobi / Gauss-Seidel / SOR / SSOR iteration matrices
                         (Sec. IX comparison).
* ``adjoint_gradients``  gradient of ``L = sum x^2`` w.r.t. branch
                         conductances, ground conductances and injections by a
                         dense adjoint solve.

Readings where the paper is silent (stopping rule: ``||b - A x^k||_2 /
||b||_2 <= tol`` checked after every sweep; one sweep = every sub-circuit
solves once, simultaneously; lagged controlled-source couplings) are stated
where they are used.

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
(closed forms, the paper's fixed-point and convergence theorems, brute force
on tiny circuits, the four-node example).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# Basic linear-algebra references
# ---------------------------------------------------------------------------

def csr_matrix(indptr, indices, data, n) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(data, np.float64), np.asarray(indices), np.asarray(indptr)),
                         shape=(n, n))


def residual_norms(A: sp.csr_matrix, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Relative residual ``||b - A x||_2 / ||b||_2`` per right-hand side.

    ``x`` and ``b`` have shape (nrhs, n)."""
    r = b - (A @ x.T).T
    return np.linalg.norm(r, axis=1) / np.linalg.norm(b, axis=1)


def direct_solve(A: sp.csr_matrix, b: np.ndarray) -> np.ndarray:
    """``x = A^-1 b`` (Eq. 1).  Dense LU with partial pivoting up to 4096
    unknowns, sparse LU (SuperLU) above.  ``b``: (nrhs, n)."""
    n = A.shape[0]
    if n <= 4096:
        lu = sla.lu_factor(A.toarray())
        return sla.lu_solve(lu, b.T).T
    lu = spla.splu(A.tocsc())
    return lu.solve(np.ascontiguousarray(b.T)).T


# ---------------------------------------------------------------------------
# Wire tearing of a disjoint node partition (Sec. V, reading R1/R2)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Tearing:
    """Result of ``tear_midpoint``.

    ``port_node[s]``   node ell(s) of the sub-circuit that owns port s
    ``port_remote[s]`` the node on the other end of the torn branch
    ``port_g[s]``      branch conductance g_e (each twin gets 2 g_e)
    ``port_tile[s]``   owning sub-circuit
    ``twin[s]``        the port at the other end of the same virtual line
    ``tile_ports[P]``  ports of P ordered by (ell, remote)
    ``tile_nodes[P]``  nodes of P in increasing order
    ``lag_*``          cut couplings that are not a branch (controlled
                       sources): entry (i, j) with value rho, applied with
                       one sweep of delay
    """

    n: int
    nparts: int
    partition: np.ndarray
    tile_nodes: list
    tile_ports: list
    port_node: np.ndarray
    port_remote: np.ndarray
    port_g: np.ndarray
    port_tile: np.ndarray
    twin: np.ndarray
    lag_i: np.ndarray
    lag_j: np.ndarray
    lag_rho: np.ndarray
    A_in: sp.csr_matrix  # A with every cut entry removed (block diagonal)


def tear_midpoint(A: sp.csr_matrix, partition: np.ndarray, nparts: int) -> Tearing:
    """Wire tearing (Sec. V, Steps 1-4) of a disjoint node partition.

    The paper tears at interfacial *nodes* shared by two sub-circuits.  With
    a disjoint partition every branch between nodes i in P and j in Q (P != Q)
    is first replaced by two conductances 2g in series meeting at a new node
    m (this changes nothing: eliminating m gives back a_ii and a_ij = -g).
    m is the interfacial node (Step 1); it is split into twins, one per side
    (Step 2); each twin keeps one of the two 2g conductances and no current
    source (Step 3: C = 2g + 2g, f = 0 + 0; Fig. 4 caption); the twins are
    joined by a lossless virtual line (Step 4).  This is level-one tearing.

    For a cut pair the branch conductance is the symmetric negative part
    g = -(a_ij + a_ji)/2.  If g > 0 the pair carries a virtual line and any
    remainder rho_ij = a_ij + g, rho_ji = a_ji + g is a lagged coupling; if
    g <= 0 both entries are lagged couplings (reading R2).
    """
    A = A.tocsr()
    n = A.shape[0]
    part = np.asarray(partition, dtype=np.int64)
    coo = A.tocoo()
    r, c, v = coo.row.astype(np.int64), coo.col.astype(np.int64), coo.data
    cut = part[r] != part[c]
    rc, cc, vc = r[cut], c[cut], v[cut]
    lo = np.minimum(rc, cc)
    hi = np.maximum(rc, cc)
    key = lo * n + hi
    ukey, inv = np.unique(key, return_inverse=True)
    a_lohi = np.zeros(len(ukey))
    a_hilo = np.zeros(len(ukey))
    fwd = rc < cc
    np.add.at(a_lohi, inv[fwd], vc[fwd])
    np.add.at(a_hilo, inv[~fwd], vc[~fwd])
    plo = ukey // n
    phi = ukey % n
    g = -(a_lohi + a_hilo) / 2.0
    wire = g > 0
    rho_lohi = np.where(wire, a_lohi + np.where(wire, g, 0.0), a_lohi)
    rho_hilo = np.where(wire, a_hilo + np.where(wire, g, 0.0), a_hilo)
    lag_i = np.concatenate([plo[rho_lohi != 0], phi[rho_hilo != 0]])
    lag_j = np.concatenate([phi[rho_lohi != 0], plo[rho_hilo != 0]])
    lag_rho = np.concatenate([rho_lohi[rho_lohi != 0], rho_hilo[rho_hilo != 0]])

    wlo, whi, wg = plo[wire], phi[wire], g[wire]
    # two ports per line; order inside each tile by (node, remote node)
    pn = np.concatenate([wlo, whi])
    pr = np.concatenate([whi, wlo])
    pg = np.concatenate([wg, wg])
    pt = part[pn]
    order = np.lexsort((pr, pn, pt))
    pn, pr, pg, pt = pn[order], pr[order], pg[order], pt[order]
    nw = len(wlo)
    # twin: the port whose (node, remote) is our (remote, node)
    pkey = pn * n + pr
    tkey = pr * n + pn
    srt = np.argsort(pkey)
    twin = srt[np.searchsorted(pkey[srt], tkey)]
    assert np.all(pn[twin] == pr) and len(pn) == 2 * nw

    tile_nodes = [np.flatnonzero(part == P) for P in range(nparts)]
    bounds = np.searchsorted(pt, np.arange(nparts + 1))
    tile_ports = [np.arange(bounds[P], bounds[P + 1]) for P in range(nparts)]
    keep = ~cut
    A_in = sp.csr_matrix((v[keep], (r[keep], c[keep])), shape=(n, n))
    return Tearing(n, nparts, part, tile_nodes, tile_ports, pn, pr, pg, pt, twin,
                   lag_i, lag_j, lag_rho, A_in)


def _line_admittance(tear: Tearing, W) -> np.ndarray:
    """Characteristic admittance per port.  ``W`` is a scalar (W = alpha I,
    Sec. VIII choice 1) or one value per port (a diagonal W; both ports of a
    line must then carry the same value)."""
    Wp = np.broadcast_to(np.asarray(W, dtype=np.float64), tear.port_g.shape).copy()
    assert np.allclose(Wp, Wp[tear.twin]), "both ends of a line need one admittance"
    return Wp


def line_admittance_choice(tear: Tearing, kind: str, alpha: float = 1.0,
                           radius: int = -1) -> np.ndarray:
    """Per-port characteristic admittance from the choices of Sec. VIII,
    for the midpoint tearing, where C_P = diag(2 g_s) is diagonal:

    ``'alpha'``  W = alpha I (choice 1).
    ``'diag'``   W = diag(C): 2 g_e on line e (choice 2; C is diagonal here,
                 so choice 3, W = C, is the same).
    ``'wob'``    W = alpha C: alpha 2 g_e (choice 4).
    ``'sca'``    the partial input admittance S~ = C - E~ D~^-1 F~ (choice 5)
                 with D~ = D_P restricted to the nodes of P within ``radius``
                 branches of ell(s) (radius < 0: all of P, so S~ = S_P); its
                 small elements are dropped down to the pattern of C, i.e.
                 its diagonal 2 g_s - 4 g_s^2 [D~^-1]_(ell, ell) is kept.  The
                 two ends of a line see different S~; the line takes the value
                 of its end in the lower-numbered sub-circuit (S~_1 of Sec.
                 VIII, "W = S~_1 or S~_2").
    """
    g = tear.port_g
    if kind == "alpha":
        return np.full(len(g), float(alpha))
    if kind == "diag":
        return 2.0 * g
    if kind == "wob":
        return float(alpha) * 2.0 * g
    if kind != "sca":
        raise ValueError(kind)
    S = np.empty(len(g))
    for P in range(tear.nparts):
        nodes = tear.tile_nodes[P]
        ports = tear.tile_ports[P]
        if len(ports) == 0:
            continue
        loc = np.full(tear.n, -1, dtype=np.int64)
        loc[nodes] = np.arange(len(nodes))
        D = tear.A_in[nodes][:, nodes].tolil()
        ell = loc[tear.port_node[ports]]
        for q, s in enumerate(ports):
            D[ell[q], ell[q]] += g[s]
        D = D.tocsr()
        for q, s in enumerate(ports):
            sel = np.arange(len(nodes))
            if radius >= 0:  # breadth-first: nodes within `radius` branches
                seen = {int(ell[q])}
                front = [int(ell[q])]
                for _ in range(radius):
                    nxt = []
                    for v in front:
                        for u in D.indices[D.indptr[v]:D.indptr[v + 1]]:
                            if int(u) not in seen:
                                seen.add(int(u))
                                nxt.append(int(u))
                    front = nxt
                sel = np.array(sorted(seen))
            Dt = D[sel][:, sel].toarray()
            e = (sel == ell[q]).astype(np.float64)
            z = np.linalg.solve(Dt, e)
            S[s] = 2 * g[s] - 4 * g[s] ** 2 * float(z @ e)
    low_end = tear.port_tile <= tear.port_tile[tear.twin]
    return np.where(low_end, S, S[tear.twin])


def local_system(A: sp.csr_matrix, tear: Tearing, P: int, Wp: np.ndarray) -> sp.csc_matrix:
    """Sub-circuit P's matrix of Eq. 11, ``[[C_P + W, E_P], [F_P, D_P]]``.

    Unknowns: the twin-node voltages u (ports of P, in ``tile_ports`` order)
    then the node voltages of P (``tile_nodes`` order).
    C_P = diag(2 g_s): each twin touches only its own node through 2 g_s.
    E_P = F_P^T: -2 g_s between twin s and its node ell(s).
    D_P = A_PP + sum_s g_s e_ell e_ell^T: the node keeps a_ii (which holds g
    for the torn branch) with the branch's g replaced by 2 g toward the twin.
    """
    nodes = tear.tile_nodes[P]
    ports = tear.tile_ports[P]
    p, m = len(ports), len(nodes)
    loc = np.full(tear.n, -1, dtype=np.int64)
    loc[nodes] = np.arange(m)
    App = tear.A_in[nodes][:, nodes].tocoo()
    g = tear.port_g[ports]
    ell = loc[tear.port_node[ports]]
    assert np.all(ell >= 0)
    rows = [np.arange(p), np.arange(p), p + ell, p + App.row, p + ell]
    cols = [np.arange(p), p + ell, np.arange(p), p + App.col, p + ell]
    vals = [2 * g + Wp[ports], -2 * g, -2 * g, App.data, g]
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(p + m, p + m))
    return M.tocsc()


@dataclasses.dataclass
class VTMResult:
    x: np.ndarray            # (nrhs, n) node voltages of the last sweep
    sweeps: int              # k at which every column met tol (or max_sweeps)
    converged: bool
    history: np.ndarray      # (sweeps, nrhs) relative residuals, sweep 1..k
    u: np.ndarray            # (nrhs, nports) twin-node voltages u^k
    i: np.ndarray            # (nrhs, nports) twin inflow currents i^k
    w_in: np.ndarray         # (nrhs, nports) incident waves used at sweep k


def vtm_midpoint(A: sp.csr_matrix, partition: np.ndarray, nparts: int, b: np.ndarray,
                 W=1.0, tol: float = 1e-10, max_sweeps: int = 100000,
                 tear: Optional[Tearing] = None, min_sweeps: int = 0,
                 keep_iterates: bool = False):
    """VTM with unit line delay (Sec. VI, Eq. 11 and Eq. 14).

    Sweep k, for every sub-circuit P at once (reading R6: k advances when all
    variables are updated, Sec. IX):
        [[C_P + W, E_P], [F_P, D_P]] [u_P^k; y_P^k]
            = [W u_twin^{k-1} - i_twin^{k-1}; b_P - sum_lag rho_ij x_j^{k-1}]
        i_P^k = -W u_P^k + W u_twin^{k-1} - i_twin^{k-1}
    with u^0 = i^0 = 0 and x^0 = 0 (Sec. VI).  After each sweep the node
    voltages x^k are assembled and the full residual b - A x^k is taken
    (reading R5).  ``b``: (nrhs, n).
    """
    A = A.tocsr()
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    nrhs, n = b.shape
    if tear is None:
        tear = tear_midpoint(A, partition, nparts)
    Wp = _line_admittance(tear, W)
    nports = len(tear.port_g)
    lus = [spla.splu(local_system(A, tear, P, Wp)) for P in range(nparts)]
    u = np.zeros((nrhs, nports))
    cur = np.zeros((nrhs, nports))
    x = np.zeros((nrhs, n))
    history = []
    iterates = []
    converged = False
    k = 0
    lag = sp.csr_matrix((tear.lag_rho, (tear.lag_i, tear.lag_j)), shape=(n, n))
    while k < max_sweeps:
        k += 1
        w_in = Wp * u[:, tear.twin] - cur[:, tear.twin]  # delayed incident wave
        rhs_nodes = b - (lag @ x.T).T
        u_new = np.empty_like(u)
        x_new = np.empty_like(x)
        for P in range(nparts):
            ports = tear.tile_ports[P]
            nodes = tear.tile_nodes[P]
            rhs = np.concatenate([w_in[:, ports].T, rhs_nodes[:, nodes].T], axis=0)
            sol = lus[P].solve(np.ascontiguousarray(rhs))
            u_new[:, ports] = sol[:len(ports)].T
            x_new[:, nodes] = sol[len(ports):].T
        cur = -Wp * u_new + w_in
        u = u_new
        x = x_new
        rel = residual_norms(A, x, b)
        history.append(rel)
        if keep_iterates:
            iterates.append(x.copy())
        if k >= min_sweeps and np.all(rel <= tol):
            converged = True
            break
    res = VTMResult(x, k, converged, np.array(history), u, cur, w_in)
    if keep_iterates:
        return res, iterates
    return res


def vtm_midpoint_delayed(A: sp.csr_matrix, partition: np.ndarray, nparts: int, b: np.ndarray,
                         W=1.0, tol: float = 1e-10, max_sweeps: int = 100000, max_delay: int = 2,
                         seed: int = 0, tear: Optional[Tearing] = None):
    """VTM with stochastic line delays (Sec. XI: "if the delays of virtual
    transmission lines are different and stochastic, VTM would turn to be a
    fully asynchronous and chaotic numerical algorithm").

    As ``vtm_midpoint``, except that at sweep k the wave arriving at port s
    left its twin d sweeps earlier, d drawn uniformly from 1..max_delay for
    every (port, sweep) by ``numpy.random.default_rng(seed)``:
        w_in(s)^k = W u_twin^(k-d) - i_twin^(k-d)   (zero before sweep 1).
    max_delay = 1 is ``vtm_midpoint``.  Returns a ``VTMResult``."""
    A = A.tocsr()
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    nrhs, n = b.shape
    if tear is None:
        tear = tear_midpoint(A, partition, nparts)
    Wp = _line_admittance(tear, W)
    nports = len(tear.port_g)
    rng = np.random.default_rng(seed)
    lus = [spla.splu(local_system(A, tear, P, Wp)) for P in range(nparts)]
    # sent[j] = outgoing wave W u - i of every port after sweep k - j
    sent = [np.zeros((nrhs, nports)) for _ in range(max_delay)]
    x = np.zeros((nrhs, n))
    u = np.zeros((nrhs, nports))
    cur = np.zeros((nrhs, nports))
    w_in = np.zeros((nrhs, nports))
    history = []
    lag = sp.csr_matrix((tear.lag_rho, (tear.lag_i, tear.lag_j)), shape=(n, n))
    converged = False
    k = 0
    while k < max_sweeps:
        k += 1
        d = rng.integers(1, max_delay + 1, size=nports)
        w_in = np.empty((nrhs, nports))
        for s_ in range(nports):
            w_in[:, s_] = sent[d[s_] - 1][:, tear.twin[s_]]
        rhs_nodes = b - (lag @ x.T).T
        u_new = np.empty_like(u)
        x_new = np.empty_like(x)
        for P in range(nparts):
            ports = tear.tile_ports[P]
            nodes = tear.tile_nodes[P]
            rhs = np.concatenate([w_in[:, ports].T, rhs_nodes[:, nodes].T], axis=0)
            sol = lus[P].solve(np.ascontiguousarray(rhs))
            u_new[:, ports] = sol[:len(ports)].T
            x_new[:, nodes] = sol[len(ports):].T
        cur = -Wp * u_new + w_in
        u = u_new
        x = x_new
        sent = [Wp * u - cur] + sent[:-1]
        rel = residual_norms(A, x, b)
        history.append(rel)
        if np.all(rel <= tol):
            converged = True
            break
    return VTMResult(x, k, converged, np.array(history), u, cur, w_in)


def reflection_ops(A: sp.csr_matrix, tear: Tearing, P: int, W=1.0):
    """Input admittance and voltage reflection matrix of sub-circuit P
    (Sec. VIII, Example 3): ``S_P = C_P - E_P D_P^-1 F_P`` and
    ``T_P = (W - S_P)(W + S_P)^-1``, dense, ports in ``tile_ports`` order.
    Returns (S_P, T_P)."""
    Wp = _line_admittance(tear, W)
    nodes = tear.tile_nodes[P]
    ports = tear.tile_ports[P]
    p = len(ports)
    loc = np.full(tear.n, -1, dtype=np.int64)
    loc[nodes] = np.arange(len(nodes))
    g = tear.port_g[ports]
    ell = loc[tear.port_node[ports]]
    D = tear.A_in[nodes][:, nodes].toarray()
    np.add.at(D, (ell, ell), g)
    E = np.zeros((p, len(nodes)))
    E[np.arange(p), ell] = -2 * g
    C = np.diag(2 * g)
    S = C - E @ np.linalg.solve(D, E.T)
    Wm = np.diag(Wp[ports])
    T = (Wm - S) @ np.linalg.inv(Wm + S)
    return S, T


def port_excitation(A: sp.csr_matrix, tear: Tearing, P: int, b: np.ndarray) -> np.ndarray:
    """``r_P = f_P - E_P D_P^-1 g_P`` (Appendix, Eq. 23) with f_P = 0 and
    g_P = b restricted to P.  ``b``: (nrhs, n) -> (nrhs, p)."""
    nodes = tear.tile_nodes[P]
    ports = tear.tile_ports[P]
    loc = np.full(tear.n, -1, dtype=np.int64)
    loc[nodes] = np.arange(len(nodes))
    g = tear.port_g[ports]
    ell = loc[tear.port_node[ports]]
    D = tear.A_in[nodes][:, nodes].toarray()
    np.add.at(D, (ell, ell), g)
    E = np.zeros((len(ports), len(nodes)))
    E[np.arange(len(ports)), ell] = -2 * g
    return -(E @ np.linalg.solve(D, np.atleast_2d(b)[:, nodes].T)).T


def backward_euler_march(A: sp.csr_matrix, cdiag: np.ndarray, p: np.ndarray,
                         x0: Optional[np.ndarray] = None) -> np.ndarray:
    """Backward-Euler transient of an RC network: A = G + C/h, and for
    k = 1..nsteps  A x_k = p_k + (C/h) x_{k-1}  (cdiag = C/h per node), each
    step by a direct solve (Eq. 1).  ``p``: (nsteps, n); returns (nsteps, n)."""
    A = A.tocsr()
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    x = np.zeros(A.shape[0]) if x0 is None else np.asarray(x0, dtype=np.float64)
    out = np.empty_like(p)
    for k in range(p.shape[0]):
        x = direct_solve(A, (p[k] + cdiag * x)[None])[0]
        out[k] = x
    return out


# ---------------------------------------------------------------------------
# Vertex-separator wire tearing with a full W (Sec. V-VI, Sec. IX)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class TwinSplit:
    """Two sub-circuits of a level-one wire tearing (Example 1, Eq. 7-8).

    Sub-circuit s has unknowns [u_s (twins of the interface nodes, in
    ``interface`` order); y_s (inner nodes, ``inner[s]`` order)] and system
    ``[[C_s, E_s], [F_s, D_s]] [u_s; y_s] = [f_s; g_s] + [i_s; 0]``.
    """

    interface: np.ndarray
    inner: list
    C: list
    E: list
    F: list
    D: list
    f: list
    g: list


def twin_split(A: np.ndarray, b: np.ndarray, inner_sub: np.ndarray, alpha: float = 0.5,
               diag_split=None) -> TwinSplit:
    """Split a dense system into two sub-circuits (Sec. V, Steps 1-3).

    ``inner_sub[v]`` is 0 or 1 for an inner node and -1 for an interfacial
    node.  Step 3 splits what is attached to an interfacial node v: its
    diagonal (conductance to ground) and its source current go ``alpha`` to
    twin 1 and ``1 - alpha`` to twin 2 (C_1 + C_2 = C, f_1 + f_2 = f); an
    entry (v, k) toward an inner node k goes to the twin on k's side; an
    entry between two interfacial nodes is split like the diagonal.  Inner
    rows keep their entries, with interfacial columns renamed to their own
    side's twin.  Inner nodes of different sub-circuits must not touch
    (Eq. 6).  ``diag_split`` optionally gives per-interface-node fractions.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    n = A.shape[0]
    iface = np.flatnonzero(inner_sub < 0)
    inner = [np.flatnonzero(inner_sub == 0), np.flatnonzero(inner_sub == 1)]
    assert np.all(A[np.ix_(inner[0], inner[1])] == 0) and np.all(A[np.ix_(inner[1], inner[0])] == 0)
    q = len(iface)
    fr = np.full(q, alpha) if diag_split is None else np.asarray(diag_split, dtype=np.float64)
    C, E, F, D, f, gg = [], [], [], [], [], []
    for s in (0, 1):
        frac = fr if s == 0 else 1.0 - fr
        Cs = A[np.ix_(iface, iface)] * frac[:, None]
        Es = A[np.ix_(iface, inner[s])].copy()
        Fs = A[np.ix_(inner[s], iface)].copy()
        Ds = A[np.ix_(inner[s], inner[s])].copy()
        C.append(Cs)
        E.append(Es)
        F.append(Fs)
        D.append(Ds)
        f.append(b[:, iface] * frac[None, :])
        gg.append(b[:, inner[s]])
    return TwinSplit(iface, inner, C, E, F, D, f, gg)


def twin_schur(ts: TwinSplit, s: int):
    """``S_s = C_s - E_s D_s^-1 F_s`` and ``r_s = f_s - E_s D_s^-1 g_s``
    (Sec. VIII Example 3; Appendix Eq. 23-24)."""
    if len(ts.inner[s]) == 0:
        return ts.C[s].copy(), ts.f[s].copy()
    S = ts.C[s] - ts.E[s] @ np.linalg.solve(ts.D[s], ts.F[s])
    r = ts.f[s] - (ts.E[s] @ np.linalg.solve(ts.D[s], ts.g[s].T)).T
    return S, r


def vtm_twin(ts: TwinSplit, W: np.ndarray, nsweeps: int):
    """VTM on a two-way vertex-separator tearing with admittance matrix W
    (Sec. VI, Eq. 11 and Eq. 14; W is |interface| x |interface|).

    Returns per sweep k = 1..nsweeps the assembled solution estimate: inner
    voltages from each side and the two twin-voltage vectors u_1^k, u_2^k,
    together with the currents, as a list of dicts.
    """
    W = np.atleast_2d(np.asarray(W, dtype=np.float64))
    q = len(ts.interface)
    nrhs = ts.f[0].shape[0]
    u = [np.zeros((nrhs, q)), np.zeros((nrhs, q))]
    cur = [np.zeros((nrhs, q)), np.zeros((nrhs, q))]
    mats = []
    for s in (0, 1):
        M = np.block([[ts.C[s] + W, ts.E[s]], [ts.F[s], ts.D[s]]])
        mats.append(sla.lu_factor(M))
    out = []
    for _k in range(nsweeps):
        new_u, new_i, ys = [], [], []
        for s in (0, 1):
            o = 1 - s
            w_in = (W @ u[o].T).T - cur[o]
            rhs = np.concatenate([(ts.f[s] + w_in).T, ts.g[s].T], axis=0)
            sol = sla.lu_solve(mats[s], rhs)
            us = sol[:q].T
            new_u.append(us)
            ys.append(sol[q:].T)
            new_i.append(-(W @ us.T).T + w_in)
        u, cur = new_u, new_i
        out.append(dict(u=[x.copy() for x in u], i=[x.copy() for x in cur], y=ys))
    return out


def twin_assemble(ts: TwinSplit, n: int, state: dict, side: int = 0) -> np.ndarray:
    """Full-length voltage vector from one sweep of ``vtm_twin``: inner nodes
    from their own sub-circuit, interfacial nodes from twin ``side``."""
    nrhs = state["u"][0].shape[0]
    x = np.zeros((nrhs, n))
    x[:, ts.interface] = state["u"][side]
    for s in (0, 1):
        x[:, ts.inner[s]] = state["y"][s]
    return x


# ---------------------------------------------------------------------------
# Comparison methods (Sec. IX-X)
# ---------------------------------------------------------------------------

def block_jacobi(A: sp.csr_matrix, partition: np.ndarray, nparts: int, b: np.ndarray,
                 tol: float = 1e-10, max_sweeps: int = 100000):
    """Block Jacobi over the same sub-circuits: ``x_P^k = A_PP^-1 (b_P -
    sum_{Q != P} A_PQ x_Q^{k-1})``, x^0 = 0; same residual and stopping rule
    as ``vtm_midpoint``.  Returns (x, sweeps, converged, history)."""
    A = A.tocsr()
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    part = np.asarray(partition)
    nodes = [np.flatnonzero(part == P) for P in range(nparts)]
    lus = [spla.splu(A[nd][:, nd].tocsc()) for nd in nodes]
    coo = A.tocoo()
    off = part[coo.row] != part[coo.col]
    A_off = sp.csr_matrix((coo.data[off], (coo.row[off], coo.col[off])), shape=A.shape)
    x = np.zeros_like(b)
    hist = []
    k = 0
    conv = False
    while k < max_sweeps:
        k += 1
        rhs = b - (A_off @ x.T).T
        xn = np.empty_like(x)
        for P in range(nparts):
            xn[:, nodes[P]] = lus[P].solve(np.ascontiguousarray(rhs[:, nodes[P]].T)).T
        x = xn
        rel = residual_norms(A, x, b)
        hist.append(rel)
        if np.all(rel <= tol):
            conv = True
            break
    return x, k, conv, np.array(hist)


def stationary_iteration_matrix(A: np.ndarray, method: str, omega: float = 1.0,
                                blocks=None) -> np.ndarray:
    """Iteration matrix G of x^{k+1} = G x^k + c for the classical methods
    (Saad, ch. 4): splitting A = D - L - U (D diagonal, L strictly lower, U
    strictly upper, signs included in L and U).
    Jacobi: D^-1 (L + U).  GS: (D - L)^-1 U.  SOR: (D - wL)^-1 ((1-w) D + wU).
    SSOR: backward SOR sweep after the forward one.  BJ: block diagonal
    splitting over ``blocks`` (list of index arrays)."""
    A = np.asarray(A, dtype=np.float64)
    D = np.diag(np.diag(A))
    L = -np.tril(A, -1)
    U = -np.triu(A, 1)
    if method == "jacobi":
        return np.linalg.solve(D, L + U)
    if method == "gs":
        return np.linalg.solve(D - L, U)
    if method == "sor":
        return np.linalg.solve(D - omega * L, (1 - omega) * D + omega * U)
    if method == "ssor":
        fwd = np.linalg.solve(D - omega * L, (1 - omega) * D + omega * U)
        bwd = np.linalg.solve(D - omega * U, (1 - omega) * D + omega * L)
        return bwd @ fwd
    if method == "bj":
        M = np.zeros_like(A)
        for blk in blocks:
            M[np.ix_(blk, blk)] = A[np.ix_(blk, blk)]
        return np.linalg.solve(M, M - A)
    raise ValueError(method)


def spectral_radius(G: np.ndarray) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(G))))


# ---------------------------------------------------------------------------
# Gradients of an IR-drop loss (adjoint of Eq. 1)
# ---------------------------------------------------------------------------

def adjoint_gradients(n: int, edges: np.ndarray, g: np.ndarray, ground: np.ndarray,
                      b: np.ndarray):
    """For ``A = sum_e g_e (e_i - e_j)(e_i - e_j)^T + diag(ground)``,
    ``x = A^-1 b`` and ``L = sum_i x_i^2``: lambda = A^-T dL/dx = A^-T (2x),
    dL/db = lambda, dL/dg_e = -(lambda_i - lambda_j)(x_i - x_j),
    dL/dground_i = -lambda_i x_i.  Dense LU.  Returns
    (L, x, lam, dg, dground, db)."""
    A = np.zeros((n, n))
    i, j = edges[:, 0], edges[:, 1]
    np.add.at(A, (i, i), g)
    np.add.at(A, (j, j), g)
    np.add.at(A, (i, j), -g)
    np.add.at(A, (j, i), -g)
    A[np.arange(n), np.arange(n)] += ground
    lu = sla.lu_factor(A)
    x = sla.lu_solve(lu, b)
    L = float(np.sum(x * x))
    lam = sla.lu_solve(lu, 2 * x, trans=1)
    dg = -(lam[i] - lam[j]) * (x[i] - x[j])
    dground = -lam * x
    return L, x, lam, dg, dground, lam.copy()
