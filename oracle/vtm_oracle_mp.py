"""The oracle's VTM iteration spread over host processes (CPU baseline).

TEST INFRASTRUCTURE ONLY, like ``vtm_oracle``: only ``tests/`` and
``bench.py``'s CPU-baseline and reference legs may use it; the CUDA library
never does, and this module never touches it.

``vtm_midpoint_mp`` runs exactly the iteration of ``vtm_oracle.vtm_midpoint``
(Sec. VI, Eq. 11 / Eq. 14 with unit line delay, zero initial values, the
full residual ``||b - A x^k|| / ||b||`` after every sweep) with the
sub-circuits dealt round ``workers`` processes.  That is the paper's own
setting (Sec. VI, the three VTM steps: every processor solves its
sub-circuits, then the boundary waves travel to the neighbours): each
worker factors the twin-row systems of its sub-circuits once, and in every
sweep reads the previous sweep's (u, i) of all ports from shared memory,
solves its sub-circuits and writes their new (u, i) and node voltages; the
parent assembles nothing (the workers write into one shared x) and takes the
residual.  Every sub-circuit solve is the same SuperLU solve of the same
matrix and right-hand side as in ``vtm_midpoint``, so the iterates and the
residual history are the same bits.

Processes start with the ``spawn`` method (safe after CUDA has been used in
the parent) and exchange data through ``multiprocessing.shared_memory``; a
pipe per worker orders the exchange (the parent sends the sweep number k,
the worker answers when its sub-circuits are done; reads of sweep k see only
slot k-1, writes go to slot k: delay one sweep).  A worker that dies is
reported, not waited for.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import threading
from multiprocessing import connection as mp_connection
from multiprocessing import shared_memory

import numpy as np
import scipy.sparse.linalg as spla

from . import vtm_oracle as O


def _views(buf, nrhs, n, nports):
    """(u[2], cur[2], x[2], r) views into one shared block."""
    off = 0
    out = []
    for shape in ((2, nrhs, nports), (2, nrhs, nports), (2, nrhs, n), (nrhs, n)):
        size = int(np.prod(shape))
        out.append(np.ndarray(shape, np.float64, buffer=buf, offset=off * 8))
        off += size
    return out


def _nbytes(nrhs, n, nports):
    return 8 * (4 * nrhs * nports + 3 * nrhs * n)


def _worker(name, shape, conn):
    nrhs, n, nports = shape
    A, tear, Wp, tiles, rows, b = conn.recv()
    shm = shared_memory.SharedMemory(name=name)
    try:
        u, cur, x, r = _views(shm.buf, nrhs, n, nports)
        lus = {P: spla.splu(O.local_system(A, tear, P, Wp)) for P in tiles}
        A_rows = A[rows[0]:rows[1]]
        lag = None
        if len(tear.lag_rho):
            import scipy.sparse as sp
            lag = sp.csr_matrix((tear.lag_rho, (tear.lag_i, tear.lag_j)), shape=(n, n))
        conn.send(0)  # factored
        while True:
            k = conn.recv()  # sweep number, or 0 to stop
            if k <= 0:
                break
            prv, nxt = (k - 1) % 2, k % 2
            for P in tiles:
                ports = tear.tile_ports[P]
                nodes = tear.tile_nodes[P]
                tw = tear.twin[ports]
                w_in = Wp[ports] * u[prv][:, tw] - cur[prv][:, tw]
                rhs_nodes = b[:, nodes]
                if lag is not None:
                    rhs_nodes = rhs_nodes - (lag @ x[prv].T).T[:, nodes]
                rhs = np.concatenate([w_in.T, rhs_nodes.T], axis=0)
                sol = lus[P].solve(np.ascontiguousarray(rhs))
                u_new = sol[:len(ports)].T
                u[nxt][:, ports] = u_new
                cur[nxt][:, ports] = -Wp[ports] * u_new + w_in
                x[nxt][:, nodes] = sol[len(ports):].T
            conn.send(k)
            # the residual b - A x^k of this worker's block of rows (each entry
            # is the same sum as in the whole product)
            if conn.recv() != k:
                break
            r[:, rows[0]:rows[1]] = b[:, rows[0]:rows[1]] - (A_rows @ x[nxt].T).T
            conn.send(k)
    finally:
        del u, cur, x, r
        shm.close()


def _gather(conns, procs):
    """Wait for one message from every worker; fail if a worker died."""
    pending = set(range(len(conns)))
    while pending:
        ready = mp_connection.wait([conns[i] for i in pending], timeout=5.0)
        if not ready:
            dead = [i for i in pending if not procs[i].is_alive()]
            if dead:
                raise RuntimeError(f"oracle worker(s) {dead} exited")
            continue
        for c in ready:
            i = conns.index(c)
            c.recv()
            pending.discard(i)


def vtm_midpoint_mp(A, partition, nparts, b, W=1.0, tol=1e-10, max_sweeps=100000, workers=None):
    """``vtm_oracle.vtm_midpoint`` (same arguments, same result and history)
    with the sub-circuits spread over ``workers`` processes (default: every
    host core).  Returns a ``VTMResult``."""
    A = A.tocsr()
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    nrhs, n = b.shape
    tear = O.tear_midpoint(A, partition, nparts)
    Wp = O._line_admittance(tear, W)
    nports = len(tear.port_g)
    workers = max(1, min(int(workers or os.cpu_count() or 1), nparts))
    # deal the sub-circuits round the workers, largest first (balanced work)
    order = sorted(range(nparts), key=lambda P: -len(tear.tile_nodes[P]))
    groups = [order[i::workers] for i in range(workers)]
    bounds = np.linspace(0, n, workers + 1).astype(np.int64)
    ctx = mp.get_context("spawn")
    shm = shared_memory.SharedMemory(create=True, size=_nbytes(nrhs, n, nports))
    procs, conns = [], []
    try:
        u, cur, x, r = _views(shm.buf, nrhs, n, nports)
        u[:] = 0.0
        cur[:] = 0.0
        x[:] = 0.0
        for g in groups:
            here, there = ctx.Pipe()
            p = ctx.Process(target=_worker, args=(shm.name, (nrhs, n, nports), there), daemon=True)
            p.start()
            procs.append(p)
            conns.append(here)
        # the inputs go out on threads, so that the workers start up together
        senders = [threading.Thread(target=c.send, args=((A, tear, Wp, g, (int(bounds[i]), int(bounds[i + 1])), b),))
                   for i, (c, g) in enumerate(zip(conns, groups))]
        for t in senders:
            t.start()
        for t in senders:
            t.join()
        _gather(conns, procs)  # every worker has factored its sub-circuits
        bn = np.linalg.norm(b, axis=1)
        history = []
        k = 0
        converged = False
        while k < max_sweeps:
            k += 1
            for c in conns:
                c.send(k)
            _gather(conns, procs)  # sweep k done everywhere
            for c in conns:
                c.send(k)
            _gather(conns, procs)  # r = b - A x^k
            rel = np.linalg.norm(r, axis=1) / bn  # as residual_norms
            history.append(rel)
            if np.all(rel <= tol):
                converged = True
                break
        for c in conns:
            c.send(0)
        for p in procs:
            p.join(timeout=30)
        s = k % 2
        res = O.VTMResult(x[s].copy(), k, converged, np.array(history), u[s].copy(), cur[s].copy(),
                          Wp * u[1 - s][:, tear.twin] - cur[1 - s][:, tear.twin])
        del u, cur, x, r
        return res
    finally:
        for p in procs:
            if p.is_alive():
                p.terminate()
        shm.close()
        shm.unlink()


def cpu_model() -> str:
    """The host CPU's model name (``/proc/cpuinfo``), or the machine type."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "hardware", "cpu model"):
                    return line.split(":", 1)[1].strip()
            fh.seek(0)
            parts = {ln.split(":")[0].strip(): ln.split(":", 1)[1].strip() for ln in fh if ":" in ln}
            if "CPU implementer" in parts:
                return f"Arm implementer {parts['CPU implementer']} part {parts.get('CPU part', '?')}"
    except OSError:
        pass
    import platform
    return platform.machine()
