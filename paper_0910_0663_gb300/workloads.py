"""Seeded synthetic circuit workloads (inputs only).

This module builds nodal-analysis systems ``A x = b`` (Sec. II, Eq. 1) of
resistor / RC networks together with a node partition and the right-hand
sides.  It holds none of the Virtual Transmission Method's arithmetic: no
tearing, no wave, no reflection operator.  Both the CUDA path's tests/bench
and the CPU oracle draw their inputs from here, so that the two sides see the
same bytes.

Recipes (all with ``numpy.random.default_rng(seed)``, draw order documented
per generator):

* ``grid2d``   5-point resistor grid with per-node ground conductance.  Used
  for the 32x32 worked case (4x4 tiles of 8x8), the 1024x1024 grids
  (256 tiles of 64x64) and the 64x64 sub-grid (4x4 tiles of 16x16).
* ``power_grid``  2048x2048 power-grid-shaped system: log-uniform edge
  conductances, 1% of nodes tied to ground by 10 S pads, every other node
  sinking U[0,1e-3] A; 32x32-node tiles.
* ``thermal3d``  128x128x32 7-point RC grid in backward-Euler form
  ``G + C/h``; partitioned by seeded random axis-aligned box cuts into 400
  boxes; 64 right-hand sides.
* ``vccs_grid``  the 2-D resistor grid plus voltage-controlled current
  sources (unsymmetric entries) at 5% of the nodes.

The paper's own test matrices (Table I) are not available; these recipes
stand in for its structured-grid (Grid2d/Grid3d) and unsymmetric
(Wang/Pchip) cases.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Workload:
    """One circuit system.

    ``indptr`` (int64, n+1), ``indices`` (int32), ``data`` (float64) hold
    ``A`` in CSR with sorted column indices.  ``partition`` (int32, n) maps
    node -> tile.  ``b`` has shape (nrhs, n): right-hand side ``r`` is
    ``b[r]``, i.e. the n x nrhs matrix stored column-major.
    ``edges`` (m x 2 int64) and ``g`` (m) are the branch list; ``ground``
    (n) the node-to-ground conductances (or C/h diagonal), so that
    ``A = sum_e g_e (e_i - e_j)(e_i - e_j)^T + diag(ground)`` for the
    symmetric recipes.
    """

    name: str
    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray
    partition: np.ndarray
    nparts: int
    b: np.ndarray
    Zc: float
    edges: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None
    ground: Optional[np.ndarray] = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return int(self.b.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))


def assemble_nodal(n: int, edges: np.ndarray, g: np.ndarray, ground: np.ndarray,
                   extra: Optional[tuple] = None):
    """Nodal matrix of a resistor network (Sec. II, Eq. 1; Lemma 1).

    Each branch (i, j) of conductance g adds g at (i,i),(j,j) and -g at
    (i,j),(j,i); ``ground[i]`` adds to (i,i).  ``extra = (rows, cols, vals)``
    adds further entries (controlled sources).  Returns sorted CSR arrays.
    """
    i = edges[:, 0]
    j = edges[:, 1]
    rows = [i, j, i, j, np.arange(n)]
    cols = [i, j, j, i, np.arange(n)]
    vals = [g, g, -g, -g, ground]
    if extra is not None:
        rows.append(extra[0])
        cols.append(extra[1])
        vals.append(extra[2])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return (A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64))


def grid_edges_2d(ny: int, nx: int) -> np.ndarray:
    """Branches of an ny x nx 5-point grid, node (r, c) -> r*nx + c.

    Order: horizontal branches row-major, then vertical branches row-major.
    """
    idx = np.arange(ny * nx, dtype=np.int64).reshape(ny, nx)
    h = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    v = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    return np.concatenate([h, v], axis=0)


def grid_edges_3d(nz: int, ny: int, nx: int) -> np.ndarray:
    """Branches of a 7-point grid, node (z, y, x) -> (z*ny + y)*nx + x.

    Order: x-branches, then y-branches, then z-branches, each in node order.
    """
    idx = np.arange(nz * ny * nx, dtype=np.int64).reshape(nz, ny, nx)
    ex = np.stack([idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()], axis=1)
    ey = np.stack([idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()], axis=1)
    ez = np.stack([idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()], axis=1)
    return np.concatenate([ex, ey, ez], axis=0)


def tile_partition_2d(ny: int, nx: int, th: int, tw: int) -> tuple:
    """Rectangular tiles of th x tw nodes; tile id row-major over the tile grid."""
    r = np.arange(ny)[:, None] // th
    c = np.arange(nx)[None, :] // tw
    ntx = (nx + tw - 1) // tw
    nty = (ny + th - 1) // th
    part = (r * ntx + c).astype(np.int32).ravel()
    return part, nty * ntx


def grid2d(ny: int = 32, nx: int = 32, th: int = 8, tw: int = 8, Zc: float = 1.0,
           seed: int = 0, nrhs: int = 1, g_lo: float = 0.5, g_hi: float = 2.0,
           ground: float = 1e-3, name: str = "grid2d") -> Workload:
    """SPD resistor grid: g ~ U[g_lo, g_hi] S, ``ground`` S on every node,
    b ~ U[-1, 1] A.  Draws: branch conductances (horizontal then vertical),
    then b (nrhs x n)."""
    rng = np.random.default_rng(seed)
    n = ny * nx
    edges = grid_edges_2d(ny, nx)
    g = rng.uniform(g_lo, g_hi, size=edges.shape[0])
    gnd = np.full(n, ground)
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    indptr, indices, data = assemble_nodal(n, edges, g, gnd)
    part, nparts = tile_partition_2d(ny, nx, th, tw)
    return Workload(name, n, indptr, indices, data, part, nparts, b, Zc, edges, g, gnd,
                    dict(grid=(ny, nx), tile=(th, tw), seed=seed))


def power_grid(ny: int = 2048, nx: int = 2048, th: int = 32, tw: int = 32, Zc: float = 1.0,
               seed: int = 0, pad_frac: float = 0.01, pad_g: float = 10.0,
               name: str = "power_grid") -> Workload:
    """Power-grid-shaped SPD system.

    g = 10**U[-1, 1] S (log-uniform in [0.1, 10]); round(pad_frac*n)
    distinct pad nodes (first entries of a seeded permutation) tied to ground
    by ``pad_g`` S with b = 0; every other node sinks U[0, 1e-3] A
    (b = -U[0, 1e-3]).  No other ground.  Draws: branch exponents
    (horizontal, vertical), permutation, then the sink currents.
    """
    rng = np.random.default_rng(seed)
    n = ny * nx
    edges = grid_edges_2d(ny, nx)
    g = 10.0 ** rng.uniform(-1.0, 1.0, size=edges.shape[0])
    npads = int(round(pad_frac * n))
    pads = rng.permutation(n)[:npads]
    gnd = np.zeros(n)
    gnd[pads] = pad_g
    b = -rng.uniform(0.0, 1e-3, size=(1, n))
    b[0, pads] = 0.0
    indptr, indices, data = assemble_nodal(n, edges, g, gnd)
    part, nparts = tile_partition_2d(ny, nx, th, tw)
    return Workload(name, n, indptr, indices, data, part, nparts, b, Zc, edges, g, gnd,
                    dict(grid=(ny, nx), tile=(th, tw), seed=seed, pads=npads))


def random_boxes(rng, dims: tuple, nboxes: int) -> list:
    """Seeded axis-aligned recursive box cuts.

    Repeatedly split the largest box (ties -> lowest id) along an axis drawn
    with probability proportional to its extent, at round(U[0.3, 0.7] *
    extent) from its low face (clamped to leave both halves non-empty), until
    ``nboxes`` boxes exist.  Boxes are (z0, z1, y0, y1, x0, x1).
    """
    boxes = [(0, dims[0], 0, dims[1], 0, dims[2])]

    def vol(bx):
        return (bx[1] - bx[0]) * (bx[3] - bx[2]) * (bx[5] - bx[4])

    while len(boxes) < nboxes:
        k = int(np.argmax([vol(bx) for bx in boxes]))
        bx = boxes[k]
        ext = np.array([bx[1] - bx[0], bx[3] - bx[2], bx[5] - bx[4]], dtype=float)
        ax = int(rng.choice(3, p=ext / ext.sum()))
        lo, hi = bx[2 * ax], bx[2 * ax + 1]
        cut = lo + int(round(rng.uniform(0.3, 0.7) * (hi - lo)))
        cut = min(max(cut, lo + 1), hi - 1)
        b1 = list(bx)
        b2 = list(bx)
        b1[2 * ax + 1] = cut
        b2[2 * ax] = cut
        boxes[k] = tuple(b1)
        boxes.append(tuple(b2))
    return boxes


def thermal3d(nz: int = 32, ny: int = 128, nx: int = 128, nboxes: int = 400, nrhs: int = 64,
              h: float = 1e-3, Zc: float = 1.0, seed: int = 0, min_box: int = 200,
              max_box: int = 3000, name: str = "thermal3d") -> Workload:
    """Backward-Euler RC thermal grid ``G + C/h``.

    g ~ U[0.5, 2] S on the 7-point branches, C ~ U[1e-3, 1e-2] F per node,
    b ~ U[-1, 1] A for ``nrhs`` independent right-hand sides.  Draws:
    branches (x, y, z), capacitances, b (nrhs x n), then the box cuts
    (repeated on the same stream until every box holds [min_box, max_box]
    nodes).
    """
    rng = np.random.default_rng(seed)
    n = nz * ny * nx
    edges = grid_edges_3d(nz, ny, nx)
    g = rng.uniform(0.5, 2.0, size=edges.shape[0])
    cap = rng.uniform(1e-3, 1e-2, size=n)
    diag = cap / h
    b = rng.uniform(-1.0, 1.0, size=(nrhs, n))
    for _attempt in range(64):
        boxes = random_boxes(rng, (nz, ny, nx), nboxes)
        vols = np.array([(bx[1] - bx[0]) * (bx[3] - bx[2]) * (bx[5] - bx[4]) for bx in boxes])
        if vols.min() >= min_box and vols.max() <= max_box:
            break
    else:
        raise RuntimeError("box partition: no admissible draw")
    part = np.empty((nz, ny, nx), dtype=np.int32)
    for k, bx in enumerate(boxes):
        part[bx[0]:bx[1], bx[2]:bx[3], bx[4]:bx[5]] = k
    indptr, indices, data = assemble_nodal(n, edges, g, diag)
    return Workload(name, n, indptr, indices, data, part.ravel(), nboxes, b, Zc, edges, g, diag,
                    dict(grid=(nz, ny, nx), boxes=boxes, seed=seed, h=h,
                         box_sizes=vols.tolist()))


def vccs_grid(ny: int = 1024, nx: int = 1024, th: int = 64, tw: int = 64, Zc: float = 1.0,
              seed: int = 0, frac: float = 0.05, gain: float = 0.3, max_hops: int = 3,
              name: str = "vccs_grid") -> Workload:
    """Resistor grid (as ``grid2d``) plus voltage-controlled current sources.

    round(frac*n) distinct controlled rows i (drawn without replacement);
    each picks a target j uniformly among the in-grid nodes at Manhattan
    distance 1..max_hops, and adds c = gamma * a_ii at (i, j) with
    gamma ~ U[-gain, gain]; |c| is added to a_ii (a_ii of the resistor grid)
    so that strict row diagonal dominance is kept.  Draws: branches, b, the
    controlled rows, one U[0,1) per row for the target, then gamma.
    """
    rng = np.random.default_rng(seed)
    n = ny * nx
    edges = grid_edges_2d(ny, nx)
    g = rng.uniform(0.5, 2.0, size=edges.shape[0])
    gnd = np.full(n, 1e-3)
    b = rng.uniform(-1.0, 1.0, size=(1, n))
    nv = int(round(frac * n))
    rows = rng.choice(n, size=nv, replace=False).astype(np.int64)
    u = rng.uniform(0.0, 1.0, size=nv)
    gamma = rng.uniform(-gain, gain, size=nv)
    # diagonal of the plain resistor grid
    deg_diag = gnd.copy()
    np.add.at(deg_diag, edges[:, 0], g)
    np.add.at(deg_diag, edges[:, 1], g)
    offs = [(dr, dc) for dr in range(-max_hops, max_hops + 1) for dc in range(-max_hops, max_hops + 1)
            if 1 <= abs(dr) + abs(dc) <= max_hops]
    offs = np.array(offs, dtype=np.int64)
    r0 = rows // nx
    c0 = rows % nx
    rr = r0[:, None] + offs[None, :, 0]
    cc = c0[:, None] + offs[None, :, 1]
    valid = (rr >= 0) & (rr < ny) & (cc >= 0) & (cc < nx)
    nvalid = valid.sum(axis=1)
    pick = np.minimum((u * nvalid).astype(np.int64), nvalid - 1)
    # index of the pick-th valid offset in each row
    csum = np.cumsum(valid, axis=1) - 1
    sel = np.argmax((csum == pick[:, None]) & valid, axis=1)
    cols = rr[np.arange(nv), sel] * nx + cc[np.arange(nv), sel]
    c = gamma * deg_diag[rows]
    ex_rows = np.concatenate([rows, rows])
    ex_cols = np.concatenate([cols, rows])
    ex_vals = np.concatenate([c, np.abs(c)])
    indptr, indices, data = assemble_nodal(n, edges, g, gnd, extra=(ex_rows, ex_cols, ex_vals))
    part, nparts = tile_partition_2d(ny, nx, th, tw)
    return Workload(name, n, indptr, indices, data, part, nparts, b, Zc, edges, g, gnd,
                    dict(grid=(ny, nx), tile=(th, tw), seed=seed, vccs=nv,
                         vccs_rows=rows, vccs_cols=cols, vccs_vals=c))


# --- the named workloads -------------------------------------------------

def c1_small_grid(seed: int = 0) -> Workload:
    """32x32 SPD grid, 4x4 tiles of 8x8, Zc = 1 ohm (1024 unknowns)."""
    return grid2d(32, 32, 8, 8, Zc=1.0, seed=seed, name="grid32_tiles8")


def c2_power_grid(Zc: float = 1.0, seed: int = 0, ny: int = 2048, nx: int = 2048) -> Workload:
    """2048x2048 power grid, 32x32-node tiles (4096 subdomains)."""
    return power_grid(ny, nx, 32, 32, Zc=Zc, seed=seed, name=f"power_grid{ny}_tiles32")


def c3_thermal(seed: int = 0, nrhs: int = 64) -> Workload:
    """128x128x32 RC thermal grid, 400 random boxes, 64 RHS."""
    return thermal3d(32, 128, 128, 400, nrhs=nrhs, seed=seed, name="thermal128x128x32_boxes400")


def c4_vccs(seed: int = 0, ny: int = 1024, nx: int = 1024) -> Workload:
    """1024x1024 grid with VCCS at 5% of nodes, 256 tiles of 64x64."""
    return vccs_grid(ny, nx, 64, 64, seed=seed, name=f"vccs_grid{ny}_tiles64")


def c5_grad_grid(seed: int = 0, ny: int = 1024, nx: int = 1024, th: int = 64, tw: int = 64) -> Workload:
    """1024x1024 SPD grid (as the 32x32 case), 256 tiles; IR-drop loss sum(x^2)."""
    return grid2d(ny, nx, th, tw, Zc=1.0, seed=seed, name=f"grid{ny}_tiles{th}")


def c5_subgrid(seed: int = 0) -> Workload:
    """The 64x64 instance of the same recipe, tiled 4x4 (16 tiles of 16x16 nodes)."""
    return grid2d(64, 64, 16, 16, Zc=1.0, seed=seed, name="grid64_tiles16")
