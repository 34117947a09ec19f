"""The benchmark configurations at full size, in the modes the bench times:
what the oracle can check at any size (the FP64 residual, the reflection
matrices of sampled tiles, the tearing counts) since its literal sweeps are
far too slow for millions of unknowns.
"""
import numpy as np
import pytest
import torch

from oracle import vtm_oracle as O
from paper_0910_0663_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_CHECK = 1e-10 * (1 + 1e-4)


@pytest.fixture(scope="module")
def vtm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0910_0663_gb300 import build
    build.build()
    from paper_0910_0663_gb300 import vtm as V
    return V


@pytest.fixture(scope="module")
def power_grid():
    w = wl.c2_power_grid(Zc=1.0)
    return w, w.csr()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_power_grid_2048_as_benchmarked(vtm, power_grid, precision):
    w, A = power_grid
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                        stream=s)
        x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        x2, info2 = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)  # graph replay
    torch.cuda.synchronize()
    st = plan.stats()
    assert st["nparts"] == 4096 and st["nports"] == 516096
    assert st["sum_p2"] == 65282048 and st["sum_tri"] == 32899072
    assert st["sweep_kernel"] in (5, 6, 7, 8, 9, 10, 11) and st["packed_bytes"] > 0
    assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= TOL_CHECK
    assert torch.equal(x, x2) and info["sweeps"] == info2["sweeps"]
    plan.close()


def test_power_grid_2048_sampled_reflection_matrices(vtm, power_grid):
    w, A = power_grid
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    assert len(tear.port_g) == 516096
    node, remote, part, _ = plan.ports()
    for P in (0, 31, 2080, 4095):  # corner, edge, interior, corner tiles
        T_lib = plan.reflection(P)
        _, T_ref = O.reflection_ops(A, tear, P, 1.0 / w.Zc)
        sel = np.flatnonzero(part == P)
        ora = tear.tile_ports[P]
        pos = {k: i for i, k in enumerate(zip(tear.port_node[ora].tolist(), tear.port_remote[ora].tolist()))}
        pm = np.array([pos[k] for k in zip(node[sel].tolist(), remote[sel].tolist())])
        assert np.abs(T_lib - T_ref[np.ix_(pm, pm)]).max() < 1e-10
        # symmetric with its spectrum in (-1, 1] (Sec. VIII)
        assert np.abs(T_lib - T_lib.T).max() < 1e-12
        ev = np.linalg.eigvalsh(0.5 * (T_lib + T_lib.T))
        assert ev.min() > -1 and ev.max() <= 1 + 1e-12
    plan.close()


def test_vccs_1024_vtm_and_block_jacobi(vtm):
    # the unsymmetric configuration: both iterations reach 1e-10
    w = wl.c4_vccs()
    A = w.csr()
    b = torch.from_numpy(w.b[0]).cuda()
    for method in ("vtm", "bj"):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, method=method)
        x, info = plan.solve(b, tol=1e-10)
        assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= TOL_CHECK
        plan.close()
