"""Unsymmetric systems (controlled sources) and block Jacobi on the GPU.

Cut controlled-source entries are applied with one sweep of delay (reading
R2), inside the same sweep as the virtual lines; block Jacobi is the same
machinery without lines.  Both are compared with the oracle sweep for sweep.
"""
import numpy as np
import pytest
import torch

from oracle import vtm_oracle as O
from paper_0910_0663_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vtm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0910_0663_gb300 import build
    build.build()
    from paper_0910_0663_gb300 import vtm as V
    return V


def _same_count_and_x(k_gpu, k_ref, x_gpu, x_ref, hist, tol, x_rel=1e-11):
    if k_gpu != k_ref:
        assert abs(k_gpu - k_ref) == 1
        assert abs(hist[min(k_gpu, k_ref) - 1].max() - tol) <= 0.01 * tol
    else:
        assert np.abs(x_gpu - x_ref).max() <= x_rel * np.abs(x_ref).max()


@pytest.mark.parametrize("ny,tile", [(24, 8), (96, 32)])
def test_vccs_vtm_matches_oracle(vtm, ny, tile):
    w = wl.vccs_grid(ny, ny, tile, tile, seed=3)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    st = plan.stats()
    assert st["symmetric"] == 0 and st["nlagged"] > 0
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=1e-10)
    assert ref.converged
    _same_count_and_x(info["sweeps"], ref.sweeps, x.cpu().numpy().reshape(w.b.shape), ref.x,
                      ref.history, 1e-10)
    assert O.residual_norms(A, x.cpu().numpy().reshape(w.b.shape), w.b).max() <= 1e-10


@pytest.mark.parametrize("case", ["vccs", "spd"])
def test_block_jacobi_matches_oracle(vtm, case):
    w = wl.vccs_grid(48, 48, 12, 12, seed=5) if case == "vccs" else \
        wl.grid2d(48, 48, 12, 12, seed=5, ground=0.05)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, method="bj")
    assert plan.stats()["nports"] == 0
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    xr, kr, conv, hist = O.block_jacobi(A, w.partition, w.nparts, w.b, tol=1e-10)
    assert conv
    _same_count_and_x(info["sweeps"], kr, x.cpu().numpy().reshape(w.b.shape), xr, hist, 1e-10)


def test_residual_history_with_lagged_couplings(vtm):
    w = wl.vccs_grid(32, 32, 8, 8, seed=7)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=0.7)
    plan.set_options(history_len=40)
    plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / 0.7, tol=0, max_sweeps=40)
    assert np.allclose(plan.history, ref.history[:, 0], rtol=1e-9, atol=1e-14)


def test_adjoint_of_unsymmetric_system(vtm):
    w = wl.vccs_grid(32, 32, 8, 8, seed=8)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    gvec = np.random.default_rng(1).uniform(-1, 1, w.n)
    lam, info = plan.adjoint(torch.from_numpy(gvec).cuda(), tol=1e-11)
    lam_star = np.linalg.solve(A.toarray().T, gvec)
    assert np.abs(lam.cpu().numpy() - lam_star).max() <= 1e-8 * np.abs(lam_star).max()
