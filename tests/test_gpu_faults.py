"""Failure reporting, made on the host (nothing here faults, traps or hangs a
GPU): a NaN right-hand side, a singular sub-circuit, a divergent iteration.
Each returns its status, and the plan (or a new one) keeps working.  Also the
intermediate iterates against the oracle's: x after sweeps 1, 2 and 10.
"""
import numpy as np
import pytest
import scipy.sparse as sp
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


def test_nan_in_b_is_reported_as_divergence_and_the_plan_stays_usable(vtm):
    from paper_0910_0663_gb300 import _vtm as C
    w = wl.grid2d(32, 32, 8, 8, seed=81)
    A = w.csr()
    for precision in ("fp64", "fp32"):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision)
        b = torch.from_numpy(w.b[0].copy()).cuda()
        b[17] = float("nan")
        x = torch.empty_like(b)
        st, _ = C.vtm_solve(plan.handle, b, x, 1, 1e-10, check=False)
        assert st == C.VTM_EDIVERGED
        x2, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        assert O.residual_norms(A, x2.cpu().numpy()[None], w.b[:1]).max() <= 1e-10 * (1 + 1e-4)


def test_singular_sub_circuit_is_reported(vtm):
    # a floating two-node island (one branch, no path to ground) as its own
    # sub-circuit: its local matrix [[g, -g], [-g, g]] has a zero pivot
    from paper_0910_0663_gb300 import _vtm as C
    w = wl.grid2d(8, 8, 4, 4, seed=82)
    n = w.n + 2
    A = sp.lil_matrix((n, n))
    A[:w.n, :w.n] = w.csr()
    A[w.n, w.n] = A[w.n + 1, w.n + 1] = 1.0
    A[w.n, w.n + 1] = A[w.n + 1, w.n] = -1.0
    A = A.tocsr()
    A.sort_indices()
    part = np.concatenate([w.partition, [w.nparts, w.nparts]]).astype(np.int32)
    with pytest.raises(C.VTMError) as e:
        vtm.Plan(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, part, w.nparts + 1, Zc=1.0)
    assert e.value.status == C.VTM_ESINGULAR
    # the same system without the island is fine
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    x, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert O.residual_norms(w.csr(), x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10 * (1 + 1e-4)


def test_divergent_block_jacobi_is_reported(vtm):
    # the paper's four-node op-amp circuit (Sec. IX, Eq. 15): block Jacobi over
    # the blocks {1, 2}, {3, 4} has spectral radius 100 (pinned on the CPU)
    from paper_0910_0663_gb300 import _vtm as C
    A = sp.csr_matrix(np.array([[1, -10, 0, 0], [0, 1, 0, 10], [10, 0, 1, 0], [0, 0, 10, 1]], float))
    A.sort_indices()
    part = np.array([0, 0, 1, 1], np.int32)
    plan = vtm.Plan(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, part, 2, Zc=1.0,
                    method="bj", max_sweeps=200)
    b = torch.ones(4, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    st, info = C.vtm_solve(plan.handle, b, x, 1, 1e-10, check=False)
    assert st == C.VTM_EDIVERGED
    assert info.sweeps < 200


@pytest.mark.parametrize("k", [1, 2, 10])
def test_iterates_after_k_sweeps_match_the_oracle(vtm, k):
    # a sweep limit of k returns x of sweep k (VTM_ENOCONV); the oracle's
    # literal Eq. 11 iterate of the same sweep agrees to 1e-12
    w = wl.c1_small_grid()
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, max_sweeps=k)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-300, check=False)
    assert info["sweeps"] == k
    _, its = O.vtm_midpoint(A, w.partition, w.nparts, w.b[:1], W=1 / w.Zc, tol=0, max_sweeps=k,
                            keep_iterates=True)
    ref = its[k - 1][0]
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_stalled_refinement_is_reported(vtm, precision):
    # an inner tolerance of 0.9 lets every inner solve stop after a sweep or
    # two, so a refinement step gains less than the 10x (FP32) / 2x (BF16) a
    # step must gain: VTM_ENOCONV long before the 40-step limit, with the
    # iterate so far; the same plan with default options then solves
    from paper_0910_0663_gb300 import _vtm as C
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=83)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                    inner_tol=0.9)
    b = torch.from_numpy(w.b[0]).cuda()
    x = torch.empty_like(b)
    st, info = C.vtm_solve(plan.handle, b, x, 1, 1e-10, check=False)
    assert st == C.VTM_ENOCONV
    assert "stalled" in C.vtm_last_error_detail()
    assert 1 <= info.outer_steps < 40 and info.relres > 1e-10
    rel = O.residual_norms(A, x.cpu().numpy()[None], w.b[:1])[0]
    assert rel == pytest.approx(info.relres, rel=1e-6)
    plan.set_options(inner_tol=0.0)
    x2, info2 = plan.solve(b, tol=1e-10)
    assert O.residual_norms(A, x2.cpu().numpy()[None], w.b[:1]).max() <= 1e-10


@pytest.mark.parametrize("kernel", [8, 10])
def test_bounded_dataflow_wait_times_out_and_the_plan_recovers(vtm, kernel):
    # flow_lag = -1: every tile waits for the residual decision of its own
    # sweep, which needs that very sweep -- a wait on a flag that nothing
    # sets.  With a short poll limit (4096 polls, about a millisecond) the
    # wait gives up, the launch ends and the solve returns VTM_ETIMEOUT; the
    # same plan with the default options then solves.  The bulk-copy waits
    # of kernels 2 and 7 are not shortened (no CTA leaves with a copy into
    # its shared memory in flight).
    from paper_0910_0663_gb300 import _vtm as C
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=84)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision="fp16",
                    sweep_kernel=kernel, wait_polls=4096, flow_lag=-1)
    b = torch.from_numpy(w.b[0]).cuda()
    x = torch.empty_like(b)
    st, _ = C.vtm_solve(plan.handle, b, x, 1, 1e-10, check=False)
    assert st == C.VTM_ETIMEOUT
    assert "bounded wait" in C.vtm_last_error_detail()
    plan.set_options(wait_polls=0, flow_lag=0)
    x2, info = plan.solve(b, tol=1e-10)
    assert plan.stats()["sweep_kernel"] == kernel
    assert O.residual_norms(A, x2.cpu().numpy()[None], w.b[:1]).max() <= 1e-10
