"""Asynchronous VTM (lines with different, varying delays): one cooperative
launch in which every tile reads the waves its neighbours last wrote.  The
iterates depend on timing, so the checks are the ones the paper's fixed-point
argument gives: the FP64-verified residual meets the tolerance and x is the
direct solution; the oracle's stochastic-delay VTM converges on the same
systems (pinned on the CPU).
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


@pytest.mark.parametrize("precision,shape", [("fp32", (256, 32)), ("fp32", (192, 48)), ("bf16", (256, 32)),
                                                 ("fp16", (256, 32))])
def test_async_vtm_reaches_the_direct_solution(vtm, precision, shape):
    n, t = shape
    w = wl.power_grid(n, n, t, t, Zc=1.0, seed=71)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                    method="async")
    x_star = O.direct_solve(A, w.b)
    for _ in range(2):  # timing differs between runs; both must converge
        x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        xs = x.cpu().numpy()[None]
        assert O.residual_norms(A, xs, w.b).max() <= TOL_CHECK
        assert np.abs(xs - x_star).max() <= 1e-7 * np.abs(x_star).max()
        assert info["sweeps"] > 0


def test_async_and_synchronous_methods_switch_on_one_plan(vtm):
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=72)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision="fp32")
    b = torch.from_numpy(w.b[0]).cuda()
    x1, i1 = plan.solve(b, tol=1e-10)
    plan.set_options(method="async")
    x2, i2 = plan.solve(b, tol=1e-10)
    plan.set_options(method="vtm")
    x3, i3 = plan.solve(b, tol=1e-10)
    assert torch.equal(x1, x3) and i1["sweeps"] == i3["sweeps"]
    for x in (x1, x2):
        assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= TOL_CHECK
    with pytest.raises(vtm.VTMError):
        plan.set_options(method="bj")  # block Jacobi is planned differently


def test_async_needs_the_packed_low_precision_sweeps(vtm):
    w = wl.power_grid(64, 64, 16, 16, Zc=1.0, seed=73)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, method="async")
    with pytest.raises(vtm.VTMError):
        plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)  # FP64 plan
    plan.set_options(method="async", precision="fp32")
    plan.factor()
    x, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert O.residual_norms(w.csr(), x.cpu().numpy()[None], w.b[:1]).max() <= TOL_CHECK
