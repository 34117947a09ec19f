"""Backward-Euler time march of the RC thermal grid (A = G + C/h), each step a
VTM solve warm-started from the previous state, against the oracle's march by
direct solves.
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


def _thermal(nsteps, seed):
    return wl.thermal3d(8, 24, 24, 12, nrhs=nsteps, seed=seed, min_box=100, max_box=1200)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_march_matches_the_oracle(vtm, precision):
    # each step meets 1e-10 relative residual; cond(G + C/h) stays below ~40
    # here (C/h in [1, 10] S, g in [0.5, 2] S), so each state is within 1e-8
    w = _thermal(6, seed=51)
    A = w.csr()
    x0 = np.random.default_rng(3).uniform(-1, 1, w.n)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision)
    X, info = plan.march(w.ground, w.b, x0=x0, tol=1e-10)
    ref = O.backward_euler_march(A, w.ground, w.b, x0)
    Xs = X.cpu().numpy()
    for k in range(6):
        assert np.abs(Xs[k] - ref[k]).max() <= 1e-8 * np.abs(ref[k]).max()
    assert info["relres"] <= 1e-10
    # the first step matches one plain solve of its right-hand side
    b1 = w.b[0] + w.ground * x0
    x1, _ = plan.solve(torch.from_numpy(b1).cuda(), tol=1e-10)
    assert np.abs(x1.cpu().numpy() - Xs[0]).max() <= 1e-8 * np.abs(Xs[0]).max()


def test_warm_start_saves_sweeps_on_a_settling_transient(vtm):
    # constant injections: after the first step each state starts close to the
    # next one, so the march needs fewer sweeps than cold solves of each step
    w = _thermal(1, seed=52)
    A = w.csr()
    nsteps = 8
    p = np.tile(w.b[0], (nsteps, 1))
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    X, info = plan.march(w.ground, p, tol=1e-10)
    ref = O.backward_euler_march(A, w.ground, p)
    assert np.abs(X.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    cold = 0
    Xs = X.cpu().numpy()
    for k in range(nsteps):
        prev = Xs[k - 1] if k else np.zeros(w.n)
        _, inf = plan.solve(torch.from_numpy(p[k] + w.ground * prev).cuda(), tol=1e-10)
        cold += inf["sweeps"]
    assert info["sweeps"] < cold
