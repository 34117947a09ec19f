"""Gradients of the IR-drop loss L = sum x^2 through the VTM solve.

The forward VTM solve and the adjoint VTM solve run on the GPU (FP32 sweeps
inside FP64 refinement for the forward pass of the large case); the branch
gradient -(lam_i - lam_j)(x_i - x_j) is a CUDA kernel.  Checked against
(1) the oracle's dense adjoint on the 64x64 grid and (2) central finite
differences (step 1e-6) of the loss on 64 random parameters of the
1024x1024 grid.
"""
import math

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


def _network(vtm, w, precision="fp64", **kw):
    return vtm.Network(w.n, w.edges, w.indptr, w.indices, w.partition, w.nparts, Zc=w.Zc,
                       precision=precision, g0=w.g, ground0=w.ground, **kw)


def test_netmap_values_reproduce_the_nodal_matrix(vtm):
    w = wl.grid2d(20, 24, 5, 6, seed=3)
    net = _network(vtm, w)
    vals = net.values(torch.from_numpy(w.g).cuda(), torch.from_numpy(w.ground).cuda())
    # same entries; diagonals may differ in the last bit (summation order)
    assert torch.allclose(vals.cpu(), torch.from_numpy(w.data), rtol=1e-15, atol=0)
    net.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gradients_match_dense_adjoint_64x64(vtm, precision):
    w = wl.c5_subgrid()
    net = _network(vtm, w, precision=precision)
    g = torch.from_numpy(w.g).cuda().requires_grad_(True)
    gr = torch.from_numpy(w.ground).cuda().requires_grad_(True)
    b = torch.from_numpy(w.b[0]).cuda().requires_grad_(True)
    # 1e-11: the adjoint right-hand side 2x is smooth, so its FP64 residual
    # floor (about cond(A) * eps) sits near 1e-12
    x = net.solve(g, gr, b, tol=1e-11)
    loss = (x * x).sum()
    loss.backward()
    L, x_ref, lam, dg, dgr, db = O.adjoint_gradients(w.n, w.edges, w.g, w.ground, w.b[0])
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))
    assert rel(x.detach().cpu().numpy(), x_ref) < 1e-9
    assert rel(g.grad.cpu().numpy(), dg) < 1e-9
    assert rel(gr.grad.cpu().numpy(), dgr) < 1e-9
    assert rel(b.grad.cpu().numpy(), db) < 1e-9
    net.close()


def test_gradients_match_central_differences_1024(vtm):
    w = wl.c5_grad_grid()
    rng = np.random.default_rng(2024)
    # forward in FP32 sweeps + FP64 refinement, then the adjoint solve
    net = _network(vtm, w, precision="fp32")
    g = torch.from_numpy(w.g).cuda().requires_grad_(True)
    b = torch.from_numpy(w.b[0]).cuda().requires_grad_(True)
    gr = torch.from_numpy(w.ground).cuda()
    x = net.solve(g, gr, b, tol=1e-11)
    (x * x).sum().backward()
    dg = g.grad.cpu().numpy()
    db = b.grad.cpu().numpy()
    net.close()
    # finite differences: FP64 VTM with a fixed sweep count, so that both
    # sides of each difference run the same (smooth) iteration
    fd_net = _network(vtm, w, precision="fp64")
    _, info = fd_net.plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-11)
    K = info["sweeps"] + 20
    fd_net.plan.set_options(max_sweeps=K)

    def loss(gv, bv):
        fd_net._set(gv, gr)
        xx, inf = fd_net.plan.solve(bv, tol=1e-300, check=False)
        assert inf["sweeps"] == K
        return math.fsum((xx.cpu().numpy() ** 2).tolist())

    g0 = torch.from_numpy(w.g).cuda()
    b0 = torch.from_numpy(w.b[0]).cuda()
    L0 = loss(g0, b0)

    def fd_errors(h, edges, nodes):
        errs = []
        for e in edges:
            gp, gm = g0.clone(), g0.clone()
            gp[e] += h
            gm[e] -= h
            fd = (loss(gp, b0) - loss(gm, b0)) / (2 * h)
            errs.append(abs(fd - dg[e]) / abs(dg[e]))
        for i in nodes:
            bp, bm = b0.clone(), b0.clone()
            bp[i] += h
            bm[i] -= h
            fd = (loss(g0, bp) - loss(g0, bm)) / (2 * h)
            errs.append(abs(fd - db[i]) / abs(db[i]))
        return np.array(errs)

    # parameters whose gradient is not tiny compared with the loss noise
    big_e = np.flatnonzero(np.abs(dg) > 1e-2 * np.abs(dg).max())
    big_n = np.flatnonzero(np.abs(db) > 1e-2 * np.abs(db).max())
    edges = rng.choice(big_e, 32, replace=False)
    nodes = rng.choice(big_n, 32, replace=False)
    # step 1e-6: the difference of two losses of size L0 carries rounding of
    # about 1e-14 L0 from the sweeps, i.e. an absolute error near 1e-14 L0 / 2e-6
    err6 = fd_errors(1e-6, edges, nodes)
    noise = 1e-14 * L0 / 2e-6
    scale = np.concatenate([np.abs(dg[edges]), np.abs(db[nodes])])
    assert np.all(err6 * scale < 20 * noise + 1e-5 * scale), (err6.max(), noise)
    # step 1e-3: rounding is 1000x smaller and the truncation error of the
    # central difference (h^2 L'''/6) stays below 1e-6 relative
    err3 = fd_errors(1e-3, edges[:16], nodes[:16])
    fd_net.close()
    assert err3.max() < 1e-5, err3.max()
