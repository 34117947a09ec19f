"""Element-by-element parity of the low-precision sweeps with the oracle.

The benchmark's path stores T_P in FP16 or BF16 (FP32 for the FP32 mode),
carries the waves in FP32 and refines in FP64.  These tests compare what
that path computes with the oracle entry by entry, on the 256x256 power
grid (64 sub-circuits of 32x32 nodes, 126 ports each), at bounds that follow
from the storage precision:

* stored T_P: every entry the sweeps read (the packed 16x16 blocks) is the
  oracle's (W - S)(W + S)^-1 (Sec. VIII) rounded once to the storage type:
  |T~ - T| <= u |T| + floor, u = 2^-24 (FP32), 2^-11 (FP16), 2^-8 (BF16);
  floor = 2^-25 for FP16 (half its subnormal spacing), plus 1e-11 for the
  FP64 difference between the library's and the oracle's T (itself pinned
  at 1e-11 by the FP64 parity tests);
* the refined solution x: for SPD A, ||x - x*||_2 <= ||b - A x||_2 / lambda_min(A)
  exactly, so x is compared with the oracle's direct solution at that
  bound (residual and lambda_min both computed by the oracle), plus the
  direct solution's own error bound of the same form;
* the iterate after k sweeps of the first inner solve (the plain VTM
  iteration on b): each sweep adds at most u |T| |w| of storage rounding
  per entry and the reflection operators do not expand errors in the
  2-norm (spectrum in (-1, 1], Sec. VIII), so after k sweeps the relative
  error is at most k u gamma (gamma = max_P |||T_P|||_inf, the oracle's), doubled
  for the FP32 waves, c and recovery (FP32 band solves for BF16/FP16).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import vtm_oracle as O
from paper_0910_0663_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

U = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
FLOOR = {"fp32": 1e-40, "bf16": 1e-40, "fp16": 2.0 ** -25}


@pytest.fixture(scope="module")
def vtm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0910_0663_gb300 import build
    build.build()
    from paper_0910_0663_gb300 import vtm as V
    return V


@pytest.fixture(scope="module")
def grid():
    w = wl.power_grid(256, 256, 32, 32, Zc=1.0, seed=4)
    A = w.csr()
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    T = [O.reflection_ops(A, tear, P, 1.0 / w.Zc)[1] for P in range(w.nparts)]
    gamma = max(float(np.abs(t).sum(axis=1).max()) for t in T)
    lam_min = float(spla.eigsh(A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    x_star = O.direct_solve(A, w.b[:1])[0]
    r_star = float(np.linalg.norm(w.b[0] - A @ x_star))
    return dict(w=w, A=A, tear=tear, T=T, gamma=gamma, lam_min=lam_min, x_star=x_star, r_star=r_star)


def _perm(plan, tear, P):
    node, remote, part, _ = plan.ports()
    sel = np.flatnonzero(part == P)
    ora = tear.tile_ports[P]
    pos = {k: i for i, k in enumerate(zip(tear.port_node[ora].tolist(), tear.port_remote[ora].tolist()))}
    return np.array([pos[k] for k in zip(node[sel].tolist(), remote[sel].tolist())])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_stored_reflection_entries_are_the_oracles_rounded_once(vtm, grid, precision):
    w, tear = grid["w"], grid["tear"]
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision)
    worst = 0.0
    for P in range(w.nparts):
        Tq, esize, packed = plan.reflection_stored(P)
        assert packed and esize == (4 if precision == "fp32" else 2)
        perm = _perm(plan, tear, P)
        Tr = grid["T"][P][np.ix_(perm, perm)]
        err = np.abs(Tq - Tr)
        bound = U[precision] * np.abs(Tr) + FLOOR[precision] + 1e-11
        assert np.all(err <= bound), (P, float((err - bound).max()))
        assert np.all(np.abs(Tq) <= 1.0)  # spectrum in (-1, 1] => entries in [-1, 1]
        worst = max(worst, float((err / (np.abs(Tr) + 1e-300))[np.abs(Tr) > 1e-3].max()))
    # the rounding is really there (not the FP64 copy) and within one unit
    assert 0.1 * U[precision] < worst <= U[precision] * (1 + 1e-6) + 1e-8
    plan.close()


@pytest.mark.parametrize("precision,kernel", [("fp32", 9), ("bf16", 9), ("fp16", 9), ("bf16", 11),
                                              ("fp16", 11)])
def test_refined_solution_against_the_direct_solution(vtm, grid, precision, kernel):
    w, A = grid["w"], grid["A"]
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                    sweep_kernel=kernel)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert plan.stats()["sweep_kernel"] == kernel
    xs = x.cpu().numpy()
    r = float(np.linalg.norm(w.b[0] - A @ xs))
    assert r <= 1e-10 * np.linalg.norm(w.b[0])
    err = float(np.linalg.norm(xs - grid["x_star"]))
    bound = (r + grid["r_star"]) / grid["lam_min"]
    assert err <= bound * (1 + 1e-6), (err, bound)
    rel_inf = float(np.abs(xs - grid["x_star"]).max() / np.abs(grid["x_star"]).max())
    print(f"\n{precision} kernel {kernel}: ||x-x*||_2 = {err:.3e} <= {bound:.3e}; rel inf {rel_inf:.2e}; "
          f"sweeps {info['sweeps']}, steps {info['outer_steps']}")
    plan.close()


@pytest.mark.parametrize("precision,kernel", [("fp32", 9), ("bf16", 9), ("fp16", 9), ("bf16", 11),
                                              ("fp16", 11)])
def test_first_inner_solve_iterates_against_the_oracle(vtm, grid, precision, kernel):
    w, A = grid["w"], grid["A"]
    kmax = 10
    _, its = O.vtm_midpoint(A, w.partition, w.nparts, w.b[:1], W=1 / w.Zc, tol=0, max_sweeps=kmax,
                            keep_iterates=True)
    for k in (1, 2, kmax):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                        sweep_kernel=kernel, max_sweeps=k, inner_tol=1e-14)
        x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-300, check=False)
        assert info["sweeps"] == k and info["outer_steps"] == 1
        assert plan.stats()["sweep_kernel"] == kernel
        ref = its[k - 1][0]
        rel = float(np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max())
        bound = 2.0 * (k * U[precision] * grid["gamma"] + 64 * 2.0 ** -24)
        print(f"\n{precision} kernel {kernel} sweep {k}: rel err {rel:.3e} (bound {bound:.3e}, "
              f"gamma {grid['gamma']:.3f})")
        assert rel <= bound
        plan.close()
