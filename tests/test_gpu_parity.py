"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Floating-point bars (FP64 path):
* sweep counts equal to the oracle's (the same linear iteration and the
  same stopping rule); +-1 is accepted only when the oracle's residual at
  that sweep is within 1% of the tolerance;
* node voltages at the same sweep count within 1e-11 relative (the two
  sides evaluate the same iteration in different orders: the oracle solves
  the twin-row system of Eq. 11, the library applies the condensed
  reflection matrices);
* reflection matrices within 1e-11 of (W - S)(W + S)^-1;
* the returned relative residual <= tol (checked by the oracle's own SpMV).
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


def _match_ports(plan, tear, P):
    """Permutation from the library's port order of tile P to the oracle's."""
    node, remote, part, twin = plan.ports()
    sel = np.flatnonzero(part == P)
    lib_keys = list(zip(node[sel].tolist(), remote[sel].tolist()))
    ora = tear.tile_ports[P]
    ora_keys = list(zip(tear.port_node[ora].tolist(), tear.port_remote[ora].tolist()))
    pos = {k: i for i, k in enumerate(ora_keys)}
    return np.array([pos[k] for k in lib_keys])


def _check_against_oracle(vtm, w, tol=1e-10, x_rel=1e-11, Zc=None):
    Zc = w.Zc if Zc is None else Zc
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=Zc)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=tol)
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1.0 / Zc, tol=tol)
    assert ref.converged
    k_gpu, k_ref = info["sweeps"], ref.sweeps
    if k_gpu != k_ref:
        assert abs(k_gpu - k_ref) == 1
        near = ref.history[min(k_gpu, k_ref) - 1].max()
        assert abs(near - tol) <= 0.01 * tol
    else:
        xs = x.cpu().numpy().reshape(w.b.shape)
        assert np.abs(xs - ref.x).max() <= x_rel * np.abs(ref.x).max()
    rel = O.residual_norms(A, x.cpu().numpy().reshape(w.b.shape), w.b)
    assert rel.max() <= tol
    # both are FP64 norms of a residual that is 1e-10 of b: rounding of the
    # individual residual entries shows in the 4th-5th digit
    assert info["relres"] == pytest.approx(rel.max(), rel=1e-3)
    return plan, info, ref


def test_small_grid_fp64_matches_oracle(vtm):
    w = wl.c1_small_grid()
    plan, info, ref = _check_against_oracle(vtm, w)
    assert info["outer_steps"] == 1


def test_small_grid_reflection_matrices(vtm):
    w = wl.c1_small_grid()
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    for P in range(w.nparts):
        T_lib = plan.reflection(P)
        _, T_ref = O.reflection_ops(A, tear, P, 1.0 / w.Zc)
        perm = _match_ports(plan, tear, P)
        assert np.abs(T_lib - T_ref[np.ix_(perm, perm)]).max() < 1e-11


def test_interface_residual_history_matches_full_residual(vtm):
    # the library's residual (torn branches only) equals the oracle's full
    # b - A x^k at every sweep (interior rows are solved exactly)
    w = wl.grid2d(24, 24, 8, 6, Zc=0.5, seed=21)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    plan.set_options(history_len=60)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    h = plan.history
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=0, max_sweeps=60)
    k = min(60, info["sweeps"])
    assert np.allclose(h[:k], ref.history[:k, 0], rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("Zc", [0.25, 1.0, 4.0])
def test_power_grid_zc_sweep(vtm, Zc):
    w = wl.power_grid(128, 128, 32, 32, Zc=Zc, seed=2)
    _check_against_oracle(vtm, w)


def test_ragged_tiles_and_random_partition(vtm):
    w = wl.grid2d(21, 26, 6, 7, Zc=0.7, seed=5, ground=0.01)
    _check_against_oracle(vtm, w)
    rng = np.random.default_rng(7)
    part = rng.integers(0, 7, w.n).astype(np.int32)
    part[:7] = np.arange(7)
    w2 = wl.Workload("rand", w.n, w.indptr, w.indices, w.data, part, 7, w.b, 1.3)
    _check_against_oracle(vtm, w2)


def test_thermal_boxes_small(vtm):
    w = wl.thermal3d(6, 12, 12, 12, nrhs=3, seed=1, min_box=20, max_box=400)
    _check_against_oracle(vtm, w)


def test_single_partition_is_one_direct_solve(vtm):
    w = wl.grid2d(20, 20, 20, 20, seed=3)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, 1, Zc=1.0)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-12)
    assert info["sweeps"] == 1
    x_star = np.linalg.solve(w.csr().toarray(), w.b[0])
    assert np.abs(x.cpu().numpy() - x_star).max() <= 1e-12 * np.abs(x_star).max()


def test_fixed_point_is_direct_solution(vtm):
    w = wl.c1_small_grid()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=4.0)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-13)
    x_star = np.linalg.solve(w.csr().toarray(), w.b[0])
    assert np.abs(x.cpu().numpy() - x_star).max() <= 1e-9 * np.abs(x_star).max()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_mixed_precision_reaches_fp64_tolerance(vtm, precision):
    w = wl.power_grid(256, 256, 32, 32, Zc=1.0, seed=4)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    rel = O.residual_norms(w.csr(), x.cpu().numpy()[None], w.b)
    assert rel.max() <= 1e-10
    assert info["outer_steps"] >= 2


def test_host_and_device_buffers_agree(vtm):
    w = wl.grid2d(16, 16, 4, 8, seed=6)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    xd, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    xh, _ = plan.solve(torch.from_numpy(w.b[0]), tol=1e-10)
    assert not xh.is_cuda
    assert torch.equal(xd.cpu(), xh)
    # reruns are bit-identical (fixed-order reductions)
    xd2, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert torch.equal(xd, xd2)


def test_multiple_columns(vtm):
    # column by column (batch=1): each column is the single-RHS solve, bit for bit
    w = wl.grid2d(16, 16, 8, 8, seed=8, nrhs=3)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, batch=1)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    for r in range(3):
        xr, _ = plan.solve(torch.from_numpy(w.b[r]).cuda(), tol=1e-10)
        assert torch.equal(xr, x[r])
    # batched (default): every column meets the tolerance
    plan_b = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    xb, info_b = plan_b.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    assert O.residual_norms(w.csr(), xb.cpu().numpy(), w.b).max() <= 1e-10


def test_zero_rhs_and_errors(vtm):
    from paper_0910_0663_gb300 import _vtm as C
    w = wl.grid2d(8, 8, 4, 4, seed=9)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    x, info = plan.solve(torch.zeros(w.n, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(x) == 0
    bad = w.partition.copy()
    bad[3] = 99
    with pytest.raises(C.VTMError) as e:
        vtm.Plan(w.indptr, w.indices, w.data, bad, w.nparts, Zc=1.0)
    assert e.value.status == C.VTM_EINVAL
    empty = np.zeros(w.n, np.int32)
    with pytest.raises(C.VTMError) as e:
        vtm.Plan(w.indptr, w.indices, w.data, empty, 2, Zc=1.0)
    assert e.value.status == C.VTM_EINVAL
    with pytest.raises(C.VTMError) as e:
        vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=-1.0)
    assert e.value.status == C.VTM_EINVAL
    p2 = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, factor=False)
    with pytest.raises(C.VTMError) as e:
        p2.solve(torch.from_numpy(w.b[0]).cuda())
    assert e.value.status == C.VTM_ENOTFACTORED
    # sweep limit -> ENOCONV with the last iterate
    p3 = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, max_sweeps=5)
    x, info = p3.solve(torch.from_numpy(w.b[0]).cuda(), check=False)
    assert info["sweeps"] == 5 and info["relres"] > 1e-10


def test_set_values_then_refactor(vtm):
    w = wl.grid2d(16, 16, 8, 8, seed=10)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    g2 = w.g * 1.3
    ip, ix, d2 = wl.assemble_nodal(w.n, w.edges, g2, w.ground)
    assert np.array_equal(ip, w.indptr) and np.array_equal(ix, w.indices)
    plan.set_values(d2)
    plan.factor()
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-11)
    A2 = O.csr_matrix(ip, ix, d2, w.n)
    x_star = np.linalg.solve(A2.toarray(), w.b[0])
    assert np.abs(x.cpu().numpy() - x_star).max() <= 1e-8 * np.abs(x_star).max()


@pytest.mark.parametrize("hub", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp16"])
def test_residual_in_both_matrix_forms(vtm, precision, hub):
    # the single-column residual reads A in ELL form when every row has at
    # most 8 entries (the 5-point grid) and in CSR form otherwise (a hub node
    # tied to 12 more nodes, in its own tile and three others: a row of 15):
    # in both the reported relative residual is the oracle's ||b - A x|| / ||b||
    # of the returned x (up to the rounding of r at this level), and x solves
    # A x = b
    w = wl.grid2d(32, 32, 8, 8, seed=13)
    edges, g = w.edges, w.g
    if hub:
        extra = np.array([[0, j] for j in (2, 3, 4, 5, 6, 7, 16, 24, 34, 40, 48, 56)], dtype=edges.dtype)
        edges = np.concatenate([edges, extra])
        g = np.concatenate([g, np.full(len(extra), 0.7)])
    ip, ix, data = wl.assemble_nodal(w.n, edges, g, w.ground)
    assert (np.diff(ip).max() > 8) == hub
    plan = vtm.Plan(ip, ix, data, w.partition, w.nparts, Zc=1.0, precision=precision)
    A = O.csr_matrix(ip, ix, data, w.n)
    for _ in range(2):
        x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        xs = x.cpu().numpy()
        rel = np.linalg.norm(w.b[0] - A @ xs) / np.linalg.norm(w.b[0])
        assert rel <= 1e-10
        assert abs(info["relres"] - rel) <= 0.1 * rel
    x_star = np.linalg.solve(A.toarray(), w.b[0])
    assert np.abs(xs - x_star).max() <= 1e-7 * np.abs(x_star).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16", "fp16"])
def test_solves_before_and_after_a_refactor(vtm, precision):
    # the captured sweep graphs of every precision are rebuilt after a new
    # factorisation: single-column and 4-column solves before and after
    # set_values + factor each match the direct solution of their matrix
    w = wl.grid2d(32, 32, 8, 8, seed=11)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, precision=precision)
    B = np.random.default_rng(3).uniform(-1, 1, (4, w.n))
    for data in (w.data, wl.assemble_nodal(w.n, w.edges, w.g * 1.7, w.ground)[2]):
        if data is not w.data:
            plan.set_values(data)
            plan.factor()
        Ad = O.csr_matrix(w.indptr, w.indices, data, w.n).toarray()
        for rhs in (B[0], B):
            x, info = plan.solve(torch.from_numpy(np.ascontiguousarray(rhs)).cuda(), tol=1e-11)
            x_star = np.linalg.solve(Ad, rhs.T).T
            assert np.abs(x.cpu().numpy() - x_star).max() <= 1e-8 * np.abs(x_star).max()


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 12])
def test_every_sweep_kernel_matches_oracle(vtm, kernel):
    # direct-load, bulk-copy staged and vector-load (256 / 128 threads)
    # kernels compute the same FP64 sweep; kernel 12 the same iteration in
    # double-float arithmetic on the packed blocks (about 48 bits: the
    # iterate at equal sweep count still agrees to 1e-11)
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=12)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, sweep_kernel=kernel)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=1e-10)
    assert abs(info["sweeps"] - ref.sweeps) <= 1
    if info["sweeps"] == ref.sweeps:
        xs = x.cpu().numpy().reshape(w.b.shape)
        assert np.abs(xs - ref.x).max() <= 1e-11 * np.abs(ref.x).max()


@pytest.mark.parametrize("precision,kernel,shape", [("fp32", 5, (90, 18)), ("fp32", 6, (192, 48)),
                                                    ("fp32", 7, (90, 18)), ("fp32", 7, (192, 48)),
                                                    ("bf16", 5, (192, 48)), ("bf16", 6, (90, 18)),
                                                    ("bf16", 7, (192, 48)), ("fp32", 8, (90, 18)),
                                                    ("fp32", 8, (192, 48)), ("bf16", 8, (90, 18)),
                                                    ("fp16", 5, (192, 48)), ("fp16", 6, (90, 18)),
                                                    ("fp16", 7, (90, 18)), ("fp16", 8, (192, 48)),
                                                    ("fp32", 9, (90, 18)), ("fp32", 9, (192, 48)),
                                                    ("bf16", 9, (90, 18)), ("fp16", 9, (192, 48)),
                                                    ("fp32", 10, (90, 18)), ("fp16", 10, (192, 32)),
                                                    ("fp16", 11, (90, 18)), ("bf16", 11, (90, 18)),
                                                    ("fp16", 11, (192, 32)), ("bf16", 11, (256, 32))])
def test_packed_symmetric_sweeps_follow_the_oracle(vtm, precision, kernel, shape):
    # T_P is symmetric (scalar W, symmetric A): the packed kernels read the
    # 16x16 blocks on and above the diagonal only.  18x18 tiles have 72, 54 or
    # 36 ports (a ragged last block); 48x48 tiles up to 192 ports (12 blocks).
    # The first inner solve is the plain VTM iteration on b, so its residual
    # history follows the oracle's up to the rounding of the stored T_P.
    n, t = shape
    w = wl.grid2d(n, n, t, t, seed=16)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                    precision=precision, sweep_kernel=kernel)
    plan.set_options(history_len=40)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    st = plan.stats()
    assert st["sweep_kernel"] == kernel and st["packed_bytes"] > 0
    assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b[:1], W=1 / w.Zc, tol=0, max_sweeps=40)
    h, href = plan.history, ref.history[:, 0]
    # BF16 entries carry 2^-9 relative rounding, which shifts the slow modes:
    # compare the first 15 sweeps only; FP16 (2^-11) follows longer
    rtol, floor, kmax = {"fp32": (1e-3, 1e-4, 40), "fp16": (2e-2, 5e-3, 20), "bf16": (5e-2, 2e-2, 15)}[precision]
    k = min(kmax, int(np.count_nonzero((h > 0) & (href[: len(h)] > floor))))
    assert k >= 5
    assert np.allclose(h[:k], href[:k], rtol=rtol, atol=0)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_dataflow_sweeps_repeat_the_launch_per_sweep_kernels_bitwise(vtm, precision):
    # one cooperative launch with per-tile neighbour waits computes the same
    # iterates as one launch per sweep: kernel 8 those of kernel 5 (four warps
    # per tile, same block arithmetic and residual order), kernel 10 those of
    # kernel 9 (one warp per tile, blocks column by column; its residual is
    # summed in two fixed-order levels of its own)
    w = wl.power_grid(256, 256, 32, 32, Zc=1.0, seed=17)
    for pair in ((5, 8), (9, 10)):
        _assert_same_iterates(vtm, w, precision, pair)


def _assert_same_iterates(vtm, w, precision, kernels):
    out = []
    for kernel in kernels:
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                        precision=precision, sweep_kernel=kernel)
        plan.set_options(history_len=64)
        x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        assert plan.stats()["sweep_kernel"] == kernel
        out.append((kernel, x, info["sweeps"], info["outer_steps"], plan.history))
    for kernel, x, sweeps, steps, hist in out[1:]:
        assert (sweeps, steps) == out[0][2:4]
        if kernel == 10:
            assert np.allclose(hist, out[0][4], rtol=1e-12, atol=0)
        else:
            assert np.array_equal(hist, out[0][4])
        assert torch.equal(x, out[0][1])


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_warp_per_tile_sweep_against_kernel_5(vtm, precision):
    # one warp per tile sums each block column's partials before reducing them
    # across lanes: the same iteration up to rounding (within the stored
    # precision of T_P), bitwise repeatable, the same FP64-verified result
    w = wl.power_grid(256, 256, 32, 32, Zc=1.0, seed=17)
    A = w.csr()
    b = torch.from_numpy(w.b[0]).cuda()
    res = {}
    for kernel in (5, 9):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                        precision=precision, sweep_kernel=kernel)
        plan.set_options(history_len=40)
        x, info = plan.solve(b, tol=1e-10)
        x2, info2 = plan.solve(b, tol=1e-10)
        assert plan.stats()["sweep_kernel"] == kernel
        assert torch.equal(x, x2) and info["sweeps"] == info2["sweeps"]
        assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10
        res[kernel] = (x.cpu().numpy(), info, plan.history)
    x5, i5, h5 = res[5]
    x9, i9, h9 = res[9]
    assert abs(i9["sweeps"] - i5["sweeps"]) <= max(4, i5["sweeps"] // 20)
    assert np.abs(x9 - x5).max() <= 1e-6 * np.abs(x5).max()  # both within cond(A) x 1e-10 of A^-1 b
    rtol = {"fp32": 1e-4, "fp16": 1e-2, "bf16": 3e-2}[precision]
    k = int(np.count_nonzero((h5 > 0) & (h9 > 0))) // 2
    assert k >= 5 and np.allclose(h9[:k], h5[:k], rtol=rtol, atol=0)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tensor_core_block_products_against_kernel_9(vtm, precision):
    # kernel 11 applies each block by warp MMAs with the waves as scaled
    # 16-bit (hi, lo) pairs: the same iteration as kernel 9 up to rounding
    # well inside the stored precision of T_P, bitwise repeatable, the same
    # FP64-verified result; 32x32 tiles (126 ports, eight block rows) and
    # 24x24 tiles (94 ports, a ragged last block)
    for shape in ((256, 32), (192, 24)):
        n, t = shape
        w = wl.power_grid(n, n, t, t, Zc=1.0, seed=21)
        A = w.csr()
        b = torch.from_numpy(w.b[0]).cuda()
        res = {}
        for kernel in (9, 11):
            plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                            precision=precision, sweep_kernel=kernel)
            plan.set_options(history_len=40)
            x, info = plan.solve(b, tol=1e-10)
            x2, info2 = plan.solve(b, tol=1e-10)
            assert plan.stats()["sweep_kernel"] == kernel
            assert torch.equal(x, x2) and info["sweeps"] == info2["sweeps"]
            assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10
            res[kernel] = (x.cpu().numpy(), info, plan.history)
        x9, i9, h9 = res[9]
        x11, i11, h11 = res[11]
        assert abs(i11["sweeps"] - i9["sweeps"]) <= max(4, i9["sweeps"] // 20)
        assert np.abs(x11 - x9).max() <= 1e-6 * np.abs(x9).max()
        # the waves' rounding (2^-22 / 2^-16 of the tile's largest) is far below
        # T_P's (2^-11 / 2^-8): the residual histories agree closely
        rtol = {"fp16": 2e-3, "bf16": 5e-3}[precision]
        k = int(np.count_nonzero((h9 > 0) & (h11 > 0))) // 2
        assert k >= 5 and np.allclose(h11[:k], h9[:k], rtol=rtol, atol=0)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tensor_core_sweep_is_invariant_to_power_of_two_scaling(vtm, precision):
    # the per-tile scale of the waves is a power of two, so solving for 2^e b
    # repeats the iteration for b exactly: with 2^24 the waves are far above
    # FP16's largest number, with 2^-12 their low halves would be subnormal
    # (the FP32 residual squares stay normal at both ends)
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=22)
    b = torch.from_numpy(w.b[0]).cuda()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                    precision=precision, sweep_kernel=11)
    x, info = plan.solve(b, tol=1e-10)
    for e in (-12, 24):
        xe, ie = plan.solve(b * 2.0 ** e, tol=1e-10)
        assert ie["sweeps"] == info["sweeps"] and ie["outer_steps"] == info["outer_steps"]
        assert torch.equal(xe, x * 2.0 ** e)


def test_tensor_core_sweep_falls_back_where_it_does_not_fit(vtm):
    # FP32 blocks, or sub-circuits of more than 128 ports: the request for
    # kernel 11 runs the direct-load kernel, and the solve is the same
    for precision, shape in (("fp32", (128, 32)), ("fp16", (192, 48))):
        n, t = shape
        w = wl.power_grid(n, n, t, t, Zc=1.0, seed=23)
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                        precision=precision, sweep_kernel=11)
        x, _ = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
        assert O.residual_norms(w.csr(), x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_warp_per_tile_sweep_with_more_tiles_than_resident_warps(vtm, precision):
    # 16384 tiles of 8x8 (32 ports): 28 tile warps per CTA, 586 CTAs, several
    # waves of CTAs per sweep; every CTA still takes its sweep number from the
    # ticket before the next launch may start
    w = wl.power_grid(1024, 1024, 8, 8, Zc=1.0, seed=19)
    A = w.csr()
    b = torch.from_numpy(w.b[0]).cuda()
    xs = {}
    for kernel in ((5, 9) if precision == "fp32" else (5, 9, 11)):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                        precision=precision, sweep_kernel=kernel)
        x, info = plan.solve(b, tol=1e-10)
        x2, info2 = plan.solve(b, tol=1e-10)
        assert plan.stats()["sweep_kernel"] == kernel and plan.stats()["nparts"] == 16384
        assert torch.equal(x, x2) and info["sweeps"] == info2["sweeps"]
        assert O.residual_norms(A, x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10
        xs[kernel] = (x.cpu().numpy(), info["sweeps"])
    for kernel in xs:
        assert abs(xs[kernel][1] - xs[5][1]) <= max(4, xs[5][1] // 20)
        assert np.abs(xs[kernel][0] - xs[5][0]).max() <= 1e-6 * np.abs(xs[5][0]).max()


@pytest.mark.parametrize("precision,kernel", [("fp32", 5), ("fp32", 6), ("fp16", 7), ("bf16", 7), ("fp16", 9),
                                              ("fp16", 11), ("bf16", 11)])
def test_overlapped_sweep_launches_compute_the_same_iterates(vtm, precision, kernel):
    # packed sweeps launched as programmatic dependents of the sweep before
    # them (the default) against plain launches: same iterates, same stop,
    # in CUDA graphs (own stream) and in plain launches
    w = wl.power_grid(192, 192, 32, 32, Zc=1.0, seed=18)
    b = torch.from_numpy(w.b[0]).cuda()
    s = torch.cuda.Stream()
    out = []
    for pdl, graphs in ((0, 0), (1, 0), (0, 1)):
        with torch.cuda.stream(s):
            plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                            sweep_kernel=kernel, pdl=pdl, graphs=graphs, stream=s)
            plan.set_options(history_len=64)
            x, info = plan.solve(b, tol=1e-10)
            x2, info2 = plan.solve(b, tol=1e-10)
        torch.cuda.synchronize()
        assert plan.stats()["sweep_kernel"] == kernel
        assert torch.equal(x, x2) and info["sweeps"] == info2["sweeps"]
        out.append((x, info["sweeps"], info["outer_steps"], plan.history))
        plan.close()
    for o in out[1:]:
        assert o[1:3] == out[0][1:3]
        assert np.array_equal(o[3], out[0][3])
        assert torch.equal(o[0], out[0][0])
    assert O.residual_norms(w.csr(), out[0][0].cpu().numpy()[None], w.b[:1]).max() <= 1e-10


def test_bad_options_are_rejected_and_the_plan_keeps_its_own(vtm):
    w = wl.power_grid(64, 64, 32, 32, Zc=1.0, seed=15)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    with pytest.raises(vtm.VTMError):
        plan.set_options(sweep_kernel=13)
    with pytest.raises(vtm.VTMError):
        plan.set_options(sweep_kernel=-1)
    for kw in ({"batch_kernel": 6}, {"wait_polls": -1}, {"flow_lag": 1}, {"batch_solve": 4},
               {"band_solve": 2}):
        with pytest.raises(vtm.VTMError):
            plan.set_options(**kw)
    for bad in (4, 5, -1):
        with pytest.raises(vtm.VTMError):
            plan.set_options(precision=bad)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert O.residual_norms(w.csr(), x.cpu().numpy()[None], w.b[:1]).max() <= 1e-10


def test_graph_path_on_a_dedicated_stream(vtm):
    # a plan with its own stream replays its sweep batches from a CUDA graph
    # and autotunes its sweep kernel; the result is the same iteration
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=13)
    A = w.csr()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, stream=s,
                        precision="fp32")
        b = torch.from_numpy(w.b[0]).cuda()
        x1, info1 = plan.solve(b, tol=1e-10)
        x2, info2 = plan.solve(b, tol=1e-10)  # graph replay
    torch.cuda.synchronize()
    assert plan.stats()["sweep_kernel"] in (1, 2, 3, 4, 5, 6, 7, 8)
    assert torch.equal(x1, x2)
    rel = O.residual_norms(A, x1.cpu().numpy()[None], w.b)
    assert rel.max() <= 1e-10


def test_double_float_sweep_history_and_stored_entries(vtm):
    # kernel 12 keeps T_P as hi + lo FP32 pairs (48 bits) and computes in
    # double-float arithmetic: its interface residual history equals the
    # oracle's full b - A x^k to 1e-9 (as the FP64 kernels do), and every
    # stored pair is the library's FP64 T_P to 2^-46 relative (and the
    # oracle's within the 1e-11 the FP64 parity tests allow)
    w = wl.grid2d(24, 24, 8, 6, Zc=0.5, seed=21)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, sweep_kernel=12)
    plan.set_options(history_len=60)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    assert plan.stats()["sweep_kernel"] == 12
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=0, max_sweeps=60)
    k = min(60, info["sweeps"])
    assert np.allclose(plan.history[:k], ref.history[:k, 0], rtol=1e-9, atol=1e-13)
    assert O.residual_norms(A, x.cpu().numpy().reshape(w.b.shape), w.b).max() <= 1e-10
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    for P in range(w.nparts):
        Tq, esize, packed = plan.reflection_stored(P)
        assert esize == 8 and packed
        T64 = plan.reflection(P)
        assert np.all(np.abs(Tq - 0.5 * (T64 + T64.T)) <= 2.0 ** -46 * np.abs(T64) + 1e-300)
        _, T_ref = O.reflection_ops(A, tear, P, 1.0 / w.Zc)
        perm = _match_ports(plan, tear, P)
        assert np.abs(Tq - T_ref[np.ix_(perm, perm)]).max() < 1e-11


@pytest.mark.parametrize("k", [1, 2, 10])
def test_double_float_iterates_after_k_sweeps(vtm, k):
    # x of sweep k of kernel 12 against the oracle's literal Eq. 11 iterate
    w = wl.power_grid(128, 128, 32, 32, Zc=1.0, seed=24)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, sweep_kernel=12,
                    max_sweeps=k)
    x, info = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-300, check=False)
    assert info["sweeps"] == k and plan.stats()["sweep_kernel"] == 12
    _, its = O.vtm_midpoint(A, w.partition, w.nparts, w.b[:1], W=1 / w.Zc, tol=0, max_sweeps=k,
                            keep_iterates=True)
    ref = its[k - 1][0]
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_tensor_core_sweep_at_extreme_magnitudes(vtm, precision, scale):
    # b scaled by 1e-30 and 1e30 (not powers of two): the per-tile scale of the
    # waves (2^(13 - E)) keeps the 16-bit (hi, lo) pairs in range, and the
    # FP64 refinement reaches the tolerance the oracle's residual confirms
    w = wl.power_grid(32 * 4, 32 * 4, 32, 32, Zc=1.0, seed=25)
    A = w.csr()
    b = w.b[0] * scale
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                    sweep_kernel=11)
    x, info = plan.solve(torch.from_numpy(b).cuda(), tol=1e-10)
    assert plan.stats()["sweep_kernel"] == 11
    xs = x.cpu().numpy()
    assert np.all(np.isfinite(xs))
    assert O.residual_norms(A, xs[None], b[None]).max() <= 1e-10
    # the same iteration as the unscaled solve up to the waves' rounding
    x1, info1 = plan.solve(torch.from_numpy(w.b[0]).cuda(), tol=1e-10)
    assert abs(info["sweeps"] - info1["sweeps"]) <= max(4, info1["sweeps"] // 20)


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_band_solve_ring_and_register_forms_give_the_same_bits(vtm, precision):
    # the FP32 band solves of the refinement (half bandwidth <= 32): factor
    # columns through a bulk-copy ring (default) or register prefetch, the same
    # arithmetic in the same order -- the same iterates and the same x, bit
    # for bit; ragged edge tiles (200 x 232 nodes in 32 x 32 tiles)
    w = wl.power_grid(200, 232, 32, 32, Zc=1.0, seed=6)
    A = w.csr()
    b = torch.from_numpy(w.b[0]).cuda()
    out = {}
    for bs in (0, 1):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                        band_solve=bs)
        assert plan.stats()["max_band"] <= 32
        x, info = plan.solve(b, tol=1e-10)
        out[bs] = (x.cpu(), info["sweeps"], info["outer_steps"])
        plan.close()
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
    assert O.residual_norms(A, out[0][0].numpy()[None, :], w.b).max() <= 1e-10
