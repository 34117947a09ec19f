"""Many right-hand sides in one batched VTM iteration (RC thermal grid,
backward-Euler time-step vectors), against the oracle's multi-RHS VTM.

The batched iteration stops when every column meets the tolerance, exactly
like the oracle's multi-RHS run, so the sweep counts and the iterates agree.
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


def _thermal_small(nrhs, seed=1):
    return wl.thermal3d(8, 24, 24, 12, nrhs=nrhs, seed=seed, min_box=100, max_box=1200)


def test_batched_fp64_matches_oracle(vtm):
    w = _thermal_small(8)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b, W=1 / w.Zc, tol=1e-10)
    assert ref.converged
    xs = x.cpu().numpy()
    if info["sweeps"] == ref.sweeps:
        assert np.abs(xs - ref.x).max() <= 1e-11 * np.abs(ref.x).max()
    else:
        assert abs(info["sweeps"] - ref.sweeps) == 1
    assert O.residual_norms(A, xs, w.b).max() <= 1e-10


def test_batched_equals_column_by_column_at_equal_sweeps(vtm):
    # with the batched count forced on every column, the same iterate results
    w = _thermal_small(4, seed=2)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc)
    xb, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    K = info["sweeps"]
    plan1 = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, batch=1,
                     max_sweeps=K)
    for r in range(4):
        xr, inf = plan1.solve(torch.from_numpy(w.b[r]).cuda(), tol=1e-300, check=False)
        assert inf["sweeps"] == K
        assert torch.allclose(xr, xb[r], rtol=1e-12, atol=1e-14 * float(xb[r].abs().max()))


@pytest.mark.parametrize("precision,nrhs", [("bf16", 16), ("fp32", 5), ("bf16", 6), ("fp16", 16)])
def test_batched_low_precision_reaches_tolerance(vtm, precision, nrhs):
    w = _thermal_small(nrhs, seed=3)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc,
                    precision=precision)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    rel = O.residual_norms(A, x.cpu().numpy(), w.b)
    assert rel.max() <= 1e-10
    assert info["outer_steps"] >= 2


def test_thermal_full_size_64_rhs_bf16(vtm):
    # the 128x128x32 grid in 400 boxes with 64 right-hand sides, as timed
    w = wl.c3_thermal(nrhs=64)
    A = w.csr()
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision="bf16")
    st = plan.stats()
    assert st["nparts"] == 400
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    rel = O.residual_norms(A, x.cpu().numpy(), w.b)
    assert rel.max() <= 1e-10
    # sampled reflection matrices of three boxes against (W - S)(W + S)^-1
    tear = O.tear_midpoint(A, w.partition, w.nparts)
    node, remote, part, _ = plan.ports()
    for P in (0, 137, 399):
        T_lib = plan.reflection(P)
        _, T_ref = O.reflection_ops(A, tear, P, 1.0 / w.Zc)
        sel = np.flatnonzero(part == P)
        keys = {k: i for i, k in enumerate(zip(tear.port_node[tear.tile_ports[P]].tolist(),
                                                 tear.port_remote[tear.tile_ports[P]].tolist()))}
        perm = np.array([keys[k] for k in zip(node[sel].tolist(), remote[sel].tolist())])
        assert np.abs(T_lib - T_ref[np.ix_(perm, perm)]).max() < 1e-10


def test_batched_graph_path_on_a_dedicated_stream(vtm):
    # own stream: persistent batched sweeps replayed from a CUDA graph, the
    # tensor-core / CUDA-core choice autotuned; a second solve repeats the first
    w = _thermal_small(16, seed=4)
    A = w.csr()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, stream=s,
                        precision="bf16")
        b = torch.from_numpy(w.b).cuda()
        x1, _ = plan.solve(b, tol=1e-10)
        x2, _ = plan.solve(b, tol=1e-10)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)
    assert O.residual_norms(A, x1.cpu().numpy(), w.b).max() <= 1e-10


@pytest.mark.parametrize("precision,batch_kernel", [("fp64", 1), ("fp64", 3), ("bf16", 1), ("bf16", 2),
                                                    ("bf16", 3), ("bf16", 4), ("bf16", 5)])
def test_every_batched_variant_against_the_oracle(vtm, precision, batch_kernel):
    # each variant forced (CUDA cores or BF16 tensor-core warp MMAs; persistent
    # grid or one work item per CTA): the result is FP64-verified and the
    # first inner solve of column 0 follows the oracle's VTM iteration on b --
    # sweep by sweep to 1e-9 in FP64; within the storage rounding of T_P (and,
    # on the tensor cores, of the waves as BF16 operands) in BF16
    w = _thermal_small(16, seed=5)
    A = w.csr()
    # BF16: an inner tolerance of 1e-4 keeps the first inner solve going past
    # the default 3e-3, so that several sweeps lie above BF16's rounding floor
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                    batch_kernel=batch_kernel, inner_tol=1e-4 if precision == "bf16" else 0.0)
    plan.set_options(history_len=30)
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    assert plan.stats()["batch_kernel"] == batch_kernel
    assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10
    ref = O.vtm_midpoint(A, w.partition, w.nparts, w.b[:1], W=1 / w.Zc, tol=0, max_sweeps=30)
    h, href = plan.history, ref.history[:, 0]
    if precision == "fp64":
        k = min(30, info["sweeps"])
        assert np.allclose(h[:k], href[:k], rtol=1e-9, atol=1e-13)
    else:
        k = min(12, int(np.count_nonzero((h > 0) & (href[: len(h)] > 1e-3))))
        assert k >= 3
        assert np.allclose(h[:k], href[:k], rtol=5e-2, atol=0)


@pytest.mark.parametrize("nrhs", [64, 5])
def test_tcgen05_batched_sweep_on_the_full_thermal_grid(vtm, nrhs):
    # the tcgen05 variant on the 128x128x32 grid in 400 boxes (ports per box
    # 263-2459: up to 20 M tiles of 128 and 39 input chunks of 64, items of
    # four M tiles), 64 columns and a ragged 5 (the B operand's other columns
    # are zero): FP64-verified result, and its first inner solve follows the
    # CUDA-core BF16 variant's residual history within the waves' BF16 rounding
    w = wl.c3_thermal(nrhs=nrhs)
    A = w.csr()
    b = torch.from_numpy(w.b).cuda()
    hist = {}
    for bk in (5, 1):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision="bf16",
                        batch_kernel=bk)
        plan.set_options(history_len=12)
        x, info = plan.solve(b, tol=1e-10)
        assert plan.stats()["batch_kernel"] == bk
        assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10
        hist[bk] = plan.history
        plan.close()
    k = int(np.count_nonzero((hist[5] > 0) & (hist[1] > 0)))
    assert k >= 3 and np.allclose(hist[5][:k], hist[1][:k], rtol=2e-2, atol=0)


@pytest.mark.parametrize("nrhs", [5, 64, 70])
def test_batched_band_solve_variants_agree(vtm, nrhs):
    # the FP32 band solves of the batched iteration -- whole column block in
    # shared memory (1), row window (2), blocked with the diagonal blocks of
    # the factors inverted ahead (3) -- are the same K_P^-1 up to FP32
    # rounding: each result is FP64-verified and the first inner solves follow
    # one another's residual history (70 columns: a call of 64 and one of 6)
    w = _thermal_small(nrhs, seed=6)
    A = w.csr()
    b = torch.from_numpy(w.b).cuda()
    hist = {}
    for mode in (1, 2, 3):
        plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision="fp32",
                        batch_solve=mode)
        plan.set_options(history_len=20)
        x, info = plan.solve(b, tol=1e-10)
        assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10
        hist[mode] = plan.history
        plan.close()
    k = int(np.count_nonzero((hist[1] > 1e-5) & (hist[3] > 1e-5)))
    assert k >= 5
    for mode in (2, 3):
        assert np.allclose(hist[mode][:k], hist[1][:k], rtol=1e-3, atol=0)


def test_blocked_band_solve_needs_a_band_of_at_most_128(vtm):
    # 280 x 280 plane in four 140 x 140 quadrants: half bandwidths above 128,
    # so the blocked solve refuses (VTM_EINVAL) and the default takes the row
    # window
    w = wl.thermal3d(1, 280, 280, 4, nrhs=3, seed=7, min_box=1, max_box=280 * 280)
    iy, ix = np.divmod(np.arange(w.n), 280)
    part = ((iy >= 140).astype(np.int32) * 2 + (ix >= 140)).astype(np.int32)
    b = torch.from_numpy(w.b).cuda()
    plan = vtm.Plan(w.indptr, w.indices, w.data, part, 4, Zc=w.Zc, precision="fp32")
    assert plan.stats()["max_band"] > 128
    x, _ = plan.solve(b, tol=1e-10)
    assert O.residual_norms(w.csr(), x.cpu().numpy(), w.b).max() <= 1e-10
    plan.set_options(batch_solve=3)
    with pytest.raises(vtm.VTMError, match="half bandwidths up to 128"):
        plan.solve(b, tol=1e-10)
    plan.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batched_columns_of_very_different_magnitudes(vtm, precision):
    # the low-precision batched residuals are double-float on columns scaled
    # by 2^-f (f from max |b_c|): columns of size 1e-30, 1 and 1e30 each reach
    # the tolerance by the oracle's FP64 residual
    w = _thermal_small(3, seed=8)
    A = w.csr()
    b = w.b * np.array([1e-30, 1.0, 1e30])[:, None]
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision)
    x, info = plan.solve(torch.from_numpy(b).cuda(), tol=1e-10)
    rel = O.residual_norms(A, x.cpu().numpy(), b)
    assert rel.max() <= 1e-10, rel
    assert info["relres"] <= 1e-10


def test_batched_low_precision_without_ports(vtm):
    # one sub-circuit: no torn lines, the batched step is the FP32 band solve
    # alone, refined in FP64
    w = _thermal_small(3, seed=9)
    A = w.csr()
    part = np.zeros(w.n, np.int32)
    plan = vtm.Plan(w.indptr, w.indices, w.data, part, 1, Zc=w.Zc, precision="fp32")
    assert plan.stats()["nports"] == 0
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10


def test_batched_matrix_beyond_double_float_range(vtm):
    # nonzeros near 2^101 (outside 2^-100 .. 2^100): the residuals stay FP64;
    # the solve reaches the tolerance all the same
    w = _thermal_small(4, seed=10)
    scale = 2.0 ** 101
    A = w.csr() * scale
    plan = vtm.Plan(w.indptr, w.indices, w.data * scale, w.partition, w.nparts, Zc=w.Zc / scale,
                    precision="fp32")
    x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
    assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batched_low_precision_with_lu_factors(vtm, precision):
    # an unsymmetric A whose asymmetry stays inside the boxes (each interior
    # branch of a box gets a one-sided extra conductance, the torn branches
    # stay symmetric): LU factors, so the blocked band solve's forward and
    # backward matrices come from different factors.  FP64-verified result,
    # and the same sweep count as the row-window solve
    w = _thermal_small(6, seed=11)
    A = w.csr().tolil()
    rng = np.random.default_rng(11)
    part = np.asarray(w.partition)
    e = np.asarray(w.edges)
    inside = e[part[e[:, 0]] == part[e[:, 1]]]
    pick = inside[rng.random(len(inside)) < 0.3]
    for i, j in pick:
        A[i, j] = A[i, j] - 0.2 * abs(A[i, j])
    A = A.tocsr()
    A.sort_indices()
    xs = {}
    for mode in (3, 2):
        plan = vtm.Plan(A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, w.partition, w.nparts,
                        Zc=w.Zc, precision=precision, batch_solve=mode)
        assert plan.stats()["symmetric"] == 0 and plan.stats()["nlagged"] == 0
        x, info = plan.solve(torch.from_numpy(w.b).cuda(), tol=1e-10)
        assert O.residual_norms(A, x.cpu().numpy(), w.b).max() <= 1e-10
        xs[mode] = (x.cpu().numpy(), info["sweeps"])
        plan.close()
    assert abs(xs[3][1] - xs[2][1]) <= 1  # the same iteration, up to FP32 rounding of the band solves
