"""The allocation-free residual entry point.

vtm_residual_norm_noalloc serves callers that cannot allocate device memory
when they need a residual (their pool owns the device, or their loop must
not call cudaMalloc).  It must give the same numbers as the plan-based
vtm_residual_norm, call after call, since its scratch is a static device
array that keeps the previous call's contents.  This file is collected last
so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_0910_0663_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0910_0663_gb300 import build
    build.build()
    from paper_0910_0663_gb300 import _vtm, vtm
    return _vtm, vtm


def test_noalloc_residual_matches_plan_residual_twice(mods):
    C, vtm = mods
    w = wl.grid2d(48, 40, 12, 10, seed=31, nrhs=3, ground=0.01)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0)
    b = torch.from_numpy(w.b).cuda()
    x, _ = plan.solve(b, tol=1e-6)  # a residual well above rounding
    x = x.contiguous()
    ref = plan.residual(x, b)  # existing entry point (vtm_residual_norm)
    rp = torch.from_numpy(w.indptr).cuda()
    ci = torch.from_numpy(w.indices).cuda()
    va = torch.from_numpy(w.data).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the second call sees the first call's leftovers
        got = C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x, b, w.nrhs, stream)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert np.all(ref > 1e-9) and np.all(ref < 1e-5)
    # a different x gives a different answer (the call really computes)
    x2 = x.clone()
    x2[1, 7] += 1.0
    got2 = C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x2, b, w.nrhs, stream)
    ref2 = plan.residual(x2, b)
    np.testing.assert_allclose(got2, ref2, rtol=1e-12)
    assert got2[1] > 10 * got[1] and got2[0] == got[0]
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(mods):
    C, _ = mods
    w = wl.grid2d(8, 8, 4, 4, seed=1)
    rp = torch.from_numpy(w.indptr).cuda()
    ci = torch.from_numpy(w.indices).cuda()
    va = torch.from_numpy(w.data).cuda()
    x = torch.zeros((65, w.n), dtype=torch.float64, device="cuda")
    with pytest.raises(C.VTMError) as e:
        C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x, x, 65)
    assert e.value.status == C.VTM_EINVAL
    with pytest.raises(C.VTMError) as e:  # host vectors are refused, not staged
        C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x.cpu(), x.cpu(), 1)
    assert e.value.status == C.VTM_EINVAL


def test_noalloc_at_its_limits_matches_plan_residual(mods):
    # more nodes than 1216 blocks x 256 threads (the grid is capped and every
    # partial slot is used) and 64 columns (the last pair of sums)
    C, vtm = mods
    w = wl.grid2d(600, 600, 60, 60, seed=32, ground=0.01)
    plan = vtm.Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=1.0, factor=False)
    g = torch.Generator().manual_seed(5)
    x = torch.rand((64, w.n), generator=g, dtype=torch.float64).cuda()
    b = torch.rand((64, w.n), generator=g, dtype=torch.float64).cuda()
    ref = plan.residual(x, b)
    rp = torch.from_numpy(w.indptr).cuda()
    ci = torch.from_numpy(w.indices).cuda()
    va = torch.from_numpy(w.data).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    assert w.n > 1216 * 256
    for _ in range(2):
        got = C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x, b, 64, stream)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    plan.close()


def test_noalloc_refuses_memory_of_another_device(mods):
    # tensors on cuda:1 while cuda:0 is current: refused before any launch
    C, _ = mods
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    w = wl.grid2d(8, 8, 4, 4, seed=1)
    d1 = torch.device("cuda", 1)
    rp = torch.from_numpy(w.indptr).to(d1)
    ci = torch.from_numpy(w.indices).to(d1)
    va = torch.from_numpy(w.data).to(d1)
    x = torch.zeros(w.n, dtype=torch.float64, device=d1)
    with torch.cuda.device(0):
        with pytest.raises(C.VTMError) as e:
            C.vtm_residual_norm_noalloc(w.n, rp, ci, va, x, x, 1)
    assert e.value.status == C.VTM_EINVAL
