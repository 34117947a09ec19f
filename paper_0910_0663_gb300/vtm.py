"""User-facing API over libvtm: torch tensors in, torch tensors out.

``Plan`` wraps one ``vtm_plan`` handle (wire tearing + port table), its
factorisation (``vtm_factor``) and the solves (``vtm_solve`` /
``vtm_adjoint``).  PyTorch supplies device memory and the CUDA stream; all
arithmetic runs in libvtm's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _vtm as C
from ._vtm import VTMError  # noqa: F401  (raised on every failing status)


def _dev(a, dtype, device):
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    return a.to(device=device, dtype=dtype).contiguous()


class Plan:
    """A torn circuit ready for VTM solves.

    indptr/indices/data: CSR of A (int64 / int32 / float64); partition: node
    -> sub-circuit (int32); Zc: characteristic impedance of the virtual lines
    (W = 1/Zc).  ``precision`` selects the arithmetic of the sweeps:
    "fp64", or "fp32"/"bf16"/"fp16" inside FP64 iterative refinement.
    """

    def __init__(self, indptr, indices, data, partition, nparts, Zc=1.0, precision="fp64",
                 device="cuda", stream=None, max_sweeps=0, check_every=0, inner_tol=0.0,
                 max_outer=0, sweep_kernel=0, method="vtm", batch=0, l2_persist=0, graphs=0,
                 batch_solve=0, pdl=0, batch_kernel=0, wait_polls=0, flow_lag=0, band_solve=0, factor=True):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n = int(len(indptr) - 1)
        self.nparts = int(nparts)
        self._opts = dict(precision=precision, max_sweeps=max_sweeps, check_every=check_every,
                          inner_tol=inner_tol, max_outer=max_outer, sweep_kernel=sweep_kernel,
                          method=method, batch=batch, l2_persist=l2_persist, graphs=graphs,
                          batch_solve=batch_solve, pdl=pdl, batch_kernel=batch_kernel,
                          wait_polls=wait_polls, flow_lag=flow_lag, band_solve=band_solve)
        self._history = None
        rp = _dev(indptr, torch.int64, self.device)
        ci = _dev(indices, torch.int32, self.device)
        va = _dev(data, torch.float64, self.device)
        pa = _dev(partition, torch.int32, self.device)
        self.handle = C.vtm_plan(self.n, rp, ci, va, pa, self.nparts, float(Zc),
                                 C.make_opts(**self._opts), self.stream.cuda_stream)
        if factor:
            self.factor()

    # -- set-up ------------------------------------------------------------
    def factor(self):
        C.vtm_factor(self.handle)

    def set_values(self, data):
        C.vtm_set_values(self.handle, _dev(data, torch.float64, self.device))

    def set_admittance(self, kind, alpha=1.0, radius=2, W=None, factor=True):
        """Line admittances (Sec. VIII): "alpha" (alpha I), "diag" (2 g_e),
        "wob" (alpha 2 g_e), "sca" (partial input admittance over `radius`
        branches) or "line" (W per port, equal at both ends of a line)."""
        if W is not None:
            W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
        C.vtm_set_admittance(self.handle, kind, alpha, radius, W)
        if factor:
            self.factor()

    def admittance(self) -> np.ndarray:
        return C.vtm_get_admittance(self.handle)

    def set_options(self, history_len=0, **kw):
        opts = {**self._opts, **kw}
        history = np.zeros(history_len, np.float64) if history_len else None
        C.vtm_set_opts(self.handle, C.make_opts(**opts, history=history))
        self._opts, self._history = opts, history

    @property
    def history(self):
        return None if self._history is None else self._history.copy()

    def stats(self) -> dict:
        return C.vtm_plan_get_stats(self.handle).as_dict()

    def ports(self):
        return C.vtm_get_ports(self.handle)

    def reflection(self, part) -> np.ndarray:
        return C.vtm_get_reflection(self.handle, part)

    def reflection_stored(self, part):
        """(T, element bytes, packed): T_P as the sweeps of the plan's
        precision read it (the rounded copy), in FP64."""
        return C.vtm_get_reflection_stored(self.handle, part)

    # -- solves --------------------------------------------------------------
    def _run(self, fn, b, tol, check):
        b = b if torch.is_tensor(b) else torch.from_numpy(np.ascontiguousarray(b))
        squeeze = b.dim() == 1
        b2 = b.reshape(1, -1) if squeeze else b
        if b2.is_cuda:
            b2 = b2.to(torch.float64).contiguous()
            x = torch.empty_like(b2)
        else:
            b2 = b2.to(torch.float64).contiguous()
            x = torch.empty_like(b2)
        st, info = fn(self.handle, b2, x, b2.shape[0], tol, check=check)
        x = x.reshape(-1) if squeeze else x
        return x, info.as_dict(), st

    def solve(self, b, tol=1e-10, check=True):
        """x with A x = b.  b: (n,) or (nrhs, n) tensor (CPU or CUDA)."""
        x, info, _ = self._run(C.vtm_solve, b, tol, check)
        return x, info

    def adjoint(self, g, tol=1e-10, check=True):
        x, info, _ = self._run(C.vtm_adjoint, g, tol, check)
        return x, info

    def march(self, cdiag, p, x0=None, tol=1e-10, check=True):
        """Backward-Euler transient: A x_k = p_k + cdiag * x_{k-1}, k = 1..nsteps,
        each step warm-started from x_{k-1}.  p: (nsteps, n); returns X
        (nsteps, n) and the summed info."""
        dev = self.device
        cd = _dev(cdiag, torch.float64, dev)
        pp = _dev(p, torch.float64, dev).reshape(-1, self.n).contiguous()
        x0d = None if x0 is None else _dev(x0, torch.float64, dev)
        X = torch.empty_like(pp)
        st, info = C.vtm_march(self.handle, cd, pp, x0d, X, pp.shape[0], tol, check=check)
        return X, info.as_dict()

    def residual(self, x, b):
        x = x.reshape(-1, self.n).to(torch.float64).contiguous()
        b = b.reshape(-1, self.n).to(torch.float64).contiguous()
        return C.vtm_residual_norm(self.handle, x, b, x.shape[0])

    def close(self):
        if getattr(self, "handle", None) is not None:
            C.vtm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_workload(w, precision="fp64", device="cuda", **kw) -> Plan:
    """Plan and factor a ``workloads.Workload``."""
    return Plan(w.indptr, w.indices, w.data, w.partition, w.nparts, Zc=w.Zc, precision=precision,
                device=device, **kw)


class Network:
    """A resistor network: branches (ei, ej) and the CSR pattern of its nodal
    matrix, with a VTM plan over a node partition.  ``solve(g, ground, b)``
    is differentiable in g, ground and b (``VTMSolve``)."""

    def __init__(self, n, edges, indptr, indices, partition, nparts, Zc=1.0, precision="fp64",
                 device="cuda", g0=None, ground0=None, **plan_kw):
        self.device = torch.device(device)
        self.n = int(n)
        self.stream = torch.cuda.current_stream(self.device)
        self.rowptr = _dev(indptr, torch.int64, self.device)
        self.colidx = _dev(indices, torch.int32, self.device)
        self.ei = _dev(np.asarray(edges)[:, 0], torch.int64, self.device)
        self.ej = _dev(np.asarray(edges)[:, 1], torch.int64, self.device)
        self.nedges = int(self.ei.numel())
        self.netmap = C.vtm_netmap_create(self.n, self.rowptr, self.colidx, self.nedges, self.ei,
                                          self.ej, self.stream.cuda_stream)
        g0 = torch.ones(self.nedges, dtype=torch.float64, device=self.device) if g0 is None else \
            _dev(g0, torch.float64, self.device)
        gr0 = None if ground0 is None else _dev(ground0, torch.float64, self.device)
        vals = self.values(g0, gr0)
        self.plan = Plan(self.rowptr, self.colidx, vals, partition, nparts, Zc=Zc,
                         precision=precision, device=self.device, stream=self.stream,
                         factor=False, **plan_kw)
        self._key = None
        self._set(g0, gr0, vals)

    def values(self, g, ground=None):
        vals = torch.empty(int(self.colidx.numel()), dtype=torch.float64, device=self.device)
        C.vtm_netmap_values(self.netmap, self.rowptr, g.contiguous(),
                            None if ground is None else ground.contiguous(), vals)
        return vals

    def _set(self, g, ground, vals=None):
        key = (g.data_ptr(), g._version, None if ground is None else (ground.data_ptr(), ground._version))
        if key == self._key:
            return
        if vals is None:
            vals = self.values(g, ground)
        self.plan.set_values(vals)
        self.plan.factor()
        self._key = key

    def gradient(self, lam, x):
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        gg = torch.empty(self.nedges, dtype=torch.float64, device=self.device)
        gr = torch.empty(self.n, dtype=torch.float64, device=self.device)
        C.vtm_netmap_gradient(self.netmap, lam.contiguous(), x.contiguous(), nrhs, gg, gr)
        return gg, gr

    def solve(self, g, ground, b, tol=1e-10):
        return VTMSolve.apply(g, ground, b, self, tol)

    def close(self):
        if getattr(self, "netmap", None) is not None:
            C.vtm_netmap_destroy(self.netmap)
            self.netmap = None
        self.plan.close()


class VTMSolve(torch.autograd.Function):
    """x = A(g, ground)^-1 b by VTM; backward by one adjoint VTM solve:
    dL/db = lam, dL/dg_e = -(lam_i - lam_j)(x_i - x_j), dL/dground = -lam x,
    with A^T lam = dL/dx."""

    @staticmethod
    def forward(ctx, g, ground, b, net, tol):
        g = g.detach().to(torch.float64).contiguous()
        gr = None if ground is None else ground.detach().to(torch.float64).contiguous()
        net._set(g, gr)
        x, info = net.plan.solve(b.detach().to(torch.float64).contiguous(), tol=tol)
        ctx.net, ctx.tol = net, tol
        ctx.has_ground = ground is not None
        ctx.save_for_backward(x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        net = ctx.net
        lam, _ = net.plan.adjoint(grad_x.to(torch.float64).contiguous(), tol=ctx.tol)
        gg, gr = net.gradient(lam, x)
        return gg, (gr if ctx.has_ground else None), lam, None, None
