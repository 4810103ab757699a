"""PyTorch-facing wrapper of the C ABI: device memory and streams come from
PyTorch; every step of the path runs in libgrf.so's CUDA kernels.

    g = GRF((4096, 4096), (1.0, 1.0), family="matern", sigma=1.0, ell=0.05, nu=2.5, max_batch=64)
    f = g.sample(seed=0, batch=64)            # (64, 4096, 4096) float32 on the current device

The autograd entry point ``grf_fields(theta, g, seed, batch)`` returns fields
whose backward gives d(loss)/d(sigma, ell, nu) through the hand-written
adjoint kernel (grf_backward).
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import _lib as L

_FAMILIES = {"matern": L.GRF_MATERN, "gaussian": L.GRF_GAUSSIAN, "paper_poly": L.GRF_PAPER_POLY}


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class GRF:
    """A plan: one grid shape, box, spectral density, algorithm and precision."""

    def __init__(self, shape: Sequence[int], lengths: Sequence[float] | None = None, family: str = "matern",
                 sigma: float = 1.0, ell: float = 0.1, nu: float = 1.5, m: float = 1.0, k: int = 1, l: int = 1,
                 n: int = 1, normalize_discrete: bool = False, alg: int = 2, precision: str = "fp32",
                 max_batch: int = 1, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("GRF needs a CUDA device; there is no CPU fallback")
        self.shape = tuple(int(s) for s in shape)
        self.d = len(self.shape)
        self.lengths = tuple(float(x) for x in (lengths if lengths is not None else [1.0] * self.d))
        self.family = family
        self.alg = int(alg)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.max_batch = int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        self._params = dict(sigma=sigma, ell=ell, nu=nu, m=m, k=k, l=l, n=n, normalize_discrete=int(normalize_discrete))
        with torch.cuda.device(self.device):
            self.handle = L.grf_plan_create(self.d, self.shape, self.lengths, self._spec(), self.alg,
                                            L.GRF_FP32 if precision == "fp32" else L.GRF_FP64, self.max_batch)

    def _spec(self):
        p = self._params
        return L.make_spectrum(_FAMILIES[self.family], p["sigma"], p["ell"], p["nu"], p["m"], p["k"], p["l"],
                               p["n"], p["normalize_discrete"])

    @property
    def params(self):
        return dict(self._params)

    def set_params(self, **kw):
        """New (sigma, ell, nu, ...) for the same family: rebuilds the tables on the current stream."""
        self._params.update(kw)
        with torch.cuda.device(self.device):
            L.grf_plan_set_spectrum(self.handle, self._spec(), _stream_ptr(self.device))

    def empty(self, batch: int) -> torch.Tensor:
        return torch.empty((batch,) + self.shape, dtype=self.dtype, device=self.device)

    def tune(self) -> dict:
        """Time the candidate schedules (radix, tiles, pipelining) and keep the best.
        A schedule this plan took from the tuning cache is kept as it is
        (GRF_TUNE_FORCE=1 times again)."""
        with torch.cuda.device(self.device):
            L.grf_plan_tune(self.handle, _stream_ptr(self.device))
        return self.schedule

    @property
    def schedule(self) -> dict:
        return L.grf_plan_schedule(self.handle)

    def sample(self, seed: int = 0, batch: int = 1, out: torch.Tensor | None = None) -> torch.Tensor:
        """batch fields; field b uses Philox key seed + b."""
        if out is None:
            out = self.empty(batch)
        assert out.is_contiguous() and out.dtype == self.dtype and out.device == self.device
        assert out.numel() == batch * self.points
        with torch.cuda.device(self.device):
            L.grf_sample(self.handle, int(seed), int(batch), out.data_ptr(), _stream_ptr(self.device))
        return out

    def sample_host(self, seed: int = 0, batch: int = 1, out: torch.Tensor | None = None) -> torch.Tensor:
        """The same fields delivered to (pinned) host memory, copies overlapped with compute."""
        if out is None:
            out = torch.empty((batch,) + self.shape, dtype=self.dtype, pin_memory=True)
        assert out.is_contiguous() and out.dtype == self.dtype and out.device.type == "cpu"
        with torch.cuda.device(self.device):
            L.grf_sample_host(self.handle, int(seed), int(batch), out.data_ptr(), _stream_ptr(self.device))
        return out

    def backward(self, seed: int, grad_out: torch.Tensor) -> torch.Tensor:
        """(batch, 3) float64 per-field d(loss)/d(sigma, ell, nu) for upstream gradient grad_out."""
        grad_out = grad_out.contiguous().to(self.dtype)
        batch = grad_out.shape[0]
        gp = torch.empty((batch, 3), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            L.grf_backward(self.handle, int(seed), batch, grad_out.data_ptr(), gp.data_ptr(), _stream_ptr(self.device))
        return gp

    def cov_origin(self, seed: int, count: int, sums: torch.Tensor | None = None) -> torch.Tensor:
        """The estimator of the paper's statistical tests: sums[j] (+)= sum_b f_b(0) f_b(x_j)
        over the fields seed .. seed + count - 1 (float64, on the device, shaped like a
        field).  Cov(x_0, x_j) = sums[j] / count.  FP32 plans."""
        if sums is None:
            sums = torch.zeros(self.shape, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            L.grf_cov_origin(self.handle, int(seed), int(count), sums.data_ptr(), _stream_ptr(self.device))
        return sums

    def rfft(self, x: torch.Tensor) -> torch.Tensor:
        """Forward real-to-complex DFT of real fields onto the half spectrum (complex64)."""
        x = x.contiguous().to(self.dtype)
        batch = x.shape[0]
        hs = self.shape[:-1] + (self.shape[-1] // 2 + 1,)
        out = torch.empty((batch,) + hs, dtype=torch.complex64, device=self.device)
        with torch.cuda.device(self.device):
            L.grf_rfft_forward(self.handle, batch, x.data_ptr(), out.data_ptr(), _stream_ptr(self.device))
        return out

    @property
    def points(self) -> int:
        return L.grf_plan_query(self.handle, 0)

    def close(self):
        if getattr(self, "handle", None) is not None:
            L.grf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GRFBoundary:
    """Fields with Neumann or Dirichlet boundary conditions on [0, L_1] x ... x [0, L_d]
    (the cosine / sine transform variant of the method): `intervals` N_i per axis,
    fields of shape (N_1 + 1, ..., N_d + 1), FP32."""

    def __init__(self, intervals: Sequence[int], lengths: Sequence[float] | None = None, bc: str = "neumann",
                 family: str = "matern", sigma: float = 1.0, ell: float = 0.1, nu: float = 1.5, m: float = 1.0,
                 k: int = 1, l: int = 1, n: int = 1, max_batch: int = 1, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("GRFBoundary needs a CUDA device; there is no CPU fallback")
        self.intervals = tuple(int(s) for s in intervals)
        self.d = len(self.intervals)
        self.shape = tuple(s + 1 for s in self.intervals)
        self.lengths = tuple(float(x) for x in (lengths if lengths is not None else [1.0] * self.d))
        self.bc = {"neumann": L.GRF_BC_NEUMANN, "dirichlet": L.GRF_BC_DIRICHLET}[bc]
        self.max_batch = int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        spec = L.make_spectrum(_FAMILIES[family], sigma, ell, nu, m, k, l, n, 0)
        with torch.cuda.device(self.device):
            self.handle = L.grf_bc_plan_create(self.d, self.intervals, self.lengths, spec, self.bc, self.max_batch)

    def sample(self, seed: int = 0, batch: int = 1, out: torch.Tensor | None = None) -> torch.Tensor:
        """batch fields of shape (N_1 + 1, ..., N_d + 1); field b uses Philox key seed + b."""
        if out is None:
            out = torch.empty((batch,) + self.shape, dtype=torch.float32, device=self.device)
        assert out.is_contiguous() and out.dtype == torch.float32 and out.device == self.device
        assert out.numel() == batch * self.points
        with torch.cuda.device(self.device):
            L.grf_sample(self.handle, int(seed), int(batch), out.data_ptr(), _stream_ptr(self.device))
        return out

    def sample_host(self, seed: int = 0, batch: int = 1, out: torch.Tensor | None = None) -> torch.Tensor:
        """The same fields delivered to (pinned) host memory."""
        if out is None:
            out = torch.empty((batch,) + self.shape, dtype=torch.float32, pin_memory=True)
        assert out.is_contiguous() and out.dtype == torch.float32 and out.device.type == "cpu"
        with torch.cuda.device(self.device):
            L.grf_sample_host(self.handle, int(seed), int(batch), out.data_ptr(), _stream_ptr(self.device))
        return out

    def set_params(self, family: str, sigma: float = 1.0, ell: float = 0.1, nu: float = 1.5, m: float = 1.0,
                   k: int = 1, l: int = 1, n: int = 1):
        """New spectral parameters of the same family: rebuilds c_K on the current stream."""
        spec = L.make_spectrum(_FAMILIES[family], sigma, ell, nu, m, k, l, n, 0)
        with torch.cuda.device(self.device):
            L.grf_plan_set_spectrum(self.handle, spec, _stream_ptr(self.device))

    def cov_origin(self, seed: int, count: int, sums: torch.Tensor | None = None) -> torch.Tensor:
        """sums[j] (+)= sum_b f_b(corner) f_b(x_j) over the fields seed .. seed + count - 1
        (float64, shaped like a field); Cov(x_0, x_j) = sums[j] / count."""
        if sums is None:
            sums = torch.zeros(self.shape, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            L.grf_cov_origin(self.handle, int(seed), int(count), sums.data_ptr(), _stream_ptr(self.device))
        return sums

    @property
    def points(self) -> int:
        return L.grf_plan_query(self.handle, 0)

    def close(self):
        if getattr(self, "handle", None) is not None:
            L.grf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _GRFFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, plan: GRF, seed: int, batch: int):
        t = theta.detach().double().cpu().tolist()
        plan.set_params(sigma=t[0], ell=t[1], nu=t[2])
        out = plan.sample(seed, batch)
        ctx.plan, ctx.seed, ctx.theta, ctx.tdev = plan, seed, t, theta.device
        return out

    @staticmethod
    def backward(ctx, grad):
        plan = ctx.plan
        cur = plan.params
        if [cur["sigma"], cur["ell"], cur["nu"]] != ctx.theta:
            plan.set_params(sigma=ctx.theta[0], ell=ctx.theta[1], nu=ctx.theta[2])
        gp = plan.backward(ctx.seed, grad)
        return gp.sum(dim=0).to(device=ctx.tdev, dtype=torch.float64), None, None, None


def grf_fields(theta: torch.Tensor, plan: GRF, seed: int, batch: int) -> torch.Tensor:
    """Differentiable sampling: theta = (sigma, ell, nu) (float64 tensor); returns
    (batch, *shape) fields of `plan` with those parameters.  The backward pass
    runs the adjoint kernel (noise regenerated from the seed, never stored)."""
    return _GRFFields.apply(theta, plan, seed, batch)


class GRFBatch:
    """Uneven batch: fields of different shapes/dimensions/parameters sampled together,
    by per-shape launches in one graph (mode "shapes", the default) or by one
    persistent kernel (mode "persistent")."""

    def __init__(self, shapes, lengths, specs, device=None, mode: str = "shapes"):
        self.shapes = [tuple(int(s) for s in shp) for shp in shapes]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        spec_objs = [L.make_spectrum(_FAMILIES[s.get("family", "matern")], s.get("sigma", 1.0), s.get("ell", 0.1),
                                     s.get("nu", 1.5)) for s in specs]
        with torch.cuda.device(self.device):
            self.handle = L.grf_batch_plan_create([len(s) for s in self.shapes], self.shapes, lengths, spec_objs)
        self.set_mode(mode)

    def set_mode(self, mode: str):
        L.grf_batch_set_mode(self.handle, {"shapes": 0, "persistent": 1}[mode])

    def empty(self):
        return [torch.empty(shp, dtype=torch.float32, device=self.device) for shp in self.shapes]

    def sample(self, seed: int, outs=None, graph: bool = False):
        if outs is None:
            outs = self.empty()
        ptrs = [o.data_ptr() for o in outs]
        with torch.cuda.device(self.device):
            fn = L.grf_batch_graph_launch if graph else L.grf_batch_sample
            fn(self.handle, int(seed), ptrs, _stream_ptr(self.device))
        return outs

    def status(self) -> int:
        with torch.cuda.device(self.device):
            return L.grf_status_word(self.handle, _stream_ptr(self.device))

    def set_debug(self, withhold_field: int = -1, timeout_ms: float = 0.0):
        L.grf_batch_set_debug(self.handle, withhold_field, timeout_ms)

    @property
    def total_points(self) -> int:
        return L.grf_plan_query(self.handle, 0)

    def close(self):
        if getattr(self, "handle", None) is not None:
            L.grf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
