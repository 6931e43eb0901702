"""GB300 (sm_103a) spherical Poisson solver: Python binding of the C ABI.

Every step of the solve runs in the library's CUDA kernels; this module only
marshals torch tensors (device memory, the current stream) into the C calls.

    import paper_1510_08094_gb300 as sp
    u = sp.solve(f)                 # f: float64 CUDA tensor [n_theta, n_lambda]
    plan = sp.Plan(n_theta, n_lambda)
    u = plan.solve(f); fbar = plan.solve_adjoint(ubar)
    u = sp.poisson(f)               # differentiable (torch.autograd.Function)
"""

from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib
from ._lib import (  # noqa: F401
    SP_FP32,
    SP_FP32_REFINE,
    SP_FP64,
    SpherePoissonError,
    library_path,
)

__all__ = ["Plan", "BatchedPlan", "solve", "solve_adjoint", "poisson", "SpherePoisson", "SpherePoissonError", "get_plan"]

_PRECISIONS = {"fp64": SP_FP64, "fp32": SP_FP32, "fp32_refine": SP_FP32_REFINE}


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_grid(t: torch.Tensor, shape, name: str, device=None):
    """Shape, dtype, contiguity and device of a grid argument; `device` is the
    plan's device (the library's tables live there and its kernels run there)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64, got {t.dtype}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the plan is on {device}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """A solver plan for one grid size (n_theta colatitudes x n_lambda longitudes).

    autotune=True times the transform tiles at plan time and keeps the fastest
    (cached in $SPHERE_POISSON_TUNE_CACHE if set).  grid="poles" is the grid
    with both poles (SP_FLAG_POLES): n_theta + 1 rows theta_i = i pi / n_theta,
    FP64 solves only."""

    def __init__(self, n_theta: int, n_lambda: int, precision: str = "fp64", refine_sweeps: int = 0,
                 device=None, autotune: bool = False, grid: str = "shifted"):
        lib = _lib.load()
        if precision not in _PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(_PRECISIONS)}")
        if grid not in ("shifted", "poles"):
            raise ValueError('grid must be "shifted" or "poles"')
        self.grid = grid
        self.n_theta, self.n_lambda = int(n_theta), int(n_lambda)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            flags = (_lib.SP_FLAG_AUTOTUNE if autotune else 0) | (_lib.SP_FLAG_POLES if grid == "poles" else 0)
            _lib.check(lib.sphere_poisson_plan(ctypes.byref(h), self.n_theta, self.n_lambda,
                                               _PRECISIONS[precision], int(refine_sweeps), flags,
                                               ctypes.byref(ws)), "sphere_poisson_plan")
        self._h = h
        self.workspace_bytes = int(ws.value)
        self._lib = lib
        self._ws = None

    @property
    def shape(self):
        return (self.n_theta + (1 if self.grid == "poles" else 0), self.n_lambda)

    def _workspace(self, workspace):
        if workspace is not None:
            if workspace.device != self.device or workspace.numel() * workspace.element_size() < self.workspace_bytes:
                raise ValueError("workspace too small or on another device")
            return workspace
        if self._ws is None:
            self._ws = torch.empty(max(1, self.workspace_bytes), dtype=torch.uint8, device=self.device)
        return self._ws

    def launches(self, adjoint: bool = False) -> int:
        n = ctypes.c_int()
        _lib.check(self._lib.sphere_poisson_launch_count(self._h, int(adjoint), ctypes.byref(n)),
                   "sphere_poisson_launch_count")
        return int(n.value)

    def solve(self, f: torch.Tensor, out: torch.Tensor | None = None, workspace=None, stream=None,
              mean_out: torch.Tensor | None = None):
        """u with Delta u = f and zero sphere mean (f: float64 CUDA [n_theta, n_lambda]).

        mean_out: optional float64 tensor on the plan's device; its first element
        receives the mean of f over the sphere (written on the stream, no sync)."""
        _check_grid(f, self.shape, "f", self.device)
        if out is None:
            out = torch.empty_like(f)
        _check_grid(out, self.shape, "out", self.device)
        mean_ptr = None
        if mean_out is not None:
            if mean_out.dtype != torch.float64 or mean_out.device != self.device or mean_out.numel() < 1:
                raise ValueError("mean_out must be a float64 tensor on the plan's device")
            mean_ptr = mean_out.data_ptr()
        ws = self._workspace(workspace)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_solve(self._h, f.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                                      ws.numel() * ws.element_size(), _stream_ptr(stream),
                                                      mean_ptr), "sphere_poisson_solve")
        return out

    def solve_adjoint(self, ubar: torch.Tensor, out: torch.Tensor | None = None, workspace=None, stream=None):
        """S^T ubar, the transpose of f -> u (the vector-Jacobian product)."""
        _check_grid(ubar, self.shape, "ubar", self.device)
        if out is None:
            out = torch.empty_like(ubar)
        _check_grid(out, self.shape, "out", self.device)
        ws = self._workspace(workspace)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_solve_adjoint(self._h, ubar.data_ptr(), out.data_ptr(),
                                                              ws.data_ptr(), ws.numel() * ws.element_size(),
                                                              _stream_ptr(stream)),
                       "sphere_poisson_solve_adjoint")
        return out

    def device_status(self, stream=None) -> int:
        """SP_OK, or SP_ERR_TIMEOUT if a kernel's bounded wait for its asynchronous
        copies gave up since the last check (synchronises `stream`; clears the status)."""
        with torch.cuda.device(self.device):
            return int(self._lib.sphere_poisson_device_status(self._h, _stream_ptr(stream)))

    def solve_noalloc(self, f: torch.Tensor, out: torch.Tensor, stream=None):
        """Allocation-free solve for callers that cannot allocate device memory when
        they solve: no workspace, the library's fixed 32 MiB scratch array is used
        instead (grids up to that size).  Calls that overlap on the GPU race on
        that shared array; `out` must be given because this call allocates nothing."""
        _check_grid(f, self.shape, "f", self.device)
        _check_grid(out, self.shape, "out", self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_solve_noalloc(self._h, f.data_ptr(), out.data_ptr(),
                                                              _stream_ptr(stream)),
                       "sphere_poisson_solve_noalloc")
        return out

    @property
    def spectrum_shape(self):
        """(n_theta, Kp) of the coefficient layout of coeffs2 / sample."""
        kp = (self.n_lambda // 2 + 2) // 2 * 2
        return (self.n_theta, kp)

    def coeffs2(self, f: torch.Tensor, stream=None) -> torch.Tensor:
        """2D Fourier coefficients X[j, k] of f~, j = 0..n_theta-1, k = 0..n_lambda/2
        (the last column is k = -n_lambda/2), as a complex128 tensor [n_theta, Kp]."""
        _check_grid(f, self.shape, "f", self.device)
        out = torch.empty(self.spectrum_shape, dtype=torch.complex128, device=self.device)
        ws = self._workspace(None)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_coeffs2(self._h, f.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                                        ws.numel(), _stream_ptr(stream)), "sphere_poisson_coeffs2")
        return out

    def sample(self, coeffs: torch.Tensor, stream=None) -> torch.Tensor:
        """Grid values of the expansion with coefficients in the coeffs2 layout."""
        if coeffs.dtype != torch.complex128 or tuple(coeffs.shape) != self.spectrum_shape or not coeffs.is_cuda:
            raise ValueError("coeffs must be a complex128 CUDA tensor of spectrum_shape")
        coeffs = coeffs.contiguous()
        out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        ws = self._workspace(None)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_sample(self._h, coeffs.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                                       ws.numel(), _stream_ptr(stream)), "sphere_poisson_sample")
        return out

    def sum2(self, f: torch.Tensor, stream=None) -> float:
        """Surface integral of f over the unit sphere (synchronises)."""
        _check_grid(f, self.shape, "f", self.device)
        res = torch.empty(2, dtype=torch.float64, device=self.device)
        ws = self._workspace(None)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_sum2(self._h, f.data_ptr(), res.data_ptr(), ws.data_ptr(),
                                                     ws.numel(), _stream_ptr(stream)), "sphere_poisson_sum2")
        return float(res[0])

    def gradient_workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        _lib.check(self._lib.sphere_poisson_gradient_workspace_size(self._h, ctypes.byref(n)),
                   "sphere_poisson_gradient_workspace_size")
        return int(n.value)

    def curl_workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        _lib.check(self._lib.sphere_poisson_curl_workspace_size(self._h, ctypes.byref(n)),
                   "sphere_poisson_curl_workspace_size")
        return int(n.value)

    def set_chop(self, rtol: float):
        """Zero the coefficients of derivative inputs with |X| <= rtol max |X|
        before the maps act (0 turns it off)."""
        _lib.check(self._lib.sphere_poisson_set_chop(self._h, float(rtol)), "sphere_poisson_set_chop")
        return self

    def _derivative_call(self, name, inputs, n_out, out, workspace, need, stream):
        for i, f in enumerate(inputs):
            _check_grid(f, self.shape, f"input {i}", self.device)
        if out is None:
            out = tuple(torch.empty_like(inputs[0]) for _ in range(n_out))
        nbytes = inputs[0].numel() * 8
        for o in out:
            _check_grid(o, self.shape, "out", self.device)
            for f in inputs:
                if abs(o.data_ptr() - f.data_ptr()) < nbytes:
                    raise ValueError("outputs must not overlap the inputs")
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
        elif workspace.numel() * workspace.element_size() < need:
            raise ValueError("workspace too small")
        with torch.cuda.device(self.device):
            _lib.check(getattr(self._lib, name)(
                self._h, *[t.data_ptr() for t in inputs], *[o.data_ptr() for o in out],
                workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream_ptr(stream)), name)
        return out

    def tangential_gradient(self, f: torch.Tensor, out=None, workspace=None, stream=None):
        """(d^t f/dx, d^t f/dy, d^t f/dz) on the grid: the Cartesian components of
        the surface gradient (Section 4, Differentiation).  out: optional tuple of
        three float64 CUDA tensors of the grid's shape."""
        return self._derivative_call("sphere_poisson_tangential_gradient", (f,), 3, out, workspace,
                                     self.gradient_workspace_bytes(), stream)

    def divergence(self, f1, f2, f3, out=None, workspace=None, stream=None):
        """Surface divergence d^t f1/dx + d^t f2/dy + d^t f3/dz (Section 4, vector calculus)."""
        r = self._derivative_call("sphere_poisson_divergence", (f1, f2, f3), 1,
                                  None if out is None else (out,), workspace, self.gradient_workspace_bytes(),
                                  stream)
        return r[0]

    def curl(self, f1, f2, f3, out=None, workspace=None, stream=None):
        """Surface curl of the field (f1, f2, f3): three components on the grid."""
        return self._derivative_call("sphere_poisson_curl", (f1, f2, f3), 3, out, workspace,
                                     self.curl_workspace_bytes(), stream)

    def scalar_curl(self, f, out=None, workspace=None, stream=None):
        """Curl of a scalar function, n x grad f (eq. CurlScalarF): three components."""
        return self._derivative_call("sphere_poisson_scalar_curl", (f,), 3, out, workspace,
                                     self.gradient_workspace_bytes(), stream)

    def vorticity(self, f1, f2, f3, out=None, workspace=None, stream=None):
        """Vorticity (curl f) . n of the field (f1, f2, f3)."""
        r = self._derivative_call("sphere_poisson_vorticity", (f1, f2, f3), 1,
                                  None if out is None else (out,), workspace, self.curl_workspace_bytes(), stream)
        return r[0]

    def lowrank_workspace_bytes(self, max_terms: int) -> int:
        n = ctypes.c_size_t()
        _lib.check(self._lib.sphere_poisson_lowrank_workspace_size(self._h, int(max_terms), ctypes.byref(n)),
                   "sphere_poisson_lowrank_workspace_size")
        return int(n.value)

    def lowrank_ge(self, f: torch.Tensor, max_terms: int | None = None, rtol: float = 1e-13,
                   alpha: float = 0.01, stream=None):
        """Structure-preserving GE of f (Section 3): (cols [T, 2 n_theta], piv [T, 2],
        rows [T, n_lambda]) with f ~= sum_t [c_t(theta) c_t(-theta)] P_t [r_t(lambda); r_t(lambda+pi)]."""
        _check_grid(f, self.shape, "f", self.device)
        T = min(self.n_theta, 1024) if max_terms is None else int(max_terms)
        m, n = 2 * self.n_theta, self.n_lambda
        cols = torch.empty(max(T, 1), m, dtype=torch.float64, device=self.device)
        rows = torch.empty(max(T, 1), n, dtype=torch.float64, device=self.device)
        piv = torch.empty(max(T, 1), 2, dtype=torch.float64, device=self.device)
        ws = torch.empty(self.lowrank_workspace_bytes(T), dtype=torch.uint8, device=self.device)
        count = ctypes.c_int()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_lowrank_ge(self._h, f.data_ptr(), T, float(rtol), float(alpha),
                                                           ctypes.byref(count), cols.data_ptr(), piv.data_ptr(),
                                                           rows.data_ptr(), ws.data_ptr(), ws.numel(),
                                                           _stream_ptr(stream)), "sphere_poisson_lowrank_ge")
        k = int(count.value)
        return cols[:k], piv[:k], rows[:k]

    def solve_lowrank(self, cols: torch.Tensor, piv: torch.Tensor, rows: torch.Tensor, out=None, stream=None):
        """u = S f for f the sum of the low-rank terms (right-hand side formed from the factors)."""
        T = int(cols.shape[0])
        m, n = 2 * self.n_theta, self.n_lambda
        for t, shape in ((cols, (T, m)), (piv, (T, 2)), (rows, (T, n))):
            if t.dtype != torch.float64 or not t.is_cuda or tuple(t.shape) != shape:
                raise ValueError("cols, piv, rows must be float64 CUDA tensors [T, 2 n_theta], [T, 2], [T, n_lambda]")
        cols, piv, rows = cols.contiguous(), piv.contiguous(), rows.contiguous()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        _check_grid(out, self.shape, "out", self.device)
        ws = torch.empty(self.lowrank_workspace_bytes(T), dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sphere_poisson_solve_lowrank(self._h, T, cols.data_ptr(), piv.data_ptr(),
                                                              rows.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                                              ws.numel(), _stream_ptr(stream)),
                       "sphere_poisson_solve_lowrank")
        return out

    def host_buffer_bytes(self) -> int:
        n = ctypes.c_size_t()
        _lib.check(self._lib.sphere_poisson_host_buffer_size(self._h, ctypes.byref(n)),
                   "sphere_poisson_host_buffer_size")
        return int(n.value)

    def solve_host(self, f_host: torch.Tensor, out: torch.Tensor | None = None, device_buffer=None,
                   stream=None, with_mean: bool = False):
        """Host-memory form: copies f in, solves, copies u out, then synchronises.

        with_mean=True returns (u, mean of f, status): status is
        SP_WARN_NONZERO_MEAN when f is not mean-zero to rounding, else SP_OK."""
        if f_host.dtype != torch.float64 or f_host.is_cuda or tuple(f_host.shape) != self.shape:
            raise ValueError("f_host must be a float64 CPU tensor of the plan's shape")
        f_host = f_host.contiguous()
        if out is None:
            out = torch.empty_like(f_host)
        need = self.host_buffer_bytes()
        if device_buffer is None:
            device_buffer = torch.empty(need, dtype=torch.uint8, device=self.device)
        elif device_buffer.device != self.device:
            raise ValueError("device_buffer is not on the plan's device")
        mean = ctypes.c_double()
        with torch.cuda.device(self.device):
            rc = _lib.check(self._lib.sphere_poisson_solve_host(self._h, f_host.data_ptr(), out.data_ptr(),
                                                                device_buffer.data_ptr(), device_buffer.numel(),
                                                                _stream_ptr(stream),
                                                                ctypes.byref(mean) if with_mean else None),
                            "sphere_poisson_solve_host")
        if with_mean:
            return out, float(mean.value), int(rc)
        return out

    def profile_begin(self, max_solves: int):
        """Start recording per-stage CUDA events for the next max_solves calls."""
        _lib.check(self._lib.sphere_poisson_profile_begin(self._h, int(max_solves)), "profile_begin")

    def profile_end(self) -> tuple[dict, int]:
        """({stage name: summed ms}, calls recorded) since profile_begin."""
        ms = (ctypes.c_double * 16)()
        n, ns = ctypes.c_int(), ctypes.c_int()
        _lib.check(self._lib.sphere_poisson_profile_end(self._h, ms, 16, ctypes.byref(n), ctypes.byref(ns)),
                   "profile_end")
        names = [self._lib.sphere_poisson_stage_name(self._h, s).decode() for s in range(ns.value)]
        return {names[s]: float(ms[s]) for s in range(ns.value)}, int(n.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sphere_poisson_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan(Plan):
    """Many independent spheres of uneven resolution solved by persistent launches (one per radix group).

    sizes: sequence of (n_theta, n_lambda).  The solve takes and returns the
    problems' grids packed back to back in one float64 CUDA tensor (see
    `offsets`, `pack`, `unpack`).  autotune=True times the transform tiles of
    every size at plan time (cached in $SPHERE_POISSON_TUNE_CACHE if set)."""

    def __init__(self, sizes, precision: str = "fp64", refine_sweeps: int = 0, autotune: bool = False,
                 device=None):
        lib = _lib.load()
        if precision not in _PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(_PRECISIONS)}")
        sizes = [(int(a), int(b)) for a, b in sizes]
        self.sizes = sizes
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        cnt = len(sizes)
        nts = (ctypes.c_int * max(cnt, 1))(*[a for a, _ in sizes])
        nls = (ctypes.c_int * max(cnt, 1))(*[b for _, b in sizes])
        h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        flags = _lib.SP_FLAG_AUTOTUNE if autotune else 0
        with torch.cuda.device(self.device):
            _lib.check(lib.sphere_poisson_plan_batched(ctypes.byref(h), cnt, nts, nls, _PRECISIONS[precision],
                                                       int(refine_sweeps), flags, ctypes.byref(ws)),
                       "sphere_poisson_plan_batched")
        self._h = h
        self._lib = lib
        self._ws = None
        self.workspace_bytes = int(ws.value)
        offs = (ctypes.c_size_t * (cnt + 1))()
        _lib.check(lib.sphere_poisson_batch_offsets(h, offs), "sphere_poisson_batch_offsets")
        self.offsets = [int(offs[i]) for i in range(cnt + 1)]
        self.n_theta, self.n_lambda = 1, self.offsets[-1]
        self.grid = "shifted"

    @property
    def shape(self):
        return (self.offsets[-1],)

    def pack(self, grids):
        """One packed float64 tensor from per-problem [n_theta, n_lambda] tensors."""
        if len(grids) != len(self.sizes):
            raise ValueError("one grid per problem")
        out = torch.empty(self.offsets[-1], dtype=torch.float64, device=self.device)
        for b, g in enumerate(grids):
            if tuple(g.shape) != self.sizes[b]:
                raise ValueError(f"grid {b} has shape {tuple(g.shape)}, expected {self.sizes[b]}")
            out[self.offsets[b]:self.offsets[b + 1]] = g.reshape(-1)
        return out

    def unpack(self, packed):
        return [packed[self.offsets[b]:self.offsets[b + 1]].view(*self.sizes[b]) for b in range(len(self.sizes))]

    def solve(self, f, out=None, workspace=None, stream=None, mean_out=None):
        if f.dim() != 1:
            raise ValueError("batched solve takes the packed 1-D array")
        return super().solve(f, out, workspace, stream, mean_out)


_plans: dict = {}
_plans_lock = threading.Lock()


def get_plan(n_theta: int, n_lambda: int, precision: str = "fp64", refine_sweeps: int = 0, device=None,
             grid: str = "shifted") -> Plan:
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    key = (int(n_theta), int(n_lambda), precision, int(refine_sweeps), dev, grid)
    with _plans_lock:
        p = _plans.get(key)
        if p is None:
            p = Plan(n_theta, n_lambda, precision, refine_sweeps, device=torch.device("cuda", dev), grid=grid)
            _plans[key] = p
        return p


def _grid_n_theta(rows: int, grid: str) -> int:
    return rows - 1 if grid == "poles" else rows


def solve(f: torch.Tensor, precision: str = "fp64", refine_sweeps: int = 0, grid: str = "shifted") -> torch.Tensor:
    """u = S f on f's device (cached plan per shape); grid="poles" takes f with
    n_theta + 1 rows on the grid with both poles."""
    return get_plan(_grid_n_theta(f.shape[0], grid), f.shape[1], precision, refine_sweeps, f.device,
                    grid).solve(f)


def solve_adjoint(ubar: torch.Tensor, precision: str = "fp64", refine_sweeps: int = 0,
                  grid: str = "shifted") -> torch.Tensor:
    return get_plan(_grid_n_theta(ubar.shape[0], grid), ubar.shape[1], precision, refine_sweeps, ubar.device,
                    grid).solve_adjoint(ubar)


class SpherePoisson(torch.autograd.Function):
    """Differentiable solve: forward u = S f, backward grad_f = S^T grad_u.

    The fp64 and fp32 forms have their own transposes.  The fp32_refine form
    computes the FP64 solution map to ~1e-13 (refined), so its backward is the
    FP64 adjoint, the transpose of the map it approximates; the refinement
    itself is not differentiated (its iterates depend on f through rounding only)."""

    @staticmethod
    def forward(ctx, f, precision="fp64", refine_sweeps=0, grid="shifted"):
        if precision not in _PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(_PRECISIONS)}")
        ctx.precision = precision
        ctx.grid = grid
        return solve(f.contiguous(), precision, refine_sweeps, grid)

    @staticmethod
    def backward(ctx, grad_u):
        adj = "fp64" if ctx.precision == "fp32_refine" else ctx.precision
        g = solve_adjoint(grad_u.contiguous(), adj, 0, ctx.grid)
        return g, None, None, None


def pipe_rates() -> dict:
    """Measured FMA issue rates of the current GPU (G instructions/s)."""
    lib = _lib.load()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(lib.sphere_poisson_pipe_rates(ctypes.byref(a), ctypes.byref(b)), "sphere_poisson_pipe_rates")
    return {"fp64_fma_gops": a.value, "fp32_fma_gops": b.value}


def poisson(f: torch.Tensor, precision: str = "fp64", refine_sweeps: int = 0, grid: str = "shifted") -> torch.Tensor:
    return SpherePoisson.apply(f, precision, refine_sweeps, grid)
